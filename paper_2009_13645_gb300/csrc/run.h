// Internal entry points of the run layer used by the serving loop.
#pragma once

#include <stdint.h>

#include "../../include/mithra.h"

namespace mithra {

// Checks of mithra_create that need no device.
int validate_request(const mithra_grid* gr, double dt_lab, const mithra_undulator* u, const mithra_bunch* b);
// mithra_create with an explicit allocator (NULLs: cudaMalloc/cudaFree).
int create_with(const mithra_grid* gr, double dt_lab, const mithra_undulator* u, const mithra_bunch* b,
                mithra_alloc_fn alloc, mithra_free_fn free_fn, void* ctx, mithra_t* out);
// The allocator installed with mithra_set_allocator (NULLs: none).
void get_allocator(mithra_alloc_fn* alloc, mithra_free_fn* free_fn, void** ctx);
// Upper bound of the device bytes a run of nsteps steps holds (what admission reserves).
int64_t footprint(const mithra_grid* gr, const mithra_undulator* u, const mithra_bunch* b, int64_t nsteps);

}  // namespace mithra
