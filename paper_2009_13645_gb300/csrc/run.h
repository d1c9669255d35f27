// Internal entry points of the run layer used by the serving loop.
#pragma once

#include <stdint.h>

#include <cuda_runtime.h>

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
// Steps of the run's captured graph (0: steps are launched one by one) and the steps enqueued so
// far; a call of exactly that many steps from a multiple of it (after the first) is one replay.
int64_t graph_steps(mithra_t r, int64_t* nstep);
// The run's captured period when its next steps are exactly one replay of it (null otherwise); the
// caller launches it - a serving group embeds it in one graph with other runs' periods - and then
// reports the replay with period_replayed (the host side advances by the period).
cudaGraph_t period_graph(mithra_t r, int64_t steps_left);
void period_replayed(mithra_t r);

}  // namespace mithra
