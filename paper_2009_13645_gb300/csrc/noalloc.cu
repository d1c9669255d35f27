// Field energy of caller-supplied E and B arrays without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need this number: code running
// inside a memory pool that is already fully carved up, a host thread that must not take the
// allocator's locks, or a real-time loop where a cudaMalloc (an implicit device synchronisation)
// would stall every stream.  This entry point therefore keeps its scratch - one FP64 partial sum
// per tile of kTileNodes nodes - in a fixed array in the library's own device memory.  That
// array exists once per GPU that loads the library and stays there until the process exits.
//
// Every call shares that array.  Each call writes every partial it later reads, so nothing has
// to be cleared between calls, but two calls whose kernels overlap on the GPU (different
// streams, or different host threads) overwrite each other's partials: callers must order them.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mithra.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int64_t kTileNodes = (int64_t)kThreads * kItems;          // nodes summed by one block
constexpr int64_t kMaxTiles = 32768;                                 // 256 KiB of partials
static_assert(MITHRA_NOALLOC_MAX_NODES == kTileNodes * kMaxTiles, "header and library disagree");

static __device__ __align__(256) double g_partial[kMaxTiles];

// Device address of g_partial for each device, looked up once with that device current.
std::mutex g_mu;
double* g_addr[64] = {};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_total(double v)
{
    __shared__ double sh[kThreads / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < kThreads / 32 ? sh[threadIdx.x] : 0.0;
    if (threadIdx.x < 32) v = warp_sum(v);
    return v;
}

// One block per tile: electric plus magnetic energy density summed over kTileNodes nodes.
template <typename real>
__global__ void __launch_bounds__(kThreads) k_energy_tiles(mithra::Fields6Soa<real> eb, int64_t n, double* partial)
{
    const int64_t base = (int64_t)blockIdx.x * kTileNodes;
    double acc = 0.0;
#pragma unroll 4
    for (int q = 0; q < kItems; ++q) {
        const int64_t t = base + (int64_t)q * kThreads + threadIdx.x;
        if (t < n)
            acc += mithra::node_energy(eb.c[0][t], eb.c[1][t], eb.c[2][t], eb.c[3][t], eb.c[4][t], eb.c[5][t]);
    }
    const double tot = block_total(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// One block adds the tile partials in a fixed order and scales by the cell volume.
__global__ void __launch_bounds__(kThreads) k_energy_finish(const double* partial, int64_t ntiles, double dv,
                                                            double* out)
{
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < ntiles; i += kThreads) s += partial[i];
    const double tot = block_total(s);
    if (threadIdx.x == 0) *out = tot * dv;
}

int set_error(int code, const char* msg) { return mithra::set_last_error(code, msg); }

}  // namespace

extern "C" int mithra_field_energy_noalloc(const void* const eb[6], int precision, int64_t n, double cell_volume,
                                           double* energy_out, void* stream)
{
    if (!eb || !energy_out) return set_error(MITHRA_EINVAL, "field_energy_noalloc: null pointer argument");
    for (int c = 0; c < 6; ++c)
        if (!eb[c] && n > 0) return set_error(MITHRA_EINVAL, "field_energy_noalloc: null field pointer");
    if (precision != 0 && precision != 1)
        return set_error(MITHRA_EINVAL, "field_energy_noalloc: precision must be 0 (double) or 1 (float)");
    if (n < 0) return set_error(MITHRA_EINVAL, "field_energy_noalloc: negative node count");
    if (n > MITHRA_NOALLOC_MAX_NODES)
        return set_error(MITHRA_EINVAL, "field_energy_noalloc: more nodes than MITHRA_NOALLOC_MAX_NODES "
                                        "(134217728); use mithra_diag, which allocates its scratch with the run");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return set_error(MITHRA_ECUDA, "field_energy_noalloc: no current CUDA device");
    }
    double* partial = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_partial);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return set_error(MITHRA_ECUDA, (std::string("field_energy_noalloc: cudaGetSymbolAddress: ") +
                                                cudaGetErrorString(e)).c_str());
            }
            g_addr[dev] = (double*)p;
        }
        partial = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ntiles = (n + kTileNodes - 1) / kTileNodes;
    if (ntiles > 0) {
        if (precision == 0) {
            mithra::Fields6Soa<double> f;
            for (int c = 0; c < 6; ++c) f.c[c] = (double*)eb[c];
            k_energy_tiles<double><<<(unsigned)ntiles, kThreads, 0, st>>>(f, n, partial);
        } else {
            mithra::Fields6Soa<float> f;
            for (int c = 0; c < 6; ++c) f.c[c] = (float*)eb[c];
            k_energy_tiles<float><<<(unsigned)ntiles, kThreads, 0, st>>>(f, n, partial);
        }
        mithra::count_launches(1);
    }
    k_energy_finish<<<1, kThreads, 0, st>>>(partial, ntiles, cell_volume, energy_out);
    mithra::count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(MITHRA_ECUDA, (std::string("field_energy_noalloc: launch: ") + cudaGetErrorString(e)).c_str());
    return MITHRA_OK;
}
