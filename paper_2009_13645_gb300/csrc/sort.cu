// Periodic counting sort of the particles by cell, so that particles that share a cell are
// neighbours in memory: the gather reads and deposit atomics of a warp then hit the same few
// cache lines.  The cells are ordered as a serpentine: x runs backwards in every other row and y
// in every other plane, so the last cell of a row (plane) touches the first of the next, and a
// block of particles that straddles two rows still covers a compact box of cells (the push's
// deposit tile).  The key is a permutation of the cell index; particles outside the node range
// go to one last bin.
#include "common.cuh"
#include "kernels.h"

namespace mithra {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Lanes of a warp that share a bin add to its counter once: the leader (lowest lane) adds their
// number, and every lane learns the value the counter had before (*base) and its own rank among
// them.  Particles that share a cell (and the many outside the node range, all in one bin) are
// neighbours in a warp, so most of their atomics on one address collapse into one.
__device__ __forceinline__ int32_t warp_aggregated_add(int32_t* ctr, int32_t bin, bool active)
{
    const unsigned act = __ballot_sync(0xffffffffu, active);
    if (!active) return 0;
    const unsigned peers = __match_any_sync(act, bin);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(ctr + bin, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    return base + __popc(peers & ((1u << lane) - 1u));
}

template <typename real>
__global__ void k_keys(Particles<real> P, int64_t np, Geom g, int32_t* __restrict__ key, int32_t* __restrict__ count,
                       int64_t nbins)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = p < np;
    int32_t kk = 0;
    if (in) {
        const int i = P.ix[p], j = P.iy[p], k = P.iz[p];
        if (i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz) {
            const int64_t row = (int64_t)k * g.ny + ((k & 1) ? g.ny - 1 - j : j);
            kk = (int32_t)(row * g.nx + ((row & 1) ? g.nx - 1 - i : i));
        } else
            kk = (int32_t)(nbins - 1);
        key[p] = kk;
    }
    warp_aggregated_add(count, kk, in);
}

// Exclusive scan of one tile per block; the tile total goes to partial[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                            int64_t n, int32_t* __restrict__ partial)
{
    __shared__ int32_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems];
    int32_t run = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t idx = base + q;
        v[q] = idx < n ? in[idx] : 0;
        run += v[q];
    }
    // inclusive scan of the per-thread totals across the warp
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    int32_t excl = incl - run + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const int64_t idx = base + q;
        if (idx < n) out[idx] = excl;
        excl += v[q];
    }
    if (threadIdx.x == kScanThreads - 1 && partial) partial[blockIdx.x] = excl;
}

__global__ void k_scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ partial)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    out[idx] += partial[idx / kScanTile];
}

size_t sort_scan_partials(int64_t nbins)
{
    size_t tot = 0;
    int64_t n = nbins;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        tot += (size_t)n;
    }
    return tot + 1;
}

// Exclusive scan of n values, in -> out, using `scratch` for the partial sums of every level.
static cudaError_t scan_exclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* scratch, cudaStream_t st)
{
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles <= 1) {
        k_scan_tile<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr);
        count_launches(1);
        return cudaGetLastError();
    }
    int32_t* partial = scratch;
    k_scan_tile<<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, partial);
    cudaError_t e = scan_exclusive(partial, partial, tiles, scratch + tiles, st);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, partial);
    count_launches(2);
    return cudaGetLastError();
}

__global__ void k_slot(const int32_t* __restrict__ key, int64_t np, int32_t* __restrict__ cursor,
                       int32_t* __restrict__ perm)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = p < np;
    const int32_t slot = warp_aggregated_add(cursor, in ? key[p] : 0, in);
    if (in) perm[p] = slot;
}

template <typename real>
__global__ void k_scatter(Particles<real> P, Particles<real> T, const int32_t* __restrict__ perm, int64_t np)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int32_t d = perm[p];
    T.ix[d] = P.ix[p];
    T.iy[d] = P.iy[p];
    T.iz[d] = P.iz[p];
    T.fx[d] = P.fx[p];
    T.fy[d] = P.fy[p];
    T.fz[d] = P.fz[p];
    T.ux[d] = P.ux[p];
    T.uy[d] = P.uy[p];
    T.uz[d] = P.uz[p];
    T.id[d] = P.id[p];
}

template <typename real>
cudaError_t launch_sort(Particles<real>& P, Particles<real>& tmp, int64_t np, const Geom& g, const SortScratch& s,
                        cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(s.count, 0, (size_t)s.nbins * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const unsigned nb = (unsigned)((np + 255) / 256);
    k_keys<real><<<nb, 256, 0, st>>>(P, np, g, s.key, s.count, s.nbins);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive(s.count, s.offset, s.nbins, s.blocksum, st)) != cudaSuccess) return e;
    k_slot<<<nb, 256, 0, st>>>(s.key, np, s.offset, s.perm);
    k_scatter<real><<<nb, 256, 0, st>>>(P, tmp, s.perm, np);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    Particles<real> t = P;
    P = tmp;
    tmp = t;
    return cudaSuccess;
}

template cudaError_t launch_sort<float>(Particles<float>&, Particles<float>&, int64_t, const Geom&, const SortScratch&,
                                        cudaStream_t);
template cudaError_t launch_sort<double>(Particles<double>&, Particles<double>&, int64_t, const Geom&,
                                         const SortScratch&, cudaStream_t);

}  // namespace mithra
