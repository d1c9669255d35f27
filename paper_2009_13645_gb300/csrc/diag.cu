// Diagnostics (manual Sec. FEL-OUTPUT "radiation-power"; field energy and bunching factor).
// All reductions run in FP64 and in a fixed order (per-block tree, then one block over the
// block partials), so a result does not depend on scheduling.
#include "common.cuh"
#include "kernels.h"

namespace mithra {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = (threadIdx.x < blockDim.x / 32) ? sh[threadIdx.x] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

// Final pass: one block adds the block partials (columns `ncol` interleaved) with
// Neumaier-compensated sums per thread, then a tree.
__global__ void k_final(const double* __restrict__ partial, int npartial, int ncol, double scale, double* __restrict__ out)
{
    __shared__ double sh[32];
    for (int c = 0; c < ncol; ++c) {
        double s = 0.0, comp = 0.0;
        for (int i = threadIdx.x; i < npartial; i += blockDim.x) {
            const double v = partial[(int64_t)i * ncol + c];
            const double t = s + v;
            comp += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
            s = t;
        }
        const double tot = block_sum(s + comp, sh);
        if (threadIdx.x == 0) out[c] = tot * scale;
    }
}

// ---- radiated power -------------------------------------------------------------------
template <typename real>
__global__ void k_power_sample(Fields6<real> eb, Geom g, int kp, double* __restrict__ ring, int slot, double omega_h,
                               double t_sample, double* __restrict__ phase_cs)
{
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int64_t pl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pl == 0) {
        double s, c;
        sincos(omega_h * t_sample, &s, &c);
        phase_cs[2 * slot] = c;
        phase_cs[2 * slot + 1] = s;
    }
    if (pl >= plane) return;
    const int64_t id = (int64_t)kp * g.sz + pl;
    double* r = ring + (int64_t)slot * 4 * plane;
    r[pl] = (double)eb.c[0][id];
    r[plane + pl] = (double)eb.c[1][id];
    r[2 * plane + pl] = (double)eb.c[3][id];
    r[3 * plane + pl] = (double)eb.c[4][id];
}

__global__ void __launch_bounds__(kRedThreads) k_power_reduce(const double* __restrict__ ring,
                                                              const double* __restrict__ phase_cs, int M, Geom g,
                                                              double* __restrict__ partial)
{
    __shared__ double sh[32];
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int64_t nin = (int64_t)(g.nx - 2) * (g.ny - 2);
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nin; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = 1 + (int)(t % (g.nx - 2));
        const int j = 1 + (int)(t / (g.nx - 2));
        const int64_t pl = (int64_t)j * g.nx + i;
        double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
        for (int m = 0; m < M; ++m) {
            const double c = phase_cs[2 * m], s = phase_cs[2 * m + 1];
            const double* r = ring + (int64_t)m * 4 * plane + pl;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double v = r[q * plane];
                re[q] += v * c;
                im[q] -= v * s;
            }
        }
        // Re(Ex By* - Ey Bx*) of the unnormalised DFT sums; the (2/M)^2 goes into `scale`
        acc += (re[0] * re[3] + im[0] * im[3]) - (re[1] * re[2] + im[1] * im[2]);
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename real>
cudaError_t power_sample_ex(const Fields6<real>& eb, const Geom& g, int kp, double* ring, int slot, double omega_h,
                            double t_sample, double* phase_cs, cudaStream_t st)
{
    const int64_t plane = (int64_t)g.nx * g.ny;
    k_power_sample<real><<<(unsigned)((plane + 255) / 256), 256, 0, st>>>(eb, g, kp, ring, slot, omega_h, t_sample,
                                                                         phase_cs);
    count_launches(1);
    return cudaGetLastError();
}
template cudaError_t power_sample_ex<float>(const Fields6<float>&, const Geom&, int, double*, int, double, double,
                                            double*, cudaStream_t);
template cudaError_t power_sample_ex<double>(const Fields6<double>&, const Geom&, int, double*, int, double, double,
                                             double*, cudaStream_t);

cudaError_t launch_power_reduce(const double* ring, const double* phase_cs, int M, const Geom& g, double scale,
                                double* partial, int npartial, double* out, cudaStream_t st)
{
    k_power_reduce<<<npartial, kRedThreads, 0, st>>>(ring, phase_cs, M, g, partial);
    k_final<<<1, kRedThreads, 0, st>>>(partial, npartial, 1, scale, out);
    count_launches(2);
    return cudaGetLastError();
}

// ---- on-axis sample -------------------------------------------------------------------
template <typename real>
__global__ void k_onaxis(const real* __restrict__ ex, int64_t id, double* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = (double)ex[id];
}

template <typename real>
cudaError_t launch_onaxis(const Fields6<real>& eb, int64_t id, double* out, cudaStream_t st)
{
    k_onaxis<real><<<1, 32, 0, st>>>(eb.c[0], id, out);
    count_launches(1);
    return cudaGetLastError();
}

// ---- field energy ----------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_energy(Fields6<real> eb, int64_t n, double* __restrict__ partial)
{
    __shared__ double sh[32];
    constexpr double eps0 = 1.0 / (kMu0 * kC * kC);
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double e2 = 0.0, b2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double e = (double)eb.c[c][t], b = (double)eb.c[3 + c][t];
            e2 += e * e;
            b2 += b * b;
        }
        acc += 0.5 * eps0 * e2 + 0.5 * b2 / kMu0;
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename real>
cudaError_t launch_energy(const Fields6<real>& eb, const Geom& g, double* partial, int npartial, double* out,
                          cudaStream_t st)
{
    k_energy<real><<<npartial, kRedThreads, 0, st>>>(eb, g.ncell, partial);
    k_final<<<1, kRedThreads, 0, st>>>(partial, npartial, 1, g.dx * g.dy * g.dz, out);
    count_launches(2);
    return cudaGetLastError();
}

// ---- bunching factor -------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_bunching(Particles<real> P, int64_t np, Geom g, double kb,
                                                          double* __restrict__ partial)
{
    __shared__ double sh[32];
    double cr = 0.0, ci = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const double z = g.z0 + ((double)P.iz[p] + (double)P.fz[p]) * g.dz;
        double s, c;
        sincos(kb * z, &s, &c);
        cr += c;
        ci += s;
    }
    const double tr = block_sum(cr, sh);
    const double ti = block_sum(ci, sh);
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = tr;
        partial[2 * blockIdx.x + 1] = ti;
    }
}

__global__ void k_bunch_final(double* out3, double inv_n)
{
    if (threadIdx.x == 0) {
        const double re = out3[1] * inv_n, im = out3[2] * inv_n;
        out3[0] = sqrt(re * re + im * im);
        out3[1] = re;
        out3[2] = im;
    }
}

template <typename real>
cudaError_t launch_bunching(const Particles<real>& P, int64_t np, const Geom& g, double kb, double* partial,
                            int npartial, double* out3, cudaStream_t st)
{
    if (np <= 0) {
        return cudaMemsetAsync(out3, 0, 3 * sizeof(double), st);
    }
    k_bunching<real><<<npartial, kRedThreads, 0, st>>>(P, np, g, kb, partial);
    k_final<<<1, kRedThreads, 0, st>>>(partial, npartial, 2, 1.0, out3 + 1);
    k_bunch_final<<<1, 32, 0, st>>>(out3, 1.0 / (double)np);
    count_launches(3);
    return cudaGetLastError();
}

#define MITHRA_INST(real)                                                                                              \
    template cudaError_t launch_onaxis<real>(const Fields6<real>&, int64_t, double*, cudaStream_t);                    \
    template cudaError_t launch_energy<real>(const Fields6<real>&, const Geom&, double*, int, double*, cudaStream_t); \
    template cudaError_t launch_bunching<real>(const Particles<real>&, int64_t, const Geom&, double, double*, int,    \
                                               double*, cudaStream_t);
MITHRA_INST(float)
MITHRA_INST(double)
#undef MITHRA_INST

}  // namespace mithra
