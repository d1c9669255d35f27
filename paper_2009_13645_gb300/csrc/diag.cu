// Diagnostics (manual Sec. FEL-OUTPUT "radiation-power"; field energy and bunching factor).
// All reductions run in FP64 and in a fixed order (per-block tree, then one block over the
// block partials), so a result does not depend on scheduling.
#include "common.cuh"
#include "kernels.h"

namespace mithra {

constexpr int kRedThreads = 256;

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
// The power step runs in the step tail (power_point in kernels.h, the launch in fields.cu).

// ---- field energy ----------------------------------------------------------------------
// The field energy (node_energy summed in FP64 over every node).
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_energy(Fields6<real> eb, int64_t n, double* __restrict__ partial)
{
    __shared__ double sh[32];
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(real) == 4) {
            const float4 e = __ldg(reinterpret_cast<const float4*>(eb.p + t * kEBStride));
            const float2 b = __ldg(reinterpret_cast<const float2*>(eb.p + t * kEBStride + 4));
            acc += node_energy(e.x, e.y, e.z, e.w, b.x, b.y);
        } else {
            acc += node_energy(eb.at(0, t), eb.at(1, t), eb.at(2, t), eb.at(3, t), eb.at(4, t), eb.at(5, t));
        }
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
                                                          const float2* __restrict__ tab, float kbdz,
                                                          double* __restrict__ partial)
{
    __shared__ double sh[32];
    double cr = 0.0, ci = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const int iz = P.iz[p];
        if (tab && iz >= 0 && iz < g.nz) {
            // the plane's phase from the FP64 table, turned by the FP32 phase of the offset
            const float2 t = __ldg(tab + iz);
            float sf, cf;
            sincosf(kbdz * (float)P.fz[p], &sf, &cf);
            cr += (double)(t.x * cf - t.y * sf);
            ci += (double)(t.y * cf + t.x * sf);
        } else {
            const double z = g.z0 + ((double)iz + (double)P.fz[p]) * g.dz;
            double s, c;
            sincos(kb * z, &s, &c);
            cr += c;
            ci += s;
        }
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

// (cos, sin) of k_b z at every node plane, in FP64, rounded to FP32.
__global__ void k_bunch_table(float2* __restrict__ tab, int nz, double z0, double dz, double kb)
{
    const int k = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (k >= nz) return;
    double s, c;
    sincos(kb * (z0 + (double)k * dz), &s, &c);
    tab[k] = make_float2((float)c, (float)s);
}

template <typename real>
cudaError_t launch_bunching(const Particles<real>& P, int64_t np, const Geom& g, double kb, double* partial,
                            int npartial, double* out3, float2* tab, cudaStream_t st)
{
    if (np <= 0) {
        return cudaMemsetAsync(out3, 0, 3 * sizeof(double), st);
    }
    // FP32 offsets: the phase of a particle is its plane's (FP64 table) plus k_b dz times its offset
    // (FP32, below k_b dz); FP64 offsets keep the whole phase in FP64
    const bool use_tab = tab && sizeof(real) == 4;
    if (use_tab) {
        k_bunch_table<<<(g.nz + 255) / 256, 256, 0, st>>>(tab, g.nz, g.z0, g.dz, kb);
        count_launches(1);
    }
    k_bunching<real><<<npartial, kRedThreads, 0, st>>>(P, np, g, kb, use_tab ? tab : nullptr, (float)(kb * g.dz),
                                                       partial);
    k_final<<<1, kRedThreads, 0, st>>>(partial, npartial, 2, 1.0, out3 + 1);
    k_bunch_final<<<1, 32, 0, st>>>(out3, 1.0 / (double)np);
    count_launches(3);
    return cudaGetLastError();
}

// ---- radiated-power spectrum ------------------------------------------------------------
// One block per (256 plane points, frequency k): the block's first thread forms the frequency's
// phases of the step; every point updates the accumulators of frequency k (adding its new
// sample, and once the window is full subtracting the sample of step n - M[k] from the ring);
// one partial flux per block.  The new sample enters the ring afterwards (k_spec_ring), once
// every frequency has read its leaving sample.
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_spec_step(Fields6<real> eb, Geom g, SpecStep s,
                                                           double* __restrict__ partial)
{
    dep_begin();
    __shared__ double sh[32];
    __shared__ double ph[4];
    const int k = blockIdx.y;
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int64_t pl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = s.sd->n;
    const int Mk = s.M[k];
    if (threadIdx.x == 0) {
        sincos(s.omega[k] * ((double)n + 0.5) * s.dt, &ph[1], &ph[0]);
        sincos(s.omega[k] * ((double)(n - Mk) + 0.5) * s.dt, &ph[3], &ph[2]);
    }
    __syncthreads();
    const bool full = n >= Mk, emit = n + 1 >= Mk;
    double contrib = 0.0;
    if (pl < plane) {
        const int64_t id = (int64_t)s.kp * g.sz + pl;
        const double x[4] = {(double)eb.at(0, id), (double)eb.at(1, id), (double)eb.at(3, id), (double)eb.at(4, id)};
        const double cn = ph[0], sn = ph[1], co = ph[2], so = ph[3];
        const double* ro = s.ring + (full ? (int64_t)((n - Mk) % s.Mh) : 0) * 4 * plane + pl;
        double* ac = s.acc + (int64_t)k * 8 * plane + pl;
        double re[4], im[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double a = ac[(2 * q) * plane], b = ac[(2 * q + 1) * plane];
            a += x[q] * cn;
            b -= x[q] * sn;
            if (full) {
                const double o = ro[q * plane];
                a -= o * co;
                b += o * so;
            }
            ac[(2 * q) * plane] = a;
            ac[(2 * q + 1) * plane] = b;
            re[q] = a;
            im[q] = b;
        }
        const int i = (int)(pl % g.nx), j = (int)(pl / g.nx);
        if (emit && i >= 1 && i <= g.nx - 2 && j >= 1 && j <= g.ny - 2)
            contrib = (re[0] * re[3] + im[0] * im[3]) - (re[1] * re[2] + im[1] * im[2]);
    }
    const double tot = block_sum(contrib, sh);
    if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = tot;
}

template <typename real>
__global__ void k_spec_ring(Fields6<real> eb, Geom g, SpecStep s)
{
    dep_begin();
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int64_t pl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pl >= plane) return;
    const int64_t id = (int64_t)s.kp * g.sz + pl;
    double* r = s.ring + (int64_t)(s.sd->n % s.Mh) * 4 * plane + pl;
    r[0] = (double)eb.at(0, id);
    r[plane] = (double)eb.at(1, id);
    r[2 * plane] = (double)eb.at(3, id);
    r[3 * plane] = (double)eb.at(4, id);
}

// One block per frequency: compensated sum of its partials.
__global__ void k_spec_final(const double* __restrict__ partial, int npartial, SpecStep s, double* __restrict__ series)
{
    dep_begin();
    __shared__ double sh[32];
    const int k = blockIdx.x;
    const int64_t n = s.sd->n;
    double sum = 0.0, comp = 0.0;
    for (int i = threadIdx.x; i < npartial; i += blockDim.x) {
        const double v = partial[(int64_t)k * npartial + i];
        const double t = sum + v;
        comp += (fabs(sum) >= fabs(v)) ? (sum - t) + v : (v - t) + sum;
        sum = t;
    }
    const double tot = block_sum(sum + comp, sh);
    if (threadIdx.x == 0) series[n * s.nf + k] = (n + 1 >= s.M[k]) ? tot * s.scale[k] : 0.0;
}

template <typename real>
cudaError_t launch_spectrum_step(const Fields6<real>& eb, const Geom& g, const SpecStep& s, double* partial,
                                 int npartial, double* series, cudaStream_t st)
{
    const int64_t plane = (int64_t)g.nx * g.ny;
    const unsigned nb = (unsigned)((plane + kRedThreads - 1) / kRedThreads);
    if ((int)nb > npartial || s.nf < 1) return cudaErrorInvalidValue;
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepOther), k_spec_step<real>, dim3(nb, s.nf),
                                          dim3(kRedThreads), 0, st, eb, g, s, partial);
        if (le != cudaSuccess) return le;
    }
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepOther), k_spec_ring<real>, dim3(nb), dim3(kRedThreads), 0,
                                          st, eb, g, s);
        if (le != cudaSuccess) return le;
    }
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepOther), k_spec_final, dim3(s.nf), dim3(kRedThreads), 0, st,
                                          partial, (int)nb, s, series);
        if (le != cudaSuccess) return le;
    }
    count_launches(3);
    return cudaGetLastError();
}

// ---- bunch sampling ------------------------------------------------------------------------
// Per-thread sums of the shifted values and their squares: FP64 on the FP64 path; on the
// FP32-mixed path FP32 per particle and per thread (positions are FP32 offsets there; the
// shifted values are formed without cancellation: x - centre from the cell index relative to the
// centre cell, gamma_lab - gamma_ref from gamma - 1 = u^2 / (1 + gamma)), FP64 across threads.
template <typename real>
__global__ void __launch_bounds__(kRedThreads) k_bunch_moments(Particles<real> P, int64_t np, Geom g, BunchSample b,
                                                               double* __restrict__ partial)
{
    dep_begin();
    __shared__ double sh[32];
    if (b.sd->n % b.every != 0) return;
    real s1[7], s2[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) s1[c] = s2[c] = (real)0;
    const real cx = (real)(0.5 * (g.nx - 1)), cy = (real)(0.5 * (g.ny - 1)), cz = (real)(0.5 * (g.nz - 1));
    const real dx = (real)g.dx, dy = (real)g.dy, dz = (real)g.dz;
    const real g0 = (real)b.g0, gb0 = (real)(b.g0 * b.b0), goff = (real)(b.g0 - b.shift[6]);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
        const real ux = (real)mom_value(P.ux[p]), uy = (real)mom_value(P.uy[p]), uz = (real)mom_value(P.uz[p]);
        const real u2 = ux * ux + uy * uy + uz * uz;
        const real gm1 = u2 / ((real)1 + sqrt((real)1 + u2));
        real d[7];
        d[0] = ((real)(P.ix[p] - (int)cx) - (cx - (real)(int)cx) + P.fx[p]) * dx;
        d[1] = ((real)(P.iy[p] - (int)cy) - (cy - (real)(int)cy) + P.fy[p]) * dy;
        d[2] = ((real)(P.iz[p] - (int)cz) - (cz - (real)(int)cz) + P.fz[p]) * dz;
        d[3] = ux;
        d[4] = uy;
        d[5] = uz;
        d[6] = g0 * gm1 + gb0 * uz + goff;   // gamma0 (gamma + beta0 u_z) - gamma_ref
#pragma unroll
        for (int c = 0; c < 7; ++c) {
            s1[c] += d[c];
            s2[c] += d[c] * d[c];
        }
    }
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        const double t1 = block_sum((double)s1[c], sh);
        const double t2 = block_sum((double)s2[c], sh);
        if (threadIdx.x == 0) {
            partial[(int64_t)blockIdx.x * 14 + c] = t1;
            partial[(int64_t)blockIdx.x * 14 + 7 + c] = t2;
        }
    }
}

__global__ void k_bunch_row(const double* __restrict__ partial, int npartial, int64_t np, BunchSample b,
                            double* __restrict__ series)
{
    dep_begin();
    __shared__ double sh[32];
    __shared__ double tot[14];
    const int64_t n = b.sd->n;
    if (n % b.every != 0) return;
    for (int c = 0; c < 14; ++c) {
        double sum = 0.0, comp = 0.0;
        for (int i = threadIdx.x; i < npartial; i += blockDim.x) {
            const double v = partial[(int64_t)i * 14 + c];
            const double t = sum + v;
            comp += (fabs(sum) >= fabs(v)) ? (sum - t) + v : (v - t) + sum;
            sum = t;
        }
        const double t = block_sum(sum + comp, sh);
        if (threadIdx.x == 0) tot[c] = t;
    }
    if (threadIdx.x == 0) {
        double* row = series + (n / b.every) * 15;
        const double inv = np > 0 ? 1.0 / (double)np : 0.0;
        row[0] = b.T0 + ((double)n + 1.5) * b.dt;
        double mean[7], sd[7];
        for (int c = 0; c < 7; ++c) {
            const double m1 = tot[c] * inv;
            mean[c] = b.shift[c] + m1;
            sd[c] = sqrt(fmax(tot[7 + c] * inv - m1 * m1, 0.0));
        }
        for (int a = 0; a < 6; ++a) {
            row[1 + a] = mean[a];
            row[7 + a] = sd[a];
        }
        row[13] = mean[6];
        row[14] = sd[6];
    }
}

template <typename real>
cudaError_t launch_bunch_sample(const Particles<real>& P, int64_t np, const Geom& g, const BunchSample& b,
                                double* partial, int npartial, double* series, cudaStream_t st)
{
    if (b.every < 1) return cudaErrorInvalidValue;
    int nb = (int)std::min<int64_t>((np + kRedThreads - 1) / kRedThreads, (int64_t)npartial);
    if (nb < 1) nb = 1;
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepOther), k_bunch_moments<real>, dim3(nb), dim3(kRedThreads),
                                          0, st, P, np, g, b, partial);
        if (le != cudaSuccess) return le;
    }
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepOther), k_bunch_row, dim3(1), dim3(kRedThreads), 0, st,
                                          partial, nb, np, b, series);
        if (le != cudaSuccess) return le;
    }
    count_launches(2);
    return cudaGetLastError();
}

#define MITHRA_INST(real)                                                                                              \
    template cudaError_t launch_spectrum_step<real>(const Fields6<real>&, const Geom&, const SpecStep&, double*, int, \
                                                    double*, cudaStream_t);                                          \
    template cudaError_t launch_bunch_sample<real>(const Particles<real>&, int64_t, const Geom&, const BunchSample&, \
                                                   double*, int, double*, cudaStream_t);                             \
    template cudaError_t launch_energy<real>(const Fields6<real>&, const Geom&, double*, int, double*, cudaStream_t); \
    template cudaError_t launch_bunching<real>(const Particles<real>&, int64_t, const Geom&, double, double*, int,    \
                                               double*, float2*, cudaStream_t);
MITHRA_INST(float)
MITHRA_INST(double)
#undef MITHRA_INST

}  // namespace mithra
