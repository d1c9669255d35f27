// Particle kernels: boost of the lab bunch into the rest frame (Eqs. LorentzTrasnformParticles,
// LorentzTransformDeltaR), and one fused pass per field step that evaluates the external
// field in FP64, gathers the self-field with linear weights (Eq. fieldInterpolation), advances
// the momentum with the Boris scheme (Eq. BorisScheme, FP64) and deposits the Umeda zigzag
// current and the linear-weight charge (Sec. "Current Deposition") with atomics.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mithra {

// Static undulator field at a particle with the phase of every planar field taken from the
// step's table (entry of the particle's z cell, in FP64) and rotated by the small angle of the
// offset within the cell and of the sub-step; cosh / sinh of the small transverse argument from
// their series.  Same fields as external_field(), evaluated with fewer FP64 operations.
__device__ __forceinline__ void static_field_fast(const ExtField& f, const PushConst& pc, int iz, double fz, int m,
                                                  double x, double y, double E[3], double B[3])
{
    double Bp[3] = {0.0, 0.0, 0.0};
    const double dzl = fma(pc.kz, fz, (double)m * pc.zstep);   // zeta beyond the cell's node plane
    const double zn = fma(pc.kz, (double)iz, pc.Z0);           // zeta of the node plane
    const int nplanar = f.kind == 1 ? 2 : 1;
    for (int j = 0; j < nplanar; ++j) {
        const double c = j ? -f.spol : f.cpol, s = j ? f.cpol : f.spol;
        const double u = (zn - (j ? f.qlam : 0.0)) + dzl;
        double sn, cs;
        if (u >= 0.0 && u <= f.Lu) {
            const double d = f.ku * dzl;
            if (fabs(d) <= 1.0) {
                const double2 t = __ldg(pc.ptab[j] + iz);
                double sd, cd;
                sincos_small(d, &sd, &cd);
                sn = fma(t.x, cd, t.y * sd);
                cs = fma(t.y, cd, -t.x * sd);
            } else {
                sincos(f.ku * u, &sn, &cs);
            }
        } else {
            const double kd = f.ku * ((u < 0.0) ? u : (u - f.Lu));
            const double g = exp(-0.5 * kd * kd);
            sn = kd * g;
            cs = g;
        }
        const double ky = f.ku * (c * y - s * x);
        double ch, sh;
        if (fabs(ky) <= 0.5) {
            coshsinh_small(ky, &ch, &sh);
        } else {
            ch = cosh(ky);
            sh = sinh(ky);
        }
        const double Bt = f.B0 * ch * sn;
        Bp[0] -= Bt * s;
        Bp[1] += Bt * c;
        Bp[2] += f.B0 * sh * cs;
    }
    // a purely magnetic lab field seen from the frame moving with beta0 along z
    const double gbc = f.g0 * f.b0 * kC;
    E[0] = -gbc * Bp[1];
    E[1] = gbc * Bp[0];
    E[2] = 0.0;
    B[0] = f.g0 * Bp[0];
    B[1] = f.g0 * Bp[1];
    B[2] = Bp[2];
}

// FP32-mixed variant: the lab coordinate of the particle (the undulator phase) and the
// Lorentz transform stay in FP64; the field shape evaluated from that phase - the rotation of
// the tabulated sin/cos by the sub-cell angle (< 1 rad) and cosh/sinh of k_u y - is computed in
// FP32, the precision of the fields it is added to.
__device__ __forceinline__ void static_field_mixed(const ExtField& f, const PushConst& pc, int iz, float fz, int m,
                                                   float x, float y, double E[3], double B[3])
{
    float Bp[3] = {0.f, 0.f, 0.f};
    const int nplanar = f.kind == 1 ? 2 : 1;
    const float ku = (float)f.ku, B0 = (float)f.B0;
    for (int j = 0; j < nplanar; ++j) {
        const float c = j ? -(float)f.spol : (float)f.cpol, s = j ? (float)f.cpol : (float)f.spol;
        const float2 t = __ldg(pc.ptab32[j] + iz);
        float sn, cs;
        if (!isnan(t.x)) {
            // the cell lies inside the undulator: rotate the exact phase of its node plane
            float sd, cd;
            sincosf(fmaf(pc.kdz, fz, pc.kzs * (float)m), &sd, &cd);
            sn = fmaf(t.x, cd, t.y * sd);
            cs = fmaf(t.y, cd, -t.x * sd);
        } else {
            const double dzl = fma(pc.kz, (double)fz, (double)m * pc.zstep);
            const double u = (fma(pc.kz, (double)iz, pc.Z0) - (j ? f.qlam : 0.0)) + dzl;
            double sd, cd;
            if (u >= 0.0 && u <= f.Lu) {
                sincos(f.ku * u, &sd, &cd);
            } else {
                const double kd = f.ku * ((u < 0.0) ? u : (u - f.Lu));
                const double g = exp(-0.5 * kd * kd);
                sd = kd * g;
                cd = g;
            }
            sn = (float)sd;
            cs = (float)cd;
        }
        const float ky = ku * (c * y - s * x);
        const float ch = coshf(ky), sh = sinhf(ky);
        const float Bt = B0 * ch * sn;
        Bp[0] -= Bt * s;
        Bp[1] += Bt * c;
        Bp[2] += B0 * sh * cs;
    }
    const double gbc = f.g0 * f.b0 * kC;
    E[0] = -gbc * (double)Bp[1];
    E[1] = gbc * (double)Bp[0];
    E[2] = 0.0;
    B[0] = f.g0 * (double)Bp[0];
    B[1] = f.g0 * (double)Bp[1];
    B[2] = (double)Bp[2];
}

// FP32 table for the mixed path: sin, cos of the exact FP64 phase at the node plane, rounded to
// FP32; NaN when [zeta, zeta + span] of the cell is not inside [0, L_u] for that planar field.
__global__ void k_phase_table32(ExtField f, double Z0, double kz, double span, int nz, float2* t0, float2* t1)
{
    const int iz = blockIdx.x * blockDim.x + threadIdx.x;
    if (iz >= nz) return;
    const double zn = fma(kz, (double)iz, Z0);
    for (int j = 0; j < (t1 ? 2 : 1); ++j) {
        const double u = zn - (j ? f.qlam : 0.0);
        float2 v = make_float2(__int_as_float(0x7fc00000), 0.f);
        if (u >= 0.0 && u + span <= f.Lu) {
            double s, c;
            sincos(f.ku * u, &s, &c);
            v = make_float2((float)s, (float)c);
        }
        (j ? t1 : t0)[iz] = v;
    }
}

cudaError_t launch_phase_table32(const ExtField& ef, double Z0, double kz, double span, int nz, float2* t0,
                                 float2* t1, cudaStream_t st)
{
    k_phase_table32<<<(nz + 127) / 128, 128, 0, st>>>(ef, Z0, kz, span, nz, t0, t1);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void k_phase_table(ExtField f, double Z0, double kz, int nz, double2* t0, double2* t1)
{
    const int iz = blockIdx.x * blockDim.x + threadIdx.x;
    if (iz >= nz) return;
    const double zn = fma(kz, (double)iz, Z0);
    double s, c;
    sincos(f.ku * zn, &s, &c);
    t0[iz] = make_double2(s, c);
    if (t1) {
        sincos(f.ku * (zn - f.qlam), &s, &c);
        t1[iz] = make_double2(s, c);
    }
}

cudaError_t launch_phase_table(const ExtField& ef, double Z0, double kz, int nz, double2* t0, double2* t1,
                               cudaStream_t st)
{
    k_phase_table<<<(nz + 127) / 128, 128, 0, st>>>(ef, Z0, kz, nz, t0, t1);
    count_launches(1);
    return cudaGetLastError();
}

__device__ __forceinline__ bool active_cell(int i, int j, int k, const Geom& g)
{
    return i >= 1 && i <= g.nx - 3 && j >= 1 && j <= g.ny - 3 && k >= 1 && k <= g.nz - 3;
}

template <typename real>
__device__ __forceinline__ void split_pos(double X, int32_t* c, real* f)
{
    const double fl = floor(X);
    real o = (real)(X - fl);
    int32_t ci = (int32_t)fl;
    if (o >= (real)1) { o -= (real)1; ci += 1; }
    *c = ci;
    *f = o;
}

// One straight piece a -> b (cell units, relative to the base cell) lying in local cell `cl`:
// current on the edges parallel to each axis with the exact path average of the linear
// weights of the two other axes.
template <typename real>
__device__ __forceinline__ void deposit_piece(const real a[3], const real b[3], const int cl[3], const int base[3],
                                              const Fields4<real>& src, const Geom& g, const PushConst& pc)
{
    real la[3], d[3], mid[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        la[l] = a[l] - (real)cl[l];
        d[l] = b[l] - a[l];
        mid[l] = la[l] + (real)0.5 * d[l];
    }
    const int64_t o = (int64_t)(base[2] + cl[2]) * g.sz + (int64_t)(base[1] + cl[1]) * g.sy + (base[0] + cl[0]);
    const int64_t st[3] = {1, g.sy, g.sz};
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        if (d[l] == (real)0) continue;
        const int m = (l + 1) % 3, n = (l + 2) % 3;
        const real F = (real)pc.qJ[l] * d[l];
        const real cross = d[m] * d[n] * (real)(1.0 / 12.0);
        const real wm1 = mid[m], wm0 = (real)1 - mid[m];
        const real wn1 = mid[n], wn0 = (real)1 - mid[n];
        real* J = src.c[l];
        atomicAdd(J + o, F * (wm0 * wn0 + cross));
        atomicAdd(J + o + st[m], F * (wm1 * wn0 - cross));
        atomicAdd(J + o + st[n], F * (wm0 * wn1 - cross));
        atomicAdd(J + o + st[m] + st[n], F * (wm1 * wn1 + cross));
    }
}

// Umeda zigzag of the move A -> B (relative to the base cell, |B - A| <= 1 per axis).
template <typename real>
__device__ __forceinline__ void zigzag(const real A[3], const real B[3], const int base[3], const Fields4<real>& src,
                                       const Geom& g, const PushConst& pc)
{
    int c1[3], c2[3];
    real R[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        c1[l] = (int)floor(A[l]);
        c2[l] = (int)floor(B[l]);
        const real lo = (real)min(c1[l], c2[l]), hi = (real)max(c1[l], c2[l]);
        const real mid = (real)0.5 * (A[l] + B[l]);
        R[l] = fmin(lo + (real)1, fmax(hi, mid));
    }
    deposit_piece(A, R, c1, base, src, g, pc);
    deposit_piece(R, B, c2, base, src, g, pc);
}

// Block-wide min/max of the cells this block deposited into (or will gather from next step),
// merged into box_out with one atomic per bound and block.
__device__ __forceinline__ void box_merge(int lo[3], int hi[3], int* box_out)
{
    __shared__ int sh[6][4];   // 128 threads = 4 warps
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int a = __reduce_min_sync(0xffffffffu, lo[d]);
        const int b = __reduce_max_sync(0xffffffffu, hi[d]);
        if (lane == 0) {
            sh[d][w] = a;
            sh[3 + d][w] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int q = threadIdx.x;
        int v = sh[q][0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) v = q < 3 ? min(v, sh[q][k]) : max(v, sh[q][k]);
        if (q < 3) {
            if (v != 0x7fffffff) atomicMin(box_out + q, v);
        } else if (v != (int)0x80000000) {
            atomicMax(box_out + q, v);
        }
    }
}

template <typename real>
__global__ void __launch_bounds__(128, sizeof(real) == 4 ? 6 : 5) k_push(Particles<real> P, int64_t np, Geom g, ExtField ef, Fields6<real> eb,
                                              Fields4<real> src, PushConst pc, int* box_out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff};
    int hi[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    if (p < np) {
        int ci[3] = {P.ix[p], P.iy[p], P.iz[p]};
        real f[3] = {P.fx[p], P.fy[p], P.fz[p]};
        double u[3] = {P.ux[p], P.uy[p], P.uz[p]};
        for (int m = 0; m < g.substeps; ++m) {
            double E[3], B[3];
            if ((std::is_same<real, float>::value ? (const void*)pc.ptab32[0] : (const void*)pc.ptab[0]) &&
                ci[2] >= 0 && ci[2] < g.nz) {
                if constexpr (std::is_same<real, float>::value) {
                    const float x = (float)g.x0 + ((float)ci[0] + f[0]) * (float)g.dx;
                    const float y = (float)g.y0 + ((float)ci[1] + f[1]) * (float)g.dy;
                    static_field_mixed(ef, pc, ci[2], f[2], m, x, y, E, B);
                } else {
                    const double x = g.x0 + ((double)ci[0] + (double)f[0]) * g.dx;
                    const double y = g.y0 + ((double)ci[1] + (double)f[1]) * g.dy;
                    static_field_fast(ef, pc, ci[2], (double)f[2], m, x, y, E, B);
                }
            } else {
                const double t = pc.t_half + (double)m * g.dtb;
                const double x = g.x0 + ((double)ci[0] + (double)f[0]) * g.dx;
                const double y = g.y0 + ((double)ci[1] + (double)f[1]) * g.dy;
                const double z = g.z0 + ((double)ci[2] + (double)f[2]) * g.dz;
                external_field(ef, x, y, z, t, E, B);
            }
            const bool a1 = active_cell(ci[0], ci[1], ci[2], g);
            real s[6] = {0, 0, 0, 0, 0, 0};
            if (a1) {
                const real wx[2] = {(real)1 - f[0], f[0]};
                const real wy[2] = {(real)1 - f[1], f[1]};
                const real wz[2] = {(real)1 - f[2], f[2]};
                const int64_t o = (int64_t)ci[2] * g.sz + (int64_t)ci[1] * g.sy + ci[0];
#pragma unroll
                for (int K = 0; K < 2; ++K)
#pragma unroll
                    for (int J = 0; J < 2; ++J)
#pragma unroll
                        for (int I = 0; I < 2; ++I) {
                            const real w = wx[I] * wy[J] * wz[K];
                            const int64_t id = o + K * g.sz + J * g.sy + I;
#pragma unroll
                            for (int c = 0; c < 6; ++c) s[c] += w * __ldg(eb.c[c] + id);
                        }
            }
            real ig;
            if constexpr (std::is_same<real, float>::value) {
                // Boris rotation in FP32 on the momentum rounded to FP32; its increment is added
                // to the FP64 momentum, and 1/gamma of the move comes from the FP64 momentum
                float uf[3] = {(float)u[0], (float)u[1], (float)u[2]};
                const float Et[3] = {(float)E[0] + s[0], (float)E[1] + s[1], (float)E[2] + s[2]};
                const float Bt[3] = {(float)B[0] + s[3], (float)B[1] + s[4], (float)B[2] + s[5]};
                const float u0[3] = {uf[0], uf[1], uf[2]};
                boris_f32(uf, Et, Bt, (float)g.dtb);
#pragma unroll
                for (int l = 0; l < 3; ++l) u[l] += (double)(uf[l] - u0[l]);
                ig = (float)rsqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    E[c] += (double)s[c];
                    B[c] += (double)s[3 + c];
                }
                boris(u, E, B, g.dtb);
                ig = 1.0 / sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            }
            real b[3];
            int nc[3];
            real nf[3];
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                b[l] = f[l] + (real)pc.cdtb[l] * ((real)u[l] * ig);
                const real fl = floor(b[l]);
                int c = (int)fl;
                real o = b[l] - fl;
                if (o >= (real)1) { o -= (real)1; c += 1; }
                b[l] = (real)c + o;   // the deposit ends exactly at the stored (cell, offset) point
                nc[l] = ci[l] + c;
                nf[l] = o;
            }
            if (a1 && active_cell(nc[0], nc[1], nc[2], g)) {
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    lo[l] = min(lo[l], min(ci[l], nc[l]));
                    hi[l] = max(hi[l], max(ci[l], nc[l]));
                }
                real mx = fmax(fabs(b[0] - f[0]), fmax(fabs(b[1] - f[1]), fabs(b[2] - f[2])));
                if (mx <= (real)1) {
                    zigzag(f, b, ci, src, g, pc);
                } else {
                    const int ns = (int)ceil((double)mx);
                    real A[3], Bq[3];
                    for (int s = 0; s < ns; ++s) {
#pragma unroll
                        for (int l = 0; l < 3; ++l) {
                            const real dl = b[l] - f[l];
                            A[l] = (s == 0) ? f[l] : f[l] + dl * ((real)s / (real)ns);
                            Bq[l] = (s == ns - 1) ? b[l] : f[l] + dl * ((real)(s + 1) / (real)ns);
                        }
                        zigzag(A, Bq, ci, src, g, pc);
                    }
                }
            }
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                ci[l] = nc[l];
                f[l] = nf[l];
            }
        }
        if (active_cell(ci[0], ci[1], ci[2], g)) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                lo[l] = min(lo[l], ci[l]);
                hi[l] = max(hi[l], ci[l]);
            }
            if (g.space_charge) {
                const real wx[2] = {(real)1 - f[0], f[0]};
                const real wy[2] = {(real)1 - f[1], f[1]};
                const real wz[2] = {(real)1 - f[2], f[2]};
                const int64_t o = (int64_t)ci[2] * g.sz + (int64_t)ci[1] * g.sy + ci[0];
                const real q = (real)pc.qrho;
#pragma unroll
                for (int K = 0; K < 2; ++K)
#pragma unroll
                    for (int J = 0; J < 2; ++J)
#pragma unroll
                        for (int I = 0; I < 2; ++I)
                            atomicAdd(src.c[3] + o + K * g.sz + J * g.sy + I, q * wx[I] * wy[J] * wz[K]);
            }
        }
        P.ix[p] = ci[0];
        P.iy[p] = ci[1];
        P.iz[p] = ci[2];
        P.fx[p] = f[0];
        P.fy[p] = f[1];
        P.fz[p] = f[2];
        P.ux[p] = u[0];
        P.uy[p] = u[1];
        P.uz[p] = u[2];
    }
    box_merge(lo, hi, box_out);
}

// Lab-frame macro-particles (x, y, z relative to the bunch reference at t' = 0, gamma*beta) to
// the rest frame at the common time T0 + dt/2 (the time of r^{1/2}).
template <typename real>
__global__ void k_boost(const double* __restrict__ lab, int64_t np, Particles<real> P, Geom g, double g0, double b0,
                        double z_ref)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double* L = lab + 6 * p;
    const double ux = L[3], uy = L[4], uzl = L[5];
    const double gl = sqrt(1.0 + ux * ux + uy * uy + uzl * uzl);
    const double uz = g0 * (uzl - b0 * gl);
    const double ig = 1.0 / sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    // ballistic shift with the rest-frame velocity over c (T0 + dt/2 - t_event)
    const double s = g0 * b0 * L[2] + 0.5 * kC * g.dt;
    const double x = L[0] + ux * ig * s;
    const double y = L[1] + uy * ig * s;
    const double z = z_ref + g0 * L[2] + uz * ig * s;
    split_pos<real>((x - g.x0) / g.dx, P.ix + p, P.fx + p);
    split_pos<real>((y - g.y0) / g.dy, P.iy + p, P.fy + p);
    split_pos<real>((z - g.z0) / g.dz, P.iz + p, P.fz + p);
    P.ux[p] = ux;
    P.uy[p] = uy;
    P.uz[p] = uz;
    P.id[p] = (int32_t)p;
}

template <typename real>
__global__ void k_set_rest(const double* __restrict__ r6, int64_t np, Particles<real> P, Geom g)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double* R = r6 + 6 * p;
    split_pos<real>((R[0] - g.x0) / g.dx, P.ix + p, P.fx + p);
    split_pos<real>((R[1] - g.y0) / g.dy, P.iy + p, P.fy + p);
    split_pos<real>((R[2] - g.z0) / g.dz, P.iz + p, P.fz + p);
    P.ux[p] = R[3];
    P.uy[p] = R[4];
    P.uz[p] = R[5];
    P.id[p] = (int32_t)p;
}

template <typename real>
__global__ void k_get_rest(Particles<real> P, int64_t np, Geom g, double* __restrict__ r6)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double* R = r6 + 6 * (int64_t)P.id[p];
    R[0] = g.x0 + ((double)P.ix[p] + (double)P.fx[p]) * g.dx;
    R[1] = g.y0 + ((double)P.iy[p] + (double)P.fy[p]) * g.dy;
    R[2] = g.z0 + ((double)P.iz[p] + (double)P.fz[p]) * g.dz;
    R[3] = P.ux[p];
    R[4] = P.uy[p];
    R[5] = P.uz[p];
}

static inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename real>
cudaError_t launch_push(const Particles<real>& P, int64_t np, const Geom& g, const ExtField& ef,
                        const Fields6<real>& eb, const Fields4<real>& src, const PushConst& pc, int* box_out,
                        cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_push<real><<<nblocks(np, 128), 128, 0, st>>>(P, np, g, ef, eb, src, pc, box_out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_boost(const double* lab6, int64_t np, const Particles<real>& P, const Geom& g, const ExtField& ef,
                         double z_ref, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_boost<real><<<nblocks(np, 256), 256, 0, st>>>(lab6, np, P, g, ef.g0, ef.b0, z_ref);
    count_launches(1);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_set_rest(const double* rest6, int64_t np, const Particles<real>& P, const Geom& g, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_set_rest<real><<<nblocks(np, 256), 256, 0, st>>>(rest6, np, P, g);
    count_launches(1);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_get_rest(const Particles<real>& P, int64_t np, const Geom& g, double* rest6, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_get_rest<real><<<nblocks(np, 256), 256, 0, st>>>(P, np, g, rest6);
    count_launches(1);
    return cudaGetLastError();
}

#define MITHRA_INST(real)                                                                                              \
    template cudaError_t launch_push<real>(const Particles<real>&, int64_t, const Geom&, const ExtField&,             \
                                           const Fields6<real>&, const Fields4<real>&, const PushConst&, int*,       \
                                           cudaStream_t);                                                              \
    template cudaError_t launch_boost<real>(const double*, int64_t, const Particles<real>&, const Geom&,              \
                                            const ExtField&, double, cudaStream_t);                                   \
    template cudaError_t launch_set_rest<real>(const double*, int64_t, const Particles<real>&, const Geom&,           \
                                               cudaStream_t);                                                          \
    template cudaError_t launch_get_rest<real>(const Particles<real>&, int64_t, const Geom&, double*, cudaStream_t);
MITHRA_INST(float)
MITHRA_INST(double)
#undef MITHRA_INST

}  // namespace mithra
