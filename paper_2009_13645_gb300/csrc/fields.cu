// Field kernels: potential update (manual Eq. updateEquation; FD = NSFD with A = 0),
// Mur absorbing boundaries (Sec. "Boundary Truncation") and E, B at nodes
// (Sec. "Field Evaluation").
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace mithra {

// ---------------------------------------------------------------------------------------
// Stencil.  Each thread owns one (i, j) column of one component lattice and marches a
// chunk of z planes, keeping the three planes k-1, k, k+1 of its own column and of its four
// transverse neighbours in registers, so that every psi^n value is loaded once per column
// that needs it (the 4 neighbour loads per plane hit L1/L2).
// ---------------------------------------------------------------------------------------
template <typename real>
struct StencilArgs {
    const real* pn[4];   // psi^{n}   (level n+1 of the step)
    const real* pm[4];   // psi^{n-1} (level n of the step)
    const real* src[4];  // J_x, J_y, J_z, rho
    real* out[4];        // psi^{n+1}
    real a1, ax, ay, a6, w, w0, s[4];   // coefficients; w = A, w0 = 1 - 2A; s = (c dt)^2 mu0 | (c dt)^2 / eps0
    int ex[4], ey[4], ez[4];            // extents of each component lattice
    int ncomp;
    int kchunk;
};

template <typename real>
__global__ void __launch_bounds__(256) k_stencil(StencilArgs<real> a, int64_t sy, int64_t sz)
{
    const int comp = blockIdx.z % a.ncomp;
    const int chunk = blockIdx.z / a.ncomp;
    const int ex = a.ex[comp], ey = a.ey[comp], ez = a.ez[comp];
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i > ex - 2 || j > ey - 2) return;
    const int k0 = 1 + chunk * a.kchunk;
    if (k0 > ez - 2) return;
    const int k1 = min(ez - 2, k0 + a.kchunk - 1);
    const real* __restrict__ p = a.pn[comp];
    const real* __restrict__ pm = a.pm[comp];
    const real* __restrict__ S = a.src[comp];
    real* __restrict__ o = a.out[comp];
    const real s = a.s[comp];
    const int64_t col = (int64_t)j * sy + i;
    // registers: [0] = k-1, [1] = k, [2] = k+1
    real c0, c1, c2, xp0, xp1, xp2, xm0, xm1, xm2, yp0, yp1, yp2, ym0, ym1, ym2;
    {
        const int64_t b0 = col + (int64_t)(k0 - 1) * sz, b1 = b0 + sz;
        c0 = __ldg(p + b0); c1 = __ldg(p + b1);
        xp0 = __ldg(p + b0 + 1); xp1 = __ldg(p + b1 + 1);
        xm0 = __ldg(p + b0 - 1); xm1 = __ldg(p + b1 - 1);
        yp0 = __ldg(p + b0 + sy); yp1 = __ldg(p + b1 + sy);
        ym0 = __ldg(p + b0 - sy); ym1 = __ldg(p + b1 - sy);
    }
    for (int k = k0; k <= k1; ++k) {
        const int64_t b = col + (int64_t)k * sz;
        const int64_t b2 = b + sz;
        c2 = __ldg(p + b2);
        xp2 = __ldg(p + b2 + 1);
        xm2 = __ldg(p + b2 - 1);
        yp2 = __ldg(p + b2 + sy);
        ym2 = __ldg(p + b2 - sy);
        // z-averaged transverse neighbours (Eq. NSFDtrick)
        const real bxp = a.w * (xp0 + xp2) + a.w0 * xp1;
        const real bxm = a.w * (xm0 + xm2) + a.w0 * xm1;
        const real byp = a.w * (yp0 + yp2) + a.w0 * yp1;
        const real bym = a.w * (ym0 + ym2) + a.w0 * ym1;
        const real v = a.a1 * c1 - __ldg(pm + b) + a.ax * (bxp + bxm) + a.ay * (byp + bym) + a.a6 * (c0 + c2)
                     + s * __ldg(S + b);
        o[b] = v;
        c0 = c1; c1 = c2;
        xp0 = xp1; xp1 = xp2;
        xm0 = xm1; xm1 = xm2;
        yp0 = yp1; yp1 = yp2;
        ym0 = ym1; ym1 = ym2;
    }
}

// ---------------------------------------------------------------------------------------
// Mur boundaries.  Points are classified by how many of their coordinates lie on a
// boundary of their lattice: faces (1), edges (2), corners (3).  Faces use the manual's
// beta / gamma update; edges and corners sum the first-order conditions of the meeting
// faces discretised at the centre of the square / cube formed with their inward
// neighbours, which gives the closed form
//   v = [ sum_{e!=0} f1_e (W_e - g) - sum_e fm_e (W_e + g) + 2 g sum_e fn_e ] / (sum_a w_a + g)
// with w_a = 1 / (2 dt D_a 2^{s-1}), W_e = sum_a w_a (+1 if e_a else -1), g = s / (c dt^2 2^s).
// Faces run first, then edges, then corners (each reads the previous class at n+1).
// ---------------------------------------------------------------------------------------
template <typename real>
struct MurArgs {
    real* n1[4];         // level n+1 (written)
    const real* n0[4];   // level n
    const real* nm[4];   // level n-1
    int ex[4], ey[4], ez[4];
    int ncomp;
    int order;
    double cdt, dt, D[3];
    // face coefficients per normal axis, in the storage type: first order beta_0 (= beta_4),
    // beta_1 (= beta_3); second order gamma_0, gamma_1 and the tangential gammas of the axes
    // (a+1)%3 and (a+2)%3
    real f0[3], f1[3], ft[3][2];
};

__device__ inline int64_t lin(int i, int j, int k, int64_t sy, int64_t sz) { return (int64_t)k * sz + (int64_t)j * sy + i; }

// One face per blockIdx.z (axis = z / 2, side = z % 2), one component per blockIdx.y.
template <typename real>
__global__ void k_mur_faces(MurArgs<real> a, int64_t sy, int64_t sz)
{
    const int comp = blockIdx.y;
    if (comp >= a.ncomp) return;
    const int ax = blockIdx.z >> 1, sd = blockIdx.z & 1;
    const int e[3] = {a.ex[comp], a.ey[comp], a.ez[comp]};
    const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;   // tangential axes, u before v
    const int nu = e[u] - 2, nv = e[v] - 2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nu * nv) return;
    int p[3];
    p[ax] = sd ? e[ax] - 1 : 0;
    p[u] = 1 + t % nu;
    p[v] = 1 + t / nu;
    const int64_t st[3] = {1, sy, sz};
    const int64_t ib = lin(p[0], p[1], p[2], sy, sz);
    const int64_t iq = ib + (sd ? -st[ax] : st[ax]);   // inward neighbour
    real* __restrict__ n1 = a.n1[comp];
    const real* __restrict__ n0 = a.n0[comp];
    const real* __restrict__ nm = a.nm[comp];
    real vout;
    if (a.order == 1) {
        const real b0 = a.f0[ax], b1 = a.f1[ax];
        vout = b0 * (nm[ib] + n1[iq]) + b1 * (n0[ib] + n0[iq]) - nm[iq];
    } else {
        // tangential neighbours at level n on the face and on the inner plane
        const int ta = (ax + 1) % 3, tb = (ax + 2) % 3;
        const real ga = a.ft[ax][0], gb = a.ft[ax][1];
        const real sa = n0[ib + st[ta]] + n0[ib - st[ta]] + n0[iq + st[ta]] + n0[iq - st[ta]];
        const real sb = n0[ib + st[tb]] + n0[ib - st[tb]] + n0[iq + st[tb]] + n0[iq - st[tb]];
        vout = a.f0[ax] * (nm[ib] + n1[iq]) + a.f1[ax] * (n0[ib] + n0[iq]) - nm[iq] + ga * sa + gb * sb;
    }
    n1[ib] = vout;
}

// Edges (cls = 2) and corners (cls = 3).
template <typename real>
__global__ void k_mur_edges(MurArgs<real> a, int64_t sy, int64_t sz, int cls, int64_t maxpts)
{
    const int comp = blockIdx.y;
    if (comp >= a.ncomp) return;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= maxpts) return;
    const int e[3] = {a.ex[comp], a.ey[comp], a.ez[comp]};
    int p[3], sg[3], axes[3], ns = 0;
    if (cls == 3) {
        if (t >= 8) return;
        for (int d = 0; d < 3; ++d) {
            const int hi = (t >> d) & 1;
            p[d] = hi ? e[d] - 1 : 0;
            sg[ns] = hi ? -1 : 1;
            axes[ns++] = d;
        }
    } else {
        // 12 edges: the free axis f runs over 1..e[f]-2, the two others sit on a boundary
        bool found = false;
        for (int f = 0; f < 3 && !found; ++f) {
            const int64_t len = e[f] - 2;
            for (int c = 0; c < 4 && !found; ++c) {
                if (t < len) {
                    const int u = (f + 1) % 3, v = (f + 2) % 3;
                    p[f] = 1 + (int)t;
                    p[u] = (c & 1) ? e[u] - 1 : 0;
                    p[v] = (c & 2) ? e[v] - 1 : 0;
                    const int lo = u < v ? u : v, hi = u < v ? v : u;
                    axes[0] = lo;
                    axes[1] = hi;
                    sg[0] = (p[lo] == 0) ? 1 : -1;
                    sg[1] = (p[hi] == 0) ? 1 : -1;
                    ns = 2;
                    found = true;
                } else {
                    t -= len;
                }
            }
        }
        if (!found) return;
    }
    real* __restrict__ n1 = a.n1[comp];
    const real* __restrict__ n0 = a.n0[comp];
    const real* __restrict__ nm = a.nm[comp];
    const int npts = 1 << ns;
    const double h = (double)(npts >> 1);
    double wa[3], wsum = 0.0;
    for (int s = 0; s < ns; ++s) {
        wa[s] = 1.0 / (2.0 * a.dt * a.D[axes[s]] * h);
        wsum += wa[s];
    }
    const double g = (double)ns / (kC * a.dt * a.dt * (double)npts);
    double num = 0.0;
    for (int ei = 0; ei < npts; ++ei) {
        int q[3] = {p[0], p[1], p[2]};
        double W = 0.0;
        for (int s = 0; s < ns; ++s) {
            const bool on = (ei >> s) & 1;
            if (on) q[axes[s]] += sg[s];
            W += on ? wa[s] : -wa[s];
        }
        const int64_t id = lin(q[0], q[1], q[2], sy, sz);
        if (ei != 0) num += (double)n1[id] * (W - g);
        num += -(double)nm[id] * (W + g) + 2.0 * g * (double)n0[id];
    }
    n1[lin(p[0], p[1], p[2], sy, sz)] = (real)(num / (wsum + g));
}

// ---------------------------------------------------------------------------------------
// E and B at interior nodes from node averages of the staggered potentials (levels n and
// n+1) and phi^n:  E = -(A^{n+1} - A^n)/dt - grad_c phi,  B = (curl_c A^n + curl_c A^{n+1}) / 2,
// in the storage type.  Per step only the nodes the particles will gather from (the box the
// push kernel reduced from the cells it deposited into) and the power plane are needed; inside
// that box the sources of the previous step are cleared in the same pass.  With box == null the
// whole interior is emitted (diagnostics) and nothing is cleared.
// ---------------------------------------------------------------------------------------
template <typename real>
struct EmitArgs {
    const real* a0[3];   // A^n
    const real* a1[3];   // A^{n+1}
    const real* phi;     // phi^n (node), may be null when space charge is off
    real* eb[6];
    real* src[4];        // sources to clear inside the box (entries may be null)
    real idt, i2dx, i2dy, i2dz;
    int kchunk;
    int kp;              // plane emitted in full (< 0: none)
    const int* box;      // cells [lo_x, lo_y, lo_z, hi_x, hi_y, hi_z] of the last deposit; null: whole grid
    int* box_reset;      // box the next push reduces into: reset to empty here (may be null)
};

template <typename real>
__device__ __forceinline__ real navg(const real* __restrict__ A, int64_t id, int64_t back)
{
    return (real)0.5 * (__ldg(A + id) + __ldg(A + id - back));
}

template <typename real>
__global__ void __launch_bounds__(256) k_emit(EmitArgs<real> a, Geom g)
{
    const int i0 = 1 + blockIdx.x * blockDim.x, j0 = 1 + blockIdx.y * blockDim.y;
    const int k0 = 1 + blockIdx.z * a.kchunk;
    const int k1 = min(g.nz - 2, k0 + a.kchunk - 1);
    if (a.box_reset && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x < 6 && threadIdx.y == 0)
        a.box_reset[threadIdx.x] = threadIdx.x < 3 ? 0x7fffffff : (int)0x80000000;
    // nodes [lo - 1, hi + 2] around the cells of the last deposit: the particles gather at their
    // cells' nodes next step, and with sub-steps they move up to one cell during that step
    int bl[3] = {1, 1, 1}, bh[3] = {g.nx - 2, g.ny - 2, g.nz - 2};
    if (a.box) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bl[d] = __ldg(a.box + d) - 1;
            bh[d] = __ldg(a.box + 3 + d) + 2;
        }
    }
    const bool plane_here = a.kp >= k0 && a.kp <= k1;
    const bool box_here = bl[0] <= min(bh[0], i0 + (int)blockDim.x - 1) && bh[0] >= i0 &&
                          bl[1] <= min(bh[1], j0 + (int)blockDim.y - 1) && bh[1] >= j0 && bl[2] <= min(bh[2], k1) &&
                          bh[2] >= k0;
    if (!plane_here && !box_here) return;
    const int i = i0 + threadIdx.x, j = j0 + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    const bool col_in = i >= bl[0] && i <= bh[0] && j >= bl[1] && j <= bh[1];
    const int64_t sy = g.sy, sz = g.sz;
    const int64_t back[3] = {1, sy, sz};
    for (int k = k0; k <= k1; ++k) {
        const bool in = col_in && k >= bl[2] && k <= bh[2];
        if (!in && k != a.kp) continue;
        const int64_t id = (int64_t)k * sz + (int64_t)j * sy + i;
        if (in && a.box) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (a.src[c]) a.src[c][id] = (real)0;
        }
        real E[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) E[c] = (navg(a.a0[c], id, back[c]) - navg(a.a1[c], id, back[c])) * a.idt;
        if (a.phi) {
            E[0] -= (__ldg(a.phi + id + 1) - __ldg(a.phi + id - 1)) * a.i2dx;
            E[1] -= (__ldg(a.phi + id + sy) - __ldg(a.phi + id - sy)) * a.i2dy;
            E[2] -= (__ldg(a.phi + id + sz) - __ldg(a.phi + id - sz)) * a.i2dz;
        }
        // node-averaged sums of the two levels, S_c = A_c^n + A_c^{n+1}, at the six neighbours
        auto S = [&](int c, int64_t at) { return navg(a.a0[c], at, back[c]) + navg(a.a1[c], at, back[c]); };
        const real bx = (S(2, id + sy) - S(2, id - sy)) * a.i2dy - (S(1, id + sz) - S(1, id - sz)) * a.i2dz;
        const real by = (S(0, id + sz) - S(0, id - sz)) * a.i2dz - (S(2, id + 1) - S(2, id - 1)) * a.i2dx;
        const real bz = (S(1, id + 1) - S(1, id - 1)) * a.i2dx - (S(0, id + sy) - S(0, id - sy)) * a.i2dy;
        a.eb[0][id] = E[0];
        a.eb[1][id] = E[1];
        a.eb[2][id] = E[2];
        a.eb[3][id] = (real)0.5 * bx;
        a.eb[4][id] = (real)0.5 * by;
        a.eb[5][id] = (real)0.5 * bz;
    }
}

// ---------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------
template <typename real>
cudaError_t launch_stencil(const FieldLevels<real>& L, const Geom& g, const StencilCoef& cf, int ncomp,
                           cudaStream_t st)
{
    StencilArgs<real> a;
    for (int c = 0; c < 4; ++c) {
        a.pn[c] = L.n1[c];
        a.pm[c] = L.n0[c];
        a.src[c] = L.src[c];
        a.out[c] = L.out[c];
        a.ex[c] = g.nx - (c == 0);
        a.ey[c] = g.ny - (c == 1);
        a.ez[c] = g.nz - (c == 2);
        a.s[c] = (real)(c < 3 ? cf.s_a : cf.s_phi);
    }
    a.a1 = (real)cf.a1;
    a.ax = (real)cf.ax;
    a.ay = (real)cf.ay;
    a.a6 = (real)cf.a6;
    a.w = (real)cf.w;
    a.w0 = (real)cf.w0;
    a.ncomp = ncomp;
    a.kchunk = 32;
    const dim3 blk(32, 8);
    const int nchunk = (g.nz - 2 + a.kchunk - 1) / a.kchunk;
    const dim3 grd((g.nx - 2 + 31) / 32, (g.ny - 2 + 7) / 8, nchunk * ncomp);
    k_stencil<real><<<grd, blk, 0, st>>>(a, g.sy, g.sz);
    count_launches(1);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mur(const FieldLevels<real>& L, const Geom& g, int order, int ncomp, cudaStream_t st)
{
    MurArgs<real> a;
    for (int c = 0; c < 4; ++c) {
        a.n1[c] = L.out[c];
        a.n0[c] = L.n1[c];
        a.nm[c] = L.n0[c];
        a.ex[c] = g.nx - (c == 0);
        a.ey[c] = g.ny - (c == 1);
        a.ez[c] = g.nz - (c == 2);
    }
    a.ncomp = ncomp;
    a.order = order;
    a.cdt = kC * g.dt;
    a.dt = g.dt;
    a.D[0] = g.dx;
    a.D[1] = g.dy;
    a.D[2] = g.dz;
    for (int ax = 0; ax < 3; ++ax) {
        const double D = a.D[ax], cdt = a.cdt, den = 1.0 / (cdt + D);
        if (order == 1) {
            a.f0[ax] = (real)((cdt - D) * den);            // beta_0 = beta_4
            a.f1[ax] = (real)(2.0 * D * den);              // beta_1 = beta_3
            a.ft[ax][0] = a.ft[ax][1] = (real)0;
        } else {
            const int ta = (ax + 1) % 3, tb = (ax + 2) % 3;
            const double ra = (cdt / a.D[ta]) * (cdt / a.D[ta]), rb = (cdt / a.D[tb]) * (cdt / a.D[tb]);
            a.f0[ax] = (real)((cdt - D) * den);            // gamma_0 = gamma_4
            a.f1[ax] = (real)(D * (2.0 - ra - rb) * den);  // gamma_1 = gamma_3
            a.ft[ax][0] = (real)(0.5 * ra * D * den);      // gamma of the (ax+1) neighbours
            a.ft[ax][1] = (real)(0.5 * rb * D * den);      // gamma of the (ax+2) neighbours
        }
    }
    int64_t maxface = 0;
    for (int c = 0; c < ncomp; ++c) {
        const int64_t e[3] = {a.ex[c], a.ey[c], a.ez[c]};
        for (int ax = 0; ax < 3; ++ax) {
            const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;
            maxface = std::max<int64_t>(maxface, (e[u] - 2) * (e[v] - 2));
        }
    }
    const int64_t nx = g.nx, ny = g.ny, nz = g.nz;
    const int64_t edges = 4 * ((nx - 2) + (ny - 2) + (nz - 2));
    const int thr = 256;
    k_mur_faces<real><<<dim3((unsigned)((maxface + thr - 1) / thr), ncomp, 6), thr, 0, st>>>(a, g.sy, g.sz);
    k_mur_edges<real><<<dim3((unsigned)((edges + thr - 1) / thr), ncomp), thr, 0, st>>>(a, g.sy, g.sz, 2, edges);
    k_mur_edges<real><<<dim3(1, ncomp), 32, 0, st>>>(a, g.sy, g.sz, 3, 8);
    count_launches(3);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_emit(const FieldLevels<real>& L, const Fields6<real>& eb, const Geom& g, const EmitBox& bx,
                        cudaStream_t st)
{
    EmitArgs<real> a;
    for (int c = 0; c < 3; ++c) {
        a.a0[c] = L.n0[c];
        a.a1[c] = L.n1[c];
    }
    a.phi = g.space_charge ? L.n0[3] : nullptr;
    for (int c = 0; c < 6; ++c) a.eb[c] = eb.c[c];
    for (int c = 0; c < 4; ++c) a.src[c] = (bx.box && bx.clear) ? (real*)L.src[c] : nullptr;
    if (!g.space_charge) a.src[3] = nullptr;
    a.idt = (real)(1.0 / g.dt);
    a.i2dx = (real)(0.5 / g.dx);
    a.i2dy = (real)(0.5 / g.dy);
    a.i2dz = (real)(0.5 / g.dz);
    a.kchunk = 16;
    a.kp = bx.kp;
    a.box = bx.box;
    a.box_reset = bx.box_reset;
    a.kchunk = bx.box ? 4 : 16;   // short z chunks spread the box over more blocks
    const dim3 blk(32, 8);
    const dim3 grd((g.nx - 2 + 31) / 32, (g.ny - 2 + 7) / 8, (g.nz - 2 + a.kchunk - 1) / a.kchunk);
    k_emit<real><<<grd, blk, 0, st>>>(a, g);
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_stencil<float>(const FieldLevels<float>&, const Geom&, const StencilCoef&, int, cudaStream_t);
template cudaError_t launch_stencil<double>(const FieldLevels<double>&, const Geom&, const StencilCoef&, int, cudaStream_t);
template cudaError_t launch_mur<float>(const FieldLevels<float>&, const Geom&, int, int, cudaStream_t);
template cudaError_t launch_mur<double>(const FieldLevels<double>&, const Geom&, int, int, cudaStream_t);
template cudaError_t launch_emit<float>(const FieldLevels<float>&, const Fields6<float>&, const Geom&, const EmitBox&,
                                        cudaStream_t);
template cudaError_t launch_emit<double>(const FieldLevels<double>&, const Fields6<double>&, const Geom&,
                                         const EmitBox&, cudaStream_t);

}  // namespace mithra
