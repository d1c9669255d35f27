// Field kernels: potential update (manual Eq. updateEquation; FD = NSFD with A = 0),
// Mur absorbing boundaries (Sec. "Boundary Truncation") and E, B at nodes
// (Sec. "Field Evaluation").
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
};

__device__ inline int64_t lin(int i, int j, int k, int64_t sy, int64_t sz) { return (int64_t)k * sz + (int64_t)j * sy + i; }

// Decode face point `t` of a lattice (e[0], e[1], e[2]): 6 faces, each interior of the
// other two axes.  Returns false when t is beyond the face count.
__device__ inline bool face_point(int64_t t, const int e[3], int ijk[3], int* axis, int* side)
{
    for (int a = 0; a < 3; ++a) {
        const int u = (a + 1) % 3, v = (a + 2) % 3;
        const int64_t nf = (int64_t)(e[u] - 2) * (e[v] - 2);
        for (int sd = 0; sd < 2; ++sd) {
            if (t < nf) {
                ijk[a] = sd ? e[a] - 1 : 0;
                ijk[u] = 1 + (int)(t % (e[u] - 2));
                ijk[v] = 1 + (int)(t / (e[u] - 2));
                *axis = a;
                *side = sd;
                return true;
            }
            t -= nf;
        }
    }
    return false;
}

template <typename real>
__global__ void k_mur_faces(MurArgs<real> a, int64_t sy, int64_t sz, int64_t maxpts)
{
    const int comp = blockIdx.y;
    if (comp >= a.ncomp) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= maxpts) return;
    const int e[3] = {a.ex[comp], a.ey[comp], a.ez[comp]};
    int p[3], ax, sd;
    if (!face_point(t, e, p, &ax, &sd)) return;
    real* __restrict__ n1 = a.n1[comp];
    const real* __restrict__ n0 = a.n0[comp];
    const real* __restrict__ nm = a.nm[comp];
    int q[3] = {p[0], p[1], p[2]};
    q[ax] += sd ? -1 : 1;   // inward neighbour
    const int64_t ib = lin(p[0], p[1], p[2], sy, sz), iq = lin(q[0], q[1], q[2], sy, sz);
    const double D = a.D[ax], cdt = a.cdt;
    const double den = 1.0 / (cdt + D);
    double v;
    if (a.order == 1) {
        const double b0 = (cdt - D) * den, b1 = 2.0 * D * den;
        v = b0 * (double)nm[ib] + b1 * (double)n0[ib] - (double)nm[iq] + b1 * (double)n0[iq] + b0 * (double)n1[iq];
    } else {
        const int u = (ax + 1) % 3, w = (ax + 2) % 3;
        const double ru = (cdt / a.D[u]) * (cdt / a.D[u]), rw = (cdt / a.D[w]) * (cdt / a.D[w]);
        const double g0 = (cdt - D) * den, g1 = D * (2.0 - ru - rw) * den;
        const double gu = 0.5 * ru * D * den, gw = 0.5 * rw * D * den;
        int t1[3], t2[3];
        double sb = 0.0, sq = 0.0;   // transverse neighbours on the face and on the inner plane
        for (int s = 0; s < 2; ++s) {
            const int ta = s ? w : u;
            const double gt = s ? gw : gu;
            for (int d = -1; d <= 1; d += 2) {
                t1[0] = p[0]; t1[1] = p[1]; t1[2] = p[2];
                t2[0] = q[0]; t2[1] = q[1]; t2[2] = q[2];
                t1[ta] += d;
                t2[ta] += d;
                sb += gt * (double)n0[lin(t1[0], t1[1], t1[2], sy, sz)];
                sq += gt * (double)n0[lin(t2[0], t2[1], t2[2], sy, sz)];
            }
        }
        v = g0 * (double)nm[ib] + g1 * (double)n0[ib] - (double)nm[iq] + g1 * (double)n0[iq] + g0 * (double)n1[iq] + sb + sq;
    }
    n1[ib] = (real)v;
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
// n+1) and phi^n:  E = -(A^{n+1} - A^n)/dt - grad_c phi,  B = (curl_c A^n + curl_c A^{n+1}) / 2.
// Each thread walks a chunk of z for one (i, j) node column.
// ---------------------------------------------------------------------------------------
template <typename real>
struct EmitArgs {
    const real* a0[3];   // A^n
    const real* a1[3];   // A^{n+1}
    const real* phi;     // phi^n (node), may be null when space charge is off
    real* eb[6];
    double idt, i2dx, i2dy, i2dz;
    int kchunk;
};

template <typename real>
__device__ inline double anode(const real* __restrict__ A, int64_t id, int64_t back)
{
    return 0.5 * ((double)__ldg(A + id) + (double)__ldg(A + id - back));
}

template <typename real>
__global__ void __launch_bounds__(256) k_emit(EmitArgs<real> a, Geom g)
{
    const int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 1 + blockIdx.y * blockDim.y + threadIdx.y;
    if (i > g.nx - 2 || j > g.ny - 2) return;
    const int k0 = 1 + blockIdx.z * a.kchunk;
    const int k1 = min(g.nz - 2, k0 + a.kchunk - 1);
    const int64_t sy = g.sy, sz = g.sz;
    for (int k = k0; k <= k1; ++k) {
        const int64_t id = (int64_t)k * sz + (int64_t)j * sy + i;
        double E[3], B[3] = {0.0, 0.0, 0.0};
        const int64_t back[3] = {1, sy, sz};
        for (int c = 0; c < 3; ++c)
            E[c] = -(anode(a.a1[c], id, back[c]) - anode(a.a0[c], id, back[c])) * a.idt;
        if (a.phi) {
            E[0] -= ((double)__ldg(a.phi + id + 1) - (double)__ldg(a.phi + id - 1)) * a.i2dx;
            E[1] -= ((double)__ldg(a.phi + id + sy) - (double)__ldg(a.phi + id - sy)) * a.i2dy;
            E[2] -= ((double)__ldg(a.phi + id + sz) - (double)__ldg(a.phi + id - sz)) * a.i2dz;
        }
        for (int l = 0; l < 2; ++l) {
            const real* const* A = l ? a.a1 : a.a0;
            B[0] += (anode(A[2], id + sy, sz) - anode(A[2], id - sy, sz)) * a.i2dy
                  - (anode(A[1], id + sz, sy) - anode(A[1], id - sz, sy)) * a.i2dz;
            B[1] += (anode(A[0], id + sz, 1) - anode(A[0], id - sz, 1)) * a.i2dz
                  - (anode(A[2], id + 1, sz) - anode(A[2], id - 1, sz)) * a.i2dx;
            B[2] += (anode(A[1], id + 1, sy) - anode(A[1], id - 1, sy)) * a.i2dx
                  - (anode(A[0], id + sy, 1) - anode(A[0], id - sy, 1)) * a.i2dy;
        }
        a.eb[0][id] = (real)E[0];
        a.eb[1][id] = (real)E[1];
        a.eb[2][id] = (real)E[2];
        a.eb[3][id] = (real)(0.5 * B[0]);
        a.eb[4][id] = (real)(0.5 * B[1]);
        a.eb[5][id] = (real)(0.5 * B[2]);
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
    const int64_t nx = g.nx, ny = g.ny, nz = g.nz;
    const int64_t faces = 2 * ((ny - 2) * (nz - 2) + (nx - 2) * (nz - 2) + (nx - 2) * (ny - 2));
    const int64_t edges = 4 * ((nx - 2) + (ny - 2) + (nz - 2));
    const int thr = 256;
    k_mur_faces<real><<<dim3((unsigned)((faces + thr - 1) / thr), ncomp), thr, 0, st>>>(a, g.sy, g.sz, faces);
    k_mur_edges<real><<<dim3((unsigned)((edges + thr - 1) / thr), ncomp), thr, 0, st>>>(a, g.sy, g.sz, 2, edges);
    k_mur_edges<real><<<dim3(1, ncomp), 32, 0, st>>>(a, g.sy, g.sz, 3, 8);
    count_launches(3);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_emit(const FieldLevels<real>& L, const Fields6<real>& eb, const Geom& g, cudaStream_t st)
{
    EmitArgs<real> a;
    for (int c = 0; c < 3; ++c) {
        a.a0[c] = L.n0[c];
        a.a1[c] = L.n1[c];
    }
    a.phi = g.space_charge ? L.n0[3] : nullptr;
    for (int c = 0; c < 6; ++c) a.eb[c] = eb.c[c];
    a.idt = 1.0 / g.dt;
    a.i2dx = 0.5 / g.dx;
    a.i2dy = 0.5 / g.dy;
    a.i2dz = 0.5 / g.dz;
    a.kchunk = 16;
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
template cudaError_t launch_emit<float>(const FieldLevels<float>&, const Fields6<float>&, const Geom&, cudaStream_t);
template cudaError_t launch_emit<double>(const FieldLevels<double>&, const Fields6<double>&, const Geom&, cudaStream_t);

}  // namespace mithra
