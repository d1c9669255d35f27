// Field kernels: potential update (manual Eq. updateEquation; FD = NSFD with A = 0),
// Mur absorbing boundaries (Sec. "Boundary Truncation") and E, B at nodes
// (Sec. "Field Evaluation").
#include <algorithm>
#include <cstring>
#include <utility>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace mithra {

// ---------------------------------------------------------------------------------------
// Stencil.  Each thread owns one (i, j) column of one component lattice and marches a
// chunk of z planes, keeping the three planes k-1, k, k+1 of its own column and the sums of its
// two x neighbours and of its two y neighbours in registers, so that every psi^n value is loaded
// once per column that needs it (the 4 neighbour loads per plane hit L1/L2) and each sum is
// formed once for the three updates that read it.
// ---------------------------------------------------------------------------------------
template <typename real>
struct StencilArgs {
    const real* pn[4];   // psi^{n}   (level n+1 of the step)
    const real* pm[4];   // psi^{n-1} (level n of the step)
    const real* src[4];  // J_x, J_y, J_z, rho
    real* out[4];        // psi^{n+1}
    real a1, ax, ay, a6, w, w0, s[4];   // coefficients; w = A, w0 = 1 - 2A; s = (c dt)^2 mu0 | (c dt)^2 / eps0
    real axw, axw0, ayw, ayw0;          // ax w, ax w0, ay w, ay w0 (products taken in FP64)
    int ex[4], ey[4], ez[4];            // extents of each component lattice
    int ncomp;
    int kchunk;
};

template <typename real>
__global__ void __launch_bounds__(256) k_stencil(StencilArgs<real> a, int64_t sy, int64_t sz)
{
    dep_begin();
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
    // registers: [0] = k-1, [1] = k, [2] = k+1; X = x-1 + x+1, Y = y-1 + y+1
    real c0, c1, c2, X0, X1, X2, Y0, Y1, Y2;
    {
        const int64_t b0 = col + (int64_t)(k0 - 1) * sz, b1 = b0 + sz;
        c0 = __ldg(p + b0);
        c1 = __ldg(p + b1);
        X0 = __ldg(p + b0 + 1) + __ldg(p + b0 - 1);
        X1 = __ldg(p + b1 + 1) + __ldg(p + b1 - 1);
        Y0 = __ldg(p + b0 + sy) + __ldg(p + b0 - sy);
        Y1 = __ldg(p + b1 + sy) + __ldg(p + b1 - sy);
    }
    for (int k = k0; k <= k1; ++k) {
        const int64_t b = col + (int64_t)k * sz;
        const int64_t b2 = b + sz;
        c2 = __ldg(p + b2);
        X2 = __ldg(p + b2 + 1) + __ldg(p + b2 - 1);
        Y2 = __ldg(p + b2 + sy) + __ldg(p + b2 - sy);
        // z-averaged transverse neighbours (Eq. NSFDtrick): ax (w (N^{k-1} + N^{k+1}) + w0 N^k)
        // over the two x neighbours, likewise along y
        const real v = a.a1 * c1 - __ldg(pm + b) + a.axw * (X0 + X2) + a.axw0 * X1 + a.ayw * (Y0 + Y2) +
                       a.ayw0 * Y1 + a.a6 * (c0 + c2) + s * __ldg(S + b);
        o[b] = v;
        c0 = c1, c1 = c2;
        X0 = X1, X1 = X2;
        Y0 = Y1, Y1 = Y2;
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
    int face0;           // first face handled (2: the TMA stencil wrote the x faces)
    int kmin, kmax;      // z range of the x faces (1 .. ez-2 unless restricted)
    // face coefficients per normal axis, in the storage type: first order beta_0 (= beta_4),
    // beta_1 (= beta_3); second order gamma_0, gamma_1 and the tangential gammas of the axes
    // (a+1)%3 and (a+2)%3
    real f0[3], f1[3], ft[3][2];
};

__device__ inline int64_t lin(int i, int j, int k, int64_t sy, int64_t sz) { return (int64_t)k * sz + (int64_t)j * sy + i; }

// Mur value of level n+1 at the face node p of face (ax, side sd) of component comp, from the
// interior value beside it (already updated) and levels n, n-1.
template <int AX, typename real>
__device__ __forceinline__ real mur_face_value_ax(const MurArgs<real>& a, int comp, int sd, const int p[3], int64_t sy,
                                                  int64_t sz)
{
    constexpr int TA = (AX + 1) % 3, TB = (AX + 2) % 3;
    const int64_t sn = AX == 0 ? 1 : (AX == 1 ? sy : sz);   // strides along the normal and the two
    const int64_t sa = TA == 0 ? 1 : (TA == 1 ? sy : sz);   // tangential axes
    const int64_t sb = TB == 0 ? 1 : (TB == 1 ? sy : sz);
    const int64_t ib = lin(p[0], p[1], p[2], sy, sz);
    const int64_t iq = ib + (sd ? -sn : sn);   // inward neighbour
    const real* __restrict__ n1 = a.n1[comp];
    const real* __restrict__ n0 = a.n0[comp];
    const real* __restrict__ nm = a.nm[comp];
    real ta = (real)0, tb = (real)0;
    if (a.order != 1) {
        // tangential neighbours at level n on the face and on the inner plane
        ta = n0[ib + sa] + n0[ib - sa] + n0[iq + sa] + n0[iq - sa];
        tb = n0[ib + sb] + n0[ib - sb] + n0[iq + sb] + n0[iq - sb];
    }
    // first order: the tangential gammas are zero
    return a.f0[AX] * (nm[ib] + n1[iq]) + a.f1[AX] * (n0[ib] + n0[iq]) - nm[iq] + a.ft[AX][0] * ta + a.ft[AX][1] * tb;
}

// The same with the normal axis ax known at run time (edges, corners, the faces beside the TF/SF
// planes): one copy of the code, the strides taken from a small table.
template <typename real>
__device__ __forceinline__ real mur_face_value(const MurArgs<real>& a, int comp, int ax, int sd, const int p[3],
                                               int64_t sy, int64_t sz)
{
    const int64_t st[3] = {1, sy, sz};
    const int64_t ib = lin(p[0], p[1], p[2], sy, sz);
    const int64_t iq = ib + (sd ? -st[ax] : st[ax]);
    const real* __restrict__ n1 = a.n1[comp];
    const real* __restrict__ n0 = a.n0[comp];
    const real* __restrict__ nm = a.nm[comp];
    real ta = (real)0, tb = (real)0;
    if (a.order != 1) {
        const int64_t sa = st[(ax + 1) % 3], sb = st[(ax + 2) % 3];
        ta = n0[ib + sa] + n0[ib - sa] + n0[iq + sa] + n0[iq - sa];
        tb = n0[ib + sb] + n0[ib - sb] + n0[iq + sb] + n0[iq - sb];
    }
    return a.f0[ax] * (nm[ib] + n1[iq]) + a.f1[ax] * (n0[ib] + n0[iq]) - nm[iq] + a.ft[ax][0] * ta + a.ft[ax][1] * tb;
}

// Rows of face (AX, side sd) of component comp: block rp takes the kFaceRows rows v = v0 +
// kFaceRows rp + r of the tangential axis v; each of its threads kFaceRowsPerThread of them at one
// position u (128 threads per row group walking the interior nodes along u: x for the y and z faces,
// coalesced).  A thread evaluates all its nodes before it stores any, so that their loads are in
// flight together.
constexpr int kTailThreads = 256;   // threads of a step-tail block
#ifndef MITHRA_FACE_ROWS_PER_THREAD
#define MITHRA_FACE_ROWS_PER_THREAD 1
#endif
constexpr int kFaceRowThreads = 128, kFaceRowsPerThread = MITHRA_FACE_ROWS_PER_THREAD;
constexpr int kFaceRows = kTailThreads / kFaceRowThreads * kFaceRowsPerThread;
template <int AX, typename real>
__device__ __forceinline__ void mur_face_rows(const MurArgs<real>& a, int comp, int sd, int rp, int64_t sy, int64_t sz)
{
    constexpr int U = AX == 0 ? 1 : 0, V = AX == 2 ? 1 : 2;   // tangential axes, u before v
    const int eu = U == 0 ? a.ex[comp] : a.ey[comp];
    const int ev = V == 1 ? a.ey[comp] : a.ez[comp];
    const int en = AX == 0 ? a.ex[comp] : (AX == 1 ? a.ey[comp] : a.ez[comp]);
    const int v0 = AX == 0 ? a.kmin : 1, v1 = AX == 0 ? min(a.kmax, ev - 2) : ev - 2;
    const int vb = v0 + kFaceRows * rp + (int)(threadIdx.x / kFaceRowThreads) * kFaceRowsPerThread;
    if (vb > v1) return;
#pragma unroll 1
    for (int u = 1 + (int)(threadIdx.x % kFaceRowThreads); u <= eu - 2; u += kFaceRowThreads) {
        real val[kFaceRowsPerThread];
        int64_t id[kFaceRowsPerThread];
#pragma unroll
        for (int r = 0; r < kFaceRowsPerThread; ++r) {
            int p[3];
            p[AX] = sd ? en - 1 : 0;
            p[U] = u;
            p[V] = min(vb + r, v1);   // rows past the face repeat its last row (stored once below)
            id[r] = lin(p[0], p[1], p[2], sy, sz);
            val[r] = mur_face_value_ax<AX>(a, comp, sd, p, sy, sz);
        }
#pragma unroll
        for (int r = 0; r < kFaceRowsPerThread; ++r)
            if (vb + r <= v1) a.n1[comp][id[r]] = val[r];
    }
}

// Face node t of face f (axis = f / 2, side = f % 2) of component comp, if it exists.
template <typename real>
__device__ __forceinline__ void mur_face_node(const MurArgs<real>& a, int comp, int f, int t, int64_t sy, int64_t sz)
{
    const int ax = f >> 1, sd = f & 1;
    const int e[3] = {a.ex[comp], a.ey[comp], a.ez[comp]};
    const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;   // tangential axes, u before v
    const int v0 = ax == 0 ? a.kmin : 1, v1 = ax == 0 ? min(a.kmax, e[v] - 2) : e[v] - 2;
    const int nu = e[u] - 2, nv = v1 - v0 + 1;
    if (nv <= 0 || t >= nu * nv) return;
    int p[3];
    p[ax] = sd ? e[ax] - 1 : 0;
    p[u] = 1 + t % nu;
    p[v] = v0 + t / nu;
    a.n1[comp][lin(p[0], p[1], p[2], sy, sz)] = mur_face_value(a, comp, ax, sd, p, sy, sz);
}

// One face per blockIdx.z (f = face0 + z), one component per blockIdx.y (the x faces next to the
// TF/SF planes after their correction).
template <typename real>
__global__ void k_mur_faces(MurArgs<real> a, int64_t sy, int64_t sz)
{
    dep_begin();
    const int comp = blockIdx.y;
    if (comp >= a.ncomp) return;
    mur_face_node(a, comp, a.face0 + (int)blockIdx.z, (int)(blockIdx.x * blockDim.x + threadIdx.x), sy, sz);
}

// Edges and corners.  Class 0..2: the edges whose free axis is 0..2 (the two other coordinates
// on a boundary); class 3: the corners.  The closed-form coefficients of each class (the FP64
// expression above, divided by sum_a w_a + g) are computed on the host.
template <typename real>
struct MurEdgeCoef {
    real A[4][8];   // n+1 values of the square / cube points (point 0, the unknown, has none)
    real B[4][8];   // n-1 values
    real C[4];      // n values (all points alike)
};

template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
// f(std::integral_constant<int, i>) for i = 0 .. N - 1, i usable as a template argument.
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// The Mur value of an edge point (class C < 3: the edges whose free axis is C) or corner (C = 3)
// p of component comp.  The boundary axes are known at compile time, so the loads of all the
// point's terms can be in flight together.  A neighbour on a face that the same launch writes
// (faces of axes >= face0 / 2; the TMA stencil wrote the x faces when face0 = 2) is evaluated
// here from the face formula, and a corner's edge neighbours from the edge formula, so that no
// point waits for the blocks that write its neighbours (the same code gives the same values).
template <int C, typename real>
__device__ __forceinline__ real mur_point_value(const MurArgs<real>& a, const MurEdgeCoef<real>& cf, int64_t sy,
                                                int64_t sz, int comp, const int p[3])
{
    constexpr int NS = C == 3 ? 3 : 2;                                    // boundary axes
    constexpr int U = (C + 1) % 3, V = (C + 2) % 3;
    constexpr int AX[3] = {C == 3 ? 0 : (U < V ? U : V), C == 3 ? 1 : (U < V ? V : U), 2};
    int sg[3];
#pragma unroll
    for (int s = 0; s < NS; ++s) sg[s] = p[AX[s]] == 0 ? 1 : -1;
    const real* __restrict__ n1 = a.n1[comp];
    const real* __restrict__ n0 = a.n0[comp];
    const real* __restrict__ nm = a.nm[comp];
    real num = (real)0;
    static_for<(1 << NS)>([&](auto eic) {
        constexpr int ei = decltype(eic)::value;
        int q[3] = {p[0], p[1], p[2]};
#pragma unroll
        for (int s = 0; s < NS; ++s)
            if ((ei >> s) & 1) q[AX[s]] += sg[s];
        const int64_t id = lin(q[0], q[1], q[2], sy, sz);
        if constexpr (ei != 0) {
            // the point's boundary axes: those not moved inward
            constexpr int nb = NS - ((ei & 1) + ((ei >> 1) & 1) + ((ei >> 2) & 1));
            constexpr int fa = !(ei & 1) ? AX[0] : (!((ei >> 1) & 1) ? AX[1] : AX[2]);   // nb = 1: that axis
            constexpr int ea = (ei & 1) ? AX[0] : (((ei >> 1) & 1) ? AX[1] : AX[2]);      // nb = 2: the moved axis
            real v;
            if constexpr (nb == 1) {
                if (2 * fa >= a.face0)
                    v = mur_face_value_ax<fa>(a, comp, q[fa] == 0 ? 0 : 1, q, sy, sz);   // a face node
                else
                    v = __ldcg(n1 + id);   // an x-face node of the stencil
            } else if constexpr (nb >= 2) {
                v = mur_point_value<ea>(a, cf, sy, sz, comp, q);   // an edge node (corners)
            } else {
                v = n1[id];                // the interior node
            }
            num += cf.A[C][ei] * v;
        }
        num += cf.B[C][ei] * nm[id] + cf.C[C] * n0[id];
    });
    return num;
}

// Edge point of class C < 3 (`which` bit 0 / 1: the high end of the lower / higher of the two
// boundary axes; pos: its index along C) or corner (C = 3, `which` bit d: the high end of axis d).
template <int C, typename real>
__device__ __forceinline__ void mur_point(const MurArgs<real>& a, const MurEdgeCoef<real>& cf, int64_t sy, int64_t sz,
                                          int comp, int which, int pos)
{
    constexpr int U = (C + 1) % 3, V = (C + 2) % 3;
    constexpr int A0 = U < V ? U : V, A1 = U < V ? V : U;
    const int e[3] = {a.ex[comp], a.ey[comp], a.ez[comp]};
    int p[3];
    if constexpr (C == 3) {
#pragma unroll
        for (int d = 0; d < 3; ++d) p[d] = ((which >> d) & 1) ? e[d] - 1 : 0;
    } else {
        p[C] = pos;
        p[A0] = (which & 1) ? e[A0] - 1 : 0;
        p[A1] = (which & 2) ? e[A1] - 1 : 0;
    }
    a.n1[comp][lin(p[0], p[1], p[2], sy, sz)] = mur_point_value<C>(a, cf, sy, sz, comp, p);
}

// The step tail, one launch of 1-D blocks of kTailThreads: blocks [0, ncomp nbe) the Mur edges and
// then the 8 corners of component b / nbe (their face and edge neighbours evaluated in place);
// then npw blocks of the power step (plane points); then npt blocks of the next step's phase
// tables (node planes); then nbb blocks that reduce the push's block records into the deposit box
// (the whole box and its z chunks' xy boxes); then the Mur faces f >= face0, per normal axis as
// many blocks per side and component as its largest face needs, which go last so that the others
// are scheduled first.  The face blocks leave without arriving; the last of the others to finish
// adds the power partials (compensated, in a fixed order) into the step's series entry once the
// window is complete, and advances the step state: nothing after this launch in the step reads
// it.

constexpr int kBoxRecs = 4 * kTailThreads;   // push records per deposit-box block of the tail
constexpr int kBoxWin = 64;                  // z chunks per block kept in shared memory
template <typename real>
__global__ void __launch_bounds__(kTailThreads) k_step_tail(MurArgs<real> a, MurEdgeCoef<real> cf, int64_t sy,
                                                            int64_t sz, int nfx, int nfy, int nfz,
                                                            int nbe, int npw, int npt, int nbb, Fields6<real> eb,
                                                            Geom g, StepTail tl, unsigned* counter)
{
    dep_begin();
    __shared__ double sh[32];
    const int ne = a.ncomp * nbe;
    const int nrest = ne + npw + npt + nbb;
    if ((int)blockIdx.x >= nrest) {
        // the faces normal to x (nfx blocks per side and component; none when the stencil wrote
        // them), then to y (nfy), then to z (nfz)
        int fi = (int)blockIdx.x - nrest, ax = 0, nf = nfx;
        if (fi >= 2 * a.ncomp * nfx) {
            fi -= 2 * a.ncomp * nfx;
            ax = 1;
            nf = nfy;
            if (fi >= 2 * a.ncomp * nfy) {
                fi -= 2 * a.ncomp * nfy;
                ax = 2;
                nf = nfz;
            }
        }
        const int side = fi / (a.ncomp * nf), r = fi - side * a.ncomp * nf;
        const int comp = r / nf, rp = r - comp * nf;
        if (ax == 0)
            mur_face_rows<0>(a, comp, side, rp, sy, sz);
        else if (ax == 1)
            mur_face_rows<1>(a, comp, side, rp, sy, sz);
        else
            mur_face_rows<2>(a, comp, side, rp, sy, sz);
        return;
    }
    const int b = (int)blockIdx.x;
    if (b < ne) {
        // point t of the 12 edges: free axis f, edge c of its four, position 1 + t along f
        int64_t t = (int64_t)(b % nbe) * blockDim.x + threadIdx.x;
        const int comp = b / nbe;
        const int e[3] = {a.ex[comp], a.ey[comp], a.ez[comp]};
        for (int f = 0; f < 3; ++f) {
            const int64_t len = e[f] - 2;
            if (t < 4 * len) {
                const int c = (int)(t / len), pos = 1 + (int)(t % len);
                if (f == 0)
                    mur_point<0>(a, cf, sy, sz, comp, c, pos);
                else if (f == 1)
                    mur_point<1>(a, cf, sy, sz, comp, c, pos);
                else
                    mur_point<2>(a, cf, sy, sz, comp, c, pos);
                t = -1;
                break;
            }
            t -= 4 * len;
        }
        if (t >= 0 && t < 8) mur_point<3>(a, cf, sy, sz, comp, (int)t, 0);   // the 8 corners after the edges
    } else if (b < ne + npw) {
        const StepDev sd = *tl.sd;
        const int64_t pl = (int64_t)(b - ne) * blockDim.x + threadIdx.x;
        const double c = pl < (int64_t)g.nx * g.ny ? power_point(eb, g, tl.power, sd, pl) : 0.0;
        const double tot = block_sum(c, sh);
        if (threadIdx.x == 0) tl.partial[b - ne] = tot;
    } else if (b < ne + npw + npt) {
        const int iz = (b - ne - npw) * (int)blockDim.x + (int)threadIdx.x;
        if (iz < tl.phase.nz) {
            // the next step's lab offset, from the same function that gives the next state; the
            // first thread also leaves that state for the last block
            const StepDev nx = step_state(tl.sd->next, tl.sc);
            phase_tables_entry(tl.phase, nx.Z0, iz);
            if (iz == 0) tl.sd[1] = nx;
        }
    } else {
        // the deposit box from the push's block records: this block takes kBoxRecs consecutive
        // records (cell order, so they span few z chunks), each thread RPT consecutive ones; the
        // whole box and the xy boxes of the chunks are reduced per warp (the warp's records reach
        // one or two chunks) and gathered with one shared-memory atomic per warp and bound in a
        // window of kBoxWin chunks, then added to the deposit box with a few atomics (a chunk
        // outside the window goes straight out)
        __shared__ int sg[6], swin[kBoxWin][4], scb;
        constexpr int RPT = kBoxRecs / kTailThreads;
        constexpr int kLo = 0x7fffffff, kHi = (int)0x80000000;
        const unsigned full = 0xffffffffu;
        const int lane = (int)threadIdx.x & 31;
        const int nchunk = emit_chunks(g.nz);
        const int64_t base = (int64_t)(b - ne - npw - npt) * kBoxRecs + (int64_t)RPT * threadIdx.x;
        if (threadIdx.x < 6) sg[threadIdx.x] = threadIdx.x < 3 ? kLo : kHi;
        for (int q = threadIdx.x; q < 4 * kBoxWin; q += blockDim.x) swin[q >> 2][q & 3] = (q & 3) < 2 ? kLo : kHi;
        if (threadIdx.x == 0) scb = kLo;
        int v[RPT][6], c0[RPT], c1[RPT];
        int lo[3] = {kLo, kLo, kLo}, hi[3] = {kHi, kHi, kHi}, cmin = kLo, cmax = kHi;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int64_t r = base + i;
#pragma unroll
            for (int q = 0; q < 6; ++q) v[i][q] = r < tl.nrec ? __ldcg(tl.box_rec + 6 * r + q) : (q < 3 ? kLo : kHi);
            // the z chunks of this record's node planes [lo_z - 1, hi_z + 2] (empty record: none)
            c0[i] = v[i][0] != kLo ? max((v[i][2] - 2) / kEmitKZ, 0) : kLo;
            c1[i] = v[i][0] != kLo ? min((v[i][5] + 1) / kEmitKZ, nchunk - 1) : kHi;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                lo[q] = min(lo[q], v[i][q]);
                hi[q] = max(hi[q], v[i][3 + q]);
            }
            cmin = min(cmin, c0[i]);
            cmax = max(cmax, c1[i]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            lo[q] = __reduce_min_sync(full, lo[q]);
            hi[q] = __reduce_max_sync(full, hi[q]);
        }
        const int wc0 = __reduce_min_sync(full, cmin), wc1 = __reduce_max_sync(full, cmax);
        __syncthreads();   // the shared bounds are initialised
        if (lane == 0 && wc0 <= wc1) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                atomicMin(sg + q, lo[q]);
                atomicMax(sg + 3 + q, hi[q]);
            }
            atomicMin(&scb, wc0);
        }
        __syncthreads();
        const int cb = scb;
        for (int c = wc0; c <= wc1; ++c) {   // the same chunks for the whole warp
            int x0 = kLo, y0 = kLo, x1 = kHi, y1 = kHi;
#pragma unroll
            for (int i = 0; i < RPT; ++i)
                if (c0[i] <= c && c <= c1[i]) {
                    x0 = min(x0, v[i][0]);
                    y0 = min(y0, v[i][1]);
                    x1 = max(x1, v[i][3]);
                    y1 = max(y1, v[i][4]);
                }
            x0 = __reduce_min_sync(full, x0);
            y0 = __reduce_min_sync(full, y0);
            x1 = __reduce_max_sync(full, x1);
            y1 = __reduce_max_sync(full, y1);
            if (lane == 0 && x0 != kLo) {
                int* w = c - cb < kBoxWin ? swin[c - cb] : tl.box_out + 6 + 4 * c;
                atomicMin(w, x0);
                atomicMin(w + 1, y0);
                atomicMax(w + 2, x1);
                atomicMax(w + 3, y1);
            }
        }
        __syncthreads();
        if (threadIdx.x < 6 && sg[0] != 0x7fffffff) {
            if (threadIdx.x < 3) atomicMin(tl.box_out + threadIdx.x, sg[threadIdx.x]);
            else atomicMax(tl.box_out + threadIdx.x, sg[threadIdx.x]);
        }
        for (int q = threadIdx.x; q < kBoxWin; q += blockDim.x)
            if (swin[q][0] != 0x7fffffff && cb + q < nchunk) {
                int* w = tl.box_out + 6 + 4 * (cb + q);
                atomicMin(w, swin[q][0]);
                atomicMin(w + 1, swin[q][1]);
                atomicMax(w + 2, swin[q][2]);
                atomicMax(w + 3, swin[q][3]);
            }
    }
    if (last_block(counter, (unsigned)nrest)) {
        const StepDev sd = *tl.sd;
        if (npw > 0 && sd.emit) {
            double s = 0.0, comp = 0.0;
            for (int i = threadIdx.x; i < npw; i += blockDim.x) {
                const double v = __ldcg(tl.partial + i);
                const double t = s + v;
                comp += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
                s = t;
            }
            const double all = block_sum(s + comp, sh);
            if (threadIdx.x == 0) tl.power.series[sd.n] = all * tl.power.scale;
        }
        __syncthreads();   // every thread of this block has read the state
        if (threadIdx.x == 0) {
            if (npt > 0) {
                // formed by the phase-table blocks (their writes are visible: read through L2)
                const unsigned long long* src = reinterpret_cast<const unsigned long long*>(tl.sd + 1);
                unsigned long long* dst = reinterpret_cast<unsigned long long*>(tl.sd);
                static_assert(sizeof(StepDev) % 8 == 0, "whole 8-byte words");
                for (int w = 0; w < (int)(sizeof(StepDev) / 8); ++w) dst[w] = __ldcg(src + w);
            } else {
                *tl.sd = step_state(sd.next, tl.sc);
            }
            *counter = 0;
        }
    }
}

// At a run's creation: block 0 sets the state of step 0, every block fills node planes of the
// phase tables of step 0.
__global__ void k_step_init(StepDev* sd, StepConst sc, PhaseTables pt)
{
    const StepDev s0 = step_state(0, sc);
    const int iz = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (iz < pt.nz) phase_tables_entry(pt, s0.Z0, iz);
    if (blockIdx.x == 0 && threadIdx.x == 0) *sd = s0;
}

cudaError_t launch_step_init(StepDev* sd, const StepConst& sc, const PhaseTables& pt, cudaStream_t st)
{
    const bool tables = pt.t32[0] || pt.t64[0];
    const int nb = tables ? (pt.nz + kTailThreads - 1) / kTailThreads : 1;
    PhaseTables p = pt;
    if (!tables) p.nz = 0;
    k_step_init<<<nb, kTailThreads, 0, st>>>(sd, sc, p);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// E and B at interior nodes from node averages of the staggered potentials (levels n and
// n+1) and phi^n:  E = -(A^{n+1} - A^n)/dt - grad_c phi,  B = (curl_c A^n + curl_c A^{n+1}) / 2,
// in the storage type.  Per step only the nodes the particles will gather from (the box the
// push kernel reduced from the cells it deposited into) and the power plane are needed; inside
// that box the sources of the previous step are cleared in the same pass.  With box == null the
// whole interior is emitted (diagnostics) and nothing is cleared.
//
// One block owns a 32 x 8 tile of node columns and marches a short run of z planes.  Each plane
// of the six potentials and phi is read once, with a one-node halo, into shared memory; the
// sums S_c = 2 (<A_c^n> + <A_c^{n+1}>) of the node averages are formed once per node there (the
// factors 1/2 live in the difference constants);
// the z neighbours (S_x, S_y and phi at k -+ 1) stay in registers, so plane k is finished while
// plane k+1 is being read.  The next plane's loads are issued before the current plane is
// computed, and one barrier per plane orders both the stage ring and the sums: the in-plane
// differences of a plane's sums are taken after the next plane's barrier.
// ---------------------------------------------------------------------------------------
template <typename real>
struct EmitArgs {
    const real* a0[3];   // A^n
    const real* a1[3];   // A^{n+1}
    const real* phi;     // phi^n (node), may be null when space charge is off
    real* eb;            // E, B interleaved (kEBStride values per node)
    real* src[4];        // sources to clear inside the box (entries may be null)
    // E from pair sums of the staggered values (0.5 / dt: the node average's 1/2 folded in), the
    // gradient of phi (0.5 / d), B from sums of two pair sums (0.125 / d: the averages' 1/2 and
    // the 1/2 of B's two time levels folded in; scaling by powers of two is exact)
    real hdt, i2dx, i2dy, i2dz, b2dx, b2dy, b2dz;
    int nchunk;          // blocks along z covering the box; a further z slice emits plane kp
    int kp;              // plane emitted in full (< 0: none)
    const int* box;      // cells [lo_x, lo_y, lo_z, hi_x, hi_y, hi_z] of the last deposit; null: whole grid
    int* box_reset;      // box the next push reduces into: reset to empty here, with the far-move flag
                         // after it (may be null)
    int* err;            // set when a bounded wait on the tensor copies expired (may be null)
};

constexpr int EX = 32, EY = 8, EKZ = kEmitKZ;        // tile and planes per block
constexpr int RL = EX + 2, RH = EY + 2;               // region: columns i0-1 .. i0+32, rows j0-1 .. j0+8
constexpr int RW = kEmitBoxW, RN = RW * RH;           // region rows are stored kEmitBoxW wide
constexpr int EHALO = 2 * RL + 2 * EY;                // region positions outside the tile
constexpr int ENT = EX * EY;                          // threads per block
static_assert(EHALO <= ENT, "emit tile: one halo position per thread at most");
static_assert(RW >= RL && RH == kEmitBoxH, "emit region inside the tensor-map box");

// Shared memory of one block: raw[s] holds A_x^n, A_x^{n+1}, A_y^n, A_y^{n+1}, A_z^n, A_z^{n+1},
// phi of plane p (s = (p - first plane) % ENS) over the region, filled ENS - 1 planes ahead;
// sum[p & 1] the sums S_x, S_y, S_z of plane p.  Each array of raw starts on a
// 128-byte boundary (the tensor copies' destination alignment).
constexpr int ENS = 4;
template <typename real>
struct EmitSmem {
    static constexpr int RS = (RN * (int)sizeof(real) + 127) / 128 * 128 / (int)sizeof(real);
    real raw[ENS][7][RS];
    real sum[2][3][RN];
    uint64_t bar[ENS];
};

// Region position of halo entry h: the rows above and below the tile, then the columns left
// and right of it.
__device__ __forceinline__ int halo_pos(int h)
{
    if (h < RL) return h;
    if (h < 2 * RL) return (RH - 1) * RW + (h - RL);
    if (h < 2 * RL + EY) return (h - 2 * RL + 1) * RW;
    return (h - 2 * RL - EY + 1) * RW + RL - 1;
}

// Asynchronous global -> shared copy of one value; n = 0 writes zero and reads nothing.
template <typename real>
__device__ __forceinline__ void cp_async_val(real* dst, const real* src, bool in)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    if (sizeof(real) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(in ? 4 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(in ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// TM: the region of each plane arrives by seven tensor copies (one per array, issued by one
// thread, completing on the stage's mbarrier); the tile grid then starts on a 16-byte boundary
// of the row, one node left of the box's first interior column rounded down.  Otherwise every
// thread copies its own node and halo position with per-element asynchronous copies.
template <typename real, bool TM>
__global__ void __launch_bounds__(ENT, sizeof(real) == 4 ? 4 : 2)
    k_emit(EmitArgs<real> a, Geom g, const __grid_constant__ EmitMaps em)
{
    dep_begin();
    extern __shared__ unsigned char emit_smem_raw[];
    EmitSmem<real>& sm = *reinterpret_cast<EmitSmem<real>*>(
        emit_smem_raw + ((128 - (mithra::su32(emit_smem_raw) & 127)) & 127));
    const int t = threadIdx.x, tx = t % EX, ty = t / EX;
    if (a.box_reset && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
        for (int q = t; q <= 6 + 4 * a.nchunk; q += ENT)
            a.box_reset[q] = q == 6 + 4 * a.nchunk ? 0
                                                    : ((q < 6 ? q < 3 : (q - 6) % 4 < 2) ? 0x7fffffff : (int)0x80000000);
    // nodes [lo - 1, hi + 2] around the cells of the last deposit: the particles gather at their
    // cells' nodes next step, and with sub-steps they move up to one cell during that step
    int bl[3] = {1, 1, 1}, bh[3] = {g.nx - 2, g.ny - 2, g.nz - 2};
    if (a.box) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            bl[d] = max(__ldg(a.box + d) - 1, 1);
            bh[d] = min(__ldg(a.box + 3 + d) + 2, d == 0 ? g.nx - 2 : (d == 1 ? g.ny - 2 : g.nz - 2));
        }
    }
    // the nodes [lo - 1, hi + 2] of z chunk c's xy box of cells (empty: x0 > x1)
    auto chunk_xy = [&](int c, int& x0, int& x1, int& y0, int& y1) {
        const int* cb = a.box + 6 + 4 * c;
        x0 = max(__ldg(cb) - 1, 1);
        y0 = max(__ldg(cb + 1) - 1, 1);
        x1 = min(__ldg(cb + 2) + 2, g.nx - 2);
        y1 = min(__ldg(cb + 3) + 2, g.ny - 2);
    };
    const bool plane_slice = (int)blockIdx.z == a.nchunk;   // the power plane, whole interior
    int xl = 1, xh = g.nx - 2, yl = 1, yh = g.ny - 2, ka, kb;
    if (plane_slice) {
        ka = kb = a.kp;
    } else {
        xl = bl[0], xh = bh[0], yl = bl[1], yh = bh[1];
        if (a.box) chunk_xy((int)blockIdx.z, xl, xh, yl, yh);   // this chunk's part of the box
        ka = max(1 + (int)blockIdx.z * EKZ, bl[2]);
        kb = min((int)(blockIdx.z + 1) * EKZ, bh[2]);
    }
    // tiles start at the region's corner, so a box that is not aligned to the tile grid costs no
    // extra tiles (the grid has enough blocks for the whole interior); with tensor copies the
    // corner is rounded down to a 16-byte boundary of the row
    constexpr int AL = TM ? 16 / (int)sizeof(real) : 1;
    const int i0 = (xl - 1) / AL * AL + 1 + (int)blockIdx.x * EX, j0 = yl + (int)blockIdx.y * EY;
    if (ka > kb || xl > xh || yl > yh || i0 > xh || j0 > yh) return;
    const int i = i0 + tx, j = j0 + ty;
    const bool emit = i >= xl && i <= xh && j >= yl && j <= yh;
    // with a box, the plane slice leaves the nodes of the chunk's box to the box blocks
    bool skip_xy = false;
    if (plane_slice && a.box && a.kp >= bl[2] && a.kp <= bh[2]) {
        int x0, x1, y0, y1;
        chunk_xy((a.kp - 1) / EKZ, x0, x1, y0, y1);
        skip_xy = i >= x0 && i <= x1 && j >= y0 && j <= y1;
    }
    const bool clear = a.box && !plane_slice;
    const int64_t sy = g.sy, sz = g.sz;

    // region positions of this thread: its node, and a halo position for the first EHALO threads
    const int qo = (ty + 1) * RW + tx + 1;
    const bool has_halo = t < EHALO;
    const int qh = has_halo ? halo_pos(t) : qo;
    // which sums the halo position needs: S_x on the rows above / below the tile, S_y on the
    // columns left / right of it, S_z and phi on both
    const bool hrow = has_halo && t < 2 * RL && (qh % RW) != 0;
    const bool hcol = has_halo && t >= 2 * RL;
    auto offset = [&](int q, bool& in) -> int64_t {
        const int ii = i0 - 1 + q % RW, jj = j0 - 1 + q / RW;
        in = ii <= g.nx - 1 && jj <= g.ny - 1;
        return in ? (int64_t)jj * sy + ii : 0;
    };
    bool in_o, in_h;
    const int64_t off_o = offset(qo, in_o), off_h = offset(qh, in_h);
    const bool use_phi = a.phi != nullptr;
    const int pfirst = ka - 1, plast = kb + 1;
    auto stage = [&](int p) { return (p - pfirst) % ENS; };
    auto parity = [&](int p) { return (uint32_t)(((p - pfirst) / ENS) & 1); };

    // copies of plane p into its stage: TM, by thread 0 (nothing past the last plane);
    // otherwise one commit group per plane and thread (empty past the last plane)
    int last_issued = pfirst - 1;
    auto issue = [&](int p) {
        if constexpr (TM) {
            if (p <= plast) {
                real(*st)[EmitSmem<real>::RS] = sm.raw[stage(p)];
                uint64_t* bar = &sm.bar[stage(p)];
                // the stage held plane p - ENS, which the block read before its last barrier
                if (p >= pfirst + ENS) mithra::fence_proxy_async_smem();
                const int nc = use_phi ? 7 : 6;
                mithra::mbar_expect_tx(bar, (uint32_t)(nc * RN * sizeof(real)));
                for (int c = 0; c < nc; ++c) mithra::tma_load_3d(st[c], &em.m[c], i0 - 1, j0 - 1, p, bar);
                last_issued = p;
            }
        } else {
            if (p <= plast) {
                const real* srcs[7] = {a.a0[0], a.a1[0], a.a0[1], a.a1[1], a.a0[2], a.a1[2], a.phi ? a.phi : a.a0[0]};
                real(*st)[EmitSmem<real>::RS] = sm.raw[stage(p)];
                const int64_t pz = (int64_t)p * sz;
#pragma unroll
                for (int c = 0; c < 7; ++c)
                    cp_async_val(&st[c][qo], srcs[c] + pz + off_o, in_o && (c < 6 || use_phi));
                if (has_halo) {
#pragma unroll
                    for (int c = 0; c < 7; ++c)
                        cp_async_val(&st[c][qh], srcs[c] + pz + off_h, in_h && (c < 6 || use_phi));
                }
            }
            cp_async_commit();
        }
    };
    auto pair = [](real u, real w) { return u + w; };   // twice the node average

    if constexpr (TM) {
        if (t == 0) {
            for (int s = 0; s < ENS; ++s) mithra::mbar_init(&sm.bar[s], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (t == 0)
            for (int d = 0; d < ENS - 1; ++d) issue(pfirst + d);
    } else {
#pragma unroll
        for (int d = 0; d < ENS - 1; ++d) issue(pfirst + d);
    }
    // per-column state: A_z at plane p-1 (own and halo position); S_x, S_y, phi at planes p-2 (0)
    // and p-1 (1); E of plane p-1 before the z derivative of phi
    real az0m = 0, az1m = 0, haz0m = 0, haz1m = 0;
    real sx0 = 0, sx1 = 0, sy0 = 0, sy1 = 0, ph0 = 0, ph1 = 0;
    real ex1 = 0, ey1 = 0, ez1 = 0;
    bool ok = true;
    int p = pfirst;
    for (; p <= plast; ++p) {
        if constexpr (TM) {
            // plane p has landed; everyone is done with plane p-1's stage
            ok = __syncthreads_and(mithra::mbar_wait(&sm.bar[stage(p)], parity(p))) != 0;
            if (!ok) break;
            if (t == 0) issue(p + ENS - 1);
        } else {
            cp_async_wait<ENS - 2>();   // this thread's copies of plane p have landed
            __syncthreads();            // everyone's have; everyone is done with plane p-1's stage
            issue(p + ENS - 1);         // into the stage of plane p-1
        }
        const real(*r)[EmitSmem<real>::RS] = sm.raw[stage(p)];
        const int b = p & 1;
        // the in-plane differences of plane p-1's sums (B_z, and the y / x derivatives of S_z in
        // B_x, B_y): its sums were written before this plane's barrier
        real bz1 = 0, bxp1 = 0, byp1 = 0;
        if (p > pfirst) {
            const real(*S)[RN] = sm.sum[b ^ 1];
            const int q = qo;
            bz1 = (S[1][q + 1] - S[1][q - 1]) * a.b2dx - (S[0][q + RW] - S[0][q - RW]) * a.b2dy;
            bxp1 = (S[2][q + RW] - S[2][q - RW]) * a.b2dy;
            byp1 = (S[2][q + 1] - S[2][q - 1]) * a.b2dx;
        }
        // node averages and sums of plane p at this thread's positions (A_z of the first plane
        // has no previous plane: its S_z and E_z are never read)
        const real az0 = r[4][qo], az1 = r[5][qo], php = use_phi ? r[6][qo] : (real)0;
        const real nx0 = pair(r[0][qo], r[0][qo - 1]), nx1 = pair(r[1][qo], r[1][qo - 1]);
        const real ny0 = pair(r[2][qo], r[2][qo - RW]), ny1 = pair(r[3][qo], r[3][qo - RW]);
        const real nz0 = pair(az0, az0m), nz1 = pair(az1, az1m);
        const real sxp = nx0 + nx1, syp = ny0 + ny1;
        sm.sum[b][0][qo] = sxp;
        sm.sum[b][1][qo] = syp;
        sm.sum[b][2][qo] = nz0 + nz1;
        az0m = az0;
        az1m = az1;
        if (has_halo) {
            if (hrow) sm.sum[b][0][qh] = pair(r[0][qh], r[0][qh - 1]) + pair(r[1][qh], r[1][qh - 1]);
            if (hcol) sm.sum[b][1][qh] = pair(r[2][qh], r[2][qh - RW]) + pair(r[3][qh], r[3][qh - RW]);
            const real h0 = r[4][qh], h1 = r[5][qh];
            sm.sum[b][2][qh] = pair(h0, haz0m) + pair(h1, haz1m);
            haz0m = h0;
            haz1m = h1;
        }
        const int q = qo;
        real ex = (nx0 - nx1) * a.hdt;
        real ey = (ny0 - ny1) * a.hdt;
        const real ez = (nz0 - nz1) * a.hdt;
        if (use_phi) {
            ex -= (r[6][q + 1] - r[6][q - 1]) * a.i2dx;
            ey -= (r[6][q + RW] - r[6][q - RW]) * a.i2dy;
        }
        // plane k = p - 1 has its z neighbours now
        const int k = p - 1;
        if (k >= ka && emit && !(skip_xy && k >= bl[2] && k <= bh[2])) {
            const int64_t id = (int64_t)k * sz + off_o;
            const real bx = bxp1 - (syp - sy0) * a.b2dz;
            const real by = (sxp - sx0) * a.b2dz - byp1;
            real ezk = ez1;
            if (use_phi) ezk -= (php - ph0) * a.i2dz;
            // the node's whole slot (unused entries zero): full 32-byte sectors, no partial writes
            real* o = a.eb + id * kEBStride;
            if constexpr (sizeof(real) == 4) {
                *reinterpret_cast<float4*>(o) = make_float4(ex1, ey1, ezk, bx);
                *reinterpret_cast<float4*>(o + 4) = make_float4(by, bz1, 0.f, 0.f);
            } else {
                *reinterpret_cast<double2*>(o) = make_double2(ex1, ey1);
                *reinterpret_cast<double2*>(o + 2) = make_double2(ezk, bx);
                *reinterpret_cast<double2*>(o + 4) = make_double2(by, bz1);
                *reinterpret_cast<double2*>(o + 6) = make_double2(0.0, 0.0);
            }
            if (clear) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (a.src[c]) a.src[c][id] = (real)0;
            }
        }
        sx0 = sx1, sx1 = sxp;
        sy0 = sy1, sy1 = syp;
        ph0 = ph1, ph1 = php;
        ex1 = ex, ey1 = ey, ez1 = ez;
        // sum[b] is read in the next plane (after its barrier) and written again two planes
        // later, after the barrier of that plane, which every thread reaches only once it is
        // done reading it
    }
    if constexpr (TM) {
        if (!ok && t == 0) {
            // a wait expired: report it and let the copies still in flight land before exiting
            if (a.err) atomicExch(a.err, 1);
            for (int pp = p; pp <= last_issued; ++pp) mithra::mbar_wait(&sm.bar[stage(pp)], parity(pp));
        }
    } else {
        cp_async_wait<0>();
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
    a.axw = (real)(cf.ax * cf.w);
    a.axw0 = (real)(cf.ax * cf.w0);
    a.ayw = (real)(cf.ay * cf.w);
    a.ayw0 = (real)(cf.ay * cf.w0);
    a.ncomp = ncomp;
    a.kchunk = 32;
    const dim3 blk(32, 8);
    const int nchunk = (g.nz - 2 + a.kchunk - 1) / a.kchunk;
    const dim3 grd((g.nx - 2 + 31) / 32, (g.ny - 2 + 7) / 8, nchunk * ncomp);
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepStencil), k_stencil<real>, dim3(grd), dim3(blk), 0, st, a,
                                          g.sy, g.sz);
        if (le != cudaSuccess) return le;
    }
    count_launches(1);
    return cudaGetLastError();
}

MurFaceCoef mur_face_coef(const Geom& g, int order)
{
    MurFaceCoef m;
    const double cdt = kC * g.dt, D3[3] = {g.dx, g.dy, g.dz};
    for (int ax = 0; ax < 3; ++ax) {
        const double D = D3[ax], den = 1.0 / (cdt + D);
        if (order == 1) {
            m.f0[ax] = (cdt - D) * den;            // beta_0 = beta_4
            m.f1[ax] = 2.0 * D * den;              // beta_1 = beta_3
            m.ft[ax][0] = m.ft[ax][1] = 0.0;
        } else {
            const int ta = (ax + 1) % 3, tb = (ax + 2) % 3;
            const double ra = (cdt / D3[ta]) * (cdt / D3[ta]), rb = (cdt / D3[tb]) * (cdt / D3[tb]);
            m.f0[ax] = (cdt - D) * den;            // gamma_0 = gamma_4
            m.f1[ax] = D * (2.0 - ra - rb) * den;  // gamma_1 = gamma_3
            m.ft[ax][0] = 0.5 * ra * D * den;      // gamma of the (ax+1) neighbours
            m.ft[ax][1] = 0.5 * rb * D * den;      // gamma of the (ax+2) neighbours
        }
    }
    return m;
}

// Edge (class f: free axis f) and corner (class 3) coefficients of the closed form, in FP64,
// divided by its denominator and rounded once to the storage type.
template <typename real>
static MurEdgeCoef<real> mur_edge_coef(const Geom& g)
{
    MurEdgeCoef<real> c{};
    const double D3[3] = {g.dx, g.dy, g.dz};
    for (int cls = 0; cls < 4; ++cls) {
        int axes[3], ns = 0;
        if (cls == 3) {
            axes[0] = 0;
            axes[1] = 1;
            axes[2] = 2;
            ns = 3;
        } else {
            const int u = (cls + 1) % 3, v = (cls + 2) % 3;
            axes[0] = u < v ? u : v;
            axes[1] = u < v ? v : u;
            ns = 2;
        }
        const int npts = 1 << ns;
        const double h = (double)(npts >> 1);
        double wa[3], wsum = 0.0;
        for (int s = 0; s < ns; ++s) {
            wa[s] = 1.0 / (2.0 * g.dt * D3[axes[s]] * h);
            wsum += wa[s];
        }
        const double gg = (double)ns / (kC * g.dt * g.dt * (double)npts);
        const double inv = 1.0 / (wsum + gg);
        for (int ei = 0; ei < npts; ++ei) {
            double W = 0.0;
            for (int s = 0; s < ns; ++s) W += ((ei >> s) & 1) ? wa[s] : -wa[s];
            c.A[cls][ei] = (real)(ei != 0 ? (W - gg) * inv : 0.0);
            c.B[cls][ei] = (real)(-(W + gg) * inv);
        }
        c.C[cls] = (real)(2.0 * gg * inv);
    }
    return c;
}

template <typename real>
cudaError_t launch_mur(const FieldLevels<real>& L, const Geom& g, int order, int ncomp, bool x_faces_done,
                       unsigned* counter, const StepTail& tail, cudaStream_t st)
{
    MurArgs<real> a;
    a.face0 = x_faces_done ? 2 : 0;
    a.kmin = 1;
    a.kmax = g.nz;
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
    const MurFaceCoef m = mur_face_coef(g, order);
    for (int ax = 0; ax < 3; ++ax) {
        a.f0[ax] = (real)m.f0[ax];
        a.f1[ax] = (real)m.f1[ax];
        a.ft[ax][0] = (real)m.ft[ax][0];
        a.ft[ax][1] = (real)m.ft[ax][1];
    }
    // face blocks per side and component along each normal axis: kFaceRows rows of the axis's
    // longest tangential v range each (mur_face_rows)
    static_assert(kTailThreads % kFaceRowThreads == 0, "whole row groups per tail block");
    int nf[3] = {0, 0, 0};
    for (int ax = a.face0 / 2; ax < 3; ++ax) {
        int rows = 0;
        for (int c = 0; c < ncomp; ++c) {
            const int e[3] = {a.ex[c], a.ey[c], a.ez[c]};
            const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;
            if (e[u] - 2 > 0) rows = std::max(rows, e[v] - 2);
        }
        nf[ax] = (rows + kFaceRows - 1) / kFaceRows;
    }
    const MurEdgeCoef<real> ec = mur_edge_coef<real>(g);
    // edge points of the widest component, then its 8 corners
    const int64_t edges = 4 * ((int64_t)(g.nx - 2) + (g.ny - 2) + (g.nz - 2)) + 8;
    const int nbe = (int)((edges + kTailThreads - 1) / kTailThreads);
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int npw = (int)((plane + kTailThreads - 1) / kTailThreads);
    if (npw > tail.npartial) return cudaErrorInvalidValue;
    const bool tables = tail.phase.t32[0] || tail.phase.t64[0];
    const int npt = tables ? (tail.phase.nz + kTailThreads - 1) / kTailThreads : 0;
    Fields6<real> E6;
    E6.p = (real*)tail.eb;
    {
        const int nface = 2 * ncomp * (nf[0] + nf[1] + nf[2]);
        // deposit-box blocks: kBoxRecs push records each
        const int nbb = (int)((tail.nrec + kBoxRecs - 1) / kBoxRecs);
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepTail), k_step_tail<real>,
                                          dim3((unsigned)(nface + ncomp * nbe + npw + npt + nbb)), dim3(kTailThreads), 0,
                                          st, a, ec, g.sy, g.sz, nf[0], nf[1], nf[2], nbe, npw, npt, nbb, E6, g,
                                          tail, counter);
        if (le != cudaSuccess) return le;
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_mur_tfsf_xfaces(const FieldLevels<real>& L, const Geom& g, int order, cudaStream_t st)
{
    MurArgs<real> a;
    a.face0 = 0;
    a.kmin = 1;
    a.kmax = 2;
    for (int c = 0; c < 4; ++c) {
        a.n1[c] = L.out[c];
        a.n0[c] = L.n1[c];
        a.nm[c] = L.n0[c];
        a.ex[c] = g.nx - (c == 0);
        a.ey[c] = g.ny - (c == 1);
        a.ez[c] = g.nz - (c == 2);
    }
    a.ncomp = 2;   // A_x, A_y
    a.order = order;
    const MurFaceCoef m = mur_face_coef(g, order);
    for (int ax = 0; ax < 3; ++ax) {
        a.f0[ax] = (real)m.f0[ax];
        a.f1[ax] = (real)m.f1[ax];
        a.ft[ax][0] = (real)m.ft[ax][0];
        a.ft[ax][1] = (real)m.ft[ax][1];
    }
    const int64_t pts = 2 * (int64_t)g.ny;
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepOther), k_mur_faces<real>,
                                          dim3((unsigned)((pts + 127) / 128), 2, 2), dim3(128), 0, st, a, g.sy, g.sz);
        if (le != cudaSuccess) return le;
    }
    count_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_mur_tfsf_xfaces<float>(const FieldLevels<float>&, const Geom&, int, cudaStream_t);
template cudaError_t launch_mur_tfsf_xfaces<double>(const FieldLevels<double>&, const Geom&, int, cudaStream_t);

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
    a.eb = eb.p;
    for (int c = 0; c < 4; ++c) a.src[c] = (bx.box && bx.clear) ? (real*)L.src[c] : nullptr;
    if (!g.space_charge) a.src[3] = nullptr;
    a.hdt = (real)(1.0 / g.dt) * (real)0.5;
    a.i2dx = (real)(0.5 / g.dx);
    a.i2dy = (real)(0.5 / g.dy);
    a.i2dz = (real)(0.5 / g.dz);
    a.b2dx = a.i2dx * (real)0.25;
    a.b2dy = a.i2dy * (real)0.25;
    a.b2dz = a.i2dz * (real)0.25;
    a.kp = bx.kp;
    a.box = bx.box;
    a.box_reset = bx.box_reset;
    a.err = bx.err;
    a.nchunk = (g.nz - 2 + EKZ - 1) / EKZ;
    constexpr int smem = (int)sizeof(EmitSmem<real>) + 128;
    if (bx.maps) {
        // tiles start up to 16 / sizeof(real) - 1 columns left of the region's first column
        const dim3 grd((g.nx - 2 + 16 / (int)sizeof(real) - 1 + EX - 1) / EX, (g.ny - 2 + EY - 1) / EY,
                       a.nchunk + (a.kp >= 1 ? 1 : 0));
        static const cudaError_t attr =
            cudaFuncSetAttribute(k_emit<real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (attr != cudaSuccess) return attr;
        {
            const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepEmit), (k_emit<real, true>), dim3(grd), dim3(ENT),
                                              smem, st, a, g, *bx.maps);
            if (le != cudaSuccess) return le;
        }
    } else {
        const dim3 grd((g.nx - 2 + EX - 1) / EX, (g.ny - 2 + EY - 1) / EY, a.nchunk + (a.kp >= 1 ? 1 : 0));
        static const cudaError_t attr =
            cudaFuncSetAttribute(k_emit<real, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (attr != cudaSuccess) return attr;
        EmitMaps none;
        memset(&none, 0, sizeof none);
        {
            const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepEmit), (k_emit<real, false>), dim3(grd), dim3(ENT),
                                              smem, st, a, g, none);
            if (le != cudaSuccess) return le;
        }
    }
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Seed through TF/SF planes.
// ---------------------------------------------------------------------------------------
// The seed potential of component c (0: A_x at (i + 1/2) dx, 1: A_y at (j + 1/2) dy) at nodes
// (i, j) of z planes 1 and 2: fbuf[((c * 2 + plane - 1) * ny + j) * nx + i].
__global__ void k_seed_eval(SeedField s, Geom g, const StepDev* sd, double T0, double* __restrict__ fbuf)
{
    dep_begin();
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 2 * plane) return;
    const int k = 1 + (int)(q / plane);
    const int64_t pl = q % plane;
    const int i = (int)(pl % g.nx), j = (int)(pl / g.nx);
    const double t = T0 + ((double)sd->n + 1.0) * g.dt;
    const double z = g.z0 + k * g.dz;
    double ax, ay, bx, by;
    seed_potential(s, g.x0 + (i + 0.5) * g.dx, g.y0 + j * g.dy, z, t, &ax, &ay);
    seed_potential(s, g.x0 + i * g.dx, g.y0 + (j + 0.5) * g.dy, z, t, &bx, &by);
    fbuf[(int64_t)(k - 1) * plane + pl] = ax;            // component 0
    fbuf[(int64_t)(2 + k - 1) * plane + pl] = by;        // component 1
}

template <typename real>
struct TfsfArgs {
    real* out[2];
    int ex[2], ey[2];
    double A, a2, a4, a6;   // NSFD coefficient, (c dt/dx)^2, (c dt/dy)^2, alpha'_6 = alpha'_7
};

template <typename real>
__global__ void k_tfsf(TfsfArgs<real> a, Geom g, const double* __restrict__ fbuf)
{
    dep_begin();
    const int c = blockIdx.y;
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(q % g.nx), j = (int)(q / g.nx);
    if (q >= plane || i < 1 || i > a.ex[c] - 2 || j < 1 || j > a.ey[c] - 2) return;
    const double* f1 = fbuf + (int64_t)(2 * c) * plane;
    const double* f2 = f1 + plane;
    auto F = [&](const double* f, int ii, int jj) { return f[(int64_t)jj * g.nx + ii]; };
    const double sf = a.A * (a.a2 * (F(f2, i + 1, j) + F(f2, i - 1, j)) + a.a4 * (F(f2, i, j + 1) + F(f2, i, j - 1))) +
                      a.a6 * F(f2, i, j);
    const double tf = a.A * (a.a2 * (F(f1, i + 1, j) + F(f1, i - 1, j)) + a.a4 * (F(f1, i, j + 1) + F(f1, i, j - 1))) +
                      a.a6 * F(f1, i, j);
    real* o = a.out[c];
    o[1 * g.sz + (int64_t)j * g.sy + i] -= (real)sf;
    o[2 * g.sz + (int64_t)j * g.sy + i] += (real)tf;
}

template <typename real>
cudaError_t launch_tfsf(real* const out[2], const Geom& g, const StencilCoef& cf, const SeedField& s,
                        const StepDev* sd, double T0, double* fbuf, cudaStream_t st)
{
    const int64_t plane = (int64_t)g.nx * g.ny;
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepOther), k_seed_eval,
                                          dim3((unsigned)((2 * plane + 127) / 128)), dim3(128), 0, st, s, g, sd, T0,
                                          fbuf);
        if (le != cudaSuccess) return le;
    }
    TfsfArgs<real> a;
    for (int c = 0; c < 2; ++c) {
        a.out[c] = out[c];
        a.ex[c] = g.nx - (c == 0);
        a.ey[c] = g.ny - (c == 1);
    }
    a.A = cf.w;
    a.a2 = cf.ax;
    a.a4 = cf.ay;
    a.a6 = cf.a6;
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepOther), k_tfsf<real>,
                                          dim3((unsigned)((plane + 127) / 128), 2), dim3(128), 0, st, a, g, fbuf);
        if (le != cudaSuccess) return le;
    }
    count_launches(2);
    return cudaGetLastError();
}

template cudaError_t launch_tfsf<float>(float* const[2], const Geom&, const StencilCoef&, const SeedField&,
                                        const StepDev*, double, double*, cudaStream_t);
template cudaError_t launch_tfsf<double>(double* const[2], const Geom&, const StencilCoef&, const SeedField&,
                                         const StepDev*, double, double*, cudaStream_t);

template cudaError_t launch_stencil<float>(const FieldLevels<float>&, const Geom&, const StencilCoef&, int, cudaStream_t);
template cudaError_t launch_stencil<double>(const FieldLevels<double>&, const Geom&, const StencilCoef&, int, cudaStream_t);
template cudaError_t launch_mur<float>(const FieldLevels<float>&, const Geom&, int, int, bool, unsigned*,
                                      const StepTail&, cudaStream_t);
template cudaError_t launch_mur<double>(const FieldLevels<double>&, const Geom&, int, int, bool, unsigned*,
                                       const StepTail&, cudaStream_t);
template cudaError_t launch_emit<float>(const FieldLevels<float>&, const Fields6<float>&, const Geom&, const EmitBox&,
                                        cudaStream_t);
template cudaError_t launch_emit<double>(const FieldLevels<double>&, const Fields6<double>&, const Geom&,
                                         const EmitBox&, cudaStream_t);

}  // namespace mithra
