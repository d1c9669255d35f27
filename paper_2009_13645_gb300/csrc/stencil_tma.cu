// Potential update (manual Eq. updateEquation; FD is the same equation with A = 0) with the
// tiles staged by the Tensor Memory Accelerator.
//
// One CTA owns a tile of TX x TY columns of one component lattice and marches a chunk of z planes.
// For every plane p it loads, with three cp.async.bulk.tensor copies completing on one mbarrier,
//   psi^n   (TX + 2 HX) x (TY + 2)  (the tile plus the x/y halo; the x origin is moved down to a
//                                     16-byte boundary, so HX = 16 bytes of elements),
//   psi^{n-1}, source  TX x TY,
// into a ring of NST shared-memory stages, NST - 1 planes ahead of the plane being computed.  The
// source is copied only for the block's own planes and only where the tile meets the nodes the
// step's push can have deposited into (the previous deposit box grown by a cell per sub-step);
// elsewhere it is zero, so early in a run, with a compact bunch, most tiles skip its bytes.
// Each thread owns the x-adjacent columns one 16-byte load fetches (four in FP32, two in FP64) and
// keeps planes k-1, k, k+1 of them and of their neighbours (the columns either side, and the rows
// above and below) in registers, reading only the new plane k+1 from shared memory with 16-byte
// loads; the results leave in one vector store (coalesced rows).  Several cells per thread share
// the per-cell cost of the loop, the barrier and the addressing (the stencil is issue bound: the
// FEL step's stencil took 137 us with one cell per thread, 102 with two, 89 with four in FP32).
//
// In FP32 the threads next to an x boundary also write the Mur value of the face node beside them
// (Sec. "First/Second Order ABCs"): every input of the face formula is already in their registers
// or in the staged tiles, whereas a separate face kernel reads one 32-byte sector per row for two
// useful values.  In FP64 that lane's arithmetic would occupy the FP64 pipe for a whole warp
// instruction (GB300's FP64 rate is low and the FP64 stencil is bound by it), so there the faces
// stay in their own kernel.  Every wait on an mbarrier has an iteration limit;
// on expiry the CTA records an error word, waits (again bounded) for its copies in flight, and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace mithra {

namespace {

#ifndef MITHRA_STENCIL_KZ
#define MITHRA_STENCIL_KZ 32
#endif
constexpr int TX = 64, TY = 8, NST = 4, KZ = MITHRA_STENCIL_KZ;   // tile, stages, planes per block

template <typename real>
struct Tile {
    static constexpr int HX = 16 / (int)sizeof(real);
    static constexpr int W = TX + 2 * HX;          // halo tile width
    static constexpr int H = TY + 2;               // halo tile height
    static constexpr int HALO_BYTES = W * H * (int)sizeof(real);
    static constexpr int BODY_BYTES = TX * TY * (int)sizeof(real);
    static constexpr int pad(int b) { return (b + 127) & ~127; }
    static constexpr int OFF_PREV = pad(HALO_BYTES);
    static constexpr int OFF_SRC = OFF_PREV + pad(BODY_BYTES);
    static constexpr int STAGE = OFF_SRC + pad(BODY_BYTES);
    static constexpr int TX_BYTES = HALO_BYTES + 2 * BODY_BYTES;   // bytes one stage receives
    static constexpr int SMEM = NST * STAGE + 128;                 // + mbarriers
};

}  // namespace

struct TmaMaps {
    CUtensorMap halo[3][4];   // psi with halo box, per ring level and component
    CUtensorMap body[3][4];   // psi without halo (used as psi^{n-1})
    CUtensorMap src[4];
    CUtensorMap emit[3][4];   // E/B emission region box (kEmitBoxW x kEmitBoxH), per level and component
};

// The maps one stencil launch reads: psi^n with halo, psi^{n-1} and the source of each component
// (1.5 KB of kernel parameters; the whole ring's maps would pass 4 KB).
struct StencilMaps {
    CUtensorMap halo[4];
    CUtensorMap body[4];
    CUtensorMap src[4];
};

template <typename real>
struct TmaArgs {
    real* out[4];
    const real* prev[4];       // psi^{n-1} arrays (read where a staged tile does not reach)
    int mur;                   // Mur order of the x faces written here (0: none)
    real mf0, mf1, mfy, mfz;   // their coefficients: f0, f1 and the tangential gammas along y, z
    int lev_n, lev_m;          // ring levels of psi^n and psi^{n-1}
    int ex[4], ey[4], ez[4];
    int ncomp;
    real a1, ax, ay, a6, w, w0, s[4];
    real axw, axw0, ayw, ayw0;   // ax w, ax w0, ay w, ay w0 (products taken in FP64)
    // the previous step's deposit box, this step's far-move flag and the box's growth in nodes
    // (sbox null: every source is read)
    const int* sbox;
    const int* sfar;
    int sgrow;
    int* err;
    // failure test: the plane pfirst + skip_plane of every block is never copied (-1: none), and
    // every wait gives up after `spin` polls
    int skip_plane;
    uint32_t spin;
};

// Cells per thread: the x-adjacent columns one 16-byte shared-memory load fetches (four in FP32,
// two in FP64), loaded and stored as one vector.
template <typename real>
constexpr int cells_per_thread()
{
    return 16 / (int)sizeof(real);
}

template <typename real, int N>
__device__ __forceinline__ void ld16(const real* p, real (&v)[N])
{
    static_assert(N * sizeof(real) == 16, "16-byte vector");
    if constexpr (sizeof(real) == 4) {
        const float4 t = *(const float4*)p;
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
        const double2 t = *(const double2*)p;
        v[0] = t.x;
        v[1] = t.y;
    }
}

template <typename real, int N>
__device__ __forceinline__ void st16(real* p, const real (&v)[N])
{
    if constexpr (sizeof(real) == 4) {
        *(float4*)p = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        *(double2*)p = make_double2(v[0], v[1]);
    }
}

template <typename real>
__global__ void __launch_bounds__(TX / cells_per_thread<real>() * TY)
    k_stencil_tma(const __grid_constant__ StencilMaps maps, TmaArgs<real> a, int64_t sy, int64_t sz)
{
    constexpr int CT = cells_per_thread<real>();
    dep_begin();
    using T = Tile<real>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = (uint64_t*)(smem + NST * T::STAGE);
    const int comp = blockIdx.z % a.ncomp;
    const int chunk = blockIdx.z / a.ncomp;
    const int ex = a.ex[comp], ey = a.ey[comp], ez = a.ez[comp];
    const int k0 = 1 + chunk * KZ;
    if (k0 > ez - 2) return;
    const int k1 = min(ez - 2, k0 + KZ - 1);
    const int xt = blockIdx.x * TX, yt = blockIdx.y * TY;
    const int tp = threadIdx.x % (TX / CT), ty = threadIdx.x / (TX / CT);
    const int cx = CT * tp;                // tile column of the thread's first cell
    const int x = xt + cx, y = yt + ty;
    const bool yin = y >= 1 && y <= ey - 2;
    bool mine[CT], all = true, any = false;   // the thread's interior cells
#pragma unroll
    for (int i = 0; i < CT; ++i) {
        mine[i] = yin && x + i >= 1 && x + i <= ex - 2;
        all = all && mine[i];
        any = any || mine[i];
    }
    const CUtensorMap* mh = &maps.halo[comp];
    const CUtensorMap* mb = &maps.body[comp];
    const CUtensorMap* ms = &maps.src[comp];
    const int pfirst = k0 - 1, plast = k1 + 1;
    // planes [zs0, zs1] whose source this block copies: the source enters the update of the
    // block's own planes only, and only where this step's push can have deposited (empty:
    // zs0 > zs1).  The box ints were written by earlier kernels of the stream and the flag by
    // the push just before: read through L2.
    int zs0 = k0, zs1 = k1;
    if (a.sbox && __ldcg(a.sfar) == 0) {
        const int d = a.sgrow;
        const int lx = __ldcg(a.sbox) - d, ly = __ldcg(a.sbox + 1) - d, lz = __ldcg(a.sbox + 2) - d;
        const int hx = __ldcg(a.sbox + 3) + 1 + d, hy = __ldcg(a.sbox + 4) + 1 + d, hz = __ldcg(a.sbox + 5) + 1 + d;
        if (lx <= xt + TX - 1 && hx >= xt && ly <= yt + TY - 1 && hy >= yt) {
            zs0 = max(zs0, lz);
            zs1 = min(zs1, hz);
        } else {
            zs1 = zs0 - 1;
        }
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(bars + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int p) {
        const int s = (p - pfirst) % NST;
        if (p - pfirst == a.skip_plane) return;   // failure test: this plane's copy never comes
        unsigned char* st = smem + s * T::STAGE;
        // the stage held plane p - NST, which the block read before its last barrier
        if (p >= pfirst + NST) fence_proxy_async_smem();
        const bool sp = p >= zs0 && p <= zs1;
        mbar_expect_tx(bars + s, (uint32_t)(sp ? T::TX_BYTES : T::TX_BYTES - T::BODY_BYTES));
        tma_load_3d(st, mh, xt - T::HX, yt - 1, p, bars + s);
        tma_load_3d(st + T::OFF_PREV, mb, xt, yt, p, bars + s);
        if (sp) tma_load_3d(st + T::OFF_SRC, ms, xt, yt, p, bars + s);
    };
    int last_issued = pfirst - 1;
    if (threadIdx.x == 0)
        for (int p = pfirst; p <= plast && p < pfirst + NST; ++p) {
            issue(p);
            last_issued = p;
        }
    bool ok = true;
    auto wait_plane = [&](int p) {
        const int s = (p - pfirst) % NST;
        const uint32_t parity = (uint32_t)(((p - pfirst) / NST) & 1);
        if (!mbar_wait(bars + s, parity, a.spin)) ok = false;
    };
    // row dy of plane p's halo tile, at the thread's first cell
    auto hrow = [&](int p, int dy) -> const real* {
        return (const real*)(smem + ((p - pfirst) % NST) * T::STAGE) + (ty + 1 + dy) * T::W + cx + T::HX;
    };
    // registers of one plane: the thread's cells c, and the sums of each cell's two x neighbours
    // (X) and of its two y neighbours (Y), formed once per plane and used in three updates; the
    // cell after the last (xq) for the Mur x face.  Planes k-1, k and k+1 are live; the loop below
    // is unrolled three times so that moving on a plane renames them instead of copying.
    struct Plane {
        real c[CT], X[CT], Y[CT], xq;
    };
    Plane P0, P1, P2;
    auto load = [&](int p, Plane& P) {
        const real* r = hrow(p, 0);
        ld16(r, P.c);
        const real xm = r[-1];
        P.xq = r[CT];
        real m[CT], q[CT];
        ld16(hrow(p, -1), m);
        ld16(hrow(p, 1), q);
#pragma unroll
        for (int i = 0; i < CT; ++i) {
            P.X[i] = (i == CT - 1 ? P.xq : P.c[i + 1]) + (i == 0 ? xm : P.c[i - 1]);
            P.Y[i] = q[i] + m[i];
        }
    };
    wait_plane(pfirst);
    wait_plane(pfirst + 1);
    load(pfirst, P0);
    load(pfirst + 1, P1);
    ok = __syncthreads_and(ok) != 0;
    if (ok && threadIdx.x == 0 && pfirst + NST <= plast) {
        issue(pfirst + NST);
        last_issued = pfirst + NST;
    }
    real* __restrict__ o = a.out[comp];
    const real s = a.s[comp];
    // plane k from planes k-1 (L), k (C) and k+1 (N, loaded here)
    auto step = [&](int k, const Plane& L, const Plane& C, Plane& N) {
        wait_plane(k + 1);
        load(k + 1, N);
        const unsigned char* stk = smem + ((k - pfirst) % NST) * T::STAGE;
        real pm[CT], sr[CT];
        ld16((const real*)(stk + T::OFF_PREV) + ty * TX + cx, pm);
        if (k >= zs0 && k <= zs1) {
            ld16((const real*)(stk + T::OFF_SRC) + ty * TX + cx, sr);
        } else {
#pragma unroll
            for (int i = 0; i < CT; ++i) sr[i] = (real)0;
        }
        if (any && ok) {
            // ax (w (N^{k-1} + N^{k+1}) + w0 N^k) over the two x neighbours, likewise along y
            real v[CT];
#pragma unroll
            for (int i = 0; i < CT; ++i)
                v[i] = a.a1 * C.c[i] - pm[i] + a.axw * (L.X[i] + N.X[i]) + a.axw0 * C.X[i] + a.ayw * (L.Y[i] + N.Y[i]) +
                       a.ayw0 * C.Y[i] + a.a6 * (L.c[i] + N.c[i]) + s * sr[i];
            const int64_t row = (int64_t)k * sz + (int64_t)y * sy;
            if (all) {
                st16(o + row + x, v);
            } else {
#pragma unroll
                for (int i = 0; i < CT; ++i)
                    if (mine[i]) o[row + x + i] = v[i];
            }
            if (tma_x_faces<real>() && a.mur) {
                // Mur x faces (the formula and the summation order of k_mur_faces): face node b,
                // its interior neighbour q
                const bool o2 = a.mur != 1;
                if (x == 0 && mine[1])   // b = x (the thread's first cell), q = x + 1
                    o[row] = a.mf0 * (pm[0] + v[1]) + a.mf1 * (C.c[0] + C.c[1]) - pm[1] +
                             a.mfy * (o2 ? C.Y[0] + C.Y[1] : (real)0) +
                             a.mfz * (o2 ? N.c[0] + L.c[0] + N.c[1] + L.c[1] : (real)0);
#pragma unroll
                for (int i = 0; i + 1 < CT; ++i)
                    if (mine[i] && x + i == ex - 2)   // q = x + i, b = x + i + 1 (a cell of this thread)
                        o[row + x + i + 1] = a.mf0 * (pm[i + 1] + v[i]) + a.mf1 * (C.c[i + 1] + C.c[i]) - pm[i] +
                                             a.mfy * (o2 ? C.Y[i + 1] + C.Y[i] : (real)0) +
                                             a.mfz * (o2 ? N.c[i + 1] + L.c[i + 1] + N.c[i] + L.c[i] : (real)0);
                if (mine[CT - 1] && x + CT - 1 == ex - 2) {   // q = the last cell, b = the next thread's first
                    const real nmb = cx + CT < TX ? ((const real*)(stk + T::OFF_PREV))[ty * TX + cx + CT]
                                                  : a.prev[comp][row + x + CT];
                    o[row + x + CT] = a.mf0 * (nmb + v[CT - 1]) + a.mf1 * (C.xq + C.c[CT - 1]) - pm[CT - 1] +
                                      a.mfy * (o2 ? hrow(k, 1)[CT] + hrow(k, -1)[CT] + C.Y[CT - 1] : (real)0) +
                                      a.mfz * (o2 ? N.xq + L.xq + N.c[CT - 1] + L.c[CT - 1] : (real)0);
                }
            }
        }
        ok = __syncthreads_and(ok) != 0;
        if (ok && threadIdx.x == 0 && k + NST <= plast) {
            issue(k + NST);
            last_issued = k + NST;
        }
    };
    int k = k0;
    while (k <= k1 && ok) {
        step(k++, P0, P1, P2);
        if (k > k1 || !ok) break;
        step(k++, P1, P2, P0);
        if (k > k1 || !ok) break;
        step(k++, P2, P0, P1);
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            if (a.err) atomicExch(a.err, 1);
            for (int p = max(pfirst, k - 1); p <= last_issued; ++p) {
                const int st = (p - pfirst) % NST;
                mbar_wait(bars + st, (uint32_t)(((p - pfirst) / NST) & 1), a.spin);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// host side: tensor maps and launch
// ---------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    });
    return fn;
}

template <typename real>
bool tma_supported(const Geom& g)
{
    return encode_fn() != nullptr && ((int64_t)g.nx * (int64_t)sizeof(real)) % 16 == 0;
}

// box: 0 the stencil's tile, 1 the stencil's tile with halo, 2 the emission region
static bool encode(CUtensorMap* m, void* base, const Geom& g, int elem, int kind)
{
    const int hx = 16 / elem;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * elem, (cuuint64_t)g.nx * g.ny * elem};
    const cuuint32_t box[3] = {(cuuint32_t)(kind == 2 ? kEmitBoxW : (kind == 1 ? TX + 2 * hx : TX)),
                               (cuuint32_t)(kind == 2 ? kEmitBoxH : (kind == 1 ? TY + 2 : TY)), 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = encode_fn()(m, elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                                   base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <typename real>
TmaMaps* make_tma_maps(real* const pot[3][4], real* const src[4], const Geom& g)
{
    if (!tma_supported<real>(g)) return nullptr;
    TmaMaps* m = new TmaMaps();
    bool ok = true;
    for (int l = 0; l < 3; ++l)
        for (int c = 0; c < 4; ++c) {
            ok = ok && encode(&m->halo[l][c], pot[l][c], g, sizeof(real), 1);
            ok = ok && encode(&m->body[l][c], pot[l][c], g, sizeof(real), 0);
            ok = ok && encode(&m->emit[l][c], pot[l][c], g, sizeof(real), 2);
        }
    for (int c = 0; c < 4; ++c) ok = ok && encode(&m->src[c], src[c], g, sizeof(real), 0);
    if (!ok) {
        delete m;
        return nullptr;
    }
    return m;
}

void free_tma_maps(TmaMaps* m) { delete m; }

bool emit_maps(const TmaMaps* maps, int lev_n, int lev_n1, EmitMaps* out)
{
    if (!maps) return false;
    for (int c = 0; c < 3; ++c) {
        out->m[2 * c] = maps->emit[lev_n][c];
        out->m[2 * c + 1] = maps->emit[lev_n1][c];
    }
    out->m[6] = maps->emit[lev_n][3];
    return true;
}

template <typename real>
cudaError_t launch_stencil_tma(const TmaMaps* maps, real* const out[4], real* const prev[4], const MurFaceCoef* mur,
                               int lev_n, int lev_m, const Geom& g, const StencilCoef& cf, int ncomp,
                               const int* src_box, const int* src_far, int src_grow, int* err, cudaStream_t st,
                               int test_skip_plane)
{
    using T = Tile<real>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_stencil_tma<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, T::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    TmaArgs<real> a;
    for (int c = 0; c < 4; ++c) {
        a.out[c] = out[c];
        a.prev[c] = prev[c];
        a.ex[c] = g.nx - (c == 0);
        a.ey[c] = g.ny - (c == 1);
        a.ez[c] = g.nz - (c == 2);
        a.s[c] = (real)(c < 3 ? cf.s_a : cf.s_phi);
    }
    a.lev_n = lev_n;
    a.lev_m = lev_m;
    a.ncomp = ncomp;
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
    a.sbox = src_box;
    a.sfar = src_far;
    a.sgrow = src_grow;
    a.err = err;
    a.skip_plane = test_skip_plane;
    a.spin = test_skip_plane >= 0 ? 1024u : kSpinLimit;
    a.mur = (mur && tma_x_faces<real>()) ? ((mur->ft[0][0] != 0.0 || mur->ft[0][1] != 0.0) ? 2 : 1) : 0;
    a.mf0 = mur ? (real)mur->f0[0] : (real)0;
    a.mf1 = mur ? (real)mur->f1[0] : (real)0;
    a.mfy = mur ? (real)mur->ft[0][0] : (real)0;
    a.mfz = mur ? (real)mur->ft[0][1] : (real)0;
    const int nchunk = (g.nz - 2 + KZ - 1) / KZ;
    const dim3 grd((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, nchunk * ncomp);
    StencilMaps sm;
    for (int c = 0; c < 4; ++c) {
        sm.halo[c] = maps->halo[lev_n][c];
        sm.body[c] = maps->body[lev_m][c];
        sm.src[c] = maps->src[c];
    }
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepStencil), k_stencil_tma<real>, dim3(grd),
                                          dim3(TX / cells_per_thread<real>() * TY),
                                          T::SMEM, st, sm, a, g.sy, g.sz);
        if (le != cudaSuccess) return le;
    }
    count_launches(1);
    return cudaGetLastError();
}

template bool tma_supported<float>(const Geom&);
template bool tma_supported<double>(const Geom&);
template TmaMaps* make_tma_maps<float>(float* const[3][4], float* const[4], const Geom&);
template TmaMaps* make_tma_maps<double>(double* const[3][4], double* const[4], const Geom&);
template cudaError_t launch_stencil_tma<float>(const TmaMaps*, float* const[4], float* const[4], const MurFaceCoef*,
                                               int, int, const Geom&, const StencilCoef&, int, const int*, const int*,
                                               int, int*, cudaStream_t, int);
template cudaError_t launch_stencil_tma<double>(const TmaMaps*, double* const[4], double* const[4],
                                                const MurFaceCoef*, int, int, const Geom&, const StencilCoef&, int,
                                                const int*, const int*, int, int*, cudaStream_t, int);

}  // namespace mithra
