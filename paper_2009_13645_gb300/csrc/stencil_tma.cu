// Potential update (manual Eq. updateEquation; FD is the same equation with A = 0) with the
// tiles staged by the Tensor Memory Accelerator.
//
// One CTA owns a tile of TX x TY columns of one component lattice and marches a chunk of z planes.
// For every plane p it loads, with three cp.async.bulk.tensor copies completing on one mbarrier,
//   psi^n   (TX + 2 HX) x (TY + 2)  (the tile plus the x/y halo; the x origin is moved down to a
//                                     16-byte boundary, so HX = 16 bytes of elements),
//   psi^{n-1}, source  TX x TY,
// into a ring of NST shared-memory stages, NST - 1 planes ahead of the plane being computed.
// Each thread owns one column and keeps planes k-1, k, k+1 of its column and of its four
// transverse neighbours in registers, reading only the new plane k+1 from shared memory.  Results
// go straight to global memory (coalesced rows).
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

namespace mithra {

namespace {

constexpr int TX = 64, TY = 8, NST = 4, KZ = 32;
constexpr uint32_t kSpinLimit = 1u << 20;

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

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(su32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
        : "memory");
}

// Bounded wait; false when the limit expired.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (uint32_t s = 0; s < kSpinLimit; ++s)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace

struct TmaMaps {
    CUtensorMap halo[3][4];   // psi with halo box, per ring level and component
    CUtensorMap body[3][4];   // psi without halo (used as psi^{n-1})
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
    int* err;
};

template <typename real>
__global__ void __launch_bounds__(TX * TY) k_stencil_tma(const __grid_constant__ TmaMaps maps, TmaArgs<real> a,
                                                          int64_t sy, int64_t sz)
{
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
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x = xt + tx, y = yt + ty;
    const bool mine = x >= 1 && x <= ex - 2 && y >= 1 && y <= ey - 2;
    const CUtensorMap* mh = &maps.halo[a.lev_n][comp];
    const CUtensorMap* mb = &maps.body[a.lev_m][comp];
    const CUtensorMap* ms = &maps.src[comp];
    const int pfirst = k0 - 1, plast = k1 + 1;   // psi^n planes needed

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(bars + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int p) {
        const int s = (p - pfirst) % NST;
        unsigned char* st = smem + s * T::STAGE;
        mbar_expect_tx(bars + s, (uint32_t)T::TX_BYTES);
        tma_load_3d(st, mh, xt - T::HX, yt - 1, p, bars + s);
        tma_load_3d(st + T::OFF_PREV, mb, xt, yt, p, bars + s);
        tma_load_3d(st + T::OFF_SRC, ms, xt, yt, p, bars + s);
    };
    int last_issued = pfirst - 1;   // meaningful in thread 0, the only thread that issues copies
    if (threadIdx.x == 0)
        for (int p = pfirst; p <= plast && p < pfirst + NST; ++p) {
            issue(p);
            last_issued = p;
        }

    bool ok = true;
    auto wait_plane = [&](int p) {
        const int s = (p - pfirst) % NST;
        const uint32_t parity = (uint32_t)(((p - pfirst) / NST) & 1);
        if (!mbar_wait(bars + s, parity)) ok = false;
    };
    auto halo_at = [&](int p, int dx, int dy) -> real {
        const real* h = (const real*)(smem + ((p - pfirst) % NST) * T::STAGE);
        return h[(ty + 1 + dy) * T::W + (tx + T::HX + dx)];
    };
    // registers: planes k-1 (0), k (1), k+1 (2) of the column and its neighbours
    real c0, c1, c2, xp0, xp1, xp2, xm0, xm1, xm2, yp0, yp1, yp2, ym0, ym1, ym2;
    wait_plane(pfirst);
    wait_plane(pfirst + 1);
    c0 = halo_at(pfirst, 0, 0);
    xp0 = halo_at(pfirst, 1, 0);
    xm0 = halo_at(pfirst, -1, 0);
    yp0 = halo_at(pfirst, 0, 1);
    ym0 = halo_at(pfirst, 0, -1);
    c1 = halo_at(pfirst + 1, 0, 0);
    xp1 = halo_at(pfirst + 1, 1, 0);
    xm1 = halo_at(pfirst + 1, -1, 0);
    yp1 = halo_at(pfirst + 1, 0, 1);
    ym1 = halo_at(pfirst + 1, 0, -1);
    // the first plane's stage is free once its halo is in registers; the decision to go on is
    // taken by the whole block
    ok = __syncthreads_and(ok) != 0;
    if (ok && threadIdx.x == 0 && pfirst + NST <= plast) {
        issue(pfirst + NST);
        last_issued = pfirst + NST;
    }
    real* __restrict__ o = a.out[comp];
    const real s = a.s[comp];
    int k = k0;
    for (; k <= k1 && ok; ++k) {
        wait_plane(k + 1);
        c2 = halo_at(k + 1, 0, 0);
        xp2 = halo_at(k + 1, 1, 0);
        xm2 = halo_at(k + 1, -1, 0);
        yp2 = halo_at(k + 1, 0, 1);
        ym2 = halo_at(k + 1, 0, -1);
        const unsigned char* stk = smem + ((k - pfirst) % NST) * T::STAGE;
        const real pm = ((const real*)(stk + T::OFF_PREV))[ty * TX + tx];
        const real sr = ((const real*)(stk + T::OFF_SRC))[ty * TX + tx];
        if (mine && ok) {
            const real bxp = a.w * (xp0 + xp2) + a.w0 * xp1;
            const real bxm = a.w * (xm0 + xm2) + a.w0 * xm1;
            const real byp = a.w * (yp0 + yp2) + a.w0 * yp1;
            const real bym = a.w * (ym0 + ym2) + a.w0 * ym1;
            const real v = a.a1 * c1 - pm + a.ax * (bxp + bxm) + a.ay * (byp + bym) + a.a6 * (c0 + c2) + s * sr;
            o[(int64_t)k * sz + (int64_t)y * sy + x] = v;
            if (tma_x_faces<real>() && a.mur && (x == 1 || x == ex - 2)) {
                // Mur x face: b = x -+ 1 on the boundary, q = x its inward neighbour (the formula
                // and the summation order of k_mur_faces)
                const int64_t row = (int64_t)k * sz + (int64_t)y * sy;
                const real* pk = (const real*)(stk + T::OFF_PREV) + ty * TX + tx;
                const int db = x == 1 ? -1 : 1;
                const real n0b = x == 1 ? xm1 : xp1;
                const real nmb = (tx + db < TX) ? pk[db] : a.prev[comp][row + x + db];
                real sa = (real)0, sb = (real)0;
                if (a.mur != 1) {
                    sa = halo_at(k, db, 1) + halo_at(k, db, -1) + yp1 + ym1;
                    sb = (x == 1 ? xm2 : xp2) + (x == 1 ? xm0 : xp0) + c2 + c0;
                }
                o[row + x + db] = a.mf0 * (nmb + v) + a.mf1 * (n0b + c1) - pm + a.mfy * sa + a.mfz * sb;
            }
        }
        c0 = c1; c1 = c2;
        xp0 = xp1; xp1 = xp2;
        xm0 = xm1; xm1 = xm2;
        yp0 = yp1; yp1 = yp2;
        ym0 = ym1; ym1 = ym2;
        // every thread is done with plane k's stage: refill it NST planes ahead
        ok = __syncthreads_and(ok) != 0;
        if (ok && threadIdx.x == 0 && k + NST <= plast) {
            issue(k + NST);
            last_issued = k + NST;
        }
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            if (a.err) atomicExch(a.err, 1);
            // wait (bounded) for the copies this CTA still has in flight before leaving
            for (int p = max(pfirst, k - 1); p <= last_issued; ++p) {
                const int st = (p - pfirst) % NST;
                mbar_wait(bars + st, (uint32_t)(((p - pfirst) / NST) & 1));
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

static bool encode(CUtensorMap* m, void* base, const Geom& g, int elem, bool halo)
{
    const int hx = 16 / elem;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * elem, (cuuint64_t)g.nx * g.ny * elem};
    const cuuint32_t box[3] = {(cuuint32_t)(halo ? TX + 2 * hx : TX), (cuuint32_t)(halo ? TY + 2 : TY), 1};
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
            ok = ok && encode(&m->halo[l][c], pot[l][c], g, sizeof(real), true);
            ok = ok && encode(&m->body[l][c], pot[l][c], g, sizeof(real), false);
        }
    for (int c = 0; c < 4; ++c) ok = ok && encode(&m->src[c], src[c], g, sizeof(real), false);
    if (!ok) {
        delete m;
        return nullptr;
    }
    return m;
}

void free_tma_maps(TmaMaps* m) { delete m; }

template <typename real>
cudaError_t launch_stencil_tma(const TmaMaps* maps, real* const out[4], real* const prev[4], const MurFaceCoef* mur,
                               int lev_n, int lev_m, const Geom& g, const StencilCoef& cf, int ncomp, int* err,
                               cudaStream_t st)
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
    a.err = err;
    a.mur = (mur && tma_x_faces<real>()) ? ((mur->ft[0][0] != 0.0 || mur->ft[0][1] != 0.0) ? 2 : 1) : 0;
    a.mf0 = mur ? (real)mur->f0[0] : (real)0;
    a.mf1 = mur ? (real)mur->f1[0] : (real)0;
    a.mfy = mur ? (real)mur->ft[0][0] : (real)0;
    a.mfz = mur ? (real)mur->ft[0][1] : (real)0;
    const int nchunk = (g.nz - 2 + KZ - 1) / KZ;
    const dim3 grd((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, nchunk * ncomp);
    k_stencil_tma<real><<<grd, TX * TY, T::SMEM, st>>>(*maps, a, g.sy, g.sz);
    count_launches(1);
    return cudaGetLastError();
}

template bool tma_supported<float>(const Geom&);
template bool tma_supported<double>(const Geom&);
template TmaMaps* make_tma_maps<float>(float* const[3][4], float* const[4], const Geom&);
template TmaMaps* make_tma_maps<double>(double* const[3][4], double* const[4], const Geom&);
template cudaError_t launch_stencil_tma<float>(const TmaMaps*, float* const[4], float* const[4], const MurFaceCoef*,
                                               int, int, const Geom&, const StencilCoef&, int, int*, cudaStream_t);
template cudaError_t launch_stencil_tma<double>(const TmaMaps*, double* const[4], double* const[4],
                                                const MurFaceCoef*, int, int, const Geom&, const StencilCoef&, int,
                                                int*, cudaStream_t);

}  // namespace mithra
