// Particle kernels: boost of the lab bunch into the rest frame (Eqs. LorentzTrasnformParticles,
// LorentzTransformDeltaR), and one fused pass per field step that evaluates the external
// field (Lorentz-transformed in FP64), gathers the self-field with linear weights (Eq.
// fieldInterpolation), advances the momentum with the Boris scheme (Eq. BorisScheme) and deposits
// the Umeda zigzag current and the linear-weight charge (Sec. "Current Deposition").  The FP32-mixed
// pass accumulates each block's deposit in a fixed-point tile in shared memory first.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

namespace mithra {

// Static undulator field at a particle with the phase of every planar field taken from the
// step's table (entry of the particle's z cell, in FP64) and rotated by the small angle of the
// offset within the cell and of the sub-step; cosh / sinh of the small transverse argument from
// their series.  Same fields as external_field(), evaluated with fewer FP64 operations.
__device__ __forceinline__ void static_field_fast(const ExtField& f, const PushConst& pc, double Z0, int iz, double fz,
                                                  int m, double x, double y, double E[3], double B[3])
{
    double Bp[3] = {0.0, 0.0, 0.0};
    const double dzl = fma(pc.kz, fz, (double)m * pc.zstep);   // zeta beyond the cell's node plane
    const double zn = fma(pc.kz, (double)iz, Z0);              // zeta of the node plane
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

// sin and cos of a small angle from their Taylor series about 0 (|t| <= 0.8: the first omitted
// terms are below 3e-9); larger angles are halved until they are small and restored with the
// double-angle formulas (never needed when a sub-step moves less than a cell).
__device__ __forceinline__ void sincos_rot32(float t, float* s, float* c)
{
    int k = 0;
    while (fabsf(t) > 0.8f && k < 24) {
        t *= 0.5f;
        ++k;
    }
    const float t2 = t * t;
    float ps = fmaf(t2, 1.f / 362880.f, -1.f / 5040.f);
    ps = fmaf(ps, t2, 1.f / 120.f);
    ps = fmaf(ps, t2, -1.f / 6.f);
    float sn = t * fmaf(ps, t2, 1.f);
    float pc = fmaf(t2, -1.f / 3628800.f, 1.f / 40320.f);
    pc = fmaf(pc, t2, -1.f / 720.f);
    pc = fmaf(pc, t2, 1.f / 24.f);
    pc = fmaf(pc, t2, -0.5f);
    float cs = fmaf(pc, t2, 1.f);
    for (; k > 0; --k) {
        const float s2 = 2.f * sn * cs;
        cs = fmaf(cs, cs, -sn * sn);
        sn = s2;
    }
    *s = sn;
    *c = cs;
}

// cosh and sinh of the transverse argument k_u y from their Taylor series (|x| <= 0.5: the first
// omitted terms are below 3e-10), the library functions beyond.
__device__ __forceinline__ void coshsinh32(float x, float* ch, float* sh)
{
    if (fabsf(x) <= 0.5f) {
        const float y = x * x;
        float pc = fmaf(y, 1.f / 40320.f, 1.f / 720.f);
        pc = fmaf(pc, y, 1.f / 24.f);
        pc = fmaf(pc, y, 0.5f);
        *ch = fmaf(pc, y, 1.f);
        float ps = fmaf(y, 1.f / 362880.f, 1.f / 5040.f);
        ps = fmaf(ps, y, 1.f / 120.f);
        ps = fmaf(ps, y, 1.f / 6.f);
        *sh = x * fmaf(ps, y, 1.f);
    } else {
        *ch = coshf(x);
        *sh = sinhf(x);
    }
}

// Window of a fringe inside a gap (Eq. fringingFieldGap) in FP32, at kd = k_u dz: cos 2a and
// cos 3a from cos a by the double- and triple-angle identities.
__device__ __forceinline__ float gap_window32(float kd, float pwin)
{
    const float c1 = cosf(kd * pwin);
    const float c2 = fmaf(2.f * c1, c1, -1.f);
    const float c3 = c1 * fmaf(2.f, c2, -1.f);
    return 0.35875f + 0.48829f * c1 + 0.14128f * c2 + 0.01168f * c3;
}

// FP32-mixed variant.  The step's table holds, per node plane and planar field, the lab field
// at the plane already Lorentz-transformed to the rest frame in FP64 (sin and cos of the plane's
// undulator phase times the FP64 amplitudes gamma0 beta0 c B, gamma0 B, B) and the phase
// distances to both ends of the undulator (of an array: of the plane's module), all rounded to
// FP32.  The transform is linear with constant coefficients, so rotating the transformed plane
// values by the sub-cell angle equals transforming the rotated ones; that rotation, the fringe
// factors outside [0, L_u] (with an array's gap windows) and cosh/sinh of k_u y are evaluated in
// FP32, the precision of the self-field they are added to.  Returns false for a particle of an
// array whose step reaches past the gap that follows the plane's module (a few node planes in
// front of each module entrance), and for a particle outside the mesh's z range in an array: it
// takes the general FP64 evaluation.
__device__ __forceinline__ bool static_field_mixed(const ExtField& f, const PushConst& pc, int iz, bool inside,
                                                   double Z0, float fz, int m, float x, float y, float E[3], float B[3])
{
    E[0] = E[1] = E[2] = 0.f;
    B[0] = B[1] = B[2] = 0.f;
    const int nplanar = f.kind == 1 ? 2 : 1;
    const float th = fmaf(pc.kdz, fz, pc.kzs * (float)m);   // phase beyond the node plane
    for (int j = 0; j < nplanar; ++j) {
        const float c = j ? -pc.spolf : pc.cpolf, s = j ? pc.cpolf : pc.spolf;
        float4 t0, t1;   // eB0 sin, eB0 cos, bB0 sin, bB0 cos; B0 sin, B0 cos, k_u u, k_u (u - L_u)
        if (inside) {
            t0 = __ldg(pc.ptab32[j] + 2 * iz);
            t1 = __ldg(pc.ptab32[j] + 2 * iz + 1);
        } else {
            // a plane outside the mesh (planar and helical fields): the table's entries formed
            // here, the phase in FP64 and reduced to [-pi, pi] in FP64, its sine and cosine in FP32
            const double ph = f.ku * (fma(pc.kz, (double)iz, Z0) - (j ? f.qlam : 0.0));
            const double n = rint(ph * (0.5 / kPi));
            float sn, cs;
            sincosf((float)fma(-n, 2.0 * kPi, ph), &sn, &cs);
            t0 = make_float4(pc.eB0f * sn, pc.eB0f * cs, pc.bB0f * sn, pc.bB0f * cs);
            t1 = make_float4(pc.B0f * sn, pc.B0f * cs, (float)ph, (float)(ph - f.ku * f.Lu));
        }
        const float ua = t1.z + th, ub = t1.w + th;
        float eS, bS, zC;   // eB0 sin, bB0 sin, B0 cos of the particle's phase
        if (ua >= 0.f && ub <= 0.f) {
            float sd, cd;
            sincos_rot32(th, &sd, &cd);
            eS = fmaf(t0.x, cd, t0.y * sd);
            bS = fmaf(t0.z, cd, t0.w * sd);
            zC = fmaf(t1.y, cd, -t1.x * sd);
        } else if (f.kind != 4) {
            const float kd = ua < 0.f ? ua : ub;
            const float g = expf(-0.5f * kd * kd);
            eS = pc.eB0f * (kd * g);
            bS = pc.bB0f * (kd * g);
            zC = pc.B0f * g;
        } else {
            // array: the plane's module i has peak field Bi (t2.x); before the first module its
            // undamped entrance fringe; after module i its exit fringe, undamped after the last
            // module, otherwise windowed and joined by the windowed entrance fringe of module
            // i + 1 (peak field t2.y) at distance k_u g further on
            const float4 t2 = __ldg(pc.ptab32a + iz);
            float Sv, Cv;
            if (ua < 0.f) {
                const float g = expf(-0.5f * ua * ua);
                Sv = t2.x * (ua * g);
                Cv = t2.x * g;
            } else {
                const bool last = t2.z != 0.f;
                if (!last && ub >= pc.kugf) return false;
                const float e1 = expf(-0.5f * ub * ub) * (last ? 1.f : gap_window32(ub, pc.pwinf));
                Sv = t2.x * (ub * e1);
                Cv = t2.x * e1;
                if (!last) {
                    const float kd2 = ub - pc.kugf;
                    const float e2 = expf(-0.5f * kd2 * kd2) * gap_window32(kd2, pc.pwinf);
                    Sv = fmaf(t2.y, kd2 * e2, Sv);
                    Cv = fmaf(t2.y, e2, Cv);
                }
            }
            eS = pc.egbf * Sv;
            bS = pc.gbf * Sv;
            zC = Cv;
        }
        float ch, sh;
        coshsinh32(pc.kuf * (c * y - s * x), &ch, &sh);
        eS *= ch;
        bS *= ch;
        E[0] -= eS * c;
        E[1] -= eS * s;
        B[0] -= bS * s;
        B[1] += bS * c;
        B[2] += sh * zC;
    }
    return true;
}

// Optical undulator (Sec. "Optical Undulator", Eqs. opticalUndulatorPW / opticalUndulatorGB,
// signalTypes) for the FP32-mixed path at the rest-frame event (x, y, z, t).  The lab coordinates
// and the retarded time tau of the counter-propagating wave are formed in FP64 and the carrier
// phase w_L tau is reduced to [-pi, pi] in FP64; the envelope, the beam profile, the Gouy and
// curvature phases and the cosines are evaluated in FP32.  A wave along -z has B_perp = z x E_perp / c
// (paraxial), so the Lorentz transform to the frame moving with +beta0 multiplies both transverse
// fields by gamma0 (1 + beta0) and leaves E_z, B_z unchanged: that factor sits in the FP64-evaluated
// amplitudes ltE, ltB, rounded once.
__device__ __forceinline__ void optical_field_mixed(const ExtField& f, const PushConst& pc, double x, double y,
                                                    double z, double t, float E[3], float B[3])
{
    const double zeta = f.g0 * fma(f.b0 * kC, t, z);
    const double tl = f.g0 * fma(f.b0 / kC, z, t);
    const double tau = (tl - f.t_f) + (zeta - f.zeta_f) / kC;
    const double ph = f.wL * tau;
    const float phr = (float)fma(-rint(ph * (0.5 / kPi)), 2.0 * kPi, ph);
    float env = 1.f;
    if (f.tp > 0.0 && !(f.signal == 1 && tau > 0.0)) {
        const float u = (float)(tau / f.tp);
        env = expf(-1.3862944f * u * u);   // 2 ln 2
    }
    float S, El = 0.f, Bl = 0.f;
    if (f.kind == 2 || f.w0 <= 0.0) {
        S = env * cosf(phr);
    } else {
        const float l = (float)(f.zeta_f - zeta);     // distance travelled past the focus
        const float lz = l * pc.izrf;
        const float q = 1.f + lz * lz;                // (w(l) / w0)^2
        const float rpar = (float)(x * f.cpol + y * f.spol), rper = (float)(y * f.cpol - x * f.spol);
        const float r2 = rpar * rpar + rper * rper;
        const float curv = pc.kLf * r2 * l / (2.f * (l * l + pc.zrf * pc.zrf));
        const float gouy = atanf(lz);
        const float iw = rsqrtf(q);                   // w0 / w(l)
        const float amp = iw * expf(-r2 / (pc.w0f * pc.w0f * q)) * env;
        S = amp * cosf(phr + gouy - curv);
        const float sl = amp * cosf(phr + 2.f * gouy - curv + 1.5707964f) * pc.izrf * iw;
        El = pc.E0f * rpar * sl;                      // E0 r_par w0 / (z_R w) amp f
        Bl = pc.E0cf * rper * sl;
    }
    E[0] = pc.ltE * S * pc.cpolf;
    E[1] = pc.ltE * S * pc.spolf;
    E[2] = -El;
    B[0] = pc.ltB * S * pc.spolf;
    B[1] = -pc.ltB * S * pc.cpolf;
    B[2] = -Bl;
}

// The phase tables the push reads (phase_entry32 / phase_entry64 in kernels.h) are filled for each
// step by the previous step's tail, and for step 0 when the run is created.

__device__ __forceinline__ bool active_cell(int i, int j, int k, const Geom& g)
{
    return i >= 1 && i <= g.nx - 3 && j >= 1 && j <= g.ny - 3 && k >= 1 && k <= g.nz - 3;
}

// A cell of the active ones or of the one-cell margin around them.  The push's bounds include the
// end cell of every particle in such a cell, so a particle entering the active cells in the next
// step deposits inside the deposit box grown by a cell per sub-step.
__device__ __forceinline__ bool recorded_cell(int i, int j, int k, const Geom& g)
{
    return (unsigned)i <= (unsigned)(g.nx - 2) && (unsigned)j <= (unsigned)(g.ny - 2) &&
           (unsigned)k <= (unsigned)(g.nz - 2);
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

// Where a deposit goes.  GlobalTarget: the four source grids (J_x, J_y, J_z, rho) in global
// memory, atomics in the grids' type.  TileTarget (FP32-mixed path): a block's tile of them in
// shared memory, node (i, j, k) at (k - oz) sz + (j - oy) sy + (i - ox), accumulated in 32-bit
// fixed point - shared-memory integer adds are native, floating-point ones are not - with a
// scale per grid chosen so that no sum can overflow (see the push kernel).
// Offsets are the target's own type: 64-bit in the grids, 32-bit in the tile (at most 4 x 1024
// entries), whose adds address shared memory directly from the tile's shared-window base.
template <typename real>
struct GlobalTarget {
    using off_t = int64_t;
    real* c[4];
    int64_t sy, sz;
    __device__ __forceinline__ int64_t at(int i, int j, int k) const { return (int64_t)k * sz + (int64_t)j * sy + i; }
    __device__ __forceinline__ void add(int comp, int64_t off, real v) const { atomicAdd(c[comp] + off, v); }
};

struct TileTarget {
    using off_t = int;
    int* t;
    unsigned base;   // shared-window address of this lane's copy of entry 0
    int sh;          // log2 of the bytes between consecutive entries (4 bytes x copies)
    int vol;
    int sy, sz;
    int ox, oy, oz;
    float scale[4];
    __device__ __forceinline__ int at(int i, int j, int k) const { return (k - oz) * sz + (j - oy) * sy + (i - ox); }
    __device__ __forceinline__ void add(int comp, int off, float v) const
    {
        const unsigned a = base + ((unsigned)(comp * vol + off) << sh);
        asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(__float2int_rn(v * scale[comp])) : "memory");
    }
};

// One straight piece a -> b (cell units, relative to the base cell) lying in local cell `cl`:
// current on the edges parallel to each axis with the exact path average of the linear
// weights of the two other axes.
template <typename real, typename Tgt>
__device__ __forceinline__ void deposit_piece(const real a[3], const real b[3], const int cl[3], const int base[3],
                                              const Tgt& T, const real qJ[3])
{
    real la[3], d[3], mid[3];
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        la[l] = a[l] - (real)cl[l];
        d[l] = b[l] - a[l];
        mid[l] = la[l] + (real)0.5 * d[l];
    }
    using off_t = typename Tgt::off_t;
    const off_t o = T.at(base[0] + cl[0], base[1] + cl[1], base[2] + cl[2]);
    const off_t st[3] = {1, (off_t)T.sy, (off_t)T.sz};
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        if (d[l] == (real)0) continue;
        const int m = (l + 1) % 3, n = (l + 2) % 3;
        const real F = qJ[l] * d[l];
        const real cross = d[m] * d[n] * (real)(1.0 / 12.0);
        const real wm1 = mid[m], wm0 = (real)1 - mid[m];
        const real wn1 = mid[n], wn0 = (real)1 - mid[n];
        T.add(l, o, F * (wm0 * wn0 + cross));
        T.add(l, o + st[m], F * (wm1 * wn0 - cross));
        T.add(l, o + st[n], F * (wm0 * wn1 - cross));
        T.add(l, o + st[m] + st[n], F * (wm1 * wn1 + cross));
    }
}

// Umeda zigzag of the move A -> B (relative to the base cell, |B - A| <= 1 per axis).  A move
// that stays in its cell has the relay point at the midpoint, so its two pieces are the halves
// of one straight segment in one cell; the path averages of the bilinear weights over the two
// halves sum to the average over the whole segment, so that move is deposited as one piece
// (same currents up to rounding, half the adds).
template <typename real, typename Tgt>
__device__ __forceinline__ void zigzag(const real A[3], const real B[3], const int base[3], const Tgt& T,
                                       const real qJ[3])
{
    int c1[3], c2[3];
    real R[3], E1[3];
    bool cross = false;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        c1[l] = (int)floor(A[l]);
        c2[l] = (int)floor(B[l]);
        const real lo = (real)min(c1[l], c2[l]), hi = (real)max(c1[l], c2[l]);
        const real mid = (real)0.5 * (A[l] + B[l]);
        R[l] = fmin(lo + (real)1, fmax(hi, mid));
        cross = cross || c1[l] != c2[l];
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) E1[l] = cross ? R[l] : B[l];
    deposit_piece(A, E1, c1, base, T, qJ);
    if (cross) deposit_piece(R, B, c2, base, T, qJ);
}

// Charge of one particle at cell c, offset fo, on the cell's eight nodes (linear weights).
template <typename real, typename Tgt>
__device__ __forceinline__ void deposit_rho(const int c[3], const real fo[3], real q, const Tgt& T)
{
    const real wx[2] = {(real)1 - fo[0], fo[0]};
    const real wy[2] = {(real)1 - fo[1], fo[1]};
    const real wz[2] = {(real)1 - fo[2], fo[2]};
    const typename Tgt::off_t o = T.at(c[0], c[1], c[2]);
#pragma unroll
    for (int K = 0; K < 2; ++K)
#pragma unroll
        for (int J = 0; J < 2; ++J)
#pragma unroll
            for (int I = 0; I < 2; ++I) T.add(3, o + K * T.sz + J * T.sy + I, q * wx[I] * wy[J] * wz[K]);
}

// The FP32-mixed deposit tile as the tile path of the push addresses it: the shared-window byte
// address of entry 0 of each source grid in this lane's copy, and the tile's pitches.
struct TileQ {
    unsigned cb[4];
    int sy, sz;
};

__device__ __forceinline__ void tile_red(unsigned a, float v)
{
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(__float2int_rn(v)) : "memory");
}

// deposit_piece on the tile: one straight piece starting at la (relative to its cell, whose tile
// entry is o) with extent d; qs = the charges qJ_l in tile units.
__device__ __forceinline__ void tile_piece(const float la[3], const float d[3], int o, const TileQ& T,
                                           const float qs[3])
{
    const int st[3] = {1, T.sy, T.sz};
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        if (d[l] == 0.f) continue;
        const int m = (l + 1) % 3, n = (l + 2) % 3;
        const float F = qs[l] * d[l];
        const float cross = d[m] * d[n] * (1.f / 12.f);
        const float wm1 = la[m] + 0.5f * d[m], wm0 = 1.f - wm1;
        const float wn1 = la[n] + 0.5f * d[n], wn0 = 1.f - wn1;
        const unsigned a0 = T.cb[l] + 4u * (unsigned)o;
        const unsigned am = 4u * (unsigned)st[m], an = 4u * (unsigned)st[n];
        tile_red(a0, F * (wm0 * wn0 + cross));
        tile_red(a0 + am, F * (wm1 * wn0 - cross));
        tile_red(a0 + an, F * (wm0 * wn1 - cross));
        tile_red(a0 + am + an, F * (wm1 * wn1 + cross));
    }
}

// The zigzag of a move from offset f of its cell (f in [0, 1), tile entry o) to b (cell units
// relative to that cell, b in [-1, 2)) on the tile, and with rho the charge at the end point
// (offset nf of the end cell): the currents of zigzag() and deposit_rho().  The start cell is
// the piece's base cell, so the cell indices need no floor: the end cell is -1, 0 or +1 per axis.
__device__ __forceinline__ void tile_move(const float f[3], const float b[3], const float nf[3], bool rho, int o,
                                          const TileQ& T, const float qs[3], float qr)
{
    float c2[3], R[3], E1[3], d1[3];
    bool cr = false;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        c2[l] = b[l] >= 1.f ? 1.f : (b[l] < 0.f ? -1.f : 0.f);
        const float mid = 0.5f * (f[l] + b[l]);
        R[l] = fminf(fminf(0.f, c2[l]) + 1.f, fmaxf(fmaxf(0.f, c2[l]), mid));
        cr = cr || c2[l] != 0.f;
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        E1[l] = cr ? R[l] : b[l];
        d1[l] = E1[l] - f[l];
    }
    tile_piece(f, d1, o, T, qs);
    const int o2 = o + (int)c2[0] + (int)c2[1] * T.sy + (int)c2[2] * T.sz;
    if (cr) {
        float la[3], d2[3];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            la[l] = R[l] - c2[l];
            d2[l] = b[l] - R[l];
        }
        tile_piece(la, d2, o2, T, qs);
    }
    if (rho) {
        const float wx0 = 1.f - nf[0], wy[2] = {1.f - nf[1], nf[1]}, wz[2] = {1.f - nf[2], nf[2]};
        const unsigned a0 = T.cb[3] + 4u * (unsigned)o2;
#pragma unroll
        for (int K = 0; K < 2; ++K)
#pragma unroll
            for (int J = 0; J < 2; ++J) {
                const float w = qr * wz[K] * wy[J];
                const unsigned a = a0 + 4u * (unsigned)(K * T.sz + J * T.sy);
                tile_red(a, w * wx0);
                tile_red(a + 4u, w * nf[0]);
            }
    }
}

// Block-wide bounding box of [lo, hi] (inclusive node ranges; empty when lo > hi), returned to
// every thread.  One barrier: every thread reduces the four warps' bounds itself.  A second call
// must not start before every thread has read the first's bounds (a barrier in between).
__device__ __forceinline__ void block_box(const int lo[3], const int hi[3], int out[6])
{
    __shared__ __align__(16) int sh[6][4];   // 128 threads = 4 warps
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
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int4 v = *reinterpret_cast<const int4*>(sh[q]);
        out[q] = q < 3 ? min(min(v.x, v.y), min(v.z, v.w)) : max(max(v.x, v.y), max(v.z, v.w));
    }
}

// Block-wide min/max of the cells this block deposited into (or will gather from next step): its
// six bounds [lo_x, lo_y, lo_z, hi_x, hi_y, hi_z] go to rec[6 b] for block b (empty bounds when it
// has no active cell).  The step tail reduces the records into the deposit box; atomics here, on
// the same few words from every block, slowed the push.
__device__ __forceinline__ void box_record(int lo[3], int hi[3], int* rec)
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
        rec[6 * (int64_t)blockIdx.x + q] = v;
    }
}

// One sub-step of one particle: external field (FP64 lab coordinate and Lorentz transform),
// gather of the self-field with linear weights, Boris push, and the move.  b = end point of the
// move in cell units relative to cell ci, (nc, nf) = the new cell and offset.  Returns whether
// the particle starts in an active cell (the gather and the deposit need its whole stencil).
template <typename real>
__device__ __forceinline__ bool push_one(int m, const int ci[3], const real f[3], mom_t<real> u[3], real b[3], int nc[3],
                                         real nf[3], const Geom& g, const ExtField& ef, const Fields6<real>& eb,
                                         const PushConst& pc, double t_half, double Z0)
{
    double E[3], B[3];    // external field in FP64 (FP64 path, and the general evaluation)
    float Ef[3], Bf[3];   // external field rounded to FP32 (FP32-mixed path)
    bool tab = false;
    if constexpr (std::is_same<real, float>::value) {
        const bool inside = ci[2] >= 0 && ci[2] < g.nz;
        if (pc.ptab32[0] && (inside || ef.kind != 4)) {
            const float x = fmaf((float)ci[0] + f[0], pc.dxf, pc.x0f);
            const float y = fmaf((float)ci[1] + f[1], pc.dyf, pc.y0f);
            tab = static_field_mixed(ef, pc, ci[2], inside, Z0, f[2], m, x, y, Ef, Bf);
        } else if (ef.kind == 2 || ef.kind == 3) {
            const double x = g.x0 + ((double)ci[0] + (double)f[0]) * g.dx;
            const double y = g.y0 + ((double)ci[1] + (double)f[1]) * g.dy;
            const double z = g.z0 + ((double)ci[2] + (double)f[2]) * g.dz;
            optical_field_mixed(ef, pc, x, y, z, t_half + (double)m * g.dtb, Ef, Bf);
            tab = true;
        }
    } else {
        if (pc.ptab[0] && ci[2] >= 0 && ci[2] < g.nz) {
            const double x = g.x0 + ((double)ci[0] + (double)f[0]) * g.dx;
            const double y = g.y0 + ((double)ci[1] + (double)f[1]) * g.dy;
            static_field_fast(ef, pc, Z0, ci[2], (double)f[2], m, x, y, E, B);
            tab = true;
        }
    }
    if (!tab) {
        const double t = t_half + (double)m * g.dtb;
        const double x = g.x0 + ((double)ci[0] + (double)f[0]) * g.dx;
        const double y = g.y0 + ((double)ci[1] + (double)f[1]) * g.dy;
        const double z = g.z0 + ((double)ci[2] + (double)f[2]) * g.dz;
        external_field(ef, x, y, z, t, E, B);
        if constexpr (std::is_same<real, float>::value) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                Ef[c] = (float)E[c];
                Bf[c] = (float)B[c];
            }
        }
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
                    const real* q = eb.p + (o + K * g.sz + J * g.sy + I) * kEBStride;
                    real v[6];
                    if constexpr (sizeof(real) == 4) {
                        const float4 a = __ldg(reinterpret_cast<const float4*>(q));
                        const float2 b = __ldg(reinterpret_cast<const float2*>(q + 4));
                        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y;
                    } else {
                        const double2 a = __ldg(reinterpret_cast<const double2*>(q));
                        const double2 b = __ldg(reinterpret_cast<const double2*>(q + 2));
                        const double2 c = __ldg(reinterpret_cast<const double2*>(q + 4));
                        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y, v[4] = c.x, v[5] = c.y;
                    }
#pragma unroll
                    for (int c = 0; c < 6; ++c) s[c] += w * v[c];
                }
    }
    real ig;
    real cdt[3];
    real um[3];   // the momentum the move uses, in the path's precision
    if constexpr (std::is_same<real, float>::value) {
        // Boris rotation in FP32 on the momentum rounded to FP32 (the pair's high part); its
        // increment is added to the pair, and the move uses the rotated FP32 momentum
        float uf[3] = {u[0].x, u[1].x, u[2].x};
        const float Et[3] = {Ef[0] + s[0], Ef[1] + s[1], Ef[2] + s[2]};
        const float Bt[3] = {Bf[0] + s[3], Bf[1] + s[4], Bf[2] + s[5]};
        const float u0[3] = {uf[0], uf[1], uf[2]};
        boris_f32(uf, Et, Bt, pc.dtbf);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            u[l] = mom_add(u[l], uf[l] - u0[l]);
            cdt[l] = pc.cdtbf[l];
            um[l] = uf[l];
        }
        // 1/gamma only scales the FP32 move: FP32 from the updated momentum's high parts
        ig = rsqrtf(fmaf(u[0].x, u[0].x, fmaf(u[1].x, u[1].x, fmaf(u[2].x, u[2].x, 1.f))));
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            E[c] += (double)s[c];
            B[c] += (double)s[3 + c];
            cdt[c] = pc.cdtb[c];
        }
        boris(u, E, B, g.dtb);
        ig = 1.0 / sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
#pragma unroll
        for (int l = 0; l < 3; ++l) um[l] = u[l];
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        b[l] = f[l] + cdt[l] * (um[l] * ig);
        const real fl = floor(b[l]);
        int c = (int)fl;
        real o = b[l] - fl;
        if (o >= (real)1) { o -= (real)1; c += 1; }
        b[l] = (real)c + o;   // the deposit ends exactly at the stored (cell, offset) point
        nc[l] = ci[l] + c;
        nf[l] = o;
    }
    return a1;
}

// Resident blocks of 128 threads per SM the push is compiled for (the register budget per thread).
#ifndef MITHRA_PUSH_MIN_BLOCKS_F32
#define MITHRA_PUSH_MIN_BLOCKS_F32 7
#endif
#ifndef MITHRA_PUSH_MIN_BLOCKS_F64
#define MITHRA_PUSH_MIN_BLOCKS_F64 5
#endif

// 32-bit entries of the FP32-mixed push's deposit tile in shared memory (all grids and copies).
#ifndef MITHRA_PUSH_TILE_INTS
#define MITHRA_PUSH_TILE_INTS 4096
#endif
constexpr int kTileInts = MITHRA_PUSH_TILE_INTS;

// The push: one thread per particle, 128 per block, the particles in cell-sorted order.
//
// Deposit (FP32-mixed path).  The block's current (and, after the last sub-step, charge) first
// accumulates in a fixed-point tile of the source grids in shared memory that covers the block's
// bounding box of touched nodes; the tile's nonzero nodes are then added to the grids in global
// memory, one atomic per node and grid.  Neighbouring particles of the sorted order share cells,
// so many shared-memory adds meet in one global add.  A block whose box does not fit the tile,
// and every move longer than a cell on some axis (split into pieces), adds to global memory
// directly, as does the whole FP64 path.
template <typename real>
__global__ void __launch_bounds__(128, sizeof(real) == 4 ? MITHRA_PUSH_MIN_BLOCKS_F32 : MITHRA_PUSH_MIN_BLOCKS_F64)
    k_push(Particles<real> P, int64_t np, Geom g, ExtField ef, Fields6<real> eb, Fields4<real> src, PushConst pc,
           int* box_rec)
{
    dep_begin();
    // FP32-mixed deposit tile (see below), cleared once here while the particle loads are in flight;
    // the flush of every sub-step but the last clears what it read
    __shared__ __align__(16) int tile[sizeof(real) == 4 ? kTileInts : 4];
    if constexpr (std::is_same<real, float>::value) {
        int4* t4 = reinterpret_cast<int4*>(tile);
        for (int i = threadIdx.x; i < kTileInts / 4; i += blockDim.x) t4[i] = make_int4(0, 0, 0, 0);
    }
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int lo[3] = {0x7fffffff, 0x7fffffff, 0x7fffffff};
    int hi[3] = {(int)0x80000000, (int)0x80000000, (int)0x80000000};
    // every thread runs the loop (the block shares the tile); threads past the end carry a
    // particle outside the grid that deposits nothing
    const bool alive = p < np;
    int ci[3] = {-4, -4, -4};
    real f[3] = {0, 0, 0};
    mom_t<real> u[3] = {};
    if (alive) {
        ci[0] = P.ix[p];
        ci[1] = P.iy[p];
        ci[2] = P.iz[p];
        f[0] = P.fx[p];
        f[1] = P.fy[p];
        f[2] = P.fz[p];
        u[0] = P.ux[p];
        u[1] = P.uy[p];
        u[2] = P.uz[p];
    }
    real qJ[3], q;
    if constexpr (std::is_same<real, float>::value) {
        qJ[0] = pc.qJf[0];
        qJ[1] = pc.qJf[1];
        qJ[2] = pc.qJf[2];
        q = pc.qrhof;
    } else {
        qJ[0] = pc.qJ[0];
        qJ[1] = pc.qJ[1];
        qJ[2] = pc.qJ[2];
        q = pc.qrho;
    }
    GlobalTarget<real> G;
    G.c[0] = src.c[0];
    G.c[1] = src.c[1];
    G.c[2] = src.c[2];
    G.c[3] = src.c[3];
    G.sy = g.sy;
    G.sz = g.sz;
    const double t_half = pc.sd->t_half, Z0 = pc.sd->Z0;
    bool rho_done = false;
    // The previous step's deposit box holds the start cell of every particle that can deposit in
    // this step (recorded_cell), so the deposits of its moves of at most one cell per sub-step stay
    // in that box grown by the sub-step count; any other deposit sets the far-move flag.  The start
    // cell is read again from the particle arrays (still unchanged) where it is needed.
    auto started_recorded = [&]() { return recorded_cell(P.ix[p], P.iy[p], P.iz[p], g); };
    for (int m = 0; m < g.substeps; ++m) {
        real b[3] = {f[0], f[1], f[2]};
        int nc[3] = {ci[0], ci[1], ci[2]};
        real nf[3] = {f[0], f[1], f[2]};
        const bool a1 = alive && push_one<real>(m, ci, f, u, b, nc, nf, g, ef, eb, pc, t_half, Z0);
        bool simple = false;   // a move of at most one cell per axis: deposited through the tile
        if (a1 && active_cell(nc[0], nc[1], nc[2], g)) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                lo[l] = min(lo[l], min(ci[l], nc[l]));
                hi[l] = max(hi[l], max(ci[l], nc[l]));
            }
            real mx = fmax(fabs(b[0] - f[0]), fmax(fabs(b[1] - f[1]), fabs(b[2] - f[2])));
            if (!(mx <= (real)1) || (m > 0 && !started_recorded())) *pc.far = 1;
            if (mx <= (real)1) {
                simple = true;
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
                    zigzag(A, Bq, ci, G, qJ);
                }
            }
        }
        // the charge at the end of the last sub-step goes through the tile with the current
        // when the move was simple; otherwise it is added directly below
        const bool last = m == g.substeps - 1;
        const bool rho_t = simple && g.space_charge && last;
        if constexpr (std::is_same<real, float>::value) {
            int tlo[3], thi[3], box[6];
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                tlo[l] = simple ? min(ci[l], nc[l]) : 0x7fffffff;
                thi[l] = simple ? max(ci[l], nc[l]) + 1 : (int)0x80000000;
            }
            block_box(tlo, thi, box);   // its barrier also orders the tile's clearing
            // the tile's rows start on a multiple of four nodes and hold whole quads of nodes, so
            // that a quad of a row is added to the grid with one vector atomic
            const int bx0 = box[0] & ~3;
            const int tx = (box[3] - bx0 + 4) & ~3, ty = box[4] - box[1] + 1, tz = box[5] - box[2] + 1;
            const int ngrid = (g.space_charge && last) ? 4 : 3;
            if (box[0] <= box[3] && (int64_t)ngrid * tx * ty * tz + 4 <= kTileInts) {
                const int vol = tx * ty * tz, nent = ngrid * vol;
                // Up to four copies of the tile, lane l adding to copy l mod copies: the sorted
                // lanes of a warp often share a cell, and the copies divide the number of lanes
                // that meet in one address of an add.  The copies lie cs = nent + 4 entries
                // apart, so that the copies of one entry sit in different banks.
                const int cs = nent + 4;
                const int lc = 4 * cs <= kTileInts ? 2 : (2 * cs <= kTileInts ? 1 : 0);
                int4* tile4 = reinterpret_cast<int4*>(tile);
                // A particle adds at most |qJ_l| to any node of J_l over its two pieces (the
                // path-averaged weights lie in [0, 1] and the pieces' extents along l sum to at
                // most one cell) and at most |q| to a node of rho, so a block of 128 sums to at most
                // 128 |qJ_l| (128 |q|): that maps to 2^30, and the rounding of each term adds at
                // most 1/2.
                TileQ T;
                const unsigned tb = (unsigned)__cvta_generic_to_shared(tile) + 4u * (unsigned)cs * (threadIdx.x & ((1u << lc) - 1u));
#pragma unroll
                for (int c = 0; c < 4; ++c) T.cb[c] = tb + 4u * (unsigned)(c * vol);
                T.sy = tx;
                T.sz = tx * ty;
                if (simple) {
                    const float qs[3] = {pc.qJt[0], pc.qJt[1], pc.qJt[2]};
                    const int o = (ci[2] - box[2]) * T.sz + (ci[1] - box[1]) * T.sy + (ci[0] - bx0);
                    tile_move(f, b, nf, rho_t, o, T, qs, pc.qrhot);
                }
                __syncthreads();
                // quad index -> (grid, k, j, quad of the row) with FP32 reciprocals: the quotients
                // are below 2^10 and (index + 1/2) / divisor stays at least 1/(2 divisor) away from
                // an integer.  With rows of the grids that are whole quads (nx a multiple of 4) a
                // quad with a nonzero node is one float4 atomic (16-byte aligned), else one atomic
                // per nonzero node.
                // approximate reciprocals: relative error below 2^-21 in the products, which moves a
                // quotient below 2^10 by less than 2^-11, inside the 1/(2 divisor) >= 2^-11 margin
                const int qx = tx >> 2, vq = vol >> 2, nq = nent >> 2;
                const float ivq = __fdividef(1.f, (float)vq), iqxy = __fdividef(1.f, (float)(qx * ty));
                const float iqx = __fdividef(1.f, (float)qx);
                const bool vec = (g.sy & 3) == 0 && (g.sz & 3) == 0;
                for (int i = threadIdx.x; i < nq; i += blockDim.x) {
                    int4 v = tile4[i];
                    for (int cp = 1; cp < (1 << lc); ++cp) {
                        const int4 w = tile4[cp * (cs >> 2) + i];
                        v.x += w.x;
                        v.y += w.y;
                        v.z += w.z;
                        v.w += w.w;
                    }
                    if (!last)
                        for (int cp = 0; cp < (1 << lc); ++cp) tile4[cp * (cs >> 2) + i] = make_int4(0, 0, 0, 0);
                    if ((v.x | v.y | v.z | v.w) != 0) {
                        const int c = (int)(((float)i + 0.5f) * ivq), r = i - c * vq;
                        const int k = (int)(((float)r + 0.5f) * iqxy), r2 = r - k * qx * ty;
                        const int j = (int)(((float)r2 + 0.5f) * iqx), iq = r2 - j * qx;
                        const float inv = c == 0 ? pc.tunit[0] : c == 1 ? pc.tunit[1] : c == 2 ? pc.tunit[2] : pc.tunit[3];
                        real* dst = (c == 0 ? src.c[0] : c == 1 ? src.c[1] : c == 2 ? src.c[2] : src.c[3]) +
                                    G.at(bx0 + 4 * iq, box[1] + j, box[2] + k);
                        const float4 fv = make_float4((float)v.x * inv, (float)v.y * inv, (float)v.z * inv, (float)v.w * inv);
                        if (vec) {
                            atomicAdd(reinterpret_cast<float4*>(dst), fv);
                        } else {
                            if (v.x) atomicAdd(dst, fv.x);
                            if (v.y) atomicAdd(dst + 1, fv.y);
                            if (v.z) atomicAdd(dst + 2, fv.z);
                            if (v.w) atomicAdd(dst + 3, fv.w);
                        }
                    }
                }
                if (!last) __syncthreads();   // the tile and the bounds are reused by the next sub-step
            } else {
                if (simple) {
                    zigzag(f, b, ci, G, qJ);
                    if (rho_t) deposit_rho(nc, nf, q, G);
                }
                if (!last) __syncthreads();   // the bounds are reused by the next sub-step
            }
        } else if (simple) {
            // FP64 path: floating-point adds straight into the grids
            zigzag(f, b, ci, G, qJ);
            if (rho_t) deposit_rho(nc, nf, q, G);
        }
        if (last) rho_done = rho_t;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            ci[l] = nc[l];
            f[l] = nf[l];
        }
    }
    if (alive && recorded_cell(ci[0], ci[1], ci[2], g)) {
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            lo[l] = min(lo[l], ci[l]);
            hi[l] = max(hi[l], ci[l]);
        }
        if (g.space_charge && !rho_done && active_cell(ci[0], ci[1], ci[2], g)) {
            if (!started_recorded()) *pc.far = 1;
            deposit_rho(ci, f, q, G);
        }
    }
    if (alive) {
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
    box_record(lo, hi, box_rec);
}

__global__ void k_finite_check(const double* __restrict__ a, int64_t n, int* flag)
{
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad = bad || !isfinite(a[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

cudaError_t launch_finite_check(const double* a, int64_t n, int* flag, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_finite_check<<<1216, 256, 0, st>>>(a, n, flag);
    count_launches(1);
    return cudaGetLastError();
}

// Lab-frame macro-particles (x, y, z relative to the bunch reference at t' = 0, gamma*beta) to
// the rest frame at the common time T0 + dt/2 (the time of r^{1/2}).  FP64 throughout; the cell
// sizes enter as their reciprocals and 1/gamma as one reciprocal square root (each within an ulp of
// the quotient): a division costs some twenty instructions of the FP64 pipe, whose rate on this
// GPU is 1/64 of the FP32 one.
template <typename real>
__global__ void k_boost(const double* __restrict__ lab, int64_t np, Particles<real> P, Geom g, double g0, double b0,
                        double z_ref, double idx, double idy, double idz)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double* L = lab + 6 * p;
    const double ux = L[3], uy = L[4], uzl = L[5];
    const double gl = sqrt(1.0 + ux * ux + uy * uy + uzl * uzl);
    const double uz = g0 * (uzl - b0 * gl);
    const double ig = rsqrt(1.0 + ux * ux + uy * uy + uz * uz);
    // ballistic shift with the rest-frame velocity over c (T0 + dt/2 - t_event)
    const double s = g0 * b0 * L[2] + 0.5 * kC * g.dt;
    const double x = L[0] + ux * ig * s;
    const double y = L[1] + uy * ig * s;
    const double z = z_ref + g0 * L[2] + uz * ig * s;
    split_pos<real>((x - g.x0) * idx, P.ix + p, P.fx + p);
    split_pos<real>((y - g.y0) * idy, P.iy + p, P.fy + p);
    split_pos<real>((z - g.z0) * idz, P.iz + p, P.fz + p);
    mom_set(P.ux + p, ux);
    mom_set(P.uy + p, uy);
    mom_set(P.uz + p, uz);
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
    mom_set(P.ux + p, R[3]);
    mom_set(P.uy + p, R[4]);
    mom_set(P.uz + p, R[5]);
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
    R[3] = mom_value(P.ux[p]);
    R[4] = mom_value(P.uy[p]);
    R[5] = mom_value(P.uz[p]);
}

static inline unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename real>
cudaError_t launch_push(const Particles<real>& P, int64_t np, const Geom& g, const ExtField& ef,
                        const Fields6<real>& eb, const Fields4<real>& src, const PushConst& pc, int* box_rec,
                        cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    {
        const cudaError_t le = launch_dep(dep_launch_on<real>(st, kDepPush), k_push<real>, dim3(nblocks(np, 128)), dim3(128), 0,
                                          st, P, np, g, ef, eb, src, pc, box_rec);
        if (le != cudaSuccess) return le;
    }
    count_launches(1);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_boost(const double* lab6, int64_t np, const Particles<real>& P, const Geom& g, const ExtField& ef,
                         double z_ref, cudaStream_t st)
{
    if (np <= 0) return cudaSuccess;
    k_boost<real><<<nblocks(np, 256), 256, 0, st>>>(lab6, np, P, g, ef.g0, ef.b0, z_ref, 1.0 / g.dx, 1.0 / g.dy,
                                                     1.0 / g.dz);
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
