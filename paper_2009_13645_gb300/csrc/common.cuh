// Internal definitions shared by the CUDA translation units of libmithra.
// Physics: MITHRA 2.0 manual (arXiv:2009.13645), Ch. "Methodology".
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace mithra {

// CODATA 2018
constexpr double kC = 299792458.0;
constexpr double kMu0 = 1.25663706212e-6;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kPi = 3.14159265358979323846;

// Rest-frame grid geometry.  Fields are stored x-fastest with row pitch nx and plane
// pitch nx*ny.  A_x/J_x index i sits at (i+1/2)dx, A_y at (j+1/2)dy, A_z at (k+1/2)dz;
// phi, rho, E and B sit on nodes.
struct Geom {
    int nx, ny, nz;
    int64_t sy, sz, ncell;
    double dx, dy, dz, dt, dtb;
    double x0, y0, z0;
    int substeps;
    int space_charge;
};

// External field of the run (lab frame) and the boost (manual Sec. "Field Initialization",
// Eqs. undulatorField, fringingField, opticalUndulatorPW, opticalUndulatorGB,
// LorentzTransformR2L, LorentzTransformElectric/Magnetic).
struct ExtField {
    int kind;           // -1 none, 0 planar, 1 helical, 2 optical plane wave, 3 optical Gaussian, 4 array
    double g0, b0;      // rest-frame gamma0, beta0
    double ku, Lu, B0;  // static undulator: wavenumber, length, peak field
    double qlam;        // helical: quarter period offset of the second planar field
    double cpol, spol;  // polarisation direction (cos, sin)
    double kL, wL, E0;  // laser wavenumber, angular frequency, peak field
    double zeta_f, t_f; // laser focus and the time its pulse centre crosses it (lab)
    double tp;          // pulse length tau (s); <= 0: continuous
    int signal;         // 0 Gaussian envelope, 1 flat-top
    double w0, zr;      // Gaussian beam waist and Rayleigh length; w0 <= 0: plane wave
    double gap, dB0;    // undulator array: gap between modules, peak-field step per module
    int nmod;           // undulator array: number of modules
};

// Planar static undulator field along (-sin, cos) in the xy-plane starting at lab
// coordinate `off`; before the entrance the manual's Neumann-type fringe, after the end
// the same fringe mirrored.  Adds to Bp.
__host__ __device__ inline void planar_add(const ExtField& f, double c, double s, double off,
                                           double xl, double yl, double zeta, double Bp[3])
{
    const double yu = c * yl - s * xl;          // coordinate along the field direction
    const double u = zeta - off;
    double sn, cs;
    if (u >= 0.0 && u <= f.Lu) {
        sincos(f.ku * u, &sn, &cs);
    } else {
        const double d = (u < 0.0) ? u : (u - f.Lu);
        const double kd = f.ku * d;
        const double g = exp(-0.5 * kd * kd);
        sn = kd * g;
        cs = g;
    }
    const double ky = f.ku * yu;
    const double ch = cosh(ky), sh = sinh(ky);
    const double Bt = f.B0 * ch * sn;   // transverse component along the field direction
    Bp[0] -= Bt * s;
    Bp[1] += Bt * c;
    Bp[2] += f.B0 * sh * cs;
}

// Window of a fringe inside a gap of length g (Eq. fringingFieldGap).
__host__ __device__ inline double gap_window(double d, double g)
{
    const double a = kPi * d / g;
    return 0.35875 + 0.48829 * cos(a) + 0.14128 * cos(2.0 * a) + 0.01168 * cos(3.0 * a);
}

// Static undulator array along (-sin, cos): module i (peak field B0 + i dB0) spans [i P, i P + Lu]
// with P = Lu + gap.  At most two modules reach a given zeta: the one whose entrance lies at or
// before it (its interior, or its exit fringe, windowed by Eq. fringingFieldGap inside the gap
// and undamped after the last module) and the next one (its entrance fringe inside the gap);
// before the first entrance only the first module's undamped entrance fringe.  Adds to Bp.
__host__ __device__ inline void array_add(const ExtField& f, double xl, double yl, double zeta, double Bp[3])
{
    const double P = f.Lu + f.gap;
    int i = (int)floor(zeta / P);
    i = i < -1 ? -1 : (i > f.nmod - 1 ? f.nmod - 1 : i);
    // keep zeta - i P in [0, P) wherever the floor rounded across a module boundary
    if (i >= 0 && zeta - i * P < 0.0) --i;
    if (i < f.nmod - 1 && zeta - (i + 1) * P >= 0.0) ++i;
    double sn = 0.0, cs = 0.0;   // peak field times the shape, summed over the modules
    auto fringe = [&](double Bm, double d, bool open) {
        const double kd = f.ku * d;
        const double e = exp(-0.5 * kd * kd) * (open ? 1.0 : gap_window(d, f.gap));
        sn += Bm * kd * e;
        cs += Bm * e;
    };
    if (i < 0) {
        fringe(f.B0, zeta, true);
    } else {
        const double u = zeta - i * P;
        const double Bi = f.B0 + i * f.dB0;
        const bool last = i == f.nmod - 1;
        if (u < f.Lu || (last && u <= f.Lu)) {
            double s, c;
            sincos(f.ku * u, &s, &c);
            sn += Bi * s;
            cs += Bi * c;
        } else if (last || u - f.Lu < f.gap) {
            fringe(Bi, u - f.Lu, last);
        }
        if (!last && P - u < f.gap) fringe(Bi + f.dB0, u - P, false);
    }
    const double yu = f.cpol * yl - f.spol * xl;
    const double ky = f.ku * yu;
    const double Bt = cosh(ky) * sn;
    Bp[0] -= Bt * f.spol;
    Bp[1] += Bt * f.cpol;
    Bp[2] += sinh(ky) * cs;
}

// Time signature f(tau, phase) of the laser (Eq. signalTypes, A0 = 1).
__host__ __device__ inline double laser_signal(const ExtField& f, double tau, double phase)
{
    const double car = cos(f.wL * tau + phase);
    if (f.tp <= 0.0 || (f.signal == 1 && tau > 0.0)) return car;
    return car * exp(-2.0 * 0.69314718055994530942 * (tau * tau) / (f.tp * f.tp));
}

// Lab-frame field at lab event (xl, yl, zeta, tl).
__host__ __device__ inline void lab_field(const ExtField& f, double xl, double yl, double zeta, double tl,
                                          double Ep[3], double Bp[3])
{
    Ep[0] = Ep[1] = Ep[2] = 0.0;
    Bp[0] = Bp[1] = Bp[2] = 0.0;
    if (f.kind == 0) {
        planar_add(f, f.cpol, f.spol, 0.0, xl, yl, zeta, Bp);
    } else if (f.kind == 1) {
        planar_add(f, f.cpol, f.spol, 0.0, xl, yl, zeta, Bp);
        // rotated by +90 degrees: (cos, sin) -> (-sin, cos)
        planar_add(f, -f.spol, f.cpol, f.qlam, xl, yl, zeta, Bp);
    } else if (f.kind == 4) {
        array_add(f, xl, yl, zeta, Bp);
    } else if (f.kind == 2 || f.kind == 3) {
        const double tau = (tl - f.t_f) + (zeta - f.zeta_f) / kC;   // counter-propagating (-z)
        double Epar, El = 0.0, Bl = 0.0;
        if (f.kind == 2 || f.w0 <= 0.0) {
            Epar = f.E0 * laser_signal(f, tau, 0.0);
        } else {
            const double l = f.zeta_f - zeta;                       // distance travelled past the focus
            const double lz = l / f.zr;
            const double wl = f.w0 * sqrt(1.0 + lz * lz);
            const double rpar = xl * f.cpol + yl * f.spol;
            const double rper = yl * f.cpol - xl * f.spol;
            const double r2 = rpar * rpar + rper * rper;
            // k r^2 / (2 R(l)) with R(l) = l (1 + (z_R/l)^2) written without dividing by l
            const double curv = f.kL * r2 * l / (2.0 * (l * l + f.zr * f.zr));
            const double gouy = atan(lz);
            const double amp = (f.w0 / wl) * exp(-r2 / (wl * wl));
            Epar = f.E0 * amp * laser_signal(f, tau, gouy - curv);
            const double sl = laser_signal(f, tau, 2.0 * gouy - curv + 0.5 * kPi);
            El = f.E0 * rpar * f.w0 / (f.zr * wl) * amp * sl;
            Bl = f.E0 * rper * f.w0 / (kC * f.zr * wl) * amp * sl;
        }
        Ep[0] = Epar * f.cpol;
        Ep[1] = Epar * f.spol;
        Ep[2] = -El;
        Bp[0] = Epar * f.spol / kC;
        Bp[1] = -Epar * f.cpol / kC;
        Bp[2] = -Bl;
    }
}

// Seed beam along +z (Sec. "Seed Field"; Sec. FIELD, field-initialization), lab parameters.
struct SeedField {
    int type;               // -1 none, 0 plane wave, 1 Gaussian beam
    double g0, b0;          // rest frame
    double A0;              // a0 m c / e
    double k, w;            // lab wavenumber and angular frequency
    double zr, w0;          // Rayleigh length and waist (Gaussian beam)
    double focus, t0;       // lab reference point and the time its pulse centre passes it
    double tp;              // pulse length tau (s); <= 0: continuous
    double cep, cpol, spol;
};

// The seed's transverse vector potential at the rest-frame event (x, y, z, t): the lab value at
// the boosted event (a transverse potential is unchanged by a boost along z).
__host__ __device__ inline void seed_potential(const SeedField& s, double x, double y, double z, double t,
                                               double* ax, double* ay)
{
    const double zeta = s.g0 * fma(s.b0 * kC, t, z);
    // retarded lab time t' - t0 - (zeta - focus)/c of the +z beam; t' - zeta/c written in rest
    // variables, (t - z/c) / (g0 (1 + b0)), avoids cancelling two nearly equal lab times
    const double tau = (t - z / kC) / (s.g0 * (1.0 + s.b0)) - s.t0 + s.focus / kC;
    double amp = 1.0, ph = 0.0;
    if (s.type == 1) {
        const double l = zeta - s.focus, lz = l / s.zr;
        const double wl = s.w0 * sqrt(1.0 + lz * lz);
        const double r2 = x * x + y * y;
        amp = (s.w0 / wl) * exp(-r2 / (wl * wl));
        ph = atan(lz) - s.k * r2 * l / (2.0 * (l * l + s.zr * s.zr));
    }
    double f = cos(s.w * tau + ph + s.cep);
    if (s.tp > 0.0) f *= exp(-2.0 * 0.69314718055994530942 * (tau * tau) / (s.tp * s.tp));
    const double a = s.A0 * amp * f;
    *ax = a * s.cpol;
    *ay = a * s.spol;
}

// External field at a rest-frame event (x, y, z, t): lab event, lab field, then the field
// transform to the frame moving with beta0 along z.
__host__ __device__ inline void external_field(const ExtField& f, double x, double y, double z, double t,
                                               double E[3], double B[3])
{
    if (f.kind < 0) {
        E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.0;
        return;
    }
    const double zeta = f.g0 * fma(f.b0 * kC, t, z);
    const double tl = f.g0 * fma(f.b0 / kC, z, t);
    double Ep[3], Bp[3];
    lab_field(f, x, y, zeta, tl, Ep, Bp);
    const double g = f.g0, bc = f.b0 * kC, bic = f.b0 / kC;
    E[0] = g * (Ep[0] - bc * Bp[1]);
    E[1] = g * (Ep[1] + bc * Bp[0]);
    E[2] = Ep[2];
    B[0] = g * (Bp[0] + bic * Ep[1]);
    B[1] = g * (Bp[1] - bic * Ep[0]);
    B[2] = Bp[2];
}

// sin and cos of a small angle |d| <= 1 in FP64 from their Taylor series (terms through d^19 /
// d^20; the first omitted term is below 1e-19 for |d| <= 1).
__host__ __device__ inline void sincos_small(double d, double* s, double* c)
{
    const double x = d * d;
    double ps = 1.0 / 121645100408832000.0;                  // 1/19!
    ps = fma(ps, -x, 1.0 / 355687428096000.0);               // 1/17!
    ps = fma(ps, -x, 1.0 / 1307674368000.0);                 // 1/15!
    ps = fma(ps, -x, 1.0 / 6227020800.0);                    // 1/13!
    ps = fma(ps, -x, 1.0 / 39916800.0);                      // 1/11!
    ps = fma(ps, -x, 1.0 / 362880.0);                        // 1/9!
    ps = fma(ps, -x, 1.0 / 5040.0);                          // 1/7!
    ps = fma(ps, -x, 1.0 / 120.0);                           // 1/5!
    ps = fma(ps, -x, 1.0 / 6.0);                             // 1/3!
    ps = fma(ps, -x, 1.0);
    *s = d * ps;
    double pc = 1.0 / 2432902008176640000.0;                 // 1/20!
    pc = fma(pc, -x, 1.0 / 6402373705728000.0);              // 1/18!
    pc = fma(pc, -x, 1.0 / 20922789888000.0);                // 1/16!
    pc = fma(pc, -x, 1.0 / 87178291200.0);                   // 1/14!
    pc = fma(pc, -x, 1.0 / 479001600.0);                     // 1/12!
    pc = fma(pc, -x, 1.0 / 3628800.0);                       // 1/10!
    pc = fma(pc, -x, 1.0 / 40320.0);                         // 1/8!
    pc = fma(pc, -x, 1.0 / 720.0);                           // 1/6!
    pc = fma(pc, -x, 1.0 / 24.0);                            // 1/4!
    pc = fma(pc, -x, 0.5);                                   // 1/2!
    *c = fma(pc, -x, 1.0);
}

// cosh and sinh of |x| <= 0.5 in FP64 from their Taylor series (through x^16 / x^17).
__host__ __device__ inline void coshsinh_small(double x, double* ch, double* sh)
{
    const double y = x * x;
    double pc = 1.0 / 20922789888000.0;                      // 1/16!
    pc = fma(pc, y, 1.0 / 87178291200.0);
    pc = fma(pc, y, 1.0 / 479001600.0);
    pc = fma(pc, y, 1.0 / 3628800.0);
    pc = fma(pc, y, 1.0 / 40320.0);
    pc = fma(pc, y, 1.0 / 720.0);
    pc = fma(pc, y, 1.0 / 24.0);
    pc = fma(pc, y, 0.5);
    *ch = fma(pc, y, 1.0);
    double ps = 1.0 / 355687428096000.0;                     // 1/17!
    ps = fma(ps, y, 1.0 / 1307674368000.0);
    ps = fma(ps, y, 1.0 / 6227020800.0);
    ps = fma(ps, y, 1.0 / 39916800.0);
    ps = fma(ps, y, 1.0 / 362880.0);
    ps = fma(ps, y, 1.0 / 5040.0);
    ps = fma(ps, y, 1.0 / 120.0);
    ps = fma(ps, y, 1.0 / 6.0);
    ps = fma(ps, y, 1.0);
    *sh = x * ps;
}

// Boris rotation of the normalised momentum u of an electron (Eq. BorisScheme), FP64.
__host__ __device__ inline void boris(double u[3], const double E[3], const double B[3], double dtb)
{
    const double h = kQe * dtb / (2.0 * kMe * kC);
    const double t1x = u[0] - h * E[0], t1y = u[1] - h * E[1], t1z = u[2] - h * E[2];
    const double a = -kQe * dtb / (2.0 * kMe * sqrt(1.0 + t1x * t1x + t1y * t1y + t1z * t1z));
    const double t2x = t1x + a * (t1y * B[2] - t1z * B[1]);
    const double t2y = t1y + a * (t1z * B[0] - t1x * B[2]);
    const double t2z = t1z + a * (t1x * B[1] - t1y * B[0]);
    const double s = 2.0 * a / (1.0 + a * a * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
    u[0] = t1x + s * (t2y * B[2] - t2z * B[1]) - h * E[0];
    u[1] = t1y + s * (t2z * B[0] - t2x * B[2]) - h * E[1];
    u[2] = t1z + s * (t2x * B[1] - t2y * B[0]) - h * E[2];
}

// The same Boris rotation in FP32 (Eq. BorisScheme); used by the FP32-mixed push, which adds
// the resulting increment to the momentum held as a pair of floats (mom_add).
__host__ __device__ inline void boris_f32(float u[3], const float E[3], const float B[3], float dtb)
{
    const float h = (float)(kQe / (2.0 * kMe * kC)) * dtb;
    const float t1x = u[0] - h * E[0], t1y = u[1] - h * E[1], t1z = u[2] - h * E[2];
    const float a = -(float)(kQe / (2.0 * kMe)) * dtb / sqrtf(1.0f + t1x * t1x + t1y * t1y + t1z * t1z);
    const float t2x = t1x + a * (t1y * B[2] - t1z * B[1]);
    const float t2y = t1y + a * (t1z * B[0] - t1x * B[2]);
    const float t2z = t1z + a * (t1x * B[1] - t1y * B[0]);
    const float s = 2.0f * a / (1.0f + a * a * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
    u[0] = t1x + s * (t2y * B[2] - t2z * B[1]) - h * E[0];
    u[1] = t1y + s * (t2z * B[0] - t2x * B[2]) - h * E[1];
    u[2] = t1z + s * (t2x * B[1] - t2y * B[0]) - h * E[2];
}

#ifdef __CUDACC__
// True in the last block of the grid to arrive (every block calls it once, with all its
// threads, after its own global writes); the writes of every block are then visible to that
// block, which reads them through L2 (__ldcg).  `counter` counts arrivals; the last block
// resets it for the next launch.
__device__ __forceinline__ bool last_block(unsigned* counter, unsigned total = 0)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        // total: the blocks that arrive (0: every block of the grid)
        if (total == 0) total = gridDim.x * gridDim.y * gridDim.z;
        last = atomicAdd(counter, 1u) == total - 1;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Sum of v over the block (the result in thread 0; sh: 32 doubles of shared memory), a fixed
// tree: warp shuffles, then the warp sums.
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

// Programmatic dependent launch.  The kernels of a step are launched with programmatic stream
// serialisation (launch_dep): a kernel's blocks may become resident while the previous kernel
// of the stream is still finishing its last blocks, which hides the launch and ramp-up of every
// kernel boundary.  Each such kernel calls dep_begin() first, in every block, before it reads
// or writes device memory: it waits until its predecessor has completed and that kernel's
// writes are visible, and only then lets its own successor launch.  So at most two kernels of
// the stream overlap, and everything before the predecessor completed before this kernel was
// launched: no block of an older kernel can still be writing, or caching in an SM's L1 a line
// this kernel later reads.  (Letting the successor launch first allowed chains of small kernels
// to be resident at once, and a kernel two launches on read a stale L1 copy of the step state
// that the older kernel was about to overwrite.)  Launched the ordinary way, the wait is a
// no-op.
__device__ __forceinline__ void dep_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

#ifndef MITHRA_DEP_LAUNCH
#define MITHRA_DEP_LAUNCH 1
#endif

// Whether a step kernel of precision `real` is launched as a programmatic dependent on stream
// st: on the FP32-mixed path when launched directly.  Steps captured into a graph already start
// back to back, and there waiting blocks of the small kernels (phase table, Mur, power) made a
// replayed period slower; the FP64 path was slower with it in both modes.
// kernel: its bit in MITHRA_DEP_MASK, the kernels that may start early.  The emission, the push
// and the stencil each gained 1-3 us per step of the FEL run 128x128x512 (steps 5-25: 0.267 ms
// with none, 0.264-0.266 with one of them); the step tail lost 10 us (its thousands of small
// blocks, resident early, wait while the stencil's last wave runs), and the optional kernels
// (spectrum, bunch sampling, seed) are small enough to lose like it.
enum DepKernel : unsigned { kDepEmit = 1, kDepPush = 2, kDepStencil = 4, kDepTail = 8, kDepOther = 16 };
#ifndef MITHRA_DEP_MASK
#define MITHRA_DEP_MASK 7u
#endif
template <typename real>
inline bool dep_launch_on(cudaStream_t st, unsigned kernel)
{
    if (!MITHRA_DEP_LAUNCH || sizeof(real) != 4 || !(kernel & (MITHRA_DEP_MASK))) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
}

// Launch kernel k, with programmatic stream serialisation when dep is set (k calls dep_begin()
// first in every block).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(bool dep, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = dep ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Stored momentum gamma*beta.  FP64 path: a double.  FP32-mixed path: an unevaluated sum of two
// floats (hi, lo) with hi the float nearest to hi + lo, about 48 significant bits: the momentum
// accumulates the FP32 Boris increments at well beyond FP32 precision without the FP64 pipe,
// and the FP32 rotation reads hi, which is the momentum rounded to FP32.
template <typename real>
struct MomStore {
    using type = double;
};
template <>
struct MomStore<float> {
    using type = float2;
};
template <typename real>
using mom_t = typename MomStore<real>::type;

__host__ __device__ inline double mom_value(double u) { return u; }
__host__ __device__ inline double mom_value(float2 u) { return (double)u.x + (double)u.y; }
__host__ __device__ inline void mom_set(double* dst, double v) { *dst = v; }
__host__ __device__ inline void mom_set(float2* dst, double v)
{
    const float h = (float)v;
    *dst = make_float2(h, (float)(v - (double)h));
}
// (hi, lo) + d: Knuth's two-sum of hi and d, the low parts added, then renormalised by a fast
// two-sum (exact error terms under round-to-nearest; no products, so nothing is contracted).
__host__ __device__ inline float2 mom_add(float2 u, float d)
{
    const float s = u.x + d;
    const float bb = s - u.x;
    const float e = (u.x - (s - bb)) + (d - bb);
    const float t = u.y + e;
    const float h = s + t;
    return make_float2(h, t - (h - s));
}

// Particle arrays (structure of arrays).  Position = node 0 + (cell + offset) * spacing,
// offset in [0, 1).  `real` is float for the FP32-mixed path, double for FP64.
template <typename real>
struct Particles {
    int32_t *ix, *iy, *iz;
    real *fx, *fy, *fz;
    mom_t<real> *ux, *uy, *uz;
    int32_t *id;
};

template <typename real>
struct Fields4 {
    real* c[4];
};

// E and B at the nodes, interleaved per node: E_x, E_y, E_z, B_x, B_y, B_z and two unused entries,
// eight values per node (32 B in FP32, 64 B in FP64), so that the six components of a node are
// read with two (FP32) or four (FP64) 16-byte loads.
constexpr int kEBStride = 8;
template <typename real>
struct Fields6 {
    real* p;
    __host__ __device__ real& at(int c, int64_t id) const { return p[id * kEBStride + c]; }
};

// Field energy density at a node, eps0 E^2 / 2 + B^2 / (2 mu0).  From FP32 components it is formed
// in FP32 (relative error below 1e-6, against the 6e-8 of the stored values), so that a sum over
// nodes in FP64 spends one conversion and one add of the FP64 pipe per node.
__device__ __forceinline__ double node_energy(float ex, float ey, float ez, float bx, float by, float bz)
{
    constexpr double eps0 = 1.0 / (kMu0 * kC * kC);
    const float e2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    const float b2 = fmaf(bx, bx, fmaf(by, by, bz * bz));
    return (double)fmaf((float)(0.5 * eps0), e2, (float)(0.5 / kMu0) * b2);
}
__device__ __forceinline__ double node_energy(double ex, double ey, double ez, double bx, double by, double bz)
{
    constexpr double eps0 = 1.0 / (kMu0 * kC * kC);
    double e2 = 0.0, b2 = 0.0;
    e2 += ex * ex;
    b2 += bx * bx;
    e2 += ey * ey;
    b2 += by * by;
    e2 += ez * ez;
    b2 += bz * bz;
    return 0.5 * eps0 * e2 + 0.5 * b2 / kMu0;
}

// Six separate arrays of E_x .. B_z (the allocation-free energy's caller arrays).
template <typename real>
struct Fields6Soa {
    real* c[6];
};

}  // namespace mithra
