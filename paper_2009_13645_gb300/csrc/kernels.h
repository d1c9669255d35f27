// Launcher declarations shared by the translation units of libmithra.
#pragma once

#include <cuda.h>

#include "../../include/mithra.h"
#include "common.cuh"

namespace mithra {

// Number of kernels launched by this library since it was loaded (all runs, all threads).
void count_launches(int64_t n);

// Quasi-random ellipsoid bunch (lab frame, n x 6) written to device memory d_out on stream st;
// particle p takes the Halton numbers of index p + 1 + j0.  Scratch for the shot noise comes from
// alloc / free_fn (ctx).  Returns a MITHRA status.
int ellipsoid_device(const mithra_ellipsoid& e, int64_t n, uint64_t j0, double* d_out, void* (*alloc)(void*, size_t),
                     void (*free_fn)(void*, void*), void* ctx, cudaStream_t st);
// Record `msg` as the calling thread's last error (read by mithra_last_error) and return `code`.
int set_last_error(int code, const char* msg);

// Pointers of one step's potential levels: n0 = psi^{n-1}, n1 = psi^n, out = psi^{n+1}, plus the
// sources J_x, J_y, J_z, rho.
template <typename real>
struct FieldLevels {
    const real* n0[4];
    const real* n1[4];
    real* out[4];
    const real* src[4];
};

// Stencil coefficients (FP64 on the host, rounded to the storage type at launch).
struct StencilCoef {
    double a1, ax, ay, a6, w, w0, s_a, s_phi;
};

template <typename real>
cudaError_t launch_stencil(const FieldLevels<real>& L, const Geom& g, const StencilCoef& cf, int ncomp,
                           cudaStream_t st);
// TMA-staged stencil (stencil_tma.cu): tensor maps of the three ring levels and the sources,
// built once per run; null when the grid's row pitch is not a multiple of 16 bytes.
struct TmaMaps;
template <typename real>
TmaMaps* make_tma_maps(real* const pot[3][4], real* const src[4], const Geom& g);
void free_tma_maps(TmaMaps* m);
// Mur face coefficients (Sec. "First/Second Order ABCs") per normal axis a: the boundary value
//   psi_b^{n+1} = f0 (psi_b^{n-1} + psi_q^{n+1}) + f1 (psi_b^n + psi_q^n) - psi_q^{n-1}
//               + ft[a][0] S_{(a+1)%3} + ft[a][1] S_{(a+2)%3},
// q the inward neighbour of b, S_t the four level-n neighbours along axis t of b and q.
struct MurFaceCoef {
    double f0[3], f1[3], ft[3][2];
};
MurFaceCoef mur_face_coef(const Geom& g, int order);

// With `mur` (not null: the run's Mur coefficients) and FP32 storage the stencil also writes the
// Mur values of the interior nodes of the x faces (x = 0 and x = ex - 1) of every lattice it
// updates; tma_x_faces<real>() tells whether it does.  test_skip_plane >= 0 (failure tests only):
// every block leaves the copy of its plane pfirst + test_skip_plane out and its waits give up
// after 1024 polls, so the bounded-wait path runs and sets *err.
// Sources: with src_box (device, the previous step's deposit box) and *src_far == 0 (device,
// the far-move flag of this step's push), a block copies the source of a plane only where the
// tile meets the nodes [lo - src_grow, hi + 1 + src_grow] of that box; elsewhere the source is
// zero (this step's push deposited nothing there and the emission cleared the last one).
// src_box null: every source is read.
template <typename real>
cudaError_t launch_stencil_tma(const TmaMaps* maps, real* const out[4], real* const prev[4], const MurFaceCoef* mur,
                               int lev_n, int lev_m, const Geom& g, const StencilCoef& cf, int ncomp,
                               const int* src_box, const int* src_far, int src_grow, int* err, cudaStream_t st,
                               int test_skip_plane = -1);

template <typename real>
constexpr bool tma_x_faces()
{
    return sizeof(real) == 4;
}

struct StepDev;
// TF/SF planes of the seed (Sec. "Seed Field") on level n+1 of A_x and A_y: the seed potential
// at the time of level n (T0 + (step + 1) dt) is evaluated once per node of z planes 1 and 2 into
// `fbuf` (2 components x 2 planes x nx x ny, FP64), then the scattered-field plane 1 subtracts
// and the total-field plane 2 adds the update terms that cross them.
template <typename real>
cudaError_t launch_tfsf(real* const out[2], const Geom& g, const StencilCoef& cf, const SeedField& s,
                        const StepDev* sd, double T0, double* fbuf, cudaStream_t st);

// Mur values of the x-face nodes of z planes 1 and 2 of A_x and A_y again, after the TF/SF
// correction changed their inward neighbours (the FP32 TMA stencil wrote them before it).
template <typename real>
cudaError_t launch_mur_tfsf_xfaces(const FieldLevels<real>& L, const Geom& g, int order, cudaStream_t st);

// Per-step values derived on the device from the step counter, so that a captured sequence of
// steps replays without host-side parameters.  Every kernel of step n reads it; the last block of
// the step's last kernel (the step tail) advances it to step n + 1, and the run's creation sets
// it to step 0.
struct StepDev {
    int64_t n;        // the step being computed
    int64_t next;     // the counter: the step after it
    double t_half;    // rest-frame time of r^{n+1/2}: T0 + (n + 1/2) dt
    double Z0;        // lab coordinate zeta of node plane 0 at t_half: gamma0 (z0 + beta0 c t_half)
    int slot;         // power-plane ring slot of step n (the slot of step n - M is the same)
    int full;         // the ring holds step n - M
    int emit;         // the power window is complete
    double cn, sn;    // cos, sin of w t_n
    double co, so;    // cos, sin of w t_{n-M}
};
struct StepConst {
    double T0, dt, g0, b0, z0, omega_h;
    int M;
};
// The StepDev of step n.
__device__ __forceinline__ StepDev step_state(int64_t n, const StepConst& c)
{
    StepDev v;
    v.n = n;
    v.next = n + 1;
    v.t_half = c.T0 + ((double)n + 0.5) * c.dt;
    v.Z0 = c.g0 * (c.z0 + c.b0 * kC * v.t_half);
    v.slot = (int)(n % c.M);
    v.full = n >= c.M ? 1 : 0;
    v.emit = n + 1 >= c.M ? 1 : 0;
    sincos(c.omega_h * ((double)n + 0.5) * c.dt, &v.sn, &v.cn);
    sincos(c.omega_h * ((double)(n - c.M) + 0.5) * c.dt, &v.so, &v.co);
    return v;
}

// The static undulator's phase tables of one node plane iz whose lab coordinate is zn (Sec. "Field
// Initialization": the planar field's phase k_u zeta per node plane, evaluated once per step in
// FP64).
// FP32-mixed path, two float4 per node plane and planar field: the sin and cos of the plane's
// phase k_u u times the FP64 rest-frame amplitudes (gamma0 beta0 c B, gamma0 B, B), and the
// distances k_u u, k_u (u - L_u) to both ends of the undulator; FP64 throughout, rounded once.
// For an array (ta != null) u is counted from the entrance of the plane's module i (the module
// whose entrance lies at or before the plane, as in the direct evaluation; before the first
// module, from the first entrance), B is that module's peak field, and ta holds per plane {B_i,
// B_{i+1} (0 after the last module), 1 for the last module, 0}.
__device__ __forceinline__ void phase_entry32(const ExtField& f, double zn, int iz, float4* t0, float4* t1, float4* ta)
{
    double Bp = f.B0, org = 0.0;
    if (ta) {
        const double P = f.Lu + f.gap;
        int i = (int)floor(zn / P);
        i = i < -1 ? -1 : (i > f.nmod - 1 ? f.nmod - 1 : i);
        if (i >= 0 && zn - i * P < 0.0) --i;
        if (i < f.nmod - 1 && zn - (i + 1) * P >= 0.0) ++i;
        const int im = i < 0 ? 0 : i;
        Bp = f.B0 + im * f.dB0;
        org = im * P;
        const bool last = i == f.nmod - 1;
        ta[iz] = make_float4((float)Bp, (float)((i >= 0 && !last) ? Bp + f.dB0 : 0.0), last ? 1.f : 0.f, 0.f);
    }
    const double eB = f.g0 * f.b0 * kC * Bp, bB = f.g0 * Bp;
    for (int j = 0; j < (t1 ? 2 : 1); ++j) {
        const double ph = f.ku * (zn - (j ? f.qlam : org));
        double s, c;
        sincos(ph, &s, &c);
        float4* t = (j ? t1 : t0) + 2 * iz;
        t[0] = make_float4((float)(eB * s), (float)(eB * c), (float)(bB * s), (float)(bB * c));
        t[1] = make_float4((float)(Bp * s), (float)(Bp * c), (float)ph, (float)(ph - f.ku * f.Lu));
    }
}
// FP64 path: sin and cos of k_u zn (and of the helical second field's k_u (zn - lambda_u / 4)).
__device__ __forceinline__ void phase_entry64(const ExtField& f, double zn, int iz, double2* t0, double2* t1)
{
    double s, c;
    sincos(f.ku * zn, &s, &c);
    t0[iz] = make_double2(s, c);
    if (t1) {
        sincos(f.ku * (zn - f.qlam), &s, &c);
        t1[iz] = make_double2(s, c);
    }
}
// The phase tables a step's push reads (null pointers: none), for the node planes 0..nz-1 at
// lab offset Z0 + kz iz.
struct PhaseTables {
    ExtField ef;
    double kz;
    int nz;
    float4 *t32[2], *ta32;
    double2* t64[2];
};
__device__ __forceinline__ void phase_tables_entry(const PhaseTables& pt, double Z0, int iz)
{
    const double zn = fma(pt.kz, (double)iz, Z0);
    if (pt.t32[0]) phase_entry32(pt.ef, zn, iz, pt.t32[0], pt.t32[1], pt.ta32);
    if (pt.t64[0]) phase_entry64(pt.ef, zn, iz, pt.t64[0], pt.t64[1]);
}

// The radiated power (Sec. FEL-OUTPUT, radiation-power): one step of the running DFT of the
// transverse fields on the power plane kp.
struct PowerStep {
    int kp;                 // plane index
    double* ring;           // M x 4 x plane samples
    double* acc;            // 8 x plane accumulators (re, im of Ex, Ey, Bx, By)
    int64_t onaxis_id;
    double* onaxis_series;  // on-axis E_x of step n goes to entry n
    double scale;           // lab factor x (2 / M)^2 x dx dy / (2 mu0)
    double* series;         // the power of step n goes to series[n] once the window is complete
};
// Plane point pl of step sd: it adds its new sample of E_x, E_y, B_x, B_y times exp(-j w t_n) to
// its accumulators and, once the window is full, subtracts the sample of step n - M kept in the
// ring (the DFT over the last M steps, updated instead of recomputed); an interior point returns
// Re(Ex By* - Ey Bx*) of its accumulators, its share of the plane's power.  The on-axis E_x of the
// step is recorded by its point.
template <typename real>
__device__ __forceinline__ double power_point(const Fields6<real>& eb, const Geom& g, const PowerStep& ps,
                                              const StepDev& sd, int64_t pl)
{
    const int64_t plane = (int64_t)g.nx * g.ny;
    const int64_t id = (int64_t)ps.kp * g.sz + pl;
    if (id == ps.onaxis_id) ps.onaxis_series[sd.n] = (double)eb.at(0, id);
    const double x[4] = {(double)eb.at(0, id), (double)eb.at(1, id), (double)eb.at(3, id), (double)eb.at(4, id)};
    double* r = ps.ring + (int64_t)sd.slot * 4 * plane + pl;
    double re[4], im[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double a = ps.acc[(2 * q) * plane + pl], b = ps.acc[(2 * q + 1) * plane + pl];
        a += x[q] * sd.cn;
        b -= x[q] * sd.sn;
        if (sd.full) {
            const double o = r[q * plane];
            a -= o * sd.co;
            b += o * sd.so;
        }
        ps.acc[(2 * q) * plane + pl] = a;
        ps.acc[(2 * q + 1) * plane + pl] = b;
        r[q * plane] = x[q];
        re[q] = a;
        im[q] = b;
    }
    const int i = (int)(pl % g.nx), j = (int)(pl / g.nx);
    if (sd.emit && i >= 1 && i <= g.nx - 2 && j >= 1 && j <= g.ny - 2)
        return (re[0] * re[3] + im[0] * im[3]) - (re[1] * re[2] + im[1] * im[2]);
    return 0.0;
}

// The end of a step (the step tail): besides the Mur edges and corners, the radiated power's
// running DFT of the step (eb: the step's E/B; series[n] once the window is complete), the phase
// tables of the next step, and the step state's advance.
struct StepTail {
    const void* eb;         // the step's E/B (Fields6 of the run's precision)
    PowerStep power;
    double* partial;        // power block partials (at most npartial)
    int npartial;
    PhaseTables phase;      // the tables of step n + 1
    StepDev* sd;            // the step state; sd[1]: the next one, written by the phase-table blocks
    StepConst sc;
    const int* box_rec;     // the push's per-block bounds (nrec records of six ints)
    int64_t nrec;
    int* box_out;           // the deposit box they reduce into (deposit_box_ints, reset to empty)
};

// Mur boundary values of level n+1 and the step tail, in one launch: the faces (x_faces_done: the
// TMA stencil of this step has written the x faces), the edges (their face neighbours evaluated
// in place), the tail's power, phase-table and deposit-box blocks, and in the last of the edge,
// power, table and box blocks to finish the corners, the power's sum and the step state's
// advance (`counter` is a zeroed device word that the launch leaves zeroed).
template <typename real>
cudaError_t launch_mur(const FieldLevels<real>& L, const Geom& g, int order, int ncomp, bool x_faces_done,
                       unsigned* counter, const StepTail& tail, cudaStream_t st);
// At a run's creation: the step state of step 0 and its phase tables.
cudaError_t launch_step_init(StepDev* sd, const StepConst& sc, const PhaseTables& pt, cudaStream_t st);
// Tensor maps of the seven arrays one E/B emission reads (A_x^n, A_x^{n+1}, A_y^n, A_y^{n+1},
// A_z^n, A_z^{n+1}, phi^n), each with a box of kEmitBoxW x kEmitBoxH x 1 (the emission tile
// plus a one-node halo, padded to whole 16-byte rows).
constexpr int kEmitBoxW = 36, kEmitBoxH = 10;
struct EmitMaps {
    CUtensorMap m[7];
};
// The emission maps of ring levels lev_n (A^n, phi^n) and lev_n1 (A^{n+1}); false without TMA.
bool emit_maps(const TmaMaps* maps, int lev_n, int lev_n1, EmitMaps* out);

// Region of one E/B emission: box == null emits the whole interior and clears nothing.
// Planes per emission block; the deposit boxes also hold, per such z chunk c of node planes
// [1 + c kEmitKZ, (c + 1) kEmitKZ], the xy box of the cells whose gather or deposit reaches it.
constexpr int kEmitKZ = 8;
__host__ __device__ inline int emit_chunks(int nz) { return (nz - 2 + kEmitKZ - 1) / kEmitKZ; }
// Ints of one deposit box: [lo_x, lo_y, lo_z, hi_x, hi_y, hi_z] of the cells, then per z chunk
// [lo_x, lo_y, hi_x, hi_y].
inline int deposit_box_ints(int nz) { return 6 + 4 * emit_chunks(nz); }
// The deposit box buffer: deposit_box_ints ints, then the push's far-move flag (PushConst::far).
inline int deposit_box_words(int nz) { return deposit_box_ints(nz) + 1; }
struct EmitBox {
    const int* box;      // device: the deposit box of the last push (deposit_box_ints)
    int* box_reset;      // device: box the next push reduces into, reset to empty (and its far flag to 0)
                         // by the emission
    int kp;              // plane always emitted in full (< 0: none)
    bool clear;          // clear the sources inside the box
    const EmitMaps* maps = nullptr;   // TMA loads (null: per-element asynchronous copies)
    int* err = nullptr;               // set when a bounded wait of the TMA loads expired
};
template <typename real>
cudaError_t launch_emit(const FieldLevels<real>& L, const Fields6<real>& eb, const Geom& g, const EmitBox& bx,
                        cudaStream_t st);



// Particles.
struct PushConst {
    const StepDev* sd;    // the step's time (t_half) and lab offset of the node planes (Z0)
    double qJ[3];         // q / (D_m D_n dt): current density per unit displacement (cells) along each axis
    double qrho;          // q / (dx dy dz)
    double cdtb[3];       // c dt_b / D_l
    // static undulator: per-step table of (sin, cos) of k_u (zeta - offset) at every z node plane
    // (one table per planar field; null: evaluate directly)
    const double2* ptab[2];
    // FP32-mixed path: per node plane and planar field two float4, {eB0 sin, eB0 cos, bB0 sin,
    // bB0 cos} and {B0 sin, B0 cos, k_u u, k_u (u - L_u)} of the plane's undulator coordinate u,
    // evaluated in FP64 and rounded to FP32
    const float4* ptab32[2];
    // undulator array, FP32-mixed path: per node plane {B_i, B_{i+1}, last module, 0} (null: no
    // array)
    const float4* ptab32a;
    double kz;            // gamma0 dz: zeta per cell along z
    double zstep;         // gamma0 beta0 c dt_b: zeta per sub-step
    float kdz, kzs;       // k_u kz and k_u zstep in FP32: the sub-cell rotation per offset and sub-step
    // FP32-mixed path: the run's constants rounded once on the host
    float x0f, y0f, dxf, dyf, dtbf, qrhof, kuf, cpolf, spolf;
    float qJf[3], cdtbf[3];
    // rest-frame amplitudes of the static undulator field, gamma0 beta0 c B0, gamma0 B0 and B0,
    // evaluated in FP64 and rounded to FP32 (the fringe of the FP32-mixed path)
    float eB0f, bB0f, B0f;
    // undulator array, FP32-mixed path: k_u g, pi / (k_u g) (the window's argument per k_u dz),
    // gamma0 beta0 c and gamma0
    float kugf, pwinf, egbf, gbf;
    // FP32-mixed deposit tile: fixed-point scale per source grid (2^30 / (128 |qJ_l|), 2^30 /
    // (128 |q|)), its inverse, and the charges in tile units (qJ_l and q times the scale)
    float tscale[4], tunit[4];
    float qJt[3], qrhot;
    // optical undulator, FP32-mixed path: the transverse rest-frame amplitudes gamma0 (1 + beta0) E0
    // and gamma0 (1 + beta0) E0 / c (the Lorentz transform of a wave travelling along -z, evaluated in
    // FP64), E0, E0 / c, the waist, 1 / z_R, z_R and k_L, rounded to FP32
    float ltE, ltB, E0f, E0cf, w0f, izrf, zrf, kLf;
    // set to 1 when a deposit of this step may fall outside the previous step's deposit box grown
    // by the sub-step count: a move longer than one cell on an axis, or a deposit by a particle
    // that started the step outside the active cells (the stencil then reads every source)
    int* far;
};

// box_rec: per block of 128 particles, the six bounds [lo_x, lo_y, lo_z, hi_x, hi_y, hi_z] of the
// cells its particles deposited into or end in (the end cells of the particles in the active
// cells or the one-cell margin around them; empty bounds: none); the step tail reduces them
// into the deposit box the next emission reads.
template <typename real>
cudaError_t launch_push(const Particles<real>& P, int64_t np, const Geom& g, const ExtField& ef,
                        const Fields6<real>& eb, const Fields4<real>& src, const PushConst& pc, int* box_rec,
                        cudaStream_t st);
// Blocks of 128 particles the push launches.
inline int64_t push_blocks(int64_t np) { return (np + 127) / 128; }

// *flag |= 1 when one of the n values at a is not finite (flag: a device word).
cudaError_t launch_finite_check(const double* a, int64_t n, int* flag, cudaStream_t st);

template <typename real>
cudaError_t launch_boost(const double* lab6, int64_t np, const Particles<real>& P, const Geom& g,
                         const ExtField& ef, double z_ref, cudaStream_t st);

template <typename real>
cudaError_t launch_set_rest(const double* rest6, int64_t np, const Particles<real>& P, const Geom& g,
                            cudaStream_t st);
template <typename real>
cudaError_t launch_get_rest(const Particles<real>& P, int64_t np, const Geom& g, double* rest6,
                            cudaStream_t st);

// Counting sort by cell.
struct SortScratch {
    int32_t* key;        // per particle
    int32_t* count;      // nbins + 1
    int32_t* offset;     // nbins + 1 (exclusive scan)
    int32_t* perm;       // per particle: destination slot
    int32_t* blocksum;   // scan partials
    int64_t nbins;
};
template <typename real>
cudaError_t launch_sort(Particles<real>& P, Particles<real>& tmp, int64_t np, const Geom& g,
                        const SortScratch& s, cudaStream_t st);
size_t sort_scan_partials(int64_t nbins);

// Diagnostics.
template <typename real>
cudaError_t launch_energy(const Fields6<real>& eb, const Geom& g, double* partial, int npartial, double* out,
                          cudaStream_t st);

// Radiated-power spectrum (Sec. FEL-OUTPUT, radiation-power, normalised-frequency sweep): for
// every frequency k the running DFT of the power plane over its own window M[k] of steps.  The
// plane samples of the last Mh >= max M[k] steps are shared by all frequencies.
struct SpecStep {
    int kp;                 // plane index
    int nf, Mh;             // frequencies, ring depth
    const StepDev* sd;
    double dt;
    const double* omega;    // device, nf rest-frame angular frequencies
    const int* M;           // device, nf windows
    const double* scale;    // device, nf: lab factor x (2 / M)^2 x dx dy / (2 mu0)
    double* ring;           // Mh x 4 x plane samples (Ex, Ey, Bx, By)
    double* acc;            // nf x 8 x plane accumulators
};
// The powers of step n go to series[n * nf + k] (zero until a frequency's window is complete).
template <typename real>
cudaError_t launch_spectrum_step(const Fields6<real>& eb, const Geom& g, const SpecStep& s, double* partial,
                                 int npartial, double* series, cudaStream_t st);

// Bunch sampling (Sec. BUNCH, bunch-sampling): after the push of every step n with n % every == 0
// the row n / every of `series` (15 values) receives the rest-frame time of the positions
// T0 + (n + 3/2) dt, the means of x, y, z (rest frame) and gamma*beta_x,y,z, their rms spreads,
// and the mean and rms spread of the lab Lorentz factor gamma0 (gamma + beta0 u_z).  Sums of
// FP64 values shifted by `shift` (the mesh centre, zero momentum, the bunch's lab gamma) keep the
// spreads free of cancellation.
struct BunchSample {
    const StepDev* sd;
    int every;
    double shift[7];
    double g0, b0, T0, dt;
};
template <typename real>
cudaError_t launch_bunch_sample(const Particles<real>& P, int64_t np, const Geom& g, const BunchSample& b,
                                double* partial, int npartial, double* series, cudaStream_t st);
// Bunching factor |<exp(i k_b z)>| and its real and imaginary parts into out3.  tab (nz entries,
// may be null): scratch for the FP32 path's table of the node planes' phases.
template <typename real>
cudaError_t launch_bunching(const Particles<real>& P, int64_t np, const Geom& g, double kb, double* partial,
                            int npartial, double* out3, float2* tab, cudaStream_t st);

}  // namespace mithra
