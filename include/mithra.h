/*
 * mithra.h - C ABI of the GB300 implementation of the rest-frame FDTD/PIC
 * time step of MITHRA 2.0 (A. Fallahi, arXiv:2009.13645).
 *
 * One run = one free-electron-laser interaction solved in the frame moving
 * with the bunch (manual Ch. "Methodology"): an explicit NSFD/FD update of the
 * potential wave equations for A and phi (Sec. "FDTD for Wave Equation",
 * "FDTD for Scalar Potential") with Mur absorbing boundaries (Sec. "Boundary
 * Truncation"), coupled to a particle-in-cell loop (Sec. "Particle In Cell":
 * field evaluation, linear gather, Boris push in the Lorentz-transformed
 * undulator or laser field, Umeda zigzag current and charge deposition).
 *
 * Conventions shared by every entry point:
 *  - Return value: MITHRA_OK (0) or a negative MITHRA_E* code.  The library
 *    never aborts and never prints; mithra_last_error() returns a
 *    thread-local message describing the last failure on the calling thread.
 *  - Units: SI.  Input structs are in the LABORATORY frame, as the manual's
 *    job files are (Ch. "User Interface": all parameters are lab-frame);
 *    the library boosts them to the rest frame itself.
 *  - Ownership: input structs and arrays are copied during the call; the
 *    caller keeps them.  Output buffers are caller-owned host memory.  Device
 *    memory belongs to the run handle and is released by mithra_destroy().
 *  - Device memory comes from the allocator installed with
 *    mithra_set_allocator() (cudaMalloc/cudaFree when none is installed).
 *  - All work of a run is enqueued on one CUDA stream (mithra_set_stream(),
 *    else a non-blocking stream the library creates); mithra_step() returns
 *    once the work is enqueued.
 *  - Thread safety: calls on different handles may come from different
 *    threads; calls on one handle must be serialised by the caller.
 */
#ifndef MITHRA_H
#define MITHRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MITHRA_OK 0
#define MITHRA_EINVAL (-1)     /* bad shape, non-finite input, unknown option */
#define MITHRA_ENOMEM (-2)     /* device allocation failed / over the HBM budget */
#define MITHRA_ERANGE (-3)     /* caller buffer too small */
#define MITHRA_ETIMEDOUT (-4)  /* a bounded device-side wait expired */
#define MITHRA_EDIVERGED (-5)  /* non-finite field energy */
#define MITHRA_ENOTFOUND (-6)  /* unknown ticket */
#define MITHRA_EAGAIN (-7)     /* request queue full, try again */
#define MITHRA_ECUDA (-8)      /* a CUDA runtime call failed */

typedef struct mithra_run *mithra_t;

/* Mesh and solver options (manual Sec. MESH).  Lengths in the lab frame. */
typedef struct mithra_grid {
    int32_t nx, ny, nz;        /* nodes per axis, each >= 6 */
    double dx, dy, dz;         /* lab resolution; the rest frame uses gamma0*dz (Sec. "Lorentz Transformation") */
    double cx, cy, cz;         /* mesh centre relative to the bunch reference point (lab) */
    int32_t solver;            /* 0 NSFD (Eq. updateEquation), 1 FD (central differences) */
    double courant;            /* FD only: dt = courant x CFL bound (Eq. CFLcondition); NSFD forces c dt = dz */
    int32_t mur_order;         /* 1 or 2 (Sec. "First/Second Order ABCs") */
    int32_t space_charge;      /* 0: phi == 0, no charge deposition (Sec. "FDTD for Scalar Potential") */
    int32_t precision;         /* 0 FP64 everywhere; 1 FP32 fields/offsets, float-pair momentum, FP64 external field, diagnostics */
    int32_t substeps;          /* N in dt_b = dt/N (Sec. "Update Algorithm"); >= 1 */
    double power_plane_dist;   /* lab distance of the radiated-power plane ahead of the bunch (Sec. FEL-OUTPUT) */
    double norm_freq;          /* normalised frequency h of the radiated-power diagnostic */
    int32_t sort_every;        /* counting sort by cell every S steps; 0 = default (20), < 0 = never */
    /* radiated-power spectrum (Sec. FEL-OUTPUT, radiation-power: minimum-normalized-frequency,
       maximum-normalized-frequency, number-of-frequency-points): nf_points frequencies
       h_k = nf_min + k (nf_max - nf_min) / (nf_points - 1) (h_0 = nf_min when nf_points = 1);
       0 .. 256 points, 0 = no spectrum; each h_k > 0 */
    double nf_min, nf_max;
    int32_t nf_points;
    /* bunch sampling (Sec. BUNCH, bunch-sampling) every bunch_every steps; 0 = off */
    int32_t bunch_every;
    /* optimize-bunch-position (Sec. MESH), static undulators (kinds 0, 1, 4) only, ignored
       otherwise: 1 moves the mesh and the power plane along z by the rest-frame drift of the bunch
       reference (on axis, Lorentz factor bunch.gamma, relative velocity
       v = (beta - beta0) / (1 - beta beta0)) until the undulator entrance reaches it, so that the
       bunch sits at the placed position inside the undulator; 0 keeps the mesh where it is placed */
    int32_t optimize_position;
} mithra_grid;

/* Undulator (manual Sec. UNDULATOR, Sec. "Field Initialization"). */
typedef struct mithra_undulator {
    int32_t kind;              /* -1 none, 0 planar static, 1 helical static (two planar, 90 deg, lambda/4 apart),
                                  2 optical plane wave, 3 optical Gaussian beam (counter-propagating, -z),
                                  4 static undulator array (Sec. "Static Undulator Array Field") */
    double K;                  /* undulator parameter K, or strength a0 of an optical undulator */
    double lambda;             /* undulator period, or laser wavelength; kind -1: rest-frame diagnostic wavelength */
    double n_periods;          /* static: undulator length in periods */
    double pol_deg;            /* polarisation angle from the x axis, degrees */
    double waist;              /* Gaussian beam waist w0 */
    double pulse_fwhm;         /* c * tau, intensity FWHM (Eq. signalTypes) */
    int32_t signal;            /* 0 modulated Gaussian, 1 flat-top (Gaussian rise, then constant) */
    double dist_to_bunch_head; /* lab distance from the bunch head to the undulator entrance / pulse */
    /* kind 4 only (Sec. UNDULATOR, static-undulator-array): n_modules planar modules of n_periods
       periods each, `gap` (lab length, >= 0) between one module's end and the next entrance,
       undulator parameter K_i = K + i * taper of module i (K of the first module fixes the rest
       frame).  Inside a gap both neighbouring fringes (Eq. fringingField) are damped by the
       window f(dz, gap) of Eq. fringingFieldGap, dz the distance to that module's end. */
    double gap;
    int32_t n_modules;         /* 1 .. 100000 */
    double taper;
} mithra_undulator;

/* The bunch (Sec. BUNCH): either macro-particles the caller gives (bunch type "file"), or, when
   lab_particles is NULL, an ellipsoid bunch generated on the device from the parameters below
   (bunch-initialization of type ellipsoid; Sec. "Electron Bunch Generation"), loaded
   quasi-randomly as mithra_ellipsoid_bunch does with
   sig = {sig_x, sig_y, sig_z}, sig_u = {eps_n_x / sig_x, eps_n_y / sig_y, gamma rel_espread}
   (a beam at its waist: the rms normalised momentum is the normalised emittance over the rms size;
   the rms energy spread sets the rms of gamma*beta_z) and the Halton index of particle p shifted by
   `seed` (index p + 1 + seed). */
typedef struct mithra_bunch {
    int64_t n;                 /* number of macro-particles (>= 0) */
    double charge_e;           /* bunch charge in electrons (> 0 when n > 0) */
    double gamma;              /* mean Lorentz factor; with the undulator it fixes the rest frame */
    double sig_z;              /* lab rms length (uniform profile: half length); the bunch head is taken
                                  3 sig_z ahead of the reference point */
    const double *lab_particles; /* host, n x 6 row-major: x, y, z (m, relative to the bunch reference point),
                                    gamma*beta_x, gamma*beta_y, gamma*beta_z; lab frame at t' = 0.
                                    NULL: generate the bunch from the fields below */
    int32_t uniform;           /* generated: 0 Gaussian current profile, 1 uniform over [-sig_z, sig_z] */
    double rel_espread;        /* generated: rms relative energy spread (>= 0) */
    double sig_x, sig_y;       /* generated: rms transverse size (>= 0) */
    double eps_n_x, eps_n_y;   /* generated: normalised emittance (>= 0; 0 when the size is 0) */
    double cse_sigma;          /* generated, uniform profile: rms of the Gaussian edges (<= 0: none) */
    double lambda_r;           /* generated: lab wavelength of the bunching and of the shot-noise slices;
                                  <= 0: the run's resonance seen in the lab, 2 pi / (k* gamma0 (1 + beta0)) */
    double bunching, bunching_phase; /* generated: bunching factor at lambda_r and its phase (rad) */
    int32_t shot_noise;        /* generated: 1 adds the shot noise of charge_e electrons per slice lambda_r */
    uint64_t seed;             /* generated: Halton index offset (n + seed < 2^32) */
} mithra_bunch;

/* Seed injected through total-field / scattered-field planes (Sec. "Seed Field"; Sec. FIELD,
   field-initialization): a beam propagating along +z, given in the laboratory frame. */
typedef struct mithra_seed {
    int32_t type;              /* -1 none, 0 plane wave, 1 Gaussian beam (paraxial) */
    double a0;                 /* strength a0 = e A0 / (m_e c) (Sec. FIELD, strength-parameter) */
    double lambda;             /* wavelength (> 0) */
    double pol_deg;            /* polarisation angle from the x axis, degrees */
    double waist;              /* Gaussian beam waist w0 (> 0 for type 1) */
    double focus;              /* lab position of the reference point / focus, measured like the
                                  undulator: from the (first) undulator entrance */
    double offset;             /* c t0: the pulse centre passes the reference point at lab time t0 */
    double pulse_fwhm;         /* c tau, intensity FWHM (Eq. signalTypes, modulated Gaussian); <= 0: continuous */
    double cep_deg;            /* carrier envelope phase, degrees */
} mithra_seed;

/* An ellipsoid bunch loaded quasi-randomly (Sec. BUNCH, bunch-initialization of type ellipsoid;
   Sec. "Electron Bunch Generation"). */
typedef struct mithra_ellipsoid {
    int32_t uniform;           /* 0 Gaussian current profile (rms sig[2]), 1 uniform over [-sig[2], sig[2]] */
    double gamma;              /* mean Lorentz factor; the mean momentum points along +z */
    double sig[3];             /* sigma-position: rms x, y (and z for a Gaussian profile), lab, m */
    double sig_u[3];           /* sigma-momentum: rms gamma*beta_x, gamma*beta_y, gamma*beta_z */
    double cse_sigma;          /* uniform profile: rms width of the Gaussian edges (<= 0: none) */
    double lambda_r;           /* lab wavelength of the bunching and of the shot-noise slices */
    double bunching;           /* bunching factor at lambda_r (0: none) */
    double bunching_phase;     /* its phase, rad */
    int32_t shot_noise;        /* 1: shot noise per slice of length lambda_r */
    double charge_e;           /* electrons in the bunch (shot-noise amplitude) */
} mithra_ellipsoid;

/* Fill out6 (host, n x 6, caller-owned: x, y, z relative to the bunch centre, gamma*beta_x,y,z;
   lab frame) with a quasi-random ellipsoid bunch, computed on the current device: particle p
   takes the Halton numbers of index p + 1 (one minus the radical inverse of the index) in the
   prime bases 2, 3 (x, y by Eq. gaussian2D), 5, 7 (transverse momenta), 11, 13 (z by Eq.
   uniform1D or gaussian1D), 17, 19 (longitudinal momentum spread).  A uniform profile with
   cse_sigma > 0 gives n L / (L + sqrt(2 pi) cse_sigma) particles to the flat part (L = 2 sig[2])
   and the rest to a Gaussian of that rms and the same peak line density whose lower half is moved
   to the tail and upper half to the head, against coherent emission from the profile's ends.
   Bunching moves z by -(2 b / k) sin(k z + phase), k = 2 pi / lambda_r; shot noise does the same
   per slice of length lambda_r with amplitude sqrt(-2 ln x_s) / sqrt(N_e,s) (Eq.
   negativeExponential; N_e,s the slice's share of charge_e) and phase 2 pi y_s, x_s and y_s the
   Halton numbers of the slice in bases 23 and 29.  Work is enqueued on `stream` (a cudaStream_t,
   NULL: legacy default stream) and the call returns when out6 is filled.  Device scratch (48 B
   per particle) comes from the installed allocator.  Errors: EINVAL, ENOMEM, ECUDA. */
int mithra_ellipsoid_bunch(const mithra_ellipsoid *e, int64_t n, double *out6, void *stream);

/* Install the device allocator used by every later mithra_create (process-wide).
   alloc(ctx, bytes) returns a device pointer or NULL; free(ctx, ptr).  Pass NULLs to restore
   cudaMalloc/cudaFree.  Runs created earlier keep the allocator they were created with.  Any
   alignment is accepted: the library asks for 256 bytes more than it needs and aligns its
   arrays to 256 bytes itself. */
typedef void *(*mithra_alloc_fn)(void *ctx, size_t bytes);
typedef void (*mithra_free_fn)(void *ctx, void *ptr);
int mithra_set_allocator(mithra_alloc_fn alloc, mithra_free_fn free_fn, void *ctx);

/* Create a run on the current CUDA device: validate and adjust the mesh as the manual's
   checks do (Sec. MESH: dx, dy scaled so sqrt((dz/dx)^2+(dz/dy)^2) = 0.99 when NSFD is
   unstable, dt = dz/c for NSFD), fix the rest frame gamma0 (Sec. "Lorentz Transformation"),
   allocate the fields and particles on the device, boost the particles
   (Eqs. LorentzTrasnformParticles, LorentzTransformDeltaR) and sort them by cell.
   dt_lab > 0 is accepted for FD only (lab field time step); <= 0 picks it automatically.
   Errors: EINVAL (sizes, non-finite values, kinds), ENOMEM, ECUDA. */
int mithra_create(const mithra_grid *grid, double dt_lab, const mithra_undulator *und,
                  const mithra_bunch *bunch, mithra_t *out);

/* Inject `seed` (copied) through the TF/SF planes of the run: node plane 1 of the z axis is the
   scattered-field plane and plane 2 the total-field plane of the transverse vector potential
   A_x, A_y.  After every potential update the update terms that cross the two planes are
   corrected by the seed's lab-frame transverse vector potential (unchanged by the boost) at
   the lattice points and the time of the level the update read: the scattered-field plane
   subtracts and the total-field plane adds them.  The seed's longitudinal potential
   (order 1/(k w0) of a paraxial beam) is not injected.  Call before the first step; a type of
   -1 removes the seed.  Errors: EINVAL (after the first step, non-finite or out-of-range
   values). */
int mithra_set_seed(mithra_t run, const mithra_seed *seed);

/* Use `stream` (a cudaStream_t) for all later work of the run. */
int mithra_set_stream(mithra_t run, void *stream);

/* Enqueue nsteps field steps (>= 0).  One step: E and B at nodes (Sec. "Field Evaluation"),
   external field + gather + Boris + zigzag/CIC deposition (Sec. "Update Algorithm",
   "Current Deposition"), potential update (Eq. updateEquation) and Mur boundaries, the
   radiated-power sample; a counting sort by cell every sort_every steps.
   Every L = lcm(6, 2 sort_every) steps (L <= 480) the run's state returns to the same buffers, so
   a whole block of L steps starting at a multiple of L (after the first) is captured once into a
   CUDA graph and replayed; the results are those of launching the steps one by one.  Capture
   needs a created stream and is skipped while profiling or with MITHRA_NO_GRAPHS=1 in the
   environment at create time.  Errors: EINVAL, ENOMEM (series growth), ECUDA. */
int mithra_step(mithra_t run, int64_t nsteps);

/* Wait for the run's stream; returns EDIVERGED if the last field energy is not finite. */
int mithra_sync(mithra_t run);

/* Field indices for mithra_fields / mithra_set_field. */
#define MITHRA_AX 0
#define MITHRA_AY 1
#define MITHRA_AZ 2
#define MITHRA_PHI 3
#define MITHRA_JX 4
#define MITHRA_JY 5
#define MITHRA_JZ 6
#define MITHRA_RHO 7
#define MITHRA_EX 8
#define MITHRA_EY 9
#define MITHRA_EZ 10
#define MITHRA_BX 11
#define MITHRA_BY 12
#define MITHRA_BZ 13

/* Copy one field (nx*ny*nz values, x fastest) to host FP64 memory.  For potentials `level`
   0 is step n and 1 is step n+1 of the next step's input (A at k dt, phi at (k+1/2) dt);
   A_x[i] sits at (i+1/2) dx, A_y at (j+1/2) dy, A_z at (k+1/2) dz; J likewise; phi, rho,
   E and B at nodes.  Synchronises the stream.  ERANGE if cap < nx*ny*nz. */
int mithra_fields(mithra_t run, int which, int level, double *host_out, size_t cap);

/* Overwrite one potential level (which 0..3, level 0..1) from host FP64 data. */
int mithra_set_field(mithra_t run, int which, int level, const double *host_in, size_t n);

/* Copy the particles (rest frame, n x 6: x, y, z, gamma*beta_x,y,z) in their input order. */
int mithra_particles(mithra_t run, double *host_out6, size_t cap_rows);

/* Replace the particles with rest-frame values (n x 6, input order). */
int mithra_set_particles(mithra_t run, const double *rest6, size_t rows);

/* Radiated power series, one value per step taken: lab-frame power (W) through the plane
   power_plane_dist ahead of the bunch at normalised frequency h, and its lab time (s).
   Power = cycle-averaged Poynting flux of the DFT over the last M = round(2 pi/(h w* dt))
   steps, times gamma0^2 (1+beta0)^2 (Sec. FEL-OUTPUT "radiation-power").
   n_out receives the series length; ERANGE if cap is smaller. */
int mithra_radiated_power(mithra_t run, double *p_lab, double *t_lab, size_t cap, size_t *n_out);

/* Radiated-power spectrum (Sec. FEL-OUTPUT, radiation-power, the normalised-frequency sweep of
   mithra_grid.nf_min .. nf_max): for every step n and frequency k, p_lab[n * nf_points + k] is the
   power of mithra_radiated_power evaluated at h_k with its own window
   M_k = round(2 pi / (h_k w* dt)) (zero until that window is complete).  h_out (nullable,
   nf_points values) receives the frequencies.  n_steps receives the number of steps; ERANGE if
   cap_values < n_steps * nf_points; EINVAL if the run has no spectrum. */
int mithra_power_spectrum(mithra_t run, double *h_out, double *p_lab, size_t cap_values, size_t *n_steps);

/* Bunch samples (Sec. BUNCH, bunch-sampling), 15 values per row, one row after the push of every
   step n with n % bunch_every == 0: the rest-frame time of the positions T0 + (n + 3/2) dt (s),
   the means of x, y, z (rest frame, m) and of gamma*beta_x, gamma*beta_y, gamma*beta_z, the rms
   spreads (population) of the same six, and the mean and rms spread of the lab Lorentz factor
   gamma0 (gamma + beta0 gamma*beta_z).  n_rows receives the number of rows; ERANGE if cap_rows is
   smaller; EINVAL if bunch sampling is off. */
int mithra_bunch_series(mithra_t run, double *out15, size_t cap_rows, size_t *n_rows);

/* On-axis E_x at the power plane, one value per step (rest frame, V/m). */
int mithra_onaxis_field(mithra_t run, double *ex, size_t cap, size_t *n_out);

/* Field energy (J, rest frame, from the last emitted E and B at nodes) and the bunching factor
   |<exp(j kb z)>| at the rest-frame ponderomotive wavenumber kb; bunching3 = {|b|, Re b, Im b}.
   Either pointer may be NULL. */
int mithra_diag(mithra_t run, double *field_energy, double *bunching3);

/* Derived constants (19 doubles): gamma0, beta0, dx, dy, dz, dt, dt_b, A_nsfd, x0, y0, z0, T0,
   omega_h, M, plane index, z_ref, macro charge, k*, kb.  hbm_bytes: device bytes held. */
int mithra_info(mithra_t run, double *info19, int64_t *hbm_bytes);

/* Per-kernel timing with CUDA events on the run's stream (off by default).  When on, every
   launch of every kernel of the step is bracketed by events; mithra_kernel_stats returns the
   summed device time (ms) and launch count per kernel id since the last reset. */
#define MITHRA_K_EMIT 0
#define MITHRA_K_PUSH 1
#define MITHRA_K_STENCIL 2
#define MITHRA_K_MUR 3
#define MITHRA_K_POWER 4
#define MITHRA_K_SORT 5
#define MITHRA_K_CLEAR 6
#define MITHRA_K_COUNT 7
int mithra_set_profiling(mithra_t run, int on);
/* Number of CUDA kernels this library has launched since it was loaded (all runs, all threads). */
int64_t mithra_kernel_launches(void);
int mithra_kernel_stats(mithra_t run, int kernel_id, double *total_ms, int64_t *launches);
const char *mithra_kernel_name(int kernel_id);

/* Serving (continuous batching).  Requests - each one run of its own grid, bunch, undulator,
   precision and step count - are queued by mithra_submit and admitted first come, first served
   as soon as their device-memory footprint fits in the serving pool; every admitted request is
   a run on its own CUDA stream, advanced in chunks of steps by one scheduler thread, so the
   kernels of concurrent requests overlap on the GPU.  A finished request returns its memory to
   the pool and its results wait in host memory until mithra_release.  Results do not depend on
   what else is being served (each run owns its buffers).  Times are seconds on the server's
   monotonic clock. */
typedef struct mithra_result {
    int32_t status;            /* MITHRA_OK, or the request's error (ENOMEM: larger than the pool) */
    int32_t state;             /* 0 queued, 1 running, 2 done */
    int64_t steps;             /* steps taken (done) or enqueued so far (running) */
    double t_submit, t_admit, t_done;
    double field_energy;       /* J, rest frame, after the last step */
    double bunching;           /* |<exp(j kb z)>| after the last step */
    double power_last;         /* lab radiated power at the last step (W) */
    double power_peak;         /* largest lab radiated power of the series (W) */
    int64_t hbm_bytes;         /* device bytes the run held */
    int64_t reserved_bytes;    /* footprint reserved at admission */
} mithra_result;

/* Start the server on the current device with a pool of hbm_budget_bytes (allocated once, from
   the installed allocator), at most max_active requests on the device, a queue of at most
   queue_capacity waiting requests, and steps_per_chunk steps enqueued per request at a time. */
int mithra_serve_start(size_t hbm_budget_bytes, int max_active, int queue_capacity, int steps_per_chunk);
/* As mithra_serve_start; grouped = 1 also advances the admitted requests together: whenever two or
   more of them are at a step from which their next steps are one replay of their captured period
   (see mithra_step), one graph whose child graphs are those periods advances all of them with one
   launch, rebuilt when its members change; a request's own steps keep their order (the group
   waits for each member's stream and each member's stream waits for the group).  Requests outside
   a group step on their own streams as with grouped = 0.  Results do not depend on the grouping. */
int mithra_serve_start_grouped(size_t hbm_budget_bytes, int max_active, int queue_capacity, int steps_per_chunk,
                               int grouped);
/* out = {group launches, request periods advanced by them} since mithra_serve_start*. */
int mithra_serve_group_stats(int64_t out[2]);
/* Queue one request (inputs copied; never blocks).  EAGAIN when the queue is full, EINVAL as
   mithra_create, and when no server is running. */
int mithra_submit(const mithra_grid *grid, const mithra_undulator *und, const mithra_bunch *bunch, int64_t nsteps,
                  uint64_t *ticket);
/* State and scalar results of a request; done = 1 once it has finished.  ENOTFOUND: unknown ticket. */
int mithra_poll(uint64_t ticket, int *done, mithra_result *out);
/* Radiated-power series of a finished request (as mithra_radiated_power).  EAGAIN if not finished. */
int mithra_result_series(uint64_t ticket, double *p_lab, double *t_lab, size_t cap, size_t *n_out);
/* Forget a finished request and its results. */
int mithra_release(uint64_t ticket);
/* stats = {completed, active, queued, reserved bytes, pool bytes in use, pool peak bytes}. */
int mithra_serve_stats(int64_t stats[6]);
/* Stop the scheduler (unfinished requests end with ETIMEDOUT) and free the pool. */
int mithra_serve_stop(void);

/* Field energy of caller-supplied E and B arrays, computed without allocating any device memory.
   No counterpart in the paper: it serves callers that cannot call cudaMalloc at that moment
   (a pool that is already fully carved up, a thread that must not take allocator locks, a
   real-time loop where an allocation's implicit synchronisation would stall every stream).
   eb[0..5]: device pointers to E_x, E_y, E_z, B_x, B_y, B_z (n values each, FP64 when precision
   is 0, FP32 when 1); energy_out: caller-owned device pointer to one double, written with
   sum(eps0 E^2/2 + B^2/(2 mu0)) * cell_volume; the work is enqueued on `stream` (a cudaStream_t,
   NULL for the legacy default stream) and the call returns without waiting.
   Scratch: one FP64 partial per 4096 nodes in a fixed 256 KiB array inside the library's device
   memory, present on every GPU that loads the library until the process exits; hence n may not
   exceed MITHRA_NOALLOC_MAX_NODES (EINVAL otherwise).  The first call on a device looks up that
   array's device address with the device current (cudaGetSymbolAddress) and keeps it for the
   process; make that first call before any stream capture.  A cudaDeviceReset destroys the array
   with the context: do not call this entry point on that device after a reset (every run handle
   and device buffer of the device is gone as well).  All calls share the array: calls whose work overlaps on the GPU
   race, so order them on one stream.  Each call writes every partial it reads; nothing needs
   clearing between calls.  Errors: EINVAL, ECUDA. */
#define MITHRA_NOALLOC_MAX_NODES (134217728LL)
int mithra_field_energy_noalloc(const void *const eb[6], int precision, int64_t n, double cell_volume,
                                double *energy_out, void *stream);

/* Release everything the run holds (waits for its stream).  NULL is ignored. */
void mithra_destroy(mithra_t run);

const char *mithra_last_error(void);
int mithra_version(void);

#ifdef __cplusplus
}
#endif
#endif
