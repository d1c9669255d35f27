/*
 * FP64 CPU oracle for the rest-frame FDTD/PIC time step of MITHRA 2.0
 * (A. Fallahi, arXiv:2009.13645).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this code: only the test-suite, the smoke check and the bench's CPU
 * baseline leg use it.  It shares no code, header or constant table with the
 * CUDA library; both receive the same lab-frame particle arrays from the
 * seeded input generator and nothing else.
 *
 * The oracle is plain and unblocked: every function follows one equation of the
 * manual in its own order and notation.  Loops whose iterations are independent of
 * one another (the stencil, the E/B evaluation, the per-particle push) may run on
 * several threads (OpenMP); every accumulation runs serially in a fixed order, so the
 * results are the same for any thread count.
 *
 * Parity pins (tests/test_oracle_*.py) tie it to what the paper and the
 * mathematics fix: the discrete dispersion relations (Eqs. numericalDispersionCD,
 * NSFDDispersionCD), the exact one-cell shift of NSFD at c dt = dz, the Mur
 * coefficient formulas and the Engquist-Majda reflection curves, the Mur edge and
 * corner values (a field satisfying every meeting face's outgoing condition is
 * reproduced exactly), E and B at nodes (exact for potentials linear in space) and
 * the field energy of uniform fields, discrete charge continuity, the Lorentz gauge
 * residual, Boris rotation invariants, Lorentz invariants of the transformed
 * undulator field, the single-electron undulator trajectory and the
 * optimize-bunch-position drift, the on-axis resonance of planar, helical and
 * optical undulators, the plane-wave flux and coherent scaling of the radiated
 * power, and the absolute power of a weak-undulator electron against the flux of
 * the equivalent rest-frame dipole through the plane (within 8 %).
 */
#ifndef MITHRA_ORACLE_H
#define MITHRA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_params {
    /* mesh, lab frame (Sec. MESH: mesh-lengths, mesh-resolution, mesh-center) */
    int32_t nx, ny, nz;
    double dx, dy, dz;        /* lab resolution; the rest frame uses dz*gamma0 (Eq. LorentzTransformB) */
    double cx, cy, cz;        /* mesh centre relative to the bunch reference point, lab */
    int32_t solver;           /* 0 NSFD (Eq. updateEquation), 1 FD (central differences) */
    double courant;           /* FD: dt = courant x the CFL bound (Eq. CFLcondition) */
    int32_t mur_order;        /* 1 or 2 */
    int32_t space_charge;     /* 0: phi == 0 and no charge deposition */
    int32_t substeps;         /* N in dt_b = dt / N */
    int32_t periodic[3];      /* test-only periodic axes (no Mur on them) */
    double plane_dist;        /* lab distance of the power plane ahead of the bunch reference */
    double norm_freq;         /* normalised frequency h of the power diagnostic */
    /* undulator (Sec. UNDULATOR) */
    int32_t und_kind;         /* -1 none, 0 planar static, 1 helical static, 2 optical plane wave, 3 optical Gaussian,
                                 4 static undulator array */
    double K;                 /* undulator parameter, or a0 for an optical undulator */
    double lambda_u;          /* period, or laser wavelength */
    double n_periods;
    double pol_deg;
    double waist;
    double pulse_fwhm;        /* c tau, intensity FWHM */
    int32_t signal;           /* 0 modulated Gaussian, 1 flat-top */
    double dist_head;
    /* bunch */
    double gamma;             /* mean Lorentz factor (sets the rest frame) */
    double charge_e;          /* electrons in the bunch */
    double sig_z;             /* lab rms length: the head sits 3 sig_z ahead of the centre */
    /* static undulator array (Sec. UNDULATOR, static-undulator-array): n_modules planar modules
       of n_periods periods each, `gap` apart (lab length), K_i = K + i * taper */
    double gap;
    int32_t n_modules;
    double taper;
    /* radiated-power spectrum (Sec. FEL-OUTPUT, radiation-power: minimum / maximum normalised
       frequency, number of frequency points); nf_points = 0: off */
    double nf_min, nf_max;
    int32_t nf_points;
    /* bunch sampling (Sec. BUNCH, bunch-sampling) every `bunch_every` steps; 0: off */
    int32_t bunch_every;
    /* seed injected through TF/SF planes (Sec. "Seed Field"; Sec. FIELD, field-initialization):
       -1 none, 0 plane wave, 1 Gaussian beam, propagating along +z; lab-frame parameters */
    int32_t seed_type;
    double seed_a0;           /* strength a0 = e A0 / (m c) */
    double seed_lambda;       /* wavelength */
    double seed_pol_deg;      /* polarisation angle from x */
    double seed_waist;        /* Gaussian beam waist w0 */
    double seed_focus;        /* lab coordinate of the reference point / focus (from the undulator entrance) */
    double seed_offset;       /* c t0: the pulse centre passes the reference point at lab time t0 */
    double seed_pulse_fwhm;   /* c tau (intensity FWHM); <= 0: continuous wave */
    double seed_cep_deg;      /* carrier envelope phase */
    /* optimize-bunch-position (Sec. MESH): static undulators only; 1 shifts the mesh and the
       power plane along z by the rest-frame drift of the bunch reference before the undulator
       entrance reaches it, so that the bunch sits at its placed position inside the undulator */
    int32_t optimize_position;
} orc_params;

typedef struct orc_run orc_run;

/* Threads the oracle's independent loops use (OpenMP; 1 when built without it).  The stencil,
   the E/B evaluation and the per-particle push run their iterations on several threads; every
   sum whose order matters (the deposition, the diagnostics) stays serial, so results do not
   depend on the thread count. */
int orc_threads(void);
/* Use n threads for the later steps (n >= 1; no effect without OpenMP). */
void orc_set_threads(int n);

/* Create a run from lab-frame particles lab6 (np x 6: x, y, z, ux, uy, uz; copied). */
orc_run *orc_create(const orc_params *p, const double *lab6, int64_t np);
void orc_destroy(orc_run *r);

/* Advance nsteps field steps (Sec. step order: E/B, push+deposit, stencil, Mur, power). */
void orc_step(orc_run *r, int64_t nsteps);

/* Derived constants: out[0..] = gamma0, beta0, dx, dy, dz, dt, dtb, A_nsfd, x0, y0, z0, T0,
   omega_h, M (window), kp (plane index), z_ref, q (macro charge), kstar, kb. */
void orc_info(const orc_run *r, double out[19]);

/* Field access.  which: 0..3 = Ax, Ay, Az, phi at level lev (0: n, 1: n+1 of the current step);
   4..7 = Jx, Jy, Jz, rho (last deposit); 8..13 = Ex, Ey, Ez, Bx, By, Bz at nodes (last emitted). */
void orc_get_field(const orc_run *r, int which, int lev, double *out);
void orc_set_field(orc_run *r, int which, int lev, const double *in);

/* Particles in the rest frame: (np x 6) x, y, z, ux, uy, uz. */
void orc_get_particles(const orc_run *r, double *out6);
void orc_set_particles(orc_run *r, const double *rest6);
int64_t orc_num_particles(const orc_run *r);

/* Per-step series (length = steps taken): lab power (W), lab time (s), on-axis Ex (V/m). */
int64_t orc_series(const orc_run *r, double *power_lab, double *t_lab, double *onaxis_ex);

/* Radiated-power spectrum: h_out[k] (nf_points) the normalised frequencies h_k = nf_min + k
   (nf_max - nf_min) / (nf_points - 1), p_lab (steps x nf_points) the lab power at each of them,
   defined as the series of orc_series with h = h_k and its own window M_k = round(2 pi /
   (h_k w* dt)).  Returns the number of steps. */
int64_t orc_spectrum(const orc_run *r, double *h_out, double *p_lab);

/* Bunch samples (rows x 15): rest-frame time of the positions (T0 + (n + 3/2) dt after step n),
   mean x, y, z (rest frame, m), mean gamma*beta_x,y,z, rms spread of x, y, z and of
   gamma*beta_x,y,z, mean and rms spread of the lab Lorentz factor gamma0 (gamma + beta0 u_z);
   taken after the push of every step n with n % bunch_every == 0.  Returns the number of rows. */
int64_t orc_bunch_series(const orc_run *r, double *out);

/* Diagnostics from the last emitted E/B and the current particles: field energy (J, rest
   frame) and the bunching factor at the rest-frame ponderomotive wavenumber kb:
   bunching[0] = |<exp(j kb z)>|, bunching[1], bunching[2] = real and imaginary parts. */
void orc_diag(const orc_run *r, double *field_energy, double *bunching);

/* Single pieces, for the pins. */
void orc_external_field(const orc_run *r, double x, double y, double z, double t,
                        double E[3], double B[3]);
void orc_lab_field(const orc_run *r, double xl, double yl, double zeta, double tl,
                   double Ep[3], double Bp[3]);
void orc_boris(double u[3], const double E[3], const double B[3], double dtb);
/* Seed: the lab-frame transverse vector potential (Ax, Ay) of the seed at the rest-frame
   event (x, y, z, t). */
void orc_seed_potential(const orc_run *r, double x, double y, double z, double t, double A[2]);
/* One Mur update of component `which` (0..3): writes boundary points of level n+2
   from levels n+2 (interior), n+1, n. */
void orc_mur(orc_run *r, int which);
/* The interior stencil alone for component `which`. */
void orc_stencil(orc_run *r, int which);
void orc_rotate_levels(orc_run *r);
/* Deposition alone: J of the move old6 -> new6 (rest frame, n x 6) and rho at new6. */
void orc_deposit_moves(orc_run *r, const double *old6, const double *new6, int64_t n);

/* Quasi-random bunch loading (Sec. "Electron Bunch Generation"; Sec. BUNCH, ellipsoid). */
typedef struct orc_ellipsoid {
    int32_t uniform;          /* 0 Gaussian current profile, 1 uniform over [-sig_z, sig_z] */
    double gamma;             /* mean Lorentz factor (momentum along +z) */
    double sig[3];            /* position spreads (sig_z: half length when uniform) */
    double sig_u[3];          /* spreads of gamma*beta_x, gamma*beta_y, gamma*beta_z */
    double cse_sigma;         /* uniform profile: rms width of the Gaussian edges (<= 0: none) */
    double lambda_r;          /* wavelength of the bunching and of the shot-noise slices */
    double bunching;          /* bunching factor b_f at lambda_r */
    double bunching_phase;    /* its phase (rad) */
    int32_t shot_noise;       /* 1: shot-noise modulation per slice of length lambda_r */
    double charge_e;          /* electrons in the bunch (shot-noise amplitude) */
} orc_ellipsoid;

/* The Halton number of index j in the i-th prime base (i < 20): one minus the radical inverse
   of j (the digits of j in base p mirrored about the radix point). */
double orc_halton(unsigned i, unsigned j);

/* n lab-frame macro-particles (n x 6: x, y, z, gamma*beta_x, gamma*beta_y, gamma*beta_z). */
void orc_ellipsoid_bunch(const orc_ellipsoid *e, int64_t n, double *out6);

#ifdef __cplusplus
}
#endif
#endif
