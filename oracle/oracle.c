/*
 * FP64 CPU oracle for one rest-frame FDTD/PIC time step of MITHRA 2.0
 * (A. Fallahi, "MITHRA 2.0: A Full-Wave Simulation Tool for Free Electron
 * Lasers", arXiv:2009.13645).  TEST INFRASTRUCTURE ONLY: see oracle.h.
 *
 * Readings of the manual that this file implements (each one also listed in
 * the design notes of the repository):
 *  - Source sign (Eq. WaveA/WaveF vs the update equations): psi^{n+1} = ...
 *    + (c dt)^2 mu0 J for A and + (c dt)^2 rho/eps0 for phi.
 *  - NSFD coefficient alpha'_6 = alpha'_7 = (c dt/dz)^2 - 2A(c dt/dx)^2 - 2A(c dt/dy)^2
 *    (the printed form repeats the dx term).
 *  - Layout: A_l and J_l live on edge centres (A_x at (i+1/2, j, k) ...), phi and
 *    rho on nodes; the same scalar update is applied to every component lattice.
 *    E and B at nodes use the manual's central-difference formulas applied to
 *    node averages of the staggered potentials (Sec. "Field Evaluation").
 *  - Time centring: level k of A is at k dt, level k of phi at (k+1/2) dt;
 *    particles hold r at half steps and u at integer steps.
 *  - Interpolation weights: linear, w0 = 1 - d/D, w1 = d/D (Eq. fieldInterpolation
 *    prints a weight that is wrong above d/D = 1/2).
 *  - Zigzag (Umeda) split at the relay point; each straight piece inside one
 *    cell deposits the exact path integral of the linear weights of the other
 *    two axes (midpoint product + D_a D_b / 12).  The midpoint product alone
 *    conserves charge only in 2D.
 *  - Mur edges and corners: the first-order conditions of the faces that meet
 *    there, discretised at the centre of the square (edge) or cube (corner),
 *    summed, and solved for the boundary value (Sec. "Second Order ABCs").
 *  - Particles outside the node range with a one-cell margin are pushed in the
 *    external field alone and deposit nothing.
 *  - Lorentz boost of particles: z = gamma0 z', u_z = gamma0 (u'_z - beta0 gamma'),
 *    and a ballistic shift to a common rest-frame time (Eq. LorentzTransformDeltaR)
 *    that is zero at the bunch reference point.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 */
#define C0 299792458.0
#define MU0 1.25663706212e-6
#define QE 1.602176634e-19
#define ME 9.1093837015e-31
#define PI 3.14159265358979323846

struct orc_run {
    orc_params p;
    int nx, ny, nz;
    int64_t ncell;
    int ext[4][3];
    double gamma0, beta0;
    double dx, dy, dz, dt, dtb, cdt, A;
    double x0, y0, z0;
    double T0, zeta_ref, z_ref;
    double shift;   /* optimize-bunch-position: z shift of the mesh and the power plane */
    double q;
    double B0, ku, Lu;
    double E0, kL, zeta_f, t_f;
    double kstar, kb, omega_h;
    int M, kp;
    double *lev[3][4];
    double *src[4];
    double *eb[6];
    int64_t np;
    double *pr;   /* np x 6: position relative to node (0,0,0) (m), then gamma*beta */
    int64_t step;
    double *ring;
    double *ring_t;
    int64_t nser, cap;
    double *ser_p, *ser_t, *ser_e;
    /* spectrum: history of the plane samples (Mh slots) and the power per step and frequency */
    int nf, Mh;
    double *hk;
    int *Mk;
    double *hist, *hist_t;
    double *spec;
    /* bunch samples */
    int64_t nbs, bcap;
    double *bser;
};

static double eps0(void) { return 1.0 / (MU0 * C0 * C0); }

static inline int64_t IDX(const orc_run *r, int i, int j, int k)
{
    return (int64_t)i + (int64_t)r->nx * ((int64_t)j + (int64_t)r->ny * (int64_t)k);
}

static inline int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

/* ------------------------------------------------------------------------- */
/* Set-up: rest frame (Sec. "Lorentz Transformation"), mesh adjustment        */
/* (Sec. MESH, checks before the run), bunch boost (Eq. LorentzTrasnformParticles, */
/* Eq. LorentzTransformDeltaR).                                                */
/* ------------------------------------------------------------------------- */

static void boost_particle(const orc_run *r, const double *lab, double *rest)
{
    const double g0 = r->gamma0, b0 = r->beta0;
    const double ux = lab[3], uy = lab[4], uzp = lab[5];
    const double gp = sqrt(1.0 + ux * ux + uy * uy + uzp * uzp);
    const double uz = g0 * (uzp - b0 * gp);
    const double g = sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    /* event (t'=0, zeta_ref + z') -> rest (z, t); propagate with the rest-frame
       velocity to the common time T0 + dt/2 (the time of r^{1/2}). */
    const double z = r->z_ref + g0 * lab[2];
    const double s = g0 * b0 * lab[2] + 0.5 * C0 * r->dt; /* c (T0 + dt/2 - t_p) */
    rest[0] = lab[0] + ux / g * s;
    rest[1] = lab[1] + uy / g * s;
    rest[2] = z + uz / g * s;
    rest[3] = ux;
    rest[4] = uy;
    rest[5] = uz;
}

orc_run *orc_create(const orc_params *p, const double *lab6, int64_t np)
{
    orc_run *r = (orc_run *)calloc(1, sizeof(orc_run));
    r->p = *p;
    r->nx = p->nx;
    r->ny = p->ny;
    r->nz = p->nz;
    r->ncell = (int64_t)p->nx * p->ny * p->nz;
    for (int c = 0; c < 4; ++c) {
        const int n[3] = {p->nx, p->ny, p->nz};
        for (int a = 0; a < 3; ++a) r->ext[c][a] = n[a] - ((c == a && !p->periodic[a]) ? 1 : 0);
    }

    /* rest frame: gamma0 = gamma / sqrt(1 + K^2/2) for a planar undulator or a
       linearly polarised laser (a0 as K); helical: gamma / sqrt(1 + K^2). */
    double g0 = p->gamma;
    if (p->und_kind == 0 || p->und_kind == 2 || p->und_kind == 3 || p->und_kind == 4)
        g0 = p->gamma / sqrt(1.0 + 0.5 * p->K * p->K);   /* array: the first module's K */
    else if (p->und_kind == 1) g0 = p->gamma / sqrt(1.0 + p->K * p->K);
    r->gamma0 = g0;
    r->beta0 = sqrt(1.0 - 1.0 / (g0 * g0));

    /* mesh boost and adjustment */
    r->dz = g0 * p->dz;
    r->dx = p->dx;
    r->dy = p->dy;
    if (p->solver == 0) {
        double ratio = sqrt(pow(r->dz / r->dx, 2) + pow(r->dz / r->dy, 2));
        if (ratio >= 1.0) {
            const double s = ratio / 0.99;
            r->dx *= s;
            r->dy *= s;
            ratio = 0.99;
        }
        r->A = 0.25 * (1.0 + 0.02 / (pow(r->dz / r->dx, 2) + pow(r->dz / r->dy, 2)));
        r->dt = r->dz / C0;
    } else {
        r->A = 0.0;
        r->dt = p->courant / (C0 * sqrt(1.0 / (r->dx * r->dx) + 1.0 / (r->dy * r->dy) + 1.0 / (r->dz * r->dz)));
    }
    r->cdt = C0 * r->dt;
    r->dtb = r->dt / (p->substeps > 0 ? p->substeps : 1);

    /* undulator */
    r->ku = 2.0 * PI / p->lambda_u;
    r->Lu = p->n_periods * p->lambda_u;
    r->B0 = 2.0 * PI * ME * C0 * p->K / (QE * p->lambda_u);
    r->kL = 2.0 * PI / p->lambda_u;
    r->E0 = p->K * ME * C0 * (C0 * r->kL) / QE;
    if (p->und_kind == 0 || p->und_kind == 1 || p->und_kind == 4) r->kstar = g0 * r->beta0 * r->ku;
    else if (p->und_kind == 2 || p->und_kind == 3) r->kstar = g0 * (1.0 + r->beta0) * r->kL;
    else r->kstar = 2.0 * PI / p->lambda_u;
    r->omega_h = p->norm_freq * C0 * r->kstar;
    /* bunching wavenumber: the rest-frame ponderomotive wave, pump + radiation
       (static: gamma0 k_u + k*; optical: 2 k*).  It is the lab resonant bunching
       wavenumber seen from the rest frame. */
    if (p->und_kind == 0 || p->und_kind == 1 || p->und_kind == 4) r->kb = g0 * r->ku + r->kstar;
    else if (p->und_kind == 2 || p->und_kind == 3) r->kb = 2.0 * r->kstar;
    else r->kb = r->kstar;

    /* placement: the rest-frame origin is the boost of the lab event (t'=0, undulator
       entrance).  A static undulator starts with its entrance dist_head/gamma0 ahead of the
       bunch head (head = centre + 3 sig_z) in the rest frame; an optical undulator
       starts with the bunch reference at the origin. */
    if (p->und_kind == 0 || p->und_kind == 1 || p->und_kind == 4) {
        const double h = 3.0 * p->sig_z;
        r->zeta_ref = -(p->dist_head + g0 * g0 * h);
    } else {
        r->zeta_ref = 0.0;
    }
    r->z_ref = g0 * r->zeta_ref;
    r->T0 = -g0 * r->beta0 * r->zeta_ref / C0;
    /* optical undulator timing: pulse centre at zeta = dist_head at t'=0, moving -z;
       it meets the bunch reference at the focus. */
    r->t_f = p->dist_head / (C0 * (1.0 + r->beta0));
    r->zeta_f = r->beta0 * p->dist_head / (1.0 + r->beta0);

    r->x0 = p->cx - 0.5 * (p->nx - 1) * r->dx;
    r->y0 = p->cy - 0.5 * (p->ny - 1) * r->dy;
    r->z0 = r->z_ref + g0 * p->cz - 0.5 * (p->nz - 1) * r->dz;

    /* optimize-bunch-position (Sec. MESH): the bunch is to sit at its placed position once it
       has passed the undulator entrance.  Before the entrance the reference particle (on axis,
       Lorentz factor gamma) moves in the rest frame with v = (beta - beta0) / (1 - beta beta0)
       (velocity addition); the entrance moves with -beta0 c and, at the reference's time T0,
       lies g0 zeta_ref (beta0^2 - 1) = -zeta_ref / g0 ahead of it.  They meet after
       t = (-zeta_ref / g0) / ((v + beta0) c), by which the reference has moved v c t: the mesh
       and the power plane move by that distance. */
    r->shift = 0.0;
    if (p->optimize_position && (p->und_kind == 0 || p->und_kind == 1 || p->und_kind == 4)) {
        const double beta = sqrt(1.0 - 1.0 / (p->gamma * p->gamma));
        const double v = (beta - r->beta0) / (1.0 - beta * r->beta0);
        const double t = (-r->zeta_ref / g0) / ((v + r->beta0) * C0);
        r->shift = v * C0 * t;
    }
    r->z0 += r->shift;

    for (int l = 0; l < 3; ++l)
        for (int c = 0; c < 4; ++c) r->lev[l][c] = (double *)calloc((size_t)r->ncell, sizeof(double));
    for (int c = 0; c < 4; ++c) r->src[c] = (double *)calloc((size_t)r->ncell, sizeof(double));
    for (int c = 0; c < 6; ++c) r->eb[c] = (double *)calloc((size_t)r->ncell, sizeof(double));

    r->np = np;
    r->pr = (double *)malloc((size_t)(np > 0 ? np : 1) * 6 * sizeof(double));
    for (int64_t i = 0; i < np; ++i) {
        double *q = r->pr + 6 * i;
        boost_particle(r, lab6 + 6 * i, q);
        /* a particle is located by its distance to the grid corner (Sec. "Field Evaluation"):
           far from the origin this keeps the resolution of the step-by-step displacements */
        q[0] -= r->x0;
        q[1] -= r->y0;
        q[2] -= r->z0;
    }
    /* macro-particle charge: the bunch charge spread over the macro-particles */
    r->q = (np > 0) ? -QE * p->charge_e / (double)np : 0.0;

    /* power diagnostic */
    {
        const double zp = r->z_ref + r->shift + g0 * p->plane_dist;
        long kp = lround((zp - r->z0) / r->dz);
        if (kp < 1) kp = 1;
        if (kp > p->nz - 2) kp = p->nz - 2;
        r->kp = (int)kp;
        long M = lround(2.0 * PI / (r->omega_h * r->dt));
        r->M = (int)(M < 1 ? 1 : M);
        r->ring = (double *)calloc((size_t)r->M * 4 * p->nx * p->ny, sizeof(double));
        r->ring_t = (double *)calloc((size_t)r->M, sizeof(double));
    }
    /* spectrum: frequencies h_k and windows M_k = round(2 pi / (h_k w* dt)) */
    if (p->nf_points > 0) {
        r->nf = p->nf_points;
        r->hk = (double *)malloc((size_t)r->nf * sizeof(double));
        r->Mk = (int *)malloc((size_t)r->nf * sizeof(int));
        r->Mh = 1;
        for (int k = 0; k < r->nf; ++k) {
            r->hk[k] = r->nf == 1 ? p->nf_min : p->nf_min + k * (p->nf_max - p->nf_min) / (r->nf - 1);
            long Mk = lround(2.0 * PI / (r->hk[k] * C0 * r->kstar * r->dt));
            r->Mk[k] = (int)(Mk < 1 ? 1 : Mk);
            if (r->Mk[k] > r->Mh) r->Mh = r->Mk[k];
        }
        r->hist = (double *)calloc((size_t)r->Mh * 4 * p->nx * p->ny, sizeof(double));
        r->hist_t = (double *)calloc((size_t)r->Mh, sizeof(double));
    }
    return r;
}

void orc_destroy(orc_run *r)
{
    if (!r) return;
    for (int l = 0; l < 3; ++l)
        for (int c = 0; c < 4; ++c) free(r->lev[l][c]);
    for (int c = 0; c < 4; ++c) free(r->src[c]);
    for (int c = 0; c < 6; ++c) free(r->eb[c]);
    free(r->pr);
    free(r->ring);
    free(r->ring_t);
    free(r->ser_p);
    free(r->ser_t);
    free(r->ser_e);
    free(r->hk);
    free(r->Mk);
    free(r->hist);
    free(r->hist_t);
    free(r->spec);
    free(r->bser);
    free(r);
}

/* ------------------------------------------------------------------------- */
/* Field update (Sec. "FDTD for Wave Equation", Eq. updateEquation; FD is the */
/* same equation with the NSFD coefficient set to zero).                      */
/* ------------------------------------------------------------------------- */

void orc_stencil(orc_run *r, int c)
{
    const int *e = r->ext[c];
    const int *per = r->p.periodic;
    const double A = r->A;
    const double rx = pow(r->cdt / r->dx, 2), ry = pow(r->cdt / r->dy, 2), rz = pow(r->cdt / r->dz, 2);
    const double a1 = 2.0 * (1.0 - (1.0 - 2.0 * A) * rx - (1.0 - 2.0 * A) * ry - rz);
    const double a2 = rx, a3 = rx, a4 = ry, a5 = ry;
    const double a6 = rz - 2.0 * A * rx - 2.0 * A * ry, a7 = a6;
    const double a8 = r->cdt * r->cdt;
    const double sfac = (c < 3) ? MU0 : 1.0 / eps0();
    const double *pn = r->lev[1][c], *pm = r->lev[0][c], *S = r->src[c];
    double *out = r->lev[2][c];
    const int lo[3] = {per[0] ? 0 : 1, per[1] ? 0 : 1, per[2] ? 0 : 1};
    const int hi[3] = {per[0] ? e[0] : e[0] - 1, per[1] ? e[1] : e[1] - 1, per[2] ? e[2] : e[2] - 1};
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k < hi[2]; ++k) {
        const int km = wrap(k - 1, e[2]), kq = wrap(k + 1, e[2]);
        for (int j = lo[1]; j < hi[1]; ++j) {
            const int jm = wrap(j - 1, e[1]), jq = wrap(j + 1, e[1]);
            for (int i = lo[0]; i < hi[0]; ++i) {
                const int im = wrap(i - 1, e[0]), iq = wrap(i + 1, e[0]);
#define P(ii, jj, kk) pn[IDX(r, ii, jj, kk)]
                const double v = -pm[IDX(r, i, j, k)] + a1 * P(i, j, k)
                    + a2 * (A * P(iq, j, km) + (1.0 - 2.0 * A) * P(iq, j, k) + A * P(iq, j, kq))
                    + a3 * (A * P(im, j, km) + (1.0 - 2.0 * A) * P(im, j, k) + A * P(im, j, kq))
                    + a4 * (A * P(i, jq, km) + (1.0 - 2.0 * A) * P(i, jq, k) + A * P(i, jq, kq))
                    + a5 * (A * P(i, jm, km) + (1.0 - 2.0 * A) * P(i, jm, k) + A * P(i, jm, kq))
                    + a6 * P(i, j, kq) + a7 * P(i, j, km) + a8 * sfac * S[IDX(r, i, j, k)];
#undef P
                out[IDX(r, i, j, k)] = v;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Seed (Sec. "Seed Field"; Sec. FIELD, field-initialization; Eq. signalTypes).*/
/* ------------------------------------------------------------------------- */

/* Transverse vector potential of the seed, a beam propagating along +z in the lab, at the lab
   event of the rest-frame event (x, y, z, t) (Eq. LorentzTransformR2L with the time coordinate).
   A transverse potential is unchanged by the boost along z, so the lab value is the rest-frame
   value.  Plane wave: A0 f(tau, 0); Gaussian beam (paraxial, waist w0 at the reference point):
   A0 (w0/w(l)) exp(-r^2/w(l)^2) f(tau, atan(l/z_R) - k r^2 l / (2 (l^2 + z_R^2))), with l the
   distance travelled past the reference point and tau = t' - t0 - (zeta - zeta_f)/c the retarded
   lab time (t' - zeta/c = (t - z/c) / (g0 (1 + b0)) for the rest-frame event); f the modulated Gaussian of Eq. signalTypes (continuous for a non-positive pulse
   length) with the carrier envelope phase.  The polarisation angle rotates A in the xy-plane. */
void orc_seed_potential(const orc_run *r, double x, double y, double z, double t, double A[2])
{
    const orc_params *p = &r->p;
    A[0] = A[1] = 0.0;
    if (p->seed_type < 0) return;
    const double g0 = r->gamma0, b0 = r->beta0;
    const double zeta = g0 * (z + b0 * C0 * t);
    const double k = 2.0 * PI / p->seed_lambda, w = C0 * k;
    const double A0 = p->seed_a0 * ME * C0 / QE;
    /* retarded lab time t' - zeta/c of the +z beam, written as (t - z/c) / (g0 (1 + b0)): the
       same quantity as the boosted t' and zeta (Eq. LorentzTransformR2L) without the
       cancellation of two nearly equal lab times (a factor 2 g0^2 on a carrier phase of
       thousands of radians) */
    const double tau = (t - z / C0) / (g0 * (1.0 + b0)) - p->seed_offset / C0 + p->seed_focus / C0;
    const double cep = p->seed_cep_deg * PI / 180.0;
    double amp = 1.0, ph = 0.0;
    if (p->seed_type == 1) {
        const double w0 = p->seed_waist, zr = PI * w0 * w0 / p->seed_lambda;
        const double l = zeta - p->seed_focus;
        const double wl = w0 * sqrt(1.0 + (l / zr) * (l / zr));
        const double r2 = x * x + y * y;
        amp = (w0 / wl) * exp(-r2 / (wl * wl));
        ph = atan(l / zr) - k * r2 * l / (2.0 * (l * l + zr * zr));
    }
    double f = cos(w * tau + ph + cep);
    if (p->seed_pulse_fwhm > 0.0) {
        const double tp = p->seed_pulse_fwhm / C0;
        f *= exp(-2.0 * log(2.0) * tau * tau / (tp * tp));
    }
    const double th = p->seed_pol_deg * PI / 180.0;
    A[0] = A0 * amp * f * cos(th);
    A[1] = A0 * amp * f * sin(th);
}

/* Seed potential component c at lattice point (i, j, k) of component c's lattice (A_x sits at
   (i + 1/2) dx, A_y at (j + 1/2) dy) and rest time t. */
static double fval(const orc_run *r, int c, double hx, double hy, int i, int j, int k, double t)
{
    double A[2];
    orc_seed_potential(r, r->x0 + (i + hx) * r->dx, r->y0 + (j + hy) * r->dy, r->z0 + k * r->dz, t, A);
    return A[c];
}

/* TF/SF planes of the seed (Sec. "Seed Field"): node plane 1 of the z axis is the scattered-field
   plane, plane 2 the total-field plane.  After the update of level n+1 from level n, the terms
   of the update equation that reach across the two planes are corrected by the excitation f^n,
   the seed potential at the lattice points at the time of level n: the SF plane loses the
   contribution of f on plane 2 (it must see the scattered field there), the TF plane gains the
   contribution of f on plane 1 (it must see the total field there).  (The printed corrections
   carry the opposite signs; with these, a plane wave leaves the SF region at zero and the TF
   region equal to f.)  Only the transverse components A_x, A_y are excited. */
static void tfsf(orc_run *r, int c)
{
    if (r->p.seed_type < 0 || c > 1) return;
    const int *e = r->ext[c];
    if (e[2] < 4) return;
    const double A = r->A;
    const double rx = pow(r->cdt / r->dx, 2), ry = pow(r->cdt / r->dy, 2), rz = pow(r->cdt / r->dz, 2);
    const double a2 = rx, a3 = rx, a4 = ry, a5 = ry;
    const double a6 = rz - 2.0 * A * rx - 2.0 * A * ry, a7 = a6;
    /* level n of the update that produced lev[2] is lev[1], at rest time T0 + (step + 1) dt */
    const double t = r->T0 + ((double)r->step + 1.0) * r->dt;
    const double hx = (c == 0) ? 0.5 : 0.0, hy = (c == 1) ? 0.5 : 0.0;
    const int per0 = r->p.periodic[0], per1 = r->p.periodic[1];
    const int ilo = per0 ? 0 : 1, ihi = per0 ? e[0] : e[0] - 1;
    const int jlo = per1 ? 0 : 1, jhi = per1 ? e[1] : e[1] - 1;
    double *out = r->lev[2][c];
#define F(ii, jj, kk) fval(r, c, hx, hy, ii, jj, kk, t)
    for (int j = jlo; j < jhi; ++j)
        for (int i = ilo; i < ihi; ++i) {
            const double sf = A * (a2 * F(i + 1, j, 2) + a3 * F(i - 1, j, 2) + a4 * F(i, j + 1, 2) + a5 * F(i, j - 1, 2))
                              + a6 * F(i, j, 2);
            const double tf = A * (a2 * F(i + 1, j, 1) + a3 * F(i - 1, j, 1) + a4 * F(i, j + 1, 1) + a5 * F(i, j - 1, 1))
                              + a7 * F(i, j, 1);
            out[IDX(r, i, j, 1)] -= sf;
            out[IDX(r, i, j, 2)] += tf;
        }
#undef F
}

/* Mur boundary (Sec. "Boundary Truncation").  Level naming as in the manual:
   xi^{n+1} = lev[2], xi^n = lev[1], xi^{n-1} = lev[0]. */

static int bset(const orc_run *r, int c, const int ijk[3], int *axes, int *sig)
{
    int ns = 0;
    for (int a = 0; a < 3; ++a) {
        if (r->p.periodic[a]) continue;
        if (ijk[a] == 0) { axes[ns] = a; sig[ns] = +1; ++ns; }
        else if (ijk[a] == r->ext[c][a] - 1) { axes[ns] = a; sig[ns] = -1; ++ns; }
    }
    return ns;
}

static double dl(const orc_run *r, int a) { return a == 0 ? r->dx : (a == 1 ? r->dy : r->dz); }

/* Face update with the manual's beta (first order) or gamma (second order) coefficients. */
static void mur_face_point(orc_run *r, int c, const int ijk[3], int a, int sg)
{
    const double *xn1 = r->lev[2][c], *xn = r->lev[1][c], *xm = r->lev[0][c];
    double *out = r->lev[2][c];
    const double cdt = r->cdt, D = dl(r, a);
    int in[3] = {ijk[0], ijk[1], ijk[2]};
    in[a] += sg;
    const int64_t b = IDX(r, ijk[0], ijk[1], ijk[2]), q = IDX(r, in[0], in[1], in[2]);
    double v;
    if (r->p.mur_order == 1) {
        const double b0 = (cdt - D) / (cdt + D), b1 = 2.0 * D / (cdt + D), b2 = -1.0, b3 = b1, b4 = b0;
        v = b0 * xm[b] + b1 * xn[b] + b2 * xm[q] + b3 * xn[q] + b4 * xn1[q];
    } else {
        const int t1 = (a + 1) % 3, t2 = (a + 2) % 3; /* the two tangential axes */
        const double D1 = dl(r, t1), D2 = dl(r, t2);
        const double r1 = pow(cdt / D1, 2), r2 = pow(cdt / D2, 2);
        const double g0 = (cdt - D) / (cdt + D), g4 = g0, g2 = -1.0;
        const double g1 = D * (2.0 - r1 - r2) / (cdt + D), g3 = g1;
        const double g5 = r1 * D / (2.0 * (cdt + D)), g6 = g5, g9 = g5, g10 = g5;
        const double g7 = r2 * D / (2.0 * (cdt + D)), g8 = g7, g11 = g7, g12 = g7;
        int pp[3], mm[3];
        double sin_ = 0, sfa = 0;
        /* neighbours along t1 on the inner plane (gamma5, gamma6) and the face (gamma9, gamma10) */
        for (int s = 0; s < 2; ++s) {
            const int t = s == 0 ? t1 : t2;
            const double gi = s == 0 ? g5 : g7, gj = s == 0 ? g6 : g8;
            const double fi = s == 0 ? g9 : g11, fj = s == 0 ? g10 : g12;
            memcpy(pp, in, sizeof pp);
            memcpy(mm, in, sizeof mm);
            pp[t] = wrap(pp[t] + 1, r->ext[c][t]);
            mm[t] = wrap(mm[t] - 1, r->ext[c][t]);
            sin_ += gi * xn[IDX(r, pp[0], pp[1], pp[2])] + gj * xn[IDX(r, mm[0], mm[1], mm[2])];
            memcpy(pp, ijk, sizeof pp);
            memcpy(mm, ijk, sizeof mm);
            pp[t] = wrap(pp[t] + 1, r->ext[c][t]);
            mm[t] = wrap(mm[t] - 1, r->ext[c][t]);
            sfa += fi * xn[IDX(r, pp[0], pp[1], pp[2])] + fj * xn[IDX(r, mm[0], mm[1], mm[2])];
        }
        v = g0 * xm[b] + g1 * xn[b] + g2 * xm[q] + g3 * xn[q] + g4 * xn1[q] + sin_ + sfa;
    }
    out[b] = v;
}

/* Edge (ns = 2) or corner (ns = 3): the sum of the first-order conditions of the
   meeting faces, each discretised at the centre of the square / cube spanned by the
   boundary point and its inward neighbours, is affine in the unknown; solve it. */
static double edge_residual(const orc_run *r, int c, const int ijk[3], int ns, const int *axes,
                            const int *sig, double v)
{
    const double *xn1 = r->lev[2][c], *xn = r->lev[1][c], *xm = r->lev[0][c];
    const int npts = 1 << ns;
    double f1[8], f0[8], fm[8];
    for (int e = 0; e < npts; ++e) {
        int pt[3] = {ijk[0], ijk[1], ijk[2]};
        for (int s = 0; s < ns; ++s)
            if (e & (1 << s)) pt[axes[s]] += sig[s];
        const int64_t id = IDX(r, pt[0], pt[1], pt[2]);
        f1[e] = (e == 0) ? v : xn1[id];
        f0[e] = xn[id];
        fm[e] = xm[id];
    }
    double res = 0.0;
    const double dt = r->dt;
    for (int s = 0; s < ns; ++s) {
        double pn1 = 0, mn1 = 0, pm1 = 0, mm1 = 0;
        for (int e = 0; e < npts; ++e) {
            if (e & (1 << s)) { pn1 += f1[e]; pm1 += fm[e]; }
            else { mn1 += f1[e]; mm1 += fm[e]; }
        }
        const double h = (double)(npts / 2);
        res += ((pn1 - mn1) / h - (pm1 - mm1) / h) / (2.0 * dt * dl(r, axes[s]));
    }
    double tt = 0;
    for (int e = 0; e < npts; ++e) tt += f1[e] - 2.0 * f0[e] + fm[e];
    res -= (double)ns * (tt / npts) / (C0 * dt * dt);
    return res;
}

static void mur_corner_point(orc_run *r, int c, const int ijk[3], int ns, const int *axes, const int *sig)
{
    const double r0 = edge_residual(r, c, ijk, ns, axes, sig, 0.0);
    const double r1 = edge_residual(r, c, ijk, ns, axes, sig, 1.0);
    r->lev[2][c][IDX(r, ijk[0], ijk[1], ijk[2])] = -r0 / (r1 - r0);
}

void orc_mur(orc_run *r, int c)
{
    const int *e = r->ext[c];
    for (int pass = 1; pass <= 3; ++pass) {
        for (int a = 0; a < 3; ++a) {
            if (r->p.periodic[a]) continue;
            for (int side = 0; side < 2; ++side) {
                const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
                int ijk[3];
                ijk[a] = side == 0 ? 0 : e[a] - 1;
                for (int u = 0; u < e[t2]; ++u) {
                    for (int w = 0; w < e[t1]; ++w) {
                        ijk[t1] = w;
                        ijk[t2] = u;
                        int axes[3], sig[3];
                        const int ns = bset(r, c, ijk, axes, sig);
                        if (ns != pass || axes[0] != a) continue; /* each point once */
                        if (ns == 1) mur_face_point(r, c, ijk, a, sig[0]);
                        else mur_corner_point(r, c, ijk, ns, axes, sig);
                    }
                }
            }
        }
    }
}

void orc_rotate_levels(orc_run *r)
{
    for (int c = 0; c < 4; ++c) {
        double *t = r->lev[0][c];
        r->lev[0][c] = r->lev[1][c];
        r->lev[1][c] = r->lev[2][c];
        r->lev[2][c] = t;
    }
}

/* ------------------------------------------------------------------------- */
/* E and B at nodes (Sec. "Field Evaluation") from node averages of the      */
/* staggered potentials: levels n (lev[0]) and n+1 (lev[1]), phi^n (lev[0]). */
/* ------------------------------------------------------------------------- */

static double anode(const orc_run *r, int lev, int c, int i, int j, int k)
{
    const double *a = r->lev[lev][c];
    int m[3] = {i, j, k};
    if (c < 3) {
        const int n = r->ext[c][c] + (r->p.periodic[c] ? 0 : 1);
        m[c] = r->p.periodic[c] ? wrap(m[c] - 1, n) : m[c] - 1;
        return 0.5 * (a[IDX(r, i, j, k)] + a[IDX(r, m[0], m[1], m[2])]);
    }
    return a[IDX(r, i, j, k)];
}

static void emit_eb(orc_run *r)
{
    const int *per = r->p.periodic;
    const int n[3] = {r->nx, r->ny, r->nz};
    const int lo[3] = {per[0] ? 0 : 1, per[1] ? 0 : 1, per[2] ? 0 : 1};
    const int hi[3] = {per[0] ? n[0] : n[0] - 1, per[1] ? n[1] : n[1] - 1, per[2] ? n[2] : n[2] - 1};
    const double dt = r->dt, dx = r->dx, dy = r->dy, dz = r->dz;
    const int sc = r->p.space_charge;
    for (int c = 0; c < 6; ++c) memset(r->eb[c], 0, (size_t)r->ncell * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = lo[2]; k < hi[2]; ++k) {
        const int km = wrap(k - 1, n[2]), kq = wrap(k + 1, n[2]);
        for (int j = lo[1]; j < hi[1]; ++j) {
            const int jm = wrap(j - 1, n[1]), jq = wrap(j + 1, n[1]);
            for (int i = lo[0]; i < hi[0]; ++i) {
                const int im = wrap(i - 1, n[0]), iq = wrap(i + 1, n[0]);
                const int64_t id = IDX(r, i, j, k);
                const double *ph = r->lev[0][3];
                const double gx = sc ? (ph[IDX(r, iq, j, k)] - ph[IDX(r, im, j, k)]) / (2 * dx) : 0.0;
                const double gy = sc ? (ph[IDX(r, i, jq, k)] - ph[IDX(r, i, jm, k)]) / (2 * dy) : 0.0;
                const double gz = sc ? (ph[IDX(r, i, j, kq)] - ph[IDX(r, i, j, km)]) / (2 * dz) : 0.0;
                r->eb[0][id] = -(anode(r, 1, 0, i, j, k) - anode(r, 0, 0, i, j, k)) / dt - gx;
                r->eb[1][id] = -(anode(r, 1, 1, i, j, k) - anode(r, 0, 1, i, j, k)) / dt - gy;
                r->eb[2][id] = -(anode(r, 1, 2, i, j, k) - anode(r, 0, 2, i, j, k)) / dt - gz;
                double bx = 0, by = 0, bz = 0;
                for (int l = 0; l < 2; ++l) {
                    bx += (anode(r, l, 2, i, jq, k) - anode(r, l, 2, i, jm, k)) / (2 * dy)
                        - (anode(r, l, 1, i, j, kq) - anode(r, l, 1, i, j, km)) / (2 * dz);
                    by += (anode(r, l, 0, i, j, kq) - anode(r, l, 0, i, j, km)) / (2 * dz)
                        - (anode(r, l, 2, iq, j, k) - anode(r, l, 2, im, j, k)) / (2 * dx);
                    bz += (anode(r, l, 1, iq, j, k) - anode(r, l, 1, im, j, k)) / (2 * dx)
                        - (anode(r, l, 0, i, jq, k) - anode(r, l, 0, i, jm, k)) / (2 * dy);
                }
                r->eb[3][id] = 0.5 * bx;
                r->eb[4][id] = 0.5 * by;
                r->eb[5][id] = 0.5 * bz;
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* External fields (Sec. "Field Initialization"): lab-frame undulator / laser,*/
/* then Eqs. LorentzTransformElectric / LorentzTransformMagnetic.            */
/* ------------------------------------------------------------------------- */

/* Planar static undulator (Eqs. undulatorField, fringingField) whose magnetic field
   points along (-sin th, cos th), starting at lab coordinate `off`.  Past its end the
   entrance fringe is mirrored. */
static void planar_field(const orc_run *r, double th, double off, double xl, double yl, double zeta,
                         double Bp[3])
{
    const double ku = r->ku, B0 = r->B0;
    const double ct = cos(th), st = sin(th);
    const double yu = -xl * st + yl * ct;
    const double zl = zeta - off;
    double s, c;
    if (zl < 0.0) {
        const double g = exp(-0.5 * (ku * zl) * (ku * zl));
        s = ku * zl * g;
        c = g;
    } else if (zl > r->Lu) {
        const double d = zl - r->Lu;
        const double g = exp(-0.5 * (ku * d) * (ku * d));
        s = ku * d * g;
        c = g;
    } else {
        s = sin(ku * zl);
        c = cos(ku * zl);
    }
    const double Bb = B0 * cosh(ku * yu) * s;
    const double Bz = B0 * sinh(ku * yu) * c;
    Bp[0] += -Bb * st;
    Bp[1] += Bb * ct;
    Bp[2] += Bz;
}

/* Window of the fringe fields inside a gap of length g (Eq. fringingFieldGap): 1 at the end of
   the module (dz = 0), about 6e-5 at the far end of the gap (dz = g). */
static double gap_window(double dz, double g)
{
    const double a = PI * dz / g;
    return 0.35875 + 0.48829 * cos(a) + 0.14128 * cos(2.0 * a) + 0.01168 * cos(3.0 * a);
}

/* Static undulator array (Sec. "Static Undulator Array Field"; Sec. UNDULATOR,
   static-undulator-array): n_modules planar modules of length L = n_periods lambda_u, module i
   starting at i (L + gap) with undulator parameter K_i = K + i taper.  Each module contributes
   the field of Eq. undulatorField in its own coordinate u (from its entrance) inside [0, L], and
   outside the fringe of Eq. fringingField with dz the distance to its nearer end: undamped where
   no module follows on that side (before the first entrance, after the last exit), damped by the
   window f(dz, gap) of Eq. fringingFieldGap inside a gap and zero beyond it.  The field is the
   sum over all modules.  Module i owns [0, L) of its coordinate and the last module [0, L]. */
static void array_field(const orc_run *r, double th, double xl, double yl, double zeta, double Bp[3])
{
    const double ku = r->ku, L = r->Lu, gap = r->p.gap;
    const int N = r->p.n_modules;
    const double ct = cos(th), st = sin(th);
    const double yu = -xl * st + yl * ct;
    for (int i = 0; i < N; ++i) {
        const double Ki = r->p.K + i * r->p.taper;
        const double B0i = 2.0 * PI * ME * C0 * Ki / (QE * r->p.lambda_u);
        const double u = zeta - i * (L + gap);
        double s = 0.0, c = 0.0;
        if (u >= 0.0 && (u < L || (i == N - 1 && u <= L))) {
            s = sin(ku * u);
            c = cos(ku * u);
        } else {
            const double dz = u < 0.0 ? u : u - L;
            const int open = u < 0.0 ? (i == 0) : (i == N - 1);
            if (open || fabs(dz) < gap) {
                const double e = exp(-0.5 * (ku * dz) * (ku * dz));
                const double w = open ? 1.0 : gap_window(dz, gap);
                s = ku * dz * e * w;
                c = e * w;
            }
        }
        const double Bb = B0i * cosh(ku * yu) * s;
        Bp[0] += -Bb * st;
        Bp[1] += Bb * ct;
        Bp[2] += B0i * sinh(ku * yu) * c;
    }
}

/* Time signature f(t, t0, phi) (Eq. signalTypes) with A0 = 1, t - t0 = tau. */
static double envelope_signal(const orc_run *r, double tau, double phase)
{
    const double w = C0 * r->kL;
    const double tp = r->p.pulse_fwhm / C0;
    const double carrier = cos(w * tau + phase);
    if (r->p.signal == 1 && tau > 0.0) return carrier;
    if (tp <= 0.0) return carrier;
    return carrier * exp(-2.0 * log(2.0) * tau * tau / (tp * tp));
}

void orc_lab_field(const orc_run *r, double xl, double yl, double zeta, double tl, double Ep[3], double Bp[3])
{
    Ep[0] = Ep[1] = Ep[2] = 0.0;
    Bp[0] = Bp[1] = Bp[2] = 0.0;
    const double th = r->p.pol_deg * PI / 180.0;
    switch (r->p.und_kind) {
    case 0:
        planar_field(r, th, 0.0, xl, yl, zeta, Bp);
        break;
    case 1:
        planar_field(r, th, 0.0, xl, yl, zeta, Bp);
        planar_field(r, th + 0.5 * PI, 0.25 * r->p.lambda_u, xl, yl, zeta, Bp);
        break;
    case 4:
        array_field(r, th, xl, yl, zeta, Bp);
        break;
    case 2:
    case 3: {
        /* counter-propagating beam along -z, polarisation (cos th, sin th, 0) */
        const double ct = cos(th), st = sin(th);
        const double tau = (tl - r->t_f) + (zeta - r->zeta_f) / C0;
        double Epar, El = 0.0, Bl = 0.0;
        if (r->p.und_kind == 2 || r->p.waist <= 0.0) {
            Epar = r->E0 * envelope_signal(r, tau, 0.0);
        } else {
            const double w0 = r->p.waist, k0 = r->kL;
            const double zr = PI * w0 * w0 / r->p.lambda_u;
            const double l = -(zeta - r->zeta_f);
            const double w = w0 * sqrt(1.0 + (l / zr) * (l / zr));
            const double rpar = xl * ct + yl * st, rperp = -xl * st + yl * ct;
            const double r2 = rpar * rpar + rperp * rperp;
            const double curv = (l == 0.0) ? 0.0 : k0 * r2 / (2.0 * l * (1.0 + (zr / l) * (zr / l)));
            const double gouy = atan(l / zr);
            const double amp = (w0 / w) * exp(-r2 / (w * w));
            Epar = r->E0 * amp * envelope_signal(r, tau, -curv + gouy);
            El = r->E0 * rpar * w0 / (zr * w) * amp * envelope_signal(r, tau, -curv + 2.0 * gouy + 0.5 * PI);
            Bl = r->E0 * rperp * w0 / (C0 * zr * w) * amp * envelope_signal(r, tau, -curv + 2.0 * gouy + 0.5 * PI);
        }
        Ep[0] = Epar * ct;
        Ep[1] = Epar * st;
        Ep[2] = -El;
        Bp[0] = Epar * st / C0;
        Bp[1] = -Epar * ct / C0;
        Bp[2] = -Bl;
        break;
    }
    default:
        break;
    }
}

void orc_external_field(const orc_run *r, double x, double y, double z, double t, double E[3], double B[3])
{
    const double g0 = r->gamma0, b0 = r->beta0;
    if (r->p.und_kind < 0) {
        E[0] = E[1] = E[2] = B[0] = B[1] = B[2] = 0.0;
        return;
    }
    /* rest -> lab event (Eq. LorentzTransformR2L, with the time coordinate) */
    const double zeta = g0 * (z + b0 * C0 * t);
    const double tl = g0 * (t + b0 * z / C0);
    double Ep[3], Bp[3];
    orc_lab_field(r, x, y, zeta, tl, Ep, Bp);
    /* E = g0 (E' + c b0 z x B') - (g0 - 1) E'_z z ;  B = g0 (B' - b0 z x E' / c) - (g0 - 1) B'_z z */
    E[0] = g0 * (Ep[0] - C0 * b0 * Bp[1]);
    E[1] = g0 * (Ep[1] + C0 * b0 * Bp[0]);
    E[2] = g0 * Ep[2] - (g0 - 1.0) * Ep[2];
    B[0] = g0 * (Bp[0] + b0 * Ep[1] / C0);
    B[1] = g0 * (Bp[1] - b0 * Ep[0] / C0);
    B[2] = g0 * Bp[2] - (g0 - 1.0) * Bp[2];
}

/* ------------------------------------------------------------------------- */
/* Boris scheme (Eq. BorisScheme), electron charge -e.                       */
/* ------------------------------------------------------------------------- */

void orc_boris(double u[3], const double E[3], const double B[3], double dtb)
{
    const double h = QE * dtb / (2.0 * ME * C0);
    double t1[3], t2[3], t3[3];
    for (int l = 0; l < 3; ++l) t1[l] = u[l] - h * E[l];
    const double alpha = -QE * dtb / (2.0 * ME * sqrt(1.0 + t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]));
    t2[0] = t1[0] + alpha * (t1[1] * B[2] - t1[2] * B[1]);
    t2[1] = t1[1] + alpha * (t1[2] * B[0] - t1[0] * B[2]);
    t2[2] = t1[2] + alpha * (t1[0] * B[1] - t1[1] * B[0]);
    const double f = 2.0 * alpha / (1.0 + alpha * alpha * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]));
    t3[0] = t1[0] + f * (t2[1] * B[2] - t2[2] * B[1]);
    t3[1] = t1[1] + f * (t2[2] * B[0] - t2[0] * B[2]);
    t3[2] = t1[2] + f * (t2[0] * B[1] - t2[1] * B[0]);
    for (int l = 0; l < 3; ++l) u[l] = t3[l] - h * E[l];
}

/* ------------------------------------------------------------------------- */
/* Gather (Eq. fieldInterpolation, linear weights) and deposition            */
/* (Sec. "Current Deposition", Umeda zigzag).                                */
/* ------------------------------------------------------------------------- */

/* cell coordinates of a position given relative to node (0,0,0) */
static void cellpos(const orc_run *r, const double *pos, double X[3])
{
    X[0] = pos[0] / r->dx;
    X[1] = pos[1] / r->dy;
    X[2] = pos[2] / r->dz;
}

static int active(const orc_run *r, const double X[3])
{
    const int n[3] = {r->nx, r->ny, r->nz};
    for (int a = 0; a < 3; ++a) {
        const double f = floor(X[a]);
        if (!(f >= 1.0 && f <= (double)(n[a] - 3))) return 0;
    }
    return 1;
}

static void gather(const orc_run *r, const double X[3], double E[3], double B[3])
{
    const int i = (int)floor(X[0]), j = (int)floor(X[1]), k = (int)floor(X[2]);
    const double f[3] = {X[0] - i, X[1] - j, X[2] - k};
    double out[6] = {0, 0, 0, 0, 0, 0};
    for (int K = 0; K < 2; ++K)
        for (int J = 0; J < 2; ++J)
            for (int I = 0; I < 2; ++I) {
                const double w = (I ? f[0] : 1.0 - f[0]) * (J ? f[1] : 1.0 - f[1]) * (K ? f[2] : 1.0 - f[2]);
                const int64_t id = IDX(r, i + I, j + J, k + K);
                for (int c = 0; c < 6; ++c) out[c] += w * r->eb[c][id];
            }
    for (int c = 0; c < 3; ++c) {
        E[c] = out[c];
        B[c] = out[3 + c];
    }
}

/* Straight piece a -> b (cell units) inside cell `cell`.  Only nodes of the z planes
   klo <= k < khi are written (a thread of the deposition owns those planes). */
static void deposit_piece(orc_run *r, const double a[3], const double b[3], const int cell[3], int klo, int khi)
{
    const double D[3] = {r->dx, r->dy, r->dz};
    double la[3], lb[3], mid[3], d[3];
    for (int l = 0; l < 3; ++l) {
        la[l] = a[l] - cell[l];
        lb[l] = b[l] - cell[l];
        mid[l] = 0.5 * (la[l] + lb[l]);
        d[l] = lb[l] - la[l];
    }
    for (int l = 0; l < 3; ++l) {
        const int m = (l + 1) % 3, n = (l + 2) % 3;
        /* current density on the edges parallel to axis l: q * (displacement along l) /
           (transverse cell area * dt), times the path average of the two linear weights */
        const double F = r->q * d[l] / (D[m] * D[n] * r->dt);
        for (int Jm = 0; Jm < 2; ++Jm)
            for (int Jn = 0; Jn < 2; ++Jn) {
                const double wm = Jm ? mid[m] : 1.0 - mid[m];
                const double wn = Jn ? mid[n] : 1.0 - mid[n];
                const double sm = Jm ? 1.0 : -1.0, sn = Jn ? 1.0 : -1.0;
                const double W = wm * wn + sm * sn * d[m] * d[n] / 12.0;
                int idx[3] = {cell[0], cell[1], cell[2]};
                idx[m] += Jm;
                idx[n] += Jn;
                if (idx[2] >= klo && idx[2] < khi) r->src[l][IDX(r, idx[0], idx[1], idx[2])] += F * W;
            }
    }
}

static void zigzag(orc_run *r, const double A[3], const double Bp[3], int klo, int khi)
{
    int c1[3], c2[3];
    double R[3];
    for (int l = 0; l < 3; ++l) {
        c1[l] = (int)floor(A[l]);
        c2[l] = (int)floor(Bp[l]);
        const double lo = (double)(c1[l] < c2[l] ? c1[l] : c2[l]);
        const double hi = (double)(c1[l] > c2[l] ? c1[l] : c2[l]);
        const double mid = 0.5 * (A[l] + Bp[l]);
        R[l] = fmin(lo + 1.0, fmax(hi, mid));
    }
    deposit_piece(r, A, R, c1, klo, khi);
    deposit_piece(r, R, Bp, c2, klo, khi);
}

static void deposit_move(orc_run *r, const double X1[3], const double X2[3], int klo, int khi)
{
    double m = 0.0;
    for (int l = 0; l < 3; ++l) m = fmax(m, fabs(X2[l] - X1[l]));
    const int ns = m > 1.0 ? (int)ceil(m) : 1;
    double A[3], B[3];
    for (int s = 0; s < ns; ++s) {
        for (int l = 0; l < 3; ++l) {
            A[l] = (s == 0) ? X1[l] : X1[l] + (X2[l] - X1[l]) * ((double)s / ns);
            B[l] = (s == ns - 1) ? X2[l] : X1[l] + (X2[l] - X1[l]) * ((double)(s + 1) / ns);
        }
        zigzag(r, A, B, klo, khi);
    }
}

static void deposit_rho(orc_run *r, const double X[3], int klo, int khi)
{
    const int i = (int)floor(X[0]), j = (int)floor(X[1]), k = (int)floor(X[2]);
    const double f[3] = {X[0] - i, X[1] - j, X[2] - k};
    const double rho = r->q / (r->dx * r->dy * r->dz);
    for (int K = 0; K < 2; ++K)
        for (int J = 0; J < 2; ++J)
            for (int I = 0; I < 2; ++I) {
                const double w = (I ? f[0] : 1.0 - f[0]) * (J ? f[1] : 1.0 - f[1]) * (K ? f[2] : 1.0 - f[2]);
                if (k + K >= klo && k + K < khi) r->src[3][IDX(r, i + I, j + J, k + K)] += rho * w;
            }
}

void orc_deposit_moves(orc_run *r, const double *old6, const double *new6, int64_t n)
{
    for (int c = 0; c < 4; ++c) memset(r->src[c], 0, (size_t)r->ncell * sizeof(double));
    for (int64_t p = 0; p < n; ++p) {
        double X1[3], X2[3];
        const double a[3] = {old6[6 * p] - r->x0, old6[6 * p + 1] - r->y0, old6[6 * p + 2] - r->z0};
        const double b[3] = {new6[6 * p] - r->x0, new6[6 * p + 1] - r->y0, new6[6 * p + 2] - r->z0};
        cellpos(r, a, X1);
        cellpos(r, b, X2);
        if (active(r, X1) && active(r, X2)) deposit_move(r, X1, X2, 0, r->nz);
        if (active(r, X2)) deposit_rho(r, X2, 0, r->nz);
    }
}

/* One particle's field step (external field, gather, Boris, move) for every sub-step, without
   depositing: the sub-step's end points in cell units go to X (N + 1 points), whether the
   sub-step's move is deposited to dep (both ends active) and whether the final charge is to
   rest_ok.  The particle's position and momentum are updated in place. */
static void push_particle(const orc_run *r, double *s, int N, double *X, char *dep, char *rho_ok)
{
    double pos[3] = {s[0], s[1], s[2]}, u[3] = {s[3], s[4], s[5]};
    cellpos(r, pos, X);
    for (int m = 0; m < N; ++m) {
        const double t = r->T0 + ((double)r->step + 0.5) * r->dt + m * r->dtb;
        double E[3], B[3], Es[3] = {0, 0, 0}, Bs[3] = {0, 0, 0};
        const double *X1 = X + 3 * m;
        double *X2 = X + 3 * (m + 1);
        orc_external_field(r, r->x0 + pos[0], r->y0 + pos[1], r->z0 + pos[2], t, E, B);
        const int a1 = active(r, X1);
        if (a1) gather(r, X1, Es, Bs);
        for (int l = 0; l < 3; ++l) {
            E[l] += Es[l];
            B[l] += Bs[l];
        }
        orc_boris(u, E, B, r->dtb);
        const double g = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double np_[3];
        for (int l = 0; l < 3; ++l) np_[l] = pos[l] + C0 * r->dtb * u[l] / g;
        cellpos(r, np_, X2);
        dep[m] = (char)(a1 && active(r, X2));
        for (int l = 0; l < 3; ++l) pos[l] = np_[l];
    }
    *rho_ok = (char)(r->p.space_charge && active(r, X + 3 * N));
    s[0] = pos[0];
    s[1] = pos[1];
    s[2] = pos[2];
    s[3] = u[0];
    s[4] = u[1];
    s[5] = u[2];
}

/* Push every particle (independent of one another: several threads may share the loop), then
   deposit in particle order and, per particle, in sub-step order, as one serial loop would. */
static void push_deposit(orc_run *r)
{
    const int N = r->p.substeps > 0 ? r->p.substeps : 1;
    for (int c = 0; c < 4; ++c) memset(r->src[c], 0, (size_t)r->ncell * sizeof(double));
    const int64_t chunk = 65536;
    double *X = (double *)malloc((size_t)chunk * 3 * (N + 1) * sizeof(double));
    char *dep = (char *)malloc((size_t)chunk * (N + 1));
    for (int64_t p0 = 0; p0 < r->np; p0 += chunk) {
        const int64_t n = r->np - p0 < chunk ? r->np - p0 : chunk;
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; ++q)
            push_particle(r, r->pr + 6 * (p0 + q), N, X + q * 3 * (N + 1), dep + q * (N + 1), dep + q * (N + 1) + N);
        /* each thread adds to its own z planes only, visiting the particles in order: every
           node receives its terms in the order of one serial loop */
#pragma omp parallel
        {
            int klo = 0, khi = r->nz;
#ifdef _OPENMP
            const int nt = omp_get_num_threads(), t = omp_get_thread_num();
            klo = (int)((int64_t)r->nz * t / nt);
            khi = (int)((int64_t)r->nz * (t + 1) / nt);
#endif
            for (int64_t q = 0; q < n; ++q) {
                const double *Xq = X + q * 3 * (N + 1);
                for (int m = 0; m < N; ++m) {
                    if (!dep[q * (N + 1) + m]) continue;
                    /* a move from z1 to z2 writes the node planes floor(min) .. floor(max) + 1 */
                    const double z1 = Xq[3 * m + 2], z2 = Xq[3 * (m + 1) + 2];
                    if (floor(fmax(z1, z2)) + 1.0 < (double)klo || floor(fmin(z1, z2)) >= (double)khi) continue;
                    deposit_move(r, Xq + 3 * m, Xq + 3 * (m + 1), klo, khi);
                }
                if (dep[q * (N + 1) + N]) deposit_rho(r, Xq + 3 * N, klo, khi);
            }
        }
    }
    free(X);
    free(dep);
}

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* Radiated power: running DFT over the last M steps of E_perp, B_perp on the */
/* plane, cycle-averaged Poynting flux, Doppler factor to the lab frame.     */
/* ------------------------------------------------------------------------- */

static void power_sample(orc_run *r)
{
    const int nx = r->nx, ny = r->ny, M = r->M;
    const int64_t plane = (int64_t)nx * ny;
    const int slot = (int)(r->step % M);
    const double ts = ((double)r->step + 0.5) * r->dt;
    double *ring = r->ring + (int64_t)slot * 4 * plane;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int64_t id = IDX(r, i, j, r->kp), pl = (int64_t)j * nx + i;
            ring[0 * plane + pl] = r->eb[0][id];
            ring[1 * plane + pl] = r->eb[1][id];
            ring[2 * plane + pl] = r->eb[3][id];
            ring[3 * plane + pl] = r->eb[4][id];
        }
    r->ring_t[slot] = ts;
    double P = 0.0;
    if (r->step + 1 >= M) {
        for (int j = 1; j < ny - 1; ++j)
            for (int i = 1; i < nx - 1; ++i) {
                const int64_t pl = (int64_t)j * nx + i;
                double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
                for (int m = 0; m < M; ++m) {
                    const double ph = r->omega_h * r->ring_t[m];
                    const double cr = cos(ph), ci = -sin(ph);
                    for (int c = 0; c < 4; ++c) {
                        const double v = r->ring[((int64_t)m * 4 + c) * plane + pl];
                        re[c] += v * cr;
                        im[c] += v * ci;
                    }
                }
                for (int c = 0; c < 4; ++c) {
                    re[c] *= 2.0 / M;
                    im[c] *= 2.0 / M;
                }
                /* Re(Ex By* - Ey Bx*) */
                P += (re[0] * re[3] + im[0] * im[3]) - (re[1] * re[2] + im[1] * im[2]);
            }
        P *= r->dx * r->dy / (2.0 * MU0);
    }
    if (r->nser >= r->cap) {
        r->cap = r->cap ? 2 * r->cap : 1024;
        r->ser_p = (double *)realloc(r->ser_p, (size_t)r->cap * sizeof(double));
        r->ser_t = (double *)realloc(r->ser_t, (size_t)r->cap * sizeof(double));
        r->ser_e = (double *)realloc(r->ser_e, (size_t)r->cap * sizeof(double));
    }
    const double g0 = r->gamma0, b0 = r->beta0;
    const double zp = r->z0 + r->kp * r->dz;
    r->ser_p[r->nser] = g0 * g0 * (1.0 + b0) * (1.0 + b0) * P;
    r->ser_t[r->nser] = g0 * (r->T0 + ts + b0 * zp / C0);
    r->ser_e[r->nser] = r->eb[0][IDX(r, nx / 2, ny / 2, r->kp)];
    r->nser++;
}

/* Radiated-power spectrum (Sec. FEL-OUTPUT, radiation-power, the normalised-frequency sweep):
   at every frequency h_k the definition of power_sample with its own window M_k, each
   recomputed from the stored plane samples of the last M_k steps. */
static void spectrum_sample(orc_run *r)
{
    if (r->nf == 0) return;
    const int nx = r->nx, ny = r->ny, Mh = r->Mh;
    const int64_t plane = (int64_t)nx * ny;
    const int slot = (int)(r->step % Mh);
    const double ts = ((double)r->step + 0.5) * r->dt;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int64_t id = IDX(r, i, j, r->kp), pl = (int64_t)j * nx + i;
            r->hist[((int64_t)slot * 4 + 0) * plane + pl] = r->eb[0][id];
            r->hist[((int64_t)slot * 4 + 1) * plane + pl] = r->eb[1][id];
            r->hist[((int64_t)slot * 4 + 2) * plane + pl] = r->eb[3][id];
            r->hist[((int64_t)slot * 4 + 3) * plane + pl] = r->eb[4][id];
        }
    r->hist_t[slot] = ts;
    r->spec = (double *)realloc(r->spec, (size_t)(r->step + 1) * r->nf * sizeof(double));
    const double g0 = r->gamma0, b0 = r->beta0;
    for (int k = 0; k < r->nf; ++k) {
        const int M = r->Mk[k];
        const double w = r->hk[k] * C0 * r->kstar;
        double P = 0.0;
        if (r->step + 1 >= M) {
            for (int j = 1; j < ny - 1; ++j)
                for (int i = 1; i < nx - 1; ++i) {
                    const int64_t pl = (int64_t)j * nx + i;
                    double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
                    for (int m = 0; m < M; ++m) {
                        const int sl = (int)((r->step - m) % Mh);
                        const double ph = w * r->hist_t[sl];
                        for (int c = 0; c < 4; ++c) {
                            const double v = r->hist[((int64_t)sl * 4 + c) * plane + pl];
                            re[c] += v * cos(ph);
                            im[c] -= v * sin(ph);
                        }
                    }
                    for (int c = 0; c < 4; ++c) {
                        re[c] *= 2.0 / M;
                        im[c] *= 2.0 / M;
                    }
                    P += (re[0] * re[3] + im[0] * im[3]) - (re[1] * re[2] + im[1] * im[2]);
                }
            P *= r->dx * r->dy / (2.0 * MU0);
        }
        r->spec[r->step * r->nf + k] = g0 * g0 * (1.0 + b0) * (1.0 + b0) * P;
    }
}

/* Bunch sampling (Sec. BUNCH, bunch-sampling): mean and rms spread (population) of the
   rest-frame positions and normalised momenta, and of the lab Lorentz factor
   gamma0 (gamma + beta0 u_z) (Eq. LorentzTrasnformParticles inverted for the energy), over all
   particles, in two passes. */
static void bunch_sample(orc_run *r)
{
    if (r->p.bunch_every <= 0 || r->step % r->p.bunch_every != 0) return;
    if (r->nbs >= r->bcap) {
        r->bcap = r->bcap ? 2 * r->bcap : 256;
        r->bser = (double *)realloc(r->bser, (size_t)r->bcap * 15 * sizeof(double));
    }
    double *row = r->bser + r->nbs * 15;
    const double org[3] = {r->x0, r->y0, r->z0};
    double mean[7] = {0, 0, 0, 0, 0, 0, 0}, var[7] = {0, 0, 0, 0, 0, 0, 0};
    const int64_t n = r->np;
    for (int pass = 0; pass < 2; ++pass)
        for (int64_t p = 0; p < n; ++p) {
            const double *q = r->pr + 6 * p;
            double v[7];
            for (int a = 0; a < 3; ++a) v[a] = q[a] + org[a];
            for (int a = 0; a < 3; ++a) v[3 + a] = q[3 + a];
            const double g = sqrt(1.0 + q[3] * q[3] + q[4] * q[4] + q[5] * q[5]);
            v[6] = r->gamma0 * (g + r->beta0 * q[5]);
            for (int c = 0; c < 7; ++c) {
                if (pass == 0) mean[c] += v[c] / (double)n;
                else var[c] += (v[c] - mean[c]) * (v[c] - mean[c]) / (double)n;
            }
        }
    row[0] = r->T0 + ((double)r->step + 1.5) * r->dt;
    for (int a = 0; a < 6; ++a) {
        row[1 + a] = mean[a];
        row[7 + a] = sqrt(var[a]);
    }
    row[13] = mean[6];
    row[14] = sqrt(var[6]);
    r->nbs++;
}

/* ------------------------------------------------------------------------- */

void orc_step(orc_run *r, int64_t nsteps)
{
    for (int64_t s = 0; s < nsteps; ++s) {
        emit_eb(r);
        push_deposit(r);
        bunch_sample(r);
        for (int c = 0; c < 4; ++c) {
            if (c == 3 && !r->p.space_charge) continue;
            orc_stencil(r, c);
            tfsf(r, c);
            orc_mur(r, c);
        }
        power_sample(r);
        spectrum_sample(r);
        orc_rotate_levels(r);
        r->step++;
    }
}

void orc_info(const orc_run *r, double out[19])
{
    out[0] = r->gamma0;
    out[1] = r->beta0;
    out[2] = r->dx;
    out[3] = r->dy;
    out[4] = r->dz;
    out[5] = r->dt;
    out[6] = r->dtb;
    out[7] = r->A;
    out[8] = r->x0;
    out[9] = r->y0;
    out[10] = r->z0;
    out[11] = r->T0;
    out[12] = r->omega_h;
    out[13] = r->M;
    out[14] = r->kp;
    out[15] = r->z_ref;
    out[16] = r->q;
    out[17] = r->kstar;
    out[18] = r->kb;
}

static double *field_ptr(const orc_run *r, int which, int lev)
{
    if (which < 4) return r->lev[lev][which];
    if (which < 8) return r->src[which - 4];
    return r->eb[which - 8];
}

void orc_get_field(const orc_run *r, int which, int lev, double *out)
{
    memcpy(out, field_ptr(r, which, lev), (size_t)r->ncell * sizeof(double));
}

void orc_set_field(orc_run *r, int which, int lev, const double *in)
{
    memcpy(field_ptr(r, which, lev), in, (size_t)r->ncell * sizeof(double));
}

void orc_get_particles(const orc_run *r, double *out6)
{
    memcpy(out6, r->pr, (size_t)r->np * 6 * sizeof(double));
    for (int64_t p = 0; p < r->np; ++p) {
        out6[6 * p + 0] += r->x0;
        out6[6 * p + 1] += r->y0;
        out6[6 * p + 2] += r->z0;
    }
}

void orc_set_particles(orc_run *r, const double *rest6)
{
    memcpy(r->pr, rest6, (size_t)r->np * 6 * sizeof(double));
    for (int64_t p = 0; p < r->np; ++p) {
        r->pr[6 * p + 0] -= r->x0;
        r->pr[6 * p + 1] -= r->y0;
        r->pr[6 * p + 2] -= r->z0;
    }
}

int64_t orc_num_particles(const orc_run *r) { return r->np; }

int64_t orc_series(const orc_run *r, double *power_lab, double *t_lab, double *onaxis_ex)
{
    if (power_lab) memcpy(power_lab, r->ser_p, (size_t)r->nser * sizeof(double));
    if (t_lab) memcpy(t_lab, r->ser_t, (size_t)r->nser * sizeof(double));
    if (onaxis_ex) memcpy(onaxis_ex, r->ser_e, (size_t)r->nser * sizeof(double));
    return r->nser;
}

int64_t orc_spectrum(const orc_run *r, double *h_out, double *p_lab)
{
    if (h_out && r->nf) memcpy(h_out, r->hk, (size_t)r->nf * sizeof(double));
    if (p_lab && r->nf) memcpy(p_lab, r->spec, (size_t)r->step * r->nf * sizeof(double));
    return r->nf ? r->step : 0;
}

int64_t orc_bunch_series(const orc_run *r, double *out)
{
    if (out && r->nbs) memcpy(out, r->bser, (size_t)r->nbs * 15 * sizeof(double));
    return r->nbs;
}

/* Neumaier summation */
static void nsum(double *s, double *comp, double v)
{
    const double t = *s + v;
    if (fabs(*s) >= fabs(v)) *comp += (*s - t) + v;
    else *comp += (v - t) + *s;
    *s = t;
}

void orc_diag(const orc_run *r, double *field_energy, double *bunching)
/* bunching[0] = |<exp(j kb z)>|, bunching[1..2] = its real and imaginary parts */
{
    if (field_energy) {
        double s = 0, cs = 0;
        const double e0 = eps0();
        for (int64_t id = 0; id < r->ncell; ++id) {
            const double e2 = r->eb[0][id] * r->eb[0][id] + r->eb[1][id] * r->eb[1][id] + r->eb[2][id] * r->eb[2][id];
            const double b2 = r->eb[3][id] * r->eb[3][id] + r->eb[4][id] * r->eb[4][id] + r->eb[5][id] * r->eb[5][id];
            nsum(&s, &cs, 0.5 * e0 * e2 + 0.5 * b2 / MU0);
        }
        *field_energy = (s + cs) * r->dx * r->dy * r->dz;
    }
    if (bunching) {
        double re = 0, cre = 0, im = 0, cim = 0;
        for (int64_t p = 0; p < r->np; ++p) {
            const double ph = r->kb * (r->z0 + r->pr[6 * p + 2]);
            nsum(&re, &cre, cos(ph));
            nsum(&im, &cim, sin(ph));
        }
        re += cre;
        im += cim;
        const double n = r->np ? (double)r->np : 1.0;
        bunching[0] = sqrt(re * re + im * im) / n;
        bunching[1] = re / n;
        bunching[2] = im / n;
    }
}

/* ------------------------------------------------------------------------- */
/* Quasi-random bunch loading (Sec. "Electron Bunch Generation": Halton       */
/* numbers, Eqs. uniform1D, gaussian1D, gaussian2D, bunchingFactor,           */
/* negativeExponential; CSE edges of the uniform profile).                    */
/* ------------------------------------------------------------------------- */

static const unsigned PRIMES[20] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61, 67, 71};

double orc_halton(unsigned i, unsigned j)
{
    const unsigned p = PRIMES[i];
    double x = 0.0, scale = 1.0 / p;
    while (j > 0) {
        x += (double)(j % p) * scale;   /* digit d_m of j lands at p^-(m+1) */
        j /= p;
        scale /= p;
    }
    return 1.0 - x;
}

/* Base assignment (the manual leaves it open): transverse positions (Eq. gaussian2D) from the
   bases 2 and 3, transverse momenta from 5 and 7, the longitudinal position from 11 (and 13 for
   a Gaussian profile, Eq. gaussian1D), the longitudinal momentum spread from 17 and 19, the
   shot-noise amplitude and phase of slice s from 23 and 29 at index s + 1.  Particle p uses
   index p + 1 (index 0 is the same point in every base).  Uniform profile with CSE edges: of
   the n particles, n_u = round(n L / (L + sqrt(2 pi) w)) fill [-sig_z, sig_z] (L = 2 sig_z) by
   Eq. uniform1D, the others form a Gaussian of rms w with the same peak line density whose lower
   half is moved to the tail (-sig_z + z) and upper half to the head (sig_z + z). */
void orc_ellipsoid_bunch(const orc_ellipsoid *e, int64_t n, double *out6)
{
    const double L = 2.0 * e->sig[2];
    int64_t nu = n;
    if (e->uniform && e->cse_sigma > 0.0) nu = (int64_t)llround((double)n * L / (L + sqrt(2.0 * PI) * e->cse_sigma));
    const double uz0 = sqrt(e->gamma * e->gamma - 1.0);
    for (int64_t p = 0; p < n; ++p) {
        const unsigned j = (unsigned)(p + 1);
        double *q = out6 + 6 * p;
        const double r1 = sqrt(-2.0 * log(orc_halton(0, j))), a1 = 2.0 * PI * orc_halton(1, j);
        q[0] = e->sig[0] * r1 * cos(a1);
        q[1] = e->sig[1] * r1 * sin(a1);
        const double r2 = sqrt(-2.0 * log(orc_halton(2, j))), a2 = 2.0 * PI * orc_halton(3, j);
        q[3] = e->sig_u[0] * r2 * cos(a2);
        q[4] = e->sig_u[1] * r2 * sin(a2);
        double z;
        if (!e->uniform) {
            z = e->sig[2] * sqrt(-2.0 * log(orc_halton(4, j))) * cos(2.0 * PI * orc_halton(5, j));
        } else if (p < nu) {
            z = L * (orc_halton(4, j) - 0.5);
        } else {
            const unsigned je = (unsigned)(p - nu + 1);
            const double ze = e->cse_sigma * sqrt(-2.0 * log(orc_halton(4, je))) * cos(2.0 * PI * orc_halton(5, je));
            z = ze < 0.0 ? -e->sig[2] + ze : e->sig[2] + ze;
        }
        q[2] = z;
        q[5] = uz0 + e->sig_u[2] * sqrt(-2.0 * log(orc_halton(6, j))) * cos(2.0 * PI * orc_halton(7, j));
    }
    /* bunching (Eq. bunchingFactor, read in the lab before the boost): z -> z - (2 b / k) sin(k z + phi) */
    if (e->lambda_r > 0.0 && (e->bunching > 0.0 || e->shot_noise)) {
        const double k = 2.0 * PI / e->lambda_r;
        if (e->bunching > 0.0)
            for (int64_t p = 0; p < n; ++p) {
                double *z = out6 + 6 * p + 2;
                *z -= (2.0 * e->bunching / k) * sin(k * *z + e->bunching_phase);
            }
        if (e->shot_noise && n > 0) {
            /* slice s = floor(z / lambda_r) - s0: electrons N_e,s = charge_e n_s / n; amplitude
               sqrt(-2 ln x_s) / sqrt(N_e,s) (Eq. negativeExponential), phase 2 pi y_s */
            int64_t s0 = INT64_MAX, s1 = INT64_MIN;
            for (int64_t p = 0; p < n; ++p) {
                const int64_t s = (int64_t)floor(out6[6 * p + 2] / e->lambda_r);
                if (s < s0) s0 = s;
                if (s > s1) s1 = s;
            }
            const int64_t ns = s1 - s0 + 1;
            int64_t *cnt = (int64_t *)calloc((size_t)ns, sizeof(int64_t));
            for (int64_t p = 0; p < n; ++p) cnt[(int64_t)floor(out6[6 * p + 2] / e->lambda_r) - s0]++;
            for (int64_t p = 0; p < n; ++p) {
                double *z = out6 + 6 * p + 2;
                const int64_t s = (int64_t)floor(*z / e->lambda_r) - s0;
                const double ne = e->charge_e * (double)cnt[s] / (double)n;
                const double b = sqrt(-2.0 * log(orc_halton(8, (unsigned)(s + 1)))) / sqrt(ne);
                const double ph = 2.0 * PI * orc_halton(9, (unsigned)(s + 1));
                *z -= (2.0 * b / k) * sin(k * *z + ph);
            }
            free(cnt);
        }
    }
}
