"""Pins of the oracle's spectrum sweep and bunch sampling (Sec. FEL-OUTPUT, radiation-power with
minimum / maximum normalised frequency and number of frequency points; Sec. BUNCH,
bunch-sampling); and the seed injected through TF/SF planes (Sec. "Seed Field").

* spectrum: a forward plane wave in a transversely periodic NSFD box (c dt = dz, so the
  discrete wave is an exact one-cell shift per step) is a pure sampled cosine at the plane; the
  power at every swept frequency and every step is then a constant times |X_k(n)|^2, X_k(n) the
  normalised DFT of that cosine over the frequency's own window, summed directly from its
  samples here; the constant is the cycle-averaged flux of the existing single-frequency pin,
  and one frequency equal to the main diagnostic's reproduces its series;
* bunch sampling, free streaming (no external field, no space charge, a negligible charge): the
  transverse normalised
  momenta and the lab Lorentz factor reproduce the lab input bunch's statistics (the last one
  inverts the boost), the mean position advances by n c dt <beta> and the position spreads grow
  as the spread of r_0 + n c dt beta;
* seed: in one dimension (transversely periodic NSFD at c dt = dz, first-order Mur at normal
  incidence, both exact) a plane-wave pulse leaves the scattered-field planes at zero and the
  total-field region equal to the incident potential to rounding -- the test that fixes the
  signs of the TF/SF corrections; a paraxial Gaussian pulse in 3D leaks below 2 % into the
  scattered-field planes and follows the incident potential on the axis.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.helpers import C0, MU0, vacuum


def _plane_wave_run(nf_min, nf_max, nf_points, lam_cells=32, nz=160):
    nx, ny = 6, 5
    w = vacuum(nx, ny, nz, 3e-4, 2.5e-4, 1.0e-4, solver=0, space_charge=0)
    r0 = oracle.Run(oracle.params_from(w, periodic=(1, 1, 0)))
    dz = r0.info()["dz"]
    w = workloads.scaled(w, lambda_u=lam_cells * dz, plane_dist=0.3 * nz * dz, nf_min=nf_min,
                         nf_max=nf_max, nf_points=nf_points)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 0)))
    inf = r.info()
    k = 2 * math.pi / (lam_cells * dz)
    om = C0 * k
    a = 1.0e6
    z = inf["z0"] + np.arange(nz) * dz
    for lev, tt in ((0, 0.0), (1, inf["dt"])):
        Ax = (a / om) * np.sin(k * z - om * tt)
        r.set_field("Ax", lev, np.broadcast_to(Ax[:, None, None], (nz, ny, nx)))
    return r, w, inf, k, om, a


def test_spectrum_of_a_plane_wave():
    lam_cells = 32
    r, w, inf, k, om, a = _plane_wave_run(0.7, 1.3, 7, lam_cells)
    nsteps = int(inf["kp"]) - 8
    r.step(nsteps)
    h, p = r.spectrum()
    assert np.allclose(h, np.linspace(0.7, 1.3, 7), rtol=0, atol=1e-15)
    assert p.shape == (nsteps, 7)
    dt = inf["dt"]
    zp = inf["z0"] + inf["kp"] * inf["dz"]
    area = (w.nx - 2) * (w.ny - 2) * inf["dx"] * inf["dy"]
    ratios = []
    for kk, hk in enumerate(h):
        M = int(round(lam_cells / hk))
        wk = hk * om
        for n in range(M + 2, nsteps):
            m = np.arange(M)
            tm = (n - m + 0.5) * dt
            X = (2.0 / M) * np.sum(np.cos(k * zp - om * tm) * np.exp(-1j * wk * tm))
            if abs(X) > 0.05:
                ratios.append(p[n, kk] / abs(X) ** 2)
            else:
                assert abs(p[n, kk]) < 0.01 * a * a * area / (2 * MU0 * C0)
            if n < M - 1:
                assert p[n, kk] == 0.0
    ratios = np.array(ratios)
    assert len(ratios) > 500
    # the same constant at every frequency and step: the fields are an exact sampled cosine
    assert np.max(np.abs(ratios / ratios[0] - 1)) < 1e-9
    # and that constant is the cycle-averaged flux a^2/(2 mu0 c) of a unit DFT amplitude (the
    # difference quotients of the potentials reduce the amplitude by O((w dt)^2))
    assert abs(ratios[0] / (a * a / (2 * MU0 * C0) * area) - 1) < 0.025


def test_spectrum_point_equals_the_power_series():
    r, w, inf, k, om, a = _plane_wave_run(1.0, 1.0, 1)
    r.step(60)
    h, p = r.spectrum()
    ps, _, _ = r.series()
    assert h.tolist() == [1.0]
    assert np.max(np.abs(p[:, 0] - ps)) <= 1e-12 * np.max(np.abs(ps))


def test_bunch_sampling_free_streaming():
    base = workloads.WORKLOADS["undulator_24x24x96"]
    # a negligible charge: the current it deposits would otherwise act back through A
    w = workloads.scaled(base, und_kind=-1, space_charge=0, n_particles=3000, bunch_every=5,
                         sig_ux=0.05, sig_uy=0.03, rel_espread=2e-3, charge_e=1e-3)
    lab = workloads.lab_bunch(w)
    r = oracle.Run(oracle.params_from(w), lab)
    r.step(41)
    bs = r.bunch_series()
    assert bs.shape == (9, 15)   # steps 0, 5, ..., 40
    inf = r.info()
    dt = inf["dt"]
    assert np.allclose(bs[:, 0], inf["T0"] + (np.arange(9) * 5 + 1.5) * dt, rtol=1e-15, atol=0)
    # momenta do not change: transverse ones are the lab ones, the lab gamma inverts the boost
    g_lab = np.sqrt(1 + np.sum(lab[:, 3:] ** 2, axis=1))
    for row in bs:
        assert abs(row[4] - lab[:, 3].mean()) < 1e-15 and abs(row[5] - lab[:, 4].mean()) < 1e-15
        assert abs(row[10] - lab[:, 3].std()) < 1e-14 and abs(row[11] - lab[:, 4].std()) < 1e-14
        assert abs(row[13] - g_lab.mean()) < 1e-12 * g_lab.mean()
        assert abs(row[14] - g_lab.std()) < 1e-9 * g_lab.std()
    # positions stream: r_n = r_0 + n c dt u / gamma (rest frame, momenta fixed)
    rest = r.particles()
    u = rest[:, 3:]
    v = C0 * dt * u / np.sqrt(1 + np.sum(u * u, axis=1))[:, None]
    r0 = rest[:, :3] - 40 * v
    for i, row in enumerate(bs):
        rn = r0 + (5 * i) * v
        assert np.max(np.abs(row[1:4] - rn.mean(axis=0))) < 1e-12 * np.max(np.abs(rn))
        assert np.max(np.abs(row[7:10] - rn.std(axis=0)) / rn.std(axis=0)) < 1e-9


# ---- seed through TF/SF planes (Sec. "Seed Field") --------------------------------------------

def _seed_box(nx, ny, nz, seed_type, lam_cells, periodic, **kw):
    dz = 1.0e-4
    w = vacuum(nx, ny, nz, 2.0e-4, 2.0e-4, dz, solver=0, space_charge=0, mur_order=kw.pop("mur_order", 1))
    w = workloads.scaled(w, seed_type=seed_type, seed_a0=1e-3, seed_lambda=lam_cells * dz, **kw)
    return oracle.Run(oracle.params_from(w, periodic=periodic)), w


def test_plane_wave_seed_exact_in_one_dimension():
    """NSFD at c dt = dz shifts a z-only field by exactly one cell per step and first-order Mur is
    exact at normal incidence, so a plane-wave pulse injected through the TF/SF planes must leave
    the scattered-field planes (z index 0, 1) at zero and make the total-field region equal to
    the incident potential, node for node, to rounding."""
    nz = 160
    # the pulse centre starts 220 cells behind the domain, so the incident field inside the
    # domain at t = 0 is below 1e-32 of its amplitude (the run starts from zero fields)
    r, w = _seed_box(4, 4, nz, 0, 20, (1, 1, 0), seed_pulse_fwhm=30 * 1.0e-4,
                     seed_offset=300 * 1.0e-4, seed_pol_deg=30.0, seed_cep_deg=40.0)
    inf = r.info()
    assert inf["gamma0"] == 1.0 and inf["T0"] == 0.0
    A0 = 1e-3 * 9.1093837015e-31 * C0 / 1.602176634e-19
    peak = 0.0
    for s in range(1, 25):
        r.step(20)
        t = (r.info()["dt"]) * (20 * s + 1)     # level n+1 after 20 s steps
        for c in (0, 1):
            a = r.field(c, 1)
            z = inf["z0"] + np.arange(nz) * inf["dz"]
            f = np.array([r.seed_potential(inf["x0"] + 0.5 * inf["dx"] * (c == 0), inf["y0"], zz, t)[c]
                          for zz in z])
            assert np.max(np.abs(a[:2])) <= 1e-12 * A0
            assert np.max(np.abs(a[2:] - f[2:, None, None])) <= 1e-11 * A0, (s, c)
            peak = max(peak, float(np.max(np.abs(f))))
    assert peak > 0.5 * A0 * math.sin(math.radians(30.0))


def test_gaussian_seed_enters_the_total_field_region():
    """A paraxial Gaussian-beam pulse (k w0 = 4 pi, focus at the middle of the box) through the
    TF/SF planes: the scattered-field planes see only what the transverse boundaries and the
    omitted longitudinal potential leave (below 2 % of the incident amplitude), and the total
    field on the axis follows the incident potential within 10 % of its amplitude: at 8 cells
    per wavelength the NSFD dispersion scales the transverse (diffraction) term by
    1 - 4 A sin^2(k dz / 2) = 0.85, which shifts the Gouy phase by a few hundredths of a radian
    over the box (the exact one-dimensional pin above carries the injection's signs, time levels
    and coefficients)."""
    nx = ny = 40
    nz = 120
    dz = 1.0e-4
    r, w = _seed_box(nx, ny, nz, 1, 8, (0, 0, 0), seed_waist=16 * 2.0e-4, seed_focus=0.0,
                     seed_pulse_fwhm=30 * dz, seed_offset=220 * dz, mur_order=2)
    inf = r.info()
    A0 = 1e-3 * 9.1093837015e-31 * C0 / 1.602176634e-19
    r.step(220)
    t = inf["dt"] * 221
    a = r.field(0, 1)
    i0, j0 = nx // 2, ny // 2
    z = inf["z0"] + np.arange(nz) * inf["dz"]
    x = inf["x0"] + (i0 + 0.5) * inf["dx"]
    y = inf["y0"] + j0 * inf["dy"]
    f = np.array([r.seed_potential(x, y, zz, t)[0] for zz in z])
    assert np.max(np.abs(f)) > 0.5 * A0
    assert np.max(np.abs(a[:2])) < 0.02 * A0
    assert np.max(np.abs(a[4:nz - 4, j0, i0] - f[4:nz - 4])) < 0.10 * A0
