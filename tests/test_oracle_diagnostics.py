"""Pins of the oracle's spectrum sweep and bunch sampling (Sec. FEL-OUTPUT, radiation-power with
minimum / maximum normalised frequency and number of frequency points; Sec. BUNCH,
bunch-sampling).

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
  as the spread of r_0 + n c dt beta.
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
