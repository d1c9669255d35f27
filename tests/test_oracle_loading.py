"""Pins of the oracle's quasi-random bunch loading (Sec. "Electron Bunch Generation": Halton
numbers, Eqs. uniform1D, gaussian1D, gaussian2D; the Gaussian CSE edges of a uniform profile;
Eqs. bunchingFactor, negativeExponential read as G8).

* Halton numbers are one minus the radical inverse: base 2 gives 1/2, 3/4, 1/4, 7/8, 3/8, ...
  and base 3 gives 2/3, 1/3, 8/9, 5/9, ... (digit reversal by hand); the first p^k indices in
  base p fill the grid {m / p^k} exactly;
* quasi-random filling: the sample moments of 2^14 Gaussian particles are far closer to the
  target than random sampling would give (1/sqrt(N)), and the bunching of an unmodulated bunch
  at an arbitrary wavelength is far below the random level 1/sqrt(N) (the manual's point:
  no spurious initial bunching);
* uniform profile with CSE edges: a flat line density over [-sig_z, sig_z] joined to
  Gaussian edges of the same peak density, with the particle split of the two parts;
* an imposed bunching factor b is recovered at the wavelength to first order.
"""
import math

import numpy as np

import oracle


def _ell(**kw):
    e = oracle.Ellipsoid()
    e.uniform = kw.get("uniform", 0)
    e.gamma = kw.get("gamma", 100.0)
    for a, v in enumerate(kw.get("sig", (50e-6, 40e-6, 7e-6))):
        e.sig[a] = v
    for a, v in enumerate(kw.get("sig_u", (0.02, 0.03, 0.01))):
        e.sig_u[a] = v
    e.cse_sigma = kw.get("cse_sigma", 0.0)
    e.lambda_r = kw.get("lambda_r", 0.0)
    e.bunching = kw.get("bunching", 0.0)
    e.bunching_phase = kw.get("bunching_phase", 0.0)
    e.shot_noise = kw.get("shot_noise", 0)
    e.charge_e = kw.get("charge_e", 1e9)
    return e


def test_halton_values_by_hand():
    base2 = [0.5, 0.75, 0.25, 0.875, 0.375, 0.625, 0.125]
    base3 = [2 / 3, 1 / 3, 8 / 9, 5 / 9, 2 / 9, 7 / 9, 4 / 9]
    assert [oracle.halton(0, j) for j in range(1, 8)] == base2
    assert max(abs(oracle.halton(1, j) - v) for j, v in zip(range(1, 8), base3)) < 3e-16
    assert oracle.halton(4, 0) == 1.0


def test_halton_first_power_of_the_base_is_a_grid():
    for i, p, k in ((0, 2, 12), (1, 3, 7), (2, 5, 5), (5, 13, 3)):
        N = p ** k
        v = np.sort([1.0 - oracle.halton(i, j) for j in range(N)])
        assert np.max(np.abs(v - np.arange(N) / N)) < 1e-15


def test_gaussian_moments_are_quasi_random():
    N = 1 << 14
    b = oracle.ellipsoid_bunch(_ell(), N)
    sig = (50e-6, 40e-6, 7e-6)
    for a in range(3):
        assert abs(b[:, a].mean()) < 0.02 * sig[a] / math.sqrt(N) * 10
        assert abs(b[:, a].std() / sig[a] - 1) < 2e-3          # random: ~ 1 / sqrt(2 N) = 5.5e-3
    sig_u = (0.02, 0.03)
    for a in range(2):
        assert abs(b[:, 3 + a].std() / sig_u[a] - 1) < 2e-3
    assert abs(b[:, 5].mean() - math.sqrt(100.0 ** 2 - 1)) < 1e-3 * 0.01
    # no spurious bunching: averaged over wavelengths shorter than the bunch, |<exp(i k z)>|
    # minus the profile's own form factor stays far below the random level 1 / sqrt(N) (random
    # loading averages about 0.9 of it)
    lams = np.geomspace(0.5e-6, 20e-6, 30)
    excess = [abs(np.mean(np.exp(2j * math.pi * b[:, 2] / lam))) - math.exp(-0.5 * (2 * math.pi * 7e-6 / lam) ** 2)
              for lam in lams]
    assert np.mean(excess) * math.sqrt(N) < 0.4


def test_uniform_profile_with_cse_edges():
    N = 1 << 15
    sz, w = 50e-6, 1.5e-6
    b = oracle.ellipsoid_bunch(_ell(uniform=1, sig=(30e-6, 30e-6, sz), cse_sigma=w), N)
    z = b[:, 2]
    L = 2 * sz
    nu = round(N * L / (L + math.sqrt(2 * math.pi) * w))
    inside = np.abs(z) <= sz
    assert abs(inside.sum() - (nu + 0)) <= (N - nu) * 0.01 + 2
    # flat line density in the middle equal to the edges' peak density
    h, edges = np.histogram(z, bins=40, range=(-sz, sz))
    dens = h / (edges[1] - edges[0])
    assert np.max(np.abs(dens / (nu / L) - 1)) < 0.01
    head = z[z > sz] - sz
    tail = sz + z[z < -sz]
    assert abs(len(head) - len(tail)) <= 0.01 * (len(head) + len(tail))
    for part in (head, -tail):
        assert abs(np.sqrt(np.mean(part ** 2)) / w - 1) < 0.02     # half-Gaussians of rms w
    # the quasi-random uniform bunch starts without bunching: at wavelengths of the order of the
    # edges (0.5 .. 2 um) at most 0.4 and on average 0.15 of the random level 1/sqrt(N)
    lev = [abs(np.mean(np.exp(2j * math.pi * z / lam))) * math.sqrt(N) for lam in np.geomspace(0.5e-6, 2e-6, 15)]
    assert max(lev) < 0.4 and np.mean(lev) < 0.15


def test_imposed_bunching_is_recovered():
    N = 1 << 14
    lam = 1.0e-6
    b = oracle.ellipsoid_bunch(_ell(uniform=1, sig=(30e-6, 30e-6, 20e-6), lambda_r=lam, bunching=0.05,
                                    bunching_phase=0.7), N)
    B = np.mean(np.exp(1j * 2 * math.pi * b[:, 2] / lam))
    assert abs(abs(B) - 0.05) < 0.002
