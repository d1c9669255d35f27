"""Pins of the oracle's static undulator array (Sec. "Static Undulator Array Field", Eq.
fringingFieldGap; Sec. UNDULATOR, static-undulator-array: K_i = K_0 + i dK).

* a one-module array is the single planar undulator (Eqs. undulatorField, fringingField);
* inside module i the peak field is B_0 K_i / K_0 at the positions i (L + g) + (m + 1/4) lambda_u;
* at the middle of a gap the exit fringe of module i and the entrance fringe of module i+1 are
  mirror images: the transverse field is (B_0,i - B_0,i+1) cosh(k_u y) k_u (g/2)
  exp(-(k_u g/2)^2/2) f(g/2, g) and the longitudinal one (B_0,i + B_0,i+1) sinh(k_u y)
  exp(-(k_u g/2)^2/2) f(g/2, g), with f(g/2, g) = 0.35875 - 0.14128 from the window's cosines at
  pi/2, pi, 3 pi/2;
* the field is continuous across every module end up to the window's residue at the far end of
  the gap (f(g, g) = 6e-5 times the neighbour's fringe there);
* div B' = 0 and curl B' = 0 inside the modules and div B' = 0 in the open fringes; inside a gap
  the window leaves div B' = B_0 sinh(k_u y) exp(-(k_u dz)^2/2) df/d(dz) per fringe (the printed
  gap field is not divergence-free), checked against that closed form;
* a single electron's normalised transverse momentum swings with amplitude K_i in module i
  (p_x / (m c) = -K_i cos(k_u z) in a planar undulator), and its lab energy stays constant.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.helpers import C0, ME, QE

LU = 0.02


def _array_run(K=1.2, n_periods=3, gap=0.75 * LU, n_modules=3, taper=0.1, gamma=30.0, **kw):
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, und_kind=4, K=K, gamma=gamma, lambda_u=LU, n_periods=n_periods,
                         gap=gap, n_modules=n_modules, taper=taper, n_particles=0, **kw)
    return oracle.Run(oracle.params_from(w)), w


def _B0(K):
    return 2 * math.pi * ME * C0 * K / (QE * LU)


def test_one_module_is_the_planar_undulator():
    ra, w = _array_run(n_modules=1, n_periods=7, taper=0.3, pol_deg=31.0)
    rp, _ = _array_run(n_modules=1, n_periods=7, taper=0.3, pol_deg=31.0)
    rp = oracle.Run(oracle.params_from(workloads.scaled(w, und_kind=0)))
    rng = np.random.default_rng(4)
    for zeta in rng.uniform(-3, 10, 200) * LU:
        x, y = rng.normal(0, 2e-3, 2)
        Ba = ra.lab_field(x, y, zeta, 0.0)[1]
        Bp = rp.lab_field(x, y, zeta, 0.0)[1]
        assert np.max(np.abs(Ba - Bp)) <= 1e-15 * _B0(1.2) * 10


def test_peak_field_of_each_module_follows_the_taper():
    K0, dK, g, L = 1.2, 0.1, 0.75 * LU, 3 * LU
    r, _ = _array_run(K=K0, taper=dK, gap=g)
    for i in range(3):
        for m in range(3):
            zeta = i * (L + g) + (m + 0.25) * LU
            B = r.lab_field(0.0, 0.0, zeta, 0.0)[1]
            assert abs(B[1] - _B0(K0 + i * dK)) < 1e-12 * _B0(K0)
            assert abs(B[0]) + abs(B[2]) < 1e-12 * _B0(K0)


@pytest.mark.parametrize("taper", [0.0, 0.15])
def test_gap_midpoint_closed_form(taper):
    K0, g, L = 1.2, 0.75 * LU, 3 * LU
    ku = 2 * math.pi / LU
    r, _ = _array_run(K=K0, taper=taper, gap=g)
    f_half = 0.35875 - 0.14128
    damp = math.exp(-0.5 * (ku * g / 2) ** 2)
    for i in range(2):
        zeta = i * (L + g) + L + g / 2
        for y in (0.0, 1.3e-3, -2.1e-3):
            B = r.lab_field(0.0, y, zeta, 0.0)[1]
            bi, bj = _B0(K0 + i * taper), _B0(K0 + (i + 1) * taper)
            By = (bi - bj) * math.cosh(ku * y) * ku * (g / 2) * damp * f_half
            Bz = (bi + bj) * math.sinh(ku * y) * damp * f_half
            assert abs(B[1] - By) < 1e-13 * _B0(K0), (i, y, B[1], By)
            assert abs(B[2] - Bz) < 1e-13 * _B0(K0), (i, y, B[2], Bz)
            assert B[0] == 0.0


def test_field_continuous_at_module_ends():
    K0, g, L = 1.2, 0.75 * LU, 3 * LU
    ku = 2 * math.pi / LU
    r, _ = _array_run(K=K0, taper=0.1, gap=g)
    # the neighbour's windowed fringe at the far end of the gap: f(g, g) < 6e-5 times the fringe
    # shape, k_u g exp(-(k_u g)^2/2) for the transverse and exp(-(k_u g)^2/2) for the
    # longitudinal component
    resid = 6e-5 * max(1.0, ku * g) * math.exp(-0.5 * (ku * g) ** 2) * 1.5
    h = 1e-12
    for i in range(3):
        for end in (i * (L + g), i * (L + g) + L):
            for y in (0.0, 1.7e-3):
                Bm = r.lab_field(0.0, y, end - h, 0.0)[1]
                Bp = r.lab_field(0.0, y, end + h, 0.0)[1]
                scale = _B0(K0 + 2 * 0.1) * math.cosh(ku * y)
                assert np.max(np.abs(Bm - Bp)) < (resid + 1e-9) * scale, (i, end, Bm, Bp)


def test_div_and_curl():
    """Inside the modules and in the open fringes div B' = curl B' = 0 (curl only inside).  In a
    gap the window breaks the divergence-free form: with B_y = B_0 cosh(k_u y) k_u dz e f and
    B_z = B_0 sinh(k_u y) e f (e = exp(-(k_u dz)^2/2)), dB_y/dy + dB_z/dz = B_0 sinh(k_u y) e
    df/d(dz) for each of the two fringes, dz signed from the module's end."""
    K0, dK, L, g = 1.2, 0.1, 3 * LU, 0.75 * LU
    r, _ = _array_run(K=K0, taper=dK, gap=g, pol_deg=23.0)
    th = math.radians(23.0)
    h = 1e-6
    ku = 2 * math.pi / LU

    def fprime(dz):
        a = math.pi / g
        return -a * (0.48829 * math.sin(a * dz) + 2 * 0.14128 * math.sin(2 * a * dz)
                     + 3 * 0.01168 * math.sin(3 * a * dz))

    rng = np.random.default_rng(11)
    zs = np.concatenate([rng.uniform(-2, 13, 40) * LU,
                         [i * (L + g) + L + f * g for i in range(2) for f in (0.2, 0.5, 0.8)]])
    for zeta in zs:
        x, y = rng.normal(0, 1e-3, 2)

        def Bf(dx_, dy_, dz_):
            return r.lab_field(x + dx_, y + dy_, zeta + dz_, 0.0)[1]

        d = [(Bf(h, 0, 0) - Bf(-h, 0, 0)) / (2 * h), (Bf(0, h, 0) - Bf(0, -h, 0)) / (2 * h),
             (Bf(0, 0, h) - Bf(0, 0, -h)) / (2 * h)]
        div = d[0][0] + d[1][1] + d[2][2]
        expect = 0.0
        i = int(zeta // (L + g))
        u = zeta - i * (L + g)
        if 0 <= i < 2 and L < u < L + g:   # gap between modules i and i + 1
            yu = -x * math.sin(th) + y * math.cos(th)
            for side, dz in ((i, u - L), (i + 1, u - L - g)):
                e = math.exp(-0.5 * (ku * dz) ** 2)
                expect += _B0(K0 + side * dK) * math.sinh(ku * yu) * e * fprime(dz)
        assert abs(div - expect) < 1e-5 * _B0(1.4) * ku, (zeta, div, expect)
        if 0 <= i < 3 and 0.05 * LU < u < L - 0.05 * LU:
            curl = np.array([d[1][2] - d[2][1], d[2][0] - d[0][2], d[0][1] - d[1][0]])
            assert np.max(np.abs(curl)) < 1e-5 * _B0(1.4) * ku


def test_single_electron_momentum_swing_per_module():
    gamma, K0, dK, npm, g = 20.0, 1.0, 0.2, 3, 1.5 * 0.03
    lu = 0.03
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, n_particles=1, charge_e=1.0, gamma=gamma, und_kind=4, K=K0,
                         lambda_u=lu, n_periods=npm, gap=g, n_modules=3, taper=dK, space_charge=0)
    lab = np.array([[0.0, 0.0, 0.0, 0.0, 0.0, math.sqrt(gamma * gamma - 1)]])
    r = oracle.Run(oracle.params_from(w), lab)
    inf = r.info()
    g0, b0, dt = inf["gamma0"], inf["beta0"], inf["dt"]
    L = npm * lu
    tr = []
    for _ in range(820):
        r.step(1)
        tr.append(r.particles()[0].copy())
    tr = np.array(tr)
    n = np.arange(len(tr)) + 1
    t = inf["T0"] + (n + 0.5) * dt
    zeta = g0 * (tr[:, 2] + b0 * C0 * t)
    assert zeta[-1] > 3 * L + 2 * g + 0.5 * lu
    u = tr[:, 3:]
    glab = g0 * (np.sqrt(1 + np.sum(u * u, axis=1)) + b0 * u[:, 2])
    assert np.max(np.abs(glab - gamma)) / gamma < 1e-3
    for i in range(3):
        a = i * (L + g)
        sel = (zeta > a + 0.2 * lu) & (zeta < a + L - 0.2 * lu)
        assert sel.sum() > 60
        swing = 0.5 * (u[sel, 0].max() - u[sel, 0].min())
        assert abs(swing - (K0 + i * dK)) < 0.01 * K0, (i, swing)
