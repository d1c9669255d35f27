"""Pins of the oracle's particle side and of the coupled step.

* Boris (Eq. BorisScheme): exact |u| conservation and the exact rotation angle
  2 atan(e B dt / (2 m gamma)) in a pure magnetic field; exact linear momentum gain in
  a pure electric field;
* discrete charge continuity (rho^{n+3/2} - rho^{n+1/2})/dt + div J^{n+1} = 0 at every node,
  and the total current moment sum J dV = q sum dr / dt;
* external field: Lorentz invariants E.B and E^2 - c^2 B^2 of the transformed field, the
  rest-frame on-axis values, div B' = 0 everywhere and curl B' = 0 inside the undulator,
  the Gaussian beam tending to the plane wave for a large waist;
* zigzag current of a move that stays in its cell: on each of the cell's 12 edges the current
  is q D_l / (V dt) times the path average of the two transverse linear weights along the
  straight move, the average taken here by Gauss-Legendre quadrature (the relay point of such a
  move is its midpoint, so the two zigzag pieces are the halves of one segment);
* particle boost: the inverse Lorentz transform recovers the lab particles;
* Lorentz gauge: with charge-conserving deposition the gauge residual G evolves as a
  source-free field (the manual's claim that the gauge holds automatically).
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.helpers import C0, EPS0, ME, MU0, QE, vacuum


def test_boris_pure_magnetic_rotation():
    B = np.array([0.3, -0.2, 1.1])
    u = np.array([2.0, -1.0, 0.5])
    g = math.sqrt(1 + u @ u)
    dt = 1e-12
    Bm = np.linalg.norm(B)
    theta = 2 * math.atan(QE * Bm * dt / (2 * ME * g))
    bh = B / Bm
    upar = (u @ bh) * bh
    u0p = u - upar
    cur = u.copy()
    n = 500
    for _ in range(n):
        cur = oracle.boris(cur, np.zeros(3), B, dt)
    assert abs(np.linalg.norm(cur) - np.linalg.norm(u)) < 1e-13 * np.linalg.norm(u)
    uperp = cur - (cur @ bh) * bh
    ang = math.atan2(np.cross(u0p, uperp) @ bh, u0p @ uperp)
    # electrons rotate in the positive sense about B
    expect = math.remainder(n * theta, 2 * math.pi)
    assert abs(math.remainder(ang - expect, 2 * math.pi)) < 1e-10


def test_boris_pure_electric_exact():
    E = np.array([1e9, -2e8, 5e8])
    u = np.array([0.1, 0.2, -0.3])
    dt = 3e-13
    cur = u.copy()
    for _ in range(100):
        cur = oracle.boris(cur, E, np.zeros(3), dt)
    exp = u - 100 * QE * dt * E / (ME * C0)
    assert np.max(np.abs(cur - exp)) < 1e-12 * np.max(np.abs(exp))


def _div_J(r, J, dx, dy, dz):
    Jx, Jy, Jz = J
    d = np.zeros_like(Jx)
    d[:, :, 1:] += (Jx[:, :, 1:] - Jx[:, :, :-1]) / dx
    d[:, :, 0] += Jx[:, :, 0] / dx
    d[:, 1:, :] += (Jy[:, 1:, :] - Jy[:, :-1, :]) / dy
    d[:, 0, :] += Jy[:, 0, :] / dy
    d[1:, :, :] += (Jz[1:, :, :] - Jz[:-1, :, :]) / dz
    d[0, :, :] += Jz[0, :, :] / dz
    return d


@pytest.mark.parametrize("maxmove", [0.4, 0.99, 2.7])
def test_charge_continuity_and_current_moment(maxmove):
    nx, ny, nz = 16, 14, 18
    dx, dy, dz = 1.1e-3, 0.9e-3, 1.3e-3
    w = vacuum(nx, ny, nz, dx, dy, dz, solver=1, courant=0.5)
    w = workloads.scaled(w, charge_e=1e6)
    rng = np.random.default_rng(11)
    n = 300
    lab = np.zeros((n, 6))
    r = oracle.Run(oracle.params_from(w), lab)
    inf = r.info()
    x0, y0, z0, dt = inf["x0"], inf["y0"], inf["z0"], inf["dt"]
    D = np.array([dx, dy, dz])
    lo = np.array([x0, y0, z0]) + 4 * D
    hi = np.array([x0 + (nx - 5) * dx, y0 + (ny - 5) * dy, z0 + (nz - 5) * dz])
    old = np.zeros((n, 6))
    old[:, :3] = lo + rng.random((n, 3)) * (hi - lo)
    new = old.copy()
    new[:, :3] += (rng.random((n, 3)) * 2 - 1) * maxmove * D
    # some particles exactly on nodes / crossing exactly at nodes
    old[:5, :3] = np.array([x0, y0, z0]) + np.array([6, 7, 8]) * D
    r.deposit_moves(old, old)
    rho0 = r.field("rho")
    r.deposit_moves(old, new)
    rho1 = r.field("rho")
    J = [r.field("Jx"), r.field("Jy"), r.field("Jz")]
    res = (rho1 - rho0) / dt + _div_J(r, J, dx, dy, dz)
    scale = np.max(np.abs(rho1)) / dt
    assert np.max(np.abs(res)) < 1e-12 * scale, np.max(np.abs(res)) / scale
    q = inf["q"]
    vol = dx * dy * dz
    for l, name in enumerate(("Jx", "Jy", "Jz")):
        moment = np.sum(J[l]) * vol
        expect = q * np.sum(new[:, l] - old[:, l]) / dt
        assert abs(moment - expect) < 1e-11 * abs(q * maxmove * D[l] * n / dt)
    assert abs(np.sum(rho1) * vol - q * n) < 1e-12 * abs(q * n)


def test_zigzag_current_of_a_move_inside_one_cell():
    nx, ny, nz = 12, 11, 13
    D = np.array([1.1e-3, 0.9e-3, 1.3e-3])
    w = vacuum(nx, ny, nz, *D, solver=1, courant=0.5)
    w = workloads.scaled(w, charge_e=1e6)
    r = oracle.Run(oracle.params_from(w), np.zeros((1, 6)))
    inf = r.info()
    org = np.array([inf["x0"], inf["y0"], inf["z0"]])
    q, dt, vol = inf["q"], inf["dt"], float(np.prod(D))
    tq, wq = np.polynomial.legendre.leggauss(4)   # exact for the quadratic integrands
    tq, wq = 0.5 * (tq + 1.0), 0.5 * wq
    rng = np.random.default_rng(5)
    names = ("Jx", "Jy", "Jz")
    for trial in range(20):
        cell = rng.integers(4, 7, 3)
        fa = rng.uniform(0.02, 0.98, 3)
        fb = np.clip(fa + rng.uniform(-0.5, 0.5, 3), 0.01, 0.99)
        old = np.zeros((1, 6))
        new = np.zeros((1, 6))
        old[0, :3] = org + (cell + fa) * D
        new[0, :3] = org + (cell + fb) * D
        r.deposit_moves(old, new)
        J = [r.field(n) for n in names]
        path = fa[None, :] + tq[:, None] * (fb - fa)[None, :]   # offsets along the move
        for l in range(3):
            m, n = (l + 1) % 3, (l + 2) % 3
            pre = q * (fb[l] - fa[l]) * D[l] / (vol * dt)
            got = np.zeros((2, 2))
            want = np.zeros((2, 2))
            for sm in (0, 1):
                for sn in (0, 1):
                    wm = path[:, m] if sm else 1.0 - path[:, m]
                    wn = path[:, n] if sn else 1.0 - path[:, n]
                    want[sm, sn] = pre * np.sum(wq * wm * wn)
                    idx = [0, 0, 0]
                    idx[l] = cell[l]
                    idx[m] = cell[m] + sm
                    idx[n] = cell[n] + sn
                    got[sm, sn] = J[l][idx[2], idx[1], idx[0]]
            scale = abs(pre)
            assert np.max(np.abs(got - want)) <= 1e-12 * scale, (trial, l, got, want)
            # nothing else on that grid
            assert abs(np.sum(J[l]) - np.sum(got)) <= 1e-12 * scale


def _undulator_run(kind, K=1.2, gamma=30.0, lu=0.02, **kw):
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, und_kind=kind, K=K, gamma=gamma, lambda_u=lu, n_periods=20,
                         n_particles=0, **kw)
    return oracle.Run(oracle.params_from(w)), w


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_external_field_lorentz_invariants(kind):
    extra = {}
    if kind >= 2:
        extra = dict(lu=1e-6, K=0.5, waist=20e-6, pulse_fwhm=3e-3, gamma=60.0)
    r, w = _undulator_run(kind, pol_deg=17.0, **extra)
    inf = r.info()
    g0, b0 = inf["gamma0"], inf["beta0"]
    rng = np.random.default_rng(4)
    lam = w.lambda_u
    for _ in range(40):
        x, y = rng.normal(0, 3e-4 if kind < 2 else 5e-6, 2)
        z = rng.uniform(-5, 5) * lam
        t = rng.uniform(0, 50) * lam / C0
        E, B = r.external_field(x, y, z, t)
        zeta, tl = g0 * (z + b0 * C0 * t), g0 * (t + b0 * z / C0)
        Ep, Bp = r.lab_field(x, y, zeta, tl)
        s = max(np.linalg.norm(Ep) ** 2 + (C0 * np.linalg.norm(Bp)) ** 2, 1e-300)
        assert abs(E @ B - Ep @ Bp) * C0 < 1e-11 * s
        assert abs((E @ E - C0 ** 2 * B @ B) - (Ep @ Ep - C0 ** 2 * Bp @ Bp)) < 1e-11 * s * g0 ** 2
        # inverse transform (frame moving at -beta0) recovers the lab field
        Ex = g0 * (E[0] + C0 * b0 * B[1])
        By = g0 * (B[1] + b0 * E[0] / C0)
        Ey = g0 * (E[1] - C0 * b0 * B[0])
        Bx = g0 * (B[0] - b0 * E[1] / C0)
        sc = math.sqrt(s)
        assert abs(Ex - Ep[0]) < 1e-9 * sc and abs(Ey - Ep[1]) < 1e-9 * sc
        assert abs(C0 * (Bx - Bp[0])) < 1e-9 * sc and abs(C0 * (By - Bp[1])) < 1e-9 * sc


def test_external_field_on_axis_rest_frame():
    r, w = _undulator_run(0)
    inf = r.info()
    g0, b0 = inf["gamma0"], inf["beta0"]
    ku = 2 * math.pi / w.lambda_u
    B0 = 2 * math.pi * ME * C0 * w.K / (QE * w.lambda_u)
    for zeta in (0.3 * w.lambda_u, 3.77 * w.lambda_u, 11.1 * w.lambda_u):
        # pick the rest-frame event with lab coordinate zeta at t = 0
        z = zeta / g0
        E, B = r.external_field(0.0, 0.0, z, 0.0)
        Bpy = B0 * math.sin(ku * zeta)
        assert abs(E[0] + g0 * b0 * C0 * Bpy) < 1e-9 * g0 * C0 * B0
        assert abs(B[1] - g0 * Bpy) < 1e-12 * g0 * B0
        assert abs(E[1]) + abs(E[2]) + abs(B[0]) + abs(B[2]) < 1e-12 * g0 * C0 * B0


@pytest.mark.parametrize("kind", [0, 1])
def test_static_undulator_field_div_curl(kind):
    r, w = _undulator_run(kind, pol_deg=23.0)
    h = 1e-6
    lam = w.lambda_u
    rng = np.random.default_rng(9)
    B0 = 2 * math.pi * ME * C0 * w.K / (QE * lam)
    ku = 2 * math.pi / lam
    for zeta in list(rng.uniform(-2, 22, 30) * lam):
        x, y = rng.normal(0, 1e-3, 2)

        def Bf(dx_, dy_, dz_):
            return r.lab_field(x + dx_, y + dy_, zeta + dz_, 0.0)[1]

        d = [(Bf(h, 0, 0) - Bf(-h, 0, 0)) / (2 * h), (Bf(0, h, 0) - Bf(0, -h, 0)) / (2 * h),
             (Bf(0, 0, h) - Bf(0, 0, -h)) / (2 * h)]
        div = d[0][0] + d[1][1] + d[2][2]
        assert abs(div) < 1e-5 * B0 * ku
        inside = 0.3 * lam < zeta < 19.7 * lam
        if inside:
            curl = np.array([d[1][2] - d[2][1], d[2][0] - d[0][2], d[0][1] - d[1][0]])
            assert np.max(np.abs(curl)) < 1e-5 * B0 * ku


def test_gaussian_beam_tends_to_plane_wave():
    ra, wa = _undulator_run(3, lu=1e-6, K=0.5, waist=5e-2, pulse_fwhm=3e-3, gamma=60.0)
    rb, wb = _undulator_run(2, lu=1e-6, K=0.5, waist=0.0, pulse_fwhm=3e-3, gamma=60.0)
    rng = np.random.default_rng(2)
    for _ in range(10):
        x, y = rng.normal(0, 1e-6, 2)
        zeta, t = rng.uniform(-3e-6, 3e-6), rng.uniform(-1e-14, 1e-14)
        Ea, Ba = ra.lab_field(x, y, zeta, t)
        Eb, Bb = rb.lab_field(x, y, zeta, t)
        s = np.linalg.norm(Eb) + 1e-3 * wa.K * ME * C0 ** 2 * 2 * math.pi / (QE * 1e-6)
        assert np.max(np.abs(Ea - Eb)) < 1e-6 * s
        assert np.max(np.abs(Ba - Bb)) * C0 < 1e-6 * s


def test_particle_boost_inverse():
    w = workloads.scaled(workloads.WORKLOADS["fel_128x128x512"], n_particles=500, nx=8, ny=8, nz=8)
    lab = workloads.lab_bunch(w)
    r = oracle.Run(oracle.params_from(w), lab)
    inf = r.info()
    g0, b0, zr, dt = inf["gamma0"], inf["beta0"], inf["z_ref"], inf["dt"]
    rest = r.particles()
    u = rest[:, 3:]
    g = np.sqrt(1 + np.sum(u * u, axis=1))
    uz_lab = g0 * (u[:, 2] + b0 * g)
    assert np.max(np.abs(uz_lab - lab[:, 5])) < 1e-10 * np.max(lab[:, 5])
    assert np.max(np.abs(u[:, :2] - lab[:, 3:5])) == 0.0
    # z = z_ref + g0 z' + (u_z/g) (g0 b0 z' + c dt/2) -> solve for z'
    zp = (rest[:, 2] - zr - u[:, 2] / g * 0.5 * C0 * dt) / (g0 + u[:, 2] / g * g0 * b0)
    assert np.max(np.abs(zp - lab[:, 2])) < 1e-9 * w.sig_z + 1e-15 * abs(zr)
    s = g0 * b0 * zp + 0.5 * C0 * dt
    assert np.max(np.abs(rest[:, 0] - u[:, 0] / g * s - lab[:, 0])) < 1e-10 * w.sig_x


def test_gauge_residual_evolves_source_free():
    """G^n = div A^n + (phi[n] - phi[n-1])/(c^2 dt) obeys the free update in the interior once
    the charge-conserving deposit feeds A and phi (checked for n >= 3)."""
    nx, ny, nz = 20, 20, 24
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, nx=nx, ny=ny, nz=nz, n_particles=400, solver=0, sig_x=2e-4,
                         sig_y=2e-4, sig_z=4e-6, charge_e=1e9, dist_head=0.002)
    lab = workloads.lab_bunch(w)
    r = oracle.Run(oracle.params_from(w), lab)
    inf = r.info()
    dx, dy, dz, dt = inf["dx"], inf["dy"], inf["dz"], inf["dt"]
    Gs = []
    for s in range(7):
        r.step(1)
        Ax, Ay, Az = r.field("Ax", 1), r.field("Ay", 1), r.field("Az", 1)
        ph1, ph0 = r.field("phi", 1), r.field("phi", 0)
        div = np.zeros_like(Ax)
        div[:, :, 1:] += (Ax[:, :, 1:] - Ax[:, :, :-1]) / dx
        div[:, 1:, :] += (Ay[:, 1:, :] - Ay[:, :-1, :]) / dy
        div[1:, :, :] += (Az[1:, :, :] - Az[:-1, :, :]) / dz
        Gs.append(div + (ph1 - ph0) / (C0 * C0 * dt))
    # free update of G with the oracle's own (pinned) stencil, on a scratch vacuum run
    wv = vacuum(nx, ny, nz, w.dx, w.dy, dz, solver=0)
    sc = oracle.Run(oracle.params_from(wv))
    assert abs(sc.info()["A"] - inf["A"]) < 1e-15 and abs(sc.info()["dt"] - dt) < 1e-25
    part = r.particles()
    X = (part[:, 0] - inf["x0"]) / dx
    assert np.all((X > 3) & (X < nx - 5))
    sl = (slice(4, nz - 4), slice(4, ny - 4), slice(4, nx - 4))
    mag = max(np.max(np.abs(g[sl])) for g in Gs)
    assert mag > 0
    for m in range(2, len(Gs) - 1):
        sc.set_field(3, 0, Gs[m - 1])
        sc.set_field(3, 1, Gs[m])
        sc.set_field(7, 0, np.zeros_like(Gs[m]))
        sc.stencil(3)
        pred = sc.field(3, 2)
        err = np.max(np.abs(pred[sl] - Gs[m + 1][sl]))
        assert err < 1e-12 * mag, (m, err, mag)
