"""Pins of the oracle's field solver against what the manual and mathematics fix.

* discrete dispersion relations of FD (Eq. numericalDispersionCD) and NSFD
  (Eq. NSFDDispersionCD): a standing mode cos(k.x) evolves exactly as cos(n w dt);
* the NSFD update at c dt = dz moves a z-plane wave by exactly one cell per step;
  this holds only with alpha'_6 = (c dt/dz)^2 - 2A (c dt/dx)^2 - 2A (c dt/dy)^2;
* CFL bound (Eq. CFLcondition) and the NSFD mesh adjustment;
* Mur: exact 1D absorption at c dt = dz, the printed beta/gamma coefficients agree
  with the printed finite-difference discretisation, and the discrete reflection
  coefficient follows the Engquist-Majda curves of first and second order;
* Mur edges and corners (reading G19): the boundary value solves the first-order outgoing
  conditions of the meeting faces, summed; a field that satisfies each of those conditions and
  is quadratic in space and time is reproduced exactly at every edge and corner node.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from tests.helpers import C0, vacuum


def _mode_run(solver, courant, dx, dy, dz, n=(12, 10, 16), A_override=None):
    w = vacuum(n[0], n[1], n[2], dx, dy, dz, solver=solver, courant=courant, space_charge=1)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 1)))
    return r, r.info()


@pytest.mark.parametrize("solver,courant", [(1, 0.9), (1, 0.5), (0, 1.0)])
@pytest.mark.parametrize("m", [(1, 2, 3), (3, 1, 5), (0, 0, 4), (5, 4, 7)])
def test_dispersion_standing_mode(solver, courant, m):
    nx, ny, nz = 12, 10, 16
    dx, dy, dz = 1.3e-3, 1.7e-3, 1.0e-3
    r, inf = _mode_run(solver, courant, dx, dy, dz, (nx, ny, nz))
    kx, ky, kz = (2 * math.pi * m[0] / (nx * dx), 2 * math.pi * m[1] / (ny * dy), 2 * math.pi * m[2] / (nz * dz))
    cdt = C0 * inf["dt"]
    A = inf["A"]
    sx, sy, sz = (math.sin(kx * dx / 2) / dx) ** 2, (math.sin(ky * dy / 2) / dy) ** 2, (math.sin(kz * dz / 2) / dz) ** 2
    if solver == 0:
        s2 = cdt ** 2 * ((1 - 4 * A * math.sin(kz * dz / 2) ** 2) * (sx + sy) + sz)
    else:
        s2 = cdt ** 2 * (sx + sy + sz)
    assert s2 < 1.0
    wdt = 2 * math.asin(math.sqrt(s2))
    z, y, x = np.meshgrid(np.arange(nz) * dz, np.arange(ny) * dy, np.arange(nx) * dx, indexing="ij")
    mode = np.cos(kx * x + ky * y + kz * z)
    for c in range(4):
        r.set_field(c, 0, mode)
        r.set_field(c, 1, mode * math.cos(wdt))
    nsteps = 200
    r.step(nsteps)
    for c in range(4):
        got = r.field(c, 1)
        exp = mode * math.cos((nsteps + 1) * wdt)
        assert np.max(np.abs(got - exp)) < 1e-10, (c, np.max(np.abs(got - exp)))


def test_nsfd_exact_one_cell_shift():
    """k_x = k_y = 0 at c dt = dz: psi^{n+1}_k = psi^n_{k+1} + psi^n_{k-1} - psi^{n-1}_k.
    dx != dy so that the printed alpha'_6 (dx term twice) would fail."""
    nx, ny, nz = 6, 7, 64
    w = vacuum(nx, ny, nz, 1.4e-3, 2.1e-3, 1.0e-3, solver=0)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 1)))
    assert abs(C0 * r.info()["dt"] - 1.0e-3) < 1e-18
    k = np.arange(nz)

    def f(s):
        s = np.mod(s, nz)
        return np.exp(-((s - 20.0) / 3.0) ** 2) + 0.3 * np.sin(2 * math.pi * s / nz)

    base = np.broadcast_to(f(k)[:, None, None], (nz, ny, nx))
    r.set_field(0, 0, base)
    r.set_field(0, 1, np.broadcast_to(f(k - 1)[:, None, None], (nz, ny, nx)))
    nsteps = 40
    r.step(nsteps)
    exp = np.broadcast_to(f(k - 1 - nsteps)[:, None, None], (nz, ny, nx))
    assert np.max(np.abs(r.field(0, 1) - exp)) < 1e-12


def _grow(solver, courant, steps=300):
    nx, ny, nz = 10, 10, 10
    w = vacuum(nx, ny, nz, 1e-3, 1e-3, 1e-3, solver=solver, courant=courant)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 1)))
    rng = np.random.default_rng(5)
    a = rng.standard_normal((nz, ny, nx))
    r.set_field(0, 0, a)
    r.set_field(0, 1, a)
    r.step(steps)
    return np.max(np.abs(r.field(0, 1)))


def test_cfl_bound():
    assert _grow(1, 0.99) < 50.0
    assert _grow(1, 1.02) > 1e6


def test_nsfd_mesh_adjustment():
    """sqrt((dz/dx)^2 + (dz/dy)^2) >= 1 is adjusted by scaling dx, dy; the run is then stable."""
    w = vacuum(10, 10, 10, 0.5e-3, 0.5e-3, 1e-3, solver=0)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 1)))
    inf = r.info()
    ratio = math.hypot(inf["dz"] / inf["dx"], inf["dz"] / inf["dy"])
    assert ratio < 1.0 and abs(ratio - 0.99) < 1e-12
    assert abs(C0 * inf["dt"] - inf["dz"]) < 1e-18
    assert abs(inf["A"] - 0.25 * (1 + 0.02 / ratio ** 2)) < 1e-15
    rng = np.random.default_rng(1)
    a = rng.standard_normal((10, 10, 10))
    r.set_field(0, 0, a)
    r.set_field(0, 1, a)
    r.step(300)
    assert np.max(np.abs(r.field(0, 1))) < 50.0


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("direction", [-1, +1])
def test_mur_exact_1d_absorption(order, direction):
    """At c dt = dz a z-travelling pulse leaves through either z face without reflection."""
    nx, ny, nz = 5, 6, 80
    w = vacuum(nx, ny, nz, 1.3e-3, 1.6e-3, 1.0e-3, solver=0, mur_order=order)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 0)))
    k = np.arange(nz, dtype=float)

    def f(s):
        return np.exp(-((s - 40.0) / 4.0) ** 2)

    for c in range(4):
        r.set_field(c, 0, np.broadcast_to(f(k)[:, None, None], (nz, ny, nx)))
        r.set_field(c, 1, np.broadcast_to(f(k + direction)[:, None, None], (nz, ny, nx)))
    r.step(120)
    for c in range(4):
        assert np.max(np.abs(r.field(c, 1))) < 1e-12, (c, np.max(np.abs(r.field(c, 1))))


def test_mur_face_matches_printed_discretisation():
    """The gamma update (printed coefficients) zeroes the printed finite-difference form of the
    second-order condition at z = -l_z/2 and z = +l_z/2.  The printed coefficients belong to the
    condition with +(c/2)(d_xx + d_yy) (the Engquist-Majda form); the printed differential
    equation carries the opposite sign on these two terms, a typo that this test records."""
    nx, ny, nz = 7, 8, 9
    dx, dy, dz = 1.2e-3, 1.5e-3, 1.0e-3
    w = vacuum(nx, ny, nz, dx, dy, dz, solver=1, courant=0.7, mur_order=2)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 0)))
    dt = r.info()["dt"]
    rng = np.random.default_rng(3)
    lv = [rng.standard_normal((nz, ny, nx)) for _ in range(3)]
    for l in range(3):
        r.set_field(3, l, lv[l])
    r.mur(3)
    new = r.field(3, 2)
    m1, n0, n1 = lv[0], lv[1], new   # xi^{n-1}, xi^n, xi^{n+1}

    def lap_x(a):
        return (np.roll(a, -1, axis=1) - 2 * a + np.roll(a, 1, axis=1)) / dx ** 2

    def lap_y(a):
        return (np.roll(a, -1, axis=0) - 2 * a + np.roll(a, 1, axis=0)) / dy ** 2

    for b, q, sgn in ((0, 1, +1), (nz - 1, nz - 2, +1)):  # -d_z at z=+l_z/2: inward minus face
        dzt = (1 / (2 * dt)) * (((n1[q] - n1[b]) - (m1[q] - m1[b])) / dz) * sgn
        dtt = (1 / (2 * C0)) * ((n1[q] - 2 * n0[q] + m1[q]) + (n1[b] - 2 * n0[b] + m1[b])) / dt ** 2
        dxx = (C0 / 4) * (lap_x(n0[q]) + lap_x(n0[b]))
        dyy = (C0 / 4) * (lap_y(n0[q]) + lap_y(n0[b]))
        res = dzt - dtt + dxx + dyy
        scale = np.max(np.abs(dtt)) + np.max(np.abs(dzt))
        assert np.max(np.abs(res)) < 1e-12 * scale, np.max(np.abs(res)) / scale


def _reflection(order, theta, kd=0.02):
    """Discrete reflection coefficient of the oracle's z-min Mur face for a plane wave at
    incidence angle theta (measured from the normal), periodic in x."""
    nx, ny, nz = 64, 4, 6
    dz = 1.0e-3
    kmag = kd / dz
    kx = kmag * math.sin(theta)
    # choose dx so that kx is a periodic mode with one wavelength across the box
    dx = 2 * math.pi / (kx * nx)
    kx = 2 * math.pi / (nx * dx)
    kz = math.sqrt(kmag ** 2 - kx ** 2)
    w = vacuum(nx, ny, nz, dx, 1.0e-3, dz, solver=1, courant=0.5, mur_order=order)
    r = oracle.Run(oracle.params_from(w, periodic=(1, 1, 0)))
    dt = r.info()["dt"]
    s2 = (C0 * dt) ** 2 * ((math.sin(kx * dx / 2) / dx) ** 2 + (math.sin(kz * dz / 2) / dz) ** 2)
    om = 2 * math.asin(math.sqrt(s2)) / dt
    z, y, x = np.meshgrid(np.arange(nz) * dz, np.arange(ny) * 1e-3, np.arange(nx) * dx, indexing="ij")

    def mode(Rc, n):
        inc = np.exp(1j * (om * n * dt + kz * z)) * np.exp(1j * kx * x)   # travelling to -z
        ref = Rc * np.exp(1j * (om * n * dt - kz * z)) * np.exp(1j * kx * x)
        return inc + ref

    def face(Rc):
        out = []
        for part in (np.real, np.imag):
            for lvl, n in ((0, -1), (1, 0), (2, 1)):
                r.set_field(3, lvl, part(mode(Rc, n)))
            r.mur(3)
            out.append(r.field(3, 2)[0, 1, 5])
        return out[0] + 1j * out[1]

    exact0 = mode(0.0, 1)[0, 1, 5]
    exact1 = mode(1.0, 1)[0, 1, 5]
    f0, f1 = face(0.0), face(1.0)
    # face(R) = f0 + R (f1 - f0) must equal exact0 + R (exact1 - exact0)
    R = (f0 - exact0) / ((exact1 - exact0) - (f1 - f0))
    return R, math.atan2(kx, kz)


@pytest.mark.parametrize("deg", [10.0, 30.0, 45.0, 60.0])
def test_mur_reflection_engquist_majda(deg):
    for order in (1, 2):
        R, th = _reflection(order, math.radians(deg))
        r1 = (1 - math.cos(th)) / (1 + math.cos(th))
        expect = r1 if order == 1 else r1 * r1
        assert abs(abs(R) - expect) < 0.03 * expect + 2e-5, (order, deg, abs(R), expect)


@pytest.mark.parametrize("comp", [3, 0, 2])
@pytest.mark.parametrize("corner", list(itertools.product((0, 1), repeat=3)))
def test_mur_edges_and_corners_solve_the_summed_first_order_conditions(comp, corner):
    """Reading G19: an edge (corner) node takes the value that satisfies the sum of the first-order
    outgoing conditions d psi/d n_in - (1/c) d psi/dt = 0 of its two (three) faces, discretised
    at the centre of the square (cube) it spans with its inward neighbours.  The field
    psi = F(sum_s sigma_s x_s + c t), sigma_s = +1 at a low face and -1 at a high one, satisfies
    the outgoing condition of each face that meets at the chosen corner of the box, hence their
    sum; with F quadratic the centred differences are exact, so the boundary update of a level
    ring filled with psi must return psi at t + dt at every edge and corner node next to that
    corner (and at its face nodes, first order).  A wrong sign, a wrong count of the summed time
    terms or a wrong averaging factor of the face differences breaks the equality."""
    nx, ny, nz = 7, 8, 9
    D = (1.1e-3, 1.3e-3, 0.9e-3)
    w = vacuum(nx, ny, nz, *D, solver=1, courant=0.9, mur_order=1)
    r = oracle.Run(oracle.params_from(w))
    dt = r.info()["dt"]
    stag = {0: (0.5, 0, 0), 1: (0, 0.5, 0), 2: (0, 0, 0.5), 3: (0, 0, 0)}[comp]
    ext = [n - (1 if comp == a else 0) for a, n in enumerate((nx, ny, nz))]
    z, y, x = np.meshgrid((np.arange(nz) + stag[2]) * D[2], (np.arange(ny) + stag[1]) * D[1],
                          (np.arange(nx) + stag[0]) * D[0], indexing="ij")
    sig = [1.0 if c == 0 else -1.0 for c in corner]
    L = 1e-3

    def F(t):
        xi = (sig[0] * x + sig[1] * y + sig[2] * z + C0 * t) / L
        return 0.3 + 0.7 * xi - 0.05 * xi * xi

    for lev, t in ((0, -dt), (1, 0.0), (2, dt)):
        r.set_field(comp, lev, F(t))
    r.mur(comp)
    got = r.field(comp, 2)
    exp = F(dt)
    checked = {1: 0, 2: 0, 3: 0}
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                ijk = (i, j, k)
                if any(ijk[a] >= ext[a] for a in range(3)):
                    continue
                sides = []
                for a in range(3):
                    if ijk[a] == 0:
                        sides.append((a, 0))
                    elif ijk[a] == ext[a] - 1:
                        sides.append((a, 1))
                if not sides or any(corner[a] != sd for a, sd in sides):
                    continue
                assert abs(got[k, j, i] - exp[k, j, i]) <= 1e-12 * np.max(np.abs(exp)), (ijk, got[k, j, i], exp[k, j, i])
                checked[len(sides)] += 1
    # the corner, the three edges leaving it (their far ends are other corners) and the faces
    assert checked[3] == 1 and checked[2] == sum(e - 2 for e in ext) and checked[1] > 0
