"""Pins of the oracle's E and B at nodes (Sec. "Field Evaluation") and of its field energy.

E = -(A^{n+1} - A^n)/dt - grad phi^n and B = (curl A^n + curl A^{n+1}) / 2 at the nodes, from node
averages of the staggered potentials (A_x at (i + 1/2) dx, ...; reading G5) and central
differences.  Node averages and central differences are exact for potentials that are linear in
space, so every emitted component must equal the closed-form value of such potentials to
rounding, at every interior node:
  B_x = dA_z/dy - dA_y/dz,  B_y = dA_x/dz - dA_z/dx,  B_z = dA_y/dx - dA_x/dy,
each averaged over the two levels.  Every one of the nine derivatives gets its own random slope,
so a swapped component (the printed B_z with A_x in place of A_y, reading G3), a wrong sign, a
missing half or a dropped level fails.

The field energy is sum over nodes of eps0 E^2 / 2 + B^2 / (2 mu0) times the cell volume: for
fields that are uniform over the interior nodes it is that density times the interior volume.
"""
import numpy as np
import pytest

import oracle
from tests.helpers import EPS0, MU0, vacuum

NX, NY, NZ = 9, 8, 11
DX, DY, DZ = 1.1e-3, 1.3e-3, 0.9e-3


def _run(space_charge=1):
    w = vacuum(NX, NY, NZ, DX, DY, DZ, solver=1, courant=0.9, space_charge=space_charge)
    return oracle.Run(oracle.params_from(w))


def _coords(offset):
    """Node coordinates (z, y, x arrays) shifted by `offset` cells per axis (staggering)."""
    z, y, x = np.meshgrid((np.arange(NZ) + offset[2]) * DZ, (np.arange(NY) + offset[1]) * DY,
                          (np.arange(NX) + offset[0]) * DX, indexing="ij")
    return x, y, z


STAG = {0: (0.5, 0.0, 0.0), 1: (0.0, 0.5, 0.0), 2: (0.0, 0.0, 0.5), 3: (0.0, 0.0, 0.0)}


def _load_linear(r, grads, consts):
    """grads[lev][c] = gradient (3,) of potential c at level lev, consts[lev][c] its value at 0."""
    for lev in (0, 1):
        for c in range(4):
            x, y, z = _coords(STAG[c])
            g = grads[lev][c]
            r.set_field(c, lev, g[0] * x + g[1] * y + g[2] * z + consts[lev][c])


def _interior(a):
    return a[1:-1, 1:-1, 1:-1]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_emitted_fields_of_linear_potentials(seed):
    rng = np.random.default_rng(seed)
    r = _run()
    dt = r.info()["dt"]
    # A ~ 1e-6 V s/m over a 1e-3 m cell: B ~ 1e-3 T; potential differences between levels give E ~ 1e5 V/m
    grads = [[rng.uniform(-1, 1, 3) * 1e-3 for _ in range(4)] for _ in range(2)]
    for lev in (0, 1):
        grads[lev][3] = grads[lev][3] * 3e8          # phi: V/m
    consts = [[rng.uniform(-1, 1) * 1e-6 for _ in range(4)] for _ in range(2)]
    consts[0][3] = consts[1][3] = 0.0
    _load_linear(r, grads, consts)
    r.step(1)
    x, y, z = _coords((0.0, 0.0, 0.0))
    X = (x, y, z)
    gphi = grads[0][3]
    for l in range(3):
        dA = sum((grads[1][l][a] - grads[0][l][a]) * X[a] for a in range(3)) + (consts[1][l] - consts[0][l])
        exp = -dA / dt - gphi[l]
        got = r.field(8 + l)
        scale = np.max(np.abs(exp))
        assert np.max(np.abs(_interior(got - exp))) <= 1e-9 * scale, ("E", l)

    def curl(g):
        return np.array([g[2][1] - g[1][2], g[0][2] - g[2][0], g[1][0] - g[0][1]])

    B = 0.5 * (curl(grads[0]) + curl(grads[1]))
    for l in range(3):
        got = _interior(r.field(11 + l))
        assert np.max(np.abs(got - B[l])) <= 1e-12 * np.max(np.abs(B)), ("B", l, got.flat[0], B[l])


def test_emitted_fields_without_space_charge_ignore_phi():
    """space-charge off (Sec. MESH): phi is zero throughout, so E is -dA/dt alone."""
    r = _run(space_charge=0)
    dt = r.info()["dt"]
    g = [np.array([0.0, 0.0, 0.0])] * 4
    grads = [g, [np.array([0.0, 0.0, 0.0])] * 3 + [np.array([5e5, -2e5, 1e5])]]
    consts = [[0.0, 0.0, 0.0, 0.0], [2e-6, -1e-6, 3e-6, 0.0]]
    _load_linear(r, grads, consts)
    r.step(1)
    for l in range(3):
        got = _interior(r.field(8 + l))
        assert np.max(np.abs(got + consts[1][l] / dt)) <= 1e-12 * abs(consts[1][l] / dt)


def test_field_energy_of_uniform_fields():
    rng = np.random.default_rng(7)
    r = _run()
    dt = r.info()["dt"]
    # uniform E from a level difference and uniform B from a linear A
    Bw = rng.uniform(-1, 1, 3) * 2e-3
    Ew = rng.uniform(-1, 1, 3) * 5e5
    # A = (B x r)/2 has curl B; the same at both levels, plus a constant step that gives E
    grads = []
    for lev in (0, 1):
        gA = [np.array([0.0, -Bw[2] / 2, Bw[1] / 2]),
              np.array([Bw[2] / 2, 0.0, -Bw[0] / 2]),
              np.array([-Bw[1] / 2, Bw[0] / 2, 0.0]),
              np.zeros(3)]
        grads.append(gA)
    consts = [[0.0, 0.0, 0.0, 0.0], [-Ew[0] * dt, -Ew[1] * dt, -Ew[2] * dt, 0.0]]
    _load_linear(r, grads, consts)
    r.step(1)
    for l in range(3):
        assert np.allclose(_interior(r.field(8 + l)), Ew[l], rtol=1e-12, atol=0)
        assert np.allclose(_interior(r.field(11 + l)), Bw[l], rtol=1e-12, atol=0)
    fe, _ = r.diag()
    n_int = (NX - 2) * (NY - 2) * (NZ - 2)
    dens = 0.5 * EPS0 * np.dot(Ew, Ew) + 0.5 * np.dot(Bw, Bw) / MU0
    exp = dens * n_int * DX * DY * DZ
    assert abs(fe - exp) <= 1e-12 * exp, (fe, exp)
    # the electric and magnetic parts separately (a misplaced eps0 or mu0 changes one of them)
    consts0 = [[0.0] * 4, [0.0] * 4]
    r2 = _run()
    _load_linear(r2, grads, consts0)
    r2.step(1)
    fe_b, _ = r2.diag()
    assert abs(fe_b - 0.5 * np.dot(Bw, Bw) / MU0 * n_int * DX * DY * DZ) <= 1e-12 * fe_b
