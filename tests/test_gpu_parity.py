"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances:
* FP64 path: 1e-11 relative (max |gpu - oracle| / max |oracle|) on fields and potentials, the
  stated bound, allowing for the reordering of atomic sums: the deposited current of a cell is
  a sum of contributions of both signs, so the order of the floating-point atomic additions
  moves it by more than one rounding.  That floor is measured in each test by a second GPU run
  with the particles in reverse order, no sorting, and lab momenta moved by two units in the last
  place (which also exposes how much the dynamics amplify rounding-level differences such as FMA
  contraction); the bound is 1e-11 + 4 x floor.
* FP32-mixed path: fields stored in FP32 (unit round-off 6e-8), momentum accumulated as a pair
  of floats (about 48 bits), external field and reductions in FP64: 1e-4 relative field energy
  and 1 % radiated power.
"""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests.helpers import C0, vacuum

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2009_13645_gb300 as mithra  # noqa: E402


def rel(a, b):
    s = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (s if s > 0 else 1.0))


def pair(w, precision, lab=None, sort_every=0):
    lab = workloads.lab_bunch(w) if lab is None else lab
    o = oracle.Run(oracle.params_from(w), lab)
    g = mithra.Run.from_workload(w, lab, precision=precision, sort_every=sort_every)
    return o, g


SMALL = workloads.scaled(workloads.WORKLOADS["undulator_24x24x96"], nx=21, ny=19, nz=45,
                         n_particles=1500)


@pytest.mark.parametrize("name", list(workloads.WORKLOADS))
def test_derived_constants_match(name):
    w = workloads.scaled(workloads.WORKLOADS[name], n_particles=16)
    o, g = pair(w, 0)
    io, ig = o.info(), g.info()
    for k in oracle.INFO_KEYS:
        a, b = ig[k], io[k]
        assert abs(a - b) <= 1e-13 * max(abs(b), 1e-300) + (1e-13 * abs(io["z_ref"]) if k in ("z0",) else 0), (k, a, b)


@pytest.mark.parametrize("solver,courant,order", [(0, 1.0, 2), (0, 1.0, 1), (1, 0.9, 2), (1, 0.6, 1)])
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 3e-5)])
def test_vacuum_fields(solver, courant, order, precision, tol):
    nx, ny, nz = 37, 29, 45     # several 32x8 tiles and z chunks with ragged tails
    w = vacuum(nx, ny, nz, 1.3e-3, 1.1e-3, 1.0e-3, solver=solver, courant=courant, mur_order=order)
    o = oracle.Run(oracle.params_from(w))
    g = mithra.Run.from_workload(w, np.zeros((0, 6)), precision=precision)
    rng = np.random.default_rng(7)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for c in range(4):
        for lev in range(2):
            a = rng.standard_normal((nz, ny, nx)) * 0.1
            a += np.exp(-((x - 18 - 3 * c) ** 2 + (y - 14) ** 2 + (z - 22 + lev) ** 2) / 20.0)
            if precision == 1:
                a = a.astype(np.float32).astype(np.float64)
            o.set_field(c, lev, a)
            g.set_field(c, lev, a)
    o.step(40)
    g.step(40)
    for c in range(4):
        for lev in range(2):
            e = rel(g.field(c, lev), o.field(c, lev))
            assert e < tol, (c, lev, e)
    for name in ("Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        e = rel(g.field(name), o.field(name))
        assert e < tol * 10, (name, e)


@pytest.mark.parametrize("kind", [0, 1, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_boost_matches(kind, precision):
    base = workloads.WORKLOADS["ics_192x192x768" if kind == 3 else "fel_128x128x512"]
    w = workloads.scaled(base, n_particles=3000, nx=16, ny=16, nz=24, und_kind=kind)
    o, g = pair(w, precision, sort_every=-1)
    po, pg = o.particles(), g.particles()
    inf = o.info()
    D = np.array([inf["dx"], inf["dy"], inf["dz"]])
    scale = np.maximum(np.abs(po[:, :3]).max(axis=0), D)
    tolx = 1e-13 if precision == 0 else 1e-6
    # u_z = gamma0 (u'_z - beta0 gamma') cancels: bound its error by the size of its terms
    lab = workloads.lab_bunch(w)
    du = 1e-14 * inf["gamma0"] * np.max(np.abs(lab[:, 5]))
    assert np.max(np.abs(pg[:, 3:] - po[:, 3:])) < du
    # positions (cells): rounding of the position itself, plus du carried by the ballistic
    # shift gamma0 beta0 z' to the common rest-frame time
    shift = inf["gamma0"] * np.max(np.abs(lab[:, 2])) + 1e-300
    assert np.max(np.abs(pg[:, :3] - po[:, :3]) / D) < tolx * np.max(scale / D) + du * shift / np.min(D)


def _fields(run):
    out = {}
    for c in range(4):
        for lev in range(2):
            out[(c, lev)] = run.field(c, lev)
    for name in ("Jx", "Jy", "Jz", "rho", "Ex", "Ey", "Ez", "Bx", "By", "Bz"):
        out[name] = run.field(name)
    return out


def _floor_fields(w, lab, precision, steps):
    """GPU run with the particle order reversed, no sort and the lab momenta perturbed by two
    units in the last place: differs from the first run only at the rounding level."""
    pert = lab[::-1].copy()
    sgn = np.where(np.random.default_rng(3).random(pert[:, 3:].shape) < 0.5, -1.0, 1.0)
    pert[:, 3:] *= 1.0 + 4.4e-16 * sgn
    r = mithra.Run.from_workload(w, pert, precision=precision, sort_every=-1)
    r.step(steps)
    f = _fields(r)
    p = r.particles()[::-1]
    r.close()
    return f, p


def _compare_run(o, g, steps, tol_field, tol_part, w=None, lab=None, precision=0):
    o.step(steps)
    g.step(steps)
    fg = _fields(g)
    floor, pfl = (None, None)
    if w is not None and lab is not None and len(lab):
        floor, pfl = _floor_fields(w, lab, precision, steps)
    for key, a in fg.items():
        b = o.field(*key) if isinstance(key, tuple) else o.field(key)
        fl = rel(a, floor[key]) if floor is not None else 0.0
        t = (tol_field if isinstance(key, tuple) else tol_field * 10) + 4.0 * fl
        e = rel(a, b)
        assert e < t, (key, e, fl)
    po, pg = o.particles(), g.particles()
    inf = o.info()
    D = np.array([inf["dx"], inf["dy"], inf["dz"]])
    if len(po):
        flp = np.max(np.abs(pg[:, :3] - pfl[:, :3]) / D) if pfl is not None else 0.0
        flu = np.max(np.abs(pg[:, 3:] - pfl[:, 3:])) if pfl is not None else 0.0
        assert np.max(np.abs(pg[:, :3] - po[:, :3]) / D) < tol_part + 4 * flp
        assert np.max(np.abs(pg[:, 3:] - po[:, 3:])) < tol_part * max(1.0, np.max(np.abs(po[:, 3:]))) + 4 * flu
    return po, pg


def test_full_step_fp64_undulator_small():
    """The full coupled step (config-1 physics on a ragged grid), FP64 path vs oracle."""
    lab = workloads.lab_bunch(SMALL)
    o, g = pair(SMALL, 0, lab=lab)
    _compare_run(o, g, 200, 1e-11, 1e-10, SMALL, lab)
    po, to, eo = o.series()
    pg, tg, eg = g.series()
    assert len(pg) == len(po) == 200
    assert rel(pg, po) < 1e-9 and rel(eg, eo) < 1e-9
    assert np.max(np.abs(tg - to)) <= 1e-15 * np.max(np.abs(to))
    fo, bo = o.diag()
    fg, bg = g.diag()
    assert abs(fg - fo) < 1e-10 * fo
    assert abs(bg - bo) < 1e-12
    assert abs(g.bunching_complex() - o.bunching_complex()) < 1e-12


@pytest.mark.parametrize("kind,substeps,solver,order", [(0, 3, 1, 1), (1, 1, 0, 2), (1, 2, 1, 2), (3, 1, 0, 2),
                                                        (2, 2, 0, 1)])
def test_full_step_fp64_kinds(kind, substeps, solver, order):
    if kind >= 2:
        base = workloads.WORKLOADS["ics_192x192x768"]
        w = workloads.scaled(base, nx=22, ny=20, nz=40, n_particles=1200, sig_x=2e-9, sig_y=2e-9,
                             sig_z=2e-9, und_kind=kind, substeps=substeps, solver=solver, mur_order=order,
                             courant=0.8, charge_e=2e3)
    else:
        base = workloads.WORKLOADS["fel_128x128x512"]
        w = workloads.scaled(base, nx=22, ny=20, nz=40, n_particles=1200, und_kind=kind, substeps=substeps,
                             solver=solver, mur_order=order, courant=0.8, sig_z=0.3e-6, dist_head=1e-4,
                             sig_x=1.5e-5, sig_y=1.5e-5, charge_e=1e7)
    lab = workloads.lab_bunch(w)
    o, g = pair(w, 0, lab=lab)
    _compare_run(o, g, 60, 1e-11, 1e-10, w, lab)


@pytest.mark.parametrize("kind", [2, 3])
def test_full_step_fp32_mixed_optical(kind):
    """FP32-mixed path in an optical undulator (plane wave and Gaussian beam): the carrier phase
    reduced in FP64, profile and envelope in FP32, the transverse Lorentz factor gamma0 (1 + beta0)
    in FP64-evaluated amplitudes.  Field energy within the stated 1e-4, momenta within 1e-5 of
    their scale after 60 steps (FP32 offsets and fields)."""
    base = workloads.WORKLOADS["ics_192x192x768"]
    w = workloads.scaled(base, nx=22, ny=20, nz=40, n_particles=1200, sig_x=2e-9, sig_y=2e-9,
                         sig_z=2e-9, und_kind=kind, substeps=2, solver=0, mur_order=2, charge_e=2e3)
    lab = workloads.lab_bunch(w)
    o, g = pair(w, 1, lab=lab)
    o.step(60)
    g.step(60)
    fo, _ = o.diag()
    fg, _ = g.diag()
    assert abs(fg - fo) / fo < 1e-4, (fg, fo)
    po, pg = o.particles(), g.particles()
    assert np.max(np.abs(pg[:, 3:] - po[:, 3:])) < 1e-5 * np.max(np.abs(po[:, 3:]))
    inf = o.info()
    D = np.array([inf["dx"], inf["dy"], inf["dz"]])
    assert np.max(np.abs(pg[:, :3] - po[:, :3]) / D) < 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_full_step_undulator_array(precision):
    """Static undulator array (one-period modules half a period apart, K tapered by 0.1 per
    module): within the run the bunch crosses the first module, its exit fringe, the gap with
    both windowed fringes and the second module's entrance.  FP64: the parity bound; FP32-mixed:
    the field-energy bound."""
    base = workloads.WORKLOADS["fel_array_128x128x512"]
    w = workloads.scaled(base, nx=22, ny=20, nz=40, n_particles=1200, n_periods=1, gap=0.009,
                         n_modules=3, taper=0.1, substeps=2, sig_z=0.3e-6, dist_head=1e-4,
                         sig_x=1.5e-5, sig_y=1.5e-5, charge_e=1e7)
    lab = workloads.lab_bunch(w)
    o, g = pair(w, precision, lab=lab)
    steps = 70
    if precision == 0:
        _compare_run(o, g, steps, 1e-11, 1e-10, w, lab)
    else:
        o.step(steps)
        g.step(steps)
        fo, _ = o.diag()
        fg, _ = g.diag()
        assert abs(fg - fo) / fo < 1e-4, (fg, fo)
        po, pg = o.particles(), g.particles()
        assert np.max(np.abs(pg[:, 3:] - po[:, 3:])) < 1e-5 * np.max(np.abs(po[:, 3:]))
    inf = o.info()
    t = inf["T0"] + (steps + 0.5) * inf["dt"]
    zeta = inf["gamma0"] * (o.particles()[:, 2] + inf["beta0"] * C0 * t)
    assert np.median(zeta) > w.n_periods * w.lambda_u + w.gap + 0.1 * w.lambda_u


def test_full_step_fp32_mixed_bounds():
    """FP32-mixed path: field energy within 1e-4 and radiated power within 1 % of the oracle."""
    w = workloads.WORKLOADS["undulator_24x24x96"]
    o, g = pair(w, 1)
    o.step(300)
    g.step(300)
    fo, bo = o.diag()
    fg, bg = g.diag()
    assert abs(fg - fo) / fo < 1e-4, (fg, fo)
    assert abs(bg - bo) < 1e-4
    po, _, _ = o.series()
    pg, _, _ = g.series()
    sig = np.abs(po) > 1e-3 * np.max(np.abs(po))
    assert sig.sum() > 100
    assert np.max(np.abs(pg[sig] - po[sig]) / np.abs(po[sig])) < 0.01
    for c in range(4):
        assert rel(g.field(c, 1), o.field(c, 1)) < 1e-3


def test_sort_does_not_change_physics():
    w = SMALL
    lab = workloads.lab_bunch(w)
    a = mithra.Run.from_workload(w, lab, precision=0, sort_every=1)
    b = mithra.Run.from_workload(w, lab, precision=0, sort_every=-1)
    a.step(50)
    b.step(50)
    for c in range(4):
        assert rel(a.field(c, 1), b.field(c, 1)) < 1e-12
    assert np.max(np.abs(a.particles() - b.particles())) < 1e-12 * np.max(np.abs(b.particles()))


def test_edge_cases_empty_and_outside():
    # no particles at all
    w0 = workloads.scaled(SMALL, n_particles=0)
    o, g = pair(w0, 0, lab=np.zeros((0, 6)))
    _compare_run(o, g, 10, 1e-11, 1e-10)
    # every particle far outside the grid: pushed by the external field only
    w1 = workloads.scaled(SMALL, n_particles=64)
    lab = workloads.lab_bunch(w1)
    lab[:, 0] += 1.0
    o, g = pair(w1, 0, lab=lab)
    _compare_run(o, g, 20, 1e-11, 1e-10, w1, lab)
    assert np.max(np.abs(g.field("rho"))) == 0.0
    # a bunch much longer than the grid (most particles outside, some inside)
    w2 = workloads.scaled(SMALL, n_particles=2000, sig_z=40e-6)
    lab2 = workloads.lab_bunch(w2)
    o, g = pair(w2, 0, lab=lab2)
    _compare_run(o, g, 30, 1e-11, 1e-10, w2, lab2)


@pytest.mark.parametrize("precision", [0, 1])
def test_sources_where_particles_enter_the_grid(precision, monkeypatch):
    """The TMA stencil reads a source only inside the previous step's deposit box grown by a cell
    per sub-step, unless the push flags a deposit that may lie outside it.  In a bunch longer than
    the grid, particles enter the active cells at most steps (0 to 3 per step here, counted with the
    oracle); the box holds the end cells of the particles in the one-cell margin around the active
    cells, so their first deposits lie inside it.  FP64: the parity bound against the oracle; FP32-mixed: the TMA run against
    the plain stencil, which reads every source, within 1e-4 of the maximum: the two stencils'
    rounding differences grow to about 2e-5 over the 30 steps, while one particle more or less
    moves the potentials by 6e-3 to 3e-2 of their maximum (oracle runs with and without it)."""
    w = workloads.scaled(workloads.WORKLOADS["undulator_24x24x96"], nx=24, ny=20, nz=48,
                         n_particles=2000, sig_z=40e-6)
    lab = workloads.lab_bunch(w)
    if precision == 0:
        o, g = pair(w, 0, lab=lab)
        _compare_run(o, g, 30, 1e-11, 1e-10, w, lab)
        return
    runs = {}
    for tag, env in (("tma", "0"), ("plain", "1")):
        monkeypatch.setenv("MITHRA_NO_TMA", env)
        runs[tag] = mithra.Run.from_workload(w, lab, precision=1)
        runs[tag].step(30)
    for c in range(4):
        for lev in range(2):
            assert rel(runs["tma"].field(c, lev), runs["plain"].field(c, lev)) < 1e-4, (c, lev)
    for r in runs.values():
        r.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_non_finite_particle_rejected(precision):
    """A non-finite value among the given lab particles is found on the device after the copy:
    mithra_create returns EINVAL and leaves no run; the same bunch without it creates one."""
    w = workloads.scaled(SMALL, n_particles=5000)
    lab = workloads.lab_bunch(w)
    for bad in (np.nan, np.inf, -np.inf):
        l2 = lab.copy()
        l2[4321, 4] = bad
        with pytest.raises(mithra.MithraError) as ei:
            mithra.Run.from_workload(w, l2, precision=precision)
        assert ei.value.code == mithra.EINVAL
    g = mithra.Run.from_workload(w, lab, precision=precision)
    g.step(1)
    g.close()


def test_fullsize_fel_two_steps():
    """The full 128x128x512 grid with 2M macro-particles, in the bench's launch configuration,
    two steps against the oracle (all potentials, a sample of particles).  Errors of the vector
    potential are measured against its largest component (|A| as a vector): after two steps
    A_y and A_z are sums of contributions of both signs (random transverse momenta).  FP32-mixed:
    those displacements come from FP32 offsets (about 1e-5 relative for a move of 0.01 cell),
    so the potentials are held to 1e-3 and the field energy to the stated 1e-4."""
    w = workloads.WORKLOADS["fel_128x128x512"]
    lab = workloads.lab_bunch(w)
    o = oracle.Run(oracle.params_from(w), lab)
    o.step(2)
    fo, bo = o.diag()
    ref = {(c, lev): o.field(c, lev) for c in range(4) for lev in range(2)}
    for precision, tol in ((0, 1e-11), (1, 1e-3)):
        g = mithra.Run.from_workload(w, lab, precision=precision)
        g.step(2)
        floor, pfl = _floor_fields(w, lab, precision, 2)
        for lev in range(2):
            amax = max(np.max(np.abs(ref[(c, lev)])) for c in range(3))
            for c in range(4):
                b = ref[(c, lev)]
                s = amax if c < 3 else np.max(np.abs(b))
                if s == 0:
                    continue
                a = g.field(c, lev)
                fl = float(np.max(np.abs(a - floor[(c, lev)])) / s)
                e = float(np.max(np.abs(a - b)) / s)
                assert e < tol + 4 * fl, (precision, c, lev, e, fl)
        fg, bg = g.diag()
        assert abs(fg - fo) <= (1e-10 if precision == 0 else 1e-4) * fo, (precision, fg, fo)
        assert abs(bg - bo) <= (1e-12 if precision == 0 else 1e-6)
        po, pg = o.particles(), g.particles()
        inf = o.info()
        D = np.array([inf["dx"], inf["dy"], inf["dz"]])
        idx = np.random.default_rng(0).choice(len(po), 20000, replace=False)
        assert np.max(np.abs(pg[idx, :3] - po[idx, :3]) / D) < (1e-9 if precision == 0 else 1e-5)
        g.close()


@pytest.mark.parametrize("shape", [(40, 29, 45), (64, 9, 70), (132, 17, 38), (66, 11, 21)])
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 3e-5)])
@pytest.mark.parametrize("order", [1, 2])
def test_tma_stencil_matches_oracle_and_plain_kernel(shape, precision, tol, order, monkeypatch):
    """Row pitches that are multiples of 16 bytes take the TMA-staged stencil; it must match the
    oracle and the plain z-marching kernel (MITHRA_NO_TMA=1) on tiles with ragged edges.  The
    TMA stencil also writes the Mur x faces of both orders; with 66 nodes in FP64 the last
    interior column of A_x (x = 63) closes a 64-wide tile, so psi^{n-1} of its face node comes
    from global memory (66 FP32 values are not a multiple of 16 bytes: plain kernel)."""
    nx, ny, nz = shape
    w = vacuum(nx, ny, nz, 1.3e-3, 1.1e-3, 1.0e-3, solver=0, mur_order=order)
    o = oracle.Run(oracle.params_from(w))
    runs = {}
    for tag, env in (("tma", "0"), ("plain", "1")):
        monkeypatch.setenv("MITHRA_NO_TMA", env)
        runs[tag] = mithra.Run.from_workload(w, np.zeros((0, 6)), precision=precision)
    rng = np.random.default_rng(3)
    for c in range(4):
        for lev in range(2):
            a = rng.standard_normal((nz, ny, nx))
            if precision == 1:
                a = a.astype(np.float32).astype(np.float64)
            o.set_field(c, lev, a)
            for r in runs.values():
                r.set_field(c, lev, a)
    o.step(25)
    for r in runs.values():
        r.step(25)
        r.sync()
    for c in range(4):
        for lev in range(2):
            a, b = runs["tma"].field(c, lev), runs["plain"].field(c, lev)
            assert rel(a, o.field(c, lev)) < tol
            # the two kernels evaluate the same expression, but the compiler may contract it into
            # FMAs differently (the TMA kernel updates four cells per FP32 thread): FP32 rounding
            # differences grow to a few 1e-6 over 25 steps of random fields
            assert rel(a, b) <= (1e-14 if precision == 0 else 1e-5)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
def test_graph_replay_matches_step_launches(precision, tol, monkeypatch):
    """Steps replayed from a captured CUDA graph give what step-by-step launches give.  With a
    sort every 3 steps a graph spans 6 steps and replays from every multiple of 6 after the
    first; calls of 5, 40 and 7 steps mix captured, replayed and single steps."""
    w = SMALL
    lab = workloads.lab_bunch(w)
    runs = {}
    for tag, env in (("graph", "0"), ("plain", "1")):
        monkeypatch.setenv("MITHRA_NO_GRAPHS", env)
        runs[tag] = mithra.Run.from_workload(w, lab, precision=precision, sort_every=3)
    launches = {}
    for tag, r in runs.items():
        l0 = mithra.kernel_launches()
        for n in (5, 40, 7):
            r.step(n)
        r.sync()
        launches[tag] = mithra.kernel_launches() - l0
    a, b = runs["graph"], runs["plain"]
    # the replayed kernels are counted as launches
    assert launches["graph"] == launches["plain"]
    for c in range(4):
        for lev in range(2):
            assert rel(a.field(c, lev), b.field(c, lev)) < tol
    pa, pb = a.particles(), b.particles()
    assert np.max(np.abs(pa - pb)) <= tol * np.max(np.abs(pb))
    sa, sb = a.series(), b.series()
    assert len(sa[0]) == len(sb[0]) == 52
    assert np.array_equal(sa[1], sb[1])
    assert rel(sa[0], sb[0]) < 100 * tol and rel(sa[2], sb[2]) < 100 * tol
    for r in runs.values():
        r.close()
