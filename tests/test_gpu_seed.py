"""GPU against the oracle: a seed injected through the TF/SF planes (Sec. "Seed Field"), in
vacuum (the potentials alone, on grids that take the TMA-staged and the plain stencil) and in a
full coupled step (undulator, bunch and seed).  Tolerances: FP64 1e-11 relative (vacuum) and the
parity bound with its measured floor (coupled), as in test_gpu_parity; FP32-mixed 1e-4: a clean
wave crossing the box is the case where the FP32 rounding of the stencil coefficients matters
most -- at c dt = dz the alpha' terms cancel exactly only in exact arithmetic, so each step
leaves a residue of order the FP32 unit round-off that the pulse accumulates coherently over
its 90-step path (random fields, as in the plain vacuum test, average it out)."""
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
from tests.test_gpu_parity import _compare_run, rel  # noqa: E402


@pytest.mark.parametrize("shape", [(37, 29, 60), (40, 28, 60)])
@pytest.mark.parametrize("seed_type", [0, 1])
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-4)])
def test_seeded_vacuum_matches_oracle(shape, seed_type, precision, tol):
    nx, ny, nz = shape
    dz = 1.0e-3
    w = vacuum(nx, ny, nz, 1.6e-3, 1.4e-3, dz, solver=0, mur_order=2)
    w = workloads.scaled(w, seed_type=seed_type, seed_a0=2e-3, seed_lambda=9 * dz, seed_pol_deg=25.0,
                         seed_waist=9e-3, seed_focus=0.01, seed_offset=0.045, seed_pulse_fwhm=20 * dz,
                         seed_cep_deg=10.0)
    o = oracle.Run(oracle.params_from(w))
    g = mithra.Run.from_workload(w, np.zeros((0, 6)), precision=precision)
    o.step(90)
    g.step(90)
    assert np.max(np.abs(o.field(0, 1))) > 0   # the pulse has entered
    for c in range(4):
        for lev in range(2):
            e = rel(g.field(c, lev), o.field(c, lev))
            assert e < tol, (c, lev, e)


def test_seeded_full_step_fp64():
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, nx=21, ny=20, nz=45, n_particles=1500, seed_type=1, seed_a0=5e-3,
                         seed_lambda=base.lambda_u * (1 + 0.5 * base.K ** 2) / (2 * base.gamma ** 2),
                         seed_waist=3e-4, seed_focus=0.05, seed_offset=0.0, seed_pulse_fwhm=0.0)
    lab = workloads.lab_bunch(w)
    o = oracle.Run(oracle.params_from(w), lab)
    g = mithra.Run.from_workload(w, lab, precision=0)
    _compare_run(o, g, 80, 1e-11, 1e-10, w, lab)


def test_set_seed_rejected_after_stepping():
    w = vacuum(24, 24, 24, 1e-3, 1e-3, 1e-3)
    g = mithra.Run.from_workload(w, np.zeros((0, 6)), precision=0)
    g.step(1)
    s = mithra.seed_from(workloads.scaled(w, seed_type=0, seed_a0=1e-3, seed_lambda=1e-2))
    with pytest.raises(mithra.MithraError):
        g.set_seed(s)
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_example2_seed_power_is_10_kW(precision):
    """Example 2's seed (Gaussian beam, a0 = 9.857e-7 at 0.265187 um, waist 183.74 um; the table
    gives its power, 10 kW) on the example's transverse mesh (84 x 84 at 30 um) without
    particles.  Its focus is placed at the power plane's lab position at the measurement time:
    the beam stays within 1.3 w0 between the TF/SF planes and the power plane 150 cells
    downstream, far inside the 2.5 mm plane.  A long Gaussian pulse (300 steps FWHM at a fixed
    rest-frame point) replaces the continuous wave so that the field rises smoothly from zero
    (a switched-on wave would put a Nyquist-frequency transient through the DFT window); its
    centre crosses the plane at step 900, 2.5 FWHM after the start.  At the pulse peak the
    radiated-power diagnostic at the resonance (h = 1) reads the seed's lab power; the
    envelope's curvature over the 27-step DFT window lowers it by 0.3 %."""
    w0 = workloads.WORKLOADS["seeded_uv_84x84x8250"]
    nz = 400
    w = workloads.scaled(w0, nz=nz, n_particles=0, plane_dist=(150 - nz // 2) * w0.dz, seed_type=-1)
    g = mithra.Run.from_workload(w, np.zeros((0, 6)), precision=precision)
    inf = g.info()
    assert abs(int(inf["kp"]) - 150) <= 1
    g0, b0 = inf["gamma0"], inf["beta0"]
    n_meas = 900
    t = inf["T0"] + (n_meas + 0.5) * inf["dt"]
    zp = inf["z0"] + inf["kp"] * inf["dz"]
    focus = g0 * (zp + b0 * C0 * t)               # lab position of the plane at the peak
    t_lab = g0 * (t + b0 * zp / C0)               # and the lab time of that event
    fwhm = 300 * w0.dz / (1 + b0)                 # c tau_lab of 300 steps at a fixed rest point
    g.set_seed(mithra.seed_from(workloads.scaled(w0, seed_focus=focus, seed_offset=C0 * t_lab,
                                                 seed_pulse_fwhm=fwhm)))
    g.step(n_meas + 60)
    p, _, _ = g.series()
    assert np.max(np.abs(p[:200])) < 1e-3 * 1e4   # the pulse starts from zero
    peak = np.max(p[n_meas - 40:n_meas + 40])
    assert abs(peak / 1.0e4 - 1.0) < 0.02, peak
    g.close()
