"""GPU against the oracle: the radiated-power spectrum sweep (Sec. FEL-OUTPUT, radiation-power,
minimum / maximum normalised frequency and number of points) and the bunch samples (Sec. BUNCH,
bunch-sampling), through the C ABI.

Tolerances as for the single-frequency power series in test_gpu_parity: FP64 1e-9 relative to
the largest value of the spectrum; FP32-mixed 1 % where the power is above 1e-3 of its maximum.
Bunch moments: FP64 1e-11 of the spread (means) and 1e-9 (spreads); FP32-mixed positions carry
FP32 cell offsets (6e-8 of a cell) and FP32 fields act on the momenta, so 1e-6 and 1e-4; in both
plus the rounding level of the quantity itself (momenta: storage precision x the largest
momentum spread; lab gamma: storage precision x gamma).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2009_13645_gb300 as mithra  # noqa: E402

W = workloads.scaled(workloads.WORKLOADS["undulator_24x24x96"], nx=21, ny=19, nz=45, n_particles=1500,
                     nf_min=0.5, nf_max=3.0, nf_points=11, bunch_every=7)


@pytest.mark.parametrize("precision", [0, 1])
def test_spectrum_and_bunch_samples_match_oracle(precision):
    lab = workloads.lab_bunch(W)
    o = oracle.Run(oracle.params_from(W), lab)
    g = mithra.Run.from_workload(W, lab, precision=precision, sort_every=5)
    o.step(120)
    g.step(120)
    ho, po = o.spectrum()
    hg, pg = g.spectrum()
    assert np.array_equal(ho, hg)
    assert po.shape == pg.shape == (120, 11)
    s = np.max(np.abs(po))
    assert s > 0
    if precision == 0:
        assert np.max(np.abs(pg - po)) < 1e-9 * s
    else:
        sig = np.abs(po) > 1e-3 * s
        assert sig.sum() > 200
        assert np.max(np.abs(pg[sig] - po[sig]) / np.abs(po[sig])) < 0.01
    # the spectrum point at the main diagnostic's frequency reproduces the main series
    k1 = int(np.argmin(np.abs(hg - W.norm_freq)))
    assert hg[k1] == W.norm_freq
    pm, _, _ = g.series()
    assert np.max(np.abs(pg[:, k1] - pm)) <= 1e-12 * np.max(np.abs(pm))

    bo, bg = o.bunch_series(), g.bunch_series()
    assert bo.shape == bg.shape == (18, 15)
    assert np.array_equal(bg[:, 0], bo[:, 0]) or np.max(np.abs(bg[:, 0] - bo[:, 0])) < 1e-15 * np.max(np.abs(bo[:, 0]))
    spread = np.concatenate([bo[:, 7:13], bo[:, 14:15]], axis=1)
    mean_err = np.abs(np.concatenate([bg[:, 1:7] - bo[:, 1:7], bg[:, 13:14] - bo[:, 13:14]], axis=1))
    sd_err = np.abs(np.concatenate([bg[:, 7:13] - bo[:, 7:13], bg[:, 14:15] - bo[:, 14:15]], axis=1))
    # tolerance per column: a fraction of its spread, plus the rounding level of the quantity
    # itself: for positions 1e-6 of the largest position spread, for the momenta the storage
    # precision times the largest momentum spread (a planar undulator leaves gamma*beta_y at
    # rounding level, and FP32 rotations act on momenta of the size K), for the lab gamma the
    # storage precision times gamma
    t, tu, tg = (1e-11, 1e-12, 1e-13) if precision == 0 else (1e-6, 1e-6, 2e-7)
    for err, tt in ((mean_err, t), (sd_err, 100 * t)):
        tol = tt * spread
        tol[:, 0:3] = np.maximum(tol[:, 0:3], tt * 1e-6 * np.max(spread[:, 0:3]))
        tol[:, 3:6] += tu * np.max(spread[:, 3:6])
        tol[:, 6] += tg * np.abs(bo[:, 13])
        excess = err / tol
        r, c = np.unravel_index(int(np.argmax(excess)), excess.shape)
        assert excess[r, c] <= 1.0, (tt, r, c, err[r, c], spread[r, c])
    g.close()


def test_diagnostics_off_are_rejected():
    w = workloads.scaled(W, nf_points=0, bunch_every=0)
    g = mithra.Run.from_workload(w, workloads.lab_bunch(w), precision=0)
    g.step(3)
    with pytest.raises(mithra.MithraError):
        g.spectrum()
    with pytest.raises(mithra.MithraError):
        g.bunch_series()
    g.close()
