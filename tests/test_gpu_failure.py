"""Failure detection without a GPU fault: the library's own bounded waiting.  Every TMA-staged
stencil block (the potential update, Eq. updateEquation) waits on mbarriers for its
tensor copies; each wait has an iteration limit, after which the block records an error word, waits
(again bounded) for the copies it did issue, and returns.  The test leaves one plane's copy out of
every block (MITHRA_TEST_TMA_SKIP_PLANE, read at create) with a short limit: nothing faults or
hangs, mithra_sync reports ETIMEDOUT, and the context stays usable - a run created afterwards
matches the oracle."""
import numpy as np
import pytest

import oracle
from tests.helpers import vacuum

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2009_13645_gb300 as mithra  # noqa: E402

SHAPE = (64, 9, 70)   # 64 FP32 values per row: a multiple of 16 bytes, the TMA stencil runs


def _grid():
    nx, ny, nz = SHAPE
    return vacuum(nx, ny, nz, 1.3e-3, 1.1e-3, 1.0e-3, solver=0, mur_order=2)


def test_expired_tma_wait_reports_etimedout_and_the_context_recovers(monkeypatch):
    w = _grid()
    monkeypatch.setenv("MITHRA_TEST_TMA_SKIP_PLANE", "1")
    r = mithra.Run.from_workload(w, np.zeros((0, 6)), precision=1)
    monkeypatch.delenv("MITHRA_TEST_TMA_SKIP_PLANE")
    r.step(1)
    with pytest.raises(mithra.MithraError) as ei:
        r.sync()
    assert ei.value.code == mithra.ETIMEDOUT
    r.close()
    # the device is fine: a new run of the same grid matches the oracle
    o = oracle.Run(oracle.params_from(w))
    g = mithra.Run.from_workload(w, np.zeros((0, 6)), precision=1)
    rng = np.random.default_rng(5)
    nx, ny, nz = SHAPE
    for c in range(4):
        for lev in range(2):
            a = rng.standard_normal((nz, ny, nx)).astype(np.float32).astype(np.float64)
            o.set_field(c, lev, a)
            g.set_field(c, lev, a)
    o.step(10)
    g.step(10)
    g.sync()
    for c in range(4):
        b = o.field(c, 1)
        assert np.max(np.abs(g.field(c, 1) - b)) < 3e-5 * np.max(np.abs(b))
    g.close()
