"""The field-energy entry point that allocates no device memory agrees with mithra_diag.

Some callers of this library cannot allocate device memory when they want a diagnostic: code
whose memory pool is already fully carved up, a thread that must not take the allocator's locks,
or a real-time loop where an allocation's implicit synchronisation would stall every stream.
mithra_field_energy_noalloc serves them from a fixed array inside the library.  These tests call
it through the C ABI twice in a row on the E and B fields of a run and check both results against
the run's own field energy (mithra_diag, which allocates its scratch with the run), within the
FP64 summation-order tolerance of the other tests.  The file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2009_13645_gb300 as m  # noqa: E402
import workloads  # noqa: E402

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_energy_matches_diag_two_calls(precision):
    w = workloads.scaled(workloads.WORKLOADS["undulator_24x24x96"], n_particles=4096)
    run = m.Run.from_workload(w, precision=precision)
    run.step(60)
    fe_ref, _ = run.diag()
    assert fe_ref > 0
    dtype = torch.float64 if precision == 0 else torch.float32
    eb = [torch.from_numpy(run.field(nm)).to(device="cuda", dtype=dtype).contiguous()
          for nm in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")]
    n = eb[0].numel()
    inf = run.info()
    dv = inf["dx"] * inf["dy"] * inf["dz"]
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(2):
        m.mithra_field_energy_noalloc([t.data_ptr() for t in eb], precision, n, dv,
                                      out.data_ptr() + 8 * k, stream.cuda_stream)
    stream.synchronize()
    got = out.cpu().numpy()
    for g in got:
        assert abs(g - fe_ref) <= 1e-12 * fe_ref, (g, fe_ref)
    assert got[0] == got[1]
    run.close()


def test_noalloc_energy_many_tiles_ragged():
    n = 3 * 4096 * 97 + 1234
    rng = np.random.default_rng(5)
    host = [rng.standard_normal(n) * (1e6 if c < 3 else 1e-2) for c in range(6)]
    eb = [torch.from_numpy(h).cuda() for h in host]
    e2 = sum(h * h for h in host[:3])
    b2 = sum(h * h for h in host[3:])
    ref = float(np.sum(0.5 * EPS0 * e2 + 0.5 * b2 / MU0)) * 2.5e-12
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for k in range(2):
        m.mithra_field_energy_noalloc([t.data_ptr() for t in eb], 0, n, 2.5e-12, out.data_ptr() + 8 * k,
                                      stream.cuda_stream)
    stream.synchronize()
    for g in out.cpu().numpy():
        assert abs(g - ref) <= 1e-12 * ref


def test_noalloc_rejects_more_than_the_maximum():
    eb = [torch.zeros(8, dtype=torch.float64, device="cuda") for _ in range(6)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(m.MithraError) as ei:
        m.mithra_field_energy_noalloc([t.data_ptr() for t in eb], 0, m.NOALLOC_MAX_NODES + 1, 1.0,
                                      out.data_ptr(), 0)
    assert ei.value.code == m.EINVAL and "MITHRA_NOALLOC_MAX_NODES" in str(ei.value)
