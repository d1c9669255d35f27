"""Serving loop (mithra_submit / mithra_poll): requests of different grids, bunches and
precisions overlap on the GPU, are admitted by device-memory footprint, and each result is the
same alone and in the mix.

"Alone" is the same request run by itself (mithra_create + mithra_step); "in the mix" is the
request served while others run concurrently.  Runs own their buffers, so the only difference is
the order of floating-point atomic additions in the deposition, which differs between any two
runs, alone or not.  FP64 requests agree to 1e-9 of the peak power and of the field energy.
FP32-mixed requests: the run-to-run spread (the largest difference among the same request run
alone three times) is measured, and the difference in the mix must stay within the stated FP32
tolerance (1 % of the peak power, 1e-4 of the field energy; the bunching factor to 1e-3 of itself)
plus four times that spread: over a few hundred steps the dynamics amplify the rounding-order
differences, and a long request can differ from itself by more than 1e-4.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2009_13645_gb300 as m  # noqa: E402
import workloads  # noqa: E402


SMALL_GRIDS = ((32, 32, 128), (64, 64, 192))
TOL = {0: (1e-9, 1e-9, 1e-12), 1: (1e-2, 1e-4, 1e-6)}   # power (of the peak), field energy, bunching


def _requests(n, steps=(60, 160), seed=11):
    # the small grids keep the test short
    return [w for _, w in workloads.serving_requests(n, rate_hz=100.0, seed=seed, steps_range=steps,
                                                     np_range=(2e3, 3e4), grids=SMALL_GRIDS)]


def _alone(w):
    lab = workloads.lab_bunch(w)
    r = m.Run.from_workload(w, lab)
    r.step(w.steps)
    p, t, _ = r.series()
    fe, b = r.diag()
    r.close()
    return p, fe, b


def _wait(tickets, timeout=300.0):
    t0 = time.time()
    while True:
        states = [m.poll(t) for t in tickets]
        if all(d for d, _ in states):
            return [r for _, r in states]
        assert time.time() - t0 < timeout, "served requests did not finish"
        time.sleep(0.01)


@pytest.mark.parametrize("grouped", [False, True])
def test_results_same_alone_and_in_the_mix(grouped):
    """grouped: the requests that reach their captured period (sort every 20 steps: 120 steps,
    captured at step 120, replayed from step 240) advance together by one graph launch; with
    480-600 steps every request has at least two periods to replay."""
    reqs = _requests(6, steps=(480, 600) if grouped else (60, 160))
    assert {w.precision for w in reqs} == {0, 1}
    m.serve_start(8 << 30, max_active=6, queue_capacity=64, steps_per_chunk=8, grouped=grouped)
    try:
        tickets = [m.submit(w) for w in reqs]
        results = _wait(tickets)
        stats = m.serve_stats()
        assert stats["completed"] == len(reqs)
        if grouped:
            gs = m.serve_group_stats()
            print("group launches", gs)
            assert gs["group_launches"] >= 1 and gs["group_periods"] >= 2
        # the requests really overlapped: some were admitted before others finished
        admits = sorted(r.t_admit for r in results)
        dones = sorted(r.t_done for r in results)
        assert admits[-1] < dones[0]
        for w, t, res in zip(reqs, tickets, results):
            assert res.status == 0 and res.steps == w.steps
            p_mix, _ = m.result_series(t)
            p_alone, fe_alone, b_alone = _alone(w)
            tp, te, tb = TOL[w.precision]
            scale = max(np.max(np.abs(p_alone)), 1e-300)
            mix = (np.max(np.abs(p_mix - p_alone)) / scale, abs(res.field_energy - fe_alone) / fe_alone,
                   abs(res.bunching - b_alone))
            floor = (0.0, 0.0, 0.0)
            if w.precision == 1:
                # the run-to-run spread: the largest difference among three runs alone
                runs = [(p_alone, fe_alone, b_alone), _alone(w), _alone(w)]
                floor = tuple(max(d) for d in zip(*[
                    (np.max(np.abs(a[0] - b[0])) / scale, abs(a[1] - b[1]) / fe_alone, abs(a[2] - b[2]))
                    for i, a in enumerate(runs) for b in runs[i + 1:]]))
                tb = max(tb, 1e-3 * b_alone)
                print(f"{w.name} steps {w.steps} FP32 alone vs alone {floor}, alone vs mix {mix}")
            assert mix[0] <= tp + 4 * floor[0], (w.name, w.precision, mix, floor)
            assert mix[1] <= te + 4 * floor[1], (w.name, w.precision, mix, floor)
            assert mix[2] <= tb + 4 * floor[2], (w.name, w.precision, mix, floor)
            m.release(t)
    finally:
        m.serve_stop()


def test_admission_by_footprint_serialises_when_only_one_fits():
    w = workloads.scaled(_requests(1, steps=(40, 40), seed=5)[0], precision=1)
    m.serve_start(8 << 30, max_active=4, queue_capacity=8, steps_per_chunk=8)
    try:
        need = _wait([m.submit(w)])[0].reserved_bytes
    finally:
        m.serve_stop()
    # a pool that holds one such request but not two: admission must serialise them
    m.serve_start(int(need * 1.5), max_active=4, queue_capacity=8, steps_per_chunk=8)
    try:
        t = [m.submit(w) for _ in range(3)]
        res = _wait(t)
        assert all(r.status == 0 for r in res)
        spans = sorted((r.t_admit, r.t_done) for r in res)
        for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
            assert a1 >= d0
        st = m.serve_stats()
        assert st["pool_peak"] <= int(need * 1.5)
        assert st["reserved"] == 0 and st["active"] == 0
        p = [m.result_series(x)[0] for x in t]
        assert np.max(np.abs(p[1] - p[0])) <= TOL[1][0] * np.max(np.abs(p[0]))   # 40 steps: within 1 %
    finally:
        m.serve_stop()


def test_rejections():
    big = workloads.scaled(workloads.WORKLOADS["fel_128x128x512"], n_particles=1000, steps=10)
    small = workloads.scaled(workloads.WORKLOADS["undulator_24x24x96"], n_particles=64, steps=5)
    m.serve_start(64 << 20, max_active=1, queue_capacity=2, steps_per_chunk=4)
    try:
        tb = m.submit(big)
        res = _wait([tb])[0]
        assert res.status == m.ENOMEM
        ts = [m.submit(small), m.submit(small)]
        # the queue holds two; a third may find it full while the first ones wait
        try:
            ts.append(m.submit(small))
        except m.MithraError as e:
            assert e.code == m.EAGAIN
        res = _wait(ts)
        assert all(r.status == 0 for r in res)
        with pytest.raises(m.MithraError) as ei:
            m.poll(987654321)
        assert ei.value.code == m.ENOTFOUND
    finally:
        m.serve_stop()
    with pytest.raises(m.MithraError) as ei:
        m.submit(small)
    assert ei.value.code == m.EINVAL
