#!/usr/bin/env python
"""Throughput of the rest-frame FDTD/PIC time step on GB300.

One step = one field step of the whole hot path: E and B at nodes, external field + gather +
Boris + zigzag/charge deposition for every particle, the potential update with Mur
boundaries, the radiated-power DFT sample (and the counting sort every 20 steps).

Workload: the FEL-like run, 128x128x512 nodes (8.39 M cells), 2 M macro-particles, planar
undulator K = 1.4, lambda_u = 1.8 cm, gamma = 100, shot-noise phases (synthetic, seeded).
Headline value: cell-updates/s of the FP32-mixed path; particle-pushes/s and the FP64 path are
reported beside it.  With --gpus N each rank runs an independent replica (weak scaling, no
collective on the data path).

--impl reference times the FP64 CPU oracle (the plain program the kernels are checked against)
on the same workload and metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-pushes/s + cell-updates/s (FP32-mixed vs FP64) at stated error; served p99"
WORKLOAD = "fel_128x128x512"
FALLBACK_HBM_GBS = 6800.0


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max_over_ranks(x: float, ws: int, device: str) -> float:
    """The maximum of x over the ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier_ranks(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(ws: int, units_per_rank_step: float, steps: int, ms_max: float) -> float:
    """Units per second of the whole job: every rank processes its own replica's units each
    step (weak scaling), over the slowest rank's time."""
    return ws * units_per_rank_step * steps / (ms_max * 1e-3)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def snapshot(self):
        """One reading, taken right before and right after the timed region (a short region may
        see no sample of the periodic query)."""
        try:
            out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            self.lines.extend(l.strip() for l in out.stdout.splitlines() if l.strip())
        except Exception:
            pass

    def start(self):
        self.snapshot()
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "5"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None and not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)
        self.snapshot()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _source_hash(files):
    """Hash of the sources a capture was taken from: a path stands for the whole file; a dict
    {"file": path, "sections": [[from, to], ...]} for the text from each `from` marker up to the
    next `to` marker (the kernel's own code in a file that holds several kernels)."""
    h = hashlib.sha256()
    for f in files:
        if isinstance(f, dict):
            with open(os.path.join(ROOT, f["file"]), encoding="utf-8") as fh:
                text = fh.read()
            for a, b in f["sections"]:
                i = text.index(a)
                h.update(text[i:text.index(b, i)].encode())
        else:
            with open(os.path.join(ROOT, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[kernel]
        if e["source_hash"] != _source_hash(e["sources"]):
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def oracle_leg(w, lab, steps: int, skip: int = 4):
    """The oracle on all host cores (OpenMP; its independent loops only, so the results are those
    of one thread): `steps` steps, the rate taken over the steps after the first `skip`.  Returns
    the run (at `steps`), the rate in steps/s and the threads used."""
    import oracle
    o = oracle.Run(oracle.params_from(w), lab)
    o.step(skip)
    t1 = time.perf_counter()
    o.step(steps - skip)
    dt = time.perf_counter() - t1
    return o, (steps - skip) / dt, oracle.threads()


def oracle_serial_rate(w, lab, steps: int = 2):
    """The same oracle on one thread (the serial reference), over a couple of steps."""
    import oracle
    n = oracle.threads()
    oracle.set_threads(1)
    try:
        o = oracle.Run(oracle.params_from(w), lab)
        o.step(1)
        t1 = time.perf_counter()
        o.step(steps)
        dt = time.perf_counter() - t1
        o.close()
    finally:
        oracle.set_threads(n)
    return steps / dt


def precision_errors(a: dict, b: dict, M: int) -> dict:
    """Errors of run a against run b: relative L2 and maximum norm of the potentials (A as a
    vector, phi), the radiated power over complete DFT windows (max |dp| / max |p|), the field
    energy and the bunching factor."""
    import numpy as np
    A_a, A_b = np.stack(a["pot"][:3]), np.stack(b["pot"][:3])
    nphi = max(float(np.linalg.norm(b["pot"][3])), 1e-300)
    pa, pb = a["p"][M - 1:], b["p"][M - 1:]
    return {"field_l2_rel_A": float(np.linalg.norm(A_a - A_b) / np.linalg.norm(A_b)),
            "field_l2_rel_phi": float(np.linalg.norm(a["pot"][3] - b["pot"][3]) / nphi),
            "field_max_rel_A": float(np.max(np.abs(A_a - A_b)) / np.max(np.abs(A_b))),
            "power_rel": float(np.max(np.abs(pa - pb)) / max(float(np.max(np.abs(pb))), 1e-300)),
            "field_energy_rel": abs(a["diag"][0] - b["diag"][0]) / b["diag"][0],
            "bunching_abs": abs(a["diag"][1] - b["diag"][1])}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import workloads
    w = workloads.WORKLOADS[WORKLOAD]
    lab = workloads.lab_bunch(w)
    import oracle
    o = oracle.Run(oracle.params_from(w), lab)
    o.step(min(args.warmup, 1))   # the oracle has no cache to warm; one step settles page faults
    budget = float(os.environ.get("MITHRA_REF_BUDGET_S", "150"))
    cores = oracle.threads()
    t1 = time.perf_counter()
    steps = 0
    while steps < args.steps:
        o.step(1)
        steps += 1
        if time.perf_counter() - t1 > budget:
            break
    dt = time.perf_counter() - t1
    cells = w.nx * w.ny * w.nz
    val = cells * steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "cell-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "steps_timed": steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [w.nx, w.ny, w.nz], "particles": w.n_particles,
                       "precision": f"fp64 (CPU oracle, {cores} threads)"},
            "particle_pushes_per_s": w.n_particles * steps / dt,
            "cpu_baseline": {"value": val, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(), "nproc": os.cpu_count(),
                             "sample": f"{steps} full field steps of {WORKLOAD} ({cells} cells, "
                                       f"{w.n_particles} particles), FP64 C on {cores} threads (OpenMP)"},
            "e2e": {"value": val, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def serving_run(m, workloads, all_fp64: bool, n_requests: int, rate_hz: float, grouped: bool = False):
    """The serving stream: Poisson arrivals, mixed grids, bunches and precision flags.  grouped: the
    requests at a replay of their captured period advance together, one graph launch for all."""
    reqs = workloads.serving_requests(n_requests, rate_hz)
    if all_fp64:
        reqs = [(t, workloads.scaled(w, precision=0)) for t, w in reqs]
    labs = [workloads.lab_bunch(w) for _, w in reqs]
    m.serve_start(64 << 30, max_active=16, queue_capacity=4 * n_requests, steps_per_chunk=16, grouped=grouped)
    try:
        t0 = time.perf_counter()
        tickets = []
        for (arr, w), lab in zip(reqs, labs):
            d = t0 + arr - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(m.submit(w, lab))
        while True:
            res = [m.poll(t) for t in tickets]
            if all(d for d, _ in res):
                break
            time.sleep(0.005)
        res = [r for _, r in res]
        peak = m.serve_stats()["pool_peak"]
        gstats = m.serve_group_stats()
        for t in tickets:
            m.release(t)
    finally:
        m.serve_stop()
    ok = [r for r in res if r.status == 0]
    lat = sorted(r.t_done - r.t_submit for r in ok)
    wait = sorted(r.t_admit - r.t_submit for r in ok)
    service = sorted(r.t_done - r.t_admit for r in ok)
    span = max(r.t_done for r in ok) - min(r.t_submit for r in ok)
    cells = sum(w.nx * w.ny * w.nz * w.steps for (_, w), r in zip(reqs, res) if r.status == 0)
    pushes = sum(w.n_particles * w.steps for (_, w), r in zip(reqs, res) if r.status == 0)

    def q(v, f):
        return v[min(len(v) - 1, int(math.ceil(f * len(v))) - 1)]

    return {"requests": n_requests, "completed": len(ok), "arrival_rate_hz": rate_hz,
            "p50_s": q(lat, 0.50), "p99_s": q(lat, 0.99), "max_s": lat[-1], "makespan_s": span,
            "queue_wait_p50_s": q(wait, 0.50), "queue_wait_p99_s": q(wait, 0.99),
            "service_p50_s": q(service, 0.50), "service_p99_s": q(service, 0.99),
            "latency": "time to result = queue wait (submit to admission) + service (admission to done)",
            "cell_updates_per_s": cells / span, "particle_pushes_per_s": pushes / span,
            "pool_peak_bytes": peak, "precision": "fp64 for every request" if all_fp64 else "50/50 FP32-mixed/FP64",
            "design": ("grouped: ready requests' captured periods as child graphs of one graph launch"
                       if grouped else "per-request streams, each replaying its own captured period"),
            "group_launches": gstats["group_launches"], "group_periods": gstats["group_periods"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=64)
    ap.add_argument("--workload", default=WORKLOAD, help="workload name from workloads.WORKLOADS")
    ap.add_argument("--no-array", action="store_true", help="skip the undulator-array workload")
    ap.add_argument("--no-diag", action="store_true", help="skip the spectrum / bunch-sampling run")
    ap.add_argument("--no-seeded", action="store_true", help="skip the seeded UV FEL workload")
    ap.add_argument("--no-loading", action="store_true", help="skip the quasi-random bunch loading")
    ap.add_argument("--no-big", action="store_true", help="skip the 256x256x1024 and 192x192x768 workloads")
    ap.add_argument("--error-windows", type=int, default=3,
                    help="radiated-power DFT windows of the error-against-oracle leg (0: skip it)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_2009_13645_gb300 as m
    import workloads

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    m.use_torch_allocator(True)
    wname = args.workload
    w = workloads.WORKLOADS[wname]
    lab = workloads.lab_bunch(w)
    cells = w.nx * w.ny * w.nz
    K, W = args.steps, max(args.warmup, 3)

    def barrier():
        barrier_ranks(ws)
        torch.cuda.synchronize()

    def reduce_max(x: float) -> float:
        return reduce_max_over_ranks(x, ws, "cuda")

    def emitted_nodes(run, wl) -> int:
        """Nodes one E/B emission writes (at least): per z chunk of 8 node planes, the xy box of
        the active cells whose nodes [lo - 1, hi + 2] reach the chunk, over the planes of the
        deposit box [lo_z - 1, hi_z + 2]; plus the power plane outside its chunk's box.  The
        push widens each chunk's box by whole blocks of particles, so the emission writes a few
        more: the count is a lower bound."""
        inf = run.info()
        P = run.particles()
        c = [np.floor((P[:, d] - inf[o]) / inf[s_]).astype(np.int64)
             for d, (o, s_) in enumerate((("x0", "dx"), ("y0", "dy"), ("z0", "dz")))]
        n = (wl.nx, wl.ny, wl.nz)
        act = np.ones(len(P), bool)
        for d in range(3):
            act &= (c[d] >= 1) & (c[d] <= n[d] - 3)
        plane = (wl.nx - 2) * (wl.ny - 2)
        if not act.any():
            return plane
        x, y, z = c[0][act], c[1][act], c[2][act]
        zl, zh = max(int(z.min()) - 1, 1), min(int(z.max()) + 2, n[2] - 2)
        kp = int(inf["kp"])
        total, kp_box = 0, 0
        for c0 in range(1, n[2] - 1, 8):
            c1 = c0 + 7
            a, b = max(c0, zl), min(c1, zh)
            if a > b:
                continue
            sel = (z - 1 <= c1) & (z + 2 >= c0)
            if not sel.any():
                continue
            ex = min(int(x[sel].max()) + 2, n[0] - 2) - max(int(x[sel].min()) - 1, 1) + 1
            ey = min(int(y[sel].max()) + 2, n[1] - 2) - max(int(y[sel].min()) - 1, 1) + 1
            total += ex * ey * (b - a + 1)
            if a <= kp <= b:
                kp_box = ex * ey
        return total + plane - kp_box

    def source_nodes(run, wl) -> int:
        """Nodes the step's deposit can reach: the box of the nodes [lo, hi + 1] of the cells of
        the active particles (the stencil needs a source there only; elsewhere it is zero)."""
        inf = run.info()
        P = run.particles()
        c = [np.floor((P[:, d] - inf[o]) / inf[s_]).astype(np.int64)
             for d, (o, s_) in enumerate((("x0", "dx"), ("y0", "dy"), ("z0", "dz")))]
        n = (wl.nx, wl.ny, wl.nz)
        act = np.ones(len(P), bool)
        for d in range(3):
            act &= (c[d] >= 1) & (c[d] <= n[d] - 3)
        if not act.any():
            return 0
        tot = 1
        for d in range(3):
            tot *= int(c[d][act].max()) + 1 - int(c[d][act].min()) + 1
        return tot

    def timed_run(precision: int, steps: int, sample_clocks: bool, wl=None, labl=None):
        """K timed steps as a user runs them (captured graphs replayed), then K more steps with
        CUDA events around every kernel (launched one by one) for the per-kernel times."""
        wl = w if wl is None else wl
        labl = lab if labl is None else labl
        stream = torch.cuda.Stream()
        run = m.Run.from_workload(wl, labl, precision=precision, stream=stream.cuda_stream)
        run.step(W)
        run.sync()
        barrier()
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.start()
        l0 = m.kernel_launches()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        run.step(steps)
        ev1.record(stream)
        ev1.synchronize()
        launches = m.kernel_launches() - l0
        barrier()
        clocks = clk.stop() if clk else None
        ms = ev0.elapsed_time(ev1)
        nodes0 = emitted_nodes(run, wl)
        src0 = source_nodes(run, wl)
        run.set_profiling(True)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        run.step(steps)
        e3.record(stream)
        e3.synchronize()
        ms_prof = e2.elapsed_time(e3)
        stats = run.kernel_stats()
        info = run.info()
        info["emitted_nodes"] = 0.5 * (nodes0 + emitted_nodes(run, wl))
        info["source_nodes"] = 0.5 * (src0 + source_nodes(run, wl))
        run.close()
        return ms, stats, launches, clocks, info, ms_prof

    # ---- FP32-mixed (headline) and FP64 ----------------------------------------------------
    ms32, stats32, launches, clocks, info, ms32_prof = timed_run(1, K, True)
    ms32 = reduce_max(ms32)
    res64 = None
    if not args.no_fp64:
        K64 = max(10, K // 2)
        ms64, stats64, _, _, _, _ = timed_run(0, K64, False)
        ms64 = reduce_max(ms64)
        res64 = {"value": whole_job_rate(ws, cells, K64, ms64), "unit": "cell-updates/s",
                 "particle_pushes_per_s": whole_job_rate(ws, w.n_particles, K64, ms64), "ms_per_step": ms64 / K64,
                 "steps": K64, "kernel_ms_per_step": {k: v[0] / K64 for k, v in stats64.items() if v[1]}}

    # ---- the same step through an undulator line (modules, gaps, taper) ----------------------
    arr = None
    if not args.no_array:
        wa = workloads.WORKLOADS["fel_array_128x128x512"]
        laba = workloads.lab_bunch(wa)
        msa, statsa, _, _, _, _ = timed_run(1, K, False, wa, laba)
        msa = reduce_max(msa)
        ca = wa.nx * wa.ny * wa.nz
        arr = {"workload": wa.name, "value": whole_job_rate(ws, ca, K, msa), "unit": "cell-updates/s",
               "particle_pushes_per_s": whole_job_rate(ws, wa.n_particles, K, msa), "ms_per_step": msa / K,
               "steps": K, "precision": "fp32-mixed",
               "undulator": f"{wa.n_modules} modules x {wa.n_periods:g} periods, gap {wa.gap:g} m, "
                            f"K = {wa.K:g} + i x {wa.taper:g}",
               "kernel_ms_per_step": {k: v[0] / K for k, v in statsa.items() if v[1]}}
        del laba

    # ---- the same step with the spectrum sweep and per-step bunch sampling on ----------------
    diag = None
    if not args.no_diag:
        wd = workloads.scaled(w, nf_min=0.5, nf_max=3.5, nf_points=32, bunch_every=1)
        msd, statsd, _, _, _, _ = timed_run(1, K, False, wd, lab)
        msd = reduce_max(msd)
        diag = {"ms_per_step": msd / K, "overhead_ms_per_step": (msd - ms32) / K,
                "value": whole_job_rate(ws, cells, K, msd), "unit": "cell-updates/s",
                "what": "radiated power at 32 normalised frequencies 0.5 .. 3.5 (own DFT window each) and "
                        "bunch moments after every step, FP32-mixed",
                "kernel_ms_per_step": {k: v[0] / K for k, v in statsd.items() if v[1]}}

    # ---- seeded UV FEL (Example 2's job file: 84 x 84 x 8250 nodes, 4.2 M particles, TF/SF seed) --
    seeded = None
    if not args.no_seeded:
        wsd = workloads.WORKLOADS["seeded_uv_84x84x8250"]
        labs = workloads.lab_bunch(wsd)
        Ks = max(10, K // 5)
        mss, statss, _, _, _, _ = timed_run(1, Ks, False, wsd, labs)
        mss = reduce_max(mss)
        cs = wsd.nx * wsd.ny * wsd.nz
        seeded = {"workload": wsd.name, "value": whole_job_rate(ws, cs, Ks, mss), "unit": "cell-updates/s",
                  "particle_pushes_per_s": whole_job_rate(ws, wsd.n_particles, Ks, mss), "ms_per_step": mss / Ks,
                  "steps": Ks, "precision": "fp32-mixed",
                  "seed": "Gaussian beam, a0 9.857e-7 (10 kW) at 0.265187 um, waist 183.74 um, TF/SF planes",
                  "kernel_ms_per_step": {k: v[0] / Ks for k, v in statss.items() if v[1]}}
        del labs

    # ---- the large helical run (256 x 256 x 1024, 32 M particles) and the inverse-Compton run ----
    big = {}
    if not args.no_big:
        for wn in ("helical_256x256x1024", "ics_192x192x768"):
            wb = workloads.WORKLOADS[wn]
            labb = workloads.lab_bunch(wb)
            Kb = max(10, K // 2)
            msb, statsb, _, _, infob, _ = timed_run(1, Kb, False, wb, labb)
            msb = reduce_max(msb)
            cb = wb.nx * wb.ny * wb.nz
            plb = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in statsb.items()}
            ent = {"value": whole_job_rate(ws, cb, Kb, msb), "unit": "cell-updates/s",
                   "particle_pushes_per_s": whole_job_rate(ws, wb.n_particles, Kb, msb), "ms_per_step": msb / Kb,
                   "steps": Kb, "grid": [wb.nx, wb.ny, wb.nz], "particles": wb.n_particles,
                   "precision": "fp32-mixed", "kernel_ms_per_step": {k: v[0] / Kb for k, v in statsb.items() if v[1]}}
            if plb.get("stencil"):
                sb = 48 * cb + 16 * infob["source_nodes"]
                a = sb / (plb["stencil"] * 1e-3) / 1e9
                ent["stencil_roofline"] = {"achieved": a, "frac": a / _peaks()[0], "ms_per_launch": plb["stencil"],
                                           "alg_bytes_per_launch": sb}
            if plb.get("push_deposit"):
                a = 80 * wb.n_particles / (plb["push_deposit"] * 1e-3) / 1e9
                ent["push_roofline"] = {"achieved": a, "frac": a / _peaks()[0], "ms_per_launch": plb["push_deposit"]}
            big[wn] = ent
            del labb

    # ---- quasi-random loading of a 32 M-particle ellipsoid bunch (Halton, uniform + CSE edges) --
    loading = None
    if not args.no_loading:
        e = m.Ellipsoid()
        e.uniform, e.gamma = 1, 200.0
        for a, v in enumerate((40e-6, 40e-6, 2e-6)):
            e.sig[a] = v
        for a, v in enumerate((0.02, 0.02, 0.02)):
            e.sig_u[a] = v
        e.cse_sigma, e.lambda_r, e.bunching, e.shot_noise, e.charge_e = 2.5e-7, 2.5e-7, 0.01, 1, 6.2e8
        nload = 32_000_000
        pinned_out = torch.empty((nload, 6), dtype=torch.float64, pin_memory=True)
        import ctypes
        buf = ctypes.cast(ctypes.c_void_p(pinned_out.data_ptr()), ctypes.POINTER(ctypes.c_double))
        m.load().mithra_ellipsoid_bunch(ctypes.byref(e), 1000, buf, None)   # warm-up
        barrier()
        t0 = time.perf_counter()
        rc = m.load().mithra_ellipsoid_bunch(ctypes.byref(e), nload, buf, None)
        dtl = time.perf_counter() - t0
        if rc == 0:
            loading = {"particles": nload, "seconds": dtl, "particles_per_s": nload / dtl,
                       "what": "mithra_ellipsoid_bunch: uniform profile with CSE edges, bunching 1 %, shot noise, "
                               "generated on the GPU and copied to pinned host memory (1.5 GB)"}
        del pinned_out

    # ---- end to end through the C ABI from pinned host memory -------------------------------
    # the median of three whole runs (a single one of about 8 ms varies by several per cent with
    # the host)
    pinned = torch.empty(lab.shape, dtype=torch.float64, pin_memory=True)
    pinned.numpy()[:] = lab
    import ctypes
    t_runs = []
    for _ in range(3):
        barrier()
        t0 = time.perf_counter()
        b = m.Bunch()
        b.n = lab.shape[0]
        b.charge_e, b.gamma, b.sig_z = w.charge_e, w.gamma, w.sig_z
        b.lab_particles = ctypes.cast(ctypes.c_void_p(pinned.data_ptr()), ctypes.POINTER(ctypes.c_double))
        run = m.Run(m.grid_from(w, 1), m.undulator_from(w), b)
        run.step(K)
        p_ser, t_ser, _ = run.series()
        fe, bunch = run.diag()
        t_runs.append(time.perf_counter() - t0)
        run.close()
    t_e2e = reduce_max(sorted(t_runs)[1])
    h2d = lab.nbytes
    d2h = 2 * 8 * K + 8 * 4

    # ---- roofline of the dominant kernel -----------------------------------------------------
    hbm, peak_kind = _peaks()
    per_launch = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in stats32.items()}
    dominant = max(stats32, key=lambda k: stats32[k][0])
    ncell = cells
    # algorithmic bytes per launch (FP32-mixed)
    alg = {
        # 4 potentials x (psi^n, psi^{n-1}, psi^{n+1}) at every cell, and their sources where the
        # step's deposit can reach (zero elsewhere)
        "stencil": 4 * 3 * 4 * ncell + 4 * 4 * info["source_nodes"],
        "emit_eb": 68 * info["emitted_nodes"],              # see emit_roof below
        # particle state in and out counted as one int32 cell index, three FP32 offsets and three
        # 8-byte momenta: 40 B each way (the layout keeps three int32 cells: 48 B moved each way)
        "push_deposit": 2 * 40 * w.n_particles,
        "clear_sources": 4 * 4 * ncell,
        "mur": 0,
        "power": 0,
        "sort": 0,
    }
    roof = None
    for kern in (dominant, "stencil"):
        if alg.get(kern):
            achieved = alg[kern] / (per_launch[kern] * 1e-3) / 1e9
            roof = {"kernel": kern, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm, "traffic": _ncu_traffic(kern),
                    "state_bytes_per_launch": 2 * 48 * w.n_particles if kern == "push_deposit" else None,
                    "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
                    if peak_kind == "measured" else "fallback 6.8 TB/s",
                    "alg_bytes_per_launch": alg[kern], "ms_per_launch": per_launch[kern]}
            break
    stencil_roof = None
    if per_launch.get("stencil"):
        a = alg["stencil"] / (per_launch["stencil"] * 1e-3) / 1e9
        stencil_roof = {"achieved": a, "frac": a / hbm, "ms_per_launch": per_launch["stencil"],
                        "alg_bytes_per_launch": alg["stencil"], "source_nodes": info["source_nodes"],
                        "traffic": _ncu_traffic("stencil")}
    emit_roof = None
    if per_launch.get("emit_eb"):
        # 68 B per emitted node: A^n, A^{n+1} (3 components each) and phi^n read, 6 E/B components
        # written, 4 sources cleared; the box is the mean of the profiled steps' first and last
        eb_bytes = 68 * info["emitted_nodes"]
        a = eb_bytes / (per_launch["emit_eb"] * 1e-3) / 1e9
        emit_roof = {"achieved": a, "frac": a / hbm, "ms_per_launch": per_launch["emit_eb"],
                     "alg_bytes_per_launch": eb_bytes, "emitted_nodes": info["emitted_nodes"],
                     "traffic": _ncu_traffic("emit_eb")}

    # ---- CPU baseline (oracle) and the errors of both GPU paths against it ---------------------
    cpu = None
    err = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        M = int(round(info["M"]))
        n_err = max(args.error_windows, 1) * M
        o, rate, cores = oracle_leg(w, lab, n_err)
        serial = oracle_serial_rate(w, lab)
        cpu = {"value": cells * rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
               "cpu": cpu_model(), "nproc": os.cpu_count(),
               "sample": f"steps 5-{n_err} of {wname} ({cells} cells, {w.n_particles} particles), FP64 C, "
                         f"independent loops on {cores} threads (OpenMP), deposition serial",
               "particle_pushes_per_s": w.n_particles * rate,
               "serial": {"value": cells * serial, "unit": "cell-updates/s", "cores": 1,
                          "sample": f"2 steps of {wname} on one thread"}}
        if args.error_windows > 0:
            ref = {"pot": [o.field(c, 1) for c in range(4)], "p": o.series()[0], "diag": o.diag()}

            def gpu(prec, labx, sort_every=0):
                g = m.Run.from_workload(w, labx, precision=prec, sort_every=sort_every)
                g.step(n_err)
                out = {"pot": [g.field(c, 1) for c in range(4)], "p": g.series()[0], "diag": g.diag()}
                g.close()
                return out

            err = {"steps": n_err, "power_windows": args.error_windows, "M": M,
                   "what": "relative L2 / max of the potentials at the last step, radiated power over complete "
                           "DFT windows (max |dp| / max |p|), field energy, bunching"}
            g32 = gpu(1, lab)
            err["fp32_mixed"] = precision_errors(g32, ref, M)
            err["fp32_mixed"]["run_to_run"] = precision_errors(gpu(1, lab), g32, M)
            g64 = gpu(0, lab)
            err["fp64"] = precision_errors(g64, ref, M)
            pert = lab[::-1].copy()
            sgn = np.where(np.random.default_rng(3).random(pert[:, 3:].shape) < 0.5, -1.0, 1.0)
            pert[:, 3:] *= 1.0 + 4.4e-16 * sgn
            err["fp64"]["atomic_reordering_floor"] = precision_errors(gpu(0, pert, -1), g64, M)
            err["bounds"] = {"fp32_mixed": "field energy 1e-4, radiated power 1 %",
                             "fp64": "1e-11 on fields + 4 x the atomic-reordering floor"}
        o.close()

    served = None
    if not args.no_serving:
        served = serving_run(m, workloads, False, args.serving_requests, 4.0)
        served["grouped"] = serving_run(m, workloads, False, args.serving_requests, 4.0, grouped=True)
        served["fp64_path"] = serving_run(m, workloads, True, args.serving_requests, 4.0)

    value = whole_job_rate(ws, cells, K, ms32)
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": ws, "steps": K, "warmup": W,
        "ms_per_step": ms32 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": wname, "grid": [w.nx, w.ny, w.nz], "particles": w.n_particles,
                   "precision": "fp32-mixed (fields, offsets, gather, deposit in f32; momentum, external "
                                "field, diagnostics in f64)",
                   "l2": f"inputs larger than L2 (fields {22 * cells * 4 / 1e9:.2f} GB + particles "
                         f"{w.n_particles * 96 / 1e9:.2f} GB resident)",
                   "parallelism": f"{ws} independent replica(s)", "sort_every": 20},
        "particle_pushes_per_s": whole_job_rate(ws, w.n_particles, K, ms32),
        "kernel_ms_per_step": {k: v[0] / K for k, v in stats32.items() if v[1]},
        "kernel_ms_per_launch": {k: v[0] / v[1] for k, v in stats32.items() if v[1]},
        "kernel_times": f"CUDA events around each kernel over {K} further steps launched one by one "
                        f"({ms32_prof / K:.4f} ms/step with the events)",
        "fp64": res64,
        "undulator_array": arr,
        "spectrum_and_bunch_sampling": diag,
        "seeded_uv": seeded,
        "bunch_loading": loading,
        "roofline": roof,
        "stencil_roofline": stencil_roof,
        "emit_roofline": emit_roof,
        "cpu_baseline": cpu,
        "error_vs_oracle": err,
        "large_runs": big or None,
        "e2e": {"value": whole_job_rate(ws, cells, K, t_e2e * 1e3), "unit": "cell-updates/s", "h2d_bytes_per_step": h2d / K,
                "d2h_bytes_per_step": d2h / K, "what": "mithra_create from pinned host particles (H2D), "
                f"{K} steps, power series + diagnostics to host (D2H); median of three runs"},
        "served": served,
        "gpu_launches": launches,
        "clocks": clocks,
        "hbm_bytes": info.get("hbm_bytes"),
    }
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
