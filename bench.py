#!/usr/bin/env python
"""Benchmark of the CudaPre hull pipeline on GB300 (arXiv 1405.3454).

One step = one hull_compute over one synthetic set: 16-extreme search and
polygon (Steps 1-2), strict-inside discard + compaction (Step 3), radix sort
and monotone chain of the survivors (the hull of the remaining points).

Workload: 268,435,456 lattice points uniform in the disk of radius 2^24
(2 GiB float32 xy, seeded), the paper's circle data at HBM-bound scale.  The
input (2 GiB) is larger than L2 (129 MB), so no L2 flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its own
independent set (weak scaling, no collective on the data path).
--impl reference times the CPU oracle on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpoints/s prefilter+hull and % of HBM roofline, exact vs FP32-filtered; p99 latency"
UNIT = "Gpoints/s"
N_POINTS = 1 << 28
SEED = 1405345
WORKLOAD = ("single set of 268,435,456 points (2 GiB float32 xy), integer values uniform in a disk "
            "of radius 2^24 centred at origin (seeded)")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Hash of the two streaming kernels' sources (and their headers) with comments and
    whitespace removed: a change of code, not of comments, makes recorded
    ncu traffic stale."""
    import re
    h = hashlib.sha256()
    for f in ("k_extremes.cu", "k_filter.cu", "internal.cuh", "stream.cuh", "proj.cuh"):
        with open(os.path.join(ROOT, "paper_1405_3454_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per point of `kernel` from an ncu capture summarised under
    profiles/ (a line 'TRAFFIC <kernel> <source-hash> <bytes-per-point>'),
    or None if absent or taken on different kernel source."""
    want = kernel_source_hash()
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".md", ".txt")):
            continue
        for line in open(os.path.join(pdir, fn)):
            m = re.match(r"^TRAFFIC\s+(\S+)\s+(\S+)\s+([0-9.]+)\s*$", line.strip())
            if m and m.group(1) == kernel and m.group(2) == want:
                return float(m.group(3))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest of every rank's x (each rank passes its own); x itself on
    one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput in units per second: every rank processes its own
    units (weak scaling) and the job takes the slowest rank's time."""
    return world * units_per_rank / seconds


def cpu_oracle_sample(n_sample: int, seed: int, xy=None, threads: int = 1):
    """The CPU oracle (as it stands) on the first n_sample points of the
    workload's generator stream (or on xy when given), single-threaded or
    with its point loops split over `threads` host threads (0: all):
    (Gpoints/s, seconds, threads used)."""
    import oracle
    import synth
    if xy is None:
        xy = synth.disk(n_sample, seed)
    oracle.cudapre(xy[:1024])  # load the library outside the timing
    t0 = time.perf_counter()
    if threads == 1:
        oracle.cudapre(xy)
        used = 1
    else:
        _, used = oracle.cudapre_mt(xy, 0, threads)
    dt = time.perf_counter() - t0
    return n_sample / dt / 1e9, dt, used


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return 0
    # Bounded samples: 2^22 points per step, the oracle's point loops on all
    # host cores (a fraction of a second each).
    n_sample = 1 << 22
    import synth
    xy = synth.disk(n_sample, SEED)
    for _ in range(args.warmup):
        cpu_oracle_sample(n_sample, SEED, xy, threads=0)
    times, cores = [], 1
    for _ in range(args.steps):
        _, dt, cores = cpu_oracle_sample(n_sample, SEED, xy, threads=0)
        times.append(dt)
    t = sum(times) / len(times)
    v = n_sample / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_points_per_step": n_sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "first 2^22 points of the disk workload's generator stream per step, "
                                   "the oracle's point loops split over all host threads"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def small_set_leg(cp, torch, synth, exact, fp32, steps, sh, stream):
    """hull_compute on the 1,000,000-point square, each call timed alone by
    CUDA events after an L2 flush: microseconds per call and Gpoints/s for
    both arithmetic forms."""
    if steps <= 0:
        return None
    n1 = 1_000_000
    d1 = torch.from_numpy(synth.square(n1, SEED, 1 << 20)).cuda()
    ws_b = cp.hull_workspace_bytes(n1)
    ws1 = cp.workspace(ws_b)
    out1 = torch.empty(n1, dtype=torch.int32, device="cuda")
    cnt1 = torch.empty(1, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {"workload": "1,000,000 points, integers uniform in [-2^20, 2^20]^2 (seeded)",
           "l2": "256 MB buffer written before every timed call"}
    for name, opt in (("plain_exact", exact), ("fp32_filtered", fp32)):
        def call():
            code = cp.hull_compute(d1.data_ptr(), n1, ws1.data_ptr(), ws_b, out1.data_ptr(), cnt1.data_ptr(), opt,
                                   sh)
            if code:
                raise cp.HullError(code, "hull_compute")
        for _ in range(5):
            call()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.fill_(k & 255)
            evs[k][0].record(stream)
            call()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(b) for a, b in evs)
        mean = sum(ms) / len(ms)
        res[name] = {"us_per_call": mean * 1e3, "us_median": ms[len(ms) // 2] * 1e3,
                     "value": n1 / (mean * 1e-3) / 1e9, "unit": UNIT, "calls": steps}
    res["hull_vertices"] = int(cnt1.item())
    del d1, ws1, out1, flush
    torch.cuda.empty_cache()
    return res


def three_d_leg(cp, torch, synth, fp32, exact, steps, stream, world, timed, peak):
    """hull3_prefilter on 2^26 lattice points uniform in the ball of radius
    2^19 (768 MB, larger than L2): Gpoints/s of both arithmetic forms, the
    stage split, and the HBM fraction of the two streaming passes (12 B per
    point read by each; 4 B per survivor written by the inside test)."""
    if steps <= 0:
        return None
    n3 = 1 << 26
    x3 = torch.from_numpy(synth.ball3(n3, SEED + 51)).cuda()
    ws_b = cp.hull3_prefilter_workspace_bytes(n3)
    ws3 = cp.workspace(ws_b)
    s3 = torch.empty(n3, dtype=torch.int32, device="cuda")
    c3 = torch.empty(1, dtype=torch.int64, device="cuda")
    sh = int(stream.cuda_stream)

    def step3(opt):
        code = cp.hull3_prefilter(x3.data_ptr(), n3, ws3.data_ptr(), ws_b, s3.data_ptr(), c3.data_ptr(), 0, opt, sh)
        if code:
            raise cp.HullError(code, "hull3_prefilter")

    out = {"workload": "2^26 points, integers uniform in the ball of radius 2^19 (768 MB, seeded)",
           "rotation_axis": "z", "angles": "cumulative 0/30/75/120"}
    for name, opt, k in (("fp32_filtered", fp32, steps), ("plain_exact", exact, max(2, steps // 4))):
        for _ in range(2):
            step3(opt)
        ms = timed(step3, opt, k)
        t = cp.StageTimer(max_calls=k)
        timed(step3, opt, k, t)
        st, calls = t.read()
        t.close()
        info = cp.read_polyhedron(ws3)
        f = info["n_survivors"] / n3
        per = {kk: v / max(calls, 1) for kk, v in st.items()}
        out[name] = {"value": world * n3 / (ms * 1e-3) / 1e9, "ms_per_step": ms,
                     "stages_ms": {"extremes": per["extremes"], "polyhedron": per["polygon"],
                                   "inside_test": per["filter"]},
                     "survivor_fraction": f, "facets": len(info["planes"]), "escalations": info["n_escalated"]}
        if name == "fp32_filtered":
            ext_gbs = 12.0 * n3 / (per["extremes"] * 1e-3) / 1e9
            flt_gbs = (12.0 + 4.0 * f) * n3 / (per["filter"] * 1e-3) / 1e9
            out[name]["extremes_hbm_frac"] = ext_gbs / peak
            out[name]["inside_test_hbm_frac"] = flt_gbs / peak
    del x3, ws3, s3
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_1405_3454_gb300 as cp
    import synth
    from paper_1405_3454_gb300 import _build

    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    _build.build()
    cp.load()
    n = args.n
    host = synth.disk(n, SEED + rank)  # each rank: its own independent set
    d_xy = torch.from_numpy(host).cuda()
    fp32 = cp.Options(filter=cp.HULL_FILTER_FP32)
    exact = cp.Options(filter=cp.HULL_FILTER_EXACT)
    ws_bytes = cp.hull_workspace_bytes(n)
    ws = cp.workspace(ws_bytes)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    sh = int(stream.cuda_stream)

    def step(opt):
        code = cp.hull_compute(d_xy.data_ptr(), n, ws.data_ptr(), ws_bytes, out.data_ptr(), cnt.data_ptr(), opt, sh)
        if code:
            raise cp.HullError(code, "hull_compute")

    def prefilter_step(opt):
        code = cp.hull_prefilter(d_xy.data_ptr(), n, ws.data_ptr(), ws_bytes, out.data_ptr(), cnt.data_ptr(), 0,
                                 opt, sh)
        if code:
            raise cp.HullError(code, "hull_prefilter")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, opt, steps, timer=None):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if timer:
            timer.attach()
        e0.record(stream)
        for _ in range(steps):
            fn(opt)
        e1.record(stream)
        if timer:
            timer.detach()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / steps, dist)

    for _ in range(args.warmup):
        step(fp32)
    torch.cuda.synchronize()

    # Headline: the FP32-filtered pipeline (bit-identical to plain exact),
    # timed without instrumentation; the stage breakdown comes from a second
    # pass with the stage timer's events between the kernels.
    clocks = ClockSampler(local)
    clocks.start()
    l0 = cp.launch_count()
    ms = timed(step, fp32, args.steps)
    launches = cp.launch_count() - l0
    clk = clocks.stop()
    timer = cp.StageTimer(max_calls=max(args.steps, 1))
    ms_staged = timed(step, fp32, args.steps, timer)
    stage_ms, calls = timer.read()
    per_call = {k: v / max(calls, 1) for k, v in stage_ms.items()}
    stats = cp.read_stats(ws)
    n_surv, n_esc, n_ref = stats["n_survivors"], stats["n_escalated"], stats["n_refined"]
    n_hull = int(cnt.item())
    value = job_rate(world, n, ms * 1e-3) / 1e9

    # Plain exact method (binary64 projections, int64 orientation for every edge).
    for _ in range(2):
        step(exact)
    ms_exact = timed(step, exact, max(3, args.steps // 4))
    # The paper's comparison (section 3, case (1) against case (2)): the same
    # hull without the preprocessing (every point sorted and chained).
    noprefilter = cp.Options(filter=cp.HULL_FILTER_FP32, no_prefilter=True)
    step(noprefilter)
    ms_np = timed(step, noprefilter, max(3, args.steps // 10))
    # The float32-escalation workload: half Gaussian, half on or one unit
    # inside the Gaussian half's polygon (its polygon from this library's own
    # hull_prefilter, which the parity tests check against the oracle).
    def gpu_polygon(g):
        dg = torch.from_numpy(np.ascontiguousarray(g)).cuda()
        _, _, _, pws = cp.prefilter(dg, fp32)
        m, pxy, _ = cp.read_polygon(pws)
        del dg, pws
        return np.array(pxy, dtype=np.int64).reshape(-1, 2)[:m]

    ne_host, _ = synth.near_edge_mix(n, SEED + 41 + rank, gpu_polygon)
    ne_dev = torch.from_numpy(ne_host).cuda()
    ne_out = torch.empty(n, dtype=torch.int32, device="cuda")

    def ne_step(opt):
        code = cp.hull_compute(ne_dev.data_ptr(), n, ws.data_ptr(), ws_bytes, ne_out.data_ptr(), cnt.data_ptr(), opt,
                               sh)
        if code:
            raise cp.HullError(code, "hull_compute")

    ne_step(fp32)
    ms_ne = timed(ne_step, fp32, max(3, args.steps // 4))
    ne_stats = cp.read_stats(ws)
    ne_hull32 = ne_out[:int(cnt.item())].clone()
    ne_step(exact)
    ms_ne_exact = timed(ne_step, exact, 3)
    ne_hull64 = ne_out[:int(cnt.item())].clone()
    near_edge = {"value": job_rate(world, n, ms_ne * 1e-3) / 1e9, "ms_per_step": ms_ne,
                 "exact_value": job_rate(world, n, ms_ne_exact * 1e-3) / 1e9, "exact_ms_per_step": ms_ne_exact,
                 "escalations": ne_stats["n_escalated"], "escalation_rate": ne_stats["n_escalated"] / n,
                 "survivors": ne_stats["n_survivors"], "hull_identical_to_exact": bool(torch.equal(ne_hull32, ne_hull64)),
                 "workload": "2^28 points: 2^27 Gaussian (sigma 2^22, clipped to +-2^24) interleaved with 2^27 on or "
                             "one unit inside the edges of the Gaussian half's polygon"}
    del ne_dev, ne_out, ne_hull32, ne_hull64, ne_host
    # Prefilter alone (Steps 1-3), both forms.
    for _ in range(2):
        prefilter_step(fp32)
    ms_pre = timed(prefilter_step, fp32, args.steps)
    ms_pre_exact = timed(prefilter_step, exact, max(3, args.steps // 4))

    # Roofline of the dominant single kernel of the prefilter.
    peak, peak_kind = peaks()
    bytes_ext = 8.0 * n
    bytes_flt = 8.0 * n + 12.0 * n_surv
    cand = {"k_extremes32": (per_call["extremes"], bytes_ext), "k_filter": (per_call["filter"], bytes_flt)}
    dom = max(cand, key=lambda k: cand[k][0])
    dms, dbytes = cand[dom]
    achieved = dbytes / (dms * 1e-3) / 1e9
    tpp = recorded_traffic(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": (tpp * n if tpp is not None else None),
                "algorithmic_bytes": dbytes}
    stages_out = {k: {"ms": per_call[k]} for k in per_call}
    stages_out["extremes"].update({"GBps": bytes_ext / (per_call["extremes"] * 1e-3) / 1e9 if per_call["extremes"] else None})
    stages_out["filter"].update({"GBps": bytes_flt / (per_call["filter"] * 1e-3) / 1e9 if per_call["filter"] else None})
    pre_bytes = 16.0 * n + 12.0 * n_surv
    prefilter = {"value": world * n / (ms_pre * 1e-3) / 1e9, "unit": UNIT, "ms": ms_pre,
                 "hbm_frac": (16.0 * n + 4.0 * n_surv) / (ms_pre * 1e-3) / 1e9 / peak,
                 "exact_value": world * n / (ms_pre_exact * 1e-3) / 1e9}

    # End to end through the public API: every step copies its points from
    # pinned host memory into the device and reads its hull back.  The steps
    # are pipelined: the copy of step k+1's points (on a copy stream, into
    # the other of two device buffers) overlaps step k's call and read-back.
    pinned = torch.from_numpy(host).pin_memory()
    host_cnt = torch.empty(1, dtype=torch.int64).pin_memory()
    d_xy2 = torch.empty_like(d_xy)
    bufs = [d_xy, d_xy2]
    cstream = torch.cuda.Stream()
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_steps = max(2, min(args.steps, 10))

    def e2e_run(steps):
        d2h = 0
        with torch.cuda.stream(cstream):
            bufs[0].copy_(pinned, non_blocking=True)
        copied[0].record(cstream)
        for k in range(steps):
            b = k % 2
            if k + 1 < steps:  # the next step's copy, once step k-1 has finished with that buffer
                if k >= 1:
                    cstream.wait_event(consumed[1 - b])
                with torch.cuda.stream(cstream):
                    bufs[1 - b].copy_(pinned, non_blocking=True)
                copied[1 - b].record(cstream)
            stream.wait_event(copied[b])
            code = cp.hull_compute(bufs[b].data_ptr(), n, ws.data_ptr(), ws_bytes, out.data_ptr(), cnt.data_ptr(),
                                   fp32, sh)
            if code:
                raise cp.HullError(code, "hull_compute")
            consumed[b].record(stream)
            host_cnt.copy_(cnt, non_blocking=True)
            stream.synchronize()
            kk = int(host_cnt.item())
            _ = out[:kk].cpu()
            d2h += 8 + 4 * kk
        torch.cuda.synchronize()
        return d2h

    e2e_run(2)
    barrier()
    t0 = time.perf_counter()
    d2h = e2e_run(e2e_steps)
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)
    e2e = {"value": world * n / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": d2h // e2e_steps,
           "pipelined": "step k+1's host-to-device copy overlaps step k's call and read-back (two device buffers)"}
    del d_xy2, bufs

    # The 1,000,000-point square (integers uniform in [-2^20, 2^20]^2), both
    # arithmetic forms: latency-bound (8 MB fits in L2, so L2 is flushed by
    # writing a 256 MB buffer before every timed call).
    small = small_set_leg(cp, torch, synth, exact, fp32, args.small_steps, sh, stream)

    # The 3D extension (section 5) on 2^26 points uniform in a ball.
    three_d = three_d_leg(cp, torch, synth, fp32, exact, args.steps_3d, stream, world, timed, peak)

    # Batched workload: many independent sets in one hull_batch call.
    batch = None
    if args.batch_sets > 0:
        del ws, out
        torch.cuda.empty_cache()
        bxy, boff, _ = synth.batch(args.batch_sets, SEED + 17 + rank)
        nb = int(boff[-1])
        db = torch.from_numpy(bxy).cuda()
        do = torch.from_numpy(boff).cuda()
        del bxy
        bws_bytes = cp.hull_batch_workspace_bytes(nb, args.batch_sets)
        bws = cp.workspace(bws_bytes)
        bout = torch.empty(nb, dtype=torch.int64, device="cuda")
        bhoff = torch.empty(args.batch_sets + 1, dtype=torch.int64, device="cuda")

        def batch_step(opt):
            code = cp.hull_batch(db.data_ptr(), do.data_ptr(), args.batch_sets, nb, bws.data_ptr(), bws_bytes,
                                 bout.data_ptr(), bhoff.data_ptr(), opt, sh)
            if code:
                raise cp.HullError(code, "hull_batch")

        for _ in range(2):
            batch_step(fp32)
        ms_default = timed(batch_step, fp32, args.batch_steps)
        # launch shapes tuned on this workload (cached by GPU and size class)
        import dataclasses
        from paper_1405_3454_gb300 import tune
        tuner = tune.Tuner(torch.cuda.get_device_name(),
                           os.path.join(tempfile.gettempdir(), "cudapre_batch_shapes_%d.json" % os.getpid()))

        def run_shape(shape):
            o = dataclasses.replace(fp32, **shape)
            batch_step(o)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            batch_step(o)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)

        shape = tuner.tune(nb, args.batch_sets, run_shape, reps=1)
        topt = dataclasses.replace(fp32, **shape)
        ms_eager = timed(batch_step, topt, args.batch_steps)
        btimer = cp.StageTimer(max_calls=args.batch_steps)
        timed(batch_step, topt, args.batch_steps, btimer)
        bst, bcalls = btimer.read()
        btimer.close()
        code, bits = cp.device_status(bws)
        hull_total = int(bhoff[-1].item())
        # the same call as a CUDA graph: captured once, then replayed
        gstream = torch.cuda.Stream()
        graph = cp.Graph()

        def graph_step():
            graph.batch_ranges(db, None, do, nb, bws, bout, bhoff, topt, stream=gstream)

        with torch.cuda.stream(gstream):
            for _ in range(2):
                graph_step()
            gstream.synchronize()
            barrier()
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(gstream)
            for _ in range(args.batch_steps):
                graph_step()
            g1.record(gstream)
            barrier()
        ms_graph = max_over_ranks(g0.elapsed_time(g1) / args.batch_steps, dist)
        gcounts = graph.counts()
        graph_same = int(bhoff[-1].item()) == hull_total and cp.device_status(bws) == (0, 0)
        graph.close()
        ms_b = ms_graph
        batch = {"value": world * nb / (ms_b * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms_b, "graph": True,
                 "graph_counts": gcounts, "graph_hull_vertices_equal_eager": graph_same,
                 "eager": {"value": world * nb / (ms_eager * 1e-3) / 1e9, "ms_per_step": ms_eager},
                 "default_shape": {"value": world * nb / (ms_default * 1e-3) / 1e9, "ms_per_step": ms_default},
                 "tuned_shape": shape, "tuning_table_ms": tuner.cache[tuner.key(nb, args.batch_sets)]["table"],
                 "sets": args.batch_sets, "points": nb, "bytes": nb * 8,
                 "hbm_GBps_two_reads": 16.0 * nb / (ms_b * 1e-3) / 1e9,
                 "stages_ms": {k: v / max(bcalls, 1) for k, v in bst.items()},
                 "hull_vertices": hull_total, "device_status": bits,
                 "workload": "%d sets, sizes floor(exp(U(ln 1e3, ln 4e6))), shape per set from square "
                             "(r 2^24), disk (r 2^24), Gaussian (sigma 2^22)" % args.batch_sets}
        del db, do, bws, bout, bhoff
        torch.cuda.empty_cache()

    # Serving: open-loop Poisson arrivals over a resident pool, continuous
    # batching (serve.py); latency = completion event - arrival.
    serving = None
    if args.serve_requests > 0:
        from paper_1405_3454_gb300 import serve
        pxy, pstarts, psizes, _ = synth.serving_pool(args.serve_per_decile, SEED + 29 + rank)
        dpool = torch.from_numpy(pxy).cuda()
        del pxy
        budget = 64 << 30
        server = serve.Server(dpool, budget_bytes=budget, max_points=256 << 20, max_sets=2048, streams=2, opt=fp32)
        req_set, unit_arr = synth.serving_requests(args.serve_requests, len(psizes), SEED + 31 + rank)
        mean_size = float(psizes[req_set].mean())
        cap_gpts = batch["value"] / world if batch else value / world
        warm = min(2000, args.serve_requests)
        serve.simulate(server, pstarts, psizes, req_set[:warm], unit_arr[:warm] / (0.5 * cap_gpts * 1e9 / mean_size))
        runs = {}
        for frac in (0.8, 0.5):
            lam = frac * cap_gpts * 1e9 / mean_size
            res = serve.simulate(server, pstarts, psizes, req_set, unit_arr / lam)
            runs["load_%.1f" % frac] = dict(res.summary(), arrival_rate_per_s=lam)
        serving = {"requests": args.serve_requests, "mean_points": mean_size,
                   "pool": "%d sets (%d per size decile of [1e4, 1.6e7), log-uniform), %d points resident"
                           % (len(psizes), args.serve_per_decile, int(psizes.sum())),
                   "capacity_gpoints_per_s": cap_gpts, "streams": 2, "max_batch_points": 256 << 20,
                   "max_batch_sets": 2048, "memory_budget_bytes": budget,
                   "admission": "a batch is formed only if its workspace and outputs fit in the largest free "
                                "block of the budget's arena; the head request waits otherwise",
                   "ingestion": "excluded (pool resident)", **runs}
        del server, dpool
        torch.cuda.empty_cache()

    cpu = None
    if world == 1 and rank == 0 and not args.no_cpu:
        v, dt, used = cpu_oracle_sample(n, SEED, host, threads=0)
        v1, dt1, _ = cpu_oracle_sample(n, SEED, host, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
               "sample": "the whole workload: all %d points of the same disk (%.1f s on %d host threads)"
                         % (n, dt, used),
               "host_threads": os.cpu_count(),
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "seconds": dt1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64+int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points": n, "mode": "fp32-filtered (bit-identical to plain exact)",
                       "angles": "cumulative 0/30/75/120", "l2": "inputs (2 GiB) larger than L2; no flush",
                       "parallelism": "independent set per GPU" if world > 1 else "single GPU"},
            "variants": {"plain_exact": {"value": world * n / (ms_exact * 1e-3) / 1e9, "ms_per_step": ms_exact},
                         "fp32_filtered": {"value": value, "ms_per_step": ms},
                         "no_prefilter": {"value": job_rate(world, n, ms_np * 1e-3) / 1e9, "ms_per_step": ms_np,
                                          "cudapre_speedup": ms_np / ms},
                         "prefilter_only": prefilter,
                         "near_edge": near_edge,
                         "small_set_1m": small,
                         "three_d": three_d,
                         "batch": batch,
                         "serving": serving},
            "stages_ms_per_step": stages_out,
            "ms_per_step_staged": ms_staged,
            "survivors": n_surv, "escalations": n_esc, "refined_survivors": n_ref, "hull_vertices": n_hull,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    timer.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_POINTS)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--small-steps", type=int, default=200, help="timed calls of the 1M-point leg (0: skip it)")
    ap.add_argument("--steps-3d", type=int, default=20, help="timed calls of the 3D leg (0: skip it)")
    ap.add_argument("--batch-sets", type=int, default=4096, help="sets of the batched leg (0: skip it)")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--serve-requests", type=int, default=100_000, help="requests of the serving leg (0: skip it)")
    ap.add_argument("--serve-per-decile", type=int, default=16)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
