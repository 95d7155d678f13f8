#!/usr/bin/env python
"""Benchmark: registered frames/s of the registration scan on one GB300.

Workload (default ``c3``): a synthetic 4,096-frame series of 512x512 fp32
lattice frames (random-walk drift U(+-1) px/frame per axis, smooth field
<= 1.5 px, SNR U(3, 20) per frame, 5 % of frames with jumps of up to 8 px,
seed 1410), registered to frame 0 by the Brent-Kung scan of the operator B
over the leaves A(f_{i-1}, f_i); nonrigid control-grid model, 2-level pyramid,
FP32 arithmetic with float-float/FP64 reductions and FP64 step control.  One
step = pyramid build + all operators + results on the host, through reg_scan.

``value``: frames/s with the frames resident in HBM, through the persistent
device-queue executor with autotuned CTAs per operator (the workload's batched
form).  ``forms`` gives the same workload one operator per launch and as a
replayed CUDA graph; ``phases`` the A leaves and the B scan timed apart.
``e2e``: the same call with pinned HOST frames (host->device copy of the
series and device->host copy of the results, for the nonrigid model every
prefix's control values, inside the timed region).

Run ``python bench.py --impl reference`` for the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "registered frames/s and operator applications/s at <=0.02 px vs FP64 oracle; stream p50/p99"
UNIT = "frames/s"


def workload_spec(name: str, rank: int, frames: int = 0):
    from paper_2010_12478_gb300 import synth
    if name == "c1":
        spec = synth.spec_c1(seed=synth.DEFAULT_SEED + rank)
    elif name == "c2":
        spec = synth.spec_c2(seed=synth.DEFAULT_SEED + rank)
    elif name == "c3":
        spec = synth.spec_c3(seed=synth.DEFAULT_SEED + rank)
    else:
        raise SystemExit(f"unknown workload {name}")
    if frames > 0:   # a shorter series of the same kind (profiler captures)
        spec.n_frames = frames
    return spec


WORKLOAD_FRAMES = {"c1": 16, "c2": 256, "c3": 4096, "c4": 128}
WORKLOAD_TEXT = {
    "c1": "16 frames 128x128 fp32 lattice series, sequential-recursion workload size",
    "c2": "256 frames 512x512 fp32 lattice series (random-walk drift +-1 px/frame, field <=1.5 px, SNR 10), "
          "Brent-Kung scan of B over A leaves",
    "c3": "4096 frames 512x512 fp32 lattice series (random-walk drift +-1 px/frame, field <=1.5 px, SNR 3-20, "
          "5% jumps <=8 px), Brent-Kung scan of B over A leaves",
    "c4": "64 independent series of 128 frames, sizes drawn from {256^2, 512^2, 1024^2}, pyramids stored as "
          "fp32 / bf16 / fp16; the series of one size share one batched scan (persistent queue)",
}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smmax=float(parts[2]), power=float(parts[3]),
                                 hw=parts[5], hwt=parts[6], swt=parts[7], swpc=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sms = sorted(r["sm"] for r in rows)
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swpc", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": rows[0]["smmax"], "samples": len(rows),
                "power_w_max": max(r["power"] for r in rows), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ helpers
def world_max_ms(ms: float, dist, device) -> float:
    """The step time of the whole job: the slowest rank's (every rank waits at the barrier)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed (independent replicas, weak
    scaling) over the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(stats, H, W, levels, storage_bytes, mode):
    """Bytes the method must move per step in the operator kernels: every energy
    evaluation reads the reference and template level once (2 s P_l bytes)."""
    total = 0.0
    sizes = []
    h, w = H, W
    for _ in range(levels):
        sizes.append(h * w)
        h, w = (h + 1) // 2, (w + 1) // 2
    for s in stats:
        for l, ev in enumerate(s["evals"]):
            total += ev * 2 * storage_bytes * sizes[l]
    return total


def pyramid_bytes(N, H, W, levels, storage_bytes, mode):
    """Bytes the pyramid build must move per step: each frame read once, and each stored level
    (with its 3-sample border in the nonrigid model) and each stored B-spline model at the pixel
    centres (nonrigid) written once."""
    pad = 3 if mode == "nonrigid" else 0
    total = 4.0 * H * W
    h, w = H, W
    for _ in range(levels):
        total += storage_bytes * (w + 2 * pad) * (h + 2 * pad)
        if mode == "nonrigid":
            total += storage_bytes * w * h
        h, w = (h + 1) // 2, (w + 1) // 2
    return N * total


def profile_traffic(name: str, src: str, key: str):
    """A DRAM-traffic figure from a committed ncu summary (profiles/<name>.md), if that summary
    was taken on the current kernel source (its sha256 prefix); else None."""
    p = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(p):
        return None
    text = open(p).read()
    m = re.search(r"kernel source sha256: ([0-9a-f]{12})", text)
    t = re.search(re.escape(key) + r": ([0-9.e+]+)", text)
    if not m or not t or m.group(1) != kernel_hash(src):
        return None
    return float(t.group(1))


def kernel_hash(src: str = "reg_kernels.cu"):
    p = os.path.join(ROOT, "paper_2010_12478_gb300", "csrc", src)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:12]


# ------------------------------------------------------------------ CPU oracle baseline
def oracle_sample(frames_np, cfg_bind, budget_s: float):
    """Time the FP64 oracle on a bounded sample of the workload's operators:
    leaves A(f_i, f_{i+1}) then B over consecutive pairs of them, until the budget."""
    import numpy as np
    import oracle as O
    oc = O.Config(levels=cfg_bind.levels, max_iter=cfg_bind.max_iter, max_rejects=cfg_bind.max_rejects,
                  tol_grad=cfg_bind.tol_grad, tol_rel_e=cfg_bind.tol_rel_e, armijo_c=cfg_bind.armijo_c,
                  tau0=cfg_bind.tau0, step_cap=cfg_bind.step_cap, lam=cfg_bind.lam, mode=cfg_bind.mode,
                metric=cfg_bind.metric, sigma=cfg_bind.sigma,
                tol_coarse=cfg_bind.tol_coarse)
    t0 = time.perf_counter()
    pyr = {}
    ops = 0
    leaves = []
    i = 0
    N = frames_np.shape[0]
    while time.perf_counter() - t0 < budget_s and i + 1 < N:
        for j in (i, i + 1):
            if j not in pyr:
                pyr[j] = O.pyramid(frames_np[j], oc.levels)
        leaves.append(O.op_A(pyr, i, i + 1, oc))
        ops += 1
        if len(leaves) % 2 == 0:
            O.op_B(leaves[-2], leaves[-1], pyr, oc)
            ops += 1
        i += 1
    dt = time.perf_counter() - t0
    return ops, dt, f"{ops} operators ({len(leaves)} A leaves + {ops - len(leaves)} B) on frames 0..{i}"


def _oracle_task(args):
    """One self-contained sample task for a pool worker: A(f0, f1), A(f1, f2) and B over them
    (the 2:1 mix of leaves and B operators of a tree scan).  Returns (operators, seconds)."""
    import oracle as O
    f, cfgd = args
    oc = O.Config(**cfgd)
    t0 = time.perf_counter()
    pyr = {j: O.pyramid(f[j], oc.levels) for j in range(3)}
    a1 = O.op_A(pyr, 0, 1, oc)
    a2 = O.op_A(pyr, 1, 2, oc)
    O.op_B(a1, a2, pyr, oc)
    return 3, time.perf_counter() - t0


def oracle_sample_parallel(frames_np, cfg_bind, budget_s: float, workers: int = 0):
    """The same oracle on all host cores: independent sample tasks (frame triples) on a pool of
    spawned processes, submitted until the budget is spent.  Returns (operators, wall seconds,
    cores, sample text)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    workers = workers or os.cpu_count() or 1
    cfgd = dict(levels=cfg_bind.levels, max_iter=cfg_bind.max_iter, max_rejects=cfg_bind.max_rejects,
                tol_grad=cfg_bind.tol_grad, tol_rel_e=cfg_bind.tol_rel_e, armijo_c=cfg_bind.armijo_c,
                tau0=cfg_bind.tau0, step_cap=cfg_bind.step_cap, lam=cfg_bind.lam, mode=cfg_bind.mode,
                metric=cfg_bind.metric, sigma=cfg_bind.sigma,
                tol_coarse=cfg_bind.tol_coarse)
    N = frames_np.shape[0]
    tasks = [(frames_np[3 * q:3 * q + 3].copy(), cfgd) for q in range(max(1, (N - 1) // 3))]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_warm_worker, range(workers)))   # imports and oracle build outside the timing
        t0 = time.perf_counter()
        ops, done, q = 0, 0, 0
        running = set()
        while q < len(tasks) and len(running) < workers:
            running.add(ex.submit(_oracle_task, tasks[q]))
            q += 1
        while running:
            fin, running = cf.wait(running, return_when=cf.FIRST_COMPLETED)
            for fu in fin:
                ops += fu.result()[0]
                done += 1
            if time.perf_counter() - t0 < budget_s:
                while q < len(tasks) and len(running) < workers:
                    running.add(ex.submit(_oracle_task, tasks[q]))
                    q += 1
        dt = time.perf_counter() - t0
    return ops, dt, workers, f"{ops} operators ({done} tasks of A, A, B on frame triples) on {workers} processes"


def _warm_worker(_):
    import oracle as O
    O.lib()
    return 0


# ------------------------------------------------------------------ serving
def serving(dev, mode: str, frames_per_stream: int, seed: int = 1410, cluster: int = 0,
            lookback=None):
    """Eight acquisition streams of 256^2, 512^2 or 1024^2 frames arriving by Poisson processes of
    U(50, 400) frames/s each, registered online through reg_stream_* with a 40 GB budget.
    Returns frames/s over the run and per-frame latency (submit -> result) percentiles."""
    import numpy as np
    import torch
    from paper_2010_12478_gb300 import binding as B
    from paper_2010_12478_gb300 import synth
    rng = np.random.default_rng(seed)
    sizes = [256, 512, 1024]
    plan = []
    for k in range(8):
        S = int(sizes[rng.integers(3)])
        rate = float(rng.uniform(50.0, 400.0))
        spec = synth.SeriesSpec(frames_per_stream, S, S, step=1.0, field_amp=1.5, snr=(10.0, 10.0),
                                seed=seed + 100 + k)
        fr = synth.make_series(spec, device=dev).frames   # device-resident acquisition buffers
        t = np.cumsum(rng.exponential(1.0 / rate, size=frames_per_stream))
        plan.append((S, rate, fr, t))
    ctx = B.Context(B.Config(mode=mode, mem_budget=40 << 30, cluster=cluster))
    # warm-up, untimed: a short stream per frame size loads and runs every kernel once
    for S in sorted({p[0] for p in plan}):
        fr = next(p[2] for p in plan if p[0] == S)
        ws = B.Stream(ctx, S, S)
        for j in range(8):
            while ws.submit(fr[j], j) != B.REG_OK:
                ws.poll(256, 1000)
        got = 0
        while got < 8:
            got += len(ws.poll(256, 100000))
        ws.close()
    streams = [B.Stream(ctx, S, S) for (S, _, _, _) in plan]
    # look-back of each stream's online scan: a prefix operator B (a long span) can take longer than
    # the frame interval at these rates, so the prefixes advance in k = 2 chains side by side (two
    # frames per B); a larger k adds window operators per frame (measured: k = 4 for the 1024^2
    # streams raised p99 from 21 ms to 2.8 s)
    lookback = lookback or {256: 2, 512: 2, 1024: 2}
    for (S, _, _, _), st in zip(plan, streams):
        st.set_lookback(lookback[S])
    events = sorted((t[j], k, j) for k, (_, _, _, t) in enumerate(plan) for j in range(len(t)))
    results = [[] for _ in plan]
    refused = 0
    wait_ms = [np.zeros(len(p[3])) for p in plan]   # arrival -> admitted (a refused submit is retried)
    # one host thread drives all streams without blocking on any: frames that arrived wait in their
    # stream's queue (in order) until a submit is admitted; results are polled between attempts
    import collections
    pending = [collections.deque() for _ in plan]
    ev = 0
    t0 = time.perf_counter()
    while ev < len(events) or any(pending):
        now = time.perf_counter() - t0
        while ev < len(events) and events[ev][0] <= now:
            ta, k, j = events[ev]
            pending[k].append((ta, j))
            ev += 1
        for k, q in enumerate(pending):
            while q:
                ta, j = q[0]
                if streams[k].submit(plan[k][2][j], j) != B.REG_OK:
                    refused += 1
                    break
                wait_ms[k][j] = (time.perf_counter() - t0 - ta) * 1e3
                q.popleft()
        for q, st in enumerate(streams):
            results[q] += st.poll(256, 0)
        time.sleep(0.0002)
    while sum(len(r) for r in results) < sum(len(p[3]) for p in plan):
        for q, st in enumerate(streams):
            results[q] += st.poll(256, 1000)
    t1 = time.perf_counter()
    for st in streams:
        st.close()
    # latency from arrival: the admission wait plus submit -> result (the service's own clock)
    svc = np.array([r["done_us"] - r["submit_us"] for rs in results for r in rs]) / 1e3
    lat = np.array([wait_ms[k][r["frame_id"]] + (r["done_us"] - r["submit_us"]) / 1e3
                    for k, rs in enumerate(results) for r in rs])
    n = len(lat)
    arr = np.array([plan[k][3][r["frame_id"]] for k, rs in enumerate(results) for r in rs])
    late = lat[arr >= 1.0]   # frames arriving after the first second
    per_stream = []
    for k, rs in enumerate(results):
        lk = np.array([wait_ms[k][r["frame_id"]] + (r["done_us"] - r["submit_us"]) / 1e3 for r in rs])
        per_stream.append({"p50": round(float(np.percentile(lk, 50)), 2), "p99": round(float(np.percentile(lk, 99)), 2),
                           "max_admission_wait_ms": round(float(wait_ms[k].max()), 2)})
    last_arrival = max(float(p[3][-1]) for p in plan)
    return {"streams": [{"size": S, "rate_fps": round(rate, 1), "frames": len(t), "lookback": lookback[S],
                         "latency_from_arrival_ms": ps}
                        for (S, rate, _, t), ps in zip(plan, per_stream)],
            "mode": mode, "frames": n, "wall_s": round(t1 - t0, 3), "value": round(n / (t1 - t0), 2),
            "unit": "frames/s", "last_arrival_s": round(last_arrival, 3),
            "drain_after_last_arrival_s": round(t1 - t0 - last_arrival, 3),
            "latency_ms": {"from": "arrival (admission wait included)",
                           "p50": round(float(np.percentile(lat, 50)), 3),
                           "p99": round(float(np.percentile(lat, 99)), 3),
                           "max": round(float(lat.max()), 3)},
            "latency_after_first_second_ms": {"p50": round(float(np.percentile(late, 50)), 3) if len(late) else None,
                                              "p99": round(float(np.percentile(late, 99)), 3) if len(late) else None},
            "service_latency_ms": {"from": "admitted submit",
                                   "p50": round(float(np.percentile(svc, 50)), 3),
                                   "p99": round(float(np.percentile(svc, 99)), 3)},
            "admission_refusals": refused, "budget_bytes": 40 << 30,
            "frames_per_stream": frames_per_stream,
            "offered_fps": round(sum(rate for (_, rate, _, _) in plan), 1),
            "frames_source": "device memory (each submit copies the frame into the stream's slot)"}


# ------------------------------------------------------------------ precision
def precision(frames, mode: str, n_samples: int = 6):
    """Per pyramid storage type: scan throughput on the workload and the maximum displacement
    error of sampled neighbour operators A(f_i, f_{i+1}) against the FP64 oracle."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2010_12478_gb300 import binding as B
    N, H, W = frames.shape
    n = N - 1
    idx = [int(i) for i in np.linspace(0, n - 1, n_samples)]
    Fh = frames.cpu().numpy()
    ref = {}
    cfg0 = B.Config(mode=mode)
    oc = O.Config(levels=cfg0.levels, max_iter=cfg0.max_iter, max_rejects=cfg0.max_rejects, tol_grad=cfg0.tol_grad,
                  tol_rel_e=cfg0.tol_rel_e, armijo_c=cfg0.armijo_c, tau0=cfg0.tau0, step_cap=cfg0.step_cap,
                  lam=cfg0.lam, mode=mode, grid=cfg0.grid, metric=cfg0.metric, sigma=cfg0.sigma,
                  tol_coarse=cfg0.tol_coarse)
    for i in idx:
        ref[i] = O.op_A({i: O.pyramid(Fh[i], oc.levels), i + 1: O.pyramid(Fh[i + 1], oc.levels)}, i, i + 1, oc)
    out = {}
    for storage in ("f32", "bf16", "f16"):
        ctx = B.Context(B.Config(mode=mode, storage=storage))
        ctx.scan(frames, schedule="brent_kung", exec="persistent")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        els, st = ctx.scan(frames, schedule="brent_kung", exec="persistent", raw=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        els, st = B.elems_list(els), B.stats_list(st, ctx.cfg.levels)
        errs = []
        for i in idx:
            # leaves are the first n operators of the per-op stats; compare the operator A(f_i, f_{i+1})
            if mode == "rigid":
                errs.append(O.max_px_error(np.array(st[i]["theta"]), ref[i].phi, H, W, "rigid"))
            else:
                g = O.grid_for(W, H, cfg0.grid)
                ctx1 = B.Context(B.Config(mode=mode, storage=storage, cluster=8))
                u = torch.empty((2, H, W), device=frames.device)
                ctx1.pairwise(frames[i].contiguous(), frames[i + 1].contiguous(), field_out=u)
                errs.append(O.max_px_error(u.cpu().numpy(), O.grid_dense(g, ref[i].phi), H, W, "nonrigid"))
        out[storage] = {"frames_per_s": round(n / dt, 2), "max_px_error_vs_oracle": round(max(errs), 5),
                        "median_px_error_vs_oracle": round(float(np.median(errs)), 5),
                        "bar_px": 0.02 if storage == "f32" else 0.1,
                        "operators_over_bar": [idx[j] for j, e in enumerate(errs)
                                               if e > (0.02 if storage == "f32" else 0.1)],
                        "operators_sampled": idx}
    out["oracle_stop_reasons"] = {i: [int(v) for v in ref[i].stats.stop[:oc.levels]] for i in idx}
    return out


# ------------------------------------------------------------------ three levels
def three_levels(dev, mode: str, exec_: str, n_samples: int = 3):
    """The c2 workload (256 x 512^2) with a 3-level pyramid, the depth the workload description
    names: scan throughput and the neighbour operators A(f_i, f_{i+1}) of a few frames against the
    FP64 oracle at the same depth."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2010_12478_gb300 import binding as B
    from paper_2010_12478_gb300 import synth
    frames = synth.make_series(synth.spec_c2(), device=dev).frames
    N, H, W = frames.shape
    cfg = B.Config(mode=mode, levels=3)
    ctx = B.Context(cfg, device=dev.index or 0)
    ctx.scan(frames, schedule="brent_kung", exec=exec_)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, st = ctx.scan(frames, schedule="brent_kung", exec=exec_, raw=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = B.stats_list(st, 3)
    oc = O.Config(levels=3, max_iter=cfg.max_iter, max_rejects=cfg.max_rejects, tol_grad=cfg.tol_grad,
                  tol_rel_e=cfg.tol_rel_e, armijo_c=cfg.armijo_c, tau0=cfg.tau0, step_cap=cfg.step_cap,
                  lam=cfg.lam, mode=mode, grid=cfg.grid, metric=cfg.metric, sigma=cfg.sigma,
                  tol_coarse=cfg.tol_coarse)
    Fh = frames.cpu().numpy()
    errs = []
    for i in [int(v) for v in np.linspace(0, N - 2, n_samples)]:
        ref = O.op_A({i: O.pyramid(Fh[i], 3), i + 1: O.pyramid(Fh[i + 1], 3)}, i, i + 1, oc)
        if mode == "rigid":
            errs.append(O.max_px_error(np.array(st[i]["theta"]), ref.phi, H, W, "rigid"))
        else:
            u = torch.empty((2, H, W), device=dev)
            B.Context(B.Config(mode=mode, levels=3, cluster=8), device=dev.index or 0).pairwise(
                frames[i].contiguous(), frames[i + 1].contiguous(), field_out=u)
            errs.append(O.max_px_error(u.cpu().numpy(), O.grid_dense(O.grid_for(W, H, cfg.grid), ref.phi), H, W,
                                       "nonrigid"))
    ev = np.array([sum(x["evals"]) for x in st])
    return {"workload": "c2: 256 frames 512x512, 3-level pyramid", "mode": mode, "exec": exec_,
            "value": round((N - 1) / dt, 2), "unit": "frames/s", "evals_per_operator": round(float(ev.mean()), 2),
            "max_px_error_vs_oracle": round(max(errs), 5), "operators_sampled": len(errs), "bar_px": 0.02}


# ------------------------------------------------------------------ registered series
def registered_series(ctx, frames, mode: str, steps: int, warmup: int, peak: float, peak_src: str, world: int):
    """reg_warp on the workload: out_k = f_k o phi_{0,k} for every frame and the series mean,
    from the deformations of one scan; device-resident, CUDA events over `steps` calls."""
    import ctypes
    import torch
    from paper_2010_12478_gb300 import binding as B
    N, H, W = frames.shape
    els, _ = ctx.scan(frames, schedule="brent_kung", exec="persistent",
                      fields_out=None, want_stats=False)
    kw = {}
    if mode == "rigid":
        arr = B.elem_array(els)
        raw = torch.empty(ctypes.sizeof(arr), dtype=torch.uint8)
        ctypes.memmove(raw.data_ptr(), ctypes.addressof(arr), ctypes.sizeof(arr))
        kw["elems"] = raw.to(frames.device)
    else:
        nx, ny, _ = B.grid_dims(W, H, ctx.cfg.grid, ctx.cfg.levels)
        g = torch.empty((N - 1, ny, nx, 2), device=frames.device)
        ctx.scan_grids(g)
        kw["grids"] = g
    out = torch.empty_like(frames)
    mean = torch.empty((H, W), device=frames.device)
    for _ in range(warmup):
        ctx.warp(frames, out=out, mean=mean, **kw)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        ctx.warp(frames, out=out, mean=mean, **kw)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    alg = 8.0 * N * H * W + 4.0 * H * W   # each frame read once, each registered frame written once, the mean
    achieved = alg / (ms / 1e3) / 1e9
    tim = ctx.last_timing()
    return {"value": round(world * N / (ms / 1e3), 1), "unit": "frames/s", "ms_per_call": round(ms, 4),
            "outputs": "registered frames [N][H][W] and their mean",
            "tma_staged": bool(tim["tma_staged"]),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         # the capture is of 256 frames; each frame is read and written once, so the
                         # traffic grows in proportion to the frames of the call
                         "traffic": (lambda t: None if t is None else round(t * N / 256))(
                             profile_traffic(f"warp_kernel_c2_{mode}", "reg_warp.cu", "dram bytes per call (scaled)")),
                         "peak_source": peak_src, "kernel": "warp_kernel (+ mean_kernel)",
                         "algorithmic_bytes_per_call": alg}}


# ------------------------------------------------------------------ mixed-size batch (c4)
def mixed_batch(args, dev, world, rank, dist):
    """The c4 workload as the benchmark's line (mixed_measure)."""
    results, sizes, clocks = mixed_measure(args.mode, dev, world, rank, dist, args.steps, args.warmup)
    if rank == 0:
        line = {
            "metric": METRIC, "value": results["f32"]["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": results["f32"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"c4: {WORKLOAD_TEXT['c4']}", "series": 64, "frames_per_series": 128,
                       "sizes": sizes, "mode": args.mode,
                       "exec": "persistent (one reg_scan_batch per size)",
                       "cluster": {str(S): C4_SHAPE[S][0] for S in C4_SHAPE},
                       "l2": "inputs larger than L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "precision": results, "clocks": clocks,
            "roofline": None, "e2e": None, "cpu_baseline": None,
            "note": "per-storage throughput and error; the operator-kernel roofline and the end-to-end and CPU "
                    "baselines are reported on the c2 and c3 workloads",
            "gpu_launches": None}
        print(json.dumps(line), flush=True)


# CTAs per operator and register form for each frame size of c4 (measured on the batched scans:
# 4 / 3 CTAs per SM for 256^2, 8 / 4 for 512^2, 16 / 3 for 1024^2 took the whole batch from
# 4,086 to 4,670 frames/s against 16 CTAs for every size)
C4_SHAPE = {256: (4, 3), 512: (8, 4), 1024: (16, 3)}


def mixed_measure(mode, dev, world, rank, dist, steps, warmup):
    """64 series x 128 frames, sizes drawn from {256, 512, 1024}^2; per pyramid storage type the
    series of each size run as one reg_scan_batch call (persistent queue); frames/s over all
    series, and the displacement error of sampled neighbour operators against the FP64 oracle."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2010_12478_gb300 import binding as B
    from paper_2010_12478_gb300 import synth
    rng = np.random.default_rng(1410 + rank)
    sizes = [int(v) for v in rng.choice([256, 512, 1024], size=64)]
    groups = {}
    for q, S in enumerate(sizes):
        spec = synth.SeriesSpec(128, S, S, step=1.0, field_amp=1.5, snr=(10.0, 10.0), seed=1410 + rank, series=q)
        groups.setdefault(S, []).append(synth.make_series(spec, device=dev).frames)
    batches = {S: torch.stack(v) for S, v in groups.items()}
    del groups
    n_frames = sum(b.shape[0] * (b.shape[1] - 1) for b in batches.values())
    peak, peak_src = peaks()
    results = {}
    with ClockSampler(0 if dev.index is None else dev.index) as clk:
        for storage in ("f32", "bf16", "f16"):
            ctxs = {S: B.Context(B.Config(mode=mode, storage=storage, cluster=C4_SHAPE[S][0], ctas_per_sm=C4_SHAPE[S][1]))
                    for S in batches}
            for S, b in batches.items():   # warm-up
                for _ in range(max(1, warmup)):
                    ctxs[S].scan_batch(b, exec="persistent", want_stats=False, raw=True)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                for S, b in batches.items():
                    ctxs[S].scan_batch(b, exec="persistent", want_stats=False, raw=True)
            e1.record()
            torch.cuda.synchronize()
            ms = world_max_ms(e0.elapsed_time(e1) / steps, dist, dev)
            results[storage] = {"value": round(job_rate(n_frames, world, ms), 2), "unit": UNIT,
                                "ms_per_step": round(ms, 2)}
            del ctxs
    # precision: sampled neighbour operators of the 256^2 and 512^2 series against the oracle
    if rank == 0:
        cfg0 = B.Config(mode=mode)
        oc = O.Config(levels=cfg0.levels, max_iter=cfg0.max_iter, max_rejects=cfg0.max_rejects,
                      tol_grad=cfg0.tol_grad, tol_rel_e=cfg0.tol_rel_e, armijo_c=cfg0.armijo_c, tau0=cfg0.tau0,
                      step_cap=cfg0.step_cap, lam=cfg0.lam, mode=mode, grid=cfg0.grid,
                      metric=cfg0.metric, sigma=cfg0.sigma,
                      tol_coarse=cfg0.tol_coarse)
        samples = [(S, 0, j) for S in (256, 512) if S in batches for j in (5, 77)]
        for storage in ("f32", "bf16", "f16"):
            ctx = B.Context(B.Config(mode=mode, storage=storage, cluster=16))
            errs = []
            for S, q, j in samples:
                F = batches[S][q]
                Fh = F[j:j + 2].cpu().numpy()
                ref = O.op_A({0: O.pyramid(Fh[0], oc.levels), 1: O.pyramid(Fh[1], oc.levels)}, 0, 1, oc)
                if mode == "rigid":
                    el, _ = ctx.pairwise(F[j].contiguous(), F[j + 1].contiguous())
                    errs.append(O.max_px_error(np.array(el[2:], dtype=np.float64), ref.phi, S, S, "rigid"))
                else:
                    u = torch.empty((2, S, S), device=dev)
                    ctx.pairwise(F[j].contiguous(), F[j + 1].contiguous(), field_out=u)
                    errs.append(O.max_px_error(u.cpu().numpy(), ref.phi, S, S, "nonrigid"))
            results[storage]["max_px_error_vs_oracle"] = round(max(errs), 5)
            results[storage]["operators_sampled"] = [f"{S}^2 series {q} frames {j},{j + 1}" for S, q, j in samples]
    return results, {str(S): int(b.shape[0]) for S, b in batches.items()}, clk.summary()


# ------------------------------------------------------------------ main
def paper_bounds(N: int, P: int, C1: float = 1.0):
    """The paper's upper bounds on the speedup of the scan registration and of the full
    registration on P workers (Sec. 5.2): (N-1) / (2N/P - 1 + C1 log2 P) and
    (2N-1) / (3N/P - 1 + C1 log2 P)."""
    lg = math.log2(P) if P > 1 else 0.0
    return {"P": P, "C1": C1, "scan": round((N - 1) / (2.0 * N / P - 1.0 + C1 * lg), 2),
            "full": round((2 * N - 1) / (3.0 * N / P - 1.0 + C1 * lg), 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4"])
    ap.add_argument("--mode", default="nonrigid", choices=["rigid", "nonrigid"])
    ap.add_argument("--exec", dest="exec_", default="persistent", choices=["plain", "level", "persistent", "graph"])
    ap.add_argument("--frames", type=int, default=0, help="override the series length (small profiler cases)")
    ap.add_argument("--cluster", type=int, default=0, help="CTAs per operator; 0 = autotuned")
    ap.add_argument("--oracle-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="main timed region only (for profiler captures)")
    ap.add_argument("--warp", action="store_true", help="with --quick: also run the registered-series stage")
    ap.add_argument("--serve-frames", type=int, default=2048, help="frames per stream in the serving run")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import numpy as np
    import torch

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist = dist_
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2010_12478_gb300 import binding as B
    from paper_2010_12478_gb300 import build, synth
    build.build()
    if args.workload == "c4":
        mixed_batch(args, dev, world, rank, dist)
        return

    spec = workload_spec(args.workload, rank, args.frames)
    ser = synth.make_series(spec, device=dev)
    frames = ser.frames
    N, H, W = frames.shape

    def barrier():
        if dist:
            dist.barrier()

    def make_ctx(mode, tune_execs):
        c = B.Context(B.Config(mode=mode, cluster=args.cluster), device=local)
        c.set_timing(True)
        tuned = {}
        if args.cluster == 0 and not args.quick:
            for ex in tune_execs:
                c.autotune(frames, exec=ex)   # outside every timed region
                tuned[ex] = c.tuned_shape(tuple(frames.shape), ex)
        return c, tuned

    def tuned_cluster(tuned, ex):
        return (tuned.get(ex) or {}).get("cluster", args.cluster)

    def timed(ctx, src, exec_, steps, warmup, split=False, grids=None, grids_host=None):
        for _ in range(warmup):
            ctx.scan(src, schedule="brent_kung", exec=exec_, split=split)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        st_list, tim = [], []
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            # the records as the library wrote them on the host; their conversion to Python
            # objects is bookkeeping of this script and happens after the timed region
            _, st = ctx.scan(src, schedule="brent_kung", exec=exec_, split=split, raw=True)
            st_list.append(st)
            tim.append(ctx.last_timing())
            if grids is not None:
                # the nonrigid result proper: every prefix's control values, back on the host
                ctx.scan_grids(grids)
                grids_host.copy_(grids)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        ms = world_max_ms(e0.elapsed_time(e1) / steps, dist, dev)
        return ms, [B.stats_list(st, ctx.cfg.levels) for st in st_list], tim

    ctx, tuned = make_ctx(args.mode, [args.exec_] + (["plain"] if args.exec_ != "plain" else []))
    cfg = ctx.cfg
    # ---- main timed region (device-resident frames, the workload's stated executor)
    with ClockSampler(local) as clk:
        ms, st_list, tim = timed(ctx, frames, args.exec_, args.steps, args.warmup)
    clocks = clk.summary()
    n_ops = len(st_list[0])
    value = job_rate(N - 1, world, ms)
    ops_per_s = job_rate(n_ops, world, ms)

    # roofline of the operator kernel
    sb = 4 if cfg.storage == "f32" else 2
    alg = sum(algorithmic_bytes(st, H, W, cfg.levels, sb, cfg.mode) for st in st_list) / len(st_list)
    kms = sum(t["op_kernel_ms"] for t in tim) / len(tim)
    launches = sum(t["op_launches"] for t in tim) / len(tim)
    peak, peak_src = peaks()
    achieved = alg / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    kname = "persistent_kernel" if args.exec_ == "persistent" else "op_kernel"
    # the committed figure is for the workload's full series (scaled from a capture of its prefix)
    traffic = profile_traffic(f"{kname}_{args.workload}_{args.mode}", "reg_kernels.cu",
                              "dram bytes per step (scaled)") if N == WORKLOAD_FRAMES[args.workload] else None
    gpu_launches = int(sum(t["op_launches"] + t["pyramid_launches"] for t in tim))
    # the pyramid build (its kernels' event time within the same steps)
    pyr_ms = sum(t["pyramid_ms"] for t in tim) / len(tim)
    pyr_alg = pyramid_bytes(N, H, W, cfg.levels, sb, cfg.mode)
    pyr_gbs = pyr_alg / (pyr_ms / 1e3) / 1e9 if pyr_ms > 0 else 0.0
    pyramid = {"bound": "hbm", "achieved": round(pyr_gbs, 1), "peak": peak, "unit": "GB/s",
               "frac": round(pyr_gbs / peak, 4), "ms_per_step": round(pyr_ms, 3),
               "launches_per_step": sum(t["pyramid_launches"] for t in tim) / len(tim),
               "algorithmic_bytes_per_step": pyr_alg,
               "note": "frames read once, stored levels (with border) and B-spline models written once"}
    ev = np.array([sum(s["evals"]) for s in st_list[0]])
    nl = N - 1
    ev_a, ev_b = ev[:nl], ev[nl:]

    levels = cfg.levels
    forms = phases = e2e = other = serve = prec = reg_series = imbalance = mock = sprod = three = c4 = None
    if args.quick and args.warp:
        reg_series = registered_series(ctx, frames, args.mode, 1, 1, peak, peak_src, world)
    if not args.quick:
        # ---- the other executors on the same workload: one operator per launch, and those launches
        # captured once as a CUDA graph and replayed (same CTAs per operator as the tuned plain path)
        forms = {args.exec_: {"value": round(value, 2), "ms_per_step": round(ms, 3),
                              "cluster": tuned_cluster(tuned, args.exec_)}}
        for ex in ("plain", "graph", "persistent"):
            if ex == args.exec_:
                continue
            if ex == "graph":
                sh = tuned.get("plain") or {}
                gctx = B.Context(B.Config(mode=args.mode, cluster=sh.get("cluster", args.cluster) or 0,
                                          unroll=sh.get("unroll", 0), ctas_per_sm=sh.get("ctas_per_sm", 0)),
                                 device=local)
                gctx.set_timing(True)
                fms, _, ftim = timed(gctx, frames, ex, max(2, args.steps // 2), 2)
                del gctx
            else:
                fms, _, ftim = timed(ctx, frames, ex, max(2, args.steps // 2), 2)
            forms[ex] = {"value": round(job_rate(N - 1, world, fms), 2), "ms_per_step": round(fms, 3),
                         "op_kernel_ms": round(sum(t["op_kernel_ms"] for t in ftim) / len(ftim), 3),
                         "cluster": tuned_cluster(tuned, ex if ex != "graph" else "plain")}
        # ---- "full" vs "scan" (Sec. 5.2): the A leaves to completion, then the B operators
        pms, _, ptim = timed(ctx, frames, args.exec_, 2, 1, split=True)
        leaf_ms = sum(t["leaf_ms"] for t in ptim) / len(ptim)
        dag_ms = sum(t["dag_ms"] for t in ptim) / len(ptim)
        # operator slots: 152 SMs x 3 CTAs per SM / CTAs per operator
        workers = 152 * 3 // max(1, tuned_cluster(tuned, args.exec_) or 8)
        phases = {"exec": args.exec_, "leaf_ops": ptim[0]["leaf_ops"], "dag_ops": ptim[0]["dag_ops"],
                  "leaf_ms": round(leaf_ms, 3), "dag_ms": round(dag_ms, 3),
                  "scan_frames_per_s": round(job_rate(N - 1, world, dag_ms), 2),
                  "full_frames_per_s": round(job_rate(N - 1, world, leaf_ms + dag_ms), 2),
                  "overlapped_full_frames_per_s": round(value, 2),
                  "evals_per_op": {"A": round(float(ev_a.mean()), 2), "B": round(float(ev_b.mean()), 2)},
                  "ms_per_op": {"A": round(leaf_ms / max(1, ptim[0]["leaf_ops"]), 5),
                                "B": round(dag_ms / max(1, ptim[0]["dag_ops"]), 5)},
                  "paper_bounds_context": paper_bounds(N, max(2, workers)),
                  "note": "scan = the B operators given the A leaves (the paper's scan registration); full = "
                          "A then B; overlapped = the main value, where B operators start as soon as their "
                          "inputs exist; paper_bounds_context evaluates the paper's speedup bounds for P "
                          "concurrent operator slots (context only)"}
        # ---- load imbalance of the operators (Sec. 3.2): per-operator work from the evaluation
        # counts, over segments of the series as the paper's ranks would hold them
        imbalance = imbalance_metric(ev_a, [64, 256, 1024])
        # ---- registered series: every frame resampled onto f_0's grid by its prefix, and the mean
        reg_series = registered_series(ctx, frames, args.mode, max(3, args.steps), 3, peak, peak_src, world)
        # ---- end to end: pinned host frames through the C ABI, copies inside the timed region, the
        # prefixes (and for the nonrigid model every prefix's control values) back on the host
        host = frames.cpu().pin_memory()
        grids = grids_host = None
        gbytes = 0
        if args.mode == "nonrigid":
            nx, ny, _ = B.grid_dims(W, H, cfg.grid, cfg.levels)
            grids = torch.empty((N - 1, ny, nx, 2), device=dev)
            grids_host = torch.empty((N - 1, ny, nx, 2), pin_memory=True)
            gbytes = grids.numel() * 4
        ems, _, _ = timed(ctx, host, args.exec_, max(2, args.steps // 2), 1, grids=grids, grids_host=grids_host)
        n_nodes = (N - 1) + B.scan_work("brent_kung", N - 1)
        d2h = 4 * N * levels + 16 + 24 * n_nodes + 144 * n_ops + 20 * (N - 1) + gbytes
        e2e = {"value": round(job_rate(N - 1, world, ems), 2), "unit": UNIT,
               "h2d_bytes_per_step": int(N * H * W * 4), "d2h_bytes_per_step": int(d2h)}
        del grids, grids_host, host
        # ---- the other deformation model on the same workload
        omode = "rigid" if args.mode == "nonrigid" else "nonrigid"
        octx, otuned = make_ctx(omode, [args.exec_])
        oms, ost, _ = timed(octx, frames, args.exec_, max(2, args.steps // 2), 2)
        oev = np.array([sum(s["evals"]) for s in ost[0]])
        other = {"mode": omode, "value": round(job_rate(N - 1, world, oms), 2), "unit": UNIT,
                 "exec": args.exec_, "evals_per_operator": {"mean": round(float(oev.mean()), 2),
                                                            "max": int(oev.max())},
                 "cluster": otuned}
        del octx
        # ---- c2 at the three pyramid levels its description names
        three = three_levels(dev, args.mode, args.exec_) if rank == 0 else None
        # ---- c4: 64 series of mixed sizes, one batched scan per size, three storage types
        c4_res, c4_sizes, _ = mixed_measure(args.mode, dev, world, rank, dist, 1, 1)
        c4 = {"workload": f"c4: {WORKLOAD_TEXT['c4']}", "sizes": c4_sizes, "storage": c4_res,
              "exec": "persistent (one reg_scan_batch per size)",
              "shape_per_size": {str(S): {"cluster": v[0], "ctas_per_sm": v[1]} for S, v in C4_SHAPE.items()}}
        # ---- the nonrigid flow's scalar products on the same workload (Sec. 2.3.1 leaves it open)
        if args.mode == "nonrigid":
            sprod = {}
            shp = tuned.get(args.exec_) or {}
            for name, metric in (("gauss_newton", B.METRIC_GAUSS_NEWTON), ("mean", B.METRIC_MEAN),
                                 ("h1_sigma1", B.METRIC_H1)):
                mctx = B.Context(B.Config(mode="nonrigid", metric=metric, sigma=1.0,
                                          cluster=shp.get("cluster", args.cluster) or 0,
                                          unroll=shp.get("unroll", 0), ctas_per_sm=shp.get("ctas_per_sm", 0)),
                                 device=local)
                mms, mst, _ = timed(mctx, frames, args.exec_, 1, 1)
                mev = np.array([sum(x["evals"]) for x in mst[0]])
                sprod[name] = {"value": round(job_rate(N - 1, world, mms), 2), "unit": UNIT,
                               "evals_per_operator": round(float(mev.mean()), 2), "max_evals": int(mev.max())}
                del mctx
            sprod["note"] = ("gauss_newton: per-point curvature diagonal (the default); mean: the plain "
                             "mean over control points; h1_sigma1: identity + sigma^2 grid Laplacian, "
                             "sigma = 1 grid spacing (the gradient smoothed)")
        if rank == 0:
            # ---- serving: eight Poisson streams, online registration, p50/p99 latency
            serve = {args.mode: serving(dev, args.mode, args.serve_frames),
                     omode: serving(dev, omode, min(args.serve_frames, 256))}
            # ---- precision forms: pyramid storage fp32 / bf16 / fp16
            prec = precision(frames, args.mode)
            # ---- the paper's mock operator on the device queue and the per-depth executor
            mock = mock_study(dev)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not args.quick and world == 1:
        fr = frames[:min(N, 1200)].cpu().numpy()   # as many frames as a bounded sample reaches
        ops1, dt1, sample1 = oracle_sample(fr, cfg, args.oracle_budget)
        opsp, dtp, cores, samplep = oracle_sample_parallel(fr, cfg, args.oracle_budget)
        scale = (N - 1) / n_ops
        cpu = {"value": round(opsp / dtp * scale, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": samplep + f"; {dtp:.1f} s wall, FP64 C; frames/s = operators/s x {N - 1}/{n_ops} "
                                   f"(operators per registered frame of this scan)",
               "single_core": {"value": round(ops1 / dt1 * scale, 4), "cores": 1,
                               "sample": sample1 + f"; {dt1:.1f} s single-threaded"}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}", "frames": N, "H": H,
                       "W": W, "mode": args.mode, "levels": levels, "schedule": "brent_kung",
                       "exec": args.exec_, "cluster": args.cluster or {"autotuned": tuned},
                       "launch_shape": {k: tim[0][k] for k in ("cluster", "unroll", "ctas_per_sm")},
                       "image_model": "quadratic B-spline (nonrigid energy), bilinear (rigid energy)",
                       "stop": f"metric gradient norm < {cfg.tol_grad:g}, at most {cfg.max_iter} steps per level",
                       "l2": "inputs larger than L2 (frames %d MiB > 129 MB L2)" % (N * H * W * 4 >> 20),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "ops_per_s": round(ops_per_s, 2), "operators_per_step": n_ops,
            "evals_per_operator": {"mean": round(float(ev.mean()), 2), "max": int(ev.max()),
                                   "A": round(float(ev_a.mean()), 2), "B": round(float(ev_b.mean()), 2)},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": traffic,
                         "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                         else "fallback 6.8 TB/s",
                         "kernel": f"{kname} (operator kernel)", "algorithmic_bytes_per_step": alg,
                         "kernel_ms_per_step": round(kms, 3), "launches_per_step": launches,
                         "caveat": "issue-bound, not DRAM-bound: the two pyramids of an operator stay in L2 "
                                   "(see the committed ncu summaries); the algorithmic bytes are read from L2 "
                                   "many times over"},
            "pyramid_roofline": pyramid,
            "forms": forms,
            "phases": phases,
            "imbalance": imbalance,
            "mock_operator": mock,
            "registered_series": reg_series,
            "other_mode": other, "scalar_products": sprod, "c2_three_levels": three, "c4_mixed": c4,
            "serving": serve,
            "precision": prec,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": gpu_launches,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def mock_study(dev, n: int = 98304, t_us: float = 20.0, seed: int = 1410):
    """The paper's mock operator (Sec. 5.1) on the device executors: n elements, operators of a
    fixed duration t or of exponentially distributed durations with mean t (Mersenne Twister
    seeded 1410); per scan DAG and executor the device time of the scan.  The per-depth
    executor waits for the slowest operator of every depth; the persistent device queue starts an
    operator as soon as its inputs exist (the GPU's counterpart of the paper's work stealing)."""
    import numpy as np
    from paper_2010_12478_gb300 import binding as B
    ctx = B.Context(B.Config(), device=dev.index or 0)
    vals = np.arange(n, dtype=np.float64) % 7
    out = {"elements": n, "mean_op_us": t_us, "seed": seed, "scans": {}}
    for sched in ("brent_kung", "dissemination", "ladner_fischer", "blelloch"):
        m = B.scan_work(sched, n)
        dyn = np.random.RandomState(seed).exponential(t_us, size=m).clip(0.0, 1.0e5).astype(np.float32)
        row = {"operators": m}
        for kind, us in (("static", np.full(m, t_us, np.float32)), ("dynamic", dyn)):
            for ex in ("level", "persistent"):
                ctx.mock_scan(vals, us, schedule=sched, exec=ex)     # warm-up
                _, ms = ctx.mock_scan(vals, us, schedule=sched, exec=ex)
                row[f"{kind}_{ex}_ms"] = round(ms, 3)
        row["dynamic_queue_speedup"] = round(row["dynamic_level_ms"] / row["dynamic_persistent_ms"], 3)
        out["scans"][sched] = row
    return out


def imbalance_metric(evals, segments):
    """The load-imbalance measure of Sec. 3.2 on measured work: the series' neighbour operators A
    cut into S contiguous segments (as ranks would hold them); per segment the work T_s = sum of
    its operators' energy evaluations; imbalance = (max_s T_s - mean) / mean."""
    import numpy as np
    out = {}
    ev = np.asarray(evals, dtype=np.float64)
    for S in segments:
        if S > len(ev):
            continue
        T = np.array([seg.sum() for seg in np.array_split(ev, S)])
        out[str(S)] = round(float((T.max() - T.mean()) / T.mean()), 4)
    return {"segments": out, "work": "energy evaluations per operator A(f_i, f_i+1)",
            "per_operator": {"mean": round(float(ev.mean()), 2), "max": int(ev.max()),
                             "cv": round(float(ev.std() / ev.mean()), 4)}}


def render_prefix(spec, n):
    """Frames 0..n-1 of the series ``spec`` describes (the same parameters as the full series)."""
    import numpy as np
    from paper_2010_12478_gb300 import synth
    phase, shifts, modes, snr = synth._draw_parameters(spec)
    return np.stack([synth.render_frame(spec, phase, shifts[t], modes, t, float(snr[t])).numpy() for t in range(n)])


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    import torch
    from paper_2010_12478_gb300 import binding as B
    from paper_2010_12478_gb300 import synth
    spec = workload_spec(args.workload, 0)
    N = spec.n_frames
    # the frames a bounded sample can reach (frame triples from the start of the series), rendered
    # exactly as in the full series
    fr = render_prefix(spec, min(N, 1200))
    n_ops = (N - 1) + len(__import__("oracle").dag_brent_kung(N - 1).ops)
    cfg = B.Config(mode=args.mode)
    budget = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample_parallel(fr, cfg, budget)
    tot_ops, tot_dt = 0, 0.0
    sample = ""
    cores = 1
    for _ in range(args.steps):
        ops, dt, cores, sample = oracle_sample_parallel(fr, cfg, budget)
        tot_ops += ops
        tot_dt += dt
    ops_s = tot_ops / tot_dt
    value = ops_s * (N - 1) / n_ops
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * tot_dt / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT[args.workload]}", "frames": N,
                       "H": spec.H, "W": spec.W, "mode": args.mode, "levels": cfg.levels, "schedule": "brent_kung",
                       "image_model": "quadratic B-spline (nonrigid energy), bilinear (rigid energy)",
                       "stop": f"metric gradient norm < {cfg.tol_grad:g}, at most {cfg.max_iter} steps per level"},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {sample} (about {budget:.0f} s); frames/s = operators/s x "
                                       f"{N - 1}/{n_ops}"},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
