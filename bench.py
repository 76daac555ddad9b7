#!/usr/bin/env python3
"""Throughput of the SBR hot path on GB300 (one JSON line on stdout).

Headline metric: Mray-bounces/s of one full pass of the hot path over the
synthetic urban workload at 300 GHz (40 box buildings on an 8 x 5 grid,
51,600 triangles, 10,000,002 geodesic rays, 6 reflections, 1024 receivers):
BVH build, launch + trace + reception + dedup, effective paths with FP64
image-method refinement, path gains and per-receiver PDP / statistics. A
ray-bounce is one closest-hit query plus the reception test of one segment.

The same line carries the H(f) synthesis throughput (H tensors/s) of the
indoor MIMO workload (16x16 UPA to 64-ULA, 1024 subcarriers, H [1024, 64,
256]) in each precision form, the live roofline of the dominant kernel
(the depth-first trace kernel), the oracle's CPU throughput on a bounded sample, an
end-to-end number through host buffers, clocks sampled during the timed
region and the number of library kernels launched.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun: the ranks split the one urban trace by geodesic ray
id, all-gather their deduplicated reception records (the trace's single
exchange step) and merge them with the trace's own min (dist, ray) rule before
the paths are refined (strong scaling); rank 0 prints.
--impl reference times the FP64 CPU oracle on bounded samples of the same
workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "Mray-bounces/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
RAY_REC_BYTES = 64      # one queued ray record (origin, direction, L, id, last surface)
# algorithmic HBM bytes of one ray-bounce of the trace: the ray state (a 64 B
# record) read at the start of the segment and written for the next one
ALG_BYTES_PER_RAY_BOUNCE = 2 * RAY_REC_BYTES
# DRAM bytes of one k_trace_df launch on the headline workload (N = 1000), from
# one ncu capture of the launch (dram__bytes_read.sum + dram__bytes_write.sum)
TRACE_DRAM_BYTES = 21_319_680 + 82_202_880
# warp instructions issued by one k_trace_df launch on the same workload, from
# one ncu capture (smsp__inst_executed.sum). The issue peak is one warp
# instruction per clock on each of the 4 schedulers of the 152 SMs
TRACE_WARP_INST = 2_380_405_416
# SHA-256 (first 16 hex digits) of the trace kernel's source and the local
# headers it includes, as they were when the two counters above were captured.
# Any later edit changes it, and the counters are then reported as null
# (unmeasured) instead of describing a kernel that no longer exists.
TRACE_COUNTERS_SRC = "14f44f1765166e99"
SM_COUNT = 152
SCHEDULERS_PER_SM = 4
SEQ_BYTES = 8           # surface id and face id appended per reflection


def trace_source_hash() -> str:
    """SHA-256 over csrc/trace.cu and every local header it includes (recursively)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2208_10006_gb300", "csrc")
    seen, order, todo = set(), [], ["trace.cu"]
    while todo:
        name = todo.pop(0)
        if name in seen or not os.path.exists(os.path.join(csrc, name)):
            continue
        seen.add(name)
        order.append(name)
        src = open(os.path.join(csrc, name), "rb").read()
        todo += [x.decode() for x in re.findall(rb'#include "([^"]+)"', src)]
    h = hashlib.sha256()
    for name in order:
        h.update(name.encode() + b"\0" + open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def trace_counters_current() -> bool:
    """True when the trace kernel's source is the one the ncu counters describe."""
    return trace_source_hash() == TRACE_COUNTERS_SRC


def issue_roofline(launch_ms, clk, N):
    """Instruction-issue view of the trace kernel: warp instructions per launch
    (counted once by ncu on the N = 1000 workload) over the live launch time,
    against the issue peak at the median SM clock sampled in the timed region."""
    mhz = clk.get("sm_mhz") if clk else None
    if N != 1000 or not mhz or not trace_counters_current():
        return None
    achieved = TRACE_WARP_INST / (launch_ms / 1e3) / 1e9
    peak = SM_COUNT * SCHEDULERS_PER_SM * mhz / 1e3
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "Gwarp-inst/s",
            "frac": achieved / peak, "warp_inst_per_launch": TRACE_WARP_INST,
            "peak_from": "152 SMs x 4 schedulers x 1 warp instruction per clock x median SM clock"}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback"


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def ray_range(R: int, rank: int, world: int):
    """Rank's share of the launch grid's geodesic ids: contiguous, sizes within one."""
    return R * rank // world, R * (rank + 1) // world


def gather_records(keys, vals):
    """The exchange step of a ray-range split trace: every rank's deduplicated
    records (keys [n, 10] int32, vals [n] int64) all-gathered over the process
    group (NCCL on GPUs, gloo on CPU); the identity without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return keys, vals
    world = dist.get_world_size()
    n = torch.tensor([keys.shape[0]], dtype=torch.int64, device=keys.device)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n)
    counts = [int(x.item()) for x in ns]
    m = max(1, max(counts))
    kp = torch.zeros((m, keys.shape[1]), dtype=keys.dtype, device=keys.device)
    vp = torch.zeros(m, dtype=vals.dtype, device=vals.device)
    kp[:keys.shape[0]] = keys
    vp[:vals.shape[0]] = vals
    ks = [torch.empty_like(kp) for _ in range(world)]
    vs = [torch.empty_like(vp) for _ in range(world)]
    dist.all_gather(ks, kp)
    dist.all_gather(vs, vp)
    return (torch.cat([k[:c] for k, c in zip(ks, counts)]), torch.cat([v[:c] for v, c in zip(vs, counts)]))


def reduce_over_ranks(t_total: float, work: float, device=None):
    """Job time = the slowest rank's timed region; work = the sum over ranks.
    Returns (t_max, work_sum); a no-op without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_total, work
    t = torch.tensor([t_total], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(w[0])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling every 10 ms and wait (up to 3 s) for the first sample,
        so that the timed region that follows is covered."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "10"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.perf_counter() + 3.0
            while not self.lines and time.perf_counter() < t_end:
                time.sleep(0.01)
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, window=None) -> dict:
        """Summary of the samples taken in window = (t0, t1) (perf_counter
        seconds; the last sample before t0 counts too), else of all."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        lines = self.lines
        if window is not None:
            before = [x for x in lines if x[0] < window[0]]
            lines = before[-1:] + [x for x in lines if window[0] <= x[0] <= window[1]]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- oracle baseline
def oracle_sample(sc, n_rays: int, n_chunks: int = 16, nthreads=None):
    """Trace n_rays spread over the geodesic id range with the FP64 oracle."""
    import oracle
    R = 10 * sc["N"] ** 2 + 2
    per = max(1, n_rays // n_chunks)
    segs, t_total, cands = 0, 0.0, 0
    for c in range(n_chunks):
        b = (R * c) // n_chunks
        t0 = time.perf_counter()
        cc, fl, cnt = oracle.trace(sc, ray_begin=b, ray_end=min(R, b + per), nthreads=nthreads)
        keys, nprod, allf = oracle.dedup(cc)
        ref = oracle.refine(sc, keys)
        paths = oracle.paths_of(sc, keys, ref)
        oracle.gains(sc, paths)
        t_total += time.perf_counter() - t0
        segs += cnt["segments"]
        cands += len(cc)
    return segs, t_total, per * n_chunks


def l2_probe(torch, dev, mb: int = 32, reps: int = 50) -> float:
    """Device copy between two L2-resident buffers (read + write bytes / time)."""
    n = mb * 1024 * 1024 // 4
    a = torch.ones(n, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    for _ in range(5):
        b.copy_(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.copy_(a)
    e1.record()
    e1.synchronize()
    return 2.0 * n * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


def cpu_baseline(sc, budget_s: float = 15.0):
    import oracle
    oracle.build()
    oracle.alpha(sc["N"])                               # one-off table, cached by the oracle
    n, t = 64, 0.0
    for _ in range(3):                                  # calibrate to about budget_s
        segs, t, rays = oracle_sample(sc, n, 16)
        if t >= budget_s / 3 or n >= 400000:
            break
        n = int(min(400000, max(256, n * budget_s / max(t, 1e-3))))
    # the same oracle on one core, on a smaller sample (about budget_s / 4)
    n1 = int(max(64, rays * (budget_s / 4) / max(t, 1e-3) / oracle.nthreads_default()))
    segs1, t1, rays1 = oracle_sample(sc, n1, 16, nthreads=1)
    return {"value": segs / t / 1e6, "unit": METRIC, "cores": oracle.nthreads_default(),
            "kind": "oracle",
            "sample": "%d rays in 16 evenly spaced id ranges of the %d-ray urban workload, "
                      "trace + dedup + refine + gains (%.1f s, %d ray-bounces)" % (
                          rays, 10 * sc["N"] ** 2 + 2, t, segs),
            "one_core": {"value": segs1 / t1 / 1e6, "cores": 1,
                         "sample": "%d rays, same ranges (%.1f s, %d ray-bounces)" % (rays1, t1, segs1)}}


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    import oracle
    oracle.build()
    sc = scenes.config2()
    cfg = {"workload": "urban_300GHz_8x5_51600tri_N1000_R10000002_K6_1024rx",
           "sample_per_step": "2048 rays in 16 spread id ranges, trace + dedup + refine + gains"}
    for _ in range(args.warmup):
        oracle_sample(sc, 2048, 16)
    segs, t = 0, 0.0
    for _ in range(args.steps):
        s, tt, _ = oracle_sample(sc, 2048, 16)
        segs += s
        t += tt
    value = segs / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": oracle.nthreads_default(),
                             "kind": "oracle", "sample": cfg["sample_per_step"]},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import paper_2208_10006_gb300 as sbr

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2208_10006_gb300 import build as b
    if rank == 0:
        b.build()
    if world > 1:
        torch.distributed.barrier()
    sbr._lib.load()
    peaks, peak_src = load_peaks()

    N_w = {"urban": 1000, "urban_n400": 400}[args.workload]
    sc = scenes.config2(N=N_w)
    d = sbr.scene_to_device(sc)
    N, K = sc["N"], sc["K"]
    # alpha = 0: every trace computes the reception-sphere angle of its launch
    # grid itself, inside the timed step (Sec. II-A.3)
    alpha = 0.0
    fc = float(sc["freqs"][0])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    R = 10 * N * N + 2
    rr = ray_range(R, rank, world)

    def step(dd, df_from=0):
        bvh = sbr.build_bvh(dd["tri"], dd["surface_id"], dd["S"])
        if world == 1:
            tr = sbr.trace(bvh, dd["tx"], dd["rx"], N, K, alpha=alpha, timing=True, depth_first_from=df_from)
            pl = sbr.paths(tr, bvh)
        else:
            # ray-range split (Sec. I: rays traced in parallel): this rank's ids,
            # its deduplicated records all-gathered, merged with the trace's own
            # min (dist, ray) rule, then the paths of the whole grid
            tr = sbr.trace(bvh, dd["tx"], dd["rx"], N, K, alpha=alpha, timing=True, depth_first_from=df_from,
                           ray_range=rr)
            keys, vals = gather_records(*tr.entries())
            pl = sbr.paths(sbr.trace_merge(dd["tx"], dd["rx"], N, K, keys, vals, alpha=alpha), bvh)
        g = sbr.path_gains(pl, dd["mats"], dd["freqs"], dd["gamma"], dd["disp"], dd["pol"])
        pdp, st = sbr.pdp_angles(pl, g, 0, fc, 1e-9, 2048)
        stats = tr.stats()
        return bvh, tr, pl, g, pdp, st, stats

    for _ in range(args.warmup):
        step(d)
    torch.cuda.synchronize()
    c0 = sbr.launch_count()
    step(d)
    torch.cuda.synchronize()
    n_launch = sbr.launch_count() - c0   # library kernels in one step (counted at each launch site)

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()   # sampling before the barrier: the timed region below is covered
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_clk0 = time.perf_counter()
    times, rb, bounce_ms, bounce_bytes = [], 0, 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = step(d)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats = out[-1]
        rb += stats["ray_bounces"]
        q = stats["queue"]
        bounce_ms += sum(stats["bounce_ms"][:K + 1])
        # depth first from bounce 0: each ray's launch direction is decoded from
        # its id and each reflection appends its surface and face id; no ray
        # record goes through memory
        bounce_bytes += SEQ_BYTES * sum(q[1:K + 1])
        del out
    torch.cuda.synchronize()
    clk = clocks.stop(window=(t_clk0, time.perf_counter()))
    t_total = sum(times) / 1e3
    t_total, rb_all = reduce_over_ranks(t_total, float(rb), device=dev)
    value = rb_all / t_total / 1e6
    # the same step with every bounce breadth first (one launch per bounce over
    # compacted ray queues), for comparison
    bf_times, bf_rb = [], 0
    for _ in range(args.steps if world == 1 else 0):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = step(d, df_from=K + 1)
        e1.record()
        e1.synchronize()
        bf_times.append(e0.elapsed_time(e1))
        bf_rb += out[-1]["ray_bounces"]
        del out
    bf_value = bf_rb / (sum(bf_times) / 1e3) / 1e6 if bf_times else None

    # e2e: the same step through the public API from pinned host memory, with the
    # inputs copied in and the path list, gains, PDP and statistics copied out.
    # The inputs live in one pinned buffer (each at a 256-byte aligned offset) and
    # go to the device in one copy per step
    host_parts = {k: v.detach().cpu().contiguous() for k, v in d.items() if isinstance(v, torch.Tensor)}
    offs, nbytes = {}, 0
    for k, v in host_parts.items():
        offs[k] = nbytes
        nbytes += (v.numel() * v.element_size() + 255) // 256 * 256
    host_buf = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    for k, v in host_parts.items():
        b = v.numel() * v.element_size()
        host_buf[offs[k]:offs[k] + b].copy_(v.reshape(-1).view(torch.uint8))

    def unpack(buf):
        out = {}
        for k, v in host_parts.items():
            b = v.numel() * v.element_size()
            out[k] = buf[offs[k]:offs[k] + b].view(v.dtype).view(v.shape)
        return out

    h2d = nbytes
    e2e_t, e2e_rb, d2h = 0.0, 0, 0
    pinned = None   # pinned host destinations of the step's results, sized by the first step
    side = torch.cuda.Stream()   # the path list goes to the host on it while gains and PDP run
    for it in range(0 if args.no_e2e else max(1, args.steps // 2) + 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dd = dict(d)
        dd.update(unpack(host_buf.to(dev, non_blocking=True)))
        bvh = sbr.build_bvh(dd["tri"], dd["surface_id"], dd["S"])
        if world == 1:
            tr = sbr.trace(bvh, dd["tx"], dd["rx"], N, K, alpha=alpha, timing=True)
            pl = sbr.paths(tr, bvh)
        else:
            tr = sbr.trace(bvh, dd["tx"], dd["rx"], N, K, alpha=alpha, timing=True, ray_range=rr)
            keys, vals = gather_records(*tr.entries())
            pl = sbr.paths(sbr.trace_merge(dd["tx"], dd["rx"], N, K, keys, vals, alpha=alpha), bvh)
        ev_pl = torch.cuda.Event()
        ev_pl.record()
        # gains and PDP are enqueued first, so that the device has work while
        # the host enqueues the path list's copies on the side stream
        g = sbr.path_gains(pl, dd["mats"], dd["freqs"], dd["gamma"], dd["disp"], dd["pol"])
        if pinned is None or pinned["rx"].shape[0] != pl.n:
            ex = pl.export()
            pinned = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in ex.items()}
            pinned["pdp"] = torch.empty((max(pl.n_rx, 1), 2048), dtype=torch.float32, pin_memory=True)
            pinned["st"] = torch.empty((max(pl.n_rx, 1), sbr.NSTATS), dtype=torch.float64, pin_memory=True)
        # the PDP kernel writes its results straight into pinned host memory
        pdp, st = sbr.pdp_angles(pl, g, 0, fc, 1e-9, 2048, out=(pinned["pdp"], pinned["st"]))
        side.wait_event(ev_pl)
        pl.export(out=pinned, stream=side)
        for k, v in (("g", g),):
            if k not in pinned or pinned[k].shape != v.shape:
                pinned[k] = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
            pinned[k].copy_(v, non_blocking=True)
        stats = tr.stats()
        torch.cuda.current_stream().wait_stream(side)
        e1.record()
        e1.synchronize()
        if it == 0:
            continue   # the first round sizes the pinned buffers
        e2e_t += e0.elapsed_time(e1) / 1e3
        e2e_rb += stats["ray_bounces"]
        d2h = sum(v.numel() * v.element_size() for v in pinned.values())
    if e2e_t > 0:
        e2e_t, e2e_rb = reduce_over_ranks(e2e_t, float(e2e_rb), device=dev)
    e2e_value = e2e_rb / e2e_t / 1e6 if e2e_t > 0 else None

    synth = None
    if not args.no_synth and rank == 0:
        synth = bench_synthesis(sbr, torch, flush, peaks, peak_src, args)
    batched = None
    if not args.no_batched and rank == 0:
        batched = bench_batched(sbr, torch, args)
    surrogate = None
    if not args.no_surrogate and rank == 0:
        surrogate = bench_surrogate(sbr, torch, args)

    if rank != 0:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
        return 0
    # algorithmic on-chip (L1 + L2) bytes of the traversal, from one instrumented
    # (untimed) trace: 64 B per BVH node fetched (scene and receiver trees), 48 B
    # per triangle tested, plus the ray records. Most node fetches hit in L1, so
    # no fraction is formed against the L2 copy probe, which is given as context
    l2 = None
    bvh_i = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    st_i = sbr.trace(bvh_i, d["tx"], d["rx"], N, K, alpha=alpha, count_visits=True).stats()
    if st_i["ray_bounces"] > 0:
        per_rb = (64.0 * (st_i["node_visits"] + st_i["rx_visits"]) + 48.0 * st_i["tri_tests"]) / st_i["ray_bounces"]
        per_rb += bounce_bytes / max(rb, 1)
        probe = l2_probe(torch, dev)
        ach = per_rb * (rb / args.steps) / (bounce_ms / args.steps / 1e3) / 1e9
        l2 = {"achieved_l1_l2": ach, "unit": "GB/s",
              "l2_copy_probe": probe, "probe": "L2-resident 2 x 32 MB device copy",
              "bytes_per_ray_bounce": per_rb,
              "node_visits_per_ray_bounce": st_i["node_visits"] / st_i["ray_bounces"],
              "tri_tests_per_ray_bounce": st_i["tri_tests"] / st_i["ray_bounces"],
              "rx_visits_per_ray_bounce": st_i["rx_visits"] / st_i["ray_bounces"]}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scenes.config2(), budget_s=args.cpu_budget)
        if synth is not None:
            synthesis_vs_oracle(synth)
    if synth is not None:
        synth.pop("_samples", None)

    # the algorithmic figure: 128 B of ray state per ray-bounce; the
    # depth-first kernel keeps the ray state in registers, so what it moves
    # through memory (streamed_bytes) is far below it
    achieved = ALG_BYTES_PER_RAY_BOUNCE * rb / (bounce_ms / 1e3) / 1e9
    hbm = float(peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    roof = {"kernel": "k_trace_df", "bound": "hbm", "achieved": achieved, "peak": hbm,
            "unit": "GB/s", "frac": achieved / hbm, "traffic": TRACE_DRAM_BYTES if (N == 1000 and trace_counters_current()) else None,
            "counters_source_sha": trace_source_hash(),
            "counters_current": trace_counters_current(),
            "peak_source": peak_src,
            "schedule": "depth first from bounce 0 (one launch per trace)",
            "algorithmic_bytes": "128 B ray state (64 B read + 64 B written) per ray-bounce, "
                                 "x ray-bounces per launch",
            "algorithmic_bytes_per_launch": ALG_BYTES_PER_RAY_BOUNCE * rb / args.steps,
            "streamed_bytes_per_launch": bounce_bytes / args.steps,
            "streamed_bytes": "8 B surface and face id per reflection (launch directions are decoded "
                              "from the ray id)",
            "avg_launch_ms": bounce_ms / args.steps,
            "kernel_share_of_step": bounce_ms / sum(times), "l2": l2,
            "issue": issue_roofline(bounce_ms / args.steps, clk, N)}
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(times),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "urban_300GHz_8x5_51600tri_N%d_R%d_K6_1024rx" % (N, 10 * N * N + 2),
                   "rays": 10 * N * N + 2, "max_bounces": K, "triangles": int(len(sc["tri"])),
                   "receivers": int(len(sc["rx"])), "ray_bounces_per_step": rb // args.steps,
                   "step": "build_bvh+trace+paths+gains+pdp", "l2": "flushed (256 MB write) "
                   "between timed steps",
                   "parallelism": ("rays%d: the launch grid split into contiguous geodesic-id ranges, one "
                                   "per rank; deduplicated records all-gathered and merged" % world
                                   if world > 1 else "single GPU")},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": None if n_launch is None else n_launch * args.steps,
        "launches_per_step": n_launch,
        "clocks": clk,
        "breadth_first": ({"value": bf_value, "unit": METRIC, "ms_per_step": statistics.mean(bf_times)}
                          if bf_times else None),
        "synthesis": synth,
        "batched": batched,
        "surrogate": surrogate,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def bench_synthesis(sbr, torch, flush, peaks, peak_src, args):
    """H(f) tensors/s on the indoor MIMO workload for each precision form."""
    sc = scenes.config3()
    d = sbr.scene_to_device(sc)
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    tr = sbr.trace(bvh, d["tx"], d["rx"], sc["N"], sc["K"])
    pl = sbr.paths(tr, bvh)
    g = sbr.path_gains(pl, d["mats"], d["freqs"], d["gamma"], d["disp"], d["pol"])
    F, Nr, Nt = len(sc["freqs"]), len(sc["rx_elem"]), len(sc["tx_elem"])
    P = pl.n
    out = {"metric": "H(f) tensors/s", "workload":
           "indoor_100GHz_5736tri_N632_K4_UPA16x16_ULA64_F1024", "paths": P,
           "H_shape": [F, Nr, Nt], "forms": {}}
    H = torch.empty((F, Nr, Nt), dtype=torch.complex64, device=d["freqs"].device)
    tc_forms = (sbr.SYNTH_BF16X3, sbr.SYNTH_FP16X3)
    reps = {sbr.SYNTH_BF16X3: max(5, args.steps), sbr.SYNTH_FP16X3: max(5, args.steps),
            sbr.SYNTH_FP32: 3, sbr.SYNTH_FP64: 1}
    names = {sbr.SYNTH_BF16X3: "bf16x3_tcgen05", sbr.SYNTH_FP16X3: "fp16x3_tcgen05",
             sbr.SYNTH_FP32: "fp32_simt", sbr.SYNTH_FP64: "fp64_simt"}
    Href = None
    # sampled (f, q, p) entries of every form, compared with the oracle in the
    # CPU-baseline leg (6 frequencies x 8 receive x 16 transmit elements)
    rng = np.random.default_rng(3)
    fi = np.sort(rng.choice(F, 6, replace=False))
    qi = np.sort(rng.choice(Nr, 8, replace=False))
    pi = np.sort(rng.choice(Nt, 16, replace=False))
    ix = [torch.as_tensor(v, device=d["freqs"].device) for v in (fi, qi, pi)]
    samples = {"f": fi, "q": qi, "p": pi, "forms": {}}
    for prec in (sbr.SYNTH_FP64, sbr.SYNTH_FP32, sbr.SYNTH_BF16X3, sbr.SYNTH_FP16X3):
        try:
            sbr.synthesize_H(pl, g, d["freqs"], d["tx_elem"], d["rx_elem"], 0, prec, out=H)
        except sbr.SbrError as e:
            out["forms"][names[prec]] = {"unavailable": str(e)}
            continue
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps[prec]):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sbr.synthesize_H(pl, g, d["freqs"], d["tx_elem"], d["rx_elem"], 0, prec, out=H)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        t = statistics.median(ts)
        Hc = H.clone()
        samples["forms"][names[prec]] = Hc[ix[0]][:, ix[1]][:, :, ix[2]].cpu().numpy()
        if prec == sbr.SYNTH_FP64:
            Href = Hc
        err = med = None
        if Href is not None:
            d_abs = (Hc - Href).abs()
            a_ref = Href.abs()
            err = float(d_abs.max() / a_ref.max())
            big = a_ref > 1e-3 * a_ref.max()
            med = float((d_abs[big] / a_ref[big]).median()) if bool(big.any()) else None
        bytes_ = 8.0 * F * Nr * Nt
        flops = 8.0 * F * Nr * Nt * P
        entry = {"value": 1.0 / t, "unit": "H tensors/s", "ms": t * 1e3,
                 "achieved_GBps": bytes_ / t / 1e9, "achieved_TFLOPs": flops / t / 1e12,
                 "max_abs_err_vs_gpu_fp64_form_over_max": err,
                 "median_rel_err_vs_gpu_fp64_form_where_abs_gt_1e-3_max": med}
        if prec in tc_forms:
            hbm = float(peaks.get("hbm_gbs", 6800.0))
            tc = float(peaks.get("bf16_tflops", 1900.0))
            t_roof = max(bytes_ / (hbm * 1e9), 3 * flops / (tc * 1e12))
            entry["roofline"] = {"bound": "hbm" if bytes_ / (hbm * 1e9) >= 3 * flops / (tc * 1e12)
                                 else "tensor", "frac": t_roof / t, "peak_source": peak_src}
        out["forms"][names[prec]] = entry
    best = [v for v in out["forms"].values() if "value" in v]
    out["value"] = max(v["value"] for v in best) if best else None
    out["unit"] = "H tensors/s"
    C = sbr.capacity(H, sc["snr_db"])
    out["capacity_bits_per_s_per_hz"] = [float(x) for x in C.cpu()]
    # capacity against the Tx array size (16^2 ... 128^2 UPA, same paths and 64-ULA Rx)
    lam = 299792458.0 / 100e9
    trend = {}
    del H
    for n in (16, 32, 64, 128):
        te = torch.as_tensor(scenes.upa_yz(sc["tx"], n, n, lam / 2), dtype=torch.float64, device="cuda")
        Hn = sbr.synthesize_H(pl, g, d["freqs"], te, d["rx_elem"], 0, sbr.SYNTH_FP16X3)
        trend["%dx%d" % (n, n)] = [float(x) for x in sbr.capacity(Hn, sc["snr_db"]).cpu()]
        del Hn
    out["capacity_vs_tx_array"] = {"snr_db": [float(s) for s in sc["snr_db"]], "bits_per_s_per_hz": trend}
    ex = {k: v.cpu().numpy() for k, v in pl.export().items()}
    samples["paths"] = dict(rx=ex["rx"], nb=ex["nb"], seq=ex["seq"], pts=ex["pts"], L=ex["L"])
    samples["scene"] = sc
    del pl, g, tr, bvh
    out["per_element_reception"] = bench_per_element(sbr, torch, args)
    out["_samples"] = samples
    return out


def synthesis_vs_oracle(synth):
    """CPU-baseline leg for the synthesis: the oracle's direct FP64 sum of Eq.
    13-14 (its own gains, the GPU's path list) on the sampled (f, q, p) entries,
    timed, and each GPU form's per-output error against it."""
    import oracle
    oracle.build()
    smp = synth.pop("_samples")
    sc, paths = smp["scene"], smp["paths"]
    fi, qi, pi = smp["f"], smp["q"], smp["p"]
    t0 = time.perf_counter()
    g_ref = oracle.gains(sc, paths, freqs=sc["freqs"][fi], gamma=sc["gamma_db_km"][fi],
                         disp=sc["disp_deg_km"][fi])
    Ho = oracle.synth_H(paths, g_ref, sc["freqs"][fi], sc["tx"], sc["rx"][0], sc["tx_elem"][pi],
                        sc["rx_elem"][qi])
    t_o = time.perf_counter() - t0
    a = np.abs(Ho)
    big = a > 1e-3 * a.max()
    for name, Hs in smp["forms"].items():
        dH = np.abs(Hs - Ho)
        synth["forms"][name]["vs_oracle_sampled"] = {
            "max_abs_err_over_max": float(dH.max() / a.max()),
            "median_rel_err_where_abs_gt_1e-3_max": float(np.median(dH[big] / a[big]))}
    n = len(fi) * len(qi) * len(pi)
    full = len(sc["freqs"]) * len(sc["rx_elem"]) * len(sc["tx_elem"])
    synth["cpu_baseline"] = {
        "value": n / full / t_o, "unit": "H tensors/s", "cores": oracle.nthreads_default(),
        "kind": "oracle",
        "sample": "%d of the %d entries of H (%d f x %d q x %d p), gains + direct FP64 sum over "
                  "%d paths (%.3f s)" % (n, full, len(fi), len(qi), len(pi), len(paths["rx"]), t_o)}


def bench_per_element(sbr, torch, args):
    """Per-element reception on the indoor MIMO scene with a wide Rx array
    (64-element ULA at 8 cm, 5 m aperture; Fig. 11): every element traced as a
    receiver and its H row synthesised from its own paths, against the
    reference-point form (one traced receiver, near-field element corrections)."""
    sc = scenes.config3(rx_spacing=0.08)
    d = sbr.scene_to_device(sc)
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    rx_el = torch.as_tensor(sc["rx_elem"], dtype=torch.float64, device="cuda")
    F, Nr, Nt = len(sc["freqs"]), len(sc["rx_elem"]), len(sc["tx_elem"])

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = fn()
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return r, statistics.median(ts)

    def chan(rx, lg=0):
        for _ in range(4):
            tr = sbr.trace(bvh, d["tx"], rx, sc["N"], sc["K"], table_log2=lg)
            st = tr.stats(check=False)
            if st["status"] != 3:
                break
            lg = st["table_log2"] + 1
        pl = sbr.paths(tr, bvh)
        return pl, sbr.path_gains(pl, d["mats"], d["freqs"], d["gamma"], d["disp"], d["pol"])

    (pl_e, g_e), ms_chan_e = timed(lambda: chan(rx_el))
    (pl_r, g_r), ms_chan_r = timed(lambda: chan(d["rx"]))
    H_e, ms_syn_e = timed(lambda: sbr.synthesize_H_elements(pl_e, g_e, d["freqs"], d["tx_elem"], sbr.SYNTH_FP32))
    H_r, ms_syn_r = timed(lambda: sbr.synthesize_H(pl_r, g_r, d["freqs"], d["tx_elem"], rx_el, 0,
                                                    sbr.SYNTH_FP16X3))
    # FP32 summation against FP64 on 64 of the subcarriers
    sel = torch.arange(0, F, F // 64, device="cuda")
    fr64 = d["freqs"][sel].contiguous()
    g64 = g_e[:, sel].contiguous() if pl_e.n else g_e
    H64 = sbr.synthesize_H_elements(pl_e, g64, fr64, d["tx_elem"], sbr.SYNTH_FP64)
    H32 = sbr.synthesize_H_elements(pl_e, g64, fr64, d["tx_elem"], sbr.SYNTH_FP32)
    err = float((H32 - H64).abs().max() / H64.abs().max())
    ex = {k: v.cpu().numpy() for k, v in pl_e.export().items()}
    nb, rxi, seq = ex["nb"], ex["rx"], ex["seq"]
    n_paths = np.bincount(rxi, minlength=Nr)
    los = np.zeros(Nr, bool)
    los[rxi[nb == 0]] = True

    def port_power_db(H):   # received power per Rx port, Tx ports combined with phase (mean over f)
        return 10.0 * torch.log10((H.abs() ** 2).sum(2).mean(0)).cpu().numpy()

    pe, pr = port_power_db(H_e), port_power_db(H_r)
    C_e = [float(x) for x in sbr.capacity(H_e, sc["snr_db"]).cpu()]
    C_r = [float(x) for x in sbr.capacity(H_r, sc["snr_db"]).cpu()]
    terms = float(F) * Nt * pl_e.n
    return {"workload": "indoor_100GHz_5736tri_N632_K4_UPA16x16_wideULA64_8cm_F1024",
            "H_shape": [F, Nr, Nt], "paths_per_element": {"min": int(n_paths.min()), "max": int(n_paths.max()),
                                                           "mean": float(n_paths.mean())},
            "elements_with_los": int(los.sum()),
            "distinct_path_sets": len({frozenset(tuple(s[:m]) for s, m in zip(seq[rxi == q], nb[rxi == q]))
                                       for q in range(Nr)}),
            "port_power_db": {"per_element": {"range": float(pe.max() - pe.min()), "std": float(pe.std())},
                              "reference_point": {"range": float(pr.max() - pr.min()), "std": float(pr.std())},
                              "per_element_profile": [round(float(x), 2) for x in pe]},
            "capacity_bits_per_s_per_hz": {"snr_db": [float(s) for s in sc["snr_db"]],
                                           "per_element": C_e, "reference_point": C_r},
            "ms": {"trace_paths_gains_per_element": ms_chan_e, "trace_paths_gains_reference_point": ms_chan_r,
                   "synth_per_element_fp32": ms_syn_e, "synth_reference_point_fp16x3": ms_syn_r},
            "synth_per_element_Gterms_per_s": terms / (ms_syn_e * 1e-3) / 1e9,
            "fp32_max_abs_err_vs_fp64_over_max": err}


def job_ranges(scs, jobs):
    """The ranges a batched workload actually spans."""
    tri = [len(scs[j["scene"]]["tri"]) for j in jobs]
    nt = [len(j["tx_elem"]) for j in jobs]
    nr = [len(j["rx_elem"]) for j in jobs]
    f = [len(j["freqs"]) for j in jobs]
    r = [10 * j["N"] ** 2 + 2 for j in jobs]
    k = [j["K"] for j in jobs]
    upa = sorted({"%dx%d" % (int(round(np.ptp(j["tx_elem"][:, 1]) / max(1e-12, _spacing(j)))) + 1,
                             int(round(np.ptp(j["tx_elem"][:, 2]) / max(1e-12, _spacing(j)))) + 1)
                  for j in jobs}, key=lambda x: [int(v) for v in x.split("x")])
    return {"triangles": [min(tri), max(tri)], "rays": [min(r), max(r)], "max_bounces": [min(k), max(k)],
            "subcarriers": [min(f), max(f)], "tx_elements": [min(nt), max(nt)], "rx_elements": [min(nr), max(nr)],
            "tx_upa": [upa[0], upa[-1]], "max_H_elements": int(max(a * b * c for a, b, c in zip(nt, nr, f)))}


def _spacing(j):
    """Element spacing of a job's arrays (half the carrier wavelength)."""
    return 299792458.0 / float(np.mean(j["freqs"])) / 2.0


def bench_batched(sbr, torch, args):
    """The batched uneven workload: 4096 Tx-Rx jobs over 32 scenes (about 1k
    to 200k triangles, log-spaced), rays 1e5-1e7 log-uniform, K 2-8, 64-1024
    subcarriers, Tx UPAs up to 8 x 8 and Rx ULAs up to 64 elements (Nr x Nt up
    to 64 x 64); the batch (tuned on its first 128 jobs, one CUDA-graph launch
    per run) against a per-pair loop of the single-job calls, with the largest
    H difference between the two. A second batch of 128 jobs reads the array
    range as square Tx UPAs of 1 x 1 ... 64 x 64 elements (up to 4096)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    n_jobs = args.batch_jobs
    scs = [scenes.batch_scene(s, span=32) for s in range(32)]
    jobs = scenes.batch_jobs(scs, n_jobs=n_jobs, seed=4)
    sdev = []
    for sc in scs:   # each scene is traced by ~128 jobs: the SAH top of its BVH pays for its build
        tri = torch.as_tensor(sc["tri"].reshape(-1, 9), dtype=torch.float32, device=dev)
        sid = torch.as_tensor(sc["surface_id"], dtype=torch.int32, device=dev)
        mats = torch.as_tensor(sc["materials"], dtype=torch.float64, device=dev)
        sdev.append((sbr.build_bvh(tri, sid, len(sc["materials"]), sah_top=True), mats))
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    jdev = [dict(scene=j["scene"], N=j["N"], K=j["K"], tx=j["tx"], rx=j["rx"], pol=j["pol"],
                 freqs=t(j["freqs"], torch.float64), gamma=t(j["gamma"], torch.float32),
                 tx_elem=t(j["tx_elem"], torch.float64), rx_elem=t(j["rx_elem"], torch.float64))
            for j in jobs]
    t0 = time.perf_counter()
    sample = [dict(j) for j in jdev[:128]]
    cfg, tune_ms = sbr.batch_tune(sdev, sample)
    tune_s = time.perf_counter() - t0
    del sample
    cfg["path_cap"] = min(2048, 2 * cfg["path_cap"])   # margin over the sample's largest key count
    b = sbr.batch_create(sdev, jdev, config=cfg)
    b.run()                     # capture + first launch
    torch.cuda.synchronize()
    ts = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    n_paths, status, info = b.query()
    t_b = min(ts) / 1e3
    # per-pair loop: the single-job calls for every job, FP16x3 synthesis; each
    # trace computes the alpha of its launch grid (the batch computes one per
    # distinct N when it is created)
    Hs = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    e0.record()
    rb_pp = 0
    for j in jdev:
        bvh, mats = sdev[j["scene"]]
        rx = torch.as_tensor(np.asarray(j["rx"], dtype=np.float64).reshape(1, 3), device=dev)
        tr = sbr.trace(bvh, j["tx"], rx, j["N"], j["K"])
        pl = sbr.paths(tr, bvh)
        g = sbr.path_gains(pl, mats, j["freqs"], j["gamma"], None,
                           sbr.POL_V if j["pol"] == "V" else sbr.POL_H)
        Hs.append(sbr.synthesize_H(pl, g, j["freqs"], j["tx_elem"], j["rx_elem"], 0, sbr.SYNTH_FP16X3))
    e1.record()
    e1.synchronize()
    t_pp = e0.elapsed_time(e1) / 1e3
    wall_pp = time.perf_counter() - w0
    dmax = 0.0
    for H, j, st in zip(Hs, jdev, status):
        if st == 0:
            m = float(H.abs().max())
            if m > 0:
                dmax = max(dmax, float((H - j["H"]).abs().max()) / m)
    rbs = info["ray_bounces"]
    b.free()
    del Hs
    upa = bench_batched_upa(sbr, torch, scs, sdev, cfg, args.batch_upa_jobs) if args.batch_upa_jobs > 0 else None
    out = {"metric": "Tx-Rx jobs/s", "workload": "batched_%djobs_32scenes_R1e5-1e7_K2-8_F64-1024" % n_jobs,
           "ranges": job_ranges(scs, jobs), "upa_64x64": upa,
           "jobs": n_jobs, "rays": info["rays"], "ray_bounces": rbs, "paths": info["paths"],
           "failed_jobs": int((status != 0).sum()),
           "batched": {"ms": t_b * 1e3, "jobs_per_s": n_jobs / t_b, "Mray_bounces_per_s": rbs / t_b / 1e6,
                       "graph_kernels": info["graph_kernels"], "waves": info["n_waves"],
                       "config": info["config"], "tune_s": tune_s, "tune_sample_ms": tune_ms},
           "per_pair_loop": {"ms": t_pp * 1e3, "wall_s": wall_pp, "jobs_per_s": n_jobs / t_pp,
                             "Mray_bounces_per_s": rbs / t_pp / 1e6},
           "speedup": t_pp / t_b,
           "max_abs_dH_over_max_H_batched_vs_per_pair": dmax}
    return out


def bench_batched_upa(sbr, torch, scs, sdev, cfg, n_jobs):
    """The array range read as Tx UPAs: n_jobs jobs (seed 5) over the same 32
    scenes with square Tx UPAs of 2^a x 2^a elements, a uniform in [0, 6]
    (1 x 1 ... 64 x 64, i.e. up to 4096 transmit elements), Rx ULAs up to 64,
    64-1024 subcarriers; one batch run (the configuration tuned for the main
    workload) against the per-pair loop, with the largest H difference."""
    dev = torch.device("cuda", torch.cuda.current_device())
    jobs = scenes.batch_jobs(scs, n_jobs=n_jobs, seed=5, tx_exp_range=(0, 6), square_tx=True)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    jdev = [dict(scene=j["scene"], N=j["N"], K=j["K"], tx=j["tx"], rx=j["rx"], pol=j["pol"],
                 freqs=t(j["freqs"], torch.float64), gamma=t(j["gamma"], torch.float32),
                 tx_elem=t(j["tx_elem"], torch.float64), rx_elem=t(j["rx_elem"], torch.float64))
            for j in jobs]
    b = sbr.batch_create(sdev, jdev, config=dict(cfg))
    b.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b.run()
    e1.record()
    e1.synchronize()
    t_b = e0.elapsed_time(e1) / 1e3
    n_paths, status, info = b.query()
    torch.cuda.synchronize()
    e0.record()
    dmax = 0.0
    for j, st in zip(jdev, status):
        bvh, mats = sdev[j["scene"]]
        rx = torch.as_tensor(np.asarray(j["rx"], dtype=np.float64).reshape(1, 3), device=dev)
        tr = sbr.trace(bvh, j["tx"], rx, j["N"], j["K"])
        pl = sbr.paths(tr, bvh)
        g = sbr.path_gains(pl, mats, j["freqs"], j["gamma"], None, sbr.POL_V if j["pol"] == "V" else sbr.POL_H)
        H = sbr.synthesize_H(pl, g, j["freqs"], j["tx_elem"], j["rx_elem"], 0, sbr.SYNTH_FP16X3)
        if st == 0:
            m = float(H.abs().max())
            if m > 0:
                dmax = max(dmax, float((H - j["H"]).abs().max()) / m)
        del H
    e1.record()
    e1.synchronize()
    t_pp = e0.elapsed_time(e1) / 1e3
    h_bytes = sum(8 * len(j["freqs"]) * len(j["tx_elem"]) * len(j["rx_elem"]) for j in jobs)
    out = {"workload": "batched_%djobs_32scenes_squareUPA1x1-64x64" % n_jobs, "ranges": job_ranges(scs, jobs),
           "jobs_with_64x64_upa": int(sum(len(j["tx_elem"]) == 4096 for j in jobs)),
           "H_bytes": h_bytes, "paths": info["paths"], "failed_jobs": int((status != 0).sum()),
           "batched": {"ms": t_b * 1e3, "jobs_per_s": n_jobs / t_b, "H_GBps": h_bytes / t_b / 1e9},
           "per_pair_loop": {"ms": t_pp * 1e3, "jobs_per_s": n_jobs / t_pp},
           "speedup": t_pp / t_b, "max_abs_dH_over_max_H_batched_vs_per_pair": dmax}
    b.free()
    return out


def bench_surrogate(sbr, torch, args):
    """The learned surrogate on the urban 300 GHz scene (51,600 triangles, Tx
    (240,120,25), 10,000,002 rays, K = 6): targets of 1,048,576 receivers at 8
    frequencies over 280-320 GHz (8,388,608 samples, seed 5) from full SBR,
    training of the 4 x 256 BF16 MLP, evaluation on 1,250 held-out receivers
    at 8 other in-band frequencies (10,000 queries, seed 6) against full SBR,
    and inference throughput against full SBR's per-sample rate."""
    from paper_2208_10006_gb300 import surrogate as S
    sc = scenes.config2()
    f_train = np.linspace(280e9, 320e9, 8)
    f_test = np.sort(np.random.default_rng(6).uniform(280e9, 320e9, 8))
    rx = S.sample_receivers(sc, args.surrogate_rx, seed=5)
    rx_t = S.sample_receivers(sc, 1250, seed=6)
    d = sbr.scene_to_device(sc)
    bvh = sbr.build_bvh(d["tri"], d["surface_id"], d["S"])
    alpha = float(sbr.launch_dirs(sc["N"], with_dirs=False)[1].cpu()[0])
    S.sbr_targets(sc, rx[:16384], f_train, alpha=alpha, dev=d, bvh=bvh)      # warm-up
    t, gen_s = S.sbr_targets(sc, rx, f_train, alpha=alpha, dev=d, bvh=bvh)
    tt, _ = S.sbr_targets(sc, rx_t, f_test, alpha=alpha, dev=d, bvh=bvh)
    X, Y = S.make_xy(rx, f_train, t)
    Xt, Yt = S.make_xy(rx_t, f_test, tt)
    lo, hi = S.x_box(sc, [280e9, 320e9])
    m, hist, train_s = S.train(X, Y, lo, hi, epochs=args.surrogate_epochs)
    ev = S.evaluate(m, Xt, Yt, threshold_db=3.0)
    # inference: one call of (up to) 1,048,576 queries on a copy of the trained model
    nq = min(X.shape[0], 1 << 20)
    Xq = X[:nq].contiguous()
    mi = sbr.MLP(S.N_OUT, lo, hi, max_batch=nq, err_channel=S.CH_ERR, err_of=S.CH_PL, loss_w=S.LOSS_W,
                 y_shift=S.SHIFT, y_scale=S.SCALE, feat_log2_max=S.FEAT_LOG2_MAX)
    mi.params(1, m.params(0))
    out = torch.empty((nq, S.N_OUT), dtype=torch.float32, device="cuda")
    mi.predict(Xq, out=out)
    ts = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        mi.predict(Xq, out=out)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    t_q = min(ts)
    ok = bool(torch.allclose(out[:8192], m.predict(Xq[:8192].contiguous())))
    mi.status()
    flops = 2.0 * nq * (128 * 256 + 3 * 256 * 256 + 256 * 128)
    sbr_rate = X.shape[0] / gen_s
    q = nq / t_q
    for v in ev["fallback"].values():   # throughput with the fallback queries sent to full SBR
        v["queries_per_s"] = 1.0 / ((1.0 - v["fraction"]) / q + v["fraction"] / sbr_rate)
    return {"metric": "surrogate queries/s", "value": nq / t_q, "unit": "queries/s",
            "workload": "urban_300GHz_51600tri_N1000_K6: %d rx x 8 f train, 1250 rx x 8 f held out" % len(rx),
            "train_samples": int(X.shape[0]), "test_queries": int(Xt.shape[0]),
            "sbr_data_s": gen_s, "sbr_samples_per_s": sbr_rate,
            "train_s": train_s, "epochs": args.surrogate_epochs, "loss_first_last": [hist[0], hist[-1]],
            "inference_ms_per_1M": t_q * 1e3 * 1048576 / nq, "inference_TFLOPs": flops / t_q / 1e12,
            "speedup_vs_sbr_per_sample": (nq / t_q) / sbr_rate, "large_batch_matches_small": ok,
            "eval": ev}


def profile_case(case: str) -> int:
    """Small single-purpose runs for ncu captures (no timing, no JSON line):
    synth: the indoor MIMO workload traced, then H synthesised in the FP16x3,
           BF16x3 and FP16x3 tensor-core forms;
    batch: 48 jobs of the batched workload (seed 4) over its first 4 scenes, one
           run with plain stream launches;
    mlp:   three surrogate training steps (batch 8192) and one prediction of
           1,048,576 queries."""
    import torch
    import paper_2208_10006_gb300 as sbr
    from paper_2208_10006_gb300 import build as b
    b.build()
    if case == "synth":
        sc = scenes.config3()
        r = sbr.run_scene(sc)
        d = r["dev"]
        for prec in (sbr.SYNTH_FP16X3, sbr.SYNTH_BF16X3, sbr.SYNTH_FP16X3):
            H = sbr.synthesize_H(r["paths"], r["g"], d["freqs"], d["tx_elem"], d["rx_elem"], 0, prec)
        torch.cuda.synchronize()
        print("synth", r["paths"].n, float(H.abs().max()))
    elif case == "batch":
        scs = [scenes.batch_scene(s, span=32) for s in range(4)]
        jobs = scenes.batch_jobs(scs, n_jobs=48, seed=4)
        dev = torch.device("cuda")
        sdev = []
        for sc in scs:
            tri = torch.as_tensor(sc["tri"].reshape(-1, 9), dtype=torch.float32, device=dev)
            sid = torch.as_tensor(sc["surface_id"], dtype=torch.int32, device=dev)
            mats = torch.as_tensor(sc["materials"], dtype=torch.float64, device=dev)
            sdev.append((sbr.build_bvh(tri, sid, len(sc["materials"]), sah_top=True), mats))
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        jdev = [dict(scene=j["scene"], N=j["N"], K=j["K"], tx=j["tx"], rx=j["rx"], pol=j["pol"],
                     freqs=t(j["freqs"], torch.float64), gamma=t(j["gamma"], torch.float32),
                     tx_elem=t(j["tx_elem"], torch.float64), rx_elem=t(j["rx_elem"], torch.float64))
                for j in jobs]
        bt = sbr.batch_create(sdev, jdev, config=dict(path_cap=256, tile_n=64, use_graph=0))
        bt.run()
        n, st, info = bt.query()
        print("batch", info["rays"], info["ray_bounces"], int((st != 0).sum()))
    elif case == "mlp":
        from paper_2208_10006_gb300 import surrogate as S
        rng = np.random.default_rng(0)
        B = 8192
        x = torch.tensor(np.column_stack([rng.uniform(0, 1, B) for _ in range(4)]).astype(np.float32), device="cuda")
        y = torch.tensor(rng.normal(size=(B, S.N_OUT)).astype(np.float32), device="cuda")
        m = sbr.MLP(S.N_OUT, [0] * 4, [1] * 4, max_batch=B, err_channel=S.CH_ERR, err_of=S.CH_PL)
        for _ in range(3):
            m.train_step(x, y)
        big = torch.tensor(rng.uniform(0, 1, (1 << 20, 4)).astype(np.float32), device="cuda")
        mi = sbr.MLP(S.N_OUT, [0] * 4, [1] * 4, max_batch=1 << 20)
        mi.predict(big)
        torch.cuda.synchronize()
        m.status()
        print("mlp ok")
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-synth", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--profile-case", choices=["synth", "batch", "mlp"], default=None,
                    help="run one small workload for an ncu capture and exit")
    ap.add_argument("--surrogate-rx", type=int, default=1048576)
    ap.add_argument("--surrogate-epochs", type=int, default=40)
    ap.add_argument("--batch-jobs", type=int, default=4096)
    ap.add_argument("--batch-upa-jobs", type=int, default=128,
                    help="jobs of the square-UPA (up to 64 x 64) batch; 0 skips it")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="urban", choices=["urban", "urban_n400"],
                    help="urban: the headline workload; urban_n400: 1.6M rays (profiling case)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
