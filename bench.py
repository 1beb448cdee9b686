#!/usr/bin/env python3
"""Benchmark: CGLS iterations/s and ray-voxel updates/s of A and A^T at 256^3.

Workload (the 256^3 configuration): 256^3 FP32 volume of 1 mm voxels holding a
seeded 40-ellipsoid phantom, 384 x 288 detector of 1 mm pixels, 360 views over
360 degrees, SID 750 mm, SDD 1200 mm; b = A x_true.  One step = one ct_cgls
call of ``--iters`` x updates (default 50, as the configuration states; ERR = 0,
x0 = 0), i.e. the whole hot path: A, A^T, the fused vector updates and the FP64
Krylov scalars, with the update replayed as a CUDA graph (the product path).
The line also carries LSQR and preconditioned CGLS/LSQR rates on the same
workload, per-operator times from a separate event-timed solve, and a served
request stream.

Prints ONE JSON line (rank 0).  ``value`` = CGLS iterations per second over
all ranks (each rank solves its own replica: the path has no exchange step).
``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CGLS iters/s and Gray-voxel/s (A, Aᵀ) at 256³; served p50/p99 latency"
WORKLOAD = ("B256: 256^3 FP32 volume (1 mm voxels, 40 random ellipsoids, seed 1), 384x288 "
            "detector (1 mm pixels), 360 views over 360 deg, SID 750 mm, SDD 1200 mm; "
            "b = A x_true; one step = ct_cgls with ERR=0, x0=0")
PEAK_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=50, help="CGLS x updates per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="cgls", choices=["cgls", "ops", "serve", "precision", "pr1",
                                                     "diff"],
                    help="ops: time ct_project and ct_backproject alone (profiling aid); "
                         "serve: the continuous-batching request stream alone; pr1: A, A^T "
                         "and CGLS-20 on the 64^3 PR1 case, GPU beside the oracle; diff: the batched "
                         "autograd operators on 8 x 128^3 volumes")
    ap.add_argument("--requests", type=int, default=128, help="serve mode: requests")
    ap.add_argument("--rate", type=float, default=20.0, help="serve mode: arrivals per second")
    ap.add_argument("--slots", type=int, default=8, help="serve mode: concurrent jobs")
    ap.add_argument("--batched", action="store_true",
                    help="serve mode: FP32 CGLS requests join one ct_batch (batched projector "
                         "launches, iteration-level scheduling)")
    ap.add_argument("--batch-executors", type=int, default=1,
                    help="serve mode with --batched: batches on their own streams")
    ap.add_argument("--no-serve-equal-error", dest="serve_equal_error", action="store_false",
                    help="default mode: skip the FP32/FP16 served streams at equal error")
    ap.add_argument("--max-iter", type=int, default=50,
                    help="serve mode: update cap per request (the stop rule is NB/NB0 <= 1e-3)")
    ap.add_argument("--batch-route", default="load", choices=["load", "size"],
                    help="serve mode with --batched: a request goes to the least loaded batch, "
                         "or to the batch of its volume size")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="serve mode: CGLS Krylov-vector storage")
    ap.add_argument("--serve-requests", type=int, default=128,
                    help="default mode: requests of the served-latency block (0 = skip)")
    ap.add_argument("--workload", default="B256", choices=["B256", "P512"],
                    help="ops mode only: 256^3 (default) or the 512^3, 720-view workload")
    ap.add_argument("--projector", default="siddon", choices=["siddon", "sf_tr", "sf_tt"],
                    help="ops mode only: Siddon rays or separable footprints (TR, TT)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"],
                    help="ops mode only: storage of the volume and sinogram (FP32 sums)")
    ap.add_argument("--views", type=int, default=0,
                    help="ops mode only: use this many of the workload's views, evenly spread "
                         "(a smaller case of the same kernels for profiling)")
    ap.add_argument("--cpu-sample-views", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, device=None) -> float:
    """Max of a per-rank scalar over all ranks (the job is as slow as its
    slowest rank); the value itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units processed by all ranks together per second of the slowest rank."""
    return world * units_per_rank / (ms_max * 1e-3)


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[4 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def ncu_counters(kernel: str):
    """The committed ncu counters of a projector kernel (DRAM bytes per launch,
    L1 and L2 hit rates, the fraction of issue slots busy), or None when the
    kernel source changed since they were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2110_13526_gb300", "csrc", "projector.cu")
    try:
        with open(p) as f:
            d = json.load(f)
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        ent = d.get(kernel)
        if ent and ent.get("projector_sha256") == sha:
            return ent
    except Exception:
        pass
    return None


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, or None."""
    ent = ncu_counters(kernel)
    return float(ent["dram_bytes_per_launch"]) if ent else None


def issue_roofline(ent: dict, seconds: float, clk: dict):
    """The instruction-issue roofline of a projector kernel: its warp
    instructions per launch (committed ncu count for the same source) over the
    live launch time, against 4 warp instructions per clock on each of the
    152 SMs at the median SM clock sampled under load (the maximum clock when
    no sample was taken).  None when the source changed since the count."""
    n = ent.get("warp_inst_per_launch") if ent else None
    if not n:
        return None
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    peak = 4.0 * 152 * mhz * 1e6
    out = {"bound": "alu", "achieved": n / seconds, "peak": peak, "unit": "warp-inst/s",
           "frac": n / seconds / peak, "warp_inst_per_launch": n,
           "peak_meaning": "4 warp instructions per clock per SM x 152 SMs x %.0f MHz" % mhz}
    sec = ent.get("red_sectors_per_launch")
    if sec:
        out["l2_reduction_sectors_per_s"] = sec / seconds
    return out


def kernel_report(kernel: str, seconds: float, nnz: int, algo_bytes: float) -> dict:
    """Per-kernel figures: live CUDA-event time, ray-voxel updates per second
    and effective gather bandwidth; DRAM bandwidth (ncu bytes over the live
    time) and L1/L2 hit rates from the committed ncu counters."""
    ent = ncu_counters(kernel) or {}
    dram = ent.get("dram_bytes_per_launch")
    return {"ms_per_launch": seconds * 1e3, "gray_voxel_per_s": nnz / seconds / 1e9,
            "effective_gbs": algo_bytes / seconds / 1e9,
            "dram_gbs": dram / seconds / 1e9 if dram is not None else None,
            "l1_hit_rate": ent.get("l1_hit_rate"), "l2_hit_rate": ent.get("l2_hit_rate"),
            "issue_busy": ent.get("issue_active"),
            "counters": "ncu" if ent else None}


PHANTOM_SEED = {"B256": 1, "P512": 2}


def make_problem(ct, torch, synth, dev, workload="B256", projector="siddon"):
    cfg = synth.CONFIGS[workload]
    g = ct.Geometry(**cfg, projector=projector)
    lo, hi = synth.box_of(cfg)
    x_true = torch.from_numpy(synth.voxelize(synth.random_ellipsoids(40, PHANTOM_SEED[workload],
                                                                     lo, hi), cfg)).to(dev)
    b = ct.project(g, x_true)
    torch.cuda.synchronize()
    return cfg, g, x_true, b


def cpu_baseline(cfg, views_n, iters_per_step):
    """The oracle (FP64 C, OpenMP) on a bounded sample: A and A^T on
    ``views_n`` of the 360 views, extrapolated to one CGLS iteration."""
    import numpy as np
    import oracle
    import synth
    oracle.build()
    og_full = oracle.OGeom(**cfg)
    views = [int(round(k * cfg["nviews"] / views_n)) % cfg["nviews"] for k in range(views_n)]
    og = og_full.subset(views)
    lo, hi = synth.box_of(cfg)
    x = synth.voxelize(synth.random_ellipsoids(40, 1, lo, hi), cfg).astype(np.float64)
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    p = oracle.project(og, x, threads)
    t1 = time.perf_counter()
    oracle.backproject(og, p, threads)
    t2 = time.perf_counter()
    scale = cfg["nviews"] / views_n
    t_iter = (t2 - t0) * scale
    return {"value": 1.0 / t_iter, "unit": "iters/s", "cores": threads, "kind": "oracle",
            "sample": "A and A^T on %d of %d views (%.1f s + %.1f s), extrapolated x%.0f to "
                      "one CGLS iteration (vector updates not counted)"
                      % (views_n, cfg["nviews"], t1 - t0, t2 - t1, scale),
            "seconds": t2 - t0}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    cfg = synth.CONFIGS["B256"]
    vals = []
    for _ in range(max(a.warmup, 0)):
        cpu_baseline(cfg, a.cpu_sample_views, a.iters)
    t_total = 0.0
    last = None
    for s in range(a.steps):
        last = cpu_baseline(cfg, a.cpu_sample_views, a.iters)
        vals.append(last["value"])
        t_total += last["seconds"]
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "ms_per_step": 1000.0 * t_total / max(a.steps, 1),
            "config": {"workload": WORKLOAD, "sample_views": a.cpu_sample_views},
            "cpu_baseline": {"kind": "oracle", "cores": last["cores"], "sample": last["sample"],
                             "value": value, "unit": "iters/s"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(a):
    import torch
    import torch.distributed as dist

    import paper_2110_13526_gb300 as ct
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    cfg, g, x_true, b = make_problem(ct, torch, synth, dev)
    nnz = ct.count_nnz(g)
    n_vox, n_rays = g.sizes()
    K = a.iters

    def step():
        # the product path: ct_cgls replays one captured update as a CUDA graph
        return ct.cgls(g, b, max_iter=K)

    for _ in range(max(a.warmup, 0)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    l0 = ct.kernel_launches()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(a.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = (ct.kernel_launches() - l0) // max(a.steps, 1)
    ms = reduce_max(ev0.elapsed_time(ev1), dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()

    # per-operator times from a separate solve with CUDA events around every
    # projector launch (no graph replay), outside the timed region
    _, rep = ct.cgls(g, b, max_iter=K, timing=True)
    ms_f, ms_b, nf, nb = rep.ms_forward, rep.ms_back, rep.n_forward, rep.n_back

    # the rest of the 256^3 configuration: LSQR and preconditioned solves,
    # K updates each (weights computed inside the call), one timed call each
    solvers = {}
    for name, fn, pc in (("lsqr", ct.lsqr, "none"), ("cgls_jacobi", ct.cgls, "jacobi"),
                         ("cgls_rowcol", ct.cgls, "rowcol"), ("lsqr_rowcol", ct.lsqr, "rowcol")):
        fn(g, b, max_iter=2, precond=pc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, r = fn(g, b, max_iter=K, precond=pc)
        e1.record(stream)
        torch.cuda.synchronize()
        solvers[name] = {"iters_per_s": K / (e0.elapsed_time(e1) * 1e-3),
                         "nb_over_nb0": r.history[-1] if r.history else None}

    # end to end through the public API with host buffers: pinned b in, x out
    b_host = b.cpu().pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.e2e_steps):
        xh, _ = ct.cgls(g, b_host, max_iter=K)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / a.e2e_steps
    e2e_value = world * K / e2e_s

    peak, peak_kind = measured_peak_gbs()
    t_f = ms_f / max(nf, 1) * 1e-3           # s per launch of the forward kernel
    t_b = ms_b / max(nb, 1) * 1e-3
    bytes_f = 4.0 * nnz + 4.0 * n_rays        # one voxel load per ray-voxel pair + sinogram out
    bytes_b = 4.0 * nnz + 4.0 * n_vox         # one voxel update per pair + volume out
    dom = "forward" if ms_f >= ms_b else "backward"
    t_dom, by_dom = (t_f, bytes_f) if dom == "forward" else (t_b, bytes_b)
    achieved = by_dom / t_dom / 1e9
    # the 256^3 geometry has no ray advancing mostly along z, so A and A^T run
    # the column-major kernels
    kname = "k_forward_cm" if dom == "forward" else "k_backward_cm"
    ent = ncu_counters(kname) or {}
    dram = traffic_for(kname)
    # The projector reads (or reduces into) one voxel per ray-voxel pair, but
    # those accesses hit L1/L2: DRAM carries only the compulsory streams.  The
    # binding unit is the on-chip gather (A: L1/L2 hit latency; A^T: issue and
    # L1/L2 reduction throughput), so "bound" names it; the algorithmic bytes
    # per second are still set against the measured HBM copy peak as the
    # effective-bandwidth figure, with the real DRAM rate beside it.
    roof = {"bound": "l1_l2_gather", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": dram,
            "frac_meaning": "effective gather bandwidth (algorithmic bytes / time) over the "
                            "measured HBM copy peak (%s)" % peak_kind,
            "dram_gbs": dram / t_dom / 1e9 if dram is not None else None,
            "dram_frac": dram / t_dom / 1e9 / peak if dram is not None else None,
            "l1_hit_rate": ent.get("l1_hit_rate"), "l2_hit_rate": ent.get("l2_hit_rate"),
            "issue_busy": ent.get("issue_active"),
            "kernel": kname, "peak_source": peak_kind,
            "ms_per_launch": t_dom * 1e3,
            "algorithmic_bytes_per_launch": by_dom,
            "issue": issue_roofline(ent, t_dom, clk)}
    value = whole_job_rate(a.steps * K, world, ms)
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "cgls_iters_per_step": K,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (sinogram 159 MB; working set ~0.8 GB)",
                       "nnz": nnz},
            "gray_voxel_per_s": {"A": nnz / t_f / 1e9, "AT": nnz / t_b / 1e9},
            "ms_per_op": {"A": t_f * 1e3, "AT": t_b * 1e3},
            "kernels": {"k_forward_cm": kernel_report("k_forward_cm", t_f, nnz, bytes_f),
                        "k_backward_cm": kernel_report("k_backward_cm", t_b, nnz, bytes_b)},
            "solvers": solvers,
            "roofline": roof,
            "e2e": {"value": e2e_value, "unit": "iters/s",
                    "h2d_bytes_per_step": 4 * n_rays, "d2h_bytes_per_step": 4 * n_vox},
            "gpu_launches": int(launches) * a.steps,
            "clocks": clk}
    if a.serve_requests > 0:
        line["served"] = serve_stream(a.serve_requests, 20.0, 8)
        if a.serve_equal_error:
            # the served form with reduced-precision storage against FP32 at
            # equal reconstruction error: every request run to NB/NB0 <= 1e-3
            line["served_equal_error"] = {
                "max_iter": 200,
                "f32": serve_stream(a.serve_requests, 20.0, 8, max_iter=200),
                "f16": serve_stream(a.serve_requests, 20.0, 8, storage="f16", max_iter=200)}
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cb = cpu_baseline(cfg, a.cpu_sample_views, K)
        cb.pop("seconds", None)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_ops(a):
    """A and A^T alone on the 256^3 (or 512^3) workload: W warm-up pairs, then
    K timed pairs, each launch bracketed by CUDA events on the current stream.
    A projects the phantom; A^T backprojects a dense seeded residual (like
    CGLS's, every ray nonzero).  --views V keeps V evenly spread views."""
    import torch

    import paper_2110_13526_gb300 as ct
    import synth

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cfg = dict(synth.CONFIGS[a.workload])
    if a.views:
        import math
        cfg["angles"] = [2.0 * math.pi * k / a.views for k in range(a.views)]
        cfg["nviews"] = a.views
    g = ct.Geometry(**cfg, projector=a.projector)
    lo, hi = synth.box_of(cfg)
    x_true = torch.from_numpy(synth.voxelize(synth.random_ellipsoids(
        40, PHANTOM_SEED[a.workload], lo, hi), cfg)).to(dev)
    e = torch.from_numpy(synth.random_field(g.sino_shape, seed=7)).to(dev)
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[a.dtype]
    x_true, e = x_true.to(dt), e.to(dt)
    nnz = ct.count_nnz(g)
    r = torch.empty(g.vol_shape, device="cuda", dtype=dt)
    p = torch.empty(g.sino_shape, device="cuda", dtype=dt)
    for _ in range(a.warmup):
        ct.project(g, x_true, out=p)
        ct.backproject(g, e, out=r)
    stream = torch.cuda.current_stream()
    tf, tb = [], []
    for _ in range(a.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        ct.project(g, x_true, out=p)
        ev[1].record(stream)
        ct.backproject(g, e, out=r)
        ev[2].record(stream)
        torch.cuda.synchronize()
        tf.append(ev[0].elapsed_time(ev[1]))
        tb.append(ev[1].elapsed_time(ev[2]))
    mf, mb = statistics.median(tf), statistics.median(tb)
    print(json.dumps({"mode": "ops", "config": {"workload": a.workload, "nnz": nnz,
                                                "views": cfg["nviews"], "dtype": a.dtype,
                                                "projector": a.projector},
                      "ms_project": mf, "ms_backproject": mb,
                      "gray_voxel_per_s": {"A": nnz / mf / 1e6, "AT": nnz / mb / 1e6},
                      "note": "ct_project / ct_backproject calls, including the transpose "
                              "and combine kernels around the projector kernel; A^T of a "
                              "dense residual"}))
    return 0


_SERVE_CACHE = {}


def serve_requests(n_requests: int, rate: float):
    """The requests of the serving stream (built once per process: the
    phantoms, their projections and the geometries): Poisson arrivals
    (seed 3), volumes 64..256^3, 60..360 views, detector scaled to
    magnification 1.6, CGLS or LSQR."""
    import torch

    import paper_2110_13526_gb300 as ct
    import synth
    from paper_2110_13526_gb300.serving import Request

    key = (n_requests, rate)
    if key in _SERVE_CACHE:
        return _SERVE_CACHE[key]
    stream = synth.serving_stream(n_requests, rate, 3)
    reqs, geoms = [], {}
    for s in stream:
        cfg = synth.serving_geometry(s["n"], s["views"])
        gk = (s["n"], s["views"])
        if gk not in geoms:
            geoms[gk] = ct.Geometry(**cfg)
        x = torch.from_numpy(synth.serving_phantom(s["n"], s["phantom_seed"])).cuda()
        b = ct.project(geoms[gk], x)
        reqs.append(Request(s["rid"], cfg, b, s["solver"], s["arrival"], max_iter=50,
                            err_tol=1e-3))
    torch.cuda.synchronize()
    _SERVE_CACHE[key] = reqs
    return reqs


def serve_stream(n_requests: int, rate: float, slots: int, budget_gb: float = 150.0,
                 storage: str = "f32", batched: bool = False, batch_executors: int = 1,
                 batch_route: str = "load", max_iter: int = 50):
    """Serving workload (serve_requests), each request solved to relative
    discrepancy 1e-3 or max_iter updates, CGLS Krylov vectors in ``storage``;
    continuous batching over ``slots`` streams under an HBM budget.  Returns
    the stats dict of the run."""
    import dataclasses

    from paper_2110_13526_gb300.serving import Server

    reqs = [dataclasses.replace(r, max_iter=max_iter, storage=storage)
            for r in serve_requests(n_requests, rate)]
    stats = Server(slots=slots, hbm_budget_bytes=budget_gb * 1e9, batched=batched,
                   batch_executors=batch_executors, batch_route=batch_route).run(reqs)
    iters = stats.iterations
    reached = sum(1 for r in stats.results if r.rel_discrepancy <= 1e-3)
    return {"requests": len(reqs), "rate_per_s": rate, "slots": slots,
            "arrival_rate_per_s": rate, "served_per_s": len(reqs) / stats.wall_s,
            "max_iter": max_iter, "reached_1e-3": reached,
            "max_rel_discrepancy": float(max((r.rel_discrepancy for r in stats.results),
                                             default=0.0)),
            "p50_s": stats.p50, "p99_s": stats.p99, "wall_s": stats.wall_s,
            "requests_per_s": len(reqs) / stats.wall_s, "solver_iters_per_s": iters / stats.wall_s,
            "max_concurrent": stats.max_concurrent,
            "max_gb_in_use": stats.max_bytes_in_use / 1e9,
            "mean_iterations": iters / max(len(reqs), 1),
            "storage": storage,
            "batched": batched, "batch_executors": batch_executors if batched else 0,
            "batch_route": batch_route if batched else None,
            "batch_steps": stats.extra.get("batch_steps", 0),
            "mean_rel_discrepancy": float(sum(r.rel_discrepancy for r in stats.results)
                                          / max(len(stats.results), 1)),
            "workload": "Poisson arrivals (seed 3); n in {64,128,192,256}, views in "
                        "{60,120,180,360}, detector 1.5n x 1.125n of 1.6 mm; CGLS/LSQR to "
                        "1e-3 or %d updates; 8-ellipsoid phantoms; CGLS Krylov storage "
                        % max_iter + storage + " (LSQR FP32)"}


def run_precision(a):
    """The 512^3 precision workload: 0.5 mm voxels, 768x576 detector of
    0.75 mm pixels, 720 views; 40-ellipsoid phantom (seed 2); Poisson noise at
    1e5 photons per ray with mu = 0.02 / mm per unit density (seed 2);
    CGLS with FP32, BF16 and FP16 Krylov storage.  Errors: the reconstruction
    against the FP32-storage run, and A applied to the phantom stored in each
    type against the FP64 oracle on 16 sampled views."""
    import numpy as np
    import torch

    import oracle
    import paper_2110_13526_gb300 as ct
    import synth

    torch.cuda.set_device(0)
    cfg = synth.CONFIGS["P512"]
    g = ct.Geometry(**cfg)
    lo, hi = synth.box_of(cfg)
    x_np = synth.voxelize(synth.random_ellipsoids(40, 2, lo, hi), cfg)
    x_true = torch.from_numpy(x_np).cuda()
    mu, i0 = 0.02, 1e5
    ax = ct.project(g, x_true)
    gen = torch.Generator(device="cuda").manual_seed(2)
    counts = torch.poisson(i0 * torch.exp(-mu * ax.double()), generator=gen)
    b = (-torch.log(torch.clamp(counts, min=1.0) / i0) / mu).float()
    del counts, ax
    K = a.iters
    res = {}
    xs = {}
    for st in ("f32", "bf16", "f16"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, rep = ct.cgls(g, b, max_iter=K, storage=st, timing=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        xs[st] = x
        res[st] = {"s_per_iter": dt / K, "iters_per_s": K / dt,
                   "ms_A": rep.ms_forward / max(rep.n_forward, 1),
                   "ms_AT": rep.ms_back / max(rep.n_back, 1),
                   "rel_discrepancy": rep.history[-1]}
    for st in ("bf16", "f16"):
        res[st]["x_rel_l2_vs_f32"] = float((xs[st] - xs["f32"]).norm() / xs["f32"].norm())
    views = [int(round(k * cfg["nviews"] / 16)) % cfg["nviews"] for k in range(16)]
    og = oracle.OGeom(**cfg).subset(views)
    want = oracle.project(og, x_np.astype(np.float64))
    for st, dt in (("f32", torch.float32), ("bf16", torch.bfloat16), ("f16", torch.float16)):
        p = ct.project(g, x_true.to(dt), out_dtype=dt)[views].double().cpu().numpy()
        res[st]["A_rel_l2_vs_oracle_16_views"] = float(np.linalg.norm(p - want)
                                                       / np.linalg.norm(want))
    print(json.dumps({"mode": "precision", "workload": "P512: 512^3 (0.5 mm), 768x576 (0.75 mm), "
                      "720 views, Poisson 1e5 photons/ray, CGLS %d updates" % K,
                      "results": res}))
    return 0


def run_serve(a):
    import torch
    torch.cuda.set_device(0)
    out = {"mode": "serve"}
    out.update(serve_stream(a.requests, a.rate, a.slots, storage=a.storage, batched=a.batched,
                            batch_executors=a.batch_executors, batch_route=a.batch_route,
                            max_iter=a.max_iter))
    print(json.dumps(out))
    return 0


def run_pr1(a):
    """The 64^3, 90-view PR1 case on both sides: the GPU's A and A^T
    (CUDA events, median of 20) and ct_cgls with 20 updates (wall time with a
    device sync, median of 5), beside the oracle's full A and A^T and its
    CGLS-20 (FP64, OpenMP, on the host cores).  Each side projects its own b
    from the same phantom and adds the same seeded 1 % noise."""
    import numpy as np
    import torch

    import paper_2110_13526_gb300 as ct
    import synth

    torch.cuda.set_device(0)
    cfg = synth.CONFIGS["PR1"]
    g = ct.Geometry(**cfg)
    x_true = synth.voxelize(synth.nested_phantom(64.0, seed=0), cfg)
    xd = torch.from_numpy(x_true).cuda()
    b_gpu = synth.gaussian_noise(ct.project(g, xd).cpu().numpy(), 0.01, seed=0)
    bd = torch.from_numpy(b_gpu.astype(np.float32)).cuda()
    y = torch.randn(g.sino_shape, device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    p = torch.empty(g.sino_shape, device="cuda")
    r = torch.empty(g.vol_shape, device="cuda")
    stream = torch.cuda.current_stream()

    def ev(fn, n):
        ts = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    for _ in range(max(a.warmup, 3)):
        ct.project(g, xd, out=p)
        ct.backproject(g, y, out=r)
        ct.cgls(g, bd, max_iter=20)
    ms_a = ev(lambda: ct.project(g, xd, out=p), 20)
    ms_at = ev(lambda: ct.backproject(g, y, out=r), 20)
    walls = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = ct.cgls(g, bd, max_iter=20)
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
    gpu = {"A_ms": ms_a, "AT_ms": ms_at, "cgls20_s": statistics.median(walls),
           "cgls20_nb_over_nb0": rep.history[-1]}

    import oracle
    from oracle.solvers import cgls as ocgls
    oracle.build()
    og = oracle.OGeom(**cfg)
    th = oracle.default_threads()
    x64 = x_true.astype(np.float64)
    t0 = time.perf_counter()
    p64 = oracle.project(og, x64, th)
    t1 = time.perf_counter()
    oracle.backproject(og, p64, th)
    t2 = time.perf_counter()
    b_or = synth.gaussian_noise(p64, 0.01, seed=0)
    t3 = time.perf_counter()
    res = ocgls(oracle.Operator(og, th), b_or, K=20)
    t4 = time.perf_counter()
    orc = {"A_s": t1 - t0, "AT_s": t2 - t1, "cgls20_s": t4 - t3,
           "cgls20_nb_over_nb0": float(res.history[-1]), "cores": th}
    print(json.dumps({"mode": "pr1", "config": {"workload": "PR1: 64^3 nested phantom (1 mm), "
                                                 "128x96 detector (1 mm), 90 views, 1 % noise"},
                      "gpu": gpu, "oracle": orc,
                      "ratio": {"A": orc["A_s"] * 1e3 / ms_a, "AT": orc["AT_s"] * 1e3 / ms_at,
                                "cgls20": orc["cgls20_s"] / gpu["cgls20_s"]}}))
    return 0


def run_diff(a):
    """The differentiation workload: a batch of 8 volumes of 128^3 (192 x 144
    detector, 180 views) through the autograd operators.  CUDA events, median
    of 10 after warm-up: batched A and A^T (one persistent projector launch
    per batch), the loss ||A x - b||^2 with its gradient (one A and one A^T),
    and the checkpointed unrolled CGLS with 10 updates, forward and backward."""
    import numpy as np
    import torch

    import paper_2110_13526_gb300 as ct
    from paper_2110_13526_gb300.autograd import A, AT, unrolled_cgls
    import synth

    torch.cuda.set_device(0)
    cfg = synth.CONFIGS["DIFF"]
    g = ct.Geometry(**cfg)
    lo, hi = synth.box_of(cfg)
    xs = [synth.voxelize(synth.random_ellipsoids(20, 100 + i, lo, hi, axis_scale=0.5), cfg)
          for i in range(8)]
    x_true = torch.from_numpy(np.stack(xs)).cuda()
    gen = torch.Generator("cuda").manual_seed(4)
    with torch.no_grad():
        b = A(g, x_true) + 0.01 * torch.randn(8, *g.sino_shape, device="cuda", generator=gen)
    x = (x_true + 0.05 * torch.randn(x_true.shape, device="cuda",
                                     generator=torch.Generator("cuda").manual_seed(5)))
    stream = torch.cuda.current_stream()

    def ev(fn, n=10):
        for _ in range(max(a.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def grad_step():
        xg = x.clone().requires_grad_(True)
        ((A(g, xg) - b).double() ** 2).sum().backward()

    def cgls_step():
        bg = b.clone().requires_grad_(True)
        unrolled_cgls(g, bg, K=10).sum().backward()

    with torch.no_grad():
        ms_a = ev(lambda: A(g, x))
        ms_at = ev(lambda: AT(g, b))
    ms_grad = ev(grad_step)
    ms_cgls = ev(cgls_step, n=5)
    print(json.dumps({"mode": "diff",
                      "config": {"workload": "DIFF: 8 x 128^3 volumes (1 mm, 20-ellipsoid "
                                             "phantoms), 192x144 detector (1.6 mm), 180 views"},
                      "batch": 8, "A_ms": ms_a, "AT_ms": ms_at,
                      "A_ms_per_volume": ms_a / 8, "AT_ms_per_volume": ms_at / 8,
                      "loss_grad_ms": ms_grad, "unrolled_cgls10_fwd_bwd_ms": ms_cgls}))
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.mode == "ops":
        return run_ops(a)
    if a.mode == "serve":
        return run_serve(a)
    if a.mode == "precision":
        return run_precision(a)
    if a.mode == "pr1":
        return run_pr1(a)
    if a.mode == "diff":
        return run_diff(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
