"""Continuous-batching reconstruction server over the C ABI.

Requests (a sinogram, its scan geometry, CGLS or LSQR, a discrepancy
tolerance and an iteration cap) arrive over time.  The server admits a
request as soon as a slot is free and its device footprint fits the HBM
budget, and runs it on its own CUDA stream from a worker thread; the ctypes
calls release the GIL, so the jobs of all occupied slots overlap on the GPU.
Requests that arrive while others run wait in FIFO order and are admitted as
slots and memory free up (no head-of-line skipping, so service order is
arrival order).  Every solve is the unchanged library call (ct_cgls /
ct_lsqr): a result does not depend on which other jobs share the GPU, up to
the float-atomic summation order of the backprojection.

With ``batched=True`` the FP32 CGLS requests instead join a ct_batch
(iteration-level continuous batching; ``batch_executors`` batches on their
own streams, each request to the least loaded one, or with
``batch_route="size"`` to the batch of its volume size): a batch thread advances its
admitted CGLS jobs one update per step, with the backprojections of all of them in one
persistent kernel launch and their projections in another, inside a CUDA
graph; jobs join between steps as they are admitted and leave when their
stopping rule fires.  LSQR and reduced-storage requests keep the per-slot
streams.  A batched job's result is that of ct_cgls alone (bitwise with a
deterministic geometry).

Cancellation: ``Server.cancel(rid)`` (from any thread while ``run`` runs),
or ``Request.cancel_after`` seconds after arrival (a client that gives up).
A queued request leaves the queue without running; a batched CGLS job
leaves its batch at the next step boundary with the iterate it has; a
per-slot CGLS solve with ``cancel_chunk = k > 0`` runs as a resumable state
in chunks of k updates (ct_cgls_resume, bitwise the uninterrupted solve
with a deterministic geometry) and stops at the next chunk boundary (the
state's device buffers are allocated and freed per solve, and freeing waits
for the device, so the option costs every other slot a short stall); any
other running solve runs to its end and is marked cancelled.  Each
cancelled request yields a Result with ``cancelled`` set (x the iterate it
reached, or None if it never ran); latency percentiles cover the requests
that were not cancelled.

Latency of a request = completion time - arrival time.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np
import torch

from . import Batch, CglsState, Geometry, cgls, lsqr


@dataclass
class Request:
    rid: int
    geometry: dict                 # keyword arguments of Geometry
    b: torch.Tensor                # sinogram on the device
    solver: str = "cgls"           # "cgls" or "lsqr"
    arrival: float = 0.0           # seconds after the start of the run
    max_iter: int = 50
    err_tol: float = 1e-3
    storage: str = "f32"           # CGLS Krylov-vector storage ("f32", "bf16", "f16")
    cancel_after: Optional[float] = None   # the client cancels this long after arrival


@dataclass
class Result:
    rid: int
    x: Optional[torch.Tensor]
    iterations: int
    rel_discrepancy: float
    arrival: float
    start: float
    end: float
    cancelled: bool = False

    @property
    def latency(self) -> float:
        return self.end - self.arrival


def _vox(geometry: dict) -> int:
    return geometry["nx"] * geometry["ny"] * geometry["nz"]


def footprint_bytes(geometry: dict, solver: str, deterministic: bool = False) -> int:
    """Device bytes a solve holds: the library's workspace plus x.

    CGLS: x, z, g, transposed scratch (4 volumes) + e, p (2 sinograms);
    LSQR: x, v, w, g, transposed scratch (5 volumes) + u (1 sinogram);
    plus per-view and per-column constants and FP64 partial sums.  A
    deterministic geometry adds its int64 sums: 16 bytes per voxel (Siddon
    backprojection) or 8 bytes per ray (footprint forward projection)."""
    n = geometry["nx"] * geometry["ny"] * geometry["nz"]
    m = geometry["nviews"] * geometry["nu"] * geometry["nv"]
    vols, sinos = (4, 2) if solver == "cgls" else (5, 1)   # FP32 storage (an upper bound)
    cols = geometry["nviews"] * geometry["nu"] * 36 + geometry["nviews"] * 48
    partials = 8 * (m // 256 + n // 1024 + 4096)
    det = 0
    if deterministic:
        det = 16 * n if geometry.get("projector", "siddon") == "siddon" else 8 * m + 4 * (n + m) // 256
    return 4 * (vols * n + sinos * m) + cols + partials + det


@dataclass
class ServeStats:
    results: List[Result]
    wall_s: float
    max_concurrent: int
    max_bytes_in_use: int
    iterations: int = 0
    p50: float = 0.0
    p99: float = 0.0
    extra: dict = field(default_factory=dict)


class Server:
    def __init__(self, slots: int = 8, hbm_budget_bytes: float = 150e9, device=None,
                 deterministic: bool = False, batched: bool = False, batch_jobs: int = 32,
                 batch_executors: int = 1, batch_route: str = "load", cancel_chunk: int = 0):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        if cancel_chunk < 0:
            raise ValueError("cancel_chunk must be >= 0")
        self.cancel_chunk = cancel_chunk
        self._cancelled: set = set()
        self._cv: Optional[threading.Condition] = None
        if batch_jobs < 1 or batch_executors < 1:
            raise ValueError("batch_jobs and batch_executors must be >= 1")
        if batch_route not in ("load", "size"):
            raise ValueError("batch_route must be 'load' or 'size'")
        self.batch_route = batch_route
        self.slots = slots
        self.batched = batched
        self.batch_jobs = batch_jobs
        self.batch_executors = batch_executors
        self.deterministic = deterministic
        self.budget = int(hbm_budget_bytes)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self._geoms: Dict[Tuple, Geometry] = {}
        self._lock = threading.Lock()

    def geometry(self, cfg: dict) -> Geometry:
        key = tuple(sorted(cfg.items()))
        with self._lock:
            g = self._geoms.get(key)
            if g is None:
                with torch.cuda.device(self.device):
                    g = Geometry(**cfg, deterministic=self.deterministic)
                self._geoms[key] = g
            return g

    def cancel(self, rid: int) -> None:
        """Cancel request rid (queued or running) of the current or next run."""
        cv = self._cv
        if cv is None:
            self._cancelled.add(rid)
            return
        with cv:
            self._cancelled.add(rid)
            cv.notify_all()

    def run(self, requests: List[Request]) -> ServeStats:
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in reqs:
            fp = footprint_bytes(r.geometry, r.solver, self.deterministic)
            if fp > self.budget:
                raise ValueError("request %d needs %d bytes, budget %d" % (r.rid, fp, self.budget))
            self.geometry(r.geometry)          # geometries are built before the clock starts
        torch.cuda.synchronize(self.device)
        # size classes of the batched CGLS requests (batch_route "size"): the
        # jobs of one batch advance in lock step, so each batch takes volumes
        # of one size and no small job waits for a large one's updates
        size_class = {v: c for c, v in enumerate(sorted({_vox(r.geometry) for r in reqs}))}
        cv = threading.Condition()
        self._cv = cv
        cancelled = self._cancelled
        timers = sorted((r.arrival + r.cancel_after, r.rid) for r in reqs
                        if r.cancel_after is not None)
        state = {"free_slots": self.slots, "bytes": 0, "running": 0, "max_running": 0,
                 "max_bytes": 0, "errors": [], "batch_active": 0, "batch_stop": False,
                 "batch_steps": 0}
        # per batch executor: admitted jobs not yet in its batch, and its load
        n_ex = self.batch_executors if self.batched else 0
        inboxes: List[List[Tuple[Request, int, float]]] = [[] for _ in range(n_ex)]
        load = [0] * n_ex
        results: List[Result] = []
        streams = [torch.cuda.Stream(device=self.device) for _ in range(self.slots)]
        free_streams = list(range(self.slots))
        t0 = time.perf_counter()

        def worker(req: Request, si: int, fp: int, t_start: float):
            try:
                torch.cuda.set_device(self.device)
                s = streams[si]
                g = self.geometry(req.geometry)
                with torch.cuda.stream(s):
                    if (req.solver == "cgls" and req.storage == "f32"
                            and self.cancel_chunk > 0):
                        # a resumable state, advanced chunk by chunk
                        cs = CglsState(g)
                        try:
                            total = 0
                            while True:
                                total = min(total + self.cancel_chunk, req.max_iter)
                                x, rep = cs.run(req.b, total, err_tol=req.err_tol, stream=s)
                                if rep.iterations < total or total >= req.max_iter:
                                    break
                                with cv:
                                    if req.rid in cancelled:
                                        break
                        finally:
                            cs.close()
                    elif req.solver == "cgls":
                        x, rep = cgls(g, req.b, max_iter=req.max_iter, err_tol=req.err_tol,
                                      stream=s, storage=req.storage)
                    else:
                        x, rep = lsqr(g, req.b, max_iter=req.max_iter, err_tol=req.err_tol,
                                      stream=s)
                    s.synchronize()
                t_end = time.perf_counter() - t0
                with cv:
                    was = req.rid in cancelled
                res = Result(req.rid, x, rep.iterations, rep.nb / rep.nb0 if rep.nb0 else 0.0,
                             req.arrival, t_start, t_end, cancelled=was)
            except Exception as e:  # reported after the run
                res = None
                with cv:
                    state["errors"].append((req.rid, repr(e)))
            with cv:
                if res is not None:
                    results.append(res)
                state["free_slots"] += 1
                state["bytes"] -= fp
                state["running"] -= 1
                free_streams.append(si)
                cv.notify_all()

        def batch_worker(k: int):
            """Executor k: one ct_batch on its own stream, so that the vector
            kernels of one batch's step overlap the projector launches of
            another's."""
            inbox = inboxes[k]
            live = {}                                     # job id -> (request, bytes, start)
            done_upd = {}                                 # job id -> x updates so far
            new: List[Tuple[Request, int, float]] = []    # taken from the inbox, not yet added

            def leave(req, fp, res):
                with cv:
                    results.append(res)
                    state["bytes"] -= fp
                    state["batch_active"] -= 1
                    load[k] -= 1
                    state["running"] -= 1
                    cv.notify_all()

            try:
                torch.cuda.set_device(self.device)
                s = torch.cuda.Stream(device=self.device)
                with torch.cuda.stream(s):
                    bt = Batch(stream=s)
                    while True:
                        with cv:
                            while not inbox and not live and not state["batch_stop"]:
                                cv.wait()
                            if state["batch_stop"] and not inbox and not live:
                                break
                            new.extend(inbox)
                            inbox.clear()
                        with cv:
                            gone = {r.rid for r, _, _ in new if r.rid in cancelled}
                            gone |= {live[j][0].rid for j in live if live[j][0].rid in cancelled}
                        while new:
                            req, fp, t_start = new.pop(0)
                            if req.rid in gone:               # cancelled before it ran
                                now = time.perf_counter() - t0
                                leave(req, fp, Result(req.rid, None, 0, float("nan"),
                                                      req.arrival, now, now, cancelled=True))
                                continue
                            jid = bt.add(self.geometry(req.geometry), req.b,
                                         max_iter=req.max_iter, err_tol=req.err_tol)
                            live[jid] = (req, fp, t_start)
                            done_upd[jid] = 1                 # the first update runs in add
                        for j in [j for j in live if live[j][0].rid in gone]:
                            x = bt.cancel(j)                  # leaves between steps
                            req, fp, t_start = live.pop(j)
                            leave(req, fp, Result(req.rid, x, done_upd.pop(j), float("nan"),
                                                  req.arrival, t_start,
                                                  time.perf_counter() - t0, cancelled=True))
                        active = [j for j in live if not bt.done(j)]
                        if active:
                            bt.step()
                            for j in active:
                                done_upd[j] += 1
                            with cv:
                                state["batch_steps"] += 1
                        for j in [j for j in live if bt.done(j)]:
                            x, rep = bt.result(j)
                            req, fp, t_start = live.pop(j)
                            done_upd.pop(j, None)
                            with cv:
                                was = req.rid in cancelled
                            leave(req, fp, Result(req.rid, x, rep.iterations,
                                                  rep.nb / rep.nb0 if rep.nb0 else 0.0,
                                                  req.arrival, t_start,
                                                  time.perf_counter() - t0, cancelled=was))
                    bt.close()
            except Exception as e:  # reported after the run
                with cv:
                    state["errors"].append(("batch", repr(e)))
                    for req, fp, _ in list(live.values()) + new + inbox:
                        state["bytes"] -= fp
                        state["batch_active"] -= 1
                        load[k] -= 1
                        state["running"] -= 1
                    inbox.clear()
                    state["batch_dead"] = True
                    cv.notify_all()

        threads = []
        bthreads = [threading.Thread(target=batch_worker, args=(k,), daemon=True)
                    for k in range(n_ex)]
        for t in bthreads:
            t.start()
        pending: List[Request] = []
        i = 0
        with cv:
            while i < len(reqs) or pending or state["running"] > 0:
                now = time.perf_counter() - t0
                while i < len(reqs) and reqs[i].arrival <= now:
                    pending.append(reqs[i])
                    i += 1
                # clients that give up; queued requests cancelled leave the queue
                while timers and timers[0][0] <= now:
                    cancelled.add(timers.pop(0)[1])
                    cv.notify_all()
                for r in [r for r in pending if r.rid in cancelled]:
                    pending.remove(r)
                    results.append(Result(r.rid, None, 0, float("nan"), r.arrival, now, now,
                                          cancelled=True))
                # admit in arrival order while a slot (or the batch) and the budget allow
                while pending:
                    fp = footprint_bytes(pending[0].geometry, pending[0].solver,
                                         self.deterministic)
                    if state["bytes"] + fp > self.budget:
                        break
                    if (self.batched and pending[0].solver == "cgls"
                            and pending[0].storage == "f32"):
                        if state["batch_active"] >= self.batch_jobs or state.get("batch_dead"):
                            break
                        req = pending.pop(0)
                        if self.batch_route == "size":
                            k = size_class[_vox(req.geometry)] % n_ex   # one class per batch
                        else:
                            k = min(range(n_ex), key=lambda j: load[j])   # least loaded
                        load[k] += 1
                        state["batch_active"] += 1
                        state["bytes"] += fp
                        state["running"] += 1
                        state["max_running"] = max(state["max_running"], state["running"])
                        state["max_bytes"] = max(state["max_bytes"], state["bytes"])
                        inboxes[k].append((req, fp, now))
                        cv.notify_all()
                        continue
                    if state["free_slots"] <= 0:
                        break
                    req = pending.pop(0)
                    si = free_streams.pop(0)
                    state["free_slots"] -= 1
                    state["bytes"] += fp
                    state["running"] += 1
                    state["max_running"] = max(state["max_running"], state["running"])
                    state["max_bytes"] = max(state["max_bytes"], state["bytes"])
                    t = threading.Thread(target=worker, args=(req, si, fp, now), daemon=True)
                    threads.append(t)
                    t.start()
                if i >= len(reqs) and not pending and state["running"] == 0:
                    break
                if state.get("batch_dead") and pending:
                    break
                wait = None
                if i < len(reqs):
                    wait = reqs[i].arrival
                if timers:
                    wait = timers[0][0] if wait is None else min(wait, timers[0][0])
                if wait is not None:
                    wait = max(0.0, wait - (time.perf_counter() - t0))
                cv.wait(timeout=wait if wait is not None else 0.5)
        for t in threads:
            t.join()
        with cv:
            state["batch_stop"] = True
            cv.notify_all()
        for t in bthreads:
            t.join()
        self._cv = None
        self._cancelled = set()
        wall = time.perf_counter() - t0
        if state["errors"]:
            raise RuntimeError("requests failed: %s" % state["errors"])
        results.sort(key=lambda r: r.rid)
        lat = np.array([r.latency for r in results if not r.cancelled])
        return ServeStats(results, wall, state["max_running"], state["max_bytes"],
                          iterations=sum(r.iterations for r in results),
                          p50=float(np.percentile(lat, 50)) if len(lat) else 0.0,
                          p99=float(np.percentile(lat, 99)) if len(lat) else 0.0,
                          extra={"batch_steps": state["batch_steps"],
                                 "cancelled": sum(r.cancelled for r in results)})


def serving_geometry(n: int, views: int) -> dict:
    """Scan of an n^3 volume of 1 mm voxels with a detector scaled to the
    magnification 1200/750 = 1.6: 1.6 mm pixels, 1.5 n x 1.125 n of them."""
    return dict(nx=n, ny=n, nz=n, vx=1.0, vy=1.0, vz=1.0, nu=int(1.5 * n), nv=int(1.125 * n),
                du=1.6, dv=1.6, sid=750.0, sdd=1200.0, nviews=views)
