"""The continuous-batching server's host logic on the CPU (paper_2110_13526_gb300/serving.py).

The library calls are replaced by fakes: a geometry object, solvers that hold
their slot for a time set by the request and return a report, and no-op
stand-ins for the CUDA stream calls.  What is tested is the scheduling
itself: requests are admitted in arrival order while a slot and the HBM
budget allow, never more than `slots` at once, a request larger than the
budget is refused before the run, cancelled requests leave the queue
without running and stay out of the percentiles, a failing solve is reported
after the run, and latencies run from arrival to completion.
"""
import contextlib
import threading
import time
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import paper_2110_13526_gb300.serving as serving


class _Stream:
    def __init__(self, *a, **k):
        pass

    def synchronize(self):
        pass


class _Geometry:
    def __init__(self, **cfg):
        self.cfg = cfg


class _Solvers:
    """cgls / lsqr fakes: each call holds its slot for the request's
    `hold` seconds (carried in b) and records when it ran."""

    def __init__(self, fail_rid=None):
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.calls = []            # (rid, start, end) in seconds of perf_counter
        self.fail_rid = fail_rid

    def _run(self, g, b, max_iter, err_tol):
        rid, hold = b
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
        t0 = time.perf_counter()
        try:
            if rid == self.fail_rid:
                raise RuntimeError("CT_ERR_CUDA: injected")
            time.sleep(hold)
        finally:
            with self.lock:
                self.running -= 1
                self.calls.append((rid, t0, time.perf_counter()))
        rep = SimpleNamespace(iterations=max_iter, nb=err_tol * 0.5, nb0=1.0)
        return ("x", rid), rep

    def cgls(self, g, b, max_iter=50, err_tol=1e-3, stream=None, storage="f32"):
        return self._run(g, b, max_iter, err_tol)

    def lsqr(self, g, b, max_iter=50, err_tol=1e-3, stream=None):
        return self._run(g, b, max_iter, err_tol)


@pytest.fixture
def fake(monkeypatch):
    solvers = _Solvers()
    monkeypatch.setattr(serving, "Geometry", _Geometry)
    monkeypatch.setattr(serving, "cgls", solvers.cgls)
    monkeypatch.setattr(serving, "lsqr", solvers.lsqr)
    monkeypatch.setattr(torch.cuda, "Stream", _Stream)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "device", lambda d: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    return solvers


def _geom(n, views=60):
    return serving.serving_geometry(n, views)


def _req(rid, arrival, hold, n=64, solver="cgls", **kw):
    return serving.Request(rid=rid, geometry=_geom(n), b=(rid, hold), solver=solver,
                           arrival=arrival, **kw)


def test_fifo_admission_and_slot_limit(fake):
    # 12 requests in a burst of 0.06 s, each holding its slot 0.05 s: at most
    # 3 run at once, and they start in arrival order
    reqs = [_req(k, 0.005 * k, 0.05, solver="lsqr" if k % 3 == 2 else "cgls")
            for k in range(12)]
    stats = serving.Server(slots=3).run(reqs[::-1])          # order of the list is irrelevant
    assert [r.rid for r in stats.results] == list(range(12))
    assert fake.max_running <= 3 and stats.max_concurrent == 3
    # admission (the recorded start) follows arrival order
    starts = [r.start for r in stats.results]
    assert starts == sorted(starts)
    for r in stats.results:
        assert not r.cancelled and r.x == ("x", r.rid)
        assert r.start >= r.arrival - 1e-6 and r.end >= r.start + 0.05 - 1e-3
        assert r.rel_discrepancy == pytest.approx(0.5e-3)
    lat = np.array([r.latency for r in stats.results])
    assert stats.p50 == pytest.approx(np.percentile(lat, 50))
    assert stats.p99 == pytest.approx(np.percentile(lat, 99))
    # 12 requests of 0.05 s on 3 slots queue behind each other (the last
    # ones wait for three waves: about 0.155 s from arrival to completion)
    assert lat.max() >= 0.14
    assert stats.iterations == 12 * 50


def test_hbm_budget_limits_concurrency_and_refuses_oversize(fake):
    big = serving.footprint_bytes(_geom(128), "cgls")
    reqs = [_req(k, 0.0, 0.03, n=128) for k in range(6)]
    stats = serving.Server(slots=8, hbm_budget_bytes=2.5 * big).run(reqs)
    assert stats.max_concurrent == 2 and fake.max_running == 2
    assert stats.max_bytes_in_use <= 2.5 * big
    with pytest.raises(ValueError, match="needs"):
        serving.Server(slots=8, hbm_budget_bytes=0.5 * big).run([_req(0, 0.0, 0.01, n=128)])


def test_cancelled_requests_leave_the_queue(fake):
    # one slot held 0.2 s by request 0; request 1 is cancelled by its client
    # 0.05 s after arrival, request 2 by the server before the run: neither
    # runs, both come back cancelled, and only the others count in the
    # percentiles
    reqs = [_req(0, 0.0, 0.2), _req(1, 0.01, 0.05, cancel_after=0.05), _req(2, 0.02, 0.05),
            _req(3, 0.03, 0.01)]
    srv = serving.Server(slots=1)
    srv.cancel(2)
    stats = srv.run(reqs)
    by = {r.rid: r for r in stats.results}
    assert by[1].cancelled and by[1].x is None and by[1].iterations == 0
    assert by[2].cancelled and by[2].x is None
    assert by[1].end < 0.2             # it left the queue while request 0 still ran
    assert sorted(c[0] for c in fake.calls) == [0, 3]
    assert stats.extra["cancelled"] == 2
    lat = np.array([by[0].latency, by[3].latency])
    assert stats.p99 == pytest.approx(np.percentile(lat, 99))
    # the cancellation set is cleared after the run: the same rid runs next time
    stats2 = srv.run([_req(2, 0.0, 0.01)])
    assert not stats2.results[0].cancelled


def test_failed_solve_is_reported_after_the_run(fake):
    fake.fail_rid = 1
    with pytest.raises(RuntimeError, match=r"requests failed.*\(1, "):
        serving.Server(slots=2).run([_req(k, 0.0, 0.01) for k in range(4)])
    # every other request still ran
    assert sorted(c[0] for c in fake.calls) == [0, 1, 2, 3]


def test_server_argument_checks(fake):
    with pytest.raises(ValueError):
        serving.Server(slots=0)
    with pytest.raises(ValueError):
        serving.Server(cancel_chunk=-1)
    with pytest.raises(ValueError):
        serving.Server(batch_route="random")


def test_footprint_bytes_counts_the_solver_state():
    g = _geom(64)
    n, m = 64 ** 3, g["nviews"] * g["nu"] * g["nv"]
    cg, ls = serving.footprint_bytes(g, "cgls"), serving.footprint_bytes(g, "lsqr")
    # CGLS holds 4 volumes and 2 sinograms, LSQR 5 volumes and 1 sinogram
    assert cg - ls == 4 * (m - n)
    assert cg > 4 * (4 * n + 2 * m)
    # a deterministic Siddon geometry adds 16 bytes per voxel; a footprint one 8 per ray
    assert serving.footprint_bytes(g, "cgls", True) - cg == 16 * n
    gf = dict(g, projector="sf_tt")
    assert serving.footprint_bytes(gf, "cgls", True) - cg >= 8 * m
