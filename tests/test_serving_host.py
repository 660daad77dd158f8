"""Host logic of the serving benchmark client (no GPU): the ask/tell Nelder-Mead and
the request bookkeeping, against a fake server that answers at once."""
from __future__ import annotations

import threading

import numpy as np

import bench
from paper_1912_13132_gb300 import datagen


def test_nelder_mead_minimises_quadratic():
    target = np.array([0.3, -1.2, 2.0])
    A = np.diag([1.0, 4.0, 0.5])
    g = bench.nelder_mead(np.zeros(3), 0.5)
    x = next(g)
    best = np.inf
    for _ in range(600):
        f = float((x - target) @ A @ (x - target))
        best = min(best, f)
        x = g.send(f)
    assert best < 1e-8


def test_nelder_mead_survives_infinite_losses():
    g = bench.nelder_mead(np.zeros(2), 1.0)
    x = next(g)
    for i in range(50):
        f = np.inf if x[0] > 0.5 else float(x @ x)
        x = g.send(f)
    assert np.all(np.isfinite(x))


class FakeServer:
    """Answers every request immediately with a loss that depends on the parameters."""

    def __init__(self):
        self.lock = threading.Lock()
        self.reqs = {}
        self.next = 1

    def submit_cv(self, d, p):
        with self.lock:
            rid, self.next = self.next, self.next + 1
            self.reqs[rid] = dict(sspe=float(np.sum(np.log(p) ** 2)), status=0, latency_ms=1.0)
        return rid

    def submit_predict(self, d, p, pts):
        assert pts.shape[1] == 2 and 1000 <= len(pts) <= 100000
        with self.lock:
            rid, self.next = self.next, self.next + 1
            self.reqs[rid] = dict(yhat=np.zeros(len(pts)), status=0, latency_ms=2.0)
        return rid

    def wait(self, rid, timeout_s=0.0):
        with self.lock:
            return self.reqs.pop(rid)


def _workloads():
    ws = []
    for i in range(3):
        ws.append(datagen.Workload(f"w{i}", np.zeros((1, 2)), np.zeros(1), np.zeros(1, np.uint8), {},
                                   np.array([[1.0, 0.05, 0.02]])))
    return ws


def test_client_burst_and_open_loop():
    cl = bench.ServingClient(None, FakeServer(), _workloads(), n_runs=6, seed=1)
    cap = cl.burst(60)
    assert cap > 0 and cl.outstanding == 0
    assert sum(cl.counts.values()) == 60
    assert cl.counts["nm"] > 0 and cl.counts["predict"] > 0
    r = cl.open(300.0, 0.3, "load")
    assert r["cv_nelder_mead"] + r["cv_probe"] + r["predict"] > 0 and r["failed"] == 0
    assert r["p50_ms"] is not None and r["p99_ms"] >= r["p50_ms"]
    assert cl.outstanding == 0
    # every CV answer advanced its run; no run is left marked busy; best points improved
    assert not any(run["busy"] for run in cl.runs)
    assert all(np.isfinite(b[0]) for b in cl.best)
    cl.pool.shutdown()
