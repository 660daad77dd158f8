"""Serving loop (pcv_server_*): continuous batching over several device-resident
datasets, admission by device memory.

Each result must be the same alone and in the mix: every CV request and every
prediction request is first evaluated on its own through the plain context API,
then all are submitted together (interleaved across datasets, so they are batched
and their kernels overlap); the served results must equal the solo results
bit for bit (tasks are computed independently, sums have a fixed order).  A
second run gives the server a memory budget below the datasets' total, so workers
must release idle datasets' work memory (evictions) -- results must still match.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1912_13132_gb300 import datagen

pytestmark = pytest.mark.gpu


def _datasets():
    out = [datagen.make_uniform(1400, 600, 3, 0.06, seed=501, name="s0"),
           datagen.make_uniform(900, 500, 2, 0.08, seed=502, name="s1"),
           datagen.config_grid_1m(rho=0.05, tau2=0.02, fine=128, cells=16, buf=4, n_valid=1024, seed=503)]
    return out


def _requests(rng, nds):
    reqs = []
    for q in range(40):
        d = int(rng.integers(nds))
        p = (float(rng.uniform(0.5, 2.0)), float(np.exp(rng.uniform(np.log(0.02), np.log(0.2)))),
             float(np.exp(rng.uniform(np.log(0.005), np.log(0.2)))))
        if q % 5 == 4:
            reqs.append(("pred", d, p, rng.random((int(rng.integers(50, 400)), 2))))
        else:
            reqs.append(("cv", d, p, None))
    return reqs


def _solo(gpu_lib, ws, reqs):
    out = []
    ctxs = [gpu_lib.Context(w.xy, w.v, w.role, w.layout, max_slots=24) for w in ws]
    for kind, d, p, pts in reqs:
        if kind == "cv":
            out.append(ctxs[d].cv_loss([p], precision="mixed")["sspe"][0])
        else:
            out.append(ctxs[d].predict(p, pts, precision="mixed"))
    for c in ctxs:
        c.close()
    return out


def _served(gpu_lib, ws, reqs, budget):
    ctxs = [gpu_lib.Context(w.xy, w.v, w.role, w.layout, max_slots=24) for w in ws]
    with gpu_lib.Server(ctxs, max_batch=8, precision="mixed", hbm_budget_bytes=budget) as srv:
        ids = []
        for kind, d, p, pts in reqs:
            ids.append(srv.submit_cv(d, p) if kind == "cv" else srv.submit_predict(d, p, pts))
        res = [srv.wait(r, timeout_s=120.0) for r in ids]
        st = srv.stats()
    for c in ctxs:
        c.close()
    return res, st


@pytest.mark.parametrize("budget", ["unlimited", "tight"])
def test_alone_equals_mixed(gpu_lib, budget):
    ws = _datasets()
    reqs = _requests(np.random.default_rng(7), len(ws))
    solo = _solo(gpu_lib, ws, reqs)
    b = 0.0
    if budget == "tight":
        # the two small sets need about 65 MB of work memory each, the gridded one about
        # 0.18 GB: a 0.1 GB budget cannot hold two at once
        b = 1e8
    res, st = _served(gpu_lib, ws, reqs, b)
    for (kind, _, _, _), want, got in zip(reqs, solo, res):
        assert got["status"] in (0, 7)
        if kind == "cv":
            assert got["sspe"] == want
        else:
            assert np.array_equal(got["yhat"], want)
    assert st["completed"] == len(reqs)
    assert st["batches"] < len(reqs)          # CV requests were batched
    assert st["p99_ms"] >= st["p50_ms"] > 0
    if budget == "tight":
        assert st["evictions"] > 0
