"""Serving loop (pcv_server_*): continuous batching over several device-resident
datasets, admission by device memory.

Each result must be the same alone and in the mix: every CV request and every
prediction request is first evaluated on its own through the plain context API,
then all are submitted together (interleaved across datasets, so they are batched,
run on either of a dataset's two lanes and overlap on the device); served CV losses
must equal the solo losses bit for bit (tasks are computed independently, the lanes
are identical, sums have a fixed order), served predictions the solo ones within the
mixed tolerance (either may come from kriging weights a CV evaluation kept).  A
second run gives the server a memory budget below the datasets' total, so workers
must release idle lanes' work memory (evictions) -- results must still match.  A
request that arrives while a long batch of its dataset runs is admitted at once on
the other lane and finishes first.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_1912_13132_gb300 import datagen
from parity_util import TOL, pred_err

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
            assert pred_err(got["yhat"], want) <= TOL["mixed"]["pred"]
    assert st["completed"] == len(reqs)
    assert st["batches"] < len(reqs)          # CV requests were batched
    assert st["p99_ms"] >= st["p50_ms"] > 0
    if budget == "tight":
        assert st["evictions"] > 0


@pytest.mark.parametrize("lanes,warm", [(2, True), (2, False), (1, True)])
def test_arrival_during_a_running_batch(gpu_lib, lanes, warm):
    """A CV request that arrives while a long batch of the same dataset runs: with two
    lanes it is admitted at once and completes before the batch (its launch takes the
    SMs the running launch leaves free); with one lane it waits for the batch.  Its
    loss equals the solo evaluation bit for bit either way.  Cold (warm=False): no
    request has run on the server before, so the late request is its lane's first call,
    which must find its work memory reserved at server creation (an allocation then
    would wait for the running launch)."""
    w = datagen.config_grid_1m(rho=0.05, tau2=0.02, fine=512, cells=32, buf=8, n_valid=8192, seed=505)
    big = [(1.0, 0.05 * (1.0 + 0.02 * q), 0.02) for q in range(16)]
    late = (1.2, 0.07, 0.03)
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, max_slots=24) as ctx:
        ctx.cv_loss(big[:1])                       # work memory and tuning outside the timing
        want = ctx.cv_loss([late])["sspe"][0]
    ctx = gpu_lib.Context(w.xy, w.v, w.role, w.layout, max_slots=24)
    ctx.cv_loss(big[:1])
    with gpu_lib.Server([ctx], max_batch=16, precision="mixed", lanes=lanes) as srv:
        # warm: every lane runs once first (the second request is queued while the first
        # lane is busy, so the other lane takes it)
        if warm:
            first = srv.submit_cv(0, big[0])
            time.sleep(0.005)
            second = srv.submit_cv(0, big[1])
            srv.wait(first)
            srv.wait(second)
        t0 = time.perf_counter()
        ids = [srv.submit_cv(0, p) for p in big]
        time.sleep(0.05)
        t_late = time.perf_counter()
        lid = srv.submit_cv(0, late)
        res = [srv.wait(i, timeout_s=120.0) for i in ids]
        lres = srv.wait(lid, timeout_s=120.0)
    ctx.close()
    batch_done = max(t0 + r["latency_ms"] / 1e3 for r in res)
    late_done = t_late + lres["latency_ms"] / 1e3
    assert lres["status"] == 0 and lres["sspe"] == want
    if lanes > 1:
        assert late_done < batch_done, (late_done - t0, batch_done - t0)
    else:
        assert late_done >= batch_done - 0.01, (late_done - t0, batch_done - t0)
    print("lanes", lanes, "warm", warm, "late request done at", late_done - t0, "batch done at", batch_done - t0)
