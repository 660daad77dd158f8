"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Every test compares element by element on the same seeded inputs: local SSPE of
each subset, the total (Eq. 6) and every validation prediction (Eq. 3).
Tolerances (tests/parity_util.py): FP64 path 1e-10 relative; mixed path 1e-6 on
losses and 1e-5 on predictions.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1912_13132_gb300 import datagen
from parity_util import TOL, compare, pred_err, rel

pytestmark = pytest.mark.gpu
PRECS = ["fp64", "mixed"]


def _run(gpu_lib, w, params, prec, subsets=None, **ctx_opts):
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, **ctx_opts) as ctx:
        out = ctx.cv_loss(params, precision=prec, per_subset=True, predictions=True)
        V_off = ctx.V_off.copy()
    members = oracle.all_members(w.xy, w.role, w.layout)
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, params, members=members, subsets=subsets)
    return out, ref, V_off


@pytest.mark.parametrize("prec", PRECS)
def test_uniform_4096_full(gpu_lib, prec):
    """4096 TRAIN + 4096 VALID uniform points, 4x4 cores, shell 0.05: every subset,
    every prediction (k about 370-500, several 64/128-row tiles and a ragged tail)."""
    w = datagen.config_uniform_4096()
    P = np.array([[1.0, 0.1, 0.05], [0.7, 0.03, 0.2], [2.0, 0.3, 0.001]])
    out, ref, V_off = _run(gpu_lib, w, P, prec)
    assert np.all(out["status"] == 0), out["status"]
    assert out["n_valid"] == ref["n_valid"]
    worst = compare(out, ref, V_off, range(16), len(P), prec)
    print(prec, worst)


@pytest.mark.parametrize("prec", PRECS)
def test_ragged_and_degenerate(gpu_lib, prec):
    """Subset sizes from 0 to a few hundred, not multiples of any tile: a core with
    validation data but no training data (yhat = 0), cores without validation data
    (skipped, z = 0), a single-point subset."""
    r = np.random.default_rng(17)
    nT, nV = 900, 400
    xy = r.random((nT + nV, 2))
    xy[:nT, 0] *= 0.7                      # no training data right of x = 0.7 + shell
    role = np.zeros(nT + nV, dtype=np.uint8)
    role[nT:] = 1
    xy[nT:nT + 150, 1] *= 0.5              # validation mostly in the lower half
    role[nT + 150:nT + 300] = 2           # some IGNORE points
    v = r.standard_normal(nT + nV)
    xy[0] = [0.95, 0.95]                   # lone training point in the top-right core
    lay = dict(kind="grid", nx=5, ny=3, delta=0.013, domain=(0.0, 1.0, 0.0, 1.0))
    w = datagen.Workload("ragged", xy, v, role, lay, None)
    P = np.array([[1.0, 0.08, 0.05], [1.3, 0.2, 0.3]])
    out, ref, V_off = _run(gpu_lib, w, P, prec)
    sizes = [len(T) for T, _ in ref["members"]]
    assert 0 in sizes and 1 in sizes, sizes
    assert np.all(out["status"] == 0)
    compare(out, ref, V_off, range(len(sizes)), len(P), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_bad_parameters(gpu_lib, prec):
    w = datagen.make_uniform(400, 200, 2, 0.05, seed=5, name="bad")
    P = np.array([[1.0, 0.1, 0.05], [-1.0, 0.1, 0.05], [1.0, 0.0, 0.05], [1.0, 0.1, -0.1],
                  [np.nan, 0.1, 0.1], [1.0, 0.1, 0.0]])
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        out = ctx.cv_loss(P, precision=prec)
    st = out["status"].tolist()
    assert st[:5] == [0, 1, 1, 1, 1], st
    assert np.isnan(out["sspe"][1:5]).all() and np.isfinite(out["sspe"][0])
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P[[0, 5]])
    assert rel(out["sspe"][0], ref["sspe"][0]) <= TOL[prec]["loss"]
    # a zero nugget is a valid configuration (tau2 >= 0): it must evaluate, exactly or
    # through the mixed path's FP64 fallback, and meet the precision's own bar
    assert st[5] in ((0,) if prec == "fp64" else (0, gpu_lib.PCV_REFINE_FALLBACK)), st
    assert rel(out["sspe"][5], ref["sspe"][1]) <= TOL[prec]["loss"], (out["sspe"][5], ref["sspe"][1])


@pytest.fixture(scope="module")
def cluster():
    """Poisson-cluster workload (65,536 TRAIN, 16 x 16 cores), 8 configurations, and the
    oracle on every subset with validation data (LAPACK-backed kriging)."""
    w = datagen.config_cluster_262k(n_train=65536, n_valid=8192, fine=512, nx=16, delta=0.02)
    P = w.params[::8]
    members = oracle.all_members(w.xy, w.role, w.layout)
    act = [i for i, (_, V) in enumerate(members) if len(V) > 0]
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P, members=members, subsets=act, lapack=True)
    return w, P, act, ref


@pytest.mark.parametrize("prec", PRECS)
def test_cluster_batch_all(gpu_lib, cluster, prec):
    """Poisson-cluster locations (uneven subsets, k from a handful to ~1600, many
    degenerate), a batch of 8 configurations in one launch, every subset with
    validation data against the oracle.  The SSPE amplifies prediction errors by about
    |yhat| / |yhat - y|, so this covers the refinement's stopping rule where its margin
    is thinnest (a sample of 8 subsets passed at a tolerance whose worst subset did not)."""
    w, P, act, ref = cluster
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        out = ctx.cv_loss(P, precision=prec, per_subset=True, predictions=True)
        V_off = ctx.V_off.copy()
    assert np.all(out["status"] == 0)
    worst = compare(out, ref, V_off, act, len(P), prec, check_total=False)
    print(prec, "cluster", len(act), "subsets", worst)


@pytest.mark.parametrize("prec", PRECS)
def test_predict_new_locations(gpu_lib, prec):
    w = datagen.make_uniform(1200, 300, 3, 0.06, seed=23, name="pred")
    pts = np.random.default_rng(1).random((700, 2)) * 1.2 - 0.1   # some outside D
    p = (1.5, 0.12, 0.04)
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        yh = ctx.predict(p, pts, precision=prec)
    ref = oracle.predict(w.xy, w.v, w.role, w.layout, p, pts)
    assert pred_err(yh, ref) <= TOL[prec]["pred"]


@pytest.mark.parametrize("prec", PRECS)
def test_deterministic(gpu_lib, prec):
    w = datagen.make_uniform(800, 400, 3, 0.05, seed=31, name="det")
    P = np.array([[1.0, 0.1, 0.05], [1.0, 0.05, 0.01]])
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, max_slots=7) as ctx:
        a = ctx.cv_loss(P, precision=prec)["sspe"]
        b = ctx.cv_loss(P, precision=prec)["sspe"]
    assert np.array_equal(a, b)


def test_forced_fp64_fallback(gpu_lib):
    """The mixed path's FP64 fallback, forced for every task: one correction allowed
    and a tolerance no refinement meets, so each task lands on the device-side list and
    is recomputed by the FP64 kernel in the same stream.  Every configuration reports
    PCV_REFINE_FALLBACK (a warning: the results stand) and matches the oracle at the
    FP64 bar; the same data at the default options need no fallback."""
    w = datagen.make_uniform(800, 400, 3, 0.05, seed=41, name="fallback")
    P = np.array([[1.0, 0.1, 0.05], [1.0, 0.05, 0.01], [0.5, 0.2, 0.002]])
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, refine_max_iter=1, refine_tol=1e-300,
                         refine_loss_tol=-1.0) as ctx:
        out = ctx.cv_loss(P, precision="mixed", per_subset=True, predictions=True)
        V_off = ctx.V_off.copy()
    assert np.all(out["status"] == gpu_lib.PCV_REFINE_FALLBACK), out["status"]
    members = oracle.all_members(w.xy, w.role, w.layout)
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P, members=members)
    worst = compare(out, ref, V_off, range(len(members)), len(P), "fp64")
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        out2 = ctx.cv_loss(P, precision="mixed")
    assert np.all(out2["status"] == 0)
    print("forced fallback", worst)


def test_sigma2_invariance_gpu(gpu_lib):
    """Only lambda = tau2 / sigma2 and rho matter (remark after Eq. 3)."""
    w = datagen.make_uniform(800, 400, 2, 0.05, seed=37, name="inv")
    P = np.array([[1.0, 0.1, 0.05], [3.0, 0.1, 0.15], [0.25, 0.1, 0.0125]])
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        s = ctx.cv_loss(P, precision="fp64")["sspe"]
    assert np.all(rel(s, s[0]) <= 1e-12)


@pytest.fixture(scope="module")
def paper5m():
    return datagen.config_paper_5m()


@pytest.mark.parametrize("prec,B", [("mixed", 8), ("fp64", 1)])
def test_paper_scale_sampled(gpu_lib, paper5m, prec, B):
    """The benchmark's own workload and launch configuration (4,999,696-node grid,
    10% missing, 80/10/10 split, 40 x 40 cores, shell 0.001, batch of B
    configurations): every configuration's total is checked for status and
    finiteness; per-subset losses and predictions are compared with the oracle on
    sampled subsets (a corner, an edge, the largest, random interior ones)."""
    w = paper5m
    P = w.params[np.arange(B) * 23 % len(w.params)]
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        out = ctx.cv_loss(P, precision=prec, per_subset=True, predictions=True)
        T_off, V_off = ctx.T_off.copy(), ctx.V_off.copy()
    assert np.all(out["status"] == 0), out["status"]
    assert np.all(np.isfinite(out["sspe"]))
    k = np.diff(T_off)
    nx = w.layout["nx"]
    pick = sorted(set([0, nx - 1, nx * nx - 1, nx // 2, int(np.argmax(k))] +
                      np.random.default_rng(5).choice(nx * nx, 3, replace=False).tolist()))
    cores = oracle.layout_cores(w.layout, w.xy)
    members = {i: oracle.subset_members(w.xy, w.role, w.layout, i, cores) for i in pick}
    for b in range(0, B, max(1, B // 2)):
        ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P[b:b + 1], members=members, subsets=pick)
        sub = dict(z=out["z"][b:b + 1], yhat=out["yhat"][b:b + 1], sspe=out["sspe"][b:b + 1])
        worst = compare(sub, ref, V_off, pick, 1, prec, check_total=False)
        print("paper-scale", prec, b, worst)


@pytest.mark.parametrize("engine", ["tensor", "simt", "tensor-bf16", "tensor-tf32", "tensor-tf32x3"])
def test_mixed_engines(gpu_lib, engine):
    """Every factorisation engine of the mixed path (tcgen05 with two-term FP16 or
    three-term BF16 operands, FP32 SIMT) meets the mixed tolerance on subsets spanning
    several 128-row tiles and a ragged tail (uniform 4096 workload, three
    configurations, one with a nugget ratio of 5e-4)."""
    w = datagen.config_uniform_4096()
    P = np.array([[1.0, 0.1, 0.05], [0.7, 0.03, 0.2], [2.0, 0.3, 0.001]])
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, factor_engine=engine) as ctx:
        out = ctx.cv_loss(P, precision="mixed", per_subset=True, predictions=True)
        V_off = ctx.V_off.copy()
    members = oracle.all_members(w.xy, w.role, w.layout)
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P, members=members)
    if engine == "tensor-tf32":   # 11-bit operands: ill-conditioned tasks fall back to FP64
        assert np.all(np.isin(out["status"], (0, 7))), out["status"]
    else:
        assert np.all(out["status"] == 0), out["status"]
    worst = compare(out, ref, V_off, range(16), len(P), "mixed")
    print("mixed", engine, out["status"].tolist(), worst)


@pytest.mark.parametrize("rho,tau2", [(0.02, 0.001), (0.02, 0.1), (0.2, 0.001), (0.2, 0.01), (0.2, 0.1)])
@pytest.mark.parametrize("prec,engine", [("mixed", "tensor"), ("mixed", "tensor-bf16"), ("fp64", "tensor"),
                                         ("mixed-tf32", "tensor"), ("mixed-tf32x3", "tensor")])
def test_grid_precision_stress(gpu_lib, prec, engine, rho, tau2):
    """Gridded 1024^2 training set (fine 2048^2 grid, 131 072 validation nodes), 32-cell
    cores with 8-cell shells (k = 1600 / 1920 / 2304): the conditioning sweep of the
    precision-stress workload (rho in {0.02, 0.2}, tau2 in {0.001, 0.01, 0.1}, the
    largest condition numbers near 1e6), for every operand scheme of the tensor-core
    factorisation (FP16 x2, BF16 x3, TF32 x1, TF32 x3) and FP64.  The field's own
    parameters are evaluated; sampled subsets (corner, edge, interior) are compared
    with the oracle.  Plain TF32 (11 significant bits) is expected to fail its
    refinement on the ill-conditioned cases: those tasks are recomputed in FP64
    (status PCV_REFINE_FALLBACK) and still meet the bar; the counts are printed."""
    w = datagen.config_grid_1m(rho=rho, tau2=tau2)
    P = w.params
    nx = w.layout["nx"]
    pick = [0, nx // 2, nx * (nx // 2) + nx // 2]
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, factor_engine=engine) as ctx:
        ctx.set_timing(True)
        out = ctx.cv_loss(P, precision=prec, per_subset=True, predictions=True)
        ph = ctx.phase_cycles() if prec.startswith("mixed") else {}
        V_off = ctx.V_off.copy()
    assert out["status"][0] in (0, 7), out["status"]       # 7: some tasks recomputed in FP64
    cores = oracle.layout_cores(w.layout, w.xy)
    members = {i: oracle.subset_members(w.xy, w.role, w.layout, i, cores) for i in pick}
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P, members=members, subsets=pick)
    worst = compare(out, ref, V_off, pick, 1, prec, check_total=False)
    if prec == "mixed-tf32x3" or (prec == "mixed" and engine != "simt"):
        assert out["status"][0] == 0, out["status"]       # the 22-24-bit schemes refine every task
    counts = {k: ph.get(k) for k in ("tasks", "residual_passes", "fail_factor", "fail_nan", "fail_stall")}
    print("grid stress", prec, engine, rho, tau2, out["status"].tolist(), worst, counts)


def test_no_pivot_failures_paper_scale(gpu_lib, paper5m):
    """The FP32 factorisation of the benchmark workload never breaks down: 100
    configurations (nugget ratios 0.025-0.1, the less well-conditioned half of the
    grid) in batches of 20, 160 000 tasks, none handed to the FP64 fallback because of
    a non-positive pivot.  (A race in the padding of the last, partial diagonal
    block once made about one task in 10^4 fail here and nowhere smaller.)"""
    w = paper5m
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        ctx.set_timing(True)
        fails = 0
        for s0 in range(100, 200, 20):
            ctx.phase_cycles(reset=True)
            out = ctx.cv_loss(w.params[s0:s0 + 20])
            fails += ctx.phase_cycles()["fail_factor"]
            assert np.all(np.isin(out["status"], (0, 7)))
    assert fails == 0


@pytest.mark.parametrize("prec", PRECS)
def test_recursive_layout_with_shell_cap(gpu_lib, prec):
    """Recursive division (Sec. 2.4) into 16 sub-domains with shells of width 0.05 capped
    at 150 training points (Sec. 4.3.2): every subset's loss and predictions."""
    w = datagen.config_uniform_4096()
    layout = dict(kind="recursive", q=4, delta=0.05, domain=(0.0, 1.0, 0.0, 1.0), shell_cap=150, cap_seed=21)
    w.layout = layout
    P = np.array([[1.0, 0.1, 0.05], [0.5, 0.04, 0.01]])
    out, ref, V_off = _run(gpu_lib, w, P, prec)
    assert np.all(out["status"] == 0), out["status"]
    worst = compare(out, ref, V_off, range(16), len(P), prec)
    print("recursive", prec, worst)


@pytest.fixture(scope="module")
def paper5m_recursive():
    return datagen.config_paper_5m_recursive()


def test_paper_recursive_sampled(gpu_lib, paper5m_recursive):
    """The paper's weak-scaling layout (Sec. 4.3.2) on the 5M-point field: 512 recursive
    sub-domains, shell 0.001 capped at 2000, k about 8.3k-8.6k (ld 8704).  Mixed path,
    two configurations: all statuses clean, and the smallest, the largest and an
    interior subset compared with the oracle (LAPACK-backed kriging for these sizes)."""
    w = paper5m_recursive
    P = w.params[[0, 137]]
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        out = ctx.cv_loss(P, precision="mixed", per_subset=True, predictions=True)
        T_off, V_off = ctx.T_off.copy(), ctx.V_off.copy()
    assert np.all(out["status"] == 0), out["status"]
    assert np.all(np.isfinite(out["sspe"]))
    k = np.diff(T_off)
    pick = sorted({int(np.argmin(k)), int(np.argmax(k)), 300})
    cores = oracle.layout_cores(w.layout, w.xy)
    members = {i: oracle.subset_members(w.xy, w.role, w.layout, i, cores) for i in pick}
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P, members=members, subsets=pick, lapack=True)
    worst = compare(out, ref, V_off, pick, len(P), "mixed", check_total=False)
    print("paper recursive", [int(k[i]) for i in pick], worst)


# Mixed-path bars of the local -2 log-likelihood: its log-determinant comes from the
# FP32-accurate factor, whose relative error grows with the condition number (measured:
# 2e-6 at condition ~1e3, 5.5e-5 at ~1e5); refinement corrects solutions, not
# determinants.  The corner case (rho = 0.2, tau2 = 0.001, condition ~1e6) records where
# that leaves the mixed result (measured 9.3e-5); FP64 meets 1e-10 everywhere.
LIK_MIXED_BAR = {"uniform": 1e-4, "grid-stress": 1e-4, "grid-corner": 5e-4}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("wl", ["uniform", "grid-stress", "grid-corner"])
def test_local_neg2loglik(gpu_lib, prec, wl):
    """Local -2 log-likelihood (Eq. 2) of every subset's training data, a by-product of
    the CV factorisations, against the oracle's Eq. 2 routine: per subset and the
    fixed-order total.  FP64 path within 1e-10.  Mixed path within 1e-4 relative: the
    log-determinant comes from the FP32 factor and is not refined, so its error grows
    with the conditioning (measured 2.0e-6 on the uniform workload, 1e-3 absolute of
    -2 log L ~ 500; 3.8e-5 on the rho = 0.2 precision-stress grid, condition ~1e5)."""
    if wl == "uniform":
        w = datagen.config_uniform_4096()
        P = np.array([[1.0, 0.1, 0.05], [0.5, 0.04, 0.01], [2.0, 0.3, 0.2]])
        pick = None
    else:
        t2 = 0.01 if wl == "grid-stress" else 0.001
        w = datagen.config_grid_1m(rho=0.2, tau2=t2)
        P = np.array([[1.0, 0.2, t2]])
        nx = w.layout["nx"]
        pick = [0, nx // 2, nx * (nx // 2) + nx // 2]
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        out = ctx.neg2loglik(P, precision=prec, per_subset=True)
        V_off = ctx.V_off.copy()
    assert np.all(out["status"] == 0), out["status"]
    cores = oracle.layout_cores(w.layout, w.xy)
    subsets = range(len(cores)) if pick is None else pick
    tol = 1e-10 if prec == "fp64" else LIK_MIXED_BAR[wl]
    worst = 0.0
    for b, (s2, rho, tau) in enumerate(P):
        tot = 0.0
        for i in subsets:
            if V_off[i + 1] == V_off[i]:
                assert out["per_subset"][b, i] == 0.0
                continue
            T, _ = oracle.subset_members(w.xy, w.role, w.layout, i, cores)
            ref, st = oracle.neg2loglik(w.xy[T], w.v[T], s2, rho, tau)
            assert st == oracle.OK
            e = abs(out["per_subset"][b, i] - ref) / abs(ref)
            worst = max(worst, e)
            assert e <= tol, (prec, b, i, out["per_subset"][b, i], ref)
            tot += ref
        if pick is None:
            assert abs(out["total"][b] - tot) <= tol * abs(tot)
    print("neg2loglik", wl, prec, worst)


@pytest.mark.parametrize("prec", PRECS)
def test_predict_local_best(gpu_lib, prec):
    """Non-stationary prediction (Sec. 4.4): each subset's locally best configuration,
    chosen from the per-subset losses, predicts the new locations of its core.  The
    choice is the per-subset minimum of the returned losses and optimal for the
    oracle's losses within the tolerance; the predictions match the oracle's kriging
    with each subset's chosen parameters."""
    w = datagen.config_uniform_4096()
    P = np.array([[1.0, 0.1, 0.05], [1.0, 0.03, 0.05], [1.0, 0.3, 0.01], [1.0, 0.1, 0.3],
                  [0.5, 0.05, 0.005], [2.0, 0.2, 0.1]])
    pts = np.random.default_rng(31).random((400, 2)) * 1.1 - 0.05     # some outside D
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        out = ctx.cv_loss(P, precision=prec, per_subset=True)
        yhat, best = ctx.predict_local(P, out["z"], pts, precision=prec)
        V_off = ctx.V_off.copy()
    members = oracle.all_members(w.xy, w.role, w.layout)
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P, members=members)
    for i in range(len(members)):
        if V_off[i + 1] == V_off[i]:
            continue
        assert best[i] == int(np.argmin(out["z"][:, i]))
        assert ref["z"][best[i], i] <= ref["z"][:, i].min() * (1 + TOL[prec]["loss"])
    core = oracle.core_of(w.layout, pts, w.xy)
    worst = 0.0
    for i in np.unique(core):
        sel = np.nonzero(core == i)[0]
        s2, rho, tau = P[best[i]]
        T = members[i][0]
        want, st = oracle.krige(w.xy[T], w.v[T], pts[sel], rho, tau / s2)
        e = pred_err(yhat[sel], want)
        worst = max(worst, e)
        assert e <= TOL[prec]["pred"], (i, e)
    print("predict_local", prec, sorted(set(best.tolist())), worst)


@pytest.mark.parametrize("prec", PRECS)
def test_gls_mean(gpu_lib, prec):
    """GLS coefficients of a linear mean (Sec. 5) from prediction operations on the
    covariate columns, against the oracle's same parallel approximation: FP64 within
    1e-9, mixed within 1e-5 relative (max norm); a planted trend is recovered."""
    w = datagen.config_uniform_4096()
    n = len(w.v)
    X = np.stack([np.ones(n), w.xy[:, 0], w.xy[:, 1], w.xy[:, 0] * w.xy[:, 1]], 1)
    beta_true = np.array([1.5, -2.0, 0.7, 1.0])
    v = w.v + X @ beta_true
    param = (1.0, 0.1, 0.05)
    with gpu_lib.Context(w.xy, v, w.role, w.layout) as ctx:
        beta = ctx.gls(X, param, precision=prec)
    ref = oracle.gls(w.xy, v, w.role, w.layout, X, param)
    err = np.max(np.abs(beta - ref)) / np.max(np.abs(ref))
    assert err <= (1e-9 if prec == "fp64" else 1e-5), (beta, ref)
    assert np.allclose(beta, beta_true, atol=1.0)
    print("gls", prec, beta.tolist(), err)


def test_lattice_path(gpu_lib):
    """Lattice data (every point on one regular grid): the mixed CV loss takes its
    covariances from per-task tables by lattice offset.  The detection, parity with the
    oracle on every subset, and agreement with the general path (the same data with one
    point moved off the lattice by 1e-9)."""
    w = datagen.config_grid_1m(rho=0.05, tau2=0.02, fine=256, cells=32, buf=8, n_valid=2048, seed=77)
    P = np.array([[1.0, 0.05, 0.02], [0.7, 0.12, 0.005]])
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        lat = ctx.lattice()
        out = ctx.cv_loss(P, precision="mixed", per_subset=True, predictions=True)
        V_off = ctx.V_off.copy()
    assert lat is not None and abs(lat[0] - 1 / 256) < 1e-15 and abs(lat[1] - 1 / 256) < 1e-15
    det = gpu_lib.pcv_lattice_detect(w.xy)          # the host rule pcv_create applied
    assert det is not None and (det[0][1], det[1][1]) == lat
    assert np.all(out["status"] == 0)
    members = oracle.all_members(w.xy, w.role, w.layout)
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P, members=members)
    worst = compare(out, ref, V_off, range(len(members)), len(P), "mixed")
    xy2 = w.xy.copy()
    xy2[5, 0] += 1e-9                      # one IGNORE-free point off the lattice
    with gpu_lib.Context(xy2, w.v, w.role, w.layout) as ctx2:
        assert ctx2.lattice() is None
        out2 = ctx2.cv_loss(P, precision="mixed")
    assert np.all(np.abs(out2["sspe"] - out["sspe"]) <= 1e-6 * np.abs(out["sspe"]))
    # a whole grid column shifted by 1e-7 of the spacing keeps every gap near h, but
    # is off the lattice by far more than coordinate rounding: no snapping, and the
    # general path matches the oracle on the shifted data
    xy3 = w.xy.copy()
    col = np.isclose(xy3[:, 0], np.unique(xy3[:, 0])[100], rtol=0, atol=1e-12)
    assert col.sum() > 0
    xy3[col, 0] += 1e-7 / 256
    assert gpu_lib.pcv_lattice_detect(xy3) is None
    with gpu_lib.Context(xy3, w.v, w.role, w.layout) as ctx3:
        assert ctx3.lattice() is None
        out3 = ctx3.cv_loss(P, precision="mixed", per_subset=True, predictions=True)
        V_off3 = ctx3.V_off.copy()
    members3 = oracle.all_members(xy3, w.role, w.layout)
    ref3 = oracle.cv_loss(xy3, w.v, w.role, w.layout, P, members=members3)
    worst3 = compare(out3, ref3, V_off3, range(len(members3)), len(P), "mixed")
    print("lattice", worst, "shifted column", worst3)


def test_size_buckets_autotuned(gpu_lib, cluster):
    """Size-bucketed launch (the default for the mixed CV loss): the uneven cluster workload
    is split by training size into buckets with their own slot sizes and autotuned engines,
    launched side by side.  Every subset matches the oracle (as in test_cluster_batch_all),
    the single-launch form agrees within the mixed tolerance, and a second context with the
    same size histogram reuses the tuner's cached choice."""
    w, P, act, ref = cluster
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        out = ctx.cv_loss(P, precision="mixed", per_subset=True, predictions=True)
        desc = ctx.buckets()
        V_off = ctx.V_off.copy()
    lines = [ln for ln in desc.strip().splitlines() if ln.startswith("k ")]     # one per bucket
    assert lines and all(("tensor" in ln) or ("simt" in ln) for ln in lines), desc
    assert sum(int(ln.split(":")[1].split()[0]) for ln in lines) == len(act)
    assert np.all(out["status"] == 0)
    worst = compare(out, ref, V_off, act, len(P), "mixed", check_total=False)
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, bucketing=1) as ctx1:
        one = ctx1.cv_loss(P, precision="mixed", per_subset=True)
        one_desc = ctx1.buckets()
    assert len([ln for ln in one_desc.strip().splitlines() if ln.startswith("k ")]) == 1
    assert np.all(rel(out["sspe"], one["sspe"]) <= 2 * TOL["mixed"]["loss"])
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx2:
        again = ctx2.cv_loss(P, precision="mixed")
        assert [ln for ln in ctx2.buckets().splitlines() if ln.startswith("k ")] == lines   # the cached choice
    assert np.array_equal(again["sspe"], out["sspe"])       # same engines, same arithmetic
    print("buckets", lines, worst)


@pytest.mark.parametrize("engine", ["tensor", "simt"])
def test_loss_aware_refinement_stop(gpu_lib, cluster, engine):
    """The loss-aware stopping rule (refine_loss_tol, the default) against the solution
    rule alone (refine_loss_tol < 0) on every subset of the cluster workload: both meet
    the mixed bars against the oracle, and the loss-aware rule spends no more residual
    passes.  The rule stops a task once the estimated error left in its predictions
    moves the local SSPE by at most 2e-8 relative; the SSPE amplifies prediction errors
    by about |yhat| / |yhat - y|, which varies from subset to subset."""
    w, P, act, ref = cluster
    passes = {}
    for label, lt in (("loss-aware", 0.0), ("solution", -1.0)):
        with gpu_lib.Context(w.xy, w.v, w.role, w.layout, factor_engine=engine, refine_loss_tol=lt,
                             bucketing=1) as ctx:
            ctx.set_timing(True)
            out = ctx.cv_loss(P, precision="mixed", per_subset=True, predictions=True)
            ph = ctx.phase_cycles()
            V_off = ctx.V_off.copy()
        assert np.all(out["status"] == 0), out["status"]
        worst = compare(out, ref, V_off, act, len(P), "mixed", check_total=False)
        passes[label] = ph["residual_passes"] / max(ph["tasks"], 1)
        print(engine, label, worst, "passes per task", passes[label])
    assert passes["loss-aware"] <= passes["solution"] + 1e-9


@pytest.mark.parametrize("prec", PRECS)
def test_predict_from_kept_weights(gpu_lib, prec):
    """Predictions at new locations from the kriging weights a CV evaluation kept
    (alpha_cache): after pcv_cv_loss of a batch, pcv_predict with one of its
    configurations factors nothing (a cache hit) and matches the oracle's kriging (Eq. 3)
    at the precision's bar; a configuration not evaluated before is solved (a miss) and
    kept, so asking again hits; with the cache off every call solves."""
    w = datagen.make_uniform(1500, 700, 3, 0.06, seed=57, name="alpha")
    P = np.array([[1.0, 0.1, 0.05], [2.0, 0.05, 0.02], [0.8, 0.15, 0.01]])
    pts = np.random.default_rng(3).random((900, 2)) * 1.1 - 0.05
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout) as ctx:
        ctx.cv_loss(P, precision=prec)
        got = [ctx.predict(p, pts, precision=prec) for p in P]
        st1 = ctx.alpha_cache_stats()
        p_new = (1.3, 0.08, 0.03)
        y_new = ctx.predict(p_new, pts, precision=prec)
        y_new2 = ctx.predict(p_new, pts, precision=prec)
        st2 = ctx.alpha_cache_stats()
    assert st1["hits"] == len(P) and st1["misses"] == 0, st1
    assert st2["hits"] == len(P) + 1 and st2["misses"] == 1, st2
    for p, yh in zip(list(P) + [p_new], got + [y_new]):
        ref = oracle.predict(w.xy, w.v, w.role, w.layout, tuple(p), pts)
        assert pred_err(yh, ref) <= TOL[prec]["pred"], (p, pred_err(yh, ref))
    assert pred_err(y_new2, y_new) <= TOL[prec]["pred"]
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, alpha_cache=-1) as ctx0:
        ctx0.cv_loss(P, precision=prec)
        y0 = ctx0.predict(P[0], pts, precision=prec)
        assert ctx0.alpha_cache_stats() == dict(hits=0, misses=0, rows=0)
    assert pred_err(got[0], y0) <= TOL[prec]["pred"]


def test_bounded_wait_runs_out(gpu_lib):
    """A device wait that runs out, in the form this pool allows: the waits of the
    tensor-core pipeline are shortened to 5 ms and the TMA producer withholds the first
    operand stage of one task, so the MMA issuer's and the epilogue's waits on it expire
    (no trap, fault or unbounded wait).  The CTA lets its issued copies and products
    complete, stops using the tensor path and hands its tasks to the FP64 fallback:
    every result still meets the bar, the affected configuration reports
    PCV_REFINE_FALLBACK, and the same call without the hook runs clean."""
    w = datagen.config_uniform_4096()
    P = np.array([[1.0, 0.1, 0.05], [0.7, 0.03, 0.2]])
    members = oracle.all_members(w.xy, w.role, w.layout)
    ref = oracle.cv_loss(w.xy, w.v, w.role, w.layout, P, members=members)
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, bucketing=1, graph=1, test_wait_us=5000,
                         test_withhold_task=3) as ctx:
        ctx.set_timing(True)
        out = ctx.cv_loss(P, precision="mixed", per_subset=True, predictions=True)
        ph = ctx.phase_cycles()
        V_off = ctx.V_off.copy()
    assert 7 in out["status"].tolist(), out["status"]
    assert np.all(np.isin(out["status"], (0, 7))), out["status"]
    assert ph["fail_factor"] >= 1, ph
    compare(out, ref, V_off, range(len(members)), len(P), "mixed")
    with gpu_lib.Context(w.xy, w.v, w.role, w.layout, bucketing=1, test_wait_us=5000) as ctx:
        out2 = ctx.cv_loss(P, precision="mixed")
    assert np.all(out2["status"] == 0), out2["status"]
    print("wait ran out:", out["status"].tolist(), "fallback tasks", ph["fail_factor"])
