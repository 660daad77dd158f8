"""Pins for the CPU oracle: each checks the oracle against something other than itself.

What pins what (all CPU, no GPU):

* Cholesky:   the factor of an SPD matrix is the unique lower-triangular L with a
              positive diagonal and L L^T = A -- checked on matrices with a known
              integer factor (exact) and by reconstruction on random SPD matrices.
* Solves:     exact rational Gaussian elimination (Python ``fractions``) on the
              FP64 matrix entries, k <= 7.
* Kriging:    Eq. 3 closed forms for one and two training points; zero-nugget
              interpolation of the training data; the lambda -> infinity limit;
              the sigma^2 invariance stated under Eq. 3; an independent LU solve
              (numpy.linalg.solve, which the oracle does not use) for a few hundred
              points.
* SSPE:       Eq. 4 on hand-computed numbers.
* Likelihood: Eq. 2 closed form for one point and an independent slogdet/solve.
* Layout:     a hand-derived membership fixture (tests/golden/layout_tiny.json);
              disjointness and covering of the cores; shells containing the cores;
              a shell wider than D gives every subset all training data.
* CV~:        additivity over subsets (Eq. 5-6), N = 1 equals global CV (Sec. 4.3.1),
              invariance under permutation of the input points.

``test_planted_mistakes`` compiles copies of the oracle with one plausible mistake
each and checks that at least one pin fails for every copy.
"""
from __future__ import annotations

import json
import math
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
U = np.finfo(np.float64).eps / 2


def _rng(s=0):
    return np.random.default_rng(1000 + s)


def _exp_cov(a, b, rho):
    """Independent restatement for the pins: numpy broadcasting, Euclidean norm."""
    d = np.sqrt(((a[:, None, :] - b[None, :, :]) ** 2).sum(-1))
    return np.exp(-d / rho)


# ---------------------------------------------------------------------------
# pins (plain functions so the planted-mistake test can run them as a battery)
# ---------------------------------------------------------------------------
def pin_cholesky_known_factor():
    Lx = np.array([[2.0, 0, 0, 0], [1, 3, 0, 0], [-1, 2, 1, 0], [4, -2, 0.5, 2]])
    A = Lx @ Lx.T
    L, st = oracle.cholesky(A)
    assert st == oracle.OK
    assert np.array_equal(L, Lx), (L, Lx)


def pin_cholesky_reconstruction():
    for k in (1, 2, 5, 17, 40):
        M = _rng(k).standard_normal((k, k))
        A = M @ M.T + k * np.eye(k)
        L, st = oracle.cholesky(A)
        assert st == oracle.OK
        assert np.all(np.triu(L, 1) == 0) and np.all(np.diag(L) > 0)
        err = np.linalg.norm(L @ L.T - A) / np.linalg.norm(A)
        assert err < 4 * k * U, err


def pin_cholesky_not_spd():
    A = np.array([[1.0, 2.0], [2.0, 1.0]])
    _, st = oracle.cholesky(A)
    assert st == oracle.NOT_SPD


def _exact_solve(A, b):
    k = len(b)
    M = [[Fraction(float(A[i, j])) for j in range(k)] + [Fraction(float(b[i]))] for i in range(k)]
    for c in range(k):
        p = next(r for r in range(c, k) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(k):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return np.array([float(M[i][k] / M[i][i]) for i in range(k)])


def pin_solve_exact_rational():
    for k in (1, 3, 7):
        r = _rng(10 + k)
        s = r.random((k, 2))
        A = _exp_cov(s, s, 0.3) + 0.1 * np.eye(k)
        b = r.standard_normal(k)
        x, st = oracle.solve_spd(A, b)
        assert st == oracle.OK
        xe = _exact_solve(A, b)
        cond = np.linalg.cond(A)
        assert np.max(np.abs(x - xe)) <= 50 * k * cond * U * np.max(np.abs(xe)), (x, xe)


def pin_krige_one_point():
    sT = np.array([[0.2, 0.3]])
    sP = np.array([[0.5, 0.7], [0.2, 0.3]])
    rho, lam, y = 0.25, 0.4, 1.7
    yh, st = oracle.krige(sT, [y], sP, rho, lam)
    d = math.sqrt(0.3 ** 2 + 0.4 ** 2)          # 0.5
    want = [math.exp(-d / rho) * y / (1 + lam), y / (1 + lam)]
    assert st == oracle.OK
    assert np.allclose(yh, want, rtol=1e-14, atol=0), (yh, want)


def pin_krige_two_points():
    sT = np.array([[0.0, 0.0], [0.3, 0.4]])     # distance 0.5
    sP = np.array([[0.6, 0.8]])                  # distances 1.0 and 0.5
    rho, lam = 0.5, 0.2
    y = np.array([1.0, -2.0])
    c = math.exp(-1.0)
    det = (1 + lam) ** 2 - c * c
    inv = np.array([[1 + lam, -c], [-c, 1 + lam]]) / det
    p = np.array([math.exp(-2.0), math.exp(-1.0)])
    want = p @ inv @ y
    yh, st = oracle.krige(sT, y, sP, rho, lam)
    assert st == oracle.OK
    assert abs(yh[0] - want) <= 1e-14 * abs(want), (yh, want)


def pin_zero_nugget_interpolates():
    r = _rng(3)
    s = r.random((12, 2))
    y = r.standard_normal(12)
    yh, st = oracle.krige(s, y, s, 0.1, 0.0)
    assert st == oracle.OK
    cond = np.linalg.cond(_exp_cov(s, s, 0.1))
    assert np.max(np.abs(yh - y)) <= 100 * cond * U * np.max(np.abs(y)), np.max(np.abs(yh - y))


def pin_large_nugget_limit():
    r = _rng(4)
    s, p = r.random((20, 2)), r.random((5, 2))
    y = r.standard_normal(20)
    lam = 1e9
    yh, _ = oracle.krige(s, y, p, 0.2, lam)
    first = _exp_cov(p, s, 0.2) @ y / lam        # (Sigma + lam I)^{-1} = I/lam + O(lam^-2)
    assert np.allclose(yh, first, rtol=1e-7, atol=0)


def pin_sigma2_invariance():
    r = _rng(5)
    s, p = r.random((30, 2)), r.random((7, 2))
    y = r.standard_normal(30)
    base, _ = oracle.krige(s, y, p, 0.15, 0.05 / 1.0)
    for s2 in (0.5, 2.0, 7.0):
        lit, st = oracle.krige_literal(s, y, p, s2, 0.15, 0.05 * s2)
        assert st == oracle.OK
        assert np.allclose(lit, base, rtol=1e-12, atol=1e-14), (s2, lit - base)


def pin_krige_vs_lu():
    r = _rng(6)
    s, p = r.random((300, 2)), r.random((40, 2))
    y = r.standard_normal(300)
    rho, lam = 0.1, 0.03
    A = _exp_cov(s, s, rho) + lam * np.eye(300)
    want = _exp_cov(p, s, rho) @ np.linalg.solve(A, y)
    yh, st = oracle.krige(s, y, p, rho, lam)
    assert st == oracle.OK
    cond = np.linalg.cond(A)
    assert np.max(np.abs(yh - want)) <= 10 * cond * U * np.max(np.abs(want)) * 300 ** 0.5


def pin_sspe_hand():
    assert oracle.sspe([1.5, 2.0, 2.0], [1.0, 2.0, 3.0]) == 1.25
    assert oracle.sspe([], []) == 0.0


def pin_neg2loglik():
    v, st = oracle.neg2loglik([[0.1, 0.1]], [1.3], 2.0, 0.1, 0.5)
    want = math.log(2 * math.pi) + math.log(2.5) + 1.3 ** 2 / 2.5
    assert st == oracle.OK and abs(v - want) < 1e-14 * abs(want)
    r = _rng(7)
    s = r.random((50, 2))
    y = r.standard_normal(50)
    C = 1.5 * _exp_cov(s, s, 0.2) + 0.1 * np.eye(50)
    want = 50 * math.log(2 * math.pi) + np.linalg.slogdet(C)[1] + y @ np.linalg.solve(C, y)
    v, st = oracle.neg2loglik(s, y, 1.5, 0.2, 0.1)
    assert abs(v - want) < 1e-10 * abs(want)


def _tiny():
    with open(os.path.join(HERE, "golden", "layout_tiny.json")) as f:
        g = json.load(f)
    pts = np.array(g["points"])
    lay = dict(kind="grid", nx=g["nx"], ny=g["ny"], delta=g["delta"], domain=tuple(g["domain"]))
    return pts[:, :2].copy(), pts[:, 2].astype(np.uint8), lay, g


def pin_layout_fixture():
    xy, role, lay, g = _tiny()
    for i in range(4):
        T, V = oracle.subset_members(xy, role, lay, i)
        assert T.tolist() == g["T"][i], (i, T, g["T"][i])
        assert V.tolist() == g["V"][i], (i, V, g["V"][i])


def pin_layout_partition():
    r = _rng(8)
    xy = r.random((3000, 2))
    xy[:50] = np.round(xy[:50] * 5) / 5          # points exactly on the cut lines and on D's edge
    role = r.integers(0, 3, 3000).astype(np.uint8)
    lay = dict(kind="grid", nx=5, ny=5, delta=0.03, domain=(0.0, 1.0, 0.0, 1.0))
    mem = oracle.all_members(xy, role, lay)
    allv = np.concatenate([V for _, V in mem])
    assert sorted(allv.tolist()) == np.nonzero(role == oracle.VALID)[0].tolist()
    for i, (T, V) in enumerate(mem):
        coreT = oracle.subset_members(xy, role.copy() * 0 + np.where(role == 0, 1, 2).astype(np.uint8),
                                      lay, i)[1]   # TRAIN points re-labelled VALID: core membership
        assert set(coreT.tolist()) <= set(T.tolist())
        assert np.all(role[T] == oracle.TRAIN) and np.all(role[V] == oracle.VALID)


def pin_layout_wide_shell():
    r = _rng(9)
    xy = r.random((500, 2))
    role = (r.random(500) < 0.5).astype(np.uint8)
    lay = dict(kind="grid", nx=3, ny=2, delta=2.0, domain=(0.0, 1.0, 0.0, 1.0))
    tr = np.nonzero(role == 0)[0].tolist()
    for T, _ in oracle.all_members(xy, role, lay):
        assert T.tolist() == tr


def _small_workload(seed=11, n=700, nx=3, delta=0.08):
    r = _rng(seed)
    xy = r.random((n, 2))
    v = r.standard_normal(n)
    role = (r.random(n) < 0.35).astype(np.uint8)
    lay = dict(kind="grid", nx=nx, ny=nx, delta=delta, domain=(0.0, 1.0, 0.0, 1.0))
    return xy, v, role, lay


def pin_cv_additive_and_global():
    xy, v, role, lay = _small_workload()
    P = np.array([[1.0, 0.1, 0.05], [2.0, 0.2, 0.01]])
    res = oracle.cv_loss(xy, v, role, lay, P)
    assert np.allclose(res["sspe"], np.nansum(res["z"], axis=1), rtol=1e-15)
    lay1 = dict(lay, nx=1, ny=1)
    res1 = oracle.cv_loss(xy, v, role, lay1, P)
    T, V = np.nonzero(role == 0)[0], np.nonzero(role == 1)[0]
    for b, (s2, rho, tau) in enumerate(P):
        A = _exp_cov(xy[T], xy[T], rho) + tau / s2 * np.eye(len(T))
        yh = _exp_cov(xy[V], xy[T], rho) @ np.linalg.solve(A, v[T])
        want = float(((yh - v[V]) ** 2).sum())
        assert abs(res1["sspe"][b] - want) <= 1e-9 * want, (res1["sspe"][b], want)


def pin_cv_permutation():
    xy, v, role, lay = _small_workload(seed=12)
    P = np.array([[1.0, 0.12, 0.03]])
    a = oracle.cv_loss(xy, v, role, lay, P)
    perm = _rng(13).permutation(len(v))
    b = oracle.cv_loss(xy[perm], v[perm], role[perm], lay, P)
    assert abs(a["sspe"][0] - b["sspe"][0]) <= 1e-12 * a["sspe"][0]
    for (Ta, Va), (Tb, Vb) in zip(a["members"], b["members"]):
        assert sorted(perm[Tb].tolist()) == Ta.tolist()
        assert sorted(perm[Vb].tolist()) == Va.tolist()


PINS = [pin_cholesky_known_factor, pin_cholesky_reconstruction, pin_cholesky_not_spd,
        pin_solve_exact_rational, pin_krige_one_point, pin_krige_two_points,
        pin_zero_nugget_interpolates, pin_large_nugget_limit, pin_sigma2_invariance,
        pin_krige_vs_lu, pin_sspe_hand, pin_neg2loglik, pin_layout_fixture,
        pin_layout_partition, pin_layout_wide_shell, pin_cv_additive_and_global,
        pin_cv_permutation]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


def test_predict_uses_containing_core():
    xy, v, role, lay = _small_workload(seed=14)
    pts = np.array([[0.1, 0.1], [0.5, 0.5], [0.99, 0.2], [1.5, -0.3], [1.0, 1.0]])
    core = oracle.core_of(lay, pts)
    assert core.tolist() == [0, 4, 2, 2, 8]
    yh = oracle.predict(xy, v, role, lay, (1.0, 0.1, 0.05), pts)
    for j, i in enumerate(core):
        T, _ = oracle.subset_members(xy, role, lay, int(i))
        A = _exp_cov(xy[T], xy[T], 0.1) + 0.05 * np.eye(len(T))
        want = _exp_cov(pts[j:j + 1], xy[T], 0.1) @ np.linalg.solve(A, v[T])
        assert abs(yh[j] - want[0]) <= 1e-9 * max(1.0, abs(want[0]))


# ---------------------------------------------------------------------------
# planted mistakes: every plausible slip in the oracle must trip some pin
# ---------------------------------------------------------------------------
MUTATIONS = {
    "norm-index": ("return sqrt(dx * dx + dy * dy);", "return sqrt(dx * dx + dx * dy);"),
    "range-inverted": ("return exp(-dist2d(a, b) / theta);", "return exp(-dist2d(a, b) * theta);"),
    "nugget-dropped": ("(i == j ? nugget : 0.0)", "(i == j ? 0.0 : 0.0)"),
    "nugget-everywhere": ("(i == j ? nugget : 0.0)", "nugget"),
    "pivot-sign": ("s -= rj[p] * rj[p];", "s += rj[p] * rj[p];"),
    "offdiag-index": ("t -= ri[p] * rj[p];", "t -= ri[p] * ri[p];"),
    "divide-pivot": ("ri[j] = t / ljj;", "ri[j] = t * ljj;"),
    "backsub-transposed": ("t -= l[p * k + i] * w[p];", "t -= l[i * k + p] * w[p];"),
    "cross-cov-scale": ("t += scale * cov_exp(", "t += cov_exp("),
    "sspe-abs": ("z += e * e;", "z += fabs(e);"),
    "core-closed-low": ("if (!(x >= x0)) continue;", "if (!(x > x0)) continue;"),
    "core-closed-high": ("if (x1_incl ? !(x <= x1) : !(x < x1)) continue;",
                         "if (!(x <= x1)) continue;"),
    "logdet-half": ("logdet += 2.0 * log(", "logdet += log("),
}


def _battery() -> list[str]:
    failed = []
    for p in PINS:
        try:
            p()
        except Exception as e:  # noqa: BLE001 - any failure of a pin counts
            failed.append(f"{p.__name__}: {type(e).__name__}")
    return failed


def test_pins_pass_on_the_oracle():
    assert _battery() == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes(name):
    old, new = MUTATIONS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "pcv_oracle.c")).read()
    assert src.count(old) >= 1, name
    d = tempfile.mkdtemp()
    try:
        c = os.path.join(d, "m.c")
        so = os.path.join(d, "m.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                               "-shared", "-fPIC", c, "-o", so, "-lm"])
        with oracle.using_library(so):
            failed = _battery()
        assert failed, f"mutation {name} passed every pin"
    finally:
        shutil.rmtree(d)


@pytest.mark.parametrize("k", [1, 2, 57, 420])
def test_lapack_kriging_matches_plain_routine(k):
    """The LAPACK-backed kriging used for large subsets agrees with the pinned plain
    C routine (and, at k = 1, with Eq. 3's closed form e^{-d/rho} y / (1 + lambda))."""
    r = _rng(40 + k)
    sT, yT, sP = r.random((k, 2)), r.standard_normal(k), r.random((30, 2))
    for rho, lam in ((0.05, 0.02), (0.3, 1e-3), (0.1, 0.5)):
        a, sa = oracle.krige(sT, yT, sP, rho, lam)
        b, sb = oracle.krige_lapack(sT, yT, sP, rho, lam)
        assert sa == sb == oracle.OK
        assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.max(np.abs(a)))
        if k == 1:
            d = np.sqrt(((sP - sT[0]) ** 2).sum(1))
            assert np.allclose(b, np.exp(-d / rho) * yT[0] / (1 + lam), rtol=1e-14, atol=0)


def test_gls_one_subset_is_exact_gls():
    """Sec. 5's identity M^-1 = (I - H) / lambda: with one subset covering D the
    prediction-based GLS equals GLS by dense solves; with a linear trend planted in the
    data the estimate recovers it approximately."""
    r = _rng(60)
    n = 500
    xy = r.random((n, 2))
    role = np.zeros(n, dtype=np.uint8)
    role[::5] = 1
    X = np.stack([np.ones(n), xy[:, 0], xy[:, 1]], 1)
    v = X @ np.array([2.0, -1.0, 0.5]) + 0.3 * r.standard_normal(n)
    lay = dict(kind="grid", nx=1, ny=1, delta=0.1, domain=(0.0, 1.0, 0.0, 1.0))
    param = (1.0, 0.1, 0.05)
    a = oracle.gls(xy, v, role, lay, X, param)
    b = oracle.gls_exact(xy, v, role, X, param)
    assert np.allclose(a, b, rtol=1e-9, atol=1e-9), (a, b)
    assert np.allclose(a, [2.0, -1.0, 0.5], atol=0.3)


def test_gls_invariants():
    """Pins of both GLS estimates (Sec. 5) by properties of the estimator, on a 3 x 3
    layout with shells: data in the column space of X (y = X beta0) give beta0 exactly,
    whatever M (the prediction operator H is linear, so each subset's normal-equation
    terms are consistent); as the nugget grows, H -> 0 and the estimate tends to
    ordinary least squares over the training points (a library least-squares solve)."""
    r = _rng(61)
    n = 450
    xy = r.random((n, 2))
    role = np.zeros(n, dtype=np.uint8)
    role[::4] = 1
    X = np.stack([np.ones(n), xy[:, 0], xy[:, 1] ** 2, np.sin(3 * xy[:, 0])], 1)
    lay = dict(kind="grid", nx=3, ny=3, delta=0.08, domain=(0.0, 1.0, 0.0, 1.0))
    beta0 = np.array([1.5, -2.0, 0.75, 0.3])
    y = X @ beta0
    for param in ((1.0, 0.1, 0.05), (2.0, 0.3, 0.001)):
        assert np.allclose(oracle.gls(xy, y, role, lay, X, param), beta0, rtol=0, atol=1e-9)
        assert np.allclose(oracle.gls_exact(xy, y, role, X, param), beta0, rtol=0, atol=1e-9)
    v = y + 0.5 * r.standard_normal(n)
    T = role == 0
    ols = np.linalg.lstsq(X[T], v[T], rcond=None)[0]
    for est in (oracle.gls(xy, v, role, lay, X, (1.0, 0.1, 1e9)), oracle.gls_exact(xy, v, role, X, (1.0, 0.1, 1e9))):
        assert np.allclose(est, ols, rtol=1e-6, atol=1e-8), (est, ols)
