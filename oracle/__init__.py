"""CPU oracle for parallel cross-validation (arXiv 1912.13132).  TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
and never imports it.  FP64 throughout.

Pieces and the passages they follow:

* ``grid_cores`` / ``subset_members``: the division of the domain D into
  disjoint rectangles D_1..D_N (Sec. 2.3) and, for each, its training data in
  D_i together with the shell D_i^shell of width delta (Sec. 2.3, Eq. 5-6),
  plus the validation data in D_i.  Readings the paper leaves open are fixed
  here (see ``grid_cores``): cores are half-open and closed on D's upper edges,
  the shell is the L-infinity band of width delta, only TRAIN points enter
  the training set.
* ``recursive_cores``: the recursive division of D into 2^q rectangles of
  Sec. 2.4 (each cut balances the data of both halves, each with its shell;
  the cut axis alternates, x first) -- readings in its docstring.
* ``shell_keys`` / the shell cap in ``subset_members``: shells holding more than
  a cap of training points keep a random sample of that size (Sec. 4.3.2),
  drawn with the SplitMix64 generator's published definition.
* ``krige`` / ``krige_literal``: simple kriging, Eq. 3 (C routine).
* ``sspe``: Eq. 4 (C routine).
* ``cv_loss``: Eq. 6, sum over subsets of the local SSPE (Algorithm 1's
  combine step), subsets without validation data contribute nothing
  (Sec. 4.3.1).
* ``neg2loglik``: Eq. 2 (C routine).
* ``gls`` / ``gls_exact``: the GLS mean of Sec. 5, beta = (X^T M^-1 X)^-1 X^T M^-1 y,
  with M^-1 v = (v - H v) / lambda and H v from the subsets' kriging (the
  parallel approximation), and the same estimate from a dense solve.

Parity of every function is pinned by ``tests/test_oracle_pins.py`` against
closed forms, exact rational solves, brute force and library routines that the
oracle itself does not use.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pcv_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

TRAIN, VALID, IGNORE = 0, 1, 2
OK, NOT_SPD = 0, 6


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no FMA contraction, no fast-math)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load(path: str):
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    L.oracle_select.restype = i64
    L.oracle_select.argtypes = [dp, ctypes.POINTER(ctypes.c_uint8), i64, ctypes.c_int,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                ctypes.POINTER(i64)]
    L.oracle_cholesky.restype = ctypes.c_int
    L.oracle_cholesky.argtypes = [dp, i64]
    L.oracle_forward.restype = None
    L.oracle_forward.argtypes = [dp, i64, dp]
    L.oracle_backward.restype = None
    L.oracle_backward.argtypes = [dp, i64, dp]
    L.oracle_krige.restype = ctypes.c_int
    L.oracle_krige.argtypes = [dp, dp, i64, dp, i64, ctypes.c_double, ctypes.c_double, dp]
    L.oracle_krige_literal.restype = ctypes.c_int
    L.oracle_krige_literal.argtypes = [dp, dp, i64, dp, i64, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, dp]
    L.oracle_sspe.restype = ctypes.c_double
    L.oracle_sspe.argtypes = [dp, dp, i64]
    L.oracle_neg2loglik.restype = ctypes.c_int
    L.oracle_neg2loglik.argtypes = [dp, dp, i64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, dp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Temporarily route every oracle call through another build of pcv_oracle.c
    (used by the tests that plant mistakes in a copy of the oracle)."""
    global _lib
    old = lib()
    _lib = _load(path)
    try:
        yield
    finally:
        _lib = old


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# linear algebra pieces (exposed for the pins)
# ----------------------------------------------------------------------------
def cholesky(a: np.ndarray) -> tuple[np.ndarray, int]:
    """Lower Cholesky factor of a (copy); returns (L, status)."""
    w = _f64(a).copy()
    k = w.shape[0]
    st = lib().oracle_cholesky(_dp(w), k)
    return np.tril(w), st


def solve_spd(a: np.ndarray, b: np.ndarray) -> tuple[np.ndarray, int]:
    """x = a^{-1} b by the oracle's Cholesky, forward and back substitution."""
    w = _f64(a).copy()
    k = w.shape[0]
    st = lib().oracle_cholesky(_dp(w), k)
    x = _f64(b).copy()
    if st == OK:
        lib().oracle_forward(_dp(w), k, _dp(x))
        lib().oracle_backward(_dp(w), k, _dp(x))
    return x, st


def krige(sT, yT, sP, rho: float, lam: float) -> tuple[np.ndarray, int]:
    """Eq. 3, second line: yhat = Sigma_p^T (Sigma + lam I)^{-1} yT."""
    sT, yT, sP = _f64(sT).reshape(-1, 2), _f64(yT), _f64(sP).reshape(-1, 2)
    out = np.empty(len(sP))
    st = lib().oracle_krige(_dp(sT), _dp(yT), len(sT), _dp(sP), len(sP), rho, lam, _dp(out))
    return out, st


def krige_lapack(sT, yT, sP, rho: float, lam: float) -> tuple[np.ndarray, int]:
    """Eq. 3, second line, with library routines for the two large steps: LAPACK's
    Cholesky factorisation and triangular solves (scipy.linalg), the covariances
    written out with numpy.  For subsets too large for the plain C routine (k of
    several thousand); pinned against it in tests/test_oracle_pins.py."""
    import scipy.linalg as sla
    sT, yT, sP = _f64(sT).reshape(-1, 2), _f64(yT), _f64(sP).reshape(-1, 2)
    if len(sT) == 0:
        return np.zeros(len(sP)), OK
    dT = np.sqrt((sT[:, None, 0] - sT[None, :, 0]) ** 2 + (sT[:, None, 1] - sT[None, :, 1]) ** 2)
    A = np.exp(-dT / rho)
    A[np.diag_indices_from(A)] += lam
    try:
        L = np.linalg.cholesky(A)
    except np.linalg.LinAlgError:
        return np.full(len(sP), np.nan), NOT_SPD
    w = sla.solve_triangular(L, yT, lower=True)
    alpha = sla.solve_triangular(L.T, w, lower=False)
    dP = np.sqrt((sP[:, None, 0] - sT[None, :, 0]) ** 2 + (sP[:, None, 1] - sT[None, :, 1]) ** 2)
    return np.exp(-dP / rho) @ alpha, OK


def krige_literal(sT, yT, sP, sigma2: float, rho: float, tau: float) -> tuple[np.ndarray, int]:
    """Eq. 3, first line: sigma2 Sigma_p^T (sigma2 Sigma + tau I)^{-1} yT."""
    sT, yT, sP = _f64(sT).reshape(-1, 2), _f64(yT), _f64(sP).reshape(-1, 2)
    out = np.empty(len(sP))
    st = lib().oracle_krige_literal(_dp(sT), _dp(yT), len(sT), _dp(sP), len(sP), sigma2, rho,
                                    tau, _dp(out))
    return out, st


def sspe(yhat, yV) -> float:
    """Eq. 4."""
    yhat, yV = _f64(yhat), _f64(yV)
    return lib().oracle_sspe(_dp(yhat), _dp(yV), len(yV))


def neg2loglik(sT, yT, sigma2: float, rho: float, tau: float) -> tuple[float, int]:
    """Eq. 2 on one set of observations."""
    sT, yT = _f64(sT).reshape(-1, 2), _f64(yT)
    out = np.empty(1)
    st = lib().oracle_neg2loglik(_dp(sT), _dp(yT), len(sT), sigma2, rho, tau, _dp(out))
    return float(out[0]), st


# ----------------------------------------------------------------------------
# layout: cores, shells, membership (Sec. 2.3)
# ----------------------------------------------------------------------------
def grid_bounds(lo: float, hi: float, n: int) -> list[float]:
    """Cut points of an n-cell regular division of [lo, hi]:
    b[0] = lo, b[n] = hi, b[c] = lo + ((hi - lo) * c) / n evaluated in FP64 in that order."""
    b = [lo + ((hi - lo) * c) / n for c in range(n + 1)]
    b[0], b[n] = lo, hi
    return b


def grid_cores(layout: dict) -> list[tuple[float, float, bool, float, float, bool]]:
    """Cores of a regular nx x ny layout, subset i = cy * nx + cx.

    Each core is (x0, x1, x1_closed, y0, y1, y1_closed): the half-open rectangle
    [x0, x1) x [y0, y1), closed on the domain's upper edges so that every point of
    D lies in exactly one core (the paper's D_i are disjoint, Sec. 2.3).
    """
    X0, X1, Y0, Y1 = layout["domain"]
    nx, ny = layout["nx"], layout["ny"]
    bx, by = grid_bounds(X0, X1, nx), grid_bounds(Y0, Y1, ny)
    out = []
    for cy in range(ny):
        for cx in range(nx):
            out.append((bx[cx], bx[cx + 1], cx == nx - 1, by[cy], by[cy + 1], cy == ny - 1))
    return out


def domain_of(layout: dict, xy=None) -> tuple[float, float, float, float]:
    """D: the layout's domain, else the bounding box of all points."""
    if layout.get("domain") is not None:
        return tuple(float(t) for t in layout["domain"])
    xy = _f64(xy)
    return (float(xy[:, 0].min()), float(xy[:, 0].max()), float(xy[:, 1].min()), float(xy[:, 1].max()))


def recursive_cores(xy, layout: dict) -> list[tuple[float, float, float, float]]:
    """The recursive division of D into 2^q sub-domains (Sec. 2.4).

    A rectangle is cut in two so that both halves, each together with its shell,
    contain a similar amount of data; the cuts alternate between the two axes.
    Readings where the section leaves details open:
      * the first cut (depth 0) is a value of x (a line parallel to the y-axis),
        then y, then x, ...;
      * "amount of data" counts every point, whatever its role, in the child's
        closed window [x0 - delta, x1 + delta] x [y0 - delta, y1 + delta] (the
        shell reaches wherever it reaches; the 512 shell-free subsets of Sec. 4.3.2
        hold 9765 or 9766 residuals each, so all data are balanced);
      * candidate cuts are the midpoints of consecutive distinct coordinates of the
        points inside the parent (half-open, closed on D's upper edges); the cut
        with the smallest |count(left) - count(right)| wins, ties going to the
        smaller cut; with fewer than two distinct coordinates the parent is cut in
        the middle;
      * the sub-domains are numbered depth first, the left (lower) half first.
    Returns [(x0, x1, y0, y1)] in that order.
    """
    xy = _f64(xy)
    X0, X1, Y0, Y1 = domain_of(layout, xy)
    d = float(layout["delta"])
    q = int(layout["q"])
    x, y = xy[:, 0], xy[:, 1]
    out = []

    def in_window(idx, r):
        px, py = x[idx], y[idx]
        return idx[(px >= r[0] - d) & (px <= r[1] + d) & (py >= r[2] - d) & (py <= r[3] + d)]

    def in_rect(idx, r):
        px, py = x[idx], y[idx]
        okx = (px >= r[0]) & ((px <= r[1]) if r[1] == X1 else (px < r[1]))
        oky = (py >= r[2]) & ((py <= r[3]) if r[3] == Y1 else (py < r[3]))
        return idx[okx & oky]

    def divide(r, depth, win):
        if depth == q:
            out.append(r)
            return
        coord = x if depth % 2 == 0 else y
        lo, hi = (r[0], r[1]) if depth % 2 == 0 else (r[2], r[3])
        u = np.unique(coord[in_rect(win, r)])
        cut = (lo + hi) / 2.0
        if len(u) >= 2:
            a = np.sort(coord[win])                      # every point in the parent's window
            cand = (u[:-1] + u[1:]) / 2.0
            left = np.searchsorted(a, cand + d, side="right")       # left child's window
            right = len(a) - np.searchsorted(a, cand - d, side="left")  # right child's window
            cut = float(cand[int(np.argmin(np.abs(left - right)))])    # first minimum = smaller cut
        if depth % 2 == 0:
            halves = ((r[0], cut, r[2], r[3]), (cut, r[1], r[2], r[3]))
        else:
            halves = ((r[0], r[1], r[2], cut), (r[0], r[1], cut, r[3]))
        for h in halves:
            divide(h, depth + 1, in_window(win, h))

    root = (X0, X1, Y0, Y1)
    divide(root, 0, in_window(np.arange(len(xy)), root))
    return out


def layout_cores(layout: dict, xy=None) -> list[tuple[float, float, bool, float, float, bool]]:
    """Cores as (x0, x1, x1_closed, y0, y1, y1_closed); recursive layouts need the points."""
    if layout["kind"] == "grid":
        return grid_cores(layout)
    if layout["kind"] in ("rects", "recursive"):
        X0, X1, Y0, Y1 = domain_of(layout, xy)
        rects = layout["cores"] if layout["kind"] == "rects" else recursive_cores(xy, layout)
        return [(r[0], r[1], r[1] == X1, r[2], r[3], r[3] == Y1) for r in rects]
    raise ValueError(f"unknown layout kind {layout['kind']}")


_M64 = (1 << 64) - 1


def shell_key(seed: int, i: int, j: int) -> int:
    """Key of shell point j of subset i: output number w + 1, w = (i << 40) | j, of the
    SplitMix64 generator seeded with `seed` (Steele, Lea and Flood, OOPSLA 2014):
    the generator adds its golden-ratio increment per output and mixes the sum."""
    z = (seed + (((i << 40) | j) + 1) * 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def subset_members(xy: np.ndarray, role: np.ndarray, layout: dict, i: int,
                   cores=None) -> tuple[np.ndarray, np.ndarray]:
    """(T_i, V_i) as ascending index arrays.

    V_i: VALID points in core i.  T_i: TRAIN points in core i together with its
    shell, i.e. in the closed window [x0 - delta, x1 + delta] x [y0 - delta, y1 + delta]
    (the shell of width delta around D_i, Sec. 2.3; only training data enter it).
    """
    L = lib()
    xy = _f64(xy)
    role = np.ascontiguousarray(role, dtype=np.uint8)
    rp = role.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    if cores is None:
        cores = layout_cores(layout, xy)
    x0, x1, xc, y0, y1, yc = cores[i]
    d = float(layout["delta"])
    n = len(role)
    out = []
    for want, rect in ((TRAIN, (x0 - d, x1 + d, True, y0 - d, y1 + d, True)),
                       (VALID, (x0, x1, xc, y0, y1, yc))):
        cnt = L.oracle_select(_dp(xy), rp, n, want, rect[0], rect[1], int(rect[2]), rect[3],
                              rect[4], int(rect[5]), None)
        idx = np.empty(cnt, dtype=np.int64)
        L.oracle_select(_dp(xy), rp, n, want, rect[0], rect[1], int(rect[2]), rect[3], rect[4],
                        int(rect[5]), idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        out.append(idx)
    cap = int(layout.get("shell_cap", 0) or 0)
    if cap > 0:
        # Sec. 4.3.2: a shell with more than `cap` training points keeps a random
        # sample of `cap` of them (without replacement); the core keeps all of its own
        T = out[0]
        px, py = xy[T, 0], xy[T, 1]
        in_core = ((px >= x0) & ((px <= x1) if xc else (px < x1)) &
                   (py >= y0) & ((py <= y1) if yc else (py < y1)))
        shell = T[~in_core]
        if len(shell) > cap:
            seed = int(layout.get("cap_seed", 0)) & _M64
            ranked = sorted(shell.tolist(), key=lambda j: (shell_key(seed, i, j), j))
            out[0] = np.sort(np.concatenate([T[in_core], np.array(ranked[:cap], dtype=np.int64)]))
    return out[0], out[1]


def all_members(xy, role, layout, threads: int | None = None):
    cores = layout_cores(layout, xy)
    with ThreadPoolExecutor(threads or os.cpu_count()) as ex:
        return list(ex.map(lambda i: subset_members(xy, role, layout, i, cores), range(len(cores))))


# ----------------------------------------------------------------------------
# the method: local SSPE per subset and their sum (Eq. 6, Algorithm 1)
# ----------------------------------------------------------------------------
def subset_cv(xy, v, T: np.ndarray, V: np.ndarray, sigma2: float, rho: float, tau: float,
              lapack: bool = False):
    """Local SSPE z_i = CV(y~_T^i, y_V^i, zeta) with zeta = (tau / sigma2, rho).

    Returns (z, yhat_V, status).  A subset with no validation data returns z = 0
    and is ignored (Sec. 4.3.1).  `lapack` selects krige_lapack for large subsets.
    """
    if len(V) == 0:
        return 0.0, np.empty(0), OK
    yhat, st = (krige_lapack if lapack else krige)(xy[T], v[T], xy[V], rho, tau / sigma2)
    if st != OK:
        return float("nan"), yhat, st
    return sspe(yhat, v[V]), yhat, st


def cv_loss(xy, v, role, layout, params, members=None, subsets=None, threads: int | None = None,
            lapack: bool = False):
    """Parallel-CV loss for each parameter row (sigma2, rho, tau).

    Returns dict with 'sspe' (B,), 'z' (B, N) local SSPEs (NaN where not evaluated),
    'status' (B, N), 'n_valid' and, per evaluated (b, i), the predictions in 'yhat'.
    The combine step sums z_i in subset order 0..N-1 (Eq. 6).
    """
    xy, v = _f64(xy), _f64(v)
    params = np.atleast_2d(_f64(params))
    cores = layout_cores(layout, xy)
    N = len(cores)
    if members is None:
        members = all_members(xy, role, layout, threads)
    idx = list(range(N)) if subsets is None else list(subsets)
    B = len(params)
    z = np.full((B, N), np.nan)
    status = np.zeros((B, N), dtype=np.int32)
    yhat = {}
    jobs = [(b, i) for b in range(B) for i in idx]

    def run(job):
        b, i = job
        T, V = members[i]
        s2, rho, tau = params[b]
        return job, subset_cv(xy, v, T, V, s2, rho, tau, lapack)

    with ThreadPoolExecutor(threads or os.cpu_count()) as ex:
        for (b, i), (zi, yh, st) in ex.map(run, jobs):
            z[b, i] = zi
            status[b, i] = st
            yhat[(b, i)] = yh
    total = np.zeros(B)
    for b in range(B):
        s = 0.0
        for i in idx:
            s += z[b, i]
        total[b] = s
    n_valid = sum(len(members[i][1]) for i in idx)
    return dict(sspe=total, z=z, status=status, yhat=yhat, n_valid=n_valid, members=members)


def core_of(layout: dict, pts: np.ndarray, xy=None) -> np.ndarray:
    """Index of the core containing each point of pts (m, 2), after clamping the point
    into D (points outside D go to the nearest core).  Layouts other than the
    regular grid take the first core that contains the clamped point, else the
    nearest one (recursive layouts need the data points `xy`)."""
    if layout["kind"] != "grid":
        pts = _f64(pts).reshape(-1, 2)
        X0, X1, Y0, Y1 = domain_of(layout, xy)
        cores = layout_cores(layout, xy)
        out = np.empty(len(pts), dtype=np.int64)
        for j, (px, py) in enumerate(pts):
            px, py = min(max(px, X0), X1), min(max(py, Y0), Y1)
            best, bestd = -1, np.inf
            for i, (x0, x1, xc, y0, y1, yc) in enumerate(cores):
                if px >= x0 and (px <= x1 if xc else px < x1) and py >= y0 and (py <= y1 if yc else py < y1):
                    best = i
                    break
                dx, dy = max(x0 - px, 0.0, px - x1), max(y0 - py, 0.0, py - y1)
                if dx * dx + dy * dy < bestd:
                    best, bestd = i, dx * dx + dy * dy
            out[j] = best
        return out
    X0, X1, Y0, Y1 = layout["domain"]
    nx, ny = layout["nx"], layout["ny"]
    bx, by = np.array(grid_bounds(X0, X1, nx)), np.array(grid_bounds(Y0, Y1, ny))
    x = np.clip(pts[:, 0], X0, X1)
    y = np.clip(pts[:, 1], Y0, Y1)
    cx = np.clip(np.searchsorted(bx, x, side="right") - 1, 0, nx - 1)
    cy = np.clip(np.searchsorted(by, y, side="right") - 1, 0, ny - 1)
    return cy * nx + cx


def predict(xy, v, role, layout, param, pts, members=None):
    """Kriging prediction at new locations: each point uses the training data of the
    subset (core plus shell) whose core contains it, with the given (sigma2, rho, tau)."""
    xy, v, pts = _f64(xy), _f64(v), _f64(pts).reshape(-1, 2)
    s2, rho, tau = [float(t) for t in param]
    core = core_of(layout, pts, xy)
    cores = layout_cores(layout, xy)
    out = np.empty(len(pts))
    for i in np.unique(core):
        sel = np.nonzero(core == i)[0]
        T = members[i][0] if members is not None else subset_members(xy, role, layout, int(i), cores)[0]
        yh, st = krige(xy[T], v[T], pts[sel], rho, tau / s2)
        out[sel] = yh
    return out


# ----------------------------------------------------------------------------
# GLS mean component (Sec. 5)
# ----------------------------------------------------------------------------
def gls(xy, v, role, layout, X, param, lapack: bool = False) -> np.ndarray:
    """beta = (X^T M^-1 X)^-1 X^T M^-1 y over the TRAIN points, M = Sigma + lambda I.

    Sec. 5: M^-1 = (I - H) / lambda with H = Sigma (Sigma + lambda I)^-1 the kriging
    operator at the observed locations, so M^-1 v is found by predicting v.  Parallel
    approximation: H v at a training point is the kriging prediction from the training
    data of the subset whose core holds the point (Eq. 3 applied to the column v).
    The 1 / lambda cancels.  The sums run over the points subset by subset."""
    xy, v = _f64(xy), _f64(v)
    X = _f64(X).reshape(len(v), -1)
    s2, rho, tau = [float(t) for t in param]
    lam = tau / s2
    cores = layout_cores(layout, xy)
    p = X.shape[1]
    A = np.zeros((p, p))
    b = np.zeros(p)
    kr = krige_lapack if lapack else krige
    for i, (x0, x1, xc, y0, y1, yc) in enumerate(cores):
        T, _ = subset_members(xy, role, layout, i, cores)
        px, py = xy[T, 0], xy[T, 1]
        C = T[(px >= x0) & ((px <= x1) if xc else (px < x1)) & (py >= y0) & ((py <= y1) if yc else (py < y1))]
        if len(C) == 0:
            continue
        HX = np.stack([kr(xy[T], X[T, c], xy[C], rho, lam)[0] for c in range(p)], 1)
        Hy, _ = kr(xy[T], v[T], xy[C], rho, lam)
        A += X[C].T @ (X[C] - HX)
        b += X[C].T @ (v[C] - Hy)
    return np.linalg.solve(A, b)


def gls_exact(xy, v, role, X, param) -> np.ndarray:
    """The same estimate with M = Sigma + lambda I over all TRAIN points, by dense solves."""
    xy, v = _f64(xy), _f64(v)
    X = _f64(X).reshape(len(v), -1)
    s2, rho, tau = [float(t) for t in param]
    T = np.nonzero(np.asarray(role) == TRAIN)[0]
    d = np.sqrt(((xy[T, None, :] - xy[None, T, :]) ** 2).sum(-1))
    M = np.exp(-d / rho) + (tau / s2) * np.eye(len(T))
    MiX = np.linalg.solve(M, X[T])
    Miy = np.linalg.solve(M, v[T])
    return np.linalg.solve(X[T].T @ MiX, X[T].T @ Miy)
