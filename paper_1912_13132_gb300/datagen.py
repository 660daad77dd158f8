"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *generates inputs*: point locations, training/validation roles and
Gaussian-process realisations used as observed values.  It holds none of the
cross-validation method's arithmetic (no kriging system, no factorisation of a
subset matrix, no prediction, no loss).  Both the CUDA path and the CPU oracle
consume what it returns; neither shares any other code.

The paper's own data (the LiDAR canopy-height residuals of Sec. 4.1) are not
available, so every workload is a seeded stand-in with the same structure:

* Sec. 2.1 / Sec. 3: zero-mean GP with exponential covariance
  ``sigma2 * exp(-||s1 - s2|| / rho)`` observed with an additive nugget of
  variance ``tau2`` (the paper's ``tau``).
* Sec. 4.4: observations split at random into training, validation and test
  (role ``IGNORE``) data.

Roles: 0 = TRAIN, 1 = VALID, 2 = IGNORE (held-out test data, never used).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TRAIN, VALID, IGNORE = 0, 1, 2
BASE_SEED = 191213132


# ----------------------------------------------------------------------------
# point sets
# ----------------------------------------------------------------------------
def uniform_points(n: int, rng: np.random.Generator) -> np.ndarray:
    """n points uniform on the unit square, shape (n, 2) float64."""
    return rng.random((n, 2))


def poisson_cluster_points(n: int, rng: np.random.Generator, n_parents: int = 400,
                           sd: float = 0.02) -> np.ndarray:
    """Neyman-Scott (Thomas) cluster process on [0,1]^2.

    Parents are uniform; each child picks a parent uniformly and adds an isotropic
    N(0, sd^2) offset.  Children falling outside the unit square are redrawn.
    """
    parents = rng.random((n_parents, 2))
    out = np.empty((0, 2))
    while len(out) < n:
        need = n - len(out)
        pid = rng.integers(0, n_parents, size=2 * need + 16)
        cand = parents[pid] + sd * rng.standard_normal((len(pid), 2))
        ok = np.all((cand >= 0.0) & (cand <= 1.0), axis=1)
        out = np.concatenate([out, cand[ok][:need]])
    return out


def grid_nodes(side: int) -> np.ndarray:
    """Cell-centred nodes ((i + 1/2)/side, (j + 1/2)/side), i-major order, shape (side^2, 2)."""
    c = (np.arange(side, dtype=np.float64) + 0.5) / side
    gx, gy = np.meshgrid(c, c, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel()], axis=1)


# ----------------------------------------------------------------------------
# Gaussian-process realisations
# ----------------------------------------------------------------------------
def gp_dense(xy: np.ndarray, sigma2: float, rho: float, tau2: float,
             rng: np.random.Generator) -> np.ndarray:
    """Exact draw y ~ N(0, sigma2 * exp(-D/rho) + tau2 I) by a dense Cholesky factor.

    Only for a few thousand points (the covariance is held densely).
    """
    d = np.sqrt(((xy[:, None, :] - xy[None, :, :]) ** 2).sum(-1))
    c = sigma2 * np.exp(-d / rho)
    c[np.diag_indices_from(c)] += tau2
    f = np.linalg.cholesky(c)
    return f @ rng.standard_normal(len(xy))


@dataclass
class CirculantInfo:
    torus: int
    min_eig_ratio: float   # most negative eigenvalue / largest, before clipping


def gp_grid_circulant(side: int, sigma2: float, rho: float, rng: np.random.Generator,
                      info: list | None = None) -> np.ndarray:
    """Latent GP (no nugget) on the side x side cell-centred grid of [0,1]^2.

    Circulant embedding (Wood & Chan 1994; Dietrich & Newsam 1997): the grid is
    embedded in a torus of M >= 2*side nodes per axis, the covariance at torus lag
    (i, j) is sigma2 * exp(-h*sqrt(min(i,M-i)^2 + min(j,M-j)^2)/rho), its 2-D DFT
    gives the eigenvalues, negative eigenvalues (small, from the exponential
    kernel's truncation) are set to zero, and the real part of
    FFT2(sqrt(eig / M^2) * (Z1 + i Z2)) is one realisation.  Returns (side, side),
    index [i, j] = node ((i+1/2)/side, (j+1/2)/side).
    """
    import scipy.fft as sfft

    h = 1.0 / side
    m = sfft.next_fast_len(2 * side)
    lag = np.arange(m, dtype=np.float64)
    lag = np.minimum(lag, m - lag) * h
    dist = np.sqrt(lag[:, None] ** 2 + lag[None, :] ** 2)
    base = sigma2 * np.exp(-dist / rho)
    eig = sfft.fft2(base, workers=-1).real
    del base, dist
    lo = float(eig.min() / eig.max())
    np.maximum(eig, 0.0, out=eig)
    if info is not None:
        info.append(CirculantInfo(torus=m, min_eig_ratio=lo))
    amp = np.sqrt(eig / float(m * m))
    del eig
    z = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    z *= amp
    del amp
    y = sfft.fft2(z, workers=-1, overwrite_x=True)
    return np.ascontiguousarray(y.real[:side, :side])


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    """One dataset plus its subset layout and the parameter batch it is evaluated on."""
    name: str
    xy: np.ndarray            # (n, 2) float64
    v: np.ndarray             # (n,) float64 observed values
    role: np.ndarray          # (n,) uint8 TRAIN / VALID / IGNORE
    layout: dict              # {'kind': 'grid', 'nx', 'ny', 'delta', 'domain': (x0,x1,y0,y1)}
    params: np.ndarray        # (B, 3) float64 rows (sigma2, rho, tau2)
    meta: dict = field(default_factory=dict)


def log_grid(lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(np.linspace(math.log(lo), math.log(hi), n))


def uniform_split(n: int, rng: np.random.Generator, fr_train: float, fr_valid: float) -> np.ndarray:
    u = rng.random(n)
    role = np.full(n, IGNORE, dtype=np.uint8)
    role[u < fr_train + fr_valid] = VALID
    role[u < fr_train] = TRAIN
    return role


def make_uniform(n_train: int, n_valid: int, nx: int, delta: float, sigma2=1.0, rho=0.1,
                 tau2=0.05, seed=BASE_SEED + 1, name="uniform") -> Workload:
    """Uniform TRAIN and VALID draws on [0,1]^2, exact GP values by a dense factor."""
    rng = np.random.default_rng(seed)
    xy = uniform_points(n_train + n_valid, rng)
    v = gp_dense(xy, sigma2, rho, tau2, rng)
    role = np.zeros(len(xy), dtype=np.uint8)
    role[n_train:] = VALID
    return Workload(name, xy, v, role,
                    dict(kind="grid", nx=nx, ny=nx, delta=delta, domain=(0.0, 1.0, 0.0, 1.0)),
                    np.array([[sigma2, rho, tau2]]), dict(seed=seed))


def config_uniform_4096(seed=BASE_SEED + 1) -> Workload:
    """4096 TRAIN + 4096 VALID uniform points, GP(1, 0.1, 0.05) drawn jointly, 4x4 cores, delta 0.05.

    Roughly 250 validation and 370-500 training points per subset.
    """
    return make_uniform(4096, 4096, 4, 0.05, seed=seed, name="uniform-4096-4x4")


def config_cluster_262k(seed=BASE_SEED + 2, n_train=262144, n_valid=32768, fine=2048,
                        nx=32, delta=0.01) -> Workload:
    """Poisson-cluster locations, GP(1, 0.05, 0.02) by circulant embedding, 32x32 cores, delta 0.01.

    Parameter batch: 8 rho log-spaced in [0.025, 0.1] x 8 tau2 log-spaced in [0.01, 0.04]
    (the [x/2, 2x] grid rule of the simulation study, Sec. 3.1).
    """
    rng = np.random.default_rng(seed)
    xy = poisson_cluster_points(n_train + n_valid, rng)
    f = gp_grid_circulant(fine, 1.0, 0.05, rng)
    ij = np.clip((xy * fine).astype(np.int64), 0, fine - 1)
    v = f[ij[:, 0], ij[:, 1]] + math.sqrt(0.02) * rng.standard_normal(len(xy))
    role = np.zeros(len(xy), dtype=np.uint8)
    role[n_train:] = VALID
    rr, tt = np.meshgrid(log_grid(0.025, 0.1, 8), log_grid(0.01, 0.04, 8), indexing="ij")
    params = np.stack([np.ones(64), rr.ravel(), tt.ravel()], 1)
    return Workload(f"cluster-{n_train}-{nx}x{nx}", xy, v, role,
                    dict(kind="grid", nx=nx, ny=nx, delta=delta, domain=(0.0, 1.0, 0.0, 1.0)),
                    params, dict(seed=seed))


def config_grid_1m(rho=0.02, tau2=0.01, seed=None, fine=2048, cells=32, buf=8,
                   n_valid=131072) -> Workload:
    """Gridded precision-stress set: latent field on a fine 2048^2 grid, TRAIN on the 1024^2
    even-index sub-grid, VALID drawn without replacement from the other fine nodes.

    Cores are cells x cells training cells with a buf-cell shell (delta = buf / (fine/2)).
    """
    if seed is None:
        seed = BASE_SEED + 3 + int(round(1000 * rho)) + int(round(1e4 * tau2))
    rng = np.random.default_rng(seed)
    f = gp_grid_circulant(fine, 1.0, rho, rng)
    half = fine // 2
    ii, jj = np.meshgrid(np.arange(fine), np.arange(fine), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    even = (ii % 2 == 0) & (jj % 2 == 0)
    tr = np.nonzero(even)[0]
    rest = np.nonzero(~even)[0]
    va = np.sort(rng.choice(rest, size=n_valid, replace=False))
    sel = np.concatenate([tr, va])
    xy = np.stack([(ii[sel] + 0.5) / fine, (jj[sel] + 0.5) / fine], 1)
    v = f.ravel()[sel] + math.sqrt(tau2) * rng.standard_normal(len(sel))
    role = np.zeros(len(sel), dtype=np.uint8)
    role[len(tr):] = VALID
    nx = half // cells
    return Workload(f"grid-{half}sq-rho{rho}-tau{tau2}", xy, v, role,
                    dict(kind="grid", nx=nx, ny=nx, delta=buf / half, domain=(0.0, 1.0, 0.0, 1.0)),
                    np.array([[1.0, rho, tau2]]), dict(seed=seed))


def config_paper_5m(side=2236, nx=40, delta=0.001, seed=BASE_SEED + 5, missing=0.1) -> Workload:
    """Paper-scale stand-in: side^2 cell-centred grid (4,999,696 nodes for side 2236), a
    fraction `missing` of nodes dropped at random, GP(1, 0.05, 0.05) by circulant
    embedding, observed nodes split 80/10/10 into TRAIN / VALID / IGNORE (Sec. 4.4),
    nx x nx cores with shell width delta = 0.001 (Sec. 4.3.2).

    Parameter batch: sigma2 in {0.5, 1} x 10 rho log-spaced in [0.025, 0.1] x 10 tau2
    log-spaced in [0.025, 0.1] (200 configurations).
    """
    rng = np.random.default_rng(seed)
    f = gp_grid_circulant(side, 1.0, 0.05, rng)
    keep = rng.random(side * side) >= missing
    idx = np.nonzero(keep)[0]
    c = (np.arange(side, dtype=np.float64) + 0.5) / side
    xy = np.stack([c[idx // side], c[idx % side]], 1)
    v = f.ravel()[idx] + math.sqrt(0.05) * rng.standard_normal(len(idx))
    role = uniform_split(len(idx), rng, 0.8, 0.1)
    s2, rr, tt = np.meshgrid([0.5, 1.0], log_grid(0.025, 0.1, 10), log_grid(0.025, 0.1, 10),
                             indexing="ij")
    params = np.stack([s2.ravel(), rr.ravel(), tt.ravel()], 1)
    return Workload(f"paper-5m-{side}sq-{nx}x{nx}", xy, v, role,
                    dict(kind="grid", nx=nx, ny=nx, delta=delta, domain=(0.0, 1.0, 0.0, 1.0)),
                    params, dict(seed=seed, side=side))


def config_paper_5m_recursive(side=2236, q=9, delta=0.001, shell_cap=2000, seed=BASE_SEED + 5,
                              missing=0.0) -> Workload:
    """The paper's weak-scaling setting (Sec. 4.3.2) on the 5M-point field of
    config_paper_5m, all nodes observed (its 5M residuals, 80/10/10 split): 2^q = 512
    sub-domains by the recursive division of Sec. 2.4, shell width 0.001, shells with more
    than 2000 training points randomly thinned to 2000 (about 8.4k-8.7k training points
    per subset here; the paper's irregular LiDAR density gave 7.9k-10.5k)."""
    w = config_paper_5m(side=side, nx=40, delta=delta, seed=seed, missing=missing)
    w.layout = dict(kind="recursive", q=q, delta=delta, domain=(0.0, 1.0, 0.0, 1.0), shell_cap=shell_cap,
                    cap_seed=seed)
    w.name = f"paper-5m-{side}sq-recursive-q{q}-cap{shell_cap}"
    return w


SERVING_SIDES = (256, 320, 384, 512, 640, 768, 896, 1024)


def config_serving(sides=SERVING_SIDES, seed=BASE_SEED + 4) -> list:
    """Serving workload: one gridded dataset per side (65,536 to 1,048,576 TRAIN), each
    built like the precision-stress set (fine grid of twice the side, TRAIN on the even
    sub-grid, VALID = TRAIN/8 other fine nodes, 32-cell cores with 8-cell shells), with
    its own rho log-uniform in [0.02, 0.2] and tau2 log-uniform in [0.01, 0.1].
    """
    rng = np.random.default_rng(seed)
    out = []
    for i, side in enumerate(sides):
        rho = float(np.exp(rng.uniform(np.log(0.02), np.log(0.2))))
        tau2 = float(np.exp(rng.uniform(np.log(0.01), np.log(0.1))))
        w = config_grid_1m(rho=rho, tau2=tau2, seed=seed + 17 * (i + 1), fine=2 * side, cells=32, buf=8,
                           n_valid=side * side // 8)
        w.name = f"serve-grid-{side}sq-rho{rho:.3g}-tau{tau2:.3g}"
        out.append(w)
    return out
