"""The recursive division of Sec. 2.4 and the shell cap of Sec. 4.3.2 (CPU).

* the library's host layout builder and the oracle agree index for index
  (bit-exact membership, identical core rectangles) on uniform, clustered and
  tied coordinates, with and without shells and caps;
* pins of the oracle's division against what the paper and counting fix:
  - without shells and with distinct coordinates every sub-domain holds
    floor(n / 2^q) or ceil(n / 2^q) points (the paper's 512 shell-free subsets of
    Sec. 4.3.2 hold 9765 or 9766 of its residuals);
  - on a 2^a x 2^a grid of cell-centred nodes, q = 2a cuts without shells give the
    regular 2^a x 2^a layout;
  - every chosen cut minimises the imbalance over all candidates, recounted point
    by point (brute force);
* the cap keeps every core point, min(cap, |shell|) shell points, and the draw
  depends on the seed only.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1912_13132_gb300 import pcv


def _check_equal(xy, role, layout):
    To, Ti, Vo, Vi, cores = pcv.pcv_plan_create(xy, role, layout)
    ref = oracle.layout_cores(layout, xy)
    assert np.array_equal(cores, np.array([[c[0], c[1], c[3], c[4]] for c in ref]))
    mem = oracle.all_members(xy, role, layout)
    for i, (T, V) in enumerate(mem):
        assert np.array_equal(Ti[To[i]:To[i + 1]], T), i
        assert np.array_equal(Vi[Vo[i]:Vo[i + 1]], V), i
    return To, Ti, Vo, Vi, ref


def _roles(n, rng):
    return rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=n, p=[0.7, 0.2, 0.1])


@pytest.mark.parametrize("q,delta,cap", [(0, 0.0, 0), (1, 0.05, 0), (4, 0.0, 0), (4, 0.03, 0), (5, 0.08, 40),
                                         (6, 0.02, 25)])
def test_membership_uniform(q, delta, cap):
    rng = np.random.default_rng(10 * q + cap)
    xy = rng.random((3000, 2))
    lay = dict(kind="recursive", q=q, delta=delta, domain=(0.0, 1.0, 0.0, 1.0), shell_cap=cap, cap_seed=99)
    _check_equal(xy, _roles(len(xy), rng), lay)


@pytest.mark.parametrize("delta,cap", [(0.0, 0), (0.02, 0), (0.04, 60)])
def test_membership_clustered_and_tied(delta, cap):
    rng = np.random.default_rng(7)
    parents = rng.random((12, 2))
    xy = parents[rng.integers(0, 12, 2500)] + 0.03 * rng.standard_normal((2500, 2))
    xy = np.round(xy * 64) / 64            # many tied coordinates, points on cut candidates
    lay = dict(kind="recursive", q=5, delta=delta, shell_cap=cap, cap_seed=3)   # domain: bounding box
    _check_equal(xy, _roles(len(xy), rng), lay)


def test_cap_on_grid_layout_matches():
    rng = np.random.default_rng(11)
    xy = rng.random((4000, 2))
    lay = dict(kind="grid", nx=4, ny=3, delta=0.1, domain=(0.0, 1.0, 0.0, 1.0), shell_cap=120, cap_seed=5)
    _check_equal(xy, _roles(len(xy), rng), lay)


def test_balance_without_shells():
    rng = np.random.default_rng(2)
    n, q = 5000, 6
    xy = rng.random((n, 2))                # distinct coordinates
    role = _roles(n, rng)
    lay = dict(kind="recursive", q=q, delta=0.0, domain=(0.0, 1.0, 0.0, 1.0))
    cores = oracle.layout_cores(lay, xy)
    counts = []
    for x0, x1, xc, y0, y1, yc in cores:
        px, py = xy[:, 0], xy[:, 1]
        inside = (px >= x0) & ((px <= x1) if xc else (px < x1)) & (py >= y0) & ((py <= y1) if yc else (py < y1))
        counts.append(int(inside.sum()))
    assert sum(counts) == n
    assert set(counts) <= {n // 2 ** q, -(-n // 2 ** q)}, sorted(set(counts))


def test_grid_nodes_reproduce_regular_layout():
    a, side = 3, 48
    c = (np.arange(side) + 0.5) / side
    gx, gy = np.meshgrid(c, c, indexing="ij")
    xy = np.stack([gx.ravel(), gy.ravel()], 1)
    role = np.zeros(len(xy), dtype=np.uint8)
    role[::5] = 1
    rec = dict(kind="recursive", q=2 * a, delta=0.0, domain=(0.0, 1.0, 0.0, 1.0))
    reg = dict(kind="grid", nx=2 ** a, ny=2 ** a, delta=0.0, domain=(0.0, 1.0, 0.0, 1.0))
    m_rec = {tuple(T.tolist()) + (-1,) + tuple(V.tolist()) for T, V in oracle.all_members(xy, role, rec)}
    m_reg = {tuple(T.tolist()) + (-1,) + tuple(V.tolist()) for T, V in oracle.all_members(xy, role, reg)}
    assert m_rec == m_reg


def test_cuts_minimise_imbalance_brute_force():
    rng = np.random.default_rng(4)
    xy = np.round(rng.random((300, 2)) * 40) / 40
    d = 0.06
    lay = dict(kind="recursive", q=2, delta=d, domain=(0.0, 1.0, 0.0, 1.0))
    cores = oracle.recursive_cores(xy, lay)
    # depth first, left half first: cores 0, 1 split the left half in y, 2, 3 the right
    depth0 = cores[2][0]
    assert cores[0][1] == cores[1][1] == depth0 == cores[3][0]

    def window_count(x0, x1, y0, y1):
        return sum(1 for px, py in xy if x0 - d <= px <= x1 + d and y0 - d <= py <= y1 + d)

    xs = sorted({px for px, py in xy})
    cands = [(xs[m] + xs[m + 1]) / 2 for m in range(len(xs) - 1)]
    imb = [abs(window_count(0.0, s, 0.0, 1.0) - window_count(s, 1.0, 0.0, 1.0)) for s in cands]
    best = cands[int(np.argmin(imb))]       # first minimum: the smaller cut on ties
    assert depth0 == best


def test_cap_invariants():
    rng = np.random.default_rng(5)
    xy = rng.random((3000, 2))
    role = _roles(len(xy), rng)
    base = dict(kind="grid", nx=3, ny=3, delta=0.15, domain=(0.0, 1.0, 0.0, 1.0))
    capped = dict(base, shell_cap=50, cap_seed=1)
    other = dict(base, shell_cap=50, cap_seed=2)
    cores = oracle.layout_cores(base)
    diff = 0
    for i, (x0, x1, xc, y0, y1, yc) in enumerate(cores):
        T, V = oracle.subset_members(xy, role, base, i)
        Tc, Vc = oracle.subset_members(xy, role, capped, i)
        To, _ = oracle.subset_members(xy, role, other, i)
        px, py = xy[T, 0], xy[T, 1]
        core = T[(px >= x0) & ((px <= x1) if xc else (px < x1)) & (py >= y0) & ((py <= y1) if yc else (py < y1))]
        shell = np.setdiff1d(T, core)
        assert np.array_equal(V, Vc)
        assert np.all(np.diff(Tc) > 0) and set(Tc) <= set(T)
        assert set(core) <= set(Tc)
        assert len(Tc) == len(core) + min(50, len(shell))
        assert np.array_equal(Tc, oracle.subset_members(xy, role, capped, i)[0])   # same seed, same draw
        diff += not np.array_equal(Tc, To)
    assert diff > 0                          # another seed draws other points


def test_shell_key_is_splitmix64():
    """The shell cap's keys are outputs of the SplitMix64 generator (Steele, Lea and Flood,
    2014): seeded with 0, its first five outputs are the published sequence (the same as
    Java's SplittableRandom(0).nextLong()), and key (i, j) is output ((i << 40) | j) + 1."""
    published = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC,
                 0x1B39896A51A8749B]
    assert [oracle.shell_key(0, 0, j) for j in range(5)] == published
    # another subset index moves the stream by whole 2^40 blocks: key (1, 0) is output 2^40 + 1,
    # which a seed shifted by 2^40 increments reaches as its first output
    gamma = 0x9E3779B97F4A7C15
    assert oracle.shell_key(0, 1, 0) == oracle.shell_key((gamma << 40) & ((1 << 64) - 1), 0, 0)
    assert oracle.shell_key(7, 3, 5) != oracle.shell_key(7, 5, 3)
