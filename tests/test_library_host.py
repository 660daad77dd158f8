"""Host-side checks of the CUDA library (no GPU needed).

* the shared library loads and exports every function include/pcv.h declares;
* the library's subset membership (host layout builder) equals the oracle's,
  index for index (bit-exact), on the tiny hand-derived fixture, on points that
  sit exactly on cut lines and window edges, and on the shapes of the paper-like
  workloads;
* invalid input is rejected with PCV_ERR_ARG.
"""
from __future__ import annotations

import json
import os
import re

import numpy as np
import pytest

import oracle
from paper_1912_13132_gb300 import datagen, pcv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_exports_match_header():
    hdr = open(os.path.join(ROOT, "include", "pcv.h")).read()
    declared = set(re.findall(r"\b(pcv_[a-z0-9_]+)\s*\(", hdr))
    assert declared == set(pcv.EXPORTS), declared ^ set(pcv.EXPORTS)
    lib = pcv.load_library(pcv.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name)


def _compare_members(xy, role, layout):
    To, Ti, Vo, Vi, cores = pcv.pcv_plan_create(xy, role, layout)
    mem = oracle.all_members(xy, role, layout)
    assert len(mem) == len(To) - 1
    for i, (T, V) in enumerate(mem):
        assert np.array_equal(Ti[To[i]:To[i + 1]], T), i
        assert np.array_equal(Vi[Vo[i]:Vo[i + 1]], V), i
    ref_cores = oracle.layout_cores(layout, xy)
    assert np.array_equal(cores, np.array([[c[0], c[1], c[3], c[4]] for c in ref_cores]))
    return To, Vo


def test_membership_fixture():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "layout_tiny.json")))
    pts = np.array(g["points"])
    lay = dict(kind="grid", nx=2, ny=2, delta=g["delta"], domain=tuple(g["domain"]))
    To, Ti, Vo, Vi, _ = pcv.pcv_plan_create(pts[:, :2], pts[:, 2].astype(np.uint8), lay)
    for i in range(4):
        assert Ti[To[i]:To[i + 1]].tolist() == g["T"][i]
        assert Vi[Vo[i]:Vo[i + 1]].tolist() == g["V"][i]


@pytest.mark.parametrize("nx,ny,delta", [(1, 1, 0.0), (3, 2, 0.0), (5, 5, 0.03), (7, 4, 0.2), (4, 4, 2.0)])
def test_membership_edges(nx, ny, delta):
    r = np.random.default_rng(nx * 100 + ny)
    xy = r.random((4000, 2))
    # points on cut lines, on window edges and on D's boundary
    b = np.array(oracle.grid_bounds(0.0, 1.0, nx))
    xy[:40, 0] = r.choice(np.concatenate([b, b - delta, b + delta]), 40)
    xy[40:80, 1] = r.choice(np.concatenate([b, b - delta, b + delta]), 40)
    xy[80:90] = 1.0
    xy[90:100] = 0.0
    xy[100:110] = [1.2, 0.5]           # outside D (inside a window when delta is large)
    role = r.integers(0, 3, len(xy)).astype(np.uint8)
    _compare_members(xy, role, dict(kind="grid", nx=nx, ny=ny, delta=delta, domain=(0.0, 1.0, 0.0, 1.0)))


def test_membership_default_domain_and_rects():
    r = np.random.default_rng(5)
    xy = r.random((1500, 2)) * [3.0, 2.0] - [1.0, 0.5]
    role = r.integers(0, 3, len(xy)).astype(np.uint8)
    lo, hi = xy.min(0), xy.max(0)
    lay = dict(kind="grid", nx=3, ny=3, delta=0.1, domain=None)
    To, Ti, Vo, Vi, cores = pcv.pcv_plan_create(xy, role, lay)
    lay_explicit = dict(lay, domain=(lo[0], hi[0], lo[1], hi[1]))
    _compare_members(xy, role, lay_explicit)
    rects = [(-1.0, 0.2, -0.5, 0.4), (0.2, 2.0, -0.5, 0.4), (-1.0, 2.0, 0.4, 1.5)]
    lay_r = dict(kind="rects", cores=rects, delta=0.05, domain=(-1.0, 2.0, -0.5, 1.5))
    _compare_members(xy, role, lay_r)


def test_membership_workload_shapes():
    w = datagen.config_uniform_4096()
    To, Vo = _compare_members(w.xy, w.role, w.layout)
    k = np.diff(To)
    assert 300 < k.min() and k.max() < 600 and 200 < np.diff(Vo).mean() < 300
    r = np.random.default_rng(3)
    xy = datagen.poisson_cluster_points(60000, r)
    role = (r.random(60000) < 0.1).astype(np.uint8)
    _compare_members(xy, role, dict(kind="grid", nx=16, ny=16, delta=0.01, domain=(0.0, 1.0, 0.0, 1.0)))


def test_membership_grid_counts():
    """Gridded training data with cell-sized shells give the designed subset sizes."""
    side = 256
    nodes = datagen.grid_nodes(side)
    role = np.zeros(len(nodes), dtype=np.uint8)
    lay = dict(kind="grid", nx=8, ny=8, delta=8 / side, domain=(0.0, 1.0, 0.0, 1.0))
    To, Vo = _compare_members(nodes, role, lay)
    k = np.diff(To).reshape(8, 8)
    assert k[0, 0] == 40 * 40 and k[3, 3] == 48 * 48 and k[0, 3] == 40 * 48


@pytest.mark.parametrize("case", ["bad-role", "nan", "neg-delta", "nx0", "inverted-domain"])
def test_invalid_input(case):
    xy = np.array([[0.1, 0.2], [0.5, 0.5]])
    role = np.array([0, 1], dtype=np.uint8)
    lay = dict(kind="grid", nx=2, ny=2, delta=0.1, domain=(0.0, 1.0, 0.0, 1.0))
    if case == "bad-role":
        role = np.array([0, 7], dtype=np.uint8)
    elif case == "nan":
        xy = xy.copy()
        xy[1, 0] = np.nan
    elif case == "neg-delta":
        lay["delta"] = -0.1
    elif case == "nx0":
        lay["nx"] = 0
    elif case == "inverted-domain":
        lay["domain"] = (1.0, 0.0, 0.0, 1.0)
    with pytest.raises(pcv.PcvError) as e:
        pcv.pcv_plan_create(xy, role, lay)
    assert e.value.status == pcv.PCV_ERR_ARG


def test_lattice_detect():
    """Host-side lattice test (the rule pcv_create applies to choose the table path):
    gridded workloads pass with their spacing; a column shifted by 1e-9 of the spacing,
    scattered points and non-finite input do not; a one-ulp change of a whole column (a
    rounding-level deviation) still passes; degenerate axes count as spacing 1."""
    w = datagen.config_paper_5m(side=560, nx=10, delta=0.001 * 2236 / 560)
    got = pcv.pcv_lattice_detect(w.xy)
    assert got is not None
    (x0, hx), (y0, hy) = got
    assert x0 == w.xy[:, 0].min() and y0 == w.xy[:, 1].min()
    assert abs(hx * 560 - 1) < 1e-14 and abs(hy * 560 - 1) < 1e-14
    xs = np.unique(w.xy[:, 0])
    col = w.xy[:, 0] == xs[200]
    for shift, ok in [(1e-9 * hx, False), (1e-6 * hx, False)]:
        xy = w.xy.copy()
        xy[col, 0] += shift
        assert (pcv.pcv_lattice_detect(xy) is not None) == ok, shift
    xy = w.xy.copy()
    xy[col, 0] = np.nextafter(xy[col, 0], 2.0)
    assert pcv.pcv_lattice_detect(xy) is not None
    # large offsets (projected coordinates in metres, 1 m spacing)
    g = np.stack(np.meshgrid(5.0e5 + np.arange(40.0), 4.2e6 + np.arange(30.0), indexing="ij"), -1).reshape(-1, 2)
    (gx0, ghx), (gy0, ghy) = pcv.pcv_lattice_detect(g)
    assert (gx0, ghx, gy0, ghy) == (5.0e5, 1.0, 4.2e6, 1.0)
    # spacing that is not a binary fraction, with missing nodes
    g2 = np.stack(np.meshgrid(np.arange(50) * 0.1, np.arange(7) * 0.3, indexing="ij"), -1).reshape(-1, 2)
    g2 = g2[np.random.default_rng(3).random(len(g2)) < 0.7]
    (_, h2x), (_, h2y) = pcv.pcv_lattice_detect(g2)
    assert abs(h2x - 0.1) < 1e-15 and abs(h2y - 0.3) < 1e-15
    assert pcv.pcv_lattice_detect(np.random.default_rng(1).random((500, 2))) is None
    assert pcv.pcv_lattice_detect(np.array([[0.25, 0.5]])) == ((0.25, 1.0), (0.5, 1.0))
    assert pcv.pcv_lattice_detect(np.array([[0.0, 0.0], [0.0, 0.5], [0.0, 1.5]])) == ((0.0, 1.0), (0.0, 0.5))
    assert pcv.pcv_lattice_detect(np.array([[0.0, 0.0], [np.nan, 0.5]])) is None
    assert pcv.pcv_lattice_detect(np.zeros((0, 2))) is None


def test_null_handles_rejected():
    """Every entry point that takes a context, plan or server handle rejects NULL with
    PCV_ERR_ARG before touching the device (the header's error behaviour); destroy calls
    accept NULL; status strings exist for every status."""
    lib = pcv.load_library(pcv.LIB_PATH)
    E = pcv.PCV_ERR_ARG
    calls = {
        "pcv_plan_info": (None, None, None, None, None, None),
        "pcv_plan_cores": (None, None),
        "pcv_subset_info": (None, None, None, None, None, None),
        "pcv_cv_loss": (None, None, 1, 1, None, None, None, None, None, None),
        "pcv_cv_loss_device": (None, None, 1, 1, None, None, None, None, None),
        "pcv_neg2loglik": (None, None, 1, 1, None, None, None, None),
        "pcv_predict": (None, None, None, 0, 1, None, None),
        "pcv_predict_local": (None, None, 1, None, None, 0, 1, None, None, None),
        "pcv_gls": (None, None, 1, None, 1, None, None),
        "pcv_set_timing": (None, 1),
        "pcv_kernel_time": (None, None, None),
        "pcv_phase_cycles": (None, None, 0),
        "pcv_server_create": (None, 0, None, None),
        "pcv_server_submit_cv": (None, 0, None, None),
        "pcv_server_submit_predict": (None, 0, None, None, 0, None),
        "pcv_server_wait": (None, 0, 0.0, None, None, None, None),
        "pcv_server_stats": (None, None, None, None, None, None, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == E, name
    assert lib.pcv_lattice(None, None, None) == 0
    lib.pcv_destroy(None)
    lib.pcv_plan_destroy(None)
    lib.pcv_server_destroy(None)
    assert lib.pcv_cv_loss(None, None, 1, 1, None, None, None, None, None, None) == E
    assert b"NULL" in lib.pcv_last_error()
    for st in range(9):
        assert lib.pcv_status_str(st)
