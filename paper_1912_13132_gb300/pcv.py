"""Python binding of the C ABI in include/pcv.h (argument marshalling only).

Every step of the hot path runs in the CUDA library ``_lib/libpcv.so``; this
module converts numpy arrays / torch tensors to pointers and status codes to
exceptions.  It never computes anything itself and it has no fallback: if the
library is missing or cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build_ext

PCV_OK, PCV_ERR_ARG, PCV_ERR_OOM, PCV_ERR_CUDA, PCV_ERR_TIMEOUT = 0, 1, 2, 3, 4
PCV_ERR_BUSY, PCV_NOT_SPD, PCV_REFINE_FALLBACK, PCV_ERR_UNSUPPORTED = 5, 6, 7, 8
PCV_PREC_FP64, PCV_PREC_MIXED = 0, 1
PCV_LAYOUT_RECTS, PCV_LAYOUT_GRID, PCV_LAYOUT_RECURSIVE = 0, 1, 2
PRECISIONS = {"fp64": PCV_PREC_FP64, "mixed": PCV_PREC_MIXED, "mixed-tf32": 2, "mixed-tf32x3": 3,
              "mixed-bf16x3": 4, "mixed-f16x2": 5}


class pcv_rect(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double)]


class pcv_layout(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("cores", ctypes.POINTER(pcv_rect)), ("n_cores", ctypes.c_int32),
                ("has_domain", ctypes.c_int32), ("domain", pcv_rect), ("delta", ctypes.c_double),
                ("q", ctypes.c_int32), ("shell_cap", ctypes.c_int32), ("cap_seed", ctypes.c_uint64)]


class pcv_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("workspace_fraction", ctypes.c_double), ("refine_max_iter", ctypes.c_int32),
                ("refine_tol", ctypes.c_double), ("factor_engine", ctypes.c_int32), ("tc_stages", ctypes.c_int32),
                ("refine_loss_tol", ctypes.c_double), ("bucketing", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("alpha_cache", ctypes.c_int32), ("refine_loss_guard", ctypes.c_double),
                ("test_wait_us", ctypes.c_int32), ("test_withhold_task", ctypes.c_int32)]


class pcv_server_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_double), ("lanes", ctypes.c_int32), ("priorities", ctypes.c_int32)]


class PcvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_vp = ctypes.c_void_p

_SIGS = {
    "pcv_plan_create": (ctypes.c_int, [_dp, _u8p, ctypes.c_int64, ctypes.POINTER(pcv_layout),
                                       ctypes.POINTER(_vp)]),
    "pcv_plan_info": (ctypes.c_int, [_vp, _i32p, ctypes.POINTER(_i64p), ctypes.POINTER(_i64p),
                                     ctypes.POINTER(_i64p), ctypes.POINTER(_i64p)]),
    "pcv_plan_cores": (ctypes.c_int, [_vp, ctypes.POINTER(pcv_rect)]),
    "pcv_plan_destroy": (None, [_vp]),
    "pcv_create": (ctypes.c_int, [_dp, _dp, _u8p, ctypes.c_int64, ctypes.POINTER(pcv_layout),
                                  ctypes.c_int32, ctypes.POINTER(pcv_options), ctypes.POINTER(_vp)]),
    "pcv_subset_info": (ctypes.c_int, [_vp, _i32p, ctypes.POINTER(_i64p), ctypes.POINTER(_i64p),
                                       ctypes.POINTER(_i64p), ctypes.POINTER(_i64p)]),
    "pcv_cv_loss": (ctypes.c_int, [_vp, _dp, ctypes.c_int32, ctypes.c_int32, _dp, _dp, _dp, _i64p,
                                   _i32p, _vp]),
    "pcv_cv_loss_device": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp,
                                          _vp, _vp]),
    "pcv_predict": (ctypes.c_int, [_vp, _dp, _dp, ctypes.c_int64, ctypes.c_int32, _dp, _vp]),
    "pcv_neg2loglik": (ctypes.c_int, [_vp, _dp, ctypes.c_int32, ctypes.c_int32, _dp, _dp, _i32p, _vp]),
    "pcv_predict_local": (ctypes.c_int, [_vp, _dp, ctypes.c_int32, _dp, _dp, ctypes.c_int64, ctypes.c_int32, _dp,
                                         _i32p, _vp]),
    "pcv_gls": (ctypes.c_int, [_vp, _dp, ctypes.c_int32, _dp, ctypes.c_int32, _dp, _vp]),
    "pcv_set_timing": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "pcv_kernel_time": (ctypes.c_int, [_vp, _dp, _dp]),
    "pcv_phase_cycles": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32]),
    "pcv_cv_loss_fp64_static": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, _i64p, _vp, _i64p, _vp, _vp,
                                               _vp, _vp, ctypes.c_int32, _vp, _vp, _vp, _vp]),
    "pcv_selftest_df": (ctypes.c_int, [ctypes.c_int32, _dp, _dp, ctypes.c_int64, _dp]),
    "pcv_selftest_df_device": (ctypes.c_int, [ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp, _vp]),
    "pcv_selftest_umma": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_float)]),
    "pcv_buckets": (ctypes.c_int32, [_vp, ctypes.c_char_p, ctypes.c_int32]),
    "pcv_alpha_cache_stats": (ctypes.c_int, [_vp, _i64p, _i64p, _i32p]),
    "pcv_measure_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, _dp, _dp]),
    "pcv_selftest_umma_scheme": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_float)]),
    "pcv_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(pcv_server_options),
                                         ctypes.POINTER(_vp)]),
    "pcv_server_submit_cv": (ctypes.c_int, [_vp, ctypes.c_int32, _dp, _i64p]),
    "pcv_server_submit_predict": (ctypes.c_int, [_vp, ctypes.c_int32, _dp, _dp, ctypes.c_int64, _i64p]),
    "pcv_server_wait": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_double, _dp, _i32p, _dp, _dp]),
    "pcv_server_stats": (ctypes.c_int, [_vp, _dp, _dp, _dp, _i64p, _i64p, _i64p]),
    "pcv_server_destroy": (None, [_vp]),
    "pcv_destroy": (None, [_vp]),
    "pcv_status_str": (ctypes.c_char_p, [ctypes.c_int32]),
    "pcv_last_error": (ctypes.c_char_p, []),
    "pcv_version": (ctypes.c_int32, []),
    "pcv_launch_count": (ctypes.c_int64, [ctypes.c_int32]),
    "pcv_lattice": (ctypes.c_int32, [_vp, _dp, _dp]),
    "pcv_lattice_detect": (ctypes.c_int32, [_dp, ctypes.c_int64, _dp, _dp, _dp, _dp]),
}
EXPORTS = tuple(_SIGS)


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libpcv.so (building it in-tree first when it is absent or stale)."""
    path = path or build_ext.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not found at {path}")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load_library()
LIB_PATH = build_ext.LIB


def _check(st: int, what: str):
    if st != PCV_OK:
        raise PcvError(st, f"{what}: {_lib.pcv_status_str(st).decode()}: {_lib.pcv_last_error().decode()}")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def make_layout(layout: dict) -> tuple[pcv_layout, object]:
    """dict {'kind': 'grid'|'rects'|'recursive', 'nx', 'ny', 'cores', 'q', 'delta', 'domain',
    'shell_cap', 'cap_seed'} -> pcv_layout."""
    L = pcv_layout()
    keep = None
    if layout["kind"] == "grid":
        L.kind = PCV_LAYOUT_GRID
        L.nx, L.ny = int(layout["nx"]), int(layout["ny"])
    elif layout["kind"] == "rects":
        L.kind = PCV_LAYOUT_RECTS
        rects = (pcv_rect * len(layout["cores"]))(*[pcv_rect(*map(float, r)) for r in layout["cores"]])
        L.cores = ctypes.cast(rects, ctypes.POINTER(pcv_rect))
        L.n_cores = len(layout["cores"])
        keep = rects
    elif layout["kind"] == "recursive":
        L.kind = PCV_LAYOUT_RECURSIVE
        L.q = int(layout["q"])
    else:
        raise ValueError(layout["kind"])
    L.shell_cap = int(layout.get("shell_cap", 0) or 0)
    L.cap_seed = int(layout.get("cap_seed", 0)) & 0xFFFFFFFFFFFFFFFF
    if layout.get("domain") is not None:
        L.has_domain = 1
        L.domain = pcv_rect(*map(float, layout["domain"]))
    L.delta = float(layout["delta"])
    return L, keep


def _csr_views(fn, handle):
    N = ctypes.c_int32()
    ptrs = [_i64p() for _ in range(4)]
    _check(fn(handle, ctypes.byref(N), *[ctypes.byref(p) for p in ptrs]), "subset info")
    n = N.value
    To = np.ctypeslib.as_array(ptrs[0], shape=(n + 1,)).copy()
    Vo = np.ctypeslib.as_array(ptrs[2], shape=(n + 1,)).copy()
    def view(p, cnt):
        cnt = int(cnt)
        return np.ctypeslib.as_array(p, shape=(cnt,)).copy() if cnt else np.empty(0, np.int64)
    return To, view(ptrs[1], To[-1]), Vo, view(ptrs[3], Vo[-1])


def pcv_plan_create(xy, role, layout: dict):
    """Host-only membership (no device).  Returns (T_off, T_idx, V_off, V_idx, cores)."""
    xy = _f64(xy).reshape(-1, 2)
    role = np.ascontiguousarray(role, dtype=np.uint8)
    L, keep = make_layout(layout)
    h = _vp()
    _check(_lib.pcv_plan_create(_ptr(xy, _dp), _ptr(role, _u8p), len(role), ctypes.byref(L),
                                ctypes.byref(h)), "pcv_plan_create")
    try:
        To, Ti, Vo, Vi = _csr_views(_lib.pcv_plan_info, h)
        cores = (pcv_rect * (len(To) - 1))()
        _check(_lib.pcv_plan_cores(h, cores), "pcv_plan_cores")
        cores = np.array([[c.x0, c.x1, c.y0, c.y1] for c in cores])
    finally:
        _lib.pcv_plan_destroy(h)
    del keep
    return To, Ti, Vo, Vi, cores


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            return None
        return None
    return int(getattr(stream, "cuda_stream", stream))


# mixed-path factorisation engines (pcv_options.factor_engine)
ENGINES = {"tensor": 0, "simt": 1, "tensor-bf16": 2, "tensor-tf32": 3, "tensor-tf32x3": 4}


class Context:
    """A device-resident dataset with its subset layout (pcv_create ... pcv_destroy)."""

    def __init__(self, xy, v, role, layout: dict, device: int = 0, max_slots: int = 0,
                 workspace_fraction: float = 0.0, refine_max_iter: int = 0, refine_tol: float = 0.0,
                 factor_engine: str = "tensor", tc_stages: int = 0, refine_loss_tol: float = 0.0,
                 bucketing: int = 0, graph: int = 0, alpha_cache: int = 0, refine_loss_guard: float = 0.0,
                 test_wait_us: int = 0, test_withhold_task: int = 0):
        xy = _f64(xy).reshape(-1, 2)
        v = _f64(v)
        role = np.ascontiguousarray(role, dtype=np.uint8)
        L, keep = make_layout(layout)
        o = pcv_options(ctypes.sizeof(pcv_options), max_slots, workspace_fraction, refine_max_iter,
                        refine_tol, ENGINES[factor_engine], tc_stages, refine_loss_tol, bucketing, graph,
                        alpha_cache, refine_loss_guard, test_wait_us, test_withhold_task)
        h = _vp()
        _check(_lib.pcv_create(_ptr(xy, _dp), _ptr(v, _dp), _ptr(role, _u8p), len(v), ctypes.byref(L),
                               device, ctypes.byref(o), ctypes.byref(h)), "pcv_create")
        del keep
        self._h = h
        self.device = device
        self.T_off, self.T_idx, self.V_off, self.V_idx = _csr_views(_lib.pcv_subset_info, h)
        self.N = len(self.T_off) - 1
        self.n_valid = int(self.V_off[-1])

    def close(self):
        if getattr(self, "_h", None):
            _lib.pcv_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def cv_loss(self, params, precision="mixed", per_subset=False, predictions=False, stream=None):
        """pcv_cv_loss on host arrays: returns dict(sspe, status, n_valid[, z][, yhat])."""
        P = _f64(params).reshape(-1, 3)
        B = len(P)
        sspe = np.empty(B)
        status = np.empty(B, dtype=np.int32)
        z = np.empty((B, self.N)) if per_subset else None
        yh = np.empty((B, self.n_valid)) if predictions else None
        nv = ctypes.c_int64()
        _check(_lib.pcv_cv_loss(self._h, _ptr(P, _dp), B, PRECISIONS[precision], _ptr(sspe, _dp),
                                _ptr(z, _dp) if z is not None else None,
                                _ptr(yh, _dp) if yh is not None else None, ctypes.byref(nv),
                                _ptr(status, _i32p), _stream_ptr(stream)), "pcv_cv_loss")
        out = dict(sspe=sspe, status=status, n_valid=nv.value)
        if z is not None:
            out["z"] = z
        if yh is not None:
            out["yhat"] = yh
        return out

    def cv_loss_device(self, d_params, d_sspe, precision="mixed", d_z=None, d_yhat=None,
                       d_status=None, stream=None):
        """pcv_cv_loss_device on torch CUDA tensors (asynchronous on the stream)."""
        B = int(d_params.shape[0])
        ptr = lambda t: None if t is None else t.data_ptr()
        _check(_lib.pcv_cv_loss_device(self._h, ptr(d_params), B, PRECISIONS[precision], ptr(d_sspe),
                                       ptr(d_z), ptr(d_yhat), ptr(d_status), _stream_ptr(stream)),
               "pcv_cv_loss_device")

    def set_timing(self, enable: bool = True):
        _check(_lib.pcv_set_timing(self._h, 1 if enable else 0), "pcv_set_timing")

    def kernel_time(self) -> tuple[float, float]:
        """(task kernel ms, combine kernel ms) of the most recent timed call."""
        t, c = ctypes.c_double(), ctypes.c_double()
        _check(_lib.pcv_kernel_time(self._h, ctypes.byref(t), ctypes.byref(c)), "pcv_kernel_time")
        return t.value, c.value

    PHASES = ("gather_assemble", "tc_update", "diag", "panel_solve", "diag_io", "factor_simt", "solves",
              "residual", "predict_loss", "task", "residual_passes", "tasks", "fail_factor", "fail_nan",
              "fail_stall")

    def alpha_cache_stats(self) -> dict:
        """pcv_alpha_cache_stats: predictions served from kept kriging weights, and not."""
        h, m, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.pcv_alpha_cache_stats(self._h, ctypes.byref(h), ctypes.byref(m), ctypes.byref(r)),
               "pcv_alpha_cache_stats")
        return dict(hits=h.value, misses=m.value, rows=r.value)

    def buckets(self) -> str:
        """The mixed CV launch's size buckets (pcv_buckets), '' before the first mixed call."""
        n = _lib.pcv_buckets(self._h, None, 0)
        buf = ctypes.create_string_buffer(n + 1)
        _lib.pcv_buckets(self._h, buf, n + 1)
        return buf.value.decode()

    def lattice(self):
        """(hx, hy) when every point lies on one regular lattice, else None (pcv_lattice)."""
        hx, hy = ctypes.c_double(), ctypes.c_double()
        return (hx.value, hy.value) if _lib.pcv_lattice(self._h, ctypes.byref(hx), ctypes.byref(hy)) else None

    def phase_cycles(self, reset: bool = False) -> dict:
        """Per-phase SM cycles of the mixed kernel (see include/pcv.h)."""
        out = (ctypes.c_uint64 * 16)()
        _check(_lib.pcv_phase_cycles(self._h, out, 1 if reset else 0), "pcv_phase_cycles")
        return {name: int(out[i]) for i, name in enumerate(self.PHASES)}

    def neg2loglik(self, params, precision: str = "mixed", per_subset: bool = False, stream=None) -> dict:
        """Local -2 log-likelihoods (Eq. 2) of the subsets' training data (pcv_neg2loglik):
        'total' (B,), 'status' (B,), and 'per_subset' (B, N) on request."""
        P = _f64(params).reshape(-1, 3)
        B = len(P)
        total = np.empty(B)
        status = np.empty(B, dtype=np.int32)
        per = np.empty((B, self.N)) if per_subset else None
        _check(_lib.pcv_neg2loglik(self._h, _ptr(P, _dp), B, PRECISIONS[precision], _ptr(total, _dp),
                                   _ptr(per, _dp) if per is not None else None, _ptr(status, _i32p),
                                   _stream_ptr(stream)), "pcv_neg2loglik")
        out = dict(total=total, status=status)
        if per is not None:
            out["per_subset"] = per
        return out

    def gls(self, X, params3, precision="mixed", stream=None) -> np.ndarray:
        """pcv_gls: GLS coefficients of the covariates X (n x p, a row per input point)."""
        Xc = _f64(X)
        if Xc.ndim == 1:
            Xc = Xc.reshape(-1, 1)
        Xc = np.ascontiguousarray(Xc)
        p = Xc.shape[1]
        pr = _f64(params3).reshape(3)
        beta = np.empty(p)
        _check(_lib.pcv_gls(self._h, _ptr(Xc, _dp), p, _ptr(pr, _dp), PRECISIONS[precision], _ptr(beta, _dp),
                            _stream_ptr(stream)), "pcv_gls")
        return beta

    def predict_local(self, params, sspe_per_subset, xy_new, precision="mixed", stream=None):
        """pcv_predict_local: predictions with each subset's locally best row of params;
        returns (yhat, best row per subset)."""
        P = _f64(params).reshape(-1, 3)
        z = _f64(sspe_per_subset).reshape(len(P), self.N)
        q = _f64(xy_new).reshape(-1, 2)
        out = np.empty(len(q))
        best = np.empty(self.N, dtype=np.int32)
        _check(_lib.pcv_predict_local(self._h, _ptr(P, _dp), len(P), _ptr(z, _dp), _ptr(q, _dp), len(q),
                                      PRECISIONS[precision], _ptr(out, _dp), _ptr(best, _i32p),
                                      _stream_ptr(stream)), "pcv_predict_local")
        return out, best

    def predict(self, params3, xy_new, precision="mixed", stream=None):
        p = _f64(params3).reshape(3)
        q = _f64(xy_new).reshape(-1, 2)
        out = np.empty(len(q))
        _check(_lib.pcv_predict(self._h, _ptr(p, _dp), _ptr(q, _dp), len(q), PRECISIONS[precision],
                                _ptr(out, _dp), _stream_ptr(stream)), "pcv_predict")
        return out


class Server:
    """Continuous-batching request loop over device-resident datasets (pcv_server_*)."""

    def __init__(self, contexts, max_batch: int = 16, precision: str = "mixed", hbm_budget_bytes: float = 0.0,
                 lanes: int = 0, priorities: int = 0):
        self.contexts = list(contexts)
        arr = (_vp * len(self.contexts))(*[c._h for c in self.contexts])
        o = pcv_server_options(ctypes.sizeof(pcv_server_options), max_batch, PRECISIONS[precision],
                               float(hbm_budget_bytes), lanes, priorities)
        h = _vp()
        _check(_lib.pcv_server_create(arr, len(self.contexts), ctypes.byref(o), ctypes.byref(h)), "pcv_server_create")
        self._h = h
        self._m = {}

    def submit_cv(self, dataset: int, params3) -> int:
        p = _f64(params3).reshape(3)
        rid = ctypes.c_int64()
        _check(_lib.pcv_server_submit_cv(self._h, dataset, _ptr(p, _dp), ctypes.byref(rid)), "pcv_server_submit_cv")
        return rid.value

    def submit_predict(self, dataset: int, params3, xy_new) -> int:
        p = _f64(params3).reshape(3)
        q = _f64(xy_new).reshape(-1, 2)
        rid = ctypes.c_int64()
        _check(_lib.pcv_server_submit_predict(self._h, dataset, _ptr(p, _dp), _ptr(q, _dp), len(q),
                                              ctypes.byref(rid)), "pcv_server_submit_predict")
        self._m[rid.value] = len(q)
        return rid.value

    def wait(self, rid: int, timeout_s: float = 0.0) -> dict:
        m = self._m.pop(rid, 0)
        y = np.empty(m) if m else None
        sspe, st, lat = ctypes.c_double(), ctypes.c_int32(), ctypes.c_double()
        _check(_lib.pcv_server_wait(self._h, rid, timeout_s, ctypes.byref(sspe), ctypes.byref(st),
                                    _ptr(y, _dp) if y is not None else None, ctypes.byref(lat)), "pcv_server_wait")
        out = dict(status=st.value, latency_ms=lat.value)
        if y is not None:
            out["yhat"] = y
        else:
            out["sspe"] = sspe.value
        return out

    def stats(self) -> dict:
        p50, p99, eps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        done, batches, ev = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.pcv_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(eps),
                                     ctypes.byref(done), ctypes.byref(batches), ctypes.byref(ev)), "pcv_server_stats")
        return dict(p50_ms=p50.value, p99_ms=p99.value, cv_evals_per_s=eps.value, completed=done.value,
                    batches=batches.value, evictions=ev.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.pcv_server_destroy(self._h)
            self._h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pcv_create(xy, v, role, layout: dict, device: int = 0, **opts) -> Context:
    return Context(xy, v, role, layout, device, **opts)


def pcv_cv_loss(ctx: Context, params, precision="mixed", **kw):
    return ctx.cv_loss(params, precision, **kw)


def pcv_cv_loss_device(ctx: Context, d_params, d_sspe, precision="mixed", **kw):
    return ctx.cv_loss_device(d_params, d_sspe, precision, **kw)


def pcv_predict(ctx: Context, params3, xy_new, precision="mixed", **kw):
    return ctx.predict(params3, xy_new, precision, **kw)


def pcv_destroy(ctx: Context):
    ctx.close()


def pcv_cv_loss_fp64_static(d_x, d_y, d_v, T_off, d_T_idx, V_off, d_Vx, d_Vy, d_Vv, d_params, d_sspe,
                            d_sspe_per_subset=None, d_status=None, stream=None) -> int:
    """Allocation-free FP64 cross-validation loss (see include/pcv.h).  Device
    arguments are torch CUDA tensors; T_off / V_off are host int64 arrays.
    Returns the pcv_status code (no exception, so callers can test the limits)."""
    T_off = np.ascontiguousarray(T_off, dtype=np.int64)
    V_off = np.ascontiguousarray(V_off, dtype=np.int64)
    ptr = lambda t: None if t is None else t.data_ptr()
    return int(_lib.pcv_cv_loss_fp64_static(
        ptr(d_x), ptr(d_y), ptr(d_v), len(T_off) - 1, _ptr(T_off, _i64p), ptr(d_T_idx), _ptr(V_off, _i64p),
        ptr(d_Vx), ptr(d_Vy), ptr(d_Vv), ptr(d_params), int(d_params.shape[0]), ptr(d_sspe),
        ptr(d_sspe_per_subset), ptr(d_status), _stream_ptr(stream)))


DF_OPS = {"exp_neg": 0, "sqrt": 1, "mul": 2, "add": 3}


def pcv_selftest_df(op: str, a, b=None) -> np.ndarray:
    """Host evaluation of a double-float primitive (see include/pcv.h)."""
    a = _f64(a)
    bb = _f64(b) if b is not None else None
    out = np.empty(len(a))
    _check(_lib.pcv_selftest_df(DF_OPS[op], _ptr(a, _dp), _ptr(bb, _dp) if bb is not None else None, len(a),
                                _ptr(out, _dp)), "pcv_selftest_df")
    return out


def pcv_selftest_df_device(op: str, d_a, d_b, d_out, stream=None):
    """Device evaluation on torch CUDA tensors."""
    _check(_lib.pcv_selftest_df_device(DF_OPS[op], d_a.data_ptr(), d_b.data_ptr() if d_b is not None else None,
                                       int(d_a.numel()), d_out.data_ptr(), _stream_ptr(stream)),
           "pcv_selftest_df_device")


def pcv_selftest_umma(A, B):
    """C = A @ B.T (B has 128 rows) through the split-BF16 tcgen05 pipeline; returns (status, C)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    assert B.shape[0] == 128 and A.shape[1] == B.shape[1]
    C = np.zeros((A.shape[0], 128), dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    st = _lib.pcv_selftest_umma(A.ctypes.data_as(fp), A.shape[0], B.ctypes.data_as(fp), A.shape[1],
                                C.ctypes.data_as(fp))
    return int(st), C


PEAK_KINDS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "fp16": 4}


def pcv_measure_peak(kind: str, seconds: float = 2.0) -> dict:
    """Device throughput probe (dense FMA or tcgen05 MMA) on the current device:
    {'tflops': achieved TFLOP/s, 'seconds': timed duration}."""
    t, e = ctypes.c_double(), ctypes.c_double()
    _check(_lib.pcv_measure_peak(PEAK_KINDS[kind], float(seconds), ctypes.byref(t), ctypes.byref(e)),
           "pcv_measure_peak")
    return dict(tflops=t.value, seconds=e.value)


UMMA_SCHEMES = {"bf16x3": 0, "f16x2": 1, "tf32": 2, "tf32x3": 3}


def pcv_selftest_umma_scheme(scheme: str, A, B):
    """C = A @ B.T (B has 128 rows) through the tcgen05 pipeline with an operand scheme;
    returns (status, C)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    assert B.shape[0] == 128 and A.shape[1] == B.shape[1]
    C = np.zeros((A.shape[0], 128), dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    st = _lib.pcv_selftest_umma_scheme(UMMA_SCHEMES[scheme], A.ctypes.data_as(fp), A.shape[0], B.ctypes.data_as(fp),
                                       A.shape[1], C.ctypes.data_as(fp))
    return int(st), C


def pcv_lattice_detect(xy):
    """Host-only: ((x0, hx), (y0, hy)) if every point lies on one regular lattice by the
    rule pcv_create applies (a few FP64 ulps of slack), else None.  No device work."""
    xy = _f64(xy).reshape(-1, 2)
    out = [ctypes.c_double() for _ in range(4)]
    ok = _lib.pcv_lattice_detect(_ptr(xy, _dp), len(xy), *(ctypes.byref(o) for o in out))
    return ((out[0].value, out[1].value), (out[2].value, out[3].value)) if ok else None


def pcv_launch_count(reset: bool = False) -> int:
    return int(_lib.pcv_launch_count(1 if reset else 0))


def pcv_version() -> int:
    return int(_lib.pcv_version())
