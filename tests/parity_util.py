"""Error metrics shared by the GPU parity tests.

CV loss: |Z - Z_ref| / Z_ref (relative, per configuration and per subset).
Predictions: per subset, max_j |yhat_j - yhat_ref_j| / RMS_j(yhat_ref).
"""
from __future__ import annotations

import numpy as np

# tolerances written from the stated targets: FP64 path 1e-10 relative;
# mixed path 1e-6 on CV losses and 1e-5 on predictions.
TOL = {"fp64": dict(loss=1e-10, pred=1e-10), "mixed": dict(loss=1e-6, pred=1e-5)}
# the mixed path's explicit operand-scheme modes share its bars
for _mode in ("mixed-tf32", "mixed-tf32x3", "mixed-bf16x3", "mixed-f16x2"):
    TOL[_mode] = TOL["mixed"]


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def pred_err(yh, ref):
    yh, ref = np.asarray(yh, float), np.asarray(ref, float)
    if len(ref) == 0:
        return 0.0
    rms = np.sqrt(np.mean(ref ** 2))
    return float(np.max(np.abs(yh - ref)) / max(rms, 1e-300))


def compare(gpu: dict, ref: dict, V_off, subsets, B, prec: str, check_total=True):
    """Check per-subset losses and predictions of `gpu` (Context.cv_loss output with
    per_subset and predictions) against the oracle result `ref` on `subsets`."""
    tol = TOL[prec]
    worst = dict(loss=0.0, pred=0.0)
    for b in range(B):
        for i in subsets:
            zr = ref["z"][b, i]
            zg = gpu["z"][b, i]
            if V_off[i + 1] == V_off[i]:
                assert zg == 0.0
                continue
            e = float(rel(zg, zr))
            worst["loss"] = max(worst["loss"], e)
            assert e <= tol["loss"], (prec, b, i, zg, zr, e)
            yg = gpu["yhat"][b, V_off[i]:V_off[i + 1]]
            pe = pred_err(yg, ref["yhat"][(b, i)])
            worst["pred"] = max(worst["pred"], pe)
            assert pe <= tol["pred"], (prec, b, i, pe)
        if check_total:
            e = float(rel(gpu["sspe"][b], ref["sspe"][b]))
            worst["loss"] = max(worst["loss"], e)
            assert e <= tol["loss"], (prec, b, gpu["sspe"][b], ref["sspe"][b])
    return worst
