"""Double-float arithmetic of the mixed path (csrc/df.cuh), checked against FP64.

The refinement residuals and the predictions of the mixed path use pairs of
floats.  Host evaluation is checked against libm here; the device evaluation is
checked against CUDA's FP64 functions (through torch) in the gpu-marked test.
Bounds: ~48-bit arithmetic, so a few 1e-15 relative for sqrt / mul / add; for
exp(-t) the input itself carries a relative error of 2^-48, i.e. an absolute
error of t * 3.6e-15 in the argument, hence the bound 1e-14 * max(1, t) up to
t = 40 (covariance arguments d / rho stay far below that in practice).
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1912_13132_gb300 import pcv

RNG = np.random.default_rng(7)


def _exp_inputs():
    return np.concatenate([np.linspace(0.0, 40.0, 200001), RNG.random(100000) * 0.01,
                           RNG.random(100000) * 3.0, [0.0, 1e-30, 1e-12, 1e-6, 0.5, 1.0]])


def test_exp_neg_host():
    t = _exp_inputs()
    rel = np.abs(pcv.pcv_selftest_df("exp_neg", t) - np.exp(-t)) / np.exp(-t)
    assert np.all(rel <= 1e-14 * np.maximum(1.0, t)), rel.max()


def test_exp_neg_large_arguments_are_tiny_and_nonnegative():
    t = np.linspace(40.0, 120.0, 1001)
    e = pcv.pcv_selftest_df("exp_neg", t)
    assert np.all(e >= 0.0) and np.all(e <= np.exp(-40.0) * (1 + 1e-6))


def test_sqrt_mul_add_host():
    a = RNG.random(100000) * 4.0
    b = RNG.standard_normal(100000)
    assert np.max(np.abs(pcv.pcv_selftest_df("sqrt", a) - np.sqrt(a)) / np.sqrt(a)) <= 4e-14
    assert np.max(np.abs(pcv.pcv_selftest_df("mul", a, b) - a * b) / np.abs(a * b)) <= 4e-14
    s = a + b
    assert np.max(np.abs(pcv.pcv_selftest_df("add", a, b) - s) / np.maximum(np.abs(a) + np.abs(b), 1e-300)) <= 4e-14


@pytest.mark.gpu
def test_exp_neg_device(gpu_lib):
    import torch

    t = _exp_inputs()
    d_t = torch.tensor(t, dtype=torch.float64, device="cuda")
    d_o = torch.empty_like(d_t)
    gpu_lib.pcv_selftest_df_device("exp_neg", d_t, None, d_o)
    ref = torch.exp(-d_t)
    rel = ((d_o - ref).abs() / ref).cpu().numpy()
    assert np.all(rel <= 1e-14 * np.maximum(1.0, t)), rel.max()
    host = gpu_lib.pcv_selftest_df("exp_neg", t)
    assert np.max(np.abs(d_o.cpu().numpy() - host) / np.exp(-t)) <= 1e-14 * 40
