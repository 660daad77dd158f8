"""The split-BF16 tcgen05 pipeline on its own (pcv_selftest_umma): C = A B^T.

Three BF16 terms per operand and six products reproduce FP32-accurate products;
the accumulation is FP32 in tensor memory.  Bound: 4e-6 relative to the row-wise
sum of |A||B|^T (K up to 1024 terms of FP32-rounded products).
"""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,K", [(128, 32), (300, 256), (517, 1024)])
def test_umma_block_column(gpu_lib, M, K):
    r = np.random.default_rng(M + K)
    A = r.standard_normal((M, K)).astype(np.float32)
    B = r.standard_normal((128, K)).astype(np.float32)
    st, C = gpu_lib.pcv_selftest_umma(A, B)
    assert st == 0, st
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    err = np.abs(C - ref) / scale
    assert err.max() <= 4e-6, err.max()


# error bound relative to the row-wise sum of |A||B|^T per scheme: FP32 accumulation over
# K terms dominates the 22-24-bit schemes; TF32 operands carry 11 significant bits
SCHEME_BOUND = {"bf16x3": 4e-6, "f16x2": 8e-6, "tf32x3": 8e-6, "tf32": 2e-3}


@pytest.mark.parametrize("scheme", ["bf16x3", "f16x2", "tf32", "tf32x3"])
@pytest.mark.parametrize("M,K", [(128, 32), (300, 256)])
def test_umma_schemes(gpu_lib, scheme, M, K):
    """Every operand scheme of the tensor engines through the same pipeline (values in
    FP16 range): the split products reproduce A B^T to the scheme's accuracy."""
    r = np.random.default_rng(M + K + 7)
    A = (r.standard_normal((M, K)) * 0.3).astype(np.float32)
    B = (r.standard_normal((128, K)) * 0.3).astype(np.float32)
    st, C = gpu_lib.pcv_selftest_umma_scheme(scheme, A, B)
    assert st == 0, st
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    err = np.abs(C - ref) / scale
    print(scheme, M, K, "max rel err", err.max())
    assert err.max() <= SCHEME_BOUND[scheme], err.max()
