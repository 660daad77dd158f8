import os
import sys

# The oracle's LAPACK-backed kriging runs many subsets on a thread pool; one BLAS thread
# per call keeps the pool from oversubscribing the host cores.  Set before numpy loads.
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def has_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library (built in-tree).  Fails loudly when it cannot be loaded."""
    if not has_gpu():
        pytest.skip("no CUDA device")
    from paper_1912_13132_gb300 import pcv
    return pcv
