"""The entry point's smoke check (one small FP64 and mixed CV loss against the oracle)
runs under the GPU suite too."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke(gpu_lib):
    import __graft_entry__

    __graft_entry__.smoke()
