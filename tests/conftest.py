import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "many_blas_threads: large oracle products, keep BLAS threads")


@pytest.fixture(scope="session")
def cuda_lib():
    """The C-ABI library, built in-tree; tests marked gpu use it."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_12808_gb300 import binding
    return binding.lib()


# Modules whose oracle runs are many small matrix products: one BLAS thread
# each (threads only add contention at these sizes; tests that need more
# mark themselves with `many_blas_threads`).
_SMALL_BLAS = ("test_tolerance_evidence", "test_oracle_pins", "test_oracle_learned_pins",
               "test_oracle_block_cg", "test_oracle_mlp")


@pytest.fixture(autouse=True)
def _blas_threads(request):
    mod = request.node.module.__name__.rsplit(".", 1)[-1]
    if mod not in _SMALL_BLAS or request.node.get_closest_marker("many_blas_threads"):
        yield
        return
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:
        yield
        return
    with threadpool_limits(limits=1, user_api="blas"):
        yield
