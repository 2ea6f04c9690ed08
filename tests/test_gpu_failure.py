"""Failure detection without a GPU fault: a bounded device wait that runs
out reports COFEM_ERR_TIMEOUT through the error word and leaves the
context usable (the next launches still compute correct results)."""
import numpy as np
import pytest
import torch

from paper_2202_12808_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives(cuda_lib):
    assert B.cofem_selftest_wait_timeout(20_000_000) == 5        # 20 ms, nothing arrives
    assert B.cofem_selftest_wait_timeout(1_000) == 5
    assert B.cofem_selftest_wait_timeout(10) == 1                # limit out of range
    # the same context still runs kernels: probes stay bit-exact
    out = torch.empty((4, 256), dtype=torch.float64, device="cuda")
    B.cofem_probe_fill(7, 3, 4, 256, B.COFEM_F64, out.data_ptr(), 256)
    torch.cuda.synchronize()
    from oracle import probe_hash as ph
    np.testing.assert_array_equal(out.cpu().numpy().T, ph.probe_matrix(7, 3, 4, 256))
