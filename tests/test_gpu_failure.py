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


def test_cg_update_wait_runs_out_and_fit_survives(cuda_lib):
    """The fused CG update's wait for the block that closes an iteration:
    with no closing block every other block gives up after the limit, the
    launch returns COFEM_ERR_TIMEOUT within about that time, and a following
    fit on the same context (tensor cores, fused direction update) still
    matches the oracle."""
    import time
    from oracle import sbl
    from paper_2202_12808_gb300 import api, datagen
    nb = B.cofem_selftest_cg_update_workspace_bytes()
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    assert B.cofem_selftest_cg_update_timeout(5_000_000, ws.data_ptr(), nb) == 5   # 5 ms
    assert time.perf_counter() - t0 < 2.0
    assert B.cofem_selftest_cg_update_timeout(10, ws.data_ptr(), nb) == 1         # out of range
    assert B.cofem_selftest_cg_update_timeout(5_000_000, ws.data_ptr(), 16) == 7  # too small
    pr = datagen.dense_problem(200, 800, 10, 0.1, seed=3)
    t16 = torch.from_numpy(pr.Phi).to(torch.bfloat16)
    op = api.DenseOperator(t16.cuda())
    y32 = pr.y.astype(np.float32)
    r = api.fit(op, torch.from_numpy(y32).cuda(), pr.beta,
                api.params(vec_dtype=B.COFEM_F32, K=8, em_iters=3, cg_tol=1e-6, cg_max_iters=300,
                           seed=3))
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dense(t16.double().numpy(), y32.astype(np.float64), pr.beta, 8,
                                       3, 1e-6, 300, seed=3)
    mu = r.mu.cpu().numpy()
    assert np.linalg.norm(mu - rmu) / np.linalg.norm(rmu) <= 1e-4
