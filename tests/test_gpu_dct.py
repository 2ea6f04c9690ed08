"""Masked-DCT dictionary (the structured Phi of Sec. 4.2) on the GPU against
the oracle: operator application (A X, Phi Z, Phi^T W) at sizes whose
four-step FFT splits are 4 x 4 up to 512 x 512, and whole fits.  FP32
vectors; the FFT in FP32 leaves relative errors near log2(D) 2^-24."""
import numpy as np
import pytest
import torch

from oracle import sbl
from paper_2202_12808_gb300 import api
from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import from_block, ld_of, rel_l2, support_compare, to_block

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("D,N,ncols", [(16, 4, 1), (64, 16, 3), (1024, 256, 21),
                                       (8192, 2048, 5), (1 << 15, 1 << 13, 2),
                                       (1 << 18, 1 << 16, 21)])
def test_dct_apply(cuda_lib, D, N, ncols):
    rng = np.random.default_rng(D + N + ncols)
    idx = np.sort(rng.choice(D, N, replace=False)).astype(np.int32)
    X = rng.standard_normal((D, ncols)).astype(np.float32).astype(np.float64)
    alpha = rng.uniform(0.5, 100.0, D)
    beta = 400.0
    it = torch.from_numpy(idx).cuda()
    op = B.cofem_op_dct(D, N, it.data_ptr())
    try:
        Xb, ld = to_block(X, torch.float32)
        Yb = torch.empty_like(Xb)
        al = torch.from_numpy(alpha).cuda()
        n = B.cofem_apply_workspace_bytes(op, B.COFEM_F32, ncols)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, al.data_ptr(), beta,
                         Yb.data_ptr(), ws.data_ptr(), n)
        W = torch.zeros((ncols, ld_of(N)), dtype=torch.float32, device="cuda")
        B.cofem_op_forward(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, W.data_ptr(), ld_of(N),
                           ws.data_ptr(), n)
        Z = torch.zeros_like(Xb)
        B.cofem_op_adjoint(op, B.COFEM_F32, W.data_ptr(), ld_of(N), ncols, Z.data_ptr(), ld,
                           ws.data_ptr(), n)
        torch.cuda.synchronize()
        phi, phit, _ = sbl.dct_dictionary(idx, D)
        ref = sbl.apply_A(phi, phit, beta, alpha, X)
        got = from_block(Yb, D)
        for j in range(ncols):
            assert rel_l2(got[:, j], ref[:, j]) <= 2e-6, (j, rel_l2(got[:, j], ref[:, j]))
        Wg = W[:, :N].T.double().cpu().numpy()
        assert rel_l2(Wg, phi(X)) <= 2e-6
        assert rel_l2(from_block(Z, D), phit(Wg)) <= 2e-6
    finally:
        B.cofem_op_destroy(op)


def test_dct_rejects_bad_sizes(cuda_lib):
    it = torch.zeros(8, dtype=torch.int32, device="cuda")
    for D, N in ((100, 8), (8, 8), (1 << 23, 8), (64, 0), (64, 65)):
        with pytest.raises(B.CofemError):
            B.cofem_op_dct(D, N, it.data_ptr())


@pytest.mark.parametrize("seed", [0, 1])
def test_dct_fit_fp32(cuda_lib, seed):
    # D = 4096, N = 1024 kept samples, d = 0.04 D coefficients (the paper's
    # first DCT setting), sigma 0.01, K = 20, 20 EM iterations, eps 1e-5
    D, N = 4096, 1024
    p = datagen.dct_problem(D, N, int(0.04 * D), 0.01, seed=seed)
    op = api.DctOperator(torch.from_numpy(p.idx).cuda(), D)
    y32 = p.y.astype(np.float32)
    prm = api.params(vec_dtype=B.COFEM_F32, K=20, em_iters=20, cg_tol=1e-5, cg_max_iters=400,
                     seed=seed)
    r = api.fit(op, torch.from_numpy(y32).cuda(), p.beta, prm)
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dct(p.idx, D, y32.astype(np.float64), p.beta, 20, 20, 1e-5, 400,
                                     seed=seed)
    a, mu = r.alpha.cpu().numpy(), r.mu.cpu().numpy()
    assert rel_l2(mu, rmu) <= 1e-4, rel_l2(mu, rmu)
    eq, border = support_compare(a, ra)
    assert eq, border
    # alpha at 3e-3 (the dense and conv tests use 1e-3): with N = D/4 every
    # coordinate is still in the support after 20 EM iterations and alpha
    # follows the probe columns' truncated solves closely -- the oracle's own
    # alpha moves by 1.7e-2 to 2.9e-2 between tolerance 1e-5 and 1e-6, and an
    # FP32 emulation of the oracle (FP32 vectors and transforms) by 3.4e-4 and
    # 7.0e-4 on these two problems (tests/test_tolerance_evidence.py::
    # test_dct_alpha_sensitivity)
    sup = (a < 1e6) & (ra < 1e6)
    assert np.max(np.abs(a[sup] - ra[sup]) / ra[sup]) <= 3e-3
    assert abs(sum(r.stats["cg_iters"]) - sum(rst.cg_iters)) <= 0.05 * sum(rst.cg_iters)


def test_dct_fit_residual_replacement(cuda_lib):
    # true-residual replacement every 10 iterations (the IF node of the CG
    # loop) with the masked DCT; sigma 0.1 (beta 100) keeps the FP32 true
    # residual attainable
    D, N = 2048, 512
    p = datagen.dct_problem(D, N, int(0.04 * D), 0.1, seed=5)
    op = api.DctOperator(torch.from_numpy(p.idx).cuda(), D)
    y32 = p.y.astype(np.float32)
    prm = api.params(vec_dtype=B.COFEM_F32, K=20, em_iters=10, cg_tol=1e-5, cg_max_iters=400,
                     seed=5, resid_replace_every=10)
    r = api.fit(op, torch.from_numpy(y32).cuda(), p.beta, prm)
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dct(p.idx, D, y32.astype(np.float64), p.beta, 20, 10, 1e-5, 400,
                                     seed=5, resid_replace_every=10)
    assert rel_l2(r.mu.cpu().numpy(), rmu) <= 1e-4
    assert abs(sum(r.stats["cg_iters"]) - sum(rst.cg_iters)) <= 0.05 * sum(rst.cg_iters)
