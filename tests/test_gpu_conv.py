"""Convolutional dictionary on the GPU against the oracle: operator
application (forward, adjoint, A X) at ragged and full sizes, and whole fits.
Circular convolution, C filters of T taps, D = C L (FP32 vectors)."""
import numpy as np
import pytest
import torch

from oracle import sbl
from paper_2202_12808_gb300 import api
from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import from_block, ld_of, rel_l2, support_compare, to_block

pytestmark = pytest.mark.gpu


def _op(h):
    ht = torch.from_numpy(np.ascontiguousarray(h, dtype=np.float32)).cuda()
    return ht, B.cofem_op_conv1d


@pytest.mark.parametrize("L,C,T,ncols", [(4096, 8, 64, 17), (4160, 8, 64, 1), (4160, 3, 5, 2),
                                         (2048, 2, 64, 21), (64, 1, 64, 3)])
def test_conv_apply(cuda_lib, L, C, T, ncols):
    rng = np.random.default_rng(L + C + T)
    h = rng.standard_normal((C, T)).astype(np.float32)
    D = C * L
    X = rng.standard_normal((D, ncols)).astype(np.float32).astype(np.float64)
    alpha = rng.uniform(0.5, 100.0, D)
    beta = 400.0
    ht = torch.from_numpy(h).cuda()
    op = B.cofem_op_conv1d(L, C, T, ht.data_ptr())
    try:
        Xb, ld = to_block(X, torch.float32)
        Yb = torch.empty_like(Xb)
        al = torch.from_numpy(alpha).cuda()
        n = B.cofem_apply_workspace_bytes(op, B.COFEM_F32, ncols)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, al.data_ptr(), beta,
                         Yb.data_ptr(), ws.data_ptr(), n)
        W = torch.zeros((ncols, ld_of(L)), dtype=torch.float32, device="cuda")
        B.cofem_op_forward(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, W.data_ptr(), ld_of(L),
                           ws.data_ptr(), n)
        Z = torch.zeros_like(Xb)
        B.cofem_op_adjoint(op, B.COFEM_F32, W.data_ptr(), ld_of(L), ncols, Z.data_ptr(), ld,
                           ws.data_ptr(), n)
        torch.cuda.synchronize()
        phi, phit, _ = sbl.conv_dictionary(h.astype(np.float64), L)
        ref = sbl.apply_A(phi, phit, beta, alpha, X)
        got = from_block(Yb, D)
        for j in range(ncols):
            assert rel_l2(got[:, j], ref[:, j]) <= 1e-5, j
        Wg = W[:, :L].T.double().cpu().numpy()
        assert rel_l2(Wg, phi(X)) <= 1e-5
        assert rel_l2(from_block(Z, D), phit(Wg)) <= 1e-5
    finally:
        B.cofem_op_destroy(op)


def test_conv_apply_full_size_sampled(cuda_lib):
    # L = 2^20, 8 filters x 64 taps, 17 columns; 3 columns checked on 256
    # sampled coordinates computed by the oracle's definition
    L, C, T, ncols = 1 << 20, 8, 64, 17
    p = datagen.conv_problem(L, C, T, 1e-3, 0.05, seed=0)
    D = C * L
    rng = np.random.default_rng(3)
    X = rng.standard_normal((D, ncols)).astype(np.float32)
    alpha = rng.uniform(1.0, 1e3, D)
    ht = torch.from_numpy(p.h).cuda()
    op = B.cofem_op_conv1d(L, C, T, ht.data_ptr())
    try:
        Xb = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
        Yb = torch.empty_like(Xb)
        al = torch.from_numpy(alpha).cuda()
        n = B.cofem_apply_workspace_bytes(op, B.COFEM_F32, ncols)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), D, ncols, al.data_ptr(), p.beta,
                         Yb.data_ptr(), ws.data_ptr(), n)
        torch.cuda.synchronize()
        h64 = p.h.astype(np.float64)
        rows = np.sort(rng.choice(D, size=256, replace=False))
        for j in (0, 7, 16):
            x = X[:, j].astype(np.float64)
            w = sbl.conv_forward(h64, x.reshape(C, L))              # Phi x (length L)
            c, m = rows // L, rows % L
            adj = np.array([sum(h64[cc, t] * w[(mm + t) % L] for t in range(T))
                            for cc, mm in zip(c, m)])
            ref = p.beta * adj + alpha[rows] * x[rows]
            got = Yb[j, rows].double().cpu().numpy()
            assert rel_l2(got, ref) <= 1e-5, j
    finally:
        B.cofem_op_destroy(op)


@pytest.mark.parametrize("seed", [0, 1])
def test_conv_fit_fp32(cuda_lib, seed):
    # L = 1024, 8 filters x 64 taps (D = 8192), 0.1% nonzeros, sigma 0.05,
    # K = 16, 30 EM iterations, eps 1e-5; oracle on the materialised Phi
    L, C, T = 1024, 8, 64
    p = datagen.conv_problem(L, C, T, 1e-3, 0.05, seed=seed)
    h64 = p.h.astype(np.float64)
    ht = torch.from_numpy(p.h).cuda()
    op = api.ConvOperator(ht, L)
    y32 = p.y.astype(np.float32)
    prm = api.params(vec_dtype=B.COFEM_F32, K=16, em_iters=30, cg_tol=1e-5, cg_max_iters=400,
                     seed=seed)
    r = api.fit(op, torch.from_numpy(y32).cuda(), p.beta, prm)
    torch.cuda.synchronize()
    M = sbl.conv_matrix_vectorised(h64, L)
    ra, rmu, rs, rst = sbl.cofem_dense(M, y32.astype(np.float64), p.beta, 16, 30, 1e-5, 400,
                                       seed=seed)
    a, mu = r.alpha.cpu().numpy(), r.mu.cpu().numpy()
    assert rel_l2(mu, rmu) <= 1e-4
    eq, border = support_compare(a, ra)
    assert eq, border
    sup = (a < 1e6) & (ra < 1e6)
    assert np.max(np.abs(a[sup] - ra[sup]) / ra[sup]) <= 1e-3
