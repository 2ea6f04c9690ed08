"""Convolutional dictionary on the tensor cores (cofem_op_conv1d_set_tensor_cores):
the block Toeplitz GEMMs against the oracle on the BF16-rounded filters
(the dictionary the operator then applies, as a BF16 dense dictionary is
compared on its rounded entries): A X at ragged sizes (one partial tile,
two tiles, more than eight channels so that accumulator slots are reused,
few taps), on sampled outputs at L = 2^20, the column norms, and whole fits
(the fit prepares the Toeplitz images once)."""
import numpy as np
import pytest
import torch

from oracle import sbl
from paper_2202_12808_gb300 import api
from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import from_block, ld_of, rel_l2, support_compare, to_block

pytestmark = pytest.mark.gpu


def bf16_round(h):
    return torch.from_numpy(np.ascontiguousarray(h, dtype=np.float32)).to(
        torch.bfloat16).double().numpy()


@pytest.mark.parametrize("L,C,T,ncols", [(64, 1, 64, 3), (4096, 8, 64, 17), (8256, 3, 5, 2),
                                         (16576, 11, 64, 5), (2048, 2, 17, 21)])
def test_conv_tc_apply(cuda_lib, L, C, T, ncols):
    rng = np.random.default_rng(7 * L + C + T)
    h = rng.standard_normal((C, T)).astype(np.float32)
    D = C * L
    X = rng.standard_normal((D, ncols)).astype(np.float32).astype(np.float64)
    alpha = rng.uniform(0.5, 100.0, D)
    beta = 400.0
    ht = torch.from_numpy(h).cuda()
    op = B.cofem_op_conv1d(L, C, T, ht.data_ptr())
    B.cofem_op_conv1d_set_tensor_cores(op, 1)
    try:
        Xb, ld = to_block(X, torch.float32)
        Yb = torch.full_like(Xb, float("nan"))
        al = torch.from_numpy(alpha).cuda()
        n = B.cofem_apply_workspace_bytes(op, B.COFEM_F32, ncols)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, al.data_ptr(), beta,
                         Yb.data_ptr(), ws.data_ptr(), n)
        W = torch.zeros((ncols, ld_of(L)), dtype=torch.float32, device="cuda")
        B.cofem_op_forward(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, W.data_ptr(), ld_of(L),
                           ws.data_ptr(), n)
        torch.cuda.synchronize()
        phi, phit, _ = sbl.conv_dictionary(bf16_round(h), L)
        ref = sbl.apply_A(phi, phit, beta, alpha, X)
        got = from_block(Yb, D)
        for j in range(ncols):
            assert rel_l2(got[:, j], ref[:, j]) <= 1e-5, (j, rel_l2(got[:, j], ref[:, j]))
        # the stand-alone product uses the same rounded filters
        assert rel_l2(W[:, :L].T.double().cpu().numpy(), phi(X)) <= 1e-5
    finally:
        B.cofem_op_destroy(op)


def test_conv_tc_full_size_sampled(cuda_lib):
    # L = 2^20, 8 filters x 64 taps, 17 columns (128 tiles per column); 3
    # columns checked on 256 sampled coordinates from the definition
    L, C, T, ncols = 1 << 20, 8, 64, 17
    p = datagen.conv_problem(L, C, T, 1e-3, 0.05, seed=0)
    D = C * L
    rng = np.random.default_rng(4)
    X = rng.standard_normal((D, ncols)).astype(np.float32)
    alpha = rng.uniform(1.0, 1e3, D)
    ht = torch.from_numpy(p.h).cuda()
    op = B.cofem_op_conv1d(L, C, T, ht.data_ptr())
    B.cofem_op_conv1d_set_tensor_cores(op, 1)
    try:
        Xb = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
        Yb = torch.empty_like(Xb)
        al = torch.from_numpy(alpha).cuda()
        n = B.cofem_apply_workspace_bytes(op, B.COFEM_F32, ncols)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), D, ncols, al.data_ptr(), p.beta,
                         Yb.data_ptr(), ws.data_ptr(), n)
        torch.cuda.synchronize()
        hr = bf16_round(p.h)
        rows = np.sort(np.concatenate([[0, L - 1, L, D - 1], rng.choice(D, size=252, replace=False)]))
        for j in (0, 7, 16):
            x = X[:, j].astype(np.float64)
            w = sbl.conv_forward(hr, x.reshape(C, L))
            c, m = rows // L, rows % L
            adj = np.array([sum(hr[cc, t] * w[(mm + t) % L] for t in range(T))
                            for cc, mm in zip(c, m)])
            ref = p.beta * adj + alpha[rows] * x[rows]
            got = Yb[j, rows].double().cpu().numpy()
            assert rel_l2(got, ref) <= 1e-5, j
    finally:
        B.cofem_op_destroy(op)


def test_conv_tc_col_norms(cuda_lib):
    L, C, T = 256, 3, 40
    h = np.random.default_rng(5).standard_normal((C, T)).astype(np.float32)
    op = api.ConvOperator(torch.from_numpy(h).cuda(), L, tensor_cores=True)
    out = api.col_norms(op, "cuda").cpu().numpy()
    ref = np.repeat(np.sum(bf16_round(h) ** 2, axis=1), L)
    assert np.max(np.abs(out - ref) / ref) <= 1e-6


@pytest.mark.parametrize("seed", [0, 1])
def test_conv_tc_fit(cuda_lib, seed):
    # L = 1024, 8 filters x 64 taps (D = 8192), 0.1% nonzeros, sigma 0.05,
    # K = 16, 30 EM iterations, eps 1e-5; oracle on the materialised Phi of
    # the rounded filters; the same bars as the FP32 conv fit
    L, C, T = 1024, 8, 64
    p = datagen.conv_problem(L, C, T, 1e-3, 0.05, seed=seed)
    op = api.ConvOperator(torch.from_numpy(p.h).cuda(), L, tensor_cores=True)
    y32 = p.y.astype(np.float32)
    prm = api.params(vec_dtype=B.COFEM_F32, K=16, em_iters=30, cg_tol=1e-5, cg_max_iters=400,
                     seed=seed)
    r = api.fit(op, torch.from_numpy(y32).cuda(), p.beta, prm)
    torch.cuda.synchronize()
    M = sbl.conv_matrix_vectorised(bf16_round(p.h), L)
    ra, rmu, rs, rst = sbl.cofem_dense(M, y32.astype(np.float64), p.beta, 16, 30, 1e-5, 400,
                                       seed=seed)
    a, mu = r.alpha.cpu().numpy(), r.mu.cpu().numpy()
    assert rel_l2(mu, rmu) <= 1e-4
    eq, border = support_compare(a, ra)
    assert eq, border
    sup = (a < 1e6) & (ra < 1e6)
    assert np.max(np.abs(a[sup] - ra[sup]) / ra[sup]) <= 1e-3
    assert abs(sum(r.stats["cg_iters"]) - sum(rst.cg_iters)) <= 0.05 * sum(rst.cg_iters)


def test_conv_tc_jacobi_start(cuda_lib):
    """The learned start's all-zero network (mu_hat = 0, s_hat = 1 / c_d,
    c_d = beta ||phi_d||^2 + alpha_d with the rounded filters' column norms)
    on the tensor-core convolution against the oracle's learned loop with
    the same predictor on the materialised dictionary of the rounded
    filters; the bars of the learned dense fit.  Sigma 0.1 (beta 100), as
    there: at sigma 0.05 the solves' tolerance alone moves mu by 1e-4 after
    15 EM iterations (the oracle's own plain and Jacobi fits differ by
    1.4e-4 there, 1.9e-5 at sigma 0.1, where the GPU fit is 4.0e-5 from the
    oracle's)."""
    from oracle import mlp as omlp
    L, C, T = 1024, 8, 64
    p = datagen.conv_problem(L, C, T, 1e-3, 0.1, seed=2)
    op = api.ConvOperator(torch.from_numpy(p.h).cuda(), L, tensor_cores=True)
    y32 = p.y.astype(np.float32)
    zero_net = torch.zeros(omlp.N_PARAMS, dtype=torch.bfloat16, device="cuda")
    prm = api.params(vec_dtype=B.COFEM_F32, K=16, em_iters=15, cg_tol=1e-5, cg_max_iters=400,
                     seed=2)
    prm.mlp = zero_net.data_ptr()
    r = api.fit(op, torch.from_numpy(y32).cuda(), p.beta, prm)
    torch.cuda.synchronize()
    fb = B.cofem_last_fit_fallbacks()
    M = sbl.conv_matrix_vectorised(bf16_round(p.h), L)
    pn2 = np.sum(M * M, axis=0).astype(np.float32).astype(np.float64)

    def predict(alpha, mu_prev, s_prev):
        return omlp.predict(np.zeros((len(alpha), 2)), alpha, pn2, p.beta)

    phi, phit, D = sbl.dense_dictionary(M)
    ra, rmu, rs, rst = sbl.cofem_learned(phi, phit, D, y32.astype(np.float64), p.beta, 16, 15,
                                         1e-5, 400, predict, seed=2)
    assert fb == sum(rst.fallbacks)
    assert rel_l2(r.mu.cpu().numpy(), rmu) <= 1e-4
    eq, border = support_compare(r.alpha.cpu().numpy(), ra)
    assert eq, border
    assert abs(sum(r.stats["cg_iters"]) - sum(rst.cg_iters)) <= 0.1 * sum(rst.cg_iters)


def test_conv_tc_apply_many_tiles(cuda_lib):
    # L = 2^16 + 64 (nine tiles per column, the last one block of 64 outputs
    # wide), 8 filters x 64 taps, 17 columns: 153 work units, so the CTAs
    # take more than one tile each; every output against the oracle
    L, C, T, ncols = (1 << 16) + 64, 8, 64, 17
    p = datagen.conv_problem(L, C, T, 1e-3, 0.05, seed=3)
    D = C * L
    rng = np.random.default_rng(6)
    X = rng.standard_normal((D, ncols)).astype(np.float32).astype(np.float64)
    alpha = rng.uniform(1.0, 1e3, D)
    ht = torch.from_numpy(p.h).cuda()
    op = B.cofem_op_conv1d(L, C, T, ht.data_ptr())
    B.cofem_op_conv1d_set_tensor_cores(op, 1)
    try:
        Xb, ld = to_block(X, torch.float32)
        Yb = torch.full_like(Xb, float("nan"))
        al = torch.from_numpy(alpha).cuda()
        n = B.cofem_apply_workspace_bytes(op, B.COFEM_F32, ncols)
        ws = torch.empty(n, dtype=torch.uint8, device="cuda")
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, al.data_ptr(), p.beta,
                         Yb.data_ptr(), ws.data_ptr(), n)
        torch.cuda.synchronize()
        phi, phit, _ = sbl.conv_dictionary(bf16_round(p.h), L)
        ref = sbl.apply_A(phi, phit, p.beta, alpha, X)
        got = from_block(Yb, D)
        for j in range(ncols):
            assert rel_l2(got[:, j], ref[:, j]) <= 1e-5, (j, rel_l2(got[:, j], ref[:, j]))
    finally:
        B.cofem_op_destroy(op)


def test_conv_tc_refused_elsewhere(cuda_lib):
    t = torch.zeros(64, dtype=torch.float32, device="cuda")
    op = api.DenseOperator(t.reshape(8, 8))
    with pytest.raises(B.CofemError):
        B.cofem_op_conv1d_set_tensor_cores(op.handle, 1)
    cop = B.cofem_op_conv1d(64, 1, 8, t.data_ptr())
    try:
        with pytest.raises(B.CofemError):
            B.cofem_op_conv1d_set_tensor_cores(cop, 2)
    finally:
        B.cofem_op_destroy(cop)
