"""Multi-task CoFEM (T tasks sharing alpha, the extension named in Sec. 5)
through cofem_fit against the FP64 oracle: B = [beta Phi^T y_1 .. beta Phi^T
y_T | p_1 .. p_K], mu is T x D, alpha_d = 1 / (mean_t mu_td^2 + s_d)."""
import numpy as np
import pytest
import torch

from oracle import sbl
from paper_2202_12808_gb300 import api
from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import bf16_round, rel_l2, support_compare

pytestmark = pytest.mark.gpu


def test_multitask_fp64_fixed_iterations(cuda_lib):
    pr = datagen.multitask_problem(256, 1024, 3, 40, 0.01, seed=1)
    Phi = pr.Phi.astype(np.float64)
    op = api.DenseOperator(torch.from_numpy(Phi).cuda())
    p = api.params(vec_dtype=B.COFEM_F64, K=16, em_iters=10, cg_tol=1e-8, cg_max_iters=400,
                   fixed_cg_iters=300, seed=2)
    r = api.fit(op, torch.from_numpy(pr.Y).cuda(), pr.beta, p)
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dense(Phi, pr.Y, pr.beta, 16, 10, 1e-8, 400,
                                       fixed_cg_iters=300, seed=2)
    mu = r.mu.cpu().numpy()
    assert mu.shape == (3, 1024)
    assert r.stats["cg_iters"] == [300] * 10
    for t in range(3):
        assert rel_l2(mu[t], rmu[t]) <= 1e-9, t
    assert rel_l2(r.s.cpu().numpy(), rs) <= 1e-9
    a = r.alpha.cpu().numpy()
    ok = ra < 1e6
    assert rel_l2(a[ok], ra[ok]) <= 1e-9


def test_multitask_bf16_tensor_cores(cuda_lib):
    # T = 4 tasks + K = 20 probes = 24 columns on the tensor-core operator
    pr = datagen.multitask_problem(256, 1024, 4, 40, 0.01, seed=3)
    t16, Phi_ref = bf16_round(pr.Phi)
    op = api.DenseOperator(t16.cuda())
    Y32 = pr.Y.astype(np.float32)
    # tolerance 1e-5 (the dense workload's): at 1e-6 the FP32 solve sits near
    # its rounding floor and takes 4 % more iterations than the FP64 oracle
    p = api.params(vec_dtype=B.COFEM_F32, K=20, em_iters=30, cg_tol=1e-5, cg_max_iters=400,
                   seed=4)
    r = api.fit(op, torch.from_numpy(Y32).cuda(), pr.beta, p)
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dense(Phi_ref, Y32.astype(np.float64), pr.beta, 20, 30, 1e-5,
                                       400, seed=4)
    a, mu = r.alpha.cpu().numpy(), r.mu.cpu().numpy()
    for t in range(4):
        assert rel_l2(mu[t], rmu[t]) <= 1e-4, (t, rel_l2(mu[t], rmu[t]))
    eq, border = support_compare(a, ra)
    assert eq, border
    sup = (a < 1e6) & (ra < 1e6)
    assert np.max(np.abs(a[sup] - ra[sup]) / ra[sup]) <= 1e-3
    assert abs(sum(r.stats["cg_iters"]) - sum(rst.cg_iters)) <= 0.05 * sum(rst.cg_iters)


def test_multitask_dct_fixed_iterations(cuda_lib):
    # two tasks observed through the same masked DCT
    D, N = 2048, 512
    p1 = datagen.dct_problem(D, N, 80, 0.05, seed=6)
    p2 = datagen.dct_problem(D, N, 80, 0.05, seed=7)
    idx = p1.idx                                    # one mask for both tasks
    phi, _, _ = sbl.dct_dictionary(idx, D)
    Y = np.stack([phi(p1.z), phi(p2.z)]) + 0.05 * np.random.default_rng(8).standard_normal((2, N))
    Y32 = Y.astype(np.float32)
    op = api.DctOperator(torch.from_numpy(idx).cuda(), D)
    p = api.params(vec_dtype=B.COFEM_F32, K=16, em_iters=3, cg_tol=1e-6, cg_max_iters=100,
                   fixed_cg_iters=8, seed=9)
    r = api.fit(op, torch.from_numpy(Y32).cuda(), p1.beta, p)
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dct(idx, D, Y32.astype(np.float64), p1.beta, 16, 3, 1e-6, 100,
                                     fixed_cg_iters=8, seed=9)
    # the FP32 bars of the other fit tests (the FP32 FFTs leave 1e-6 per
    # application; 3e-5 in mu after 3 EM iterations of 8 CG iterations)
    mu = r.mu.cpu().numpy()
    for t in range(2):
        assert rel_l2(mu[t], rmu[t]) <= 1e-4, (t, rel_l2(mu[t], rmu[t]))
    assert rel_l2(r.alpha.cpu().numpy(), ra) <= 1e-3
