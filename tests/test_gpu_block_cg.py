"""Block CG on the GPU (params.solver = 1) against the oracle's block CG
(oracle/sbl.py::block_cg_solve, pinned in tests/test_oracle_block_cg.py) on
the same seeded inputs, through the C ABI.

Bars:
  FP64 vectors, a fixed number of iterations in one E-step: mu, s <= 1e-9
      (the iterate is the block-Krylov Galerkin solution, unique), at 21
      and 33 columns, with one and with several staged chunks per block.
  FP64 vectors, tol 1e-12: mu, s <= 1e-9 and equal support over 10 EM
      iterations.
  FP32 vectors (CUDA-core FP32, FP32 on the tensor cores as hi + lo, BF16):
      mu <= 1e-4, alpha on the support <= 1e-3, equal support -- the bars of
      the column-wise FP32 fits -- and fewer CG iterations in total than the
      column-wise GPU fit of the same problem.
"""
import numpy as np
import pytest
import torch

from oracle import sbl
from paper_2202_12808_gb300 import api
from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import bf16_round, rel_l2, support_compare

pytestmark = pytest.mark.gpu


def _problem(N=256, D=1024, nnz=51, sigma=0.01, seed=0):
    return datagen.dense_problem(N, D, nnz, sigma, seed)


def _hi_lo(Phi32):
    hi = torch.from_numpy(Phi32).to(torch.bfloat16)
    lo = (torch.from_numpy(Phi32) - hi.float()).to(torch.bfloat16)
    return hi.double().numpy() + lo.double().numpy()


def _op(Phi, dtype, packed=False):
    op = api.DenseOperator(torch.from_numpy(np.ascontiguousarray(Phi)).to("cuda", dtype))
    if packed:
        nb = B.cofem_op_dense_packed_bytes(op.handle)
        op.packed = torch.empty(nb, dtype=torch.uint8, device="cuda")
        B.cofem_op_dense_attach_packed(op.handle, op.packed.data_ptr(), nb)
    return op


def _fit(op, y, beta, vec, **kw):
    p = api.params(vec_dtype=vec, **kw)
    ydt = torch.float64 if vec == B.COFEM_F64 else torch.float32
    r = api.fit(op, torch.from_numpy(np.asarray(y)).to("cuda", ydt), beta, p)
    torch.cuda.synchronize()
    return r.alpha.cpu().numpy(), r.mu.cpu().numpy(), r.s.cpu().numpy(), r.stats


@pytest.mark.parametrize("k", [1, 8, 13])
def test_block_fp64_fixed_iterations_one_e_step(cuda_lib, k):
    """At t = 1 (alpha = 1) A = beta Phi^T Phi + I has the eigenvalue 1 on
    the 768-dimensional null space of Phi and 256 others, so 21 right-hand
    sides exhaust the block Krylov space after 14 iterations (the oracle's
    relative residual: 9.2e-6 after 13, 2.0e-14 after 14); k stays below."""
    prob = _problem()
    Phi = prob.Phi.astype(np.float64)
    op = _op(Phi, torch.float64)
    a, mu, s, st = _fit(op, prob.y, prob.beta, B.COFEM_F64, K=20, em_iters=1, cg_tol=1e-6,
                        cg_max_iters=400, fixed_cg_iters=k, seed=3, solver=1)
    ra, rmu, rs, rst = sbl.cofem_dense(Phi, prob.y, prob.beta, 20, 1, 1e-6, 400,
                                       fixed_cg_iters=k, seed=3, solver=1)
    assert st["cg_iters"] == [k]
    assert rel_l2(mu, rmu) <= 1e-9, rel_l2(mu, rmu)
    assert rel_l2(s, rs) <= 1e-9, rel_l2(s, rs)


@pytest.mark.parametrize("N,D,K", [(256, 1024, 32), (512, 8192, 20), (512, 8192, 32)])
def test_block_fp64_fixed_iterations_shapes(cuda_lib, N, D, K):
    """K + 1 = 33 columns take the 36-wide kernels; D = 8192 gives each gram
    block several staged 32-row chunks (256 chunks over at most one block
    per SM)."""
    prob = _problem(N=N, D=D, nnz=D // 20)
    Phi = prob.Phi.astype(np.float64)
    op = _op(Phi, torch.float64)
    k = 6
    a, mu, s, st = _fit(op, prob.y, prob.beta, B.COFEM_F64, K=K, em_iters=1, cg_tol=1e-6,
                        cg_max_iters=400, fixed_cg_iters=k, seed=3, solver=1)
    ra, rmu, rs, rst = sbl.cofem_dense(Phi, prob.y, prob.beta, K, 1, 1e-6, 400,
                                       fixed_cg_iters=k, seed=3, solver=1)
    assert rel_l2(mu, rmu) <= 1e-9, rel_l2(mu, rmu)
    assert rel_l2(s, rs) <= 1e-9, rel_l2(s, rs)


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_block_fp32_fixed_iterations_multichunk(cuda_lib, kind):
    """FP32 vectors at 512 x 8192 with 33 columns (several staged chunks per
    gram block), first E-step after 2 and 6 iterations: CUDA-core FP32
    dictionary and BF16 on the tensor cores."""
    prob = _problem(N=512, D=8192, nnz=8192 // 20)
    if kind == "f32":
        Phi_ref, tdt, Phi_in = prob.Phi.astype(np.float64), torch.float32, prob.Phi
    else:
        _, Phi_ref = bf16_round(prob.Phi)
        tdt, Phi_in = torch.bfloat16, Phi_ref
    y32 = prob.y.astype(np.float32).astype(np.float64)
    op = _op(Phi_in, tdt)
    for k in (2, 6):
        a, mu, s, st = _fit(op, y32, prob.beta, B.COFEM_F32, K=32, em_iters=1, cg_tol=1e-6,
                            cg_max_iters=400, fixed_cg_iters=k, seed=3, solver=1)
        ra, rmu, rs, rst = sbl.cofem_dense(Phi_ref, y32, prob.beta, 32, 1, 1e-6, 400,
                                           fixed_cg_iters=k, seed=3, solver=1)
        # mu: 1e-4 after two iterations, 1e-2 after six -- FP32 rounding
        # reaches the mean column through the probes' null-space directions
        # (tests/test_tolerance_evidence.py::
        # test_block_cg_fp32_first_e_step_amplifies_rounding: the FP32
        # emulation of the oracle is 6e-6 and 2.8e-3 away)
        assert rel_l2(mu, rmu) <= (1e-4 if k == 2 else 1e-2), rel_l2(mu, rmu)
        assert rel_l2(s, rs) <= 1e-4, rel_l2(s, rs)


def test_block_fp64_tight_tolerance(cuda_lib):
    prob = _problem()
    Phi = prob.Phi.astype(np.float64)
    op = _op(Phi, torch.float64)
    a, mu, s, st = _fit(op, prob.y, prob.beta, B.COFEM_F64, K=20, em_iters=10, cg_tol=1e-12,
                        cg_max_iters=1000, seed=5, solver=1)
    ra, rmu, rs, rst = sbl.cofem_dense(Phi, prob.y, prob.beta, 20, 10, 1e-12, 1000, seed=5,
                                       solver=1)
    print("cg iters gpu", st["cg_iters"], "oracle", rst.cg_iters)
    assert rel_l2(mu, rmu) <= 1e-9, rel_l2(mu, rmu)
    assert rel_l2(s, rs) <= 1e-9, rel_l2(s, rs)
    eq, _ = support_compare(a, ra)
    assert eq
    assert abs(sum(st["cg_iters"]) - sum(rst.cg_iters)) <= 0.1 * sum(rst.cg_iters)


def test_block_fp64_multitask(cuda_lib):
    """T = 2 tasks sharing alpha: B = [b_1 b_2 | probes] in one block."""
    rng = np.random.default_rng(4)
    N, D, T = 128, 512, 2
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    Z = np.zeros((T, D))
    sup = rng.choice(D, 20, replace=False)
    Z[:, sup] = rng.standard_normal((T, 20))
    Y = Z @ Phi.T + 0.01 * rng.standard_normal((T, N))
    beta = 1e4
    op = _op(Phi, torch.float64)
    p = api.params(vec_dtype=B.COFEM_F64, K=16, em_iters=8, cg_tol=1e-12, cg_max_iters=1000,
                   seed=2, solver=1)
    r = api.fit(op, torch.from_numpy(Y).cuda(), beta, p)
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dense(Phi, Y, beta, 16, 8, 1e-12, 1000, seed=2, solver=1)
    assert rel_l2(r.mu.cpu().numpy(), rmu) <= 1e-9
    assert rel_l2(r.s.cpu().numpy(), rs) <= 1e-9


@pytest.mark.parametrize("phi_kind", ["f32", "f32-tc", "bf16"])
def test_block_fp32_tolerance_mode(cuda_lib, phi_kind):
    prob = _problem()
    packed = phi_kind == "f32-tc"
    if phi_kind == "f32":
        Phi_ref, tdt, Phi_in = prob.Phi.astype(np.float64), torch.float32, prob.Phi
    elif packed:
        Phi_ref, tdt, Phi_in = _hi_lo(prob.Phi), torch.float32, prob.Phi
    else:
        _, Phi_ref = bf16_round(prob.Phi)
        tdt, Phi_in = torch.bfloat16, Phi_ref
    y32 = prob.y.astype(np.float32).astype(np.float64)
    kw = dict(K=20, em_iters=50, cg_tol=1e-6, cg_max_iters=400, seed=0)
    op = _op(Phi_in, tdt, packed)
    a, mu, s, st = _fit(op, y32, prob.beta, B.COFEM_F32, solver=1, **kw)
    a0, mu0, s0, st0 = _fit(op, y32, prob.beta, B.COFEM_F32, solver=0, **kw)
    ra, rmu, rs, rst = sbl.cofem_dense(Phi_ref, y32, prob.beta, 20, 50, 1e-6, 400, seed=0,
                                       solver=1)
    print("cg iters block", sum(st["cg_iters"]), "column", sum(st0["cg_iters"]),
          "oracle block", sum(rst.cg_iters))
    eq, border = support_compare(a, ra)
    assert eq, border
    assert rel_l2(mu, rmu) <= 1e-4, rel_l2(mu, rmu)
    sup = (ra < 1e6) & (a < 1e6)
    assert np.max(np.abs(a[sup] - ra[sup]) / ra[sup]) <= 1e-3
    assert sum(st["cg_iters"]) < sum(st0["cg_iters"])
    assert max(st["relres"]) < 1e-6


@pytest.mark.parametrize("tol", [1e-5, 1e-6])
def test_block_dct_fp32(cuda_lib, tol):
    D, N = 4096, 1024
    p = datagen.dct_problem(D, N, int(0.04 * D), 0.01, seed=0)
    op = api.DctOperator(torch.from_numpy(p.idx).cuda(), D)
    y32 = p.y.astype(np.float32)
    prm = api.params(vec_dtype=B.COFEM_F32, K=20, em_iters=10, cg_tol=tol, cg_max_iters=400,
                     seed=0, solver=1)
    r = api.fit(op, torch.from_numpy(y32).cuda(), p.beta, prm)
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dct(p.idx, D, y32.astype(np.float64), p.beta, 20, 10, tol, 400,
                                     seed=0, solver=1)
    # mu at 1e-3: at t = 1 A has only the eigenvalues 1 and beta + 1, and
    # FP32 rounding reaches the mean column through the probes (an FP32
    # emulation of the oracle's block fit is 2.3e-4 away:
    # tests/test_tolerance_evidence.py::test_block_cg_dct_fp32_mu)
    assert rel_l2(r.mu.cpu().numpy(), rmu) <= 1e-3, rel_l2(r.mu.cpu().numpy(), rmu)
    eq, border = support_compare(r.alpha.cpu().numpy(), ra)
    assert eq, border


@pytest.mark.parametrize("vec", [B.COFEM_F64, B.COFEM_F32])
def test_block_zero_y_is_deflated(cuda_lib, vec):
    """y = 0 makes b = 0 a zero right-hand side, so B^T B is singular: the
    start's factorisation drops that index, mu stays exactly 0 and the
    probe columns are solved as in the oracle (whose Householder QR gives
    the zero column a zero row of C)."""
    prob = _problem(N=64, D=256, nnz=8)
    Phi = prob.Phi.astype(np.float64)
    dt = torch.float64 if vec == B.COFEM_F64 else torch.float32
    tol, bar = (1e-12, 1e-9) if vec == B.COFEM_F64 else (1e-6, 1e-4)
    op = _op(Phi, dt)
    a, mu, s, st = _fit(op, np.zeros(64), prob.beta, vec, K=8, em_iters=2, cg_tol=tol,
                        cg_max_iters=400, seed=1, solver=1)
    ra, rmu, rs, rst = sbl.cofem_dense(Phi, np.zeros(64), prob.beta, 8, 2, tol, 400, seed=1,
                                       solver=1)
    assert not np.any(mu) and not np.any(rmu)
    assert rel_l2(s, rs) <= bar, rel_l2(s, rs)
    assert np.all(np.isfinite(a))


def _headline_op():
    c = datagen.CONFIGS["dense-n4096-d32768"]
    prob = datagen.dense_problem(c["N"], c["D"], c["n_nonzero"], c["sigma"], 0)
    hi, Phi_ref = bf16_round(prob.Phi)
    op = _op(Phi_ref, torch.bfloat16, packed=True)
    nbt = B.cofem_op_dense_autotune_workspace_bytes(op.handle, c["K"] + 1)
    wst = torch.empty(nbt, dtype=torch.uint8, device="cuda")
    B.cofem_op_dense_autotune(op.handle, c["K"] + 1, wst.data_ptr(), nbt)
    del wst
    return c, prob, Phi_ref, op


@pytest.mark.parametrize("k", [1, 3])
def test_block_headline_shape_fixed_iterations(cuda_lib, k):
    """4096 x 32768, K = 32, BF16 dictionary packed on the tensor cores: the
    first E-step after k block iterations against the oracle's (the
    Galerkin iterate) on the BF16-rounded dictionary."""
    c, prob, Phi_ref, op = _headline_op()
    y32 = prob.y.astype(np.float32).astype(np.float64)
    a, mu, s, st = _fit(op, y32, prob.beta, B.COFEM_F32, K=c["K"], em_iters=1, cg_tol=1e-6,
                        cg_max_iters=400, fixed_cg_iters=k, seed=0, solver=1)
    ra, rmu, rs, rst = sbl.cofem_dense(Phi_ref, y32, prob.beta, c["K"], 1, 1e-6, 400,
                                       fixed_cg_iters=k, seed=0, solver=1)
    assert rel_l2(mu, rmu) <= 1e-4, rel_l2(mu, rmu)
    assert rel_l2(s, rs) <= 1e-4, rel_l2(s, rs)


def test_block_headline_shape_first_e_step(cuda_lib):
    """The same in tolerance mode (tol 1e-5), checked against what the
    joint stop test guarantees: ||b - A mu|| <= tol ||B||_F (with a factor 2
    for the drift between the recursive and the true residual in FP32).
    The test does not pin mu itself here: at t = 1 the 28672-dimensional
    null space of Phi has the eigenvalue 1 against beta-sized ones on its
    range, so a mean-column residual inside the bound can still move mu by
    up to tol ||B||_F / 1 = 7.7, a third of ||mu||.  Column-wise CG keeps
    that residual in the range and lands within 1e-5 of the oracle; block CG
    mixes in the probes' null-space directions, and its FP32 iterate moves
    with rounding (the FP32 emulation of the oracle: 8e-4 after 8
    iterations at 1024 x 8192 already; the GPU: 7 % after 22)."""
    c, prob, Phi_ref, op = _headline_op()
    y32 = prob.y.astype(np.float32).astype(np.float64)
    a, mu, s, st = _fit(op, y32, prob.beta, B.COFEM_F32, K=c["K"], em_iters=1,
                        cg_tol=c["cg_tol"], cg_max_iters=c["cg_max_iters"], seed=0, solver=1)
    ra, rmu, rs, rst = sbl.cofem_dense(Phi_ref, y32, prob.beta, c["K"], 1, c["cg_tol"],
                                       c["cg_max_iters"], seed=0, solver=1)
    b = prob.beta * (Phi_ref.T @ y32)
    norm_B = np.sqrt(b @ b + c["K"] * c["D"])
    Amu = prob.beta * (Phi_ref.T @ (Phi_ref @ mu)) + mu
    res = np.linalg.norm(b - Amu) / norm_B
    print("tolerance mode iters", st["cg_iters"], rst.cg_iters, "relres", st["relres"],
          "true mean-column residual %.2e" % res, "mu %.2e s %.2e" % (rel_l2(mu, rmu), rel_l2(s, rs)))
    assert st["relres"][0] < c["cg_tol"]
    assert res <= 2 * c["cg_tol"], res
    assert rel_l2(s, rs) <= 1e-3, rel_l2(s, rs)


def test_block_refused_by_batched_fit(cuda_lib):
    prob = _problem(N=64, D=256, nnz=8)
    Phi = torch.from_numpy(prob.Phi).cuda().to(torch.bfloat16)
    y = torch.from_numpy(prob.y.astype(np.float32)).cuda()
    pr = B.cofem_problem(N=64, D=256, phi_dev=Phi.data_ptr(), ld=256, y_dev=y.data_ptr(),
                         beta=prob.beta, seed=0)
    with pytest.raises(B.CofemError) as e:
        B.cofem_batched_workspace_bytes([pr], api.params(K=8, solver=1))
    assert e.value.code == 6        # COFEM_ERR_UNSUPPORTED
