"""Evidence, from the oracle alone, for the GPU parity bars that are looser
than the oracle's own FP64 precision.  CPU only.

Each test runs the oracle's Algorithm 1 (Sec. 3.2 CG) through
oracle/emulation.py, which changes nothing but rounding: every per-column
reduction moved by one FP64 ulp, or FP32 vectors with FP32-accumulated
products as on the GPU's FP32 path.  The figures they assert are the ones
the GPU tests cite for their bars:

* tests/test_gpu_fit.py::test_fp64_tolerance_mode_config1 -- per-E-step
  iteration counts cannot be compared, totals within 2 %, mu within 1e-5;
* tests/test_gpu_fit.py::test_per_column_stop_bf16_tensor_cores -- FP32
  probe columns need more iterations on their own, totals within 6 %;
* tests/test_gpu_batched.py -- the sigma = 0.1 cases at 20 EM iterations,
  and the bars of the sigma = 0.01 case at 50 EM iterations;
* tests/test_gpu_dct.py::test_dct_fit_fp32 -- alpha on the support at 3e-3;
* tests/test_gpu_headline.py -- the full-shape fit is compared after its
  first EM iteration only;
* tests/test_gpu_fit.py::test_fp8_dictionary_fit -- alpha on the support
  at 3e-3 with the FP8 dictionary;
* tests/test_gpu_block_cg.py -- block CG with FP32 vectors in a first
  E-step (alpha = 1): mu at 1e-2 after six iterations, the masked DCT's mu
  at 1e-3.
"""
import numpy as np
import pytest
import scipy.fft as sfft
import torch

from oracle import emulation as em
from oracle import sbl
from paper_2202_12808_gb300 import datagen
from gpu_helpers import fp8_quantize_reference, rel_l2, support_compare


def _bf16(Phi32):
    return torch.from_numpy(Phi32).to(torch.bfloat16).double().numpy()


def _alpha_dev(a, r):
    sup = (a < 1e6) & (r < 1e6)
    return float(np.max(np.abs(a[sup] - r[sup]) / r[sup]))


# ------------------------------------------------- the hooks change nothing else

@pytest.mark.parametrize("kw", [dict(), dict(stop_rule=1), dict(fixed_cg_iters=7)])
def test_emulation_without_hooks_is_the_oracle(kw):
    pr = datagen.dense_problem(60, 200, 8, 0.05, seed=3)
    Phi = pr.Phi.astype(np.float64)
    ra, rmu, rs, rst = sbl.cofem_dense(Phi, pr.y, pr.beta, 6, 4, 1e-8, 300, seed=2, **kw)
    ea, emu, es, est = em.cofem_dense(Phi, pr.y, pr.beta, 6, 4, 1e-8, 300, seed=2, **kw)
    assert est.cg_iters == rst.cg_iters
    assert np.array_equal(ea, ra) and np.array_equal(emu, rmu) and np.array_equal(es, rs)


def test_fp32_products_are_fp32_accurate():
    # FP32 accumulation of 1024 products of +-N(0,1/256) x N(0,1): relative
    # error of order sqrt(1024) 2^-24 of the column sums, far below 1e-3
    pr = datagen.dense_problem(256, 1024, 10, 0.01, seed=1)
    Phi = _bf16(pr.Phi)
    phi, phit, _ = em.fp32_dense_dictionary(Phi)
    Z = np.random.default_rng(0).standard_normal((1024, 3))
    e1 = rel_l2(phi(Z), Phi @ Z.astype(np.float32).astype(np.float64))
    e2 = rel_l2(phit(Phi @ Z), Phi.T @ (Phi @ Z).astype(np.float32).astype(np.float64))
    assert 0 < e1 < 1e-5 and 0 < e2 < 1e-5


# ------------------------------------------ FP64 tolerance mode (config 1)

def test_ulp_perturbed_reductions_move_single_esteps():
    """Config 1 (256 x 1024, K 20, 50 EM iterations, tol 1e-6), the FP64
    oracle against itself with every reduction moved by one ulp: single
    E-steps end up to 4-8 iterations apart (so per-E-step counts cannot be
    compared with any implementation whose sums run in another order), the
    total moves by well under 2 %, mu by about 1e-7."""
    c = datagen.CONFIGS["dense-fp64-n256-d1024"]
    pr = datagen.dense_problem(c["N"], c["D"], c["n_nonzero"], c["sigma"], 0)
    Phi = pr.Phi.astype(np.float64)
    args = (Phi, pr.y, pr.beta, c["K"], c["em_iters"], c["cg_tol"], c["cg_max_iters"])
    ra, rmu, rs, rst = sbl.cofem_dense(*args, seed=0)
    worst = 0
    for ps in (1, 2):
        pa, pmu, pss, pst = em.cofem_dense(*args, seed=0, dperturb=em.ulp_perturber(ps))
        d = np.abs(np.array(pst.cg_iters) - np.array(rst.cg_iters))
        worst = max(worst, int(d.max()))
        assert abs(sum(pst.cg_iters) - sum(rst.cg_iters)) <= 0.005 * sum(rst.cg_iters)
        assert rel_l2(pmu, rmu) <= 1e-6
        eq, _ = support_compare(pa, ra)
        assert eq
    assert worst >= 3


# ----------------------------------------- per-column stop, FP32 vectors

def test_fp32_per_column_stop_needs_more_iterations():
    """stop_rule = 1 at tol 1e-5 on config 1 with the BF16-rounded Phi: with
    FP32 vectors and FP32-accumulated products each probe column needs more
    iterations to reach 1e-5 of its own norm (first E-step 46 against the FP64
    oracle's 31) and the fit about 5 % more in total -- more than 2 %, less
    than the GPU test's 6 %."""
    c = datagen.CONFIGS["dense-fp64-n256-d1024"]
    pr = datagen.dense_problem(c["N"], c["D"], c["n_nonzero"], c["sigma"], 0)
    Phi = _bf16(pr.Phi)
    y32 = pr.y.astype(np.float32).astype(np.float64)
    args = (Phi, y32, pr.beta, c["K"], c["em_iters"], 1e-5, c["cg_max_iters"])
    ra, rmu, rs, rst = sbl.cofem_dense(*args, seed=0, stop_rule=1)
    ea, emu, es, est = em.cofem_dense(*args, seed=0, stop_rule=1, vround=em.fp32_round,
                                      fp32_products=True)
    assert rst.cg_iters[0] == 31 and est.cg_iters[0] >= 41
    extra = (sum(est.cg_iters) - sum(rst.cg_iters)) / sum(rst.cg_iters)
    assert 0.02 < extra < 0.06, extra
    assert rel_l2(emu, rmu) <= 1e-4


# ------------------------------------------------ batched noise level

def _batched_case(N, i, sigma, em_iters):
    prob = datagen.dense_problem(N, 4 * N, max(1, 4 * N // 20), sigma, seed=7 + i)
    Phi = _bf16(prob.Phi)
    y64 = prob.y.astype(np.float32).astype(np.float64)
    args = (Phi, y64, prob.beta, 16, em_iters, 1e-5, 400)
    ra, rmu, rs, rst = sbl.cofem_dense(*args, seed=1000 + i)
    ea, emu, es, est = em.cofem_dense(*args, seed=1000 + i, vround=em.fp32_round,
                                      fp32_products=True)
    return rel_l2(emu, rmu), _alpha_dev(ea, ra), support_compare(ea, ra)[0]


def test_batched_sigma_0p01_at_20_em_iterations_is_out_of_fp32_reach():
    """The batched GPU tests' problems (N = 128 and 511 of their sizes, D = 4N,
    K 16, tol 1e-5): after 20 EM iterations at sigma = 0.01 the FP32
    emulation of the oracle is itself more than 1e-4 away from the FP64
    oracle in mu and more than 1e-3 in alpha on the support, so no FP32
    implementation can meet those bars there; at sigma = 0.1 it stays within
    them (mu 1.3e-5, alpha 3.3e-4 at most)."""
    for N, i in ((128, 0), (511, 3)):
        e_mu, e_al, _ = _batched_case(N, i, 0.01, 20)
        assert e_mu > 1e-4 and e_al > 1e-3, (N, e_mu, e_al)
        e_mu, e_al, eq = _batched_case(N, i, 0.1, 20)
        assert e_mu <= 5e-5 and e_al <= 5e-4 and eq, (N, e_mu, e_al)


def test_batched_sigma_0p01_at_50_em_iterations_bars():
    """At the batched workload's own noise level (sigma 0.01) and 50 EM
    iterations the trajectory has settled: the FP32 emulation meets mu 1e-4
    and the support exactly, but alpha on the support moves by up to 2e-3
    (1.6e-3 and 2.0e-3 here), which sets the GPU case's alpha bar at 5e-3."""
    worst = 0.0
    for N, i in ((128, 0), (511, 3)):
        e_mu, e_al, eq = _batched_case(N, i, 0.01, 50)
        assert e_mu <= 2e-5 and eq, (N, e_mu)
        worst = max(worst, e_al)
    assert 1e-3 < worst < 3e-3, worst


def test_batched_fixed_iterations_fp32_error():
    """tests/test_gpu_batched.py::test_batched_split_k_products: six fixed CG
    iterations per E-step, two E-steps, sigma 0.1.  The iterates are smooth
    functions of the products there: FP32 vectors move mu by about 2.4e-7 with
    exact products and by 1.5e-6 to 2.6e-6 with FP32-accumulated ones, so the
    GPU bar of 5e-5 leaves room only for accumulation-order effects (the GPU's
    split-K partials add over other lengths), not for a wrong K range."""
    for i, (N, D) in ((1, (150, 600)), (3, (2048, 8192))):
        prob = datagen.dense_problem(N, D, max(1, D // 20), 0.1, seed=7 + i)
        Phi = _bf16(prob.Phi)
        y64 = prob.y.astype(np.float32).astype(np.float64)
        args = (Phi, y64, prob.beta, 16, 2, 1e-5, 400)
        ra, rmu, rs, rst = sbl.cofem_dense(*args, seed=1000 + i, fixed_cg_iters=6)
        ea, emu, es, est = em.cofem_dense(*args, seed=1000 + i, fixed_cg_iters=6,
                                          vround=em.fp32_round)
        fa, fmu, fs, fst = em.cofem_dense(*args, seed=1000 + i, fixed_cg_iters=6,
                                          vround=em.fp32_round, fp32_products=True)
        assert rel_l2(emu, rmu) < 5e-7
        assert 5e-7 < rel_l2(fmu, rmu) < 5e-6


# ---------------------------------------------------------- masked DCT

def test_dct_alpha_sensitivity():
    """D = 4096, N = 1024, 0.04 D coefficients, sigma 0.01, K 20, 20 EM
    iterations (tests/test_gpu_dct.py::test_dct_fit_fp32): every coordinate is
    still in the support and alpha follows the truncated probe solves -- the
    oracle's own alpha moves by more than 1e-2 between tolerance 1e-5 and
    1e-6 -- and FP32 vectors with FP32 transforms move it by 3e-4 to 7e-4,
    within the GPU bar of 3e-3 but near 1e-3."""
    D, N = 4096, 1024
    worst = 0.0
    for seed in (0, 1):
        p = datagen.dct_problem(D, N, int(0.04 * D), 0.01, seed=seed)
        y32 = p.y.astype(np.float32).astype(np.float64)
        ra, rmu, rs, rst = sbl.cofem_dct(p.idx, D, y32, p.beta, 20, 20, 1e-5, 400, seed=seed)
        ra6, _, _, _ = sbl.cofem_dct(p.idx, D, y32, p.beta, 20, 20, 1e-6, 400, seed=seed)
        assert _alpha_dev(ra6, ra) > 1e-2
        idx = p.idx

        def phi(Z):
            return sfft.idct(np.asarray(Z).astype(np.float32), type=2, norm="ortho",
                             axis=0)[idx].astype(np.float64)

        def phit(W):
            T = np.zeros((D,) + W.shape[1:], dtype=np.float32)
            T[idx] = W.astype(np.float32)
            return sfft.dct(T, type=2, norm="ortho", axis=0).astype(np.float64)

        ea, emu, es, est = em.cofem(phi, phit, D, y32, p.beta, 20, 20, 1e-5, 400, seed=seed,
                                    vround=em.fp32_round)
        assert rel_l2(emu, rmu) <= 1e-4
        worst = max(worst, _alpha_dev(ea, ra))
    assert 2e-4 < worst < 3e-3, worst


# ---------------------------------------- the headline shape (4096 x 32768)

@pytest.mark.many_blas_threads
def test_headline_shape_trajectory_amplifies_fp32_rounding():
    """N = 4096, D = 32768, K = 32, tol 1e-5, BF16-rounded Phi: after the
    first EM iteration the FP32 emulation of the oracle is 2e-5 away in mu,
    after the second already more than 1e-2 -- the second E-step's solve
    stops at relres 1e-5 on a far worse conditioned A, whose iterate then
    depends on rounding at the level of cond(A) x 1e-5.  So the full-shape
    GPU fit is compared with the oracle after one EM iteration."""
    c = datagen.CONFIGS["dense-n4096-d32768"]
    pr = datagen.dense_problem(c["N"], c["D"], c["n_nonzero"], c["sigma"], 0)
    Phi = _bf16(pr.Phi)
    y64 = pr.y.astype(np.float32).astype(np.float64)
    args = (Phi, y64, pr.beta, c["K"], 2, c["cg_tol"], c["cg_max_iters"])
    r1 = sbl.cofem_dense(*args[:4], 1, *args[5:], seed=0)
    e1 = em.cofem_dense(*args[:4], 1, *args[5:], seed=0, vround=em.fp32_round,
                        fp32_products=True)
    assert rel_l2(e1[1], r1[1]) <= 1e-4
    r2 = sbl.cofem_dense(*args, seed=0)
    e2 = em.cofem_dense(*args, seed=0, vround=em.fp32_round, fp32_products=True)
    assert e2[3].cg_iters == r2[3].cg_iters
    assert rel_l2(e2[1], r2[1]) > 1e-2


def test_fp8_dictionary_alpha_sensitivity():
    """Config 1 with the dictionary an FP8 handle applies (E4M3, power-of-two
    tile scales, bf16(q x scale)): the FP32 emulation of the oracle stays
    within the FP32 bars for mu (6e-6) and the support, but moves alpha on
    the support by 1.3e-3, past the 1e-3 bar -- so the FP8 fit's alpha bar
    is 3e-3."""
    c = datagen.CONFIGS["dense-fp64-n256-d1024"]
    pr = datagen.dense_problem(c["N"], c["D"], c["n_nonzero"], c["sigma"], 0)
    _, _, Phi = fp8_quantize_reference(pr.Phi)
    y32 = pr.y.astype(np.float32).astype(np.float64)
    args = (Phi, y32, pr.beta, c["K"], c["em_iters"], c["cg_tol"], c["cg_max_iters"])
    ra, rmu, rs, rst = sbl.cofem_dense(*args, seed=0)
    ea, emu, es, est = em.cofem_dense(*args, seed=0, vround=em.fp32_round, fp32_products=True)
    assert rel_l2(emu, rmu) <= 1e-4
    assert support_compare(ea, ra)[0]
    assert 1e-3 < _alpha_dev(ea, ra) < 3e-3


# ------------------------------------------------- block CG (solver variant)

def test_block_emulation_without_hooks_is_the_oracle():
    rng = np.random.default_rng(3)
    Phi = rng.standard_normal((40, 120)) / np.sqrt(40)
    y = rng.standard_normal(40)
    kw = dict(seed=2, solver=1)
    r = sbl.cofem_dense(Phi, y, 50.0, 6, 4, 1e-8, 200, **kw)
    e = em.cofem_dense(Phi, y, 50.0, 6, 4, 1e-8, 200, **kw)
    for a, b in zip(r[:3], e[:3]):
        assert np.array_equal(a, b)
    assert r[3].cg_iters == e[3].cg_iters


def test_block_cg_fp32_first_e_step_amplifies_rounding():
    """N = 512, D = 8192, K = 32 (33 columns), sigma 0.01, t = 1: A = beta
    Phi^T Phi + I has the eigenvalue 1 on the 7680-dimensional null space of
    Phi and beta-sized ones on its range.  Block CG builds the mean column
    from the probes' directions, whose null-space parts are large, so FP32
    rounding reaches mu: after two iterations it is 6e-6 away from the FP64
    iterate, after six 2.8e-3 -- while column-wise CG in FP32, whose mean
    column stays in the range, is 2e-6 away.  The GPU's block CG gives 8e-6
    and 3.5e-3 here (tests/test_gpu_block_cg.py::
    test_block_fp32_fixed_iterations_multichunk, bar 1e-2)."""
    prob = datagen.dense_problem(512, 8192, 8192 // 20, 0.01, 0)
    Phi = prob.Phi.astype(np.float64)
    y32 = prob.y.astype(np.float32).astype(np.float64)
    out = {}
    for k in (2, 6):
        for solver in (0, 1):
            r = sbl.cofem_dense(Phi, y32, prob.beta, 32, 1, 1e-6, 400, fixed_cg_iters=k,
                                seed=3, solver=solver)
            e = em.cofem_dense(Phi, y32, prob.beta, 32, 1, 1e-6, 400, fixed_cg_iters=k,
                               seed=3, solver=solver, vround=em.fp32_round,
                               fp32_products=True)
            out[k, solver] = rel_l2(e[1], r[1])
    assert out[2, 1] <= 1e-4
    assert 1e-3 <= out[6, 1] <= 1e-2
    assert out[6, 0] <= 1e-5


def test_block_cg_dct_fp32_mu():
    """The masked DCT (D = 4096, N = 1024, 0.04 D coefficients, sigma 0.01,
    K 20, 10 EM iterations, tol 1e-5) with block CG: Phi Phi^T = I, so A has
    just the eigenvalues 1 and beta + alpha at t = 1, and FP32 vectors with
    FP32 transforms leave mu 2.3e-4 from the FP64 block fit (the GPU: 3e-4;
    tests/test_gpu_block_cg.py::test_block_dct_fp32, bar 1e-3)."""
    D, N = 4096, 1024
    p = datagen.dct_problem(D, N, int(0.04 * D), 0.01, seed=0)
    y32 = p.y.astype(np.float32).astype(np.float64)
    idx = p.idx

    def phi(Z):
        return sfft.idct(np.asarray(Z).astype(np.float32), type=2, norm="ortho",
                         axis=0)[idx].astype(np.float64)

    def phit(W):
        T = np.zeros((D,) + W.shape[1:], dtype=np.float32)
        T[idx] = W.astype(np.float32)
        return sfft.dct(T, type=2, norm="ortho", axis=0).astype(np.float64)

    ra, rmu, rs, rst = sbl.cofem_dct(idx, D, y32, p.beta, 20, 10, 1e-5, 400, seed=0, solver=1)
    ea, emu, es, est = em.cofem(phi, phit, D, y32, p.beta, 20, 10, 1e-5, 400, seed=0,
                                solver=1, vround=em.fp32_round)
    assert 1e-4 <= rel_l2(emu, rmu) <= 1e-3
