"""Batched fits (cofem_fit_batched): every problem runs its own Algorithm 1
(own CG recurrences, stop test and probes) inside shared grouped launches.
Checked per problem against the FP64 oracle and against single-problem GPU
fits of the same problem.

The cases use sigma = 0.1 (beta = 100) and 20 EM iterations: at beta = 1e4
and a handful of EM iterations these small problems amplify any FP32
rounding difference (an FP32 emulation of the oracle itself drifts by
3e-3 to 6e-3 in mu after 6 EM iterations), so no FP32 implementation could
be compared there at 1e-4; at beta = 100 the emulation stays near 1e-5."""
import numpy as np
import pytest
import torch

from oracle import sbl
from paper_2202_12808_gb300 import api
from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import bf16_round, rel_l2, support_compare

pytestmark = pytest.mark.gpu

SIZES = [128, 150, 300, 511, 640, 1000]      # N_i; D_i = 4 N_i (ragged vs every tile)


def _batch(K=16, em=20, tol=1e-5, seed0=7, sigma=0.1):
    phis, ys, betas, seeds, refs = [], [], [], [], []
    for i, N in enumerate(SIZES):
        D = 4 * N
        prob = datagen.dense_problem(N, D, max(1, D // 20), sigma, seed=seed0 + i)
        t16, Phi64 = bf16_round(prob.Phi)
        y32 = prob.y.astype(np.float32)
        phis.append(t16.cuda())
        ys.append(torch.from_numpy(y32).cuda())
        betas.append(prob.beta)
        seeds.append(1000 + i)
        refs.append((Phi64, y32.astype(np.float64), prob.beta))
    p = api.params(vec_dtype=B.COFEM_F32, K=K, em_iters=em, cg_tol=tol, cg_max_iters=400)
    return phis, ys, betas, seeds, refs, p


def test_batched_matches_oracle_per_problem(cuda_lib):
    phis, ys, betas, seeds, refs, p = _batch()
    alphas, mus, ss, st = api.fit_batched(phis, ys, betas, seeds, p)
    torch.cuda.synchronize()
    for i, (Phi64, y64, beta) in enumerate(refs):
        ra, rmu, rs, rst = sbl.cofem_dense(Phi64, y64, beta, p.K, p.em_iters, p.cg_tol,
                                           p.cg_max_iters, seed=seeds[i])
        a, mu = alphas[i].cpu().numpy(), mus[i].cpu().numpy()
        assert rel_l2(mu, rmu) <= 1e-4, (i, rel_l2(mu, rmu))
        eq, border = support_compare(a, ra)
        assert eq, (i, border)
        sup = (a < 1e6) & (ra < 1e6)
        assert np.max(np.abs(a[sup] - ra[sup]) / ra[sup]) <= 1e-3, i


def test_batched_matches_single_problem_fits(cuda_lib):
    phis, ys, betas, seeds, refs, p = _batch()
    alphas, mus, ss, st = api.fit_batched(phis, ys, betas, seeds, p)
    torch.cuda.synchronize()
    for i in range(len(phis)):
        op = api.DenseOperator(phis[i])
        ps = api.params(vec_dtype=B.COFEM_F32, K=p.K, em_iters=p.em_iters, cg_tol=p.cg_tol,
                        cg_max_iters=p.cg_max_iters, seed=seeds[i])
        r = api.fit(op, ys[i], betas[i], ps)
        torch.cuda.synchronize()
        assert rel_l2(mus[i].cpu().numpy(), r.mu.cpu().numpy()) <= 1e-4, i
        tot_b, tot_s = sum(st["cg_iters"][i]), sum(r.stats["cg_iters"])
        assert abs(tot_b - tot_s) <= 0.05 * tot_s, i


def test_batched_rejects_unsupported(cuda_lib):
    phis, ys, betas, seeds, refs, p = _batch(em=1)
    for bad in (dict(resid_replace_every=10), dict(vec_dtype=B.COFEM_F64)):
        q = api.params(K=16, em_iters=1, **bad)
        with pytest.raises(B.CofemError) as e:
            api.fit_batched(phis, ys, betas, seeds, q)
        assert e.value.code == 6
