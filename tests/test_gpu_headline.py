"""Fit parity at the dense workload's full shape: N = 4096, D = 32768, K = 32
probes (33 columns), BF16 Phi in the packed tile layout on the tensor cores,
autotuned pipeline, CG tol 1e-5 with residual replacement every 50
iterations -- the launch configuration that bench.py times -- against the
oracle run on the same BF16-rounded dictionary (reading R12).

The comparison covers the first E-step and M-step of Algorithm 1 (alpha = 1):
after it, the EM trajectory at this shape amplifies FP32 rounding so much
that an FP32 emulation of the oracle is itself more than 1e-2 away in mu after
two EM iterations (tests/test_tolerance_evidence.py::
test_headline_shape_trajectory_amplifies_fp32_rounding), while after one it
is 2.2e-5 away.  The whole 100-iteration fit is compared with the oracle's
own 100-iteration fit by bench.py (support and alpha at the end).  Bars: the
FP32 bars (mu 1e-4, alpha 1e-3, equal support), equal CG iteration counts.
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

CFG = datagen.CONFIGS["dense-n4096-d32768"]


@pytest.fixture(scope="module")
def headline():
    pr = datagen.dense_problem(CFG["N"], CFG["D"], CFG["n_nonzero"], CFG["sigma"], 0)
    t16, Phi64 = bf16_round(pr.Phi)
    return pr, t16, Phi64


def _operator(t16):
    N, D = t16.shape
    op = api.DenseOperator(t16.cuda())
    nb = B.cofem_dense_packed_bytes(N, D)
    packed = torch.empty(nb, dtype=torch.uint8, device="cuda")
    B.cofem_op_dense_attach_packed(op.handle, packed.data_ptr(), nb)
    nbt = B.cofem_op_dense_autotune_workspace_bytes(op.handle, CFG["K"] + 1)
    wst = torch.empty(nbt, dtype=torch.uint8, device="cuda")
    B.cofem_op_dense_autotune(op.handle, CFG["K"] + 1, wst.data_ptr(), nbt)
    return op, packed


def test_headline_shape_first_em_iteration(cuda_lib, headline):
    pr, t16, Phi64 = headline
    op, packed = _operator(t16)
    y32 = pr.y.astype(np.float32)
    kw = dict(K=CFG["K"], cg_tol=CFG["cg_tol"], cg_max_iters=CFG["cg_max_iters"],
              resid_replace_every=CFG["resid_replace_every"], seed=0)
    r = api.fit(op, torch.from_numpy(y32).cuda(), pr.beta,
                api.params(vec_dtype=B.COFEM_F32, em_iters=1, **kw))
    torch.cuda.synchronize()
    ra, rmu, rs, rst = sbl.cofem_dense(Phi64, y32.astype(np.float64), pr.beta, CFG["K"], 1,
                                       CFG["cg_tol"], CFG["cg_max_iters"],
                                       resid_replace_every=CFG["resid_replace_every"], seed=0)
    assert r.stats["cg_iters"] == rst.cg_iters
    a, mu, s = r.alpha.cpu().numpy(), r.mu.cpu().numpy(), r.s.cpu().numpy()
    assert rel_l2(mu, rmu) <= 1e-4, rel_l2(mu, rmu)
    assert rel_l2(s, rs) <= 1e-4, rel_l2(s, rs)
    eq, border = support_compare(a, ra)
    assert eq, border
    sup = (a < 1e6) & (ra < 1e6)
    assert np.max(np.abs(a[sup] - ra[sup]) / ra[sup]) <= 1e-3
