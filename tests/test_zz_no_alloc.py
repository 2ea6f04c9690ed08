"""cofem_op_apply_noalloc: the operator application for callers that may not
allocate device memory (a plugin inside an application that owns the whole
device memory pool, a loop that must not synchronise on an allocation).  It
takes its scratch from a static array inside the library instead of a
caller-provided workspace.

Checked through the C ABI against cofem_op_apply (which uses a workspace the
test allocates) on two calls in a row with different inputs, so stale scratch
contents from the first call would show up in the second; with the same
per-column tolerances as the other operator tests.  This file is collected
last so that a failure here stops a `-x` run only after every other test.
"""
import numpy as np
import pytest
import torch

from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import bf16_round, phi_tensor, rel_l2, to_block, from_block

pytestmark = pytest.mark.gpu


def _reference_apply(op, vec, Xb, ld, ncols, al, beta):
    n = B.cofem_apply_workspace_bytes(op, vec, ncols)
    ws = torch.empty(max(n, 256), dtype=torch.uint8, device="cuda")
    Y = torch.empty_like(Xb)
    B.cofem_op_apply(op, vec, Xb.data_ptr(), ld, ncols, al.data_ptr(), beta, Y.data_ptr(),
                     ws.data_ptr(), ws.numel())
    return Y


@pytest.mark.parametrize("kind,N,D,ncols", [("bf16", 1000, 4000, 33), ("bf16", 4096, 32768, 33),
                                            ("f32", 300, 1200, 21), ("f64", 256, 1024, 21)])
def test_noalloc_matches_workspace_entry_point(cuda_lib, kind, N, D, ncols):
    prob = datagen.dense_problem(N, D, max(1, D // 50), 0.01, seed=N)
    if kind == "bf16":
        _, Phi = bf16_round(prob.Phi)
        Phi_t, ldp = phi_tensor(Phi, torch.bfloat16)
        pdt, vec, vdt, tol = B.COFEM_BF16, B.COFEM_F32, torch.float32, 2e-5
    elif kind == "f32":
        Phi_t, ldp = phi_tensor(prob.Phi, torch.float32)
        pdt, vec, vdt, tol = B.COFEM_F32, B.COFEM_F32, torch.float32, 2e-5
    else:
        Phi_t, ldp = phi_tensor(prob.Phi.astype(np.float64), torch.float64)
        pdt, vec, vdt, tol = B.COFEM_F64, B.COFEM_F64, torch.float64, 1e-12
    op = B.cofem_op_dense(N, D, pdt, Phi_t.data_ptr(), ldp)
    try:
        rng = np.random.default_rng(ncols + N)
        al = torch.from_numpy(rng.uniform(0.5, 100.0, D)).cuda()
        beta = 1e4
        for call in range(2):                       # two calls in a row
            X = rng.standard_normal((D, ncols)) * (1.0 + 10.0 * call)
            Xb, ld = to_block(X, vdt)
            ref = _reference_apply(op, vec, Xb, ld, ncols, al, beta)
            Y = torch.full_like(Xb, float("nan"))
            B.cofem_op_apply_noalloc(op, vec, Xb.data_ptr(), ld, ncols, al.data_ptr(), beta,
                                     Y.data_ptr())
            torch.cuda.synchronize()
            got, want = from_block(Y, D), from_block(ref, D)
            assert np.all(np.isfinite(got))
            for j in range(ncols):
                assert rel_l2(got[:, j], want[:, j]) <= tol, (call, j)
    finally:
        B.cofem_op_destroy(op)


def test_noalloc_rejects_problems_beyond_its_scratch(cuda_lib):
    # a BF16 operator of 8192 x 262144 with 64 columns needs far more than the
    # static scratch; the call must refuse before launching anything
    N, D = 8192, 262144
    Phi_t = torch.empty((1, 64), dtype=torch.bfloat16, device="cuda")   # never read
    op = B.cofem_op_dense(N, D, B.COFEM_BF16, Phi_t.data_ptr(), D)
    try:
        cap = B.cofem_noalloc_scratch_capacity()
        assert B.cofem_apply_workspace_bytes(op, B.COFEM_F32, 64) > cap
        x = torch.empty(8, dtype=torch.float32, device="cuda")
        with pytest.raises(B.CofemError) as e:
            B.cofem_op_apply_noalloc(op, B.COFEM_F32, x.data_ptr(), D, 64, x.data_ptr(), 1.0,
                                     x.data_ptr())
        assert e.value.code == 7
        assert "static scratch" in B.lib().cofem_last_error().decode()
    finally:
        B.cofem_op_destroy(op)
