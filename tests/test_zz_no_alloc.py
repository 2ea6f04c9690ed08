"""cofem_op_apply_noalloc: the operator application for callers that may not
allocate device memory (a plugin inside an application that owns the whole
device memory pool, a loop that must not synchronise on an allocation).  It
takes its scratch from a static array inside the library instead of a
caller-provided workspace.

Checked through the C ABI against cofem_op_apply (which uses a workspace the
test allocates) on two calls in a row with different inputs, so stale scratch
contents from the first call would show up in the second.  Both entry points
run the same kernels on the same inputs with fixed-order reductions, so the
results must be bitwise equal.  The structured operators (convolution,
masked DCT), whose scratch holds tables and intermediates rebuilt on every
call, run after a dense call has left other data in the shared array.  This
file is collected last so that a failure here stops a `-x` run only after
every other test.
"""
import numpy as np
import pytest
import torch

from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import bf16_round, phi_tensor, to_block, from_block

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
        pdt, vec, vdt = B.COFEM_BF16, B.COFEM_F32, torch.float32
    elif kind == "f32":
        Phi_t, ldp = phi_tensor(prob.Phi, torch.float32)
        pdt, vec, vdt = B.COFEM_F32, B.COFEM_F32, torch.float32
    else:
        Phi_t, ldp = phi_tensor(prob.Phi.astype(np.float64), torch.float64)
        pdt, vec, vdt = B.COFEM_F64, B.COFEM_F64, torch.float64
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
            got = from_block(Y, D)
            assert np.all(np.isfinite(got))
            assert torch.equal(Y[:, :D], ref[:, :D]), (call, float((Y[:, :D] - ref[:, :D]).abs().max()))
    finally:
        B.cofem_op_destroy(op)


def _two_calls_match(op, D, ncols, seed):
    """Two noalloc applications in a row (different inputs) against the
    workspace entry point, bitwise, FP32 vectors."""
    rng = np.random.default_rng(seed)
    al = torch.from_numpy(rng.uniform(0.5, 100.0, D)).cuda()
    for call in range(2):
        X = rng.standard_normal((D, ncols)) * (1.0 + 10.0 * call)
        Xb, ld = to_block(X, torch.float32)
        ref = _reference_apply(op, B.COFEM_F32, Xb, ld, ncols, al, 400.0)
        Y = torch.full_like(Xb, float("nan"))
        B.cofem_op_apply_noalloc(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, al.data_ptr(), 400.0,
                                 Y.data_ptr())
        torch.cuda.synchronize()
        assert torch.isfinite(Y[:, :D]).all()
        assert torch.equal(Y[:, :D], ref[:, :D]), call


def _dirty_scratch_with_a_dense_call():
    prob = datagen.dense_problem(512, 4096, 40, 0.01, seed=3)
    Phi_t, ldp = phi_tensor(bf16_round(prob.Phi)[1], torch.bfloat16)
    op = B.cofem_op_dense(512, 4096, B.COFEM_BF16, Phi_t.data_ptr(), ldp)
    try:
        X = torch.randn((17, 4096), device="cuda") * 1e3
        al = torch.full((4096,), 3.0, dtype=torch.float64, device="cuda")
        Y = torch.empty_like(X)
        B.cofem_op_apply_noalloc(op, B.COFEM_F32, X.data_ptr(), 4096, 17, al.data_ptr(), 1e4,
                                 Y.data_ptr())
        torch.cuda.synchronize()
    finally:
        B.cofem_op_destroy(op)


def test_noalloc_conv_after_dense(cuda_lib):
    L, C, T, ncols = 4160, 8, 64, 17
    h = torch.from_numpy(datagen.conv_problem(L, C, T, 0.01, 0.05, seed=2).h).cuda()
    _dirty_scratch_with_a_dense_call()
    op = B.cofem_op_conv1d(L, C, T, h.data_ptr())
    try:
        _two_calls_match(op, C * L, ncols, 11)
    finally:
        B.cofem_op_destroy(op)


def test_noalloc_conv_tensor_cores_after_dense(cuda_lib):
    # the convolution on the tensor cores: its Toeplitz images and the FP32
    # copy of alpha are written into the same scratch on every call
    L, C, T, ncols = 8256, 8, 64, 17
    h = torch.from_numpy(datagen.conv_problem(L, C, T, 0.01, 0.05, seed=7).h).cuda()
    _dirty_scratch_with_a_dense_call()
    op = B.cofem_op_conv1d(L, C, T, h.data_ptr())
    B.cofem_op_conv1d_set_tensor_cores(op, 1)
    try:
        _two_calls_match(op, C * L, ncols, 13)
    finally:
        B.cofem_op_destroy(op)


def test_noalloc_dct_after_dense(cuda_lib):
    D, N, ncols = 8192, 2048, 21
    idx = torch.from_numpy(datagen.dct_problem(D, N, int(0.04 * D), 0.01, seed=4).idx).cuda()
    _dirty_scratch_with_a_dense_call()
    op = B.cofem_op_dct(D, N, idx.data_ptr())
    try:
        _two_calls_match(op, D, ncols, 12)
    finally:
        B.cofem_op_destroy(op)


def test_noalloc_rejects_problems_beyond_its_scratch(cuda_lib):
    # a BF16 operator of 8192 x 8192 with 64 columns needs more scratch than
    # the static array holds: the call must refuse before launching anything.
    # Every buffer is a real allocation of the full size, so even a call that
    # went ahead would stay in bounds.
    N, D, ncols = 8192, 8192, 64
    Phi_t = torch.zeros((N, D), dtype=torch.bfloat16, device="cuda")
    op = B.cofem_op_dense(N, D, B.COFEM_BF16, Phi_t.data_ptr(), D)
    try:
        cap = B.cofem_noalloc_scratch_capacity()
        assert B.cofem_apply_workspace_bytes(op, B.COFEM_F32, ncols) > cap
        X = torch.zeros((ncols, D), dtype=torch.float32, device="cuda")
        Y = torch.empty_like(X)
        al = torch.ones(D, dtype=torch.float64, device="cuda")
        with pytest.raises(B.CofemError) as e:
            B.cofem_op_apply_noalloc(op, B.COFEM_F32, X.data_ptr(), D, ncols, al.data_ptr(), 1.0,
                                     Y.data_ptr())
        assert e.value.code == 7
        assert "static scratch" in B.lib().cofem_last_error().decode()
    finally:
        B.cofem_op_destroy(op)
