"""Kernel-level parity: each hot-path step through the C ABI against the
oracle on the same seeded inputs.  Sizes span several tiles plus a ragged
tail; column counts include 1, 2, 17, 21, 33 and 64."""
import numpy as np
import pytest
import torch

from oracle import probe_hash as ph
from oracle import sbl
from paper_2202_12808_gb300 import binding as B
from paper_2202_12808_gb300 import datagen
from gpu_helpers import (bf16_round, fp8_applied, fp8_quantize_reference, from_block, ld_of,
                         phi_tensor, rel_l2, to_block)

pytestmark = pytest.mark.gpu


def _ws(op, vec, ncols):
    n = B.cofem_apply_workspace_bytes(op, vec, ncols)
    return torch.empty(max(n, 256), dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("K,D,t,seed", [(20, 1024, 1, 0), (20, 1024, 50, 0), (32, 32768, 7, 3),
                                        (100, 777, 2, 123456789), (1, 65, 1, 2 ** 63 + 5)])
def test_probe_fill_bit_exact(cuda_lib, K, D, t, seed):
    for dt, vec in ((torch.float64, B.COFEM_F64), (torch.float32, B.COFEM_F32)):
        ld = ld_of(D)
        out = torch.full((K, ld), 7.0, dtype=dt, device="cuda")
        B.cofem_probe_fill(seed, t, K, D, vec, out.data_ptr(), ld)
        torch.cuda.synchronize()
        got = out[:, :D].T.cpu().double().numpy()
        ref = ph.probe_matrix(seed, t, K, D)
        assert np.array_equal(got, ref)
        assert torch.all(out[:, D:] == 0)


def test_probe_fill_all_config1_iterations(cuda_lib):
    # all (t, k, d) of 50 EM iterations at K = 20, D = 1024
    ld = 1024
    out = torch.empty((20, ld), dtype=torch.float32, device="cuda")
    for t in range(1, 51):
        B.cofem_probe_fill(0, t, 20, 1024, B.COFEM_F32, out.data_ptr(), ld)
        assert np.array_equal(out.T.cpu().double().numpy(), ph.probe_matrix(0, t, 20, 1024))


APPLY_CASES = [
    # (N, D, ncols)
    (200, 1000, 1), (200, 1000, 2), (200, 1000, 17), (256, 1024, 21), (130, 515, 33),
    (96, 300, 64), (520, 1300, 33),
]


@pytest.mark.parametrize("N,D,ncols", APPLY_CASES)
@pytest.mark.parametrize("kind", ["f64", "f32", "f32-packed", "f32-packed-r256", "bf16",
                                  "bf16-t2", "bf16-t1", "bf16-simt", "bf16-packed",
                                  "bf16-packed-t1", "bf16-r256", "bf16-packed-r256", "fp8"])
def test_op_apply_dense(cuda_lib, N, D, ncols, kind):
    prob = datagen.dense_problem(N, D, max(1, D // 50), 0.01, seed=N + D + ncols)
    rng = np.random.default_rng(ncols)
    X = rng.standard_normal((D, ncols))
    alpha = rng.uniform(0.5, 1e3, D)
    beta = 1e4
    if kind == "f64":
        Phi_ref = prob.Phi.astype(np.float64)
        Phi_t, ld_phi = phi_tensor(Phi_ref, torch.float64)
        vdt, vec, tol = torch.float64, B.COFEM_F64, 1e-12
        pdt = B.COFEM_F64
    elif kind in ("f32", "f32-packed", "f32-packed-r256"):
        # f32-packed: the tensor cores with Phi = hi + lo (two BF16 terms, at
        # most 2^-17 relative per entry), against the oracle on the FP32 Phi
        Phi_ref = prob.Phi.astype(np.float64)
        Phi_t, ld_phi = phi_tensor(prob.Phi, torch.float32)
        vdt, vec, tol = torch.float32, B.COFEM_F32, 2e-5
        pdt = B.COFEM_F32
    elif kind == "fp8":
        # E4M3 bytes with a power-of-two scale per 128 x 128 tile (quantised
        # on the CPU); the oracle applies bf16(q x scale)
        q, scales, Phi_ref = fp8_quantize_reference(prob.Phi)
        ld_phi = ld_of(D)
        Phi_t = torch.zeros((N, ld_phi), dtype=torch.uint8, device="cuda")
        Phi_t[:, :D] = torch.from_numpy(q).cuda()
        scales_t = torch.from_numpy(scales).cuda()
        vdt, vec, pdt, tol = torch.float32, B.COFEM_F32, B.COFEM_FP8_E4M3, 2e-5
    else:
        t16, Phi_ref = bf16_round(prob.Phi)
        Phi_t, ld_phi = phi_tensor(Phi_ref, torch.bfloat16)
        vdt, vec, pdt = torch.float32, B.COFEM_F32, B.COFEM_BF16
        # FP32 split into 3 / 2 / 1 BF16 terms (24 / 16 / 8-bit mantissas)
        terms = {"bf16": 3, "bf16-t2": 2, "bf16-t1": 1, "bf16-simt": 0, "bf16-packed": 3,
                 "bf16-packed-t1": 1, "bf16-r256": 3, "bf16-packed-r256": 3}[kind]
        tol = {3: 2e-5, 2: 6e-5, 1: 8e-3, 0: 2e-5}[terms]
    X_in = X.astype(np.float32).astype(np.float64) if vdt == torch.float32 else X
    op = B.cofem_op_dense(N, D, pdt, Phi_t.data_ptr(), ld_phi,
                          scales_t.data_ptr() if kind == "fp8" else None)
    if pdt == B.COFEM_BF16:
        B.cofem_op_dense_set_terms(op, terms)
    if kind.endswith("-r256"):
        # two 128-row output tiles per work unit (ragged: odd tile counts)
        B.cofem_op_dense_set_tile_rows(op, 256)
        assert B.cofem_op_dense_get_pipeline(op)[2] == 256
    packed = None
    if kind.startswith("bf16-packed") or kind.startswith("f32-packed") or kind == "fp8":
        nb = B.cofem_op_dense_packed_bytes(op)
        assert nb == {"f": B.cofem_dense_packed_bytes(N, D) * 2,
                      "b": B.cofem_dense_packed_bytes(N, D),
                      "p": B.cofem_dense_packed_bytes(N, D) // 2}[kind[0] if kind != "fp8" else "p"]
        packed = torch.empty(nb, dtype=torch.uint8, device="cuda")
        B.cofem_op_dense_attach_packed(op, packed.data_ptr(), nb)
    try:
        Xb, ld = to_block(X_in, vdt)
        Yb = torch.full_like(Xb, 3.0)
        al = torch.from_numpy(alpha).cuda()
        ws = _ws(op, vec, ncols)
        B.cofem_op_apply(op, vec, Xb.data_ptr(), ld, ncols, al.data_ptr(), beta, Yb.data_ptr(),
                         ws.data_ptr(), ws.numel())
        torch.cuda.synchronize()
        phi, phit, _ = sbl.dense_dictionary(Phi_ref)
        ref = sbl.apply_A(phi, phit, beta, alpha, X_in)
        got = from_block(Yb, D)
        for j in range(ncols):
            assert rel_l2(got[:, j], ref[:, j]) <= tol, (j, rel_l2(got[:, j], ref[:, j]))
        # the two halves
        W = torch.zeros((ncols, ld_of(N)), dtype=vdt, device="cuda")
        B.cofem_op_forward(op, vec, Xb.data_ptr(), ld, ncols, W.data_ptr(), ld_of(N),
                           ws.data_ptr(), ws.numel())
        Z = torch.zeros_like(Xb)
        B.cofem_op_adjoint(op, vec, W.data_ptr(), ld_of(N), ncols, Z.data_ptr(), ld,
                           ws.data_ptr(), ws.numel())
        torch.cuda.synchronize()
        Wref = Phi_ref @ X_in
        Wg = W[:, :N].T.double().cpu().numpy()
        half_tol = 1e-12 if kind == "f64" else 2e-5     # the halves run on CUDA cores
        assert rel_l2(Wg, Wref) <= half_tol
        Zref = Phi_ref.T @ Wg
        assert rel_l2(from_block(Z, D), Zref) <= half_tol
    finally:
        B.cofem_op_destroy(op)


@pytest.mark.parametrize("K,D", [(20, 1024), (32, 1000), (5, 70), (64, 4096)])
def test_diag_mstep(cuda_lib, K, D):
    rng = np.random.default_rng(K * D)
    seed, t = 99, 4
    X = rng.standard_normal((D, K + 1)) * 1e-2
    X[:10, 0] = 0.0                       # mu = 0 ...
    X[:10, 1:] = 0.0                      # ... and s = 0: clamped denominators
    for dt, vec in ((torch.float64, B.COFEM_F64), (torch.float32, B.COFEM_F32)):
        Xin = X.astype(np.float32).astype(np.float64) if dt == torch.float32 else X
        Xb, ld = to_block(Xin, dt)
        mu = torch.empty(D, dtype=torch.float64, device="cuda")
        s = torch.empty_like(mu)
        al = torch.empty_like(mu)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        B.cofem_diag_mstep(seed, t, K, D, vec, Xb.data_ptr(), ld, 1e-12, 1e6, mu.data_ptr(),
                           s.data_ptr(), al.data_ptr(), counts.data_ptr())
        torch.cuda.synchronize()
        P = ph.probe_matrix(seed, t, K, D)
        s_ref = sbl.diag_estimate(P, Xin[:, 1:])
        mu_ref = Xin[:, 0]
        a_ref, clamps = sbl.m_step(mu_ref, s_ref)
        np.testing.assert_array_equal(mu.cpu().numpy(), mu_ref)
        # sums of K terms in another order: compare on the scale of the terms
        scale = np.abs(Xin[:, 1:]).sum(axis=1) / K
        assert np.all(np.abs(s.cpu().numpy() - s_ref) <= 1e-14 * scale + 1e-300)
        a = al.cpu().numpy()
        np.testing.assert_allclose(1.0 / a, 1.0 / a_ref, rtol=1e-12, atol=1e-14 * scale.max())
        c = counts.cpu().numpy()
        assert c[0] == clamps
        assert c[1] == int(np.sum(a < 1e6))


@pytest.mark.parametrize("N,D", [(300, 1100), (128, 128), (1000, 4096)])
def test_fp8_quantize_matches_definition(cuda_lib, N, D):
    """cofem_quantize_fp8_tiles against its definition computed on the CPU:
    power-of-two tile scales, E4M3 bytes bit for bit (tiles of very
    different magnitude, an all-zero tile, ragged edges)."""
    rng = np.random.default_rng(N + D)
    Phi = rng.standard_normal((N, D)).astype(np.float32)
    Phi *= np.exp(rng.uniform(-8, 8, ((N + 127) // 128, (D + 127) // 128))).astype(
        np.float32).repeat(128, 0).repeat(128, 1)[:N, :D]
    Phi[:min(N, 128), :min(D, 128)] = 0.0
    q_ref, s_ref, _ = fp8_quantize_reference(Phi)
    P = torch.from_numpy(Phi).cuda()
    q = torch.zeros((N, ld_of(D)), dtype=torch.uint8, device="cuda")
    sc = torch.empty(((N + 127) // 128, (D + 127) // 128), dtype=torch.float32, device="cuda")
    B.cofem_quantize_fp8_tiles(P.data_ptr(), N, D, D, q.data_ptr(), ld_of(D), sc.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(sc.cpu().numpy(), s_ref)
    np.testing.assert_array_equal(q[:, :D].cpu().numpy(), q_ref)


def test_f32_packed_terms_are_hi_plus_lo(cuda_lib):
    """The two packed images of an FP32 dictionary: applying Phi = hi + lo
    with exact-valued inputs matches the oracle's product with hi + lo
    (rounded to nearest even, from torch) far more closely than the 2^-17
    representation error of Phi itself."""
    N, D, ncols = 300, 1100, 17
    prob = datagen.dense_problem(N, D, 20, 0.01, seed=9)
    P32 = prob.Phi
    hi = torch.from_numpy(P32).to(torch.bfloat16)
    lo = (torch.from_numpy(P32) - hi.float()).to(torch.bfloat16)
    Phi_hl = hi.double().numpy() + lo.double().numpy()
    assert np.max(np.abs(Phi_hl - P32) / np.maximum(np.abs(P32), 1e-30)) <= 2.0 ** -17
    Phi_t, ld_phi = phi_tensor(P32, torch.float32)
    op = B.cofem_op_dense(N, D, B.COFEM_F32, Phi_t.data_ptr(), ld_phi)
    nb = B.cofem_op_dense_packed_bytes(op)
    pk = torch.empty(nb, dtype=torch.uint8, device="cuda")
    B.cofem_op_dense_attach_packed(op, pk.data_ptr(), nb)
    try:
        rng = np.random.default_rng(2)
        X = rng.standard_normal((D, ncols)).astype(np.float32).astype(np.float64)
        alpha = rng.uniform(0.5, 10.0, D)
        Xb, ld = to_block(X, torch.float32)
        Yb = torch.empty_like(Xb)
        al = torch.from_numpy(alpha).cuda()
        ws = _ws(op, B.COFEM_F32, ncols)
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, al.data_ptr(), 1.0,
                         Yb.data_ptr(), ws.data_ptr(), ws.numel())
        torch.cuda.synchronize()
        phi, phit, _ = sbl.dense_dictionary(Phi_hl)
        ref = sbl.apply_A(phi, phit, 1.0, alpha, X)
        got = from_block(Yb, D)
        for j in range(ncols):
            assert rel_l2(got[:, j], ref[:, j]) <= 2e-6, j
    finally:
        B.cofem_op_destroy(op)


@pytest.mark.parametrize("packed,rows", [(False, 128), (True, 128), ("f32", 128), (True, 256),
                                         ("f32", 256), ("fp8", 128)])
def test_op_apply_tensor_core_full_size(cuda_lib, packed, rows):
    # the bench workload's operator (N=4096, D=32768, 33 columns, BF16 Phi,
    # 3-term split) on sampled output rows computed one by one by the oracle
    N, D, ncols = 4096, 32768, 33
    prob = datagen.dense_problem(N, D, 655, 0.01, seed=0)
    scales_ptr = None
    if packed == "f32":
        # FP32 Phi on the tensor cores (hi + lo), against the FP32 Phi
        Phi_ref = prob.Phi.astype(np.float64)
        Phi_t, ld_phi = phi_tensor(prob.Phi, torch.float32)
        pdt = B.COFEM_F32
    elif packed == "fp8":
        # quantised by the library; the oracle applies bf16(q x scale)
        P32 = torch.from_numpy(prob.Phi).cuda()
        Phi_t = torch.zeros((N, D), dtype=torch.uint8, device="cuda")
        sc = torch.empty((N // 128, D // 128), dtype=torch.float32, device="cuda")
        B.cofem_quantize_fp8_tiles(P32.data_ptr(), N, D, D, Phi_t.data_ptr(), D, sc.data_ptr())
        torch.cuda.synchronize()
        del P32
        Phi_ref = fp8_applied(Phi_t.cpu().numpy(), sc.cpu().numpy())
        ld_phi, pdt, scales_ptr = D, B.COFEM_FP8_E4M3, sc.data_ptr()
    else:
        t16, Phi_ref = bf16_round(prob.Phi)
        Phi_t, ld_phi = phi_tensor(Phi_ref, torch.bfloat16)
        pdt = B.COFEM_BF16
    rng = np.random.default_rng(1)
    X = rng.standard_normal((D, ncols)).astype(np.float32).astype(np.float64)
    alpha = rng.uniform(0.5, 1e6, D)
    beta = 1e4
    op = B.cofem_op_dense(N, D, pdt, Phi_t.data_ptr(), ld_phi, scales_ptr)
    B.cofem_op_dense_set_tile_rows(op, rows)
    if packed:
        nb = B.cofem_op_dense_packed_bytes(op)
        pk = torch.empty(nb, dtype=torch.uint8, device="cuda")
        B.cofem_op_dense_attach_packed(op, pk.data_ptr(), nb)
    try:
        Xb, ld = to_block(X, torch.float32)
        Yb = torch.empty_like(Xb)
        al = torch.from_numpy(alpha).cuda()
        ws = _ws(op, B.COFEM_F32, ncols)
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, al.data_ptr(), beta,
                         Yb.data_ptr(), ws.data_ptr(), ws.numel())
        torch.cuda.synchronize()
        W = Phi_ref @ X                                   # N x ncols, fp64
        rows = np.sort(rng.choice(D, size=512, replace=False))
        rows[-1] = D - 1
        ref = beta * (Phi_ref[:, rows].T @ W) + alpha[rows, None] * X[rows]
        got = Yb[:, rows].T.double().cpu().numpy()
        for j in range(ncols):
            assert rel_l2(got[:, j], ref[:, j]) <= 2e-5, j
    finally:
        B.cofem_op_destroy(op)


def test_autotuner_keeps_results_correct(cuda_lib):
    N, D, ncols = 1000, 5000, 21
    prob = datagen.dense_problem(N, D, 50, 0.01, seed=4)
    _, Phi_ref = bf16_round(prob.Phi)
    Phi_t, ld_phi = phi_tensor(Phi_ref, torch.bfloat16)
    op = B.cofem_op_dense(N, D, B.COFEM_BF16, Phi_t.data_ptr(), ld_phi)
    try:
        nb = B.cofem_op_dense_autotune_workspace_bytes(op, ncols)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        st, cps, us = B.cofem_op_dense_autotune(op, ncols, ws.data_ptr(), nb)
        assert 2 <= st <= 8 and cps in (1, 2) and us > 0
        rng = np.random.default_rng(0)
        X = rng.standard_normal((D, ncols)).astype(np.float32).astype(np.float64)
        alpha = rng.uniform(1, 10, D)
        Xb, ld = to_block(X, torch.float32)
        Yb = torch.empty_like(Xb)
        al = torch.from_numpy(alpha).cuda()
        wsa = _ws(op, B.COFEM_F32, ncols)
        B.cofem_op_apply(op, B.COFEM_F32, Xb.data_ptr(), ld, ncols, al.data_ptr(), 1e4,
                         Yb.data_ptr(), wsa.data_ptr(), wsa.numel())
        torch.cuda.synchronize()
        phi, phit, _ = sbl.dense_dictionary(Phi_ref)
        ref = sbl.apply_A(phi, phit, 1e4, alpha, X)
        got = from_block(Yb, D)
        for j in range(ncols):
            assert rel_l2(got[:, j], ref[:, j]) <= 2e-5
    finally:
        B.cofem_op_destroy(op)
