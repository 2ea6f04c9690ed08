"""Shared helpers of the GPU parity tests (inputs from datagen, reference
values from oracle/ only)."""
import numpy as np
import torch

from paper_2202_12808_gb300 import binding as B


def ld_of(n):
    return (n + 63) // 64 * 64


def to_block(X, dtype, device="cuda"):
    """D x m numpy -> column-major device block (m x ld), zero padded."""
    D, m = X.shape
    ld = ld_of(D)
    out = torch.zeros((m, ld), dtype=dtype, device=device)
    out[:, :D] = torch.from_numpy(np.ascontiguousarray(X.T)).to(device=device, dtype=dtype)
    return out, ld


def from_block(Xb, D):
    return Xb[:, :D].T.double().cpu().numpy()


def bf16_round(Phi32):
    """Round a float32 matrix to bfloat16 (torch, round-to-nearest-even) and
    return (bf16 tensor on CPU, exact float64 values)."""
    t = torch.from_numpy(Phi32).to(torch.bfloat16)
    return t, t.double().numpy()


def phi_tensor(Phi, dtype, device="cuda"):
    N, D = Phi.shape
    ld = ld_of(D)
    out = torch.zeros((N, ld), dtype=dtype, device=device)
    out[:, :D] = torch.from_numpy(np.ascontiguousarray(Phi)).to(device=device, dtype=dtype)
    return out, ld


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def support_compare(alpha_gpu, alpha_ref, thr=1e6):
    """Support sets {alpha < thr}; coordinates within a factor 2 of thr in
    either path are excluded (borderline).  Returns (equal, n_borderline)."""
    a, r = np.asarray(alpha_gpu), np.asarray(alpha_ref)
    border = ((a > thr / 2) & (a < thr * 2)) | ((r > thr / 2) & (r < thr * 2))
    sa, sr = (a < thr) & ~border, (r < thr) & ~border
    return bool(np.array_equal(sa, sr)), int(border.sum())


def fp8_quantize_reference(Phi32):
    """The FP8 E4M3 quantisation the library documents, on the CPU: per
    128 x 128 tile the smallest power of two s with max |phi| / s <= 448,
    bytes e4m3(phi / s) (torch's round-to-nearest-even cast), and the
    dictionary a handle applies, bf16(float(q) x s), as float64.
    Returns (bytes N x D uint8, scales, Phi_applied)."""
    N, D = Phi32.shape
    tm, tn = (N + 127) // 128, (D + 127) // 128
    scales = np.ones((tm, tn), dtype=np.float32)
    q = np.zeros((N, D), dtype=np.uint8)
    applied = np.zeros((N, D))
    for i in range(tm):
        for j in range(tn):
            blk = Phi32[128 * i:128 * (i + 1), 128 * j:128 * (j + 1)]
            m = float(np.max(np.abs(blk)))
            s = 1.0
            if m > 0:
                f, e = np.frexp(np.float32(m) / np.float32(448.0))
                s = float(np.ldexp(1.0, int(e) - 1 if f == 0.5 else int(e)))
            scales[i, j] = s
            t = (torch.from_numpy(np.ascontiguousarray(blk)) / s).to(torch.float8_e4m3fn)
            q[128 * i:128 * (i + 1), 128 * j:128 * (j + 1)] = t.view(torch.uint8).numpy()
            deq = (t.to(torch.float32) * torch.tensor(s, dtype=torch.float32)).to(torch.bfloat16)
            applied[128 * i:128 * (i + 1), 128 * j:128 * (j + 1)] = deq.double().numpy()
    return q, scales, applied


def fp8_applied(q, scales):
    """bf16(float(q) x scale of its 128 x 128 tile) for E4M3 bytes q (N x D)."""
    N, D = q.shape
    s = np.repeat(np.repeat(scales, 128, axis=0), 128, axis=1)[:N, :D]
    v = torch.from_numpy(np.ascontiguousarray(q)).view(torch.float8_e4m3fn).to(torch.float32)
    return (v * torch.from_numpy(np.ascontiguousarray(s, dtype=np.float32))).to(
        torch.bfloat16).double().numpy()
