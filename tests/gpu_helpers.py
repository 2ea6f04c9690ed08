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
