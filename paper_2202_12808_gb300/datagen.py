"""Seeded synthetic SBL problems shaped like the paper's workloads.

This module is shared by the CUDA path's tests/bench and by the oracle's
tests: it only draws inputs (dictionary, sparse ground truth, noisy
observations) and holds none of CoFEM's arithmetic.  Every generator is a
pure function of its seed (numpy PCG64 via ``default_rng``).

Workloads (Sec. 4 uses simulated compressed-sensing data only):

* ``dense_problem``   Phi iid N(0, 1/N) (N x D), d nonzeros at uniform random
                      positions with N(0,1) (or +-1, or Laplace) amplitudes,
                      y = Phi z + N(0, sigma^2) noise (Eq. model).
* ``conv_problem``    C filters of T taps, iid N(0,1) then unit l2 norm;
                      circular convolutional dictionary over a length-L signal;
                      z has a fraction of nonzeros with Laplace(0,1) amplitudes.
* ``batched_sizes``   N_i uniform on an integer range, D_i = ratio * N_i, one
                      seed per problem derived from a master seed.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class DenseProblem:
    Phi: np.ndarray        # N x D, float32 (exactly representable values)
    z: np.ndarray          # D, float64 ground truth
    y: np.ndarray          # N, float64
    support: np.ndarray    # indices of nonzeros
    beta: float


def _amplitudes(rng, n, kind):
    if kind == "normal":
        return rng.standard_normal(n)
    if kind == "spike":
        return rng.choice(np.array([-1.0, 1.0]), size=n)
    if kind == "laplace":
        return rng.laplace(0.0, 1.0, size=n)
    raise ValueError(kind)


def dense_problem(N, D, n_nonzero, sigma, seed, amp="normal", phi_scale=None):
    """Dense compressed-sensing problem.  phi_scale defaults to 1/sqrt(N)
    (entries N(0, 1/N)); pass 1.0 for the paper's Sec. 4.1 N(0,1) entries."""
    rng = np.random.default_rng(seed)
    scale = (1.0 / np.sqrt(N)) if phi_scale is None else phi_scale
    Phi = (rng.standard_normal((N, D), dtype=np.float32) * np.float32(scale))
    support = np.sort(rng.choice(D, size=n_nonzero, replace=False))
    z = np.zeros(D)
    z[support] = _amplitudes(rng, n_nonzero, amp)
    noise = sigma * rng.standard_normal(N)
    y = Phi.astype(np.float64)[:, support] @ z[support] + noise
    return DenseProblem(Phi, z, y, support, 1.0 / sigma ** 2)


@dataclass
class ConvProblem:
    h: np.ndarray          # C x T filters, float32, unit l2 norm per filter
    z: np.ndarray          # C x L ground truth codes (float64)
    y: np.ndarray          # L observations (float64)
    beta: float


def conv_problem(L, C, T, density, sigma, seed):
    """Circular convolutional dictionary problem; y = sum_c h_c (*) z_c + noise,
    built by scattering each nonzero's shifted filter (the generative model,
    Eq. model)."""
    rng = np.random.default_rng(seed)
    h = rng.standard_normal((C, T))
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    h = h.astype(np.float32)
    D = C * L
    nnz = max(1, int(round(density * D)))
    idx = np.sort(rng.choice(D, size=nnz, replace=False))
    amps = rng.laplace(0.0, 1.0, size=nnz)
    z = np.zeros((C, L))
    z.reshape(-1)[idx] = amps
    y = sigma * rng.standard_normal(L)
    c_of, m_of = idx // L, idx % L
    h64 = h.astype(np.float64)
    for j in range(T):
        np.add.at(y, (m_of + j) % L, amps * h64[c_of, j])
    return ConvProblem(h, z, y, 1.0 / sigma ** 2 if sigma > 0 else float("inf"))


@dataclass
class DctProblem:
    idx: np.ndarray        # N kept sample indices, int32, strictly increasing
    z: np.ndarray          # D ground-truth DCT coefficients (float64)
    y: np.ndarray          # N observations (float64)
    beta: float


def dct_problem(D, N, n_nonzero, sigma, seed):
    """Masked-DCT problem of the paper's structured experiment (Sec. 4.2): N of
    the D samples kept (chosen uniformly without replacement), n_nonzero
    N(0, 1) DCT coefficients at uniform positions, y = the kept samples of
    the signal (scipy's orthonormal inverse DCT of z) plus N(0, sigma^2)
    noise (the generative model, Eq. model)."""
    import scipy.fft as sfft
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(D, size=N, replace=False)).astype(np.int32)
    z = np.zeros(D)
    z[rng.choice(D, size=n_nonzero, replace=False)] = rng.standard_normal(n_nonzero)
    y = sfft.idct(z, type=2, norm="ortho")[idx] + sigma * rng.standard_normal(N)
    return DctProblem(idx, z, y, 1.0 / sigma ** 2 if sigma > 0 else float("inf"))


@dataclass
class MultiTaskProblem:
    Phi: np.ndarray        # N x D float32, iid N(0, 1/N)
    Z: np.ndarray          # T x D ground truth (float64), one support shared by the tasks
    Y: np.ndarray          # T x N observations (float64)
    beta: float


def multitask_problem(N, D, T, n_nonzero, sigma, seed):
    """T tasks observed through one dense Phi with a common support (the
    multi-task model of the extension named in Sec. 5): n_nonzero shared
    positions, independent N(0, 1) amplitudes per task, y_t = Phi z_t +
    N(0, sigma^2) noise."""
    rng = np.random.default_rng(seed)
    Phi = (rng.standard_normal((N, D)) / np.sqrt(N)).astype(np.float32)
    Z = np.zeros((T, D))
    idx = rng.choice(D, size=n_nonzero, replace=False)
    Z[:, idx] = rng.standard_normal((T, n_nonzero))
    Y = Z @ Phi.astype(np.float64).T + sigma * rng.standard_normal((T, N))
    return MultiTaskProblem(Phi, Z, Y, 1.0 / sigma ** 2 if sigma > 0 else float("inf"))


def batched_sizes(n_problems, n_min, n_max, ratio, seed):
    """(N_i, D_i, seed_i) for each problem; N_i uniform on [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_min, n_max + 1, size=n_problems)
    seeds = rng.integers(0, 2 ** 62, size=n_problems)
    return [(int(n), int(ratio * n), int(s)) for n, s in zip(Ns, seeds)]


def orthonormal_columns(N, D, seed):
    """N x D matrix with orthonormal columns (D <= N), Q factor of a Gaussian
    matrix (Householder QR via numpy)."""
    rng = np.random.default_rng(seed)
    Q, Rm = np.linalg.qr(rng.standard_normal((N, D)))
    return Q * np.sign(np.diag(Rm))[None, :]


# Named workloads (sizes of the paper-shaped configurations).
CONFIGS = {
    # FP64 plain CoFEM: dense N=256, D=1024, 51 nonzeros, sigma 0.01, K=20,
    # 50 EM iterations, CG tol 1e-6, U=400.
    "dense-fp64-n256-d1024": dict(N=256, D=1024, n_nonzero=51, sigma=0.01, K=20,
                                  em_iters=50, cg_tol=1e-6, cg_max_iters=400),
    # Large dense: N=4096, D=32768, 2% nonzeros, beta 1e4, K=32, 100 EM
    # iterations, CG tol 1e-5, residual replacement every 50 iterations.
    "dense-n4096-d32768": dict(N=4096, D=32768, n_nonzero=655, sigma=0.01, K=32,
                               em_iters=100, cg_tol=1e-5, cg_max_iters=400,
                               resid_replace_every=50),
    # Batched: 512 dense problems, N uniform on [128, 2048], D = 4N, BF16,
    # 5% nonzeros, sigma 0.01, K=16, 50 EM iterations, CG tol 1e-5.
    "batched-512-n128-2048": dict(n_problems=512, n_min=128, n_max=2048, ratio=4,
                                  frac_nonzero=0.05, sigma=0.01, K=16, em_iters=50,
                                  cg_tol=1e-5, cg_max_iters=400),
    # Convolutional: L = 2^20, 8 filters x 64 taps, 0.1% nonzeros Laplace,
    # sigma 0.05, K=16, 30 EM iterations.
    "conv-l1m-c8-t64": dict(L=1 << 20, C=8, T=64, density=1e-3, sigma=0.05, K=16,
                            em_iters=30, cg_tol=1e-5, cg_max_iters=400),
    # Masked DCT (the paper's structured experiment at its largest size):
    # D = 2^18, N = D/4 kept samples, d = 0.1 D N(0,1) coefficients, K = 20,
    # U = 400; the paper states no noise level or tolerance: sigma 0.01 and
    # CG tol 1e-5 as for the dense workload.
    "dct-d262144": dict(D=1 << 18, N=1 << 16, n_nonzero=26214, sigma=0.01, K=20,
                        em_iters=30, cg_tol=1e-5, cg_max_iters=400),
}


def batched_problems_torch_f32(n_problems, n_min, n_max, ratio, frac_nonzero, sigma, seed,
                               device="cuda"):
    """The problems of batched_problems_torch (same sizes and seeds) with the
    dictionary kept in FP32: Phi_i iid N(0, 1/N_i) float32 and y_i = Phi_i z_i
    + N(0, sigma^2) from that FP32 dictionary.  A path that stores Phi_i in
    BF16 then approximates the dictionary the data came from.  Returns a list
    of (Phi_i float32 N_i x D_i, z_i float64, y_i float32, beta, seed_i)."""
    import torch
    out = []
    for N, D, s in batched_sizes(n_problems, n_min, n_max, ratio, seed):
        g = torch.Generator(device=device)
        g.manual_seed(s)
        Phi = torch.randn((N, D), generator=g, device=device) / float(np.sqrt(N))
        k = max(1, int(round(frac_nonzero * D)))
        idx = torch.randperm(D, generator=g, device=device)[:k]
        z = torch.zeros(D, dtype=torch.float64, device=device)
        z[idx] = torch.randn(k, generator=g, device=device, dtype=torch.float64)
        noise = sigma * torch.randn(N, generator=g, device=device, dtype=torch.float64)
        y = (Phi.double()[:, idx] @ z[idx] + noise).float()
        out.append((Phi, z, y, 1.0 / sigma ** 2, s))
    return out


def batched_problems_torch(n_problems, n_min, n_max, ratio, frac_nonzero, sigma, seed,
                           device="cuda"):
    """Many dense problems (N_i uniform on [n_min, n_max], D_i = ratio N_i,
    Phi_i iid N(0, 1/N_i) in BF16, a fraction of nonzeros with N(0,1)
    amplitudes, y_i = Phi_i z_i + N(0, sigma^2)) drawn on the device with a
    seeded torch generator per problem (host generation of the 3 G entries of
    the 512-problem workload would take minutes).  Returns a list of
    (Phi_i bf16 N_i x D_i, z_i float64, y_i float32, beta, seed_i)."""
    import torch
    out = []
    for N, D, s in batched_sizes(n_problems, n_min, n_max, ratio, seed):
        g = torch.Generator(device=device)
        g.manual_seed(s)
        Phi = (torch.randn((N, D), generator=g, device=device) / float(np.sqrt(N))).to(torch.bfloat16)
        k = max(1, int(round(frac_nonzero * D)))
        idx = torch.randperm(D, generator=g, device=device)[:k]
        z = torch.zeros(D, dtype=torch.float64, device=device)
        z[idx] = torch.randn(k, generator=g, device=device, dtype=torch.float64)
        noise = sigma * torch.randn(N, generator=g, device=device, dtype=torch.float64)
        y = (Phi.double()[:, idx] @ z[idx] + noise).float()
        out.append((Phi, z, y, 1.0 / sigma ** 2, s))
    return out
