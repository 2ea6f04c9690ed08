"""Torch-facing convenience layer over the C ABI (marshalling only).

PyTorch provides device memory and streams; every step of the method runs in
libcofem's CUDA kernels through ``binding``.  No CPU fallback exists: without
a CUDA device or without the built library these functions raise.
"""
from dataclasses import dataclass

import torch

from . import binding as B

_DT = {torch.float64: B.COFEM_F64, torch.float32: B.COFEM_F32, torch.bfloat16: B.COFEM_BF16}


def _ld(n):
    return (n + 63) // 64 * 64


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class DenseOperator:
    """Dense Phi (N x D) held on the device; keeps the tensor alive."""

    def __init__(self, Phi: torch.Tensor):
        if not Phi.is_cuda:
            raise ValueError("Phi must be a CUDA tensor")
        if Phi.dtype not in _DT:
            raise ValueError("Phi dtype must be float64, float32 or bfloat16")
        N, D = Phi.shape
        ld = _ld(D) if Phi.dtype == torch.bfloat16 else D
        if Phi.stride() != (ld, 1):
            buf = torch.zeros((N, ld), dtype=Phi.dtype, device=Phi.device)
            buf[:, :D] = Phi
            Phi = buf
        self.phi = Phi
        self.N, self.D = N, D
        self.dtype = _DT[Phi.dtype]
        self.handle = B.cofem_op_dense(N, D, self.dtype, Phi.data_ptr(), Phi.stride(0))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None:
            B.cofem_op_destroy(h)
            self.handle = None


class Fp8DenseOperator:
    """Dense Phi stored as FP8 E4M3 with a power-of-two scale per 128 x 128
    tile, quantised on the device by the library from an FP32 CUDA tensor
    (N x D), with the packed copy the tensor cores read attached.  Keeps the
    bytes, the scales and the packed copy alive."""

    def __init__(self, Phi32: torch.Tensor, stream=None):
        if not Phi32.is_cuda or Phi32.dtype != torch.float32:
            raise ValueError("Phi must be a float32 CUDA tensor")
        N, D = Phi32.shape
        Phi32 = Phi32.contiguous()
        ld = _ld(D)
        self.phi = torch.zeros((N, ld), dtype=torch.uint8, device=Phi32.device)
        self.scales = torch.empty(((N + 127) // 128, (D + 127) // 128), dtype=torch.float32,
                                  device=Phi32.device)
        st = _stream_ptr(stream)
        B.cofem_quantize_fp8_tiles(Phi32.data_ptr(), N, D, D, self.phi.data_ptr(), ld,
                                   self.scales.data_ptr(), st)
        self.N, self.D = N, D
        self.dtype = B.COFEM_FP8_E4M3
        self.handle = B.cofem_op_dense(N, D, B.COFEM_FP8_E4M3, self.phi.data_ptr(), ld,
                                       self.scales.data_ptr())
        nb = B.cofem_op_dense_packed_bytes(self.handle)
        self.packed = torch.empty(nb, dtype=torch.uint8, device=Phi32.device)
        B.cofem_op_dense_attach_packed(self.handle, self.packed.data_ptr(), nb, st)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None:
            B.cofem_op_destroy(h)
            self.handle = None


class ConvOperator:
    """Circular convolutional Phi: C filters of T taps over length-L signals."""

    def __init__(self, h: torch.Tensor, L: int, tensor_cores: bool = False):
        if not h.is_cuda or h.dtype != torch.float32:
            raise ValueError("filters must be a float32 CUDA tensor")
        self.h = h.contiguous()
        self.C, self.T = self.h.shape
        self.L = L
        self.N, self.D = L, self.C * L
        self.dtype = B.COFEM_F32
        self.handle = B.cofem_op_conv1d(L, self.C, self.T, self.h.data_ptr())
        # tensor cores: the filters are rounded to BF16 for every use of Phi
        self.tensor_cores = bool(tensor_cores)
        if self.tensor_cores:
            B.cofem_op_conv1d_set_tensor_cores(self.handle, 1)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None:
            B.cofem_op_destroy(h)
            self.handle = None


class DctOperator:
    """Masked-DCT Phi (Sec. 4.2): the orthonormal inverse DCT of length D,
    then the N samples at `idx` (an int32 CUDA tensor, strictly increasing)."""

    def __init__(self, idx: torch.Tensor, D: int):
        if not idx.is_cuda or idx.dtype != torch.int32 or idx.dim() != 1:
            raise ValueError("idx must be a 1-D int32 CUDA tensor")
        self.idx = idx.contiguous()
        self.N, self.D = int(self.idx.numel()), int(D)
        self.dtype = B.COFEM_F32
        self.handle = B.cofem_op_dct(self.D, self.N, self.idx.data_ptr())

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None:
            B.cofem_op_destroy(h)
            self.handle = None


def _op_device(op):
    """Device of the tensors an operator handle reads."""
    for name in ("phi", "h", "idx"):
        t = getattr(op, name, None)
        if t is not None:
            return t.device
    raise TypeError("unknown operator %r" % type(op).__name__)


@dataclass
class FitResult:
    alpha: torch.Tensor
    mu: torch.Tensor
    s: torch.Tensor
    stats: dict


def params(**kw):
    return B.cofem_params_default(**kw)


def workspace(op, p, device=None):
    n = B.cofem_workspace_bytes(op.handle, p)
    dev = device if device is not None else torch.device("cuda")
    return torch.empty(n, dtype=torch.uint8, device=dev)


def fit(op, y, beta, p=None, ws=None, alpha=None, stream=None, **kw):
    """Algorithm 1 on the GPU.  y: CUDA tensor of the vector dtype
    (float64 for vec_dtype=F64, float32 otherwise), N values, or T x N for
    T tasks sharing alpha (p.tasks is then set to T and mu is T x D).
    Returns FitResult."""
    if p is None:
        p = params(**kw)
    vec = torch.float64 if p.vec_dtype == B.COFEM_F64 else torch.float32
    y = y.to(device=_op_device(op), dtype=vec).contiguous()
    T = y.shape[0] if y.dim() == 2 else 1
    if y.dim() == 2:
        p.tasks = T
    dev = y.device
    if ws is None:
        ws = workspace(op, p, dev)
    mu = torch.empty((T, op.D) if y.dim() == 2 else op.D, dtype=torch.float64, device=dev)
    s = torch.empty(op.D, dtype=torch.float64, device=dev)
    if alpha is None:
        alpha = torch.empty(op.D, dtype=torch.float64, device=dev)
    stats = B.cofem_fit(op.handle, y.data_ptr(), float(beta), p, ws.data_ptr(), ws.numel(),
                        mu.data_ptr(), s.data_ptr(), alpha.data_ptr(), _stream_ptr(stream))
    return FitResult(alpha, mu, s, stats)


def apply(op, X, alpha, beta, vec_dtype=None, stream=None):
    """Y = beta Phi^T Phi X + alpha . X for a D x ncols block X (CUDA)."""
    vec = B.COFEM_F64 if X.dtype == torch.float64 else B.COFEM_F32
    D, ncols = X.shape
    ld = _ld(D)
    Xb = torch.zeros((ncols, ld), dtype=X.dtype, device=X.device)
    Xb[:, :D] = X.T
    Yb = torch.empty_like(Xb)
    n = B.cofem_apply_workspace_bytes(op.handle, vec, ncols)
    ws = torch.empty(max(n, 256), dtype=torch.uint8, device=X.device)
    B.cofem_op_apply(op.handle, vec, Xb.data_ptr(), ld, ncols, alpha.data_ptr(), float(beta),
                     Yb.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    return Yb[:, :D].T


def fit_batched(phis, ys, betas, seeds, p, ws=None, stream=None):
    """Algorithm 1 for many problems at once (BF16 dictionaries).  phis: list
    of CUDA bfloat16 (N_i x D_i) tensors; ys: CUDA float32 (N_i); returns
    (alphas, mus, ss, stats) with per-problem tensors."""
    probs, keep = [], []
    for Phi, y, beta, seed in zip(phis, ys, betas, seeds):
        N, D = Phi.shape
        ld = _ld(D)
        if Phi.stride() != (ld, 1) or Phi.dtype != torch.bfloat16:
            buf = torch.zeros((N, ld), dtype=torch.bfloat16, device=Phi.device)
            buf[:, :D] = Phi
            Phi = buf
        y = y.to(torch.float32).contiguous()
        keep += [Phi, y]
        probs.append(B.cofem_problem(N, D, Phi.data_ptr(), ld, y.data_ptr(), float(beta), int(seed)))
    dev = phis[0].device
    if ws is None:
        ws = torch.empty(B.cofem_batched_workspace_bytes(probs, p), dtype=torch.uint8, device=dev)
    dtot = sum(int(P.shape[1]) for P in phis)
    mu = torch.empty(dtot, dtype=torch.float64, device=dev)
    s = torch.empty_like(mu)
    alpha = torch.empty_like(mu)
    stats = B.cofem_fit_batched(probs, p, ws.data_ptr(), ws.numel(), mu.data_ptr(), s.data_ptr(),
                                alpha.data_ptr(), _stream_ptr(stream))
    offs = [0]
    for P in phis:
        offs.append(offs[-1] + int(P.shape[1]))
    cut = lambda t: [t[offs[i]:offs[i + 1]] for i in range(len(phis))]
    return cut(alpha), cut(mu), cut(s), stats


# ---------------------------------------------------------------- learned path

MLP_PARAMS = 1282
_MLP_SHAPES = [(32, 4), (32,), (32, 32), (32,), (2, 32), (2,)]


class LearnedWarmStart:
    """Weights of the per-coordinate MLP on the device: FP32 master copy,
    Adam moments and the BF16 copy the fit and the forward pass read."""

    def __init__(self, seed=0, device="cuda"):
        g = torch.Generator(device="cpu")
        g.manual_seed(seed)
        parts = []
        for shp in _MLP_SHAPES:
            if len(shp) == 2:     # Glorot uniform
                lim = (6.0 / (shp[0] + shp[1])) ** 0.5
                parts.append((torch.rand(shp, generator=g, dtype=torch.float64) * 2 - 1) * lim)
            else:
                parts.append(torch.zeros(shp, dtype=torch.float64))
        self.master = torch.cat([p.reshape(-1) for p in parts]).float().to(device)
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.bf16 = self.master.to(torch.bfloat16)
        self.step = 0

    def train(self, U, Y, steps, lr=3e-3, batch=65536, stream=None, seed=0):
        """Adam on (U, Y) (CUDA float32, n x 4 and n x 2) in contiguous batches of
        a shuffled copy; returns the list of batch losses."""
        n = U.shape[0]
        g = torch.Generator(device=U.device)
        g.manual_seed(seed)
        perm = torch.randperm(n, device=U.device, generator=g)
        Us, Ys = U[perm].contiguous(), Y[perm].contiguous()
        nb = max(1, n // batch)
        ws = torch.empty(B.cofem_mlp_train_workspace_bytes(min(batch, n)), dtype=torch.uint8,
                         device=U.device)
        loss = torch.zeros(steps, dtype=torch.float64, device=U.device)
        for k in range(steps):
            i = k % nb
            b = min(batch, n)
            self.step += 1
            B.cofem_mlp_adam_step(self.master.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                  self.bf16.data_ptr(), Us[i * b:].data_ptr(), Ys[i * b:].data_ptr(),
                                  b, self.step, lr, ws.data_ptr(), ws.numel(),
                                  loss[k:].data_ptr(), _stream_ptr(stream))
        return loss.cpu().tolist()

    def forward(self, U, stream=None):
        O = torch.empty((U.shape[0], 2), dtype=torch.float32, device=U.device)
        B.cofem_mlp_forward(self.bf16.data_ptr(), B.COFEM_BF16, U.data_ptr(), U.shape[0],
                            O.data_ptr(), _stream_ptr(stream))
        return O


def col_norms(op, device, stream=None):
    """||phi_d||^2 of every coordinate of a dictionary (D floats on device)."""
    pn2 = torch.empty(op.D, dtype=torch.float32, device=device)
    n = B.cofem_col_norms_workspace_bytes(op.handle)
    ws = torch.empty(n, dtype=torch.uint8, device=device) if n else None
    B.cofem_op_col_norms_ws(op.handle, pn2.data_ptr(), ws.data_ptr() if n else None, n,
                            _stream_ptr(stream))
    if ws is not None and stream is not None:
        ws.record_stream(stream)
    return pn2


def collect_training_data(op, y, beta, p, em_iters, stream=None):
    """Runs plain CoFEM one EM iteration at a time and returns (U, Y) samples
    of every coordinate for E-steps 2..em_iters: features from the alpha the
    E-step used and the previous E-step's mu, s; targets from its own mu, s."""
    dev = y.device
    D = op.D
    pn2 = col_norms(op, dev, stream)
    alpha = torch.empty(D, dtype=torch.float64, device=dev)
    Us, Ys = [], []
    mu_prev = s_prev = None
    ws = None
    for t in range(em_iters):
        q = params(**{f: getattr(p, f) for f, _ in B.cofem_params._fields_})
        q.em_iters = 1
        q.t_offset = t
        q.mlp = None
        if ws is None:
            ws = workspace(op, q, dev)
        if t == 0:
            alpha.fill_(q.alpha_init)
        a_in = alpha.clone()
        r = fit(op, y, beta, q, ws=ws, alpha=alpha, stream=stream)
        if mu_prev is not None:
            U = torch.empty((D, 4), dtype=torch.float32, device=dev)
            Yt = torch.empty((D, 2), dtype=torch.float32, device=dev)
            B.cofem_mlp_features(a_in.data_ptr(), pn2.data_ptr(), float(beta),
                                 mu_prev.data_ptr(), s_prev.data_ptr(), D, U.data_ptr(),
                                 _stream_ptr(stream))
            B.cofem_mlp_targets(a_in.data_ptr(), pn2.data_ptr(), float(beta), r.mu.data_ptr(),
                                r.s.data_ptr(), D, Yt.data_ptr(), _stream_ptr(stream))
            Us.append(U)
            Ys.append(Yt)
        mu_prev, s_prev = r.mu.clone(), r.s.clone()
        alpha = r.alpha
    return torch.cat(Us), torch.cat(Ys)
