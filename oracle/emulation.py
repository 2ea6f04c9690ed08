"""Rounding experiments on the oracle -- TEST INFRASTRUCTURE ONLY.

Some GPU parity bars are looser than the oracle's own FP64 precision (CG
iteration counts of tolerance-mode fits, mu after truncated solves, the
noise level of the batched cases).  This module produces the evidence for
those bars from the oracle alone: Algorithm 1 with the column-wise CG of
Sec. 3.2, exactly as ``sbl.cofem`` / ``sbl.cg_solve`` compute it, with two
optional hooks that change nothing but rounding:

* ``vround``   applied to every stored vector (B, X, R, P, the operator
               product Q and its intermediate W = Phi P) and to the alpha the
               operator reads -- with ``fp32_round`` this emulates FP32
               vectors (the GPU's FP32 path stores the same quantities in
               FP32 and keeps mu, s, alpha and every CG scalar in FP64); the
               products themselves are either exact FP64 products
               (``sbl.dense_dictionary``) or FP32-accumulated ones
               (``fp32_dense_dictionary``: numpy float32 matrix products, which
               accumulate in FP32 like the tensor cores' accumulators, in
               another order);
* ``dperturb`` applied to every per-column reduction (gamma_j = p_j^T q_j and
               rho_j = r_j^T r_j) -- with ``ulp_perturber`` each result is
               multiplied by (1 + u 2^-52), u = +-1 from a seeded generator:
               a re-ordering of the FP64 sums moves them by about as much.

``block_cg_solve`` carries ``vround`` over to the block CG of the solver
variant (``sbl.block_cg_solve``).

With both hooks None the functions perform exactly the arithmetic of
``sbl.cg_solve``, ``sbl.block_cg_solve`` and ``sbl.cofem`` (pinned bit for bit in
tests/test_tolerance_evidence.py), so every difference they show comes
from rounding alone.  Only the joint stop rule and the per-column rule of
``sbl.cg_solve`` are carried over; residual replacement is not.
"""
import numpy as np

from . import sbl
from .probe_hash import probe_matrix


def fp32_round(v):
    """Round to the nearest float32 and return float64 (exact)."""
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def ulp_perturber(seed, rel=2.0 ** -52):
    """Reduction hook: multiplies each value by 1 + u rel, u = +-1 drawn from
    numpy's PCG64 stream of `seed`."""
    rng = np.random.default_rng(seed)

    def f(v):
        u = rng.choice(np.array([-1.0, 1.0]), size=np.shape(v))
        return v * (1.0 + u * rel)

    return f


def fp32_dense_dictionary(Phi):
    """Dense Phi whose products Phi Z and Phi^T W run as float32 matrix
    products (FP32 inputs, FP32 accumulation), returned as float64.  Phi must
    be exactly representable in float32 (a BF16- or FP32-stored dictionary)."""
    P32 = np.asarray(Phi, dtype=np.float64).astype(np.float32)
    assert np.array_equal(P32.astype(np.float64), np.asarray(Phi, dtype=np.float64))

    def phi(Z):
        return (P32 @ np.asarray(Z).astype(np.float32)).astype(np.float64)

    def phit(W):
        return (P32.T @ np.asarray(W).astype(np.float32)).astype(np.float64)

    return phi, phit, P32.shape[1]


def _id(v):
    return v


def cg_solve(A, B, tol, max_iters, fixed_iters=0, stop_rule=0, vround=None, dperturb=None):
    """sbl.cg_solve (joint or per-column stop, X0 = 0) with the rounding
    hooks of the module header."""
    vr = vround or _id
    dp = dperturb or _id
    B = vr(np.asarray(B, dtype=np.float64))
    X = np.zeros_like(B)
    R = B.copy()
    P = R.copy()
    rho = dp(np.sum(R * R, axis=0))
    normB = np.sqrt(np.sum(B * B))
    normBj = np.sqrt(np.sum(B * B, axis=0))
    limit = fixed_iters if fixed_iters > 0 else max_iters
    if normB == 0.0:
        return sbl.CGResult(X, 0, 0.0, True)
    relres = np.sqrt(np.sum(rho)) / normB
    per_column = stop_rule == 1 and fixed_iters == 0
    if per_column:
        active = (normBj > 0) & ~(np.sqrt(rho) < tol * normBj)
        rho = np.where(active, rho, 0.0)
        if not np.any(active):
            return sbl.CGResult(X, 0, relres, True)
    elif fixed_iters == 0 and relres < tol:
        return sbl.CGResult(X, 0, relres, True)
    it = 0
    while it < limit:
        it += 1
        Q = vr(A(P))
        gamma = dp(np.sum(P * Q, axis=0))
        a = np.where(rho > 0, rho / np.where(gamma != 0, gamma, 1.0), 0.0)
        X = vr(X + a * P)
        R = vr(R - a * Q)
        rho_new = dp(np.sum(R * R, axis=0))
        relres = np.sqrt(np.sum(rho_new)) / normB
        if per_column:
            active = active & ~(np.sqrt(rho_new) < tol * normBj)
            rho_new = np.where(active, rho_new, 0.0)
            if not np.any(active):
                return sbl.CGResult(X, it, relres, True)
        elif fixed_iters == 0 and relres < tol:
            return sbl.CGResult(X, it, relres, True)
        b = np.where(rho > 0, rho_new / np.where(rho > 0, rho, 1.0), 0.0)
        P = vr(R + b * P)
        rho = rho_new
    converged = fixed_iters > 0 or (not np.any(active) if per_column else relres < tol)
    return sbl.CGResult(X, it, relres, converged)


def block_cg_solve(A, B, tol, max_iters, fixed_iters=0, vround=None):
    """sbl.block_cg_solve (X0 = 0, joint stop test) with every stored block
    (B, X, Q, P, the operator product Z = A P, V) and every small matrix
    (C, xi, M = xi C, psi) passed through vround; the QR factorisations and
    products themselves are FP64 library steps, as in the oracle."""
    vr = vround or _id
    B = vr(np.asarray(B, dtype=np.float64))
    X = np.zeros_like(B)
    normB = np.sqrt(np.sum(B * B))
    limit = fixed_iters if fixed_iters > 0 else max_iters
    if normB == 0.0:
        return sbl.CGResult(X, 0, 0.0, True)
    Q, C = np.linalg.qr(B)
    Q, C = vr(Q), vr(C)
    relres = np.sqrt(np.sum(C * C)) / normB
    if fixed_iters == 0 and relres < tol:
        return sbl.CGResult(X, 0, relres, True)
    P = Q.copy()
    it = 0
    while it < limit:
        it += 1
        Z = vr(A(P))
        xi = vr(np.linalg.inv(P.T @ Z))
        X = vr(X + P @ vr(xi @ C))
        V = vr(Q - Z @ xi)
        R = V @ C
        relres = np.sqrt(np.sum(R * R)) / normB
        if fixed_iters == 0 and relres < tol:
            return sbl.CGResult(X, it, relres, True)
        if it == limit:
            break
        Q, psi = np.linalg.qr(V)
        Q, psi = vr(Q), vr(psi)
        P = vr(Q + P @ psi.T)
        C = vr(psi @ C)
    return sbl.CGResult(X, it, relres, fixed_iters > 0 or relres < tol)


def cofem(phi, phit, D, y, beta, K, em_iters, cg_tol, cg_max_iters, seed=0,
          alpha_init=1.0, fixed_cg_iters=0, stop_rule=0, vround=None, dperturb=None,
          support_threshold=1e6, solver=0):
    """sbl.cofem (single task, t from 1) with the rounding hooks: B, X, R, P
    and the operator product pass through vround, the operator reads
    vround(alpha), every per-column reduction passes through dperturb.  mu, s
    and alpha stay float64 (as on the GPU).  solver = 1: block CG
    (block_cg_solve, vround only).  Returns (alpha, mu, s, FitStats)."""
    vr = vround or _id
    y = np.asarray(y, dtype=np.float64)
    alpha = np.broadcast_to(np.asarray(alpha_init, dtype=np.float64), (D,)).copy()
    b = beta * phit(y[:, None])
    stats = sbl.FitStats()
    mu = np.zeros(D)
    s = np.zeros(D)
    for t in range(1, em_iters + 1):
        al = vr(alpha)
        # A X = beta Phi^T (Phi X) + alpha . X (Eq. mat-eq), the intermediate
        # W = Phi X stored through vround as well
        A = lambda X, al=al: beta * phit(vr(phi(X))) + al[:, None] * X
        P = probe_matrix(seed, t, K, D)
        B = np.concatenate([b, P], axis=1)
        if solver == 1:
            res = block_cg_solve(A, B, cg_tol, cg_max_iters, fixed_cg_iters, vround)
        else:
            res = cg_solve(A, B, cg_tol, cg_max_iters, fixed_cg_iters, stop_rule, vround,
                           dperturb)
        mu = res.X[:, 0]
        s = sbl.diag_estimate(P, res.X[:, 1:])
        alpha, clamps = sbl.m_step(mu, s)
        stats.cg_iters.append(res.iters)
        stats.relres.append(res.relres)
        stats.clamps.append(clamps)
        stats.support.append(int(np.sum(alpha < support_threshold)))
    return alpha, mu, s, stats


def cofem_dense(Phi, y, beta, K, em_iters, cg_tol, cg_max_iters, fp32_products=False, **kw):
    """cofem on a dense Phi; fp32_products selects fp32_dense_dictionary."""
    dic = fp32_dense_dictionary if fp32_products else sbl.dense_dictionary
    phi, phit, D = dic(Phi)
    return cofem(phi, phit, D, y, beta, K, em_iters, cg_tol, cg_max_iters, **kw)
