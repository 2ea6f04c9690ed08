"""FP64 oracle for the SBL model, exact EM and covariance-free EM (CoFEM).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy float64;
matrix products and Cholesky factorisations are library steps, everything else
follows the paper's equations in their order:

* model            Sec. 2.1, Eq. (model):  z ~ N(0, diag(alpha)^-1),
                                            y ~ N(Phi z, beta^-1 I)
* objective        Sec. 2.1, Eq. (mle2):   log p(y | alpha)
* exact E-step     Sec. 2.2, Eq. (estep-params):
                   Sigma = (beta Phi^T Phi + diag alpha)^-1, mu = beta Sigma Phi^T y
* M-step           Sec. 2.2, Eq. (mstep):  alpha = 1 / (mu*mu + diag Sigma)
* CoFEM            Sec. 3, Eq. (mat-eq), Eq. (diag-estimate), Algorithm 1
* linear solver    Sec. 3.2: conjugate gradients on A X = B, the mat-vec
                   replaced by a mat-mat, stopped when
                   ||A X - B||_F / ||B||_F < eps or after U iterations.

Readings where the paper is silent or garbled (each also listed in the design
notes of the repository):

* Sec. 3.2 writes A = Phi^T Phi + diag(alpha) without beta; Eq. (mat-eq) and
  Algorithm 1 have beta.  beta is kept.
* "Replacing mat-vec with mat-mat" is read as independent CG recurrences per
  column (own step sizes a_j, b_j), sharing each operator application.
* The stop test is the joint Frobenius ratio on the recursive residual,
  checked after every iteration; all columns iterate until it passes.
* X0 = 0.  Column 0 of B / X holds beta Phi^T y (mu); columns 1..K hold the
  probes.  The paper lists mu last; the order does not change any result.
* mu*mu + s can be <= 0 because s is an estimate; the M-step divides by
  max(mu*mu + s, den_floor) with den_floor = 1e-12 and counts the clamps.
* A column whose residual is exactly zero gets a_j = b_j = 0 (it has
  converged; avoids 0/0).
* Optional residual replacement every R iterations: r = B - A x.
* The convolutional dictionary is circular: (Phi z)[n] = sum_c sum_j
  h[c, j] z_c[(n - j) mod L]; Phi^T is its exact adjoint (correlation).
* The DCT dictionary of Sec. 4.2 ("inverse DCT followed by an undersampling
  mask") uses the orthonormal DCT-II / DCT-III pair, so Phi Phi^T = I_N;
  the mask keeps a uniformly random set of N = D/4 samples.
* Optional per-column stop rule (stop_rule = 1): see cg_solve.
* Optional block CG (solver = 1, a solver variant; the paper's solver is
  the column-wise one): see block_cg_solve.

Parity status: every function here is pinned by a CPU test against a closed
form, a library routine on an independent formulation, brute force, or an
invariant; see tests/test_oracle_pins.py.
"""
from dataclasses import dataclass, field

import numpy as np

from .probe_hash import probe_matrix

DEN_FLOOR = 1e-12


# --------------------------------------------------------------------------
# Dictionary operators.  Each returns (apply_phi, apply_phit, D).
# --------------------------------------------------------------------------

def dense_dictionary(Phi):
    """Dense Phi (N x D).  tau_D = O(N D) (Sec. 3.2)."""
    Phi = np.asarray(Phi, dtype=np.float64)

    def phi(Z):
        return Phi @ Z

    def phit(W):
        return Phi.T @ W

    return phi, phit, Phi.shape[1]


def conv_forward(h, Z):
    """(Phi z)[n] = sum_c sum_j h[c, j] z_c[(n - j) mod L]  (circular).

    h: C x T filters.  Z: C x L (one column) or C x L x m (m columns).
    Returns L (or L x m).  np.roll(v, j)[n] = v[(n - j) mod L].
    """
    h = np.asarray(h, dtype=np.float64)
    C, T = h.shape
    out = np.zeros(Z.shape[1:], dtype=np.float64)
    for c in range(C):
        for j in range(T):
            out += h[c, j] * np.roll(Z[c], j, axis=0)
    return out


def conv_adjoint(h, W):
    """(Phi^T w)_c[m] = sum_j h[c, j] w[(m + j) mod L]  (correlation)."""
    h = np.asarray(h, dtype=np.float64)
    C, T = h.shape
    out = np.zeros((C,) + W.shape, dtype=np.float64)
    for c in range(C):
        for j in range(T):
            out[c] += h[c, j] * np.roll(W, -j, axis=0)
    return out


def conv_dictionary(h, L):
    """Convolutional Phi (L x C*L); coordinate index d = c * L + m."""
    h = np.asarray(h, dtype=np.float64)
    C = h.shape[0]

    def phi(Z):
        m = Z.shape[1:]
        return conv_forward(h, Z.reshape((C, L) + m))

    def phit(W):
        out = conv_adjoint(h, W)
        return out.reshape((C * L,) + W.shape[1:])

    return phi, phit, C * L


def dct_dictionary(idx, D):
    """Masked-DCT Phi of Sec. 4.2 (N x D): the orthonormal inverse DCT of
    length D followed by the undersampling mask that keeps samples idx.
    With C the orthonormal DCT-II matrix, Phi = C^T[idx, :]:
        Phi z = (C^T z)[idx],  Phi^T w = C (w scattered to idx, zeros elsewhere).
    The transforms are scipy's FFT-based DCTs (a library step)."""
    import scipy.fft as sfft
    idx = np.asarray(idx)

    def phi(Z):
        return sfft.idct(np.asarray(Z, dtype=np.float64), type=2, norm="ortho", axis=0)[idx]

    def phit(W):
        W = np.asarray(W, dtype=np.float64)
        T = np.zeros((D,) + W.shape[1:])
        T[idx] = W
        return sfft.dct(T, type=2, norm="ortho", axis=0)

    return phi, phit, D


def dct_matrix(D):
    """Orthonormal DCT-II matrix from its definition:
    C[k, n] = s_k cos(pi k (2n + 1) / (2D)), s_0 = sqrt(1/D), s_k = sqrt(2/D)."""
    k = np.arange(D)[:, None]
    n = np.arange(D)[None, :]
    s = np.where(k == 0, np.sqrt(1.0 / D), np.sqrt(2.0 / D))
    return s * np.cos(np.pi * k * (2 * n + 1) / (2 * D))


def conv_matrix(h, L):
    """Materialised Phi for the circular convolution (L x C*L), by index
    rule: Phi[n, c*L + m] = h[c, (n - m) mod L] when that lag is < T."""
    h = np.asarray(h, dtype=np.float64)
    C, T = h.shape
    M = np.zeros((L, C * L))
    for n in range(L):
        for c in range(C):
            for m in range(L):
                lag = (n - m) % L
                if lag < T:
                    M[n, c * L + m] += h[c, lag]
    return M


def conv_matrix_vectorised(h, L):
    """Same matrix as conv_matrix, built with array indexing (for larger L)."""
    h = np.asarray(h, dtype=np.float64)
    C, T = h.shape
    n = np.arange(L)[:, None]
    m = np.arange(L)[None, :]
    lag = (n - m) % L
    M = np.zeros((L, C * L))
    for c in range(C):
        block = np.where(lag < T, h[c, np.minimum(lag, T - 1)], 0.0)
        M[:, c * L:(c + 1) * L] = block
    return M


def apply_A(phi, phit, beta, alpha, X):
    """A X with A = beta Phi^T Phi + diag(alpha)  (Eq. mat-eq)."""
    return beta * phit(phi(X)) + alpha[:, None] * X


# --------------------------------------------------------------------------
# Conjugate gradients on A X = B (Sec. 3.2).
# --------------------------------------------------------------------------

@dataclass
class CGResult:
    X: np.ndarray
    iters: int
    relres: float            # recursive residual ||R||_F / ||B||_F at exit
    converged: bool


def cg_solve(A, B, tol, max_iters, fixed_iters=0, resid_replace_every=0, stop_rule=0):
    """Column-wise CG, stopped on the joint Frobenius residual ratio.

    A: function X -> A X.  B: D x m.  X0 = 0.
    fixed_iters > 0 runs exactly that many iterations and ignores tol.
    resid_replace_every = R > 0 recomputes r = B - A x every R iterations.
    stop_rule = 1 (an option; the paper's rule is 0): column j is frozen once
    ||r_j|| / ||b_j|| < tol (its a_j and b_j are 0 from then on) and the solve
    ends when every column is frozen; relres stays the joint ratio.
    """
    B = np.asarray(B, dtype=np.float64)
    X = np.zeros_like(B)
    R = B.copy()
    P = R.copy()
    rho = np.sum(R * R, axis=0)
    normB = np.sqrt(np.sum(B * B))
    normBj = np.sqrt(rho)
    limit = fixed_iters if fixed_iters > 0 else max_iters
    if normB == 0.0:
        return CGResult(X, 0, 0.0, True)
    relres = np.sqrt(np.sum(rho)) / normB
    per_column = stop_rule == 1 and fixed_iters == 0
    if per_column:
        active = (normBj > 0) & ~(np.sqrt(rho) < tol * normBj)
        rho = np.where(active, rho, 0.0)     # a frozen column takes a_j = b_j = 0
        if not np.any(active):
            return CGResult(X, 0, relres, True)
    elif fixed_iters == 0 and relres < tol:
        return CGResult(X, 0, relres, True)
    it = 0
    while it < limit:
        it += 1
        Q = A(P)
        gamma = np.sum(P * Q, axis=0)
        a = np.where(rho > 0, rho / np.where(gamma != 0, gamma, 1.0), 0.0)
        X = X + a * P
        if resid_replace_every > 0 and it % resid_replace_every == 0:
            R = B - A(X)
        else:
            R = R - a * Q
        rho_new = np.sum(R * R, axis=0)
        relres = np.sqrt(np.sum(rho_new)) / normB
        if per_column:
            active = active & ~(np.sqrt(rho_new) < tol * normBj)
            rho_new = np.where(active, rho_new, 0.0)
            if not np.any(active):
                return CGResult(X, it, relres, True)
        elif fixed_iters == 0 and relres < tol:
            return CGResult(X, it, relres, True)
        b = np.where(rho > 0, rho_new / np.where(rho > 0, rho, 1.0), 0.0)
        P = R + b * P
        rho = rho_new
    converged = fixed_iters > 0 or (not np.any(active) if per_column else relres < tol)
    return CGResult(X, it, relres, converged)


def pcg_solve(A, B, X0, minv, tol, max_iters, resid_replace_every=0):
    """Column-wise preconditioned CG from X0 with the diagonal preconditioner
    M^-1 = diag(minv); same joint stop test on the residual R = B - A X as
    cg_solve.  With X0 = 0 and minv = 1 it performs exactly cg_solve's
    arithmetic.  (The learned warm start / preconditioner; the paper's solver
    is the unpreconditioned case.)"""
    B = np.asarray(B, dtype=np.float64)
    X = np.array(X0, dtype=np.float64)
    R = B - A(X) if np.any(X) else B.copy()
    Z = minv[:, None] * R
    P = Z.copy()
    rho = np.sum(R * Z, axis=0)
    normB = np.sqrt(np.sum(B * B))
    if normB == 0.0:
        return CGResult(np.zeros_like(B), 0, 0.0, True)
    relres = np.sqrt(np.sum(R * R)) / normB
    if relres < tol:
        return CGResult(X, 0, relres, True)
    it = 0
    while it < max_iters:
        it += 1
        Q = A(P)
        gamma = np.sum(P * Q, axis=0)
        a = np.where(rho > 0, rho / np.where(gamma != 0, gamma, 1.0), 0.0)
        X = X + a * P
        if resid_replace_every > 0 and it % resid_replace_every == 0:
            R = B - A(X)
        else:
            R = R - a * Q
        Z = minv[:, None] * R
        rho_new = np.sum(R * Z, axis=0)
        relres = np.sqrt(np.sum(R * R)) / normB
        if relres < tol:
            return CGResult(X, it, relres, True)
        b = np.where(rho > 0, rho_new / np.where(rho > 0, rho, 1.0), 0.0)
        P = Z + b * P
        rho = rho_new
    return CGResult(X, it, relres, relres < tol)


def block_cg_solve(A, B, tol, max_iters, fixed_iters=0):
    """Block CG on A X = B: the m columns share one block Krylov space
    span{B, A B, .., A^(k-1) B} (O'Leary, Lin. Alg. Appl. 29, 1980), the
    solver slot of Sec. 3.2 filled by a block method instead of m
    independent recurrences.  This is the residual-orthonormalised form of
    Dubrulle (ETNA 12, 2001): the residual block is kept as R = Q C with
    Q^T Q = I, so that ||R||_F = ||C||_F.  With X0 = 0:

        Q C = B (QR),  P = Q
        repeat:  Z = A P;  xi = (P^T Z)^-1
                 X = X + P xi C
                 V = Q - Z xi             (R_new = V C)
                 stop when ||V C||_F / ||B||_F < tol (same joint test as cg_solve)
                 Q psi = V (QR);  P = Q + P psi^T;  C = psi C

    fixed_iters > 0 runs exactly that many iterations and ignores tol.  The
    QR factorisations are the library's (Householder); they need no special
    case for a residual block that loses rank (a zero right-hand side, or a
    column combination that has converged): C or psi then has a zero row
    and that combination takes no further part in X.
    """
    B = np.asarray(B, dtype=np.float64)
    X = np.zeros_like(B)
    normB = np.sqrt(np.sum(B * B))
    limit = fixed_iters if fixed_iters > 0 else max_iters
    if normB == 0.0:
        return CGResult(X, 0, 0.0, True)
    Q, C = np.linalg.qr(B)
    relres = np.sqrt(np.sum(C * C)) / normB
    if fixed_iters == 0 and relres < tol:
        return CGResult(X, 0, relres, True)
    P = Q.copy()
    it = 0
    while it < limit:
        it += 1
        Z = A(P)
        xi = np.linalg.inv(P.T @ Z)
        X = X + P @ (xi @ C)
        V = Q - Z @ xi
        R = V @ C
        relres = np.sqrt(np.sum(R * R)) / normB
        if fixed_iters == 0 and relres < tol:
            return CGResult(X, it, relres, True)
        if it == limit:
            break
        Q, psi = np.linalg.qr(V)
        P = Q + P @ psi.T
        C = psi @ C
    return CGResult(X, it, relres, fixed_iters > 0 or relres < tol)


# --------------------------------------------------------------------------
# Diagonal estimation (Sec. 3.1) and M-step (Eq. mstep with s).
# --------------------------------------------------------------------------

def diag_estimate(P, Xp):
    """Proposition (Sec. 3.1): s = (sum_k p_k . x_k) / (sum_k p_k . p_k),
    x_k = Sigma p_k.  For +-1 probes this is Eq. (diag-estimate)."""
    return np.sum(P * Xp, axis=1) / np.sum(P * P, axis=1)


def m_step(mu, s, den_floor=DEN_FLOOR):
    """alpha = 1 / (mu*mu + s), denominator floored at den_floor.  mu may be
    T x D (T tasks sharing alpha, the multi-task extension of Sec. 5): then
    mu*mu is the mean over the tasks, alpha_d = T / sum_t (mu_td^2 + s_d).
    Returns (alpha, number of clamped coordinates)."""
    mu = np.asarray(mu)
    m2 = mu * mu if mu.ndim == 1 else np.mean(mu * mu, axis=0)
    den = m2 + s
    clamps = int(np.sum(den < den_floor))
    return 1.0 / np.maximum(den, den_floor), clamps


# --------------------------------------------------------------------------
# Algorithm 1: CovarianceFreeEM(y, Phi, beta, T_em, K).
# --------------------------------------------------------------------------

@dataclass
class FitStats:
    cg_iters: list = field(default_factory=list)
    relres: list = field(default_factory=list)
    clamps: list = field(default_factory=list)
    support: list = field(default_factory=list)


def cofem(phi, phit, D, y, beta, K, em_iters, cg_tol, cg_max_iters,
          seed=0, alpha_init=1.0, t_offset=0, fixed_cg_iters=0,
          resid_replace_every=0, den_floor=DEN_FLOOR, probes=None,
          support_threshold=1e6, stop_rule=0, solver=0):
    """Algorithm 1.  Returns (alpha, mu, s, FitStats).

    alpha_init: scalar (Alg. 1 initialises alpha = 1) or a length-D vector
    (resume from a previous alpha).  t runs t_offset+1 .. t_offset+em_iters.
    probes: optional function t -> D x K probe block; default is the
    counter-based Rademacher generator of probe_hash.  stop_rule: see
    cg_solve.  solver = 1 solves each E-step by block CG (block_cg_solve;
    the joint stop test, no residual replacement, stop_rule 0) instead of
    the column-wise recurrences.

    Multi-task (the extension named in Sec. 5, T tasks sharing alpha): y of
    shape T x N; B = [beta Phi^T y_1 .. beta Phi^T y_T | p_1 .. p_K], mu is
    returned T x D and the M-step averages mu^2 over the tasks (m_step).
    """
    y = np.asarray(y, dtype=np.float64)
    multi = y.ndim == 2
    Y = y.T if multi else y[:, None]         # N x T
    T = Y.shape[1]
    alpha = np.broadcast_to(np.asarray(alpha_init, dtype=np.float64), (D,)).copy()
    b = beta * phit(Y)                       # beta Phi^T y_t, fixed over EM iterations
    stats = FitStats()
    mu = np.zeros((T, D) if multi else D)
    s = np.zeros(D)
    for t in range(t_offset + 1, t_offset + em_iters + 1):
        # Simplified E-step.
        A = lambda X, al=alpha: apply_A(phi, phit, beta, al, X)
        P = probes(t) if probes is not None else probe_matrix(seed, t, K, D)
        B = np.concatenate([b, P], axis=1)
        if solver == 1:
            if resid_replace_every or stop_rule:
                raise ValueError("block CG: no residual replacement, joint stop test only")
            res = block_cg_solve(A, B, cg_tol, cg_max_iters, fixed_cg_iters)
        else:
            res = cg_solve(A, B, cg_tol, cg_max_iters, fixed_cg_iters,
                           resid_replace_every, stop_rule)
        mu = res.X[:, :T].T if multi else res.X[:, 0]
        s = diag_estimate(P, res.X[:, T:])
        # M-step.
        alpha, clamps = m_step(mu, s, den_floor)
        stats.cg_iters.append(res.iters)
        stats.relres.append(res.relres)
        stats.clamps.append(clamps)
        stats.support.append(int(np.sum(alpha < support_threshold)))
    return alpha, mu, s, stats


def cofem_learned(phi, phit, D, y, beta, K, em_iters, cg_tol, cg_max_iters, predict,
                  seed=0, alpha_init=1.0, den_floor=DEN_FLOOR, support_threshold=1e6):
    """Algorithm 1 with a learned warm start and diagonal preconditioner: at
    E-step t >= 2, (mu_hat, s_hat) = predict(alpha, mu_prev, s_prev); the
    solve starts from X0 = [mu_hat | s_hat . p_k] with M^-1 = diag(s_hat);
    if it has not reached cg_tol after cg_max_iters, plain CG from zero
    (the paper's solver) is run instead.  Returns (alpha, mu, s, stats) with
    stats.cg_iters the iterations of the accepted solve plus any fallback."""
    y = np.asarray(y, dtype=np.float64)
    alpha = np.broadcast_to(np.asarray(alpha_init, dtype=np.float64), (D,)).copy()
    b = beta * phit(y)
    stats = FitStats()
    stats.fallbacks = []
    mu = np.zeros(D)
    s = np.zeros(D)
    for t in range(1, em_iters + 1):
        A = lambda X, al=alpha: apply_A(phi, phit, beta, al, X)
        P = probe_matrix(seed, t, K, D)
        B = np.concatenate([b[:, None], P], axis=1)
        if t == 1:
            res = cg_solve(A, B, cg_tol, cg_max_iters)
            fb = 0
        else:
            mu_hat, s_hat = predict(alpha, mu, s)
            X0 = np.concatenate([mu_hat[:, None], s_hat[:, None] * P], axis=1)
            res = pcg_solve(A, B, X0, s_hat, cg_tol, cg_max_iters)
            fb = 0
            if not res.converged:
                res2 = cg_solve(A, B, cg_tol, cg_max_iters)
                res = CGResult(res2.X, res.iters + res2.iters, res2.relres, res2.converged)
                fb = 1
        mu = res.X[:, 0]
        s = diag_estimate(P, res.X[:, 1:])
        alpha, clamps = m_step(mu, s, den_floor)
        stats.cg_iters.append(res.iters)
        stats.relres.append(res.relres)
        stats.clamps.append(clamps)
        stats.support.append(int(np.sum(alpha < support_threshold)))
        stats.fallbacks.append(fb)
    return alpha, mu, s, stats


def cofem_dense(Phi, y, beta, K, em_iters, cg_tol, cg_max_iters, **kw):
    phi, phit, D = dense_dictionary(Phi)
    return cofem(phi, phit, D, y, beta, K, em_iters, cg_tol, cg_max_iters, **kw)


def cofem_dct(idx, D, y, beta, K, em_iters, cg_tol, cg_max_iters, **kw):
    phi, phit, D = dct_dictionary(idx, D)
    return cofem(phi, phit, D, y, beta, K, em_iters, cg_tol, cg_max_iters, **kw)


def cofem_conv(h, y, beta, K, em_iters, cg_tol, cg_max_iters, **kw):
    L = len(y)
    phi, phit, D = conv_dictionary(h, L)
    return cofem(phi, phit, D, y, beta, K, em_iters, cg_tol, cg_max_iters, **kw)


# --------------------------------------------------------------------------
# Exact EM (Sec. 2.2) and the objective (Eq. mle2).
# --------------------------------------------------------------------------

def e_step_exact(Phi, y, beta, alpha):
    """Eq. (estep-params): Sigma by Cholesky inverse, mu = beta Sigma Phi^T y."""
    Phi = np.asarray(Phi, dtype=np.float64)
    A = beta * (Phi.T @ Phi) + np.diag(alpha)
    L = np.linalg.cholesky(A)
    Linv = np.linalg.inv(L)
    Sigma = Linv.T @ Linv
    mu = beta * (Sigma @ (Phi.T @ y))
    return mu, Sigma


def em_exact(Phi, y, beta, em_iters, alpha_init=1.0, den_floor=DEN_FLOOR):
    """Exact EM: alternate Eq. (estep-params) and Eq. (mstep).
    Returns (alpha, mu, diagSigma, alpha_history) with alpha_history[0] the
    initial alpha."""
    D = Phi.shape[1]
    alpha = np.broadcast_to(np.asarray(alpha_init, dtype=np.float64), (D,)).copy()
    hist = [alpha.copy()]
    mu = np.zeros(D)
    dS = np.zeros(D)
    for _ in range(em_iters):
        mu, Sigma = e_step_exact(Phi, y, beta, alpha)
        dS = np.diag(Sigma).copy()
        alpha, _ = m_step(mu, dS, den_floor)
        hist.append(alpha.copy())
    return alpha, mu, dS, hist


def loglik(Phi, y, beta, alpha):
    """Eq. (mle2): y | alpha ~ N(0, C) with C = beta^-1 I + Phi diag(alpha)^-1 Phi^T
    (integrating z out of Eq. (model)).  Evaluated in the N-dimensional form."""
    Phi = np.asarray(Phi, dtype=np.float64)
    N = Phi.shape[0]
    C = np.eye(N) / beta + (Phi / alpha[None, :]) @ Phi.T
    sign, logdet = np.linalg.slogdet(C)
    quad = y @ np.linalg.solve(C, y)
    return -0.5 * (N * np.log(2 * np.pi) + logdet + quad)
