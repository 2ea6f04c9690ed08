"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with a
closed form, a library routine on an independent formulation, brute force,
or an invariant.  CPU only.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import probe_hash as ph
from oracle import sbl
from paper_2202_12808_gb300 import datagen


# ---------------------------------------------------------------- probe hash

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_ints(name):
    return [int(l, 16) for l in open(os.path.join(GOLDEN, name))
            if l.strip() and not l.startswith("#")]


def test_splitmix64_published_stream():
    # SplitMix64 seeded with state 0: first three outputs of the published
    # generator (state advances by the golden gamma before each mix).
    expect = _golden_ints("splitmix64_seed0.txt")
    assert len(expect) == 3
    x = 0
    for e in expect:
        assert ph.mix64_int(x) == e
        x = (x + ph.GAMMA) & ph.MASK
    arr = ph.mix64(np.array([0, ph.GAMMA, (2 * ph.GAMMA) & ph.MASK], dtype=np.uint64))
    assert [int(v) for v in arr] == expect


def test_probe_words_match_scalar_path():
    seed, t = 12345, 7
    h = ph.probe_words(seed, t, 300, 2)
    s1 = ph.mix64_int(ph.mix64_int(seed) ^ t)
    for d in (0, 1, 17, 299):
        for w in (0, 1):
            assert int(h[d, w]) == ph.mix64_int(s1 ^ ((d << 8) | w))
    P = ph.probe_matrix(seed, t, 100, 300)
    for d in (0, 5, 299):
        for k in (0, 63, 64, 99):
            bit = (ph.mix64_int(s1 ^ ((d << 8) | (k // 64))) >> (k % 64)) & 1
            assert P[d, k] == (1.0 if bit == 0 else -1.0)


def test_probe_statistics():
    K, D = 64, 20000
    P = ph.probe_matrix(3, 1, K, D)
    n = P.size
    # mean of +-1 signs: std 1/sqrt(n)
    assert abs(P.mean()) < 5 / np.sqrt(n)
    # column correlations ~ N(0, 1/D)
    C = (P.T @ P) / D
    off = C[~np.eye(K, dtype=bool)]
    assert np.max(np.abs(off)) < 5.5 / np.sqrt(D)
    # independent across EM iterations and seeds
    P2 = ph.probe_matrix(3, 2, K, D)
    P3 = ph.probe_matrix(4, 1, K, D)
    for Q in (P2, P3):
        assert abs(np.mean(P * Q)) < 5 / np.sqrt(n)
    # each of the 64 bit positions is balanced
    col_means = P.mean(axis=0)
    assert np.max(np.abs(col_means)) < 5 / np.sqrt(D)


# ------------------------------------------------------------- CG (Sec. 3.2)

def _spd_problem(N, D, seed, beta=1.0, alpha_spread=(0.5, 5.0)):
    rng = np.random.default_rng(seed)
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    alpha = rng.uniform(*alpha_spread, size=D)
    return Phi, alpha


def test_cg_matches_cholesky():
    Phi, alpha = _spd_problem(150, 200, 1, beta=3.0)
    beta = 3.0
    A = beta * Phi.T @ Phi + np.diag(alpha)
    rng = np.random.default_rng(2)
    B = rng.standard_normal((200, 5))
    X_ref = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), B)
    phi, phit, D = sbl.dense_dictionary(Phi)
    res = sbl.cg_solve(lambda X: sbl.apply_A(phi, phit, beta, alpha, X), B, 1e-14, 2000)
    assert res.converged
    assert np.linalg.norm(res.X - X_ref) / np.linalg.norm(X_ref) <= 1e-10


def test_cg_residual_replacement_matches_cholesky():
    Phi, alpha = _spd_problem(100, 160, 5, alpha_spread=(0.01, 50.0))
    beta = 10.0
    A = beta * Phi.T @ Phi + np.diag(alpha)
    B = np.random.default_rng(6).standard_normal((160, 3))
    X_ref = np.linalg.solve(A, B)
    phi, phit, _ = sbl.dense_dictionary(Phi)
    res = sbl.cg_solve(lambda X: sbl.apply_A(phi, phit, beta, alpha, X), B, 1e-13, 3000,
                       resid_replace_every=7)
    assert res.converged
    # the recursive residual was replaced by the true one: check it is true
    true_rel = np.linalg.norm(A @ res.X - B) / np.linalg.norm(B)
    assert true_rel < 1e-12
    assert np.linalg.norm(res.X - X_ref) / np.linalg.norm(X_ref) <= 1e-10


def test_cg_diagonal_terminates_in_distinct_count():
    # CG on a matrix with m distinct eigenvalues ends in exactly m steps.
    vals = np.array([1.0, 3.0, 7.0, 20.0, 55.0])
    diag = np.repeat(vals, 40)
    rng = np.random.default_rng(0)
    B = rng.standard_normal((diag.size, 3))
    res = sbl.cg_solve(lambda X: diag[:, None] * X, B, 1e-11, 50)
    assert res.converged and res.iters == len(vals)


def test_cg_fixed_iteration_mode():
    diag = np.linspace(1, 10, 50)
    B = np.ones((50, 2))
    res = sbl.cg_solve(lambda X: diag[:, None] * X, B, 1.0, 50, fixed_iters=4)
    assert res.iters == 4
    res0 = sbl.cg_solve(lambda X: diag[:, None] * X, B, 1e-30, 4)
    assert np.array_equal(res.X, res0.X)


# ------------------------------------- E-step on orthonormal dictionaries

@pytest.mark.parametrize("K", [1, 5, 20])
def test_orthonormal_estep_closed_form(K):
    N = D = 64
    Phi = datagen.orthonormal_columns(N, D, 11)
    rng = np.random.default_rng(12)
    y = rng.standard_normal(N)
    beta, a0 = 4.0, 2.5
    alpha, mu, s, st = sbl.cofem_dense(Phi, y, beta, K, 1, 1e-14, 10, seed=9,
                                       alpha_init=a0)
    q = Phi.T @ y
    assert st.cg_iters == [1]                  # A = (beta + a0) I
    np.testing.assert_allclose(mu, beta * q / (beta + a0), rtol=1e-13)
    np.testing.assert_allclose(s, 1.0 / (beta + a0), rtol=1e-13)
    np.testing.assert_allclose(alpha, 1.0 / (mu * mu + 1.0 / (beta + a0)), rtol=1e-13)


def test_orthonormal_nonuniform_alpha_diag_exact():
    # A diagonal with 3 distinct values: s = 1/(beta+alpha) for any probes.
    N, D = 96, 60
    Phi = datagen.orthonormal_columns(N, D, 3)
    y = np.random.default_rng(4).standard_normal(N)
    beta = 2.0
    a0 = np.tile([0.5, 7.0, 100.0], D // 3)
    alpha, mu, s, st = sbl.cofem_dense(Phi, y, beta, 3, 1, 1e-13, 20, alpha_init=a0)
    assert st.cg_iters == [3]
    np.testing.assert_allclose(s, 1.0 / (beta + a0), rtol=1e-11)
    np.testing.assert_allclose(mu, beta * (Phi.T @ y) / (beta + a0), rtol=1e-11)


def test_orthonormal_em_fixed_point():
    # Orthogonal design: alpha* = 1 / (q^2 - 1/beta) where q^2 > 1/beta,
    # alpha -> infinity otherwise (Eq. estep-params + Eq. mstep per coordinate).
    N = D = 16
    Phi = datagen.orthonormal_columns(N, D, 21)
    beta = 25.0
    q = np.linspace(-1.5, 1.5, D)
    q[np.abs(q) < 0.05] = 0.03
    y = Phi @ q
    alpha, mu, dS, hist = sbl.em_exact(Phi, y, beta, 3000)
    strong = q * q > 1.0 / beta + 0.05
    weak = q * q < 1.0 / beta - 0.01
    assert strong.any() and weak.any()
    np.testing.assert_allclose(alpha[strong], 1.0 / (q[strong] ** 2 - 1.0 / beta), rtol=1e-8)
    assert np.all(alpha[weak] > 1e4)
    # CoFEM with exact diagonal (orthonormal Phi) follows exact EM.
    a_c, _, _, _ = sbl.cofem_dense(Phi, y, beta, 2, 40, 1e-15, 50)
    np.testing.assert_allclose(a_c, hist[40], rtol=1e-9)


# ------------------------------------------- diagonal estimation (Sec. 3.1)

def _small_model(N, D, seed, beta=50.0):
    rng = np.random.default_rng(seed)
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    y = rng.standard_normal(N)
    return Phi, y, beta


def test_hadamard_probes_give_exact_diagonal():
    D = 64
    Phi, y, beta = _small_model(40, D, 1)
    H = scipy.linalg.hadamard(D).astype(np.float64)
    _, mu, s, _ = sbl.cofem_dense(Phi, y, beta, D, 1, 1e-14, 1000,
                                  probes=lambda t: H)
    mu_ex, Sigma = sbl.e_step_exact(Phi, y, beta, np.ones(D))
    np.testing.assert_allclose(s, np.diag(Sigma), rtol=1e-9)
    np.testing.assert_allclose(mu, mu_ex, rtol=1e-9, atol=1e-12)


def test_all_sign_patterns_give_exact_diagonal():
    D = 8
    Phi, y, beta = _small_model(5, D, 2, beta=3.0)
    P = np.array(list(itertools.product([1.0, -1.0], repeat=D))).T   # D x 2^D
    _, _, s, _ = sbl.cofem_dense(Phi, y, beta, P.shape[1], 1, 1e-15, 100,
                                 probes=lambda t: P)
    _, Sigma = sbl.e_step_exact(Phi, y, beta, np.ones(D))
    np.testing.assert_allclose(s, np.diag(Sigma), rtol=1e-10)


def test_general_rule_equals_rademacher_form():
    rng = np.random.default_rng(0)
    P = ph.probe_matrix(1, 1, 9, 30)
    X = rng.standard_normal((30, 9))
    np.testing.assert_allclose(sbl.diag_estimate(P, X), (P * X).mean(axis=1), rtol=1e-15)
    # general (non +-1) probes: unbiased rule divides by sum p^2
    G = rng.standard_normal((30, 9))
    M = rng.standard_normal((30, 30))
    s = sbl.diag_estimate(G, M @ G)
    manual = np.array([sum(G[d, k] * (M @ G[:, k])[d] for k in range(9)) /
                       sum(G[d, k] ** 2 for k in range(9)) for d in range(30)])
    np.testing.assert_allclose(s, manual, rtol=1e-12)


def test_estimator_unbiased_with_closed_form_variance():
    # E[s_d] = Sigma_dd,  Var[s_d] = (1/K) sum_{j != d} Sigma_dj^2 (Rademacher).
    D, K, seeds = 24, 4, 400
    Phi, y, beta = _small_model(12, D, 7, beta=5.0)
    alpha = np.random.default_rng(8).uniform(0.5, 3.0, D)
    _, Sigma = sbl.e_step_exact(Phi, y, beta, alpha)
    S = np.stack([sbl.cofem_dense(Phi, y, beta, K, 1, 1e-13, 500, seed=sd,
                                  alpha_init=alpha)[2] for sd in range(seeds)])
    var = (np.sum(Sigma ** 2, axis=1) - np.diag(Sigma) ** 2) / K
    z = (S.mean(axis=0) - np.diag(Sigma)) / np.sqrt(var / seeds)
    assert np.max(np.abs(z)) < 5.0
    ratio = S.var(axis=0, ddof=1) / var
    assert 0.7 < np.median(ratio) < 1.3


@pytest.mark.parametrize("em_t,N,D", [(0, 128, 512), (5, 64, 256), (20, 64, 256)])
def test_cofem_matches_exact_em_with_many_probes(em_t, N, D):
    # K = 10^4 probes at a fixed alpha (exact EM's alpha after em_t steps):
    # relative L2 error of s against diag(Sigma) within 1e-2, D <= 512.
    prob = datagen.dense_problem(N, D, D // 25, 0.01, seed=5)
    Phi = prob.Phi.astype(np.float64)
    beta = 1e4
    _, _, _, hist = sbl.em_exact(Phi, prob.y, beta, em_t)
    alpha = hist[em_t]
    _, mu, s, _ = sbl.cofem_dense(Phi, prob.y, beta, 10000, 1, 1e-10, 2000,
                                  alpha_init=alpha, seed=1)
    mu_ex, Sigma = sbl.e_step_exact(Phi, prob.y, beta, alpha)
    dS = np.diag(Sigma)
    assert np.linalg.norm(s - dS) / np.linalg.norm(dS) <= 1e-2
    assert np.linalg.norm(mu - mu_ex) / np.linalg.norm(mu_ex) <= 1e-6


# ----------------------------------------------------- exact EM, objective

def test_loglik_two_forms_agree():
    # N-space Gaussian marginal vs the D-space form through the posterior
    # (determinant lemma); each derived separately from Eq. (model).
    N, D = 30, 50
    Phi, y, beta = _small_model(N, D, 3, beta=7.0)
    alpha = np.random.default_rng(4).uniform(0.1, 10, D)
    mu, Sigma = sbl.e_step_exact(Phi, y, beta, alpha)
    _, logdetS = np.linalg.slogdet(Sigma)
    dform = -0.5 * (N * np.log(2 * np.pi) - N * np.log(beta) - np.sum(np.log(alpha))
                    - logdetS + beta * np.sum((y - Phi @ mu) ** 2) + mu @ (alpha * mu))
    assert abs(sbl.loglik(Phi, y, beta, alpha) - dform) < 1e-9 * abs(dform)


def test_loglik_scalar_case():
    # N = D = 1: y ~ N(0, 1/beta + phi^2/alpha)
    phi, y, beta, alpha = 0.7, 1.3, 2.0, 0.5
    var = 1 / beta + phi * phi / alpha
    expect = -0.5 * (np.log(2 * np.pi * var) + y * y / var)
    got = sbl.loglik(np.array([[phi]]), np.array([y]), beta, np.array([alpha]))
    assert abs(got - expect) < 1e-14


def test_exact_em_monotone():
    prob = datagen.dense_problem(64, 256, 10, 0.05, seed=2)
    Phi = prob.Phi.astype(np.float64)
    beta = prob.beta
    _, _, _, hist = sbl.em_exact(Phi, prob.y, beta, 30)
    ll = [sbl.loglik(Phi, prob.y, beta, a) for a in hist]
    for a, b in zip(ll, ll[1:]):
        assert b >= a - 1e-9 * abs(a)
    assert ll[-1] > ll[0]


def test_m_step_clamp():
    alpha, clamps = sbl.m_step(np.array([0.0, 1.0, 1e-7]), np.array([-1.0, 0.0, 0.0]))
    assert clamps == 2
    np.testing.assert_allclose(alpha, [1e12, 1.0, 1e12])


def test_resume_equals_uninterrupted():
    prob = datagen.dense_problem(40, 160, 6, 0.01, seed=8)
    Phi = prob.Phi.astype(np.float64)
    kw = dict(seed=4)
    a6, mu6, s6, _ = sbl.cofem_dense(Phi, prob.y, 1e4, 8, 6, 1e-8, 200, **kw)
    a3, _, _, _ = sbl.cofem_dense(Phi, prob.y, 1e4, 8, 3, 1e-8, 200, **kw)
    b6, nu6, r6, _ = sbl.cofem_dense(Phi, prob.y, 1e4, 8, 3, 1e-8, 200,
                                     alpha_init=a3, t_offset=3, **kw)
    assert np.array_equal(a6, b6) and np.array_equal(mu6, nu6) and np.array_equal(s6, r6)


# -------------------------------------------------- convolutional operator

def test_conv_matches_materialised_matrix():
    rng = np.random.default_rng(0)
    C, T, L = 3, 5, 32
    h = rng.standard_normal((C, T))
    M = sbl.conv_matrix(h, L)
    phi, phit, D = sbl.conv_dictionary(h, L)
    z = rng.standard_normal((D, 2))
    w = rng.standard_normal((L, 2))
    np.testing.assert_allclose(phi(z), M @ z, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(phit(w), M.T @ w, rtol=1e-13, atol=1e-13)


def test_conv_matrix_vectorised_matches_loops():
    h = np.random.default_rng(2).standard_normal((3, 7))
    np.testing.assert_array_equal(sbl.conv_matrix_vectorised(h, 40), sbl.conv_matrix(h, 40))


def test_conv_adjoint_identity():
    rng = np.random.default_rng(1)
    C, T, L = 8, 64, 512
    h = rng.standard_normal((C, T))
    phi, phit, D = sbl.conv_dictionary(h, L)
    z = rng.standard_normal(D)
    w = rng.standard_normal(L)
    lhs = phi(z) @ w
    rhs = z @ phit(w)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.linalg.norm(z) * np.linalg.norm(w))


def test_datagen_conv_observation_matches_operator():
    # the generator's scatter of shifted filters equals the dictionary applied
    # to the ground truth (noise removed by sigma = 0)
    p = datagen.conv_problem(256, 4, 16, 0.02, 0.0, seed=3)
    phi, _, _ = sbl.conv_dictionary(p.h.astype(np.float64), 256)
    np.testing.assert_allclose(phi(p.z.reshape(-1)), p.y, rtol=1e-12, atol=1e-12)


# ------------------------------------------- preconditioned CG (learned path)

def test_pcg_identity_preconditioner_is_cg():
    Phi, alpha = _spd_problem(60, 90, 3)
    phi, phit, D = sbl.dense_dictionary(Phi)
    A = lambda X: sbl.apply_A(phi, phit, 2.0, alpha, X)
    B = np.random.default_rng(1).standard_normal((90, 4))
    r1 = sbl.cg_solve(A, B, 1e-10, 500)
    r2 = sbl.pcg_solve(A, B, np.zeros_like(B), np.ones(90), 1e-10, 500)
    assert r1.iters == r2.iters and np.array_equal(r1.X, r2.X)


def test_pcg_exact_diagonal_preconditioner_one_step():
    d = np.linspace(1, 100, 40)
    B = np.random.default_rng(2).standard_normal((40, 3))
    res = sbl.pcg_solve(lambda X: d[:, None] * X, B, np.zeros_like(B), 1.0 / d, 1e-13, 10)
    assert res.iters == 1
    np.testing.assert_allclose(res.X, B / d[:, None], rtol=1e-13)


def test_pcg_matches_cholesky_and_exact_start():
    Phi, alpha = _spd_problem(80, 120, 4, alpha_spread=(0.1, 10.0))
    beta = 5.0
    Am = beta * Phi.T @ Phi + np.diag(alpha)
    phi, phit, _ = sbl.dense_dictionary(Phi)
    A = lambda X: sbl.apply_A(phi, phit, beta, alpha, X)
    B = np.random.default_rng(5).standard_normal((120, 3))
    X_ref = np.linalg.solve(Am, B)
    minv = 1.0 / np.diag(Am)
    res = sbl.pcg_solve(A, B, np.random.default_rng(6).standard_normal((120, 3)), minv,
                        1e-13, 1000)
    assert res.converged
    assert np.linalg.norm(res.X - X_ref) / np.linalg.norm(X_ref) <= 1e-10
    res0 = sbl.pcg_solve(A, B, X_ref, minv, 1e-9, 10)
    assert res0.iters == 0


# ------------------------------------------------ per-column stop rule (c3)

def _spd_system(n=200, m=5, seed=3):
    """SPD A with eigenvalues spread over [1, 20] (CG in FP64 stays close to
    exact arithmetic), and right-hand sides that converge after 1, 3 and
    about 30-40 iterations."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.exp(rng.uniform(0.0, np.log(20.0), n))
    A = (Q * lam) @ Q.T
    A = (A + A.T) / 2
    B = rng.standard_normal((n, m)) * np.array([1e3, 1.0, 1e-2, 5.0, 1.0])[:m]
    if m > 4:
        B[:, 1] = Q[:, :3] @ np.ones(3)        # three eigenvectors: three iterations
        B[:, 4] = Q[:, 0]                      # one eigenvector: one iteration
    return A, B


def test_per_column_stop_equals_independent_cg():
    """stop_rule = 1 freezes each column at its own tolerance, so column j's
    iterates are those of a textbook CG on A x = b_j alone; scipy's cg stops
    on the same recursive-residual test ||r|| < rtol ||b||."""
    import scipy.sparse.linalg as sla
    A, B = _spd_system()
    tol = 1e-8
    res = sbl.cg_solve(lambda X: A @ X, B, tol, 500, stop_rule=1)
    assert res.converged
    iters = []
    for j in range(B.shape[1]):
        count = [0]

        def cb(xk):
            count[0] += 1
        x, info = sla.cg(A, B[:, j], rtol=tol, atol=0.0, maxiter=500, callback=cb)
        assert info == 0
        iters.append(count[0])
        # one iteration more or less moves x_j by 4e-9 or more here
        assert np.linalg.norm(res.X[:, j] - x) <= 1e-12 * np.linalg.norm(x), j
    assert res.iters == max(iters)
    assert len(set(iters)) > 2                 # the columns did stop at different points
    # every column meets its own test; the joint ratio is the reported one
    Rt = B - A @ res.X
    for j in range(B.shape[1]):
        assert np.linalg.norm(Rt[:, j]) < 1e-7 * np.linalg.norm(B[:, j])
    assert res.relres == pytest.approx(
        np.sqrt(np.sum((B - A @ res.X) ** 2)) / np.linalg.norm(B), rel=1e-3)


def test_per_column_stop_single_column_is_joint():
    """With one right-hand side the per-column and the joint rule coincide."""
    A, B = _spd_system(m=1)
    r0 = sbl.cg_solve(lambda X: A @ X, B, 1e-9, 500, stop_rule=0)
    r1 = sbl.cg_solve(lambda X: A @ X, B, 1e-9, 500, stop_rule=1)
    assert r0.iters == r1.iters
    np.testing.assert_array_equal(r0.X, r1.X)


def test_per_column_stop_ignored_with_fixed_iterations():
    A, B = _spd_system()
    r0 = sbl.cg_solve(lambda X: A @ X, B, 1e-8, 500, fixed_iters=7, stop_rule=0)
    r1 = sbl.cg_solve(lambda X: A @ X, B, 1e-8, 500, fixed_iters=7, stop_rule=1)
    assert r0.iters == r1.iters == 7
    np.testing.assert_array_equal(r0.X, r1.X)


# ------------------------------------------------ masked DCT dictionary (Sec. 4.2)

def test_dct_dictionary_matches_definition():
    """The oracle's FFT-based Phi / Phi^T equal the rows of the transposed
    DCT-II matrix written from its definition (index formula, loops)."""
    D = 64
    C = np.zeros((D, D))
    for k in range(D):
        for n in range(D):
            s = np.sqrt(1.0 / D) if k == 0 else np.sqrt(2.0 / D)
            C[k, n] = s * np.cos(np.pi * k * (2 * n + 1) / (2 * D))
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(D, 16, replace=False))
    phi, phit, _ = sbl.dct_dictionary(idx, D)
    Z = rng.standard_normal((D, 3))
    W = rng.standard_normal((16, 3))
    np.testing.assert_allclose(phi(Z), C.T[idx] @ Z, atol=1e-12)
    np.testing.assert_allclose(phit(W), C[:, idx] @ W, atol=1e-12)
    np.testing.assert_allclose(sbl.dct_matrix(D), C, atol=1e-14)


def test_dct_dictionary_closed_forms():
    """Orthonormality: Phi Phi^T = I_N; the DCT of a constant is sqrt(D) e_0
    and of the k-th cosine sqrt(D/2) e_k; the adjoint identity."""
    D = 256
    idx = np.arange(D)
    phi, phit, _ = sbl.dct_dictionary(idx, D)
    n = np.arange(D)
    e = phit(np.ones(D))
    assert abs(e[0] - np.sqrt(D)) < 1e-12 and np.max(np.abs(e[1:])) < 1e-12
    for k in (1, 5, 200):
        c = phit(np.cos(np.pi * k * (2 * n + 1) / (2 * D)))
        assert abs(c[k] - np.sqrt(D / 2)) < 1e-11
        c[k] = 0.0
        assert np.max(np.abs(c)) < 1e-11
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(D, 64, replace=False))
    phi, phit, _ = sbl.dct_dictionary(idx, D)
    W = rng.standard_normal((64, 2))
    np.testing.assert_allclose(phi(phit(W)), W, atol=1e-12)
    z, w = rng.standard_normal(D), rng.standard_normal(64)
    assert abs(phi(z) @ w - z @ phit(w)) < 1e-10


def test_dct_problem_generator():
    from paper_2202_12808_gb300 import datagen
    pr = datagen.dct_problem(1024, 256, 40, 0.0, seed=3)
    assert pr.idx.dtype == np.int32 and np.all(np.diff(pr.idx) > 0)
    assert np.count_nonzero(pr.z) == 40
    phi, _, _ = sbl.dct_dictionary(pr.idx, 1024)
    np.testing.assert_allclose(pr.y, phi(pr.z), atol=1e-12)


# ------------------------------------------------ multi-task extension (Sec. 5)

def test_multitask_identical_tasks_reduce_to_single_task():
    """T copies of one observation vector: every task's mean equals the
    single-task mean and the shared alpha equals the single-task alpha."""
    from paper_2202_12808_gb300 import datagen
    # overdetermined and well conditioned, so that the BLAS rounding of the
    # wider products (T + K columns instead of 1 + K) stays at 1e-13
    pr = datagen.dense_problem(200, 64, 8, 0.05, seed=2)
    Phi = pr.Phi.astype(np.float64)
    kw = dict(fixed_cg_iters=64, seed=3)
    a1, m1, s1, _ = sbl.cofem_dense(Phi, pr.y, pr.beta, 12, 2, 1e-8, 200, **kw)
    Y = np.stack([pr.y, pr.y, pr.y])
    a3, m3, s3, _ = sbl.cofem_dense(Phi, Y, pr.beta, 12, 2, 1e-8, 200, **kw)
    assert m3.shape == (3, 64)
    for t in range(3):
        np.testing.assert_allclose(m3[t], m1, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(a3, a1, rtol=1e-10)
    np.testing.assert_allclose(s3, s1, rtol=1e-10, atol=1e-13)


def test_multitask_matches_exact_em_step():
    """One EM step of multi-task CoFEM with converged CG and many probes
    against the exact multi-task EM step written from its definition:
    Sigma = (beta Phi^T Phi + diag alpha)^-1, mu_t = beta Sigma Phi^T y_t,
    alpha_d = 1 / (mean_t mu_td^2 + Sigma_dd)."""
    from paper_2202_12808_gb300 import datagen
    pr = datagen.multitask_problem(48, 96, 3, 6, 0.1, seed=4)
    Phi = pr.Phi.astype(np.float64)
    alpha0 = np.random.default_rng(0).uniform(0.5, 5.0, 96)
    A = pr.beta * Phi.T @ Phi + np.diag(alpha0)
    Sigma = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A), np.eye(96))
    mu_ex = pr.beta * (Sigma @ (Phi.T @ pr.Y.T)).T            # T x D
    alpha_ex = 1.0 / (np.mean(mu_ex ** 2, axis=0) + np.diag(Sigma))
    a, mu, s, _ = sbl.cofem_dense(Phi, pr.Y, pr.beta, 16000, 1, 1e-12, 500,
                                  alpha_init=alpha0, seed=5)
    np.testing.assert_allclose(mu, mu_ex, rtol=1e-7, atol=1e-10)
    assert np.linalg.norm(s - np.diag(Sigma)) <= 2e-2 * np.linalg.norm(np.diag(Sigma))
    assert np.linalg.norm(a - alpha_ex) <= 2e-2 * np.linalg.norm(alpha_ex)
