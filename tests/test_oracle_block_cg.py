"""Pins of the oracle's block CG (oracle/sbl.py::block_cg_solve and
cofem(solver=1)): the block method's defining property, its special cases
and the E-step it feeds, each checked against something other than the
recurrence itself.

* Galerkin: after k iterations from X0 = 0, every column of X is the
  A-orthogonal projection of the solution onto the block Krylov space
  span{B, A B, .., A^(k-1) B} (O'Leary 1980, Thm. 2) -- computed here by
  brute force from an orthonormal basis of that space.
* One column: the block recurrence is plain CG (Sec. 3.2's solver).
* Finite termination after D / m iterations (the block Krylov space is the
  whole space), recursive residual = true residual, a zero right-hand
  side, B = 0.
* cofem(solver=1): the closed form of an E-step with A = c I, and the
  column-wise fit at a tight tolerance.
"""
import numpy as np
import pytest

from oracle import sbl


def spd(D, lo, hi, seed):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((D, D)))
    ev = np.linspace(lo, hi, D)
    return (Qm * ev) @ Qm.T


def galerkin(A, B, k):
    """A-orthogonal projection of A^-1 B onto span{B, .., A^(k-1) B}."""
    blocks = [B]
    for _ in range(k - 1):
        blocks.append(A @ blocks[-1])
    V, _ = np.linalg.qr(np.concatenate(blocks, axis=1))
    return V @ np.linalg.solve(V.T @ A @ V, V.T @ B)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_block_cg_is_the_block_krylov_galerkin_solution(k):
    D, m = 30, 3
    A = spd(D, 1.0, 10.0, 0)
    B = np.random.default_rng(1).standard_normal((D, m))
    res = sbl.block_cg_solve(lambda X: A @ X, B, 0.0, 100, fixed_iters=k)
    assert res.iters == k
    ref = galerkin(A, B, k)
    assert np.max(np.abs(res.X - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_block_cg_one_column_is_plain_cg():
    D = 50
    A = spd(D, 0.5, 20.0, 2)
    b = np.random.default_rng(3).standard_normal((D, 1))
    r1 = sbl.block_cg_solve(lambda X: A @ X, b, 1e-10, 200)
    r0 = sbl.cg_solve(lambda X: A @ X, b, 1e-10, 200)
    assert r1.iters == r0.iters
    assert np.max(np.abs(r1.X - r0.X)) <= 1e-11 * np.max(np.abs(r0.X))
    assert abs(r1.relres - r0.relres) <= 1e-6 * r0.relres


def test_block_cg_terminates_after_d_over_m_iterations():
    D, m = 12, 3
    A = spd(D, 1.0, 50.0, 4)
    B = np.random.default_rng(5).standard_normal((D, m))
    res = sbl.block_cg_solve(lambda X: A @ X, B, 1e-11, 100)
    assert res.converged and res.iters <= D // m
    assert np.max(np.abs(res.X - np.linalg.solve(A, B))) <= 1e-9


@pytest.mark.parametrize("k", [1, 3, 6])
def test_block_cg_recursive_residual_is_the_true_residual(k):
    D, m = 40, 4
    A = spd(D, 1.0, 100.0, 6)
    B = np.random.default_rng(7).standard_normal((D, m))
    res = sbl.block_cg_solve(lambda X: A @ X, B, 0.0, 100, fixed_iters=k)
    true = np.linalg.norm(B - A @ res.X) / np.linalg.norm(B)
    assert abs(res.relres - true) <= 1e-9 * true


def test_block_cg_zero_column_and_zero_b():
    """A zero right-hand side makes the block rank-deficient: its column of
    X stays zero and the other columns still solve their systems."""
    D = 20
    A = spd(D, 1.0, 5.0, 8)
    B = np.random.default_rng(9).standard_normal((D, 3))
    B[:, 0] = 0.0
    res = sbl.block_cg_solve(lambda X: A @ X, B, 1e-12, 50)
    assert res.converged
    assert not np.any(res.X[:, 0])
    assert np.max(np.abs(res.X - np.linalg.solve(A, B))) <= 1e-10
    Z = sbl.block_cg_solve(lambda X: A @ X, np.zeros((D, 3)), 1e-8, 50)
    assert Z.iters == 0 and not np.any(Z.X)


def test_cofem_block_e_step_with_scaled_identity_system():
    """Phi with orthonormal columns and alpha = 1 (t = 1): A = (beta + 1) I,
    so block CG ends after one iteration with X = B / (beta + 1); mu =
    beta Phi^T y / (beta + 1), s_d = 1 / (beta + 1) exactly (p_kd^2 = 1),
    alpha = 1 / (mu^2 + s)."""
    N, D, K, beta = 32, 16, 3, 4.0
    rng = np.random.default_rng(10)
    Phi, _ = np.linalg.qr(rng.standard_normal((N, D)))
    y = rng.standard_normal(N)
    alpha, mu, s, st = sbl.cofem_dense(Phi, y, beta, K, 1, 1e-10, 50, solver=1)
    assert st.cg_iters == [1]
    mu_ref = beta * (Phi.T @ y) / (beta + 1.0)
    assert np.max(np.abs(mu - mu_ref)) <= 1e-13
    assert np.max(np.abs(s - 1.0 / (beta + 1.0))) <= 1e-13
    assert np.max(np.abs(alpha - 1.0 / (mu_ref ** 2 + 1.0 / (beta + 1.0)))) <= 1e-12 * np.max(alpha)


def test_cofem_block_matches_column_wise_fit_at_tight_tolerance():
    """Both solvers solve the same E-step systems; at tol 1e-12 the fits
    agree to the solves' accuracy (relative residual 1e-12 times cond(A),
    which grows with the pruned alpha, carried through five M-steps: 2e-7
    measured), with fewer block iterations."""
    rng = np.random.default_rng(11)
    N, D, K = 48, 96, 8
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    z = np.zeros(D)
    z[rng.choice(D, 6, replace=False)] = rng.standard_normal(6)
    y = Phi @ z + 0.05 * rng.standard_normal(N)
    beta = 1.0 / 0.05 ** 2
    a0, m0, s0, st0 = sbl.cofem_dense(Phi, y, beta, K, 5, 1e-12, 500)
    a1, m1, s1, st1 = sbl.cofem_dense(Phi, y, beta, K, 5, 1e-12, 500, solver=1)
    assert np.max(np.abs(a1 - a0) / a0) <= 1e-6
    assert np.max(np.abs(m1 - m0)) <= 1e-7 * np.max(np.abs(m0))
    assert sum(st1.cg_iters) < sum(st0.cg_iters)


def test_cofem_block_rejects_replacement_and_per_column_rule():
    Phi = np.eye(4)
    with pytest.raises(ValueError):
        sbl.cofem_dense(Phi, np.ones(4), 1.0, 1, 1, 1e-8, 10, solver=1, resid_replace_every=5)
    with pytest.raises(ValueError):
        sbl.cofem_dense(Phi, np.ones(4), 1.0, 1, 1, 1e-8, 10, solver=1, stop_rule=1)
