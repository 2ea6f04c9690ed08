"""Pins of the oracle's learned CoFEM loop (sbl.cofem_learned) against what
the mathematics fixes, CPU only.

The loop is Algorithm 1 with a warm start X0 = [mu_hat | s_hat . p_k] and a
diagonal preconditioner M^-1 = diag(s_hat) from E-step 2 on, plain CG at the
first E-step, and plain CG from zero when the preconditioned solve misses the
tolerance within the cap (each E-step then counts both solves).  Each test
below fails on one of the plausible mistakes: s_hat applied to the wrong
columns, the first-E-step branch skipped, the predictor fed the wrong state,
a fallback counted twice or its result dropped.
"""
import numpy as np

from oracle import sbl
from paper_2202_12808_gb300 import datagen


def _orthonormal(D=64, seed=31, beta=40.0):
    Phi = datagen.orthonormal_columns(D, D, seed)
    q = np.linspace(-0.6, 0.6, D)
    y = Phi @ q
    return Phi, y, beta, Phi.T @ y


def test_exact_predictor_needs_no_iterations():
    """Orthonormal Phi: A = diag(beta + alpha), the E-step is mu = beta q /
    (beta + alpha), Sigma_dd = 1 / (beta + alpha).  A predictor that returns
    exactly that makes X0 the solution of A X = B (s_hat applied to the probe
    columns, mu_hat to column 0), so every learned solve stops before its
    first iteration, none falls back, and alpha follows the closed-form EM
    recursion alpha' = 1 / (mu^2 + 1/(beta + alpha)).  The first E-step runs
    plain CG (one iteration: A is a multiple of I at alpha = 1)."""
    Phi, y, beta, q = _orthonormal()
    D = Phi.shape[1]
    phi, phit, _ = sbl.dense_dictionary(Phi)
    calls = []

    def predict(alpha, mu_prev, s_prev):
        calls.append(alpha.copy())
        return beta * q / (beta + alpha), 1.0 / (beta + alpha)

    em = 6
    alpha, mu, s, st = sbl.cofem_learned(phi, phit, D, y, beta, 8, em, 1e-10, 50, predict,
                                         seed=3)
    assert st.cg_iters == [1] + [0] * (em - 1)
    assert st.fallbacks == [0] * em
    assert len(calls) == em - 1                       # not called at the first E-step
    a = np.ones(D)
    for t in range(em):
        a_next = 1.0 / ((beta * q / (beta + a)) ** 2 + 1.0 / (beta + a))
        if t >= 1:
            np.testing.assert_allclose(calls[t - 1], a, rtol=1e-12)
        a = a_next
    np.testing.assert_allclose(alpha, a, rtol=1e-12)
    np.testing.assert_allclose(s, 1.0 / (beta + calls[-1]), rtol=1e-12)


def test_exact_preconditioner_converges_in_one_iteration():
    """Same orthonormal problem, predictor with the exact variance but
    mu_hat = 0: the probe columns start solved, column 0 starts at R = B, and
    PCG with M^-1 = A^-1 (A diagonal) reaches the solution in exactly one
    iteration; mu is then the exact E-step mean."""
    Phi, y, beta, q = _orthonormal(seed=32)
    D = Phi.shape[1]
    phi, phit, _ = sbl.dense_dictionary(Phi)

    def predict(alpha, mu_prev, s_prev):
        return np.zeros(D), 1.0 / (beta + alpha)

    em = 5
    alpha, mu, s, st = sbl.cofem_learned(phi, phit, D, y, beta, 4, em, 1e-10, 50, predict,
                                         seed=4)
    assert st.cg_iters == [1] * em
    assert st.fallbacks == [0] * em
    a_prev = np.ones(D)
    for _ in range(em - 1):
        a_prev = 1.0 / ((beta * q / (beta + a_prev)) ** 2 + 1.0 / (beta + a_prev))
    np.testing.assert_allclose(mu, beta * q / (beta + a_prev), rtol=1e-12)


def test_untrustworthy_prediction_falls_back_to_the_plain_fit():
    """A predictor whose s_hat is e^40 starts every learned solve from a
    residual ~1e17 ||B||: with a cap of 3 iterations every E-step from the
    second on falls back once, counts 3 + the plain solve's iterations, and
    keeps the plain solve's result -- so the whole fit equals sbl.cofem.  The
    predictor receives, at E-step t, the alpha, mu and s that the plain fit
    has after t - 1 E-steps."""
    pr = datagen.dense_problem(48, 160, 6, 0.05, seed=5)
    Phi = pr.Phi.astype(np.float64)
    phi, phit, D = sbl.dense_dictionary(Phi)
    seen = []

    def predict(alpha, mu_prev, s_prev):
        seen.append((alpha.copy(), mu_prev.copy(), s_prev.copy()))
        return np.ones(D), np.full(D, np.exp(40.0))

    em, cap, tol = 5, 3, 1e-6
    la, lmu, ls, lst = sbl.cofem_learned(phi, phit, D, pr.y, pr.beta, 6, em, tol, cap, predict,
                                         seed=8)
    # the plain fit needs more than `cap` iterations per E-step, so the cap
    # also ends the plain solves: run it with the same cap and compare
    pa, pmu, ps, pst = sbl.cofem(phi, phit, D, pr.y, pr.beta, 6, em, tol, cap, seed=8)
    assert lst.fallbacks == [0] + [1] * (em - 1)
    assert lst.cg_iters == [pst.cg_iters[0]] + [cap + c for c in pst.cg_iters[1:]]
    np.testing.assert_allclose(la, pa, rtol=1e-12)
    np.testing.assert_allclose(lmu, pmu, rtol=1e-12)
    np.testing.assert_allclose(ls, ps, rtol=1e-12)
    for t in range(2, em + 1):
        a_t, mu_t, s_t, _ = sbl.cofem(phi, phit, D, pr.y, pr.beta, 6, t - 1, tol, cap, seed=8)
        a_seen, mu_seen, s_seen = seen[t - 2]
        np.testing.assert_allclose(a_seen, a_t, rtol=1e-12)
        np.testing.assert_allclose(mu_seen, mu_t, rtol=1e-12)
        np.testing.assert_allclose(s_seen, s_t, rtol=1e-12)


def test_fallback_at_full_cap_keeps_plain_iterates():
    """With a cap the plain solve does not reach (it converges), a failed
    learned solve costs exactly `cap` iterations on top of the plain ones and
    the accepted iterates are the plain CG iterates from zero."""
    pr = datagen.dense_problem(48, 160, 6, 0.5, seed=6)     # beta = 4: well conditioned
    Phi = pr.Phi.astype(np.float64)
    phi, phit, D = sbl.dense_dictionary(Phi)

    def predict(alpha, mu_prev, s_prev):
        return np.zeros(D), np.full(D, np.exp(40.0))

    em, cap, tol = 2, 50, 1e-8
    la, lmu, ls, lst = sbl.cofem_learned(phi, phit, D, pr.y, pr.beta, 4, em, tol, cap, predict,
                                         seed=2)
    pa, pmu, ps, pst = sbl.cofem(phi, phit, D, pr.y, pr.beta, 4, em, tol, cap, seed=2)
    assert max(pst.cg_iters) < cap
    assert lst.fallbacks == [0, 1]
    assert lst.cg_iters == [pst.cg_iters[0]] + [cap + c for c in pst.cg_iters[1:]]
    assert max(lst.relres) < tol
    np.testing.assert_allclose(lmu, pmu, rtol=1e-12)
    np.testing.assert_allclose(la, pa, rtol=1e-12)


def test_learned_and_plain_first_estep_identical():
    """At the first E-step the learned loop runs the paper's plain CG: one
    EM iteration of both loops gives the same alpha, mu and s."""
    pr = datagen.dense_problem(40, 120, 5, 0.05, seed=7)
    phi, phit, D = sbl.dense_dictionary(pr.Phi.astype(np.float64))

    def predict(alpha, mu_prev, s_prev):
        raise AssertionError("no prediction at the first E-step")

    la, lmu, ls, lst = sbl.cofem_learned(phi, phit, D, pr.y, pr.beta, 5, 1, 1e-8, 300, predict,
                                         seed=9)
    pa, pmu, ps, pst = sbl.cofem(phi, phit, D, pr.y, pr.beta, 5, 1, 1e-8, 300, seed=9)
    assert lst.cg_iters == pst.cg_iters
    np.testing.assert_allclose(la, pa, rtol=1e-13)
    np.testing.assert_allclose(lmu, pmu, rtol=1e-13)
    np.testing.assert_allclose(ls, ps, rtol=1e-13)
