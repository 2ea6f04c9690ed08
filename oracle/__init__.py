"""FP64 CPU oracle for covariance-free EM (CoFEM) -- TEST INFRASTRUCTURE ONLY.

This package is the slow, plain, obviously-correct reference that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (``paper_2202_12808_gb300``) never imports, links or calls it, and
the two share no code: the only common dependency is the seeded input
generator module, which holds none of the method's arithmetic.

Everything here is float64 numpy, written in the order and notation of the
paper (Lin, Song, Bilgic, Ba, "High-Dimensional Sparse Bayesian Learning
without Covariance Matrices", ICASSP 2022):

* ``probe_hash``  -- the counter-based Rademacher probe generator (SplitMix64).
* ``sbl``         -- the dictionary operators, column-wise CG (Sec. 3.2),
                     Algorithm 1 (CoFEM), exact EM (Eq. estep-params, mstep)
                     and the type-II likelihood (Eq. mle2).
* ``mlp``         -- the per-coordinate MLP used by the learned warm start /
                     preconditioner (forward, backward, Adam).

Parity status of each function is stated in its module header.
"""
