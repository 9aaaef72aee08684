"""Plain FP64 CPU oracle for TLR quasi-Monte Carlo MVN/MVT probabilities.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The GPU library never calls it, and it shares no code with the GPU path: the
two meet only in the seeded inputs of ``synth``.

Everything here follows the paper (arXiv 2003.11183, "Exploiting low rank
covariance structures for computing high-dimensional normal and Student-t
probabilities") step by step, in float64, written for a reader to check by eye:

- ``special``  univariate functions: Phi, log Phi, Phi^-1 (scipy), chi quantile
               (Section 2.1, Section 2.2 / Algorithm 3)
- ``lattice``  Richtmyer lattice with random shifts (Section 2.1, Section 3.4)
- ``geometry`` locations, geometric indexing, covariance kernels (Section 3.2)
- ``factor``   univariate conditioning, block reordering (Algorithm 4),
               iterative block reordering during Cholesky (Algorithm 5),
               adaptive cross approximation of the off-diagonal tiles (Section 3.3)
- ``sov``      dense SOV integrand (eq. 2 / Algorithm 1, Algorithm 3), TLR
               integrand (Algorithms 6 and 7), and the QMC estimator

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, library routines or brute force; the TLR integrand also at the
full size n = 65,536, on a problem whose per-sample value has a closed form
(``tests/test_oracle_full_size.py``).
"""
