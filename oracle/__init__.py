"""FP64 CPU oracle for periodic frozen-density-embedding (subsystem) DFT.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the CUDA library computes.  Only the test-suite, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it; the product
path never does, and it shares no code with the CUDA library (both take their seeded
inputs from ``paper_1406_7803_gb300.workloads``, which holds no arithmetic of the method).

Every function cites the passage of Genova, Ceresoli & Pavanello, "Periodic Subsystem
Density-Functional Theory" (arXiv:1406.7803) it follows.  Readings of points where the
paper is silent or garbled are fixed in ``oracle.conventions`` and listed in the design
notes of the repository.

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or library routines, with these exceptions:

* parity unpinned: the absolute energies of the synthetic cells, which have no external
  value beyond the invariants (see ``oracle.scf``);
* parity unpinned: revAPBEK kappa = 1.245 and mu = 0.23889 (the cited functional's
  published constants; the tests pin only the form: F(0) = 1, F''(0) = 2 mu,
  F(inf) = 1 + kappa);
* parity unpinned: LC94 a, b, alpha, f and the split of c + d (the tests pin the
  second-order gradient expansion c + d = 5/27 to 4e-4);
* PW92 alpha_1, beta_1..beta_4 and A are pinned through the high- and low-density
  expansions (c0, c1, d0, d1) and PW92's construction beta_2 = 2 A beta_1^2; PBE kappa,
  beta and gamma through the Lieb-Oxford bound, the Ma-Brueckner coefficient and c0.
"""
