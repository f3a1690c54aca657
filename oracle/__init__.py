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
closed forms, invariants, brute force or library routines, except the absolute energies
of the synthetic cells, which have no external value ("parity unpinned" beyond the
invariants; see ``oracle.scf``).
"""
