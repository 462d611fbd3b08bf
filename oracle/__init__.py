"""CPU oracle for the sTiles arrowhead tile Cholesky (TEST INFRASTRUCTURE).

This package is a plain, slow, obviously-correct FP64 restatement of what the
method computes.  It exists only to check the CUDA library: the tests, the
smoke check and the benchmark's CPU-baseline leg may import it; the library
never does, and it shares no code with the library.

Modules
-------
ordering  partial Reverse Cuthill-McKee of the body (Section III.A) and the
          "keep the permutation only if it reduces fill" rule.
tiles     the Compressed Tile Storage Format tile map (Section III.B), the
          tile-level symbolic factorization (Section II, step 2) and the
          per-task flop count.
cholesky  the left-looking sparse tile Cholesky of Algorithm 1 (lower
          storage), the log-determinant and the forward/backward solves.

Every function states the passage it follows.  Readings of places where the
paper is silent or garbled are stated where they are used.

Parity status: all functions are pinned by the ``-m "not gpu"`` tests
(dense brute force, closed forms, hand-checked orderings, brute-force
boolean elimination, the paper's accumulation count).  None is "parity
unpinned".
"""
