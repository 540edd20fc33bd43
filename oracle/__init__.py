"""CPU oracle for the Diffuse hot path -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import anything from this package.
The product path (the C-ABI library and its Python binding) never calls it and
shares no code with it.

What it holds:
  * ``ops``      -- the element operations of the task bodies, in FP64 or in the
                    stored dtype (Section 2, Fig. 1e/1f; Section 6, Fig. 8).
  * ``ir``       -- the paper's IR and its definitions written out plainly:
                    sub-store bounds (Fig. 3e), point dependencies (Def. 1),
                    dependence maps (Def. 2), fusibility (Def. 3), the four
                    fusion constraints (Fig. 5), the greedy prefix (Section
                    4.2.2), temporaries (Def. 4) and the canonical window form
                    (Section 5.2).
  * ``interp``   -- an unfused task-stream interpreter: every index task runs
                    point by point, one loop per task, every temporary stored.
  * ``programs`` -- the workloads written as unfused programs in program order:
                    Black-Scholes, CG, the Fig. 1 Jacobi stencil and its 3-D
                    7-point analogue, BiCGSTAB.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, textbook values, invariants or brute force; none is
"parity unpinned".
"""
