"""Oracle for the BURA fractional solver — TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, obviously-correct CPU statement of what the GPU
path computes.  It is imported only by ``tests/``, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (the CUDA library and its Python binding) never imports, links or
runs anything in here, and this package shares no code with it.

Modules
-------
remez      1-BURA of t^(1-alpha) on [0,1] by the modified Remez algorithm
           (Algorithm 1, Sec. 3.2) in multi-precision, plus the
           partial-fraction coefficients c_j, d_j of eq. (simplified), Sec. 2.2.
           Equations are cited by their LaTeX labels in the paper.
operators  the scaled matrix  A = Atilde / Lambda  (eq. (algebraic), Sec. 1.2) for 5-point and
           7-point finite-difference operators -div(a grad u) on uniform grids
           with homogeneous Dirichlet data, as scipy.sparse matrices.
exact      closed-form sine-transform eigenbasis solutions on constant-
           coefficient grids (eq. (exacalg), Sec. 5.1): exact A^{-alpha} f and the
           exact BURA value  u_r = sum_j c_j (A - d_j I)^{-1} f  (eq. (Rgeneral)).
direct     the same two quantities for any operator: sparse direct solves of
           every shifted system (eq. (Rgeneral)), and dense eigendecomposition
           for tiny matrices (eq. (exacalg)).
pcg        the same method on the CPU for any operator: every shifted system solved on its own by
           multigrid-preconditioned CG in FP64 (C with OpenMP, oracle/cpu_pcg.c), then the
           weighted sum of eq. (Rgeneral); the oracle of the variable-coefficient operators and
           the timed same-method CPU baseline.
quadrature the sinc quadrature of [BP15] of the paper's comparison (eq. (BonitoPasciak), Sec. 5.3).
tables     lookup of the committed oracle-generated coefficient table.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against values the paper prints or against closed forms / invariants; see
tests/test_oracle_*.py.  No function is "parity unpinned".
"""
