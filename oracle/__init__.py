"""FP64 CPU oracle for the matrix/tensor-oriented FCGLE time stepping.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the C-ABI library,
its Python binding, ``bench.py``'s timed GPU arm) may import, call or link
anything in this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

It is written from the paper (Caliari & Cassini, "matrix- and
tensor-oriented ... space-fractional complex Ginzburg--Landau equation",
arXiv 2510.21394) and shares no code with the CUDA path:

* ``fd``      -- finite-difference coefficients g_k (Sec. 2, FD2 recurrence)
                 and their fourth-order extrapolation (Sec. 2, Eq. FD4), the
                 Toeplitz matrices D_n^alpha (Eq. Dnalpha), grids (Sec. 2).
* ``phi``     -- scalar phi_l functions (Eq. phi), FP64.
* ``brute``   -- O1: the dense Kronecker sum K (Eq. Ksum) and f(theta K) v by
                 dense solve / expm / augmented-matrix exponential.  No
                 eigendecomposition anywhere.  Tiny grids only.
* ``tensor``  -- O2: mu-mode products, the Tucker form of f(theta K) v
                 (Eq. fKu_diag) and the Kronecker-product form of exp
                 (Eq. Neudeckerd), from numpy ``eigh`` of each D_mu.
* ``schemes`` -- the time integrators written in their vector form (Sec. 4:
                 Eqs. lbdf2-v, Strang, krogstad-v) plus Lawson-Euler,
                 Heun-based Lawson-RK2 and Cox-Matthews ETD2RK (standard forms,
                 stated in ``schemes``), on top of ``tensor``.
* ``adjoint`` -- the discrete adjoint of the Lawson-RK2 step and the gradient
                 of a final-time misfit.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, mpmath, brute force,
printed numbers of the paper); see ``tests/test_oracle_*.py``.
"""
