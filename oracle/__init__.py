"""CPU oracle for the JFNK NLTE hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 restatement of what the paper computes, written from the
paper (arXiv:2406.17234) and from the published methods it cites, to check
the CUDA library against. It shares no code, headers, tables or constants
with the library under ``paper_2406_17234_gb300/`` and imports nothing from
it; the two meet only through the seeded descriptors of ``workloads``.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run this package.
The product path never routes through it.

Modules
  model     -- setup: grids, quadratures, LTE populations, Voigt profiles,
               collision rates, background (Sect. 2.1.1, Eqs. Vij-gij)
  formal    -- piecewise-linear short-characteristic formal solver
               (Eqs. Iplus/Iminus, App. A)
  residual  -- Algorithm 1 (residual F), complex-step and finite-difference
               Jacobian-vector products (Eqs. fordif-complex)
  precond   -- block-Jacobi preconditioner, "first solution" of Sect. 2.5.2
  krylov    -- GMRES (Arnoldi, Givens) and BiCGSTAB (Sect. 2.3)
  jfnk      -- Algorithm 2
  rh92      -- the reference method: linearisation with operator splitting
               and a local operator (Rybicki & Hummer 1992, full
               preconditioning)
  dense     -- dense Jacobian from unit-vector JVPs and dense Newton-Raphson
               (brute force on tiny grids)

Parity status per function is stated in each module header; every function
listed above is pinned by tests in ``tests/test_oracle_*.py``.
"""
