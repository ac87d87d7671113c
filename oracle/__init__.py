"""Plain FP64 CPU oracle for the ACM-HD flux-reconstruction right-hand side.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method that the CUDA path is checked against.  Only the
test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
(the CUDA library and its Python binding) never imports, links or calls it,
and it imports nothing from the product package.

Modules
-------
ops1d     1-D Gauss-Legendre nodes, Lagrange interpolation/derivative,
          FR correction functions (Sec. 2.1, FR divergence equation).
acmhd     ACM-HD flux, source and Rusanov/mean common flux
          (Sec. 2.2, Eqs. acmhd_2d and acmhd_nd; Sec. 5 for the common flux).
fr        The six-stage FR right-hand side of Table fr_adv, sum-factorised
          along tensor-product lines, plus a dense Kronecker-product variant
          for tiny meshes and a per-element evaluator for sampled checks.
timestep  Classical RK4 pseudo-time step, BDF2 dual time stepping and the
          FP64 velocity residual (Sec. 5).
mlp       Per-element MLP forward/backward/Adam for the learned initial guess
          (no counterpart in the paper).
pmg       P-multigrid (full approximation scheme over the orders p .. 0) and
          Anderson mixing of its cycles for the pseudo-time solve (Sec. 5).

Parity status: every module's docstring lists what pins it (closed forms,
textbook operators derived independently with sympy, invariants, brute
force, planted-mistake tests); no function is left "parity unpinned".
"""
