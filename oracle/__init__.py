"""Plain FP64 CPU oracle for the NN-corrected nodal DGSEM of arXiv 2207.11571.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library ``libdgnn.so`` and its Python binding) never imports, calls or links
anything here, and nothing here imports the product package: the two share no
code.  Inputs that both sides consume (seeded random perturbations, random
states, initial weights) are passed in as arrays.

Everything is written for a reader checking it against the paper by eye:
numpy in float64, one step of the method per function, no blocking or fusion.

Modules
  basis      Gauss-Lobatto nodes/weights, Lagrange derivative matrix, Legendre
             modal filter (the projection G of Sec. 2, Eq. 2; Sec. 2.6).
  physics    compressible Navier-Stokes fluxes (Appendix A), Roe flux, BR1
             interface viscous flux, Smagorinsky eddy viscosity (Sec. 3.1).
  dgsem      periodic hex mesh, Taylor-Green initial field (Sec. 3.1, Eq. 11),
             strong-form DGSEM operator p(q) (Eq. 1/3), BR1 lifted gradients,
             low-storage RK3 (Sec. 2, Eq. 6 generalised), diagnostics (Eq. 9).
  mlp        fully connected forcing network (Sec. 2.2, Fig. 2): forward,
             backward, MSE loss and Adam, with optional bf16 rounding points.
  algorithm1 training-pair generation, the corrected evolution (Algorithm 1,
             Eq. 4-6).

Parity pins live in ``tests/test_oracle_*.py``.  Functions without an
independent pin say "parity unpinned" in their docstring.  Parity unpinned, because
the paper does not fix them: the closure constants of
``physics.transport_coefficients`` (filter width h/(P+1) and Pr_t = 0.9; the
eddy-viscosity formula itself is pinned) and the constant of ``dgsem.stable_dt``
(its form is pinned by the order ratios printed in Sec. 2.3).
"""
