"""Plain FP64 CPU oracle of the sparse IDP DG stage update (Pazner, arXiv 2004.08503).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The GPU library never imports it, and it imports nothing from the GPU library.

The oracle writes the paper's operators out literally (Kronecker-product element
matrices, pairwise ``c_ij``/``d_ij`` coefficients, bar states, Zalesak and convex
limiting) with numpy in float64, vectorised over elements only.  Each function
cites the section / equation it follows.

Modules
  gll     -- Gauss-Lobatto nodes/weights, weighted derivative D, sparsified D-hat (Sec. 2.2, Eq. didp)
  laws    -- physical laws: constant advection, 2D Burgers, 2D Euler (Sec. 4.3, Eq. euler-eos/flux)
  scheme  -- HO residual, LO IDP residual, bar states, bounds, subcell FCT/convex limiter,
             CFL time step, SSP-RK3 (Sec. 2-4)
  curved  -- curved (mapped) quadrilateral meshes: metric terms, face normals, the conservative
             metric correction of Sec. 3.1 and the residuals on mapped elements

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
(closed forms, invariants, textbook special cases, brute force); none is "parity unpinned".
"""
from . import curved, gll, laws, scheme  # noqa: F401
