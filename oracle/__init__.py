"""Plain FP64 CPU oracle for the isogeometric single-layer BEM with interpolation FMM.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (the CUDA library and its Python binding) never calls into this
package, and this package imports nothing from the product path.

What it computes (Dölz, Harbrecht, Kurz, Schöps, Wolf, "A fast isogeometric BEM
for the three dimensional Laplace- and Helmholtz problems"):

* Gauss-Legendre rules (Sec. 4, item 4)                         -> ``gauss``
* p-open knot vectors, Cox-de Boor B-splines (Def. 2.1, Sec. 2.2) -> ``bspline``
* patch maps F_j and surface measure k_j (Eq. def::geom, Sec. 3.2) -> ``geometry``
* touching-pair detection and Duffy / Sauter-Schwab style rules
  for singular element pairs (Sec. 4, item 4)                    -> ``singular``
* the dense Galerkin matrix of the single-layer operator in the
  B-spline space S_{p,m} (Eqs. varformdisc, Sec. 3.2)             -> ``galerkin``
* cluster tree, admissibility and block cluster tree (Sec. 4.1,
  Def. 4.1)                                                      -> ``tree``
* interpolation (degenerate-kernel) far field, non-nested
  (Sec. 4.2)                                                     -> ``fmm``
* right-hand side, solvers, potential evaluation (Eq. repform)   -> ``solve``

Everything is written directly in the B-spline basis of S_{p,m}: the oracle has
no Bernstein superspace, no Bézier extraction and no nested cluster bases, so it
shares no structure with the GPU path, which works in the superspace S*_{p,m}
and with nested (M2M / L2L) transfers.

Parity status per function is recorded in the module docstrings; every public
function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""
