"""CPU FP64 oracle for the refined-wall Stokes solve (arXiv 2108.07205).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant generator with the CUDA library in
``paper_2108_07205_gb300/csrc``.

What it computes is the plain definition of the method's result: the refined
Nystrom system of Sec. 2 (Eq. interior_BIE_discretized2) assembled densely and
solved by LAPACK LU.  The extended linear system and the Woodbury formula of
Sec. 3.2 (Eq. extendedlLinearSystem, Eq. wood) are also written out densely,
for tiny meshes, with the SVD factors of Sec. 3.4 (Eq. uniform_concat).

Modules
  quadrature  Gauss-Legendre rule (Sec. 5 preamble: 16-point composite panels).
  curves      star and constricted-channel wall curves with exact derivatives.
  discretize  panels, nodes, local refinement and index sets (Sec. 3.1).
  stokes      Stokeslet, double-layer matrix with the N correction (Sec. 2,
              Remark 2.1), velocity evaluation.
  dense       dense solve of the refined system; ELS and Woodbury (Sec. 3.2-3.4).
  holes       the wall with added holes (App. B): combined-field operator of
              Eq. exterior_BIE on the holes with a graded singular rule.
  exterior    the exterior problem on one wall (Sec. 2.2, Eq. exterior_BIE),
              reference and locally refined, with the same graded rule.

Parity status of each function is stated in its module docstring; every
function here is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants or brute force.
"""
