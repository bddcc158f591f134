"""Plain FP64 CPU oracle for the 2D FMM of Luo & Duraiswami, "Alternative tilings
for the fast multipole method on the plane" (arXiv:1204.3105).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import or run anything in this
package.  The product path (the CUDA library under ``paper_1204_3105_gb300``)
never calls it and shares no code, tables or constants with it.

What is here, each file citing the passage it follows:

* ``tiling_quad``  - quadtree with Morton Z indexing (Sec. 4, Fig. 3a).
* ``tiling_sept``  - septree: GBT base-7 arithmetic from the unit-sum table
  (Sec. 5.1, Fig. 4b), Neighbors, zero-extension, CellCenter (eq. 6) and
  CellIndex (eqs. 7-9), each as the paper states it, plus an independent
  Eisenstein-integer route for the same keys.
* ``tiling_tri``   - triangle quadtree: adjacentNeighbor with Table 1,
  the 12-neighbour recursion, isUp (eq. 11), CellCenter (eq. 12) and the
  nearest-of-four CellIndex descent (eq. 13), plus an exact fixed-point
  barycentric descent for the same keys.
* ``params``       - separation ratios (Table 2, Sec. 7), the truncation
  order p(eps) and the root-cell geometry of each tiling.
* ``fmm``          - the FMM itself (Sec. 2): keys, stable sort, cells per
  level, Near / NeighborsE4 lists (Sec. 4, eq. 3), P2M, M2M, M2L, L2L, L2P
  (the Greengard-Rokhlin operators the paper defers to its references) and
  the P2P near-field sum.
* ``direct``       - brute-force O(NM) evaluation of eq. (2) with compensated
  FP64 summation.

Readings of the paper that the oracle relies on (see the docstrings):
the potential graded is Re Phi = sum_i u_i log|y_j - x_i| (the complex log
of eq. 1 is multivalued, only its real part is single valued); coincident
source/target pairs are skipped; NeighborsE4 is the set difference
Children[Parent(n) u Neighbors(Parent(n))] minus ({n} u Neighbors(n)).

Parity unpinned: the imaginary part of Phi (branch dependent, not graded).
"""
