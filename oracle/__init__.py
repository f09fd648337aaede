"""FP64 CPU oracle for the Legendre-multipole 3PCF (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_2604_08855_gb300``; the two meet only through the seeded
input generators.

Parity status of each function (what pins it is listed in the tests):
  ylm    pinned: scipy's complex spherical harmonics, the addition theorem,
         orthonormality by quadrature.
  alm    pinned through zeta (hand geometries, triplets) and the addition
         theorem on its own output.
  zeta   pinned: O(N^3) triplet sum with numpy Legendre polynomials, the
         l = 0 closed form with scipy's cKDTree neighbour counts, hand-built
         geometries with printed P_l values, invariances.
  contract  the contraction of given a_lm rows alone; pinned: it reproduces
         zeta from the oracle's own a_lm (whose zeta is pinned as above).
  ambiguous  the pairs within a relative tolerance of a bin edge; pinned:
         hand-placed pairs at and near edges, and its count equals zeta's
         namb.
  zeta_sphere  pinned: frame-free triplet sum (angles between tangent
         projections), the m = 0 closed form with scipy's cKDTree chord
         counts, a hand geometry at the pole and on the equator, rotation
         invariance.
  shared.*  the shared-neighbour-list estimate and its error bounds (3-D
         and sphere); the pins are listed in shared.py.
  edge.edge_correct  pinned: sympy's Wigner 3j symbols, exact Legendre
         quotients built with numpy's legmul, flat randoms (plain ratio),
         quadrature of N/R.
"""
from .oracle import build, ylm, alm, ambiguous, contract, zeta, zeta_sphere, max_threads, lib_path  # noqa: F401
from . import edge, shared  # noqa: F401
