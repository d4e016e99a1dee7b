"""CPU oracle for the photonic band-structure path (TEST INFRASTRUCTURE ONLY).

A plain, slow, FP64 NumPy/SciPy implementation of what the GPU path computes,
written from the paper (Boerm, Koehl, Talebi, arXiv:2304.00337) and sharing no
code with the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline / reference leg) may import it; the product path
never does.

Modules and what pins each (tests under ``tests/test_oracle_*.py``):

* ``fem``        - basis functions and Galerkin assembly (Section 3).  Pinned by
  the closed-form Bloch dispersion for constant eps, Stokes' theorem on Bloch
  plane waves (curl and gradient DOFs), ``A L = 0``, Hermitian / definiteness
  properties, hand-computed element integrals and the Galerkin coarse-grid
  identity.
* ``eigen``      - smallest non-zero eigenpairs of the pencil (dense and sparse),
  closed-form spectrum, factored Rayleigh quotients.  Pinned by the closed form,
  dense-vs-reduced brute force, and ``lambda(k) = lambda(-k)``.
* ``multigrid``  - reference edge and nodal V-cycles (Section 5).  Pinned by
  convergence of the iterated cycle to a sparse direct solve, Hermiticity of
  the symmetric cycle and exactness of each patch solve.  Its contraction
  factor is not printed in the paper: parity against the paper is unpinned,
  only the algorithm's invariants are.
* ``extrapolation`` - Rayleigh-Ritz on a span after exact gradient projection
  (Sections 4 and 7).  Pinned by Courant-Fischer bounds and exactness on an
  invariant subspace.
"""
from . import fem, eigen, multigrid, extrapolation  # noqa: F401
