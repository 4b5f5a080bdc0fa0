"""FP64 CPU oracle for the doubly periodic periodizing operator.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
links this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA library (no headers, helpers, tables or
generators).

Contents (Pei, Askham, Greengard & Jiang, "Periodic Fast Multipole Method",
arXiv 2111.01083):

* ``lattice``  -- canonical cell, wrapping, near/far image split (Sec. 1,
  Definition of Lambda_near / Lambda_far; Sec. 3 validity argument).
* ``greens``   -- free-space Green's functions: (1/2pi) log(1/r),
  (1/2pi) K0(beta r) (Sec. 1), the Stokeslet (Sec. 5.2) and the modified
  Stokeslet (Eq. msgreen).
* ``ewald``    -- the DEFINITION of the periodic operator, K^(p) q, by Ewald
  splitting, and the near-block direct sum K^near q; P2 q = K^(p) q - K^near q
  (Sec. 1, eqs. for K^near / K^far, Definition "periodizing operators").
* ``theta``    -- Jacobi-theta closed form of the Laplace periodic Green's
  function (independent pin of ``ewald`` for Laplace).
* ``brute``    -- absolutely convergent brute-force image sums for modified
  Helmholtz, whole far field or one of the four parts S/N/W/E (Eq. ksplitting2).
* ``method``   -- the paper's plain O(r(N_S+N_T)) method: direct application
  of the low-rank factorizations L D R for the south/north/west/east parts
  (Theorems south_thm, west_thm, south_thm_lap, west_thm_lap, south_thm_s,
  west_thm_s, south_thm_ms, west_thm_ms; Sec. 6 direct application), with this oracle's own
  (deliberately over-resolved) quadrature for the west/east integrals.
* ``nufft``    -- direct-sum definitions of the type-1/type-2 NUFFT sums
  (Sec. 2.3) and of Gauss-Legendre barycentric interpolation (Sec. 2.4),
  used to check the intermediate products of the NUFFT path.

Output conventions shared by every function here:
  scalar kernels ("laplace", "modhelm"): pot[nrhs, nt], grad[nrhs, 2, nt]
  "stokes", "mstokes": vel[nrhs, 2, nt] (forces f[nrhs, 2, ns])
Laplace and Stokes results are defined up to an additive constant per rhs
(per velocity component for Stokes); compare them modulo the best-fit
constant (``oracle.metrics``).
"""
