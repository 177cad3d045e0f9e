"""CPU oracle for the overlapping source-transfer DDM (arXiv 2509.20801).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The GPU
library never calls it and shares no code with it; the two meet only in the
seeded input generators of ``workloads``.

Everything here is plain, slow and complex128:

* ``fdfd``   -- SC-PML profile (Eqs. 10-13), 5-point stretched stencil
                (Eq. 2 with Eq. 9), global sparse assembly (Eq. 4) and the
                plain definition of the solution, a sparse direct solve.
* ``stddm``  -- strip partition with overlapping PML (Sec. 2.3, Fig. 3),
                local operators, the one-sweep preconditioner M^-1, the
                paper's Algorithm 1 with explicit transfer operators
                (Eqs. 14-21) and the equivalent Richardson form, and the
                symmetric multiplicative order of the same local solves.
* ``nn``     -- the learned-guess network (forward, hand-written backward,
                Adam), its image normalisation and the scaled start.
* ``krylov`` -- textbook restarted right-preconditioned GMRES(m) and
                flexible GMRES(m) with modified Gram-Schmidt and Givens
                rotations.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):

* PML profile: pinned by the 1-D closed-form reflection tests and the
  printed-value check of sigma_max; the polynomial sample positions
  themselves follow one reading of Eqs. 11-12 shared with the GPU path.
* Stencil / assembly: pinned by the exact 1-D discrete solution, the free-space
  Hankel function (2nd-order convergence), the Mie series and reciprocity.
* Local solves, M^-1, Algorithm 1: pinned by the transfer identity, by the
  Algorithm-1 == Richardson identity and by nsub = 1 reducing to A^-1.
* Multiplicative order: pinned by the product form of its error
  propagator, I - M^-1 A = (I - P_0)..(I - P_{n-1})..(I - P_0) with
  P_k = E_k A_k^-1 R_k^I A built column by column, and by one strip giving
  A^-1.
* Network: pinned by central finite differences, an independent autograd
  restatement, scipy's correlate2d and the closed-form first Adam step.
* GMRES / FGMRES: pinned by one-iteration convergence when M = A, finite
  termination on small systems, residual monotonicity and the bound by the
  Richardson residual.
"""
