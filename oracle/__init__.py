"""FP64 CPU oracle for distillation low-mode averaging (arXiv:2201.09729).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the smoke check and the CPU-baseline leg of the benchmark may
call it.  It shares no code with the CUDA library; both consume the arrays
written by the ``synth`` input generator.

Every function is a plain, slow statement of the definition it follows, in
complex128, vectorised over lattice sites with numpy (no blocking, no fusion,
no even-odd tricks beyond what the even-odd decomposition itself states).
Library routines used as single steps: numpy matrix inverse / eigh, scipy
sparse LU (the dense-LU cross-check) and ARPACK (Lanczos) for Laplacian modes
on timeslices too large for a dense eigh.

Modules
  gamma      Dirac matrices (chiral basis) and sigma_{mu nu}.
  lattice    site / parity / even-odd / neighbour index tables.
  dirac      O(a)-improved Wilson-clover operator, even-odd blocks, Schur
             complement, sparse matrix form.
  solve      CG on the normal equations of the even-odd system (CGNE).
  laplacian  the spatial covariant Laplacian of Eq. 1 and its low modes.
  dlma       distillation sources, projector, perambulator and the
             C_rest / C_mixed / C_dist contractions of Eqs. 2-4.
  dilution   colour x even-odd diluted wall sources with spin-explicit
             one-end insertion (Sec. 3) and the trace form they estimate.

Parity status: every function is pinned by a test against a closed form, an
invariant, brute force or a library routine, except the paper-level physics
(C_dist / C ratios), which needs the CLS ensembles: parity unpinned there.
"""
