"""CPU FP64 oracle for the regularized TE domain-integral-equation solver.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import anything from
this package.  The CUDA library never calls it, and it shares no code, table or
constant generator with the CUDA library; the only module both sides use is
`paper_1104_4263_gb300.workloads`, which draws seeded inputs and holds none of
the method's arithmetic.

Contents (each function cites the passage of Zouros & Budko, "Transverse
electric scattering on inhomogeneous objects: spectrum of integral operator and
preconditioning", that it follows):

  green      -- matrix elements of the discretised TE operator, Section 4,
                Eqs. (4.3)-(4.5), with the Green's function of Eq. (2.14).
  dense      -- dense 2N x 2N matrices A = I - G X and A_R = A(chi'), Eq. (3.18)
                and Section 5; incident plane wave (Section 4, end).
  fftmv      -- the same product through a zero-padded 2-D FFT (scipy.fft); the
                CPU throughput baseline for grids too large for the dense matrix.
  rows       -- exact O(N) sums for selected output rows on large grids.
  gmres      -- restarted GMRES(m) with right preconditioning (Section 4/5), and
                flexible GMRES (Saad 1993) for a step-dependent or nonlinear right
                preconditioner such as a learned one.
  deflation  -- the deflating preconditioner of Eqs. (4.12)-(4.13) built from a
                dense eigendecomposition; the deflation radius of Section 5.
  fno        -- Fourier neural operator (Li et al., ICLR 2021), forward and a
                hand-derived backward pass: the reference for the learned
                preconditioner of flexible GMRES.
  cylinder   -- closed-form series for TE scattering by a homogeneous circular
                cylinder (textbook separation of variables in the Maxwell system
                of Eq. (2.1)); a pin for the discretisation.
  tm         -- the scalar TM operator of Section 2 and its cylinder series.
  te_mag     -- the TE system with magnetic contrast, unknowns (E1, E2, H3): the
                couplings of Section 3's compact kernels, the regulariser
                A(chi'_e, chi_m), and the magneto-dielectric cylinder series.

Everything is complex128 / float64.  Parity status: every function here is pinned
by `tests/test_oracle_*.py` against closed forms, invariants or brute force; none
is "parity unpinned".
"""
