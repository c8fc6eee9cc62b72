"""FP64 CPU oracle for the matrix-free resolvent time march.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs call it.  It shares no code with the CUDA library; the
only module both sides use is ``workloads`` (seeded inputs, no arithmetic of
the method).

Layout of the oracle, each module following the paper's statement:
  frequencies  commensurate frequency grid, window length T = 2 pi / dw
               (Sec. 2.3, Delta omega = 2 pi / T)
  operators    explicit sparse system matrices A of the workloads
               (Sec. 2.1 Eq. (system); Sec. 3 Eq. (GL_timeDomain) for the GL family)
  march        RK4 time march of the direct and adjoint systems with forcing
               synthesised from Fourier coefficients and a DFT of the response
               (Sec. 2.1 Eqs. (system)-(adsystemFreqDomain); TRM Sec. 2.2; SSRM Sec. 2.3 Eq. (forceFseries))
  decay        unforced decay run of a seeded random state that sets the SSRM
               transient length (Sec. 2.3); SplitMix64 counter-based initial state
  resolvent    closed forms: continuous R(w) = (i w I - A)^{-1} (Sec. 2.1) and
               the exact resolvent of the RK4-discretised system
  rsvd         power iteration with the gain estimate of App. A Eq. (tildeSig) and
               the block (randomized-SVD) form used for the gains and modes
  weighted     weighted (B, C, W) resolvent and its SVD (Sec. 2.1)
  arnoldi      Arnoldi / Krylov suboptimal gains on the steady-state method (App. A)
  series       the transient-response method in time-series form (Sec. 2.2):
               series-driven runs, snapshot interpolation (App. C), FIR
               flattening (App. B), Fourier transforms at any frequency and the
               TRM power iteration

Parity status: every function is pinned by the not-gpu tests in
``tests/test_oracle_*.py`` (closed forms, convergence orders, identities,
special cases); none is "parity unpinned".
"""
