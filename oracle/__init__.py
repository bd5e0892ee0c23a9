"""CPU FP64 oracle of the otVMC method (arxiv 2506.23928), written from the paper.

This package is TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
CPU-baseline / reference arm may import it; the CUDA library never does, and the two
share no code.  Plain numpy in FP64 / complex128, one function per definition of the
paper, each citing the equation or section it follows:

  philox        counter-based draws (Philox4x32-10 from its published definition)
  model         Eq. 10 Hamiltonian with signed couplings, decay and dephasing jump operators
  lindblad      exact density matrix, Eq. 1 (RK4; dense Liouvillian for expm checks)
  sse           exact-state trajectories of Eq. 2 (Ito) and Eq. 4-5 (Stratonovich, App. C)
  fossfeig      closed form of App. D (h = 0, periodic chain)
  ansatz        Jastrow (Eq. 12), its tied variants LJPHd / LJH, RBM (Eq. 11): log psi, O_k, flip ratios
  tvmc          local estimators, S / F / N^n / D (after Eq. 8), shift and SNR solves,
                Metropolis sampling, the predictor-corrector step of App. C
  observables   M, C and Wineland xi^2 (LITF paragraph) from local estimators
  trajectories  MC otVMC, enumeration otVMC and exact-SSE ensembles (Eq. 3)

Parity unpinned: the SNR filter shape of tvmc.solve_snr (the paper cites the scheme but
does not print it); only its vanishing-threshold limit is pinned.
"""
