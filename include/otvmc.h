/*
 * otvmc.h -- C ABI of a GB300 (sm_103a) implementation of the data-parallel hot path of
 * open time-dependent variational Monte Carlo over quantum trajectories (otVMC):
 * Apostoli, D'Alberto, Genoni, Bertaina, Galli, "Unraveling Open Quantum Dynamics with
 * Time-Dependent Variational Monte Carlo", arXiv:2506.23928.
 *
 * Each trajectory carries complex variational parameters theta (P entries) of a
 * wavefunction psi_theta over N spins-1/2.  One trajectory step (App. C) runs two
 * *evaluations*; each evaluation samples configurations from |psi_theta|^2 (Metropolis),
 * builds the local operators O_k, the local effective energy E_eff and local noises B^n
 * (definitions after Eq. 8, effective Hamiltonian Eq. 5), the quantum geometric tensor S
 * and the vector D = -i F dt + sum_n N^n dW_n (otVMC procedure paragraph), and solves
 * (S + eps I) delta = D; the predictor-corrector scheme then moves theta.  Observables are
 * the magnetisation and spin covariance (LITF paragraph), averaged over trajectories (Eq. 3).
 *
 * Conventions common to every entry point
 * ---------------------------------------
 * - Pointers named *_d are device pointers (any allocator; 16-byte aligned); pointers
 *   named *_h are host pointers.  The caller owns every buffer it passes.  Handles
 *   (otvmc_model, otvmc_ansatz) own only small device copies of model constants.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Stage
 *   entry points enqueue work on it and return without synchronising; errors found on
 *   the device are written to the status word at the start of the workspace and are
 *   read (and cleared) by otvmc_check.  Entry points that synchronise say so.
 * - `work_d` / `work_bytes`: caller-provided device scratch, at least the size returned
 *   by otvmc_workspace_bytes for the same (ansatz, ntraj, ns, precision).  Its first 256
 *   bytes hold the status word and per-call diagnostics; the rest is carved per call.
 *   Contents do not carry over between calls unless stated.  Calls sharing a workspace
 *   must be ordered on one stream.
 * - Batches: every stage call processes `ntraj` trajectories with `ns` samples each;
 *   trajectory t of the call has global id traj0 + t (the id keys the counter-based
 *   random streams, so results do not depend on how trajectories are batched).
 * - Complex numbers are interleaved (re, im) doubles (double2); theta is [ntraj][P].
 * - Spin configurations: [ntraj][ns][W] uint64 with W = ceil(N/64); bit j % 64 of word
 *   j / 64 is set iff sigma_j = +1 (spin up, eigenvalue +1 of sigma^z_j).  Unused high
 *   bits are zero.  Sample s of a trajectory is the state of Markov chain s.
 * - Errors are returned as otvmc_status and never abort; otvmc_last_error() gives a
 *   thread-local message for the last failing call.  Device code never traps.
 *
 * Random draws (Philox4x32-10, Salmon et al. SC'11; key = (seed mod 2^32, seed >> 32)):
 *   Wiener increments : counter (n/4, step, traj, 2<<28); 4 normals per counter by two
 *                       Box-Muller pairs over words (0,1) and (2,3); dW = sqrt(dt) z.
 *   Metropolis        : counter (p/2, chain, traj, (1<<28) | (eval & 0x0FFFFFFF)); proposal
 *                       p uses words (2(p%2), 2(p%2)+1): site = (w * N) >> 32,
 *                       u = (w' + 0.5) 2^-32, accept iff u < |psi(x')/psi(x)|^2 (FP64).
 *   Initial chains    : counter (q, chain, traj, 3<<28); words 2q, 2q+1 = (w0 | w1<<32),
 *                       (w2 | w3<<32).
 *   eval = 2*step + stage (stage 0 predictor, 1 corrector; 2*n_steps for a final pass).
 */
#ifndef OTVMC_H
#define OTVMC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OTVMC_API __attribute__((visibility("default")))
#else
#define OTVMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum otvmc_status {
    OTVMC_OK = 0,
    OTVMC_ERR_INVALID = 1,     /* bad argument, size or handle */
    OTVMC_ERR_OOM = 2,         /* a handle's small device allocation failed */
    OTVMC_ERR_CUDA = 3,        /* a CUDA runtime call failed (message in otvmc_last_error) */
    OTVMC_ERR_NOT_PD = 4,      /* S + eps I not positive definite after the shift retries */
    OTVMC_ERR_TIMEOUT = 5,     /* a bounded device wait ran out (kernel returned early) */
    OTVMC_ERR_NONFINITE = 6,   /* NaN / Inf in a parameter update */
    OTVMC_ERR_RANGE = 7,       /* a fixed-point field or sample count exceeded its range */
    OTVMC_ERR_UNSUPPORTED = 8, /* combination not built (e.g. RBM with this precision) */
    OTVMC_ERR_WORKSPACE = 9    /* work_bytes smaller than otvmc_workspace_bytes */
} otvmc_status;

enum { OTVMC_JASTROW = 0, OTVMC_RBM = 1, OTVMC_LJ = 2 };
enum { OTVMC_PREC_FP64 = 0, OTVMC_PREC_MIXED = 1 };
enum { OTVMC_REG_SHIFT = 0, OTVMC_REG_SNR = 1 };
enum { OTVMC_HEUN = 0, OTVMC_MIDPOINT = 1 };

#define OTVMC_MAX_SITES 256
#define OTVMC_MOMENTS 9 /* m_x m_y m_z q_xx q_yy q_zz q_xy q_xz q_yz per trajectory */

typedef struct otvmc_model otvmc_model;
typedef struct otvmc_ansatz otvmc_ansatz;

/* ------------------------------------------------------------------- model (Eq. 10, LITF)
 * H = sum_{i<j} J_ij sz_i sz_j + h sum_i sx_i with explicit signed couplings (the
 * paper's -(J/K) sum sz sz / r^alpha - h sum sx is J_ij = -J/(K r^alpha), h -> -h).
 * Jump operators: decay L = sqrt(kappa_i) s^-_i and dephasing L = sqrt(gamma_i) sz_i,
 * operators with zero rate omitted; order: decays in site order, then dephasings. */
typedef struct otvmc_model_desc {
    int n;               /* number of spins, 1 <= n <= OTVMC_MAX_SITES */
    const double* J_h;   /* n*n row-major, symmetric, zero diagonal */
    double h;            /* transverse field */
    const double* kappa_h; /* n decay rates >= 0, or NULL for none */
    const double* gamma_h; /* n dephasing rates >= 0, or NULL for none */
} otvmc_model_desc;

/* Couplings J_ij = J / r_ij^alpha of an open (pbc = 0) or periodic (pbc = 1, nearest
 * image) chain (dim = 1, extent[0] = N) or square lattice (dim = 2, extent = {Lx, Ly},
 * row-major sites); kac = 1 divides by K(alpha) = sum_{i<j} r_ij^-alpha / (N - 1)
 * (LITF paragraph).  Host only; J_out_h has N*N entries. */
OTVMC_API otvmc_status otvmc_lattice_couplings(int dim, const int* extent, double J, double alpha,
                                     int kac, int pbc, double* J_out_h);

/* Copies the description; allocates ~N*N*8 bytes of device memory for J. */
OTVMC_API otvmc_status otvmc_model_create(const otvmc_model_desc* desc, otvmc_model** out);
OTVMC_API void otvmc_model_destroy(otvmc_model* model);
/* Number of jump operators N_L (length of each trajectory's dW and <L+L^+> rows). */
OTVMC_API int otvmc_model_nops(const otvmc_model* model);

/* ---------------------------------------------------------- ansatz (Eq. 11 RBM, Eq. 12 LJ)
 * OTVMC_JASTROW: log psi = sum a_i s_i + sum_{j<k} eta_jk s_j s_k, P = N(N+1)/2,
 *   theta = [a_0..a_{N-1}, eta_jk for j<k row-major].  n_hidden ignored.
 * OTVMC_RBM: log psi = sum a_i s_i + sum_m log 2cosh(b_m + sum_i W_im s_i),
 *   P = N + M + N M, theta = [a (N), b (M), W (N x M row-major)], M = n_hidden in
 *   [1, 4096].  Sampling uses an FP32 warp-per-chain kernel whose decisions equal the FP64
 *   ones (M <= 256; an FP64 kernel beyond); its ratios are products of flip factors
 *   cosh(g - 2 s W) / cosh g = 1 + (cosh 2W - 1) - s tanh(g) sinh 2W, tabulated per call in
 *   the workspace.  MIXED (M <= 256): the same flip factors for the estimators' ratios, FP32
 *   log 2cosh in the observables; in run_trajectories, S (P <= ns) or T (P > ns) from
 *   split-BF16 tensor-core products accumulated in FP32 and the tensor-core Cholesky, whose
 *   solution is corrected against the exact S or T (residuals from integer fixed-point sums,
 *   FP64 right-hand side): delta agrees with the FP64 oracle to about 1e-6 relative on the
 *   factorised T path at eps 1e-3; on the T path T is by default formed without O
 *   (otvmc_ansatz_set_rbm_t_build);
 *   build_S_F / solve_step of an RBM run in FP64 for either precision.
 * The ansatz keeps a pointer to the model, which must outlive it. */
OTVMC_API otvmc_status otvmc_ansatz_create(const otvmc_model* model, int kind, int n_hidden,
                                 otvmc_ansatz** out);
OTVMC_API void otvmc_ansatz_destroy(otvmc_ansatz* ansatz);
OTVMC_API int64_t otvmc_ansatz_nparams(const otvmc_ansatz* ansatz);

/* Partially inhomogeneous long-range Jastrow LJPHd (Eq. 12 and the paragraph after it): the
 * two-body parameters eta_jk are free for every pair at distance D <= d and shared by all
 * pairs at the same distance D > d; the biases a_i stay free.  D = |j - k| (pbc = 0) or the
 * nearest-image distance min(|j - k|, N - |j - k|) (pbc = 1, for a periodic chain).  d = 0 is
 * the homogeneous LJH; d at least the largest distance gives the full Jastrow (LJNH) with the
 * OTVMC_JASTROW layout.  theta = [a (N), one eta per group]: first the pairs at distance <= d
 * one by one in row-major order (j < k), then one parameter per distance D > d in increasing
 * D.  P = N + number of groups: 2N - 1 - d + N d - d(d+1)/2 for an open chain; N + N d +
 * floor(N/2) - d for a periodic one with d < N/2 (the paper prints 2N - 1 - d + N d / 2, which
 * agrees with the open-chain count at d = 0 and d = N - 1 only).
 * Kind OTVMC_LJ.  Sampling, local estimators and observables run the Jastrow kernels on the
 * expanded pair parameters (held in the workspace); build_S_F gives S in FP64 (S_d required,
 * from exact integer counts of the tied log-derivatives O_g = sum over the group of s_j s_k)
 * and D, obar folded from the exact pair sums, for either precision; solve_step then factors
 * S in FP64 (G_d unused); otvmc_solve_snr takes it as well.  N <= 200. */
OTVMC_API otvmc_status otvmc_ansatz_create_lj(const otvmc_model* model, int d, int pbc, otvmc_ansatz** out);

/* How the MIXED path of run_trajectories forms T = O_c O_c^+ / ns of an RBM on the T path
 * (P > ns; the push-through solve of the otVMC procedure).
 * OTVMC_RBM_T_FACTORED (default): from the exact factorisation of the RBM's log-derivatives,
 *   sum_k O_k(x) O_k(x')^* = A + B + A B with A = sum_i s_i s_i' (an integer) and
 *   B = sum_m tanh gamma_m(x) tanh gamma_m(x')^* (FP32), centred with obar (FP64 column sums);
 *   O(ns^2 (N + M)) work and no O in memory.  delta = O_c^+ z / ns likewise from N x (M + 1)
 *   column sums.  Same delta as the materialised form up to rounding.
 * OTVMC_RBM_T_MATERIALISED: O_c materialised (real embedding, three BF16 pieces) and T from
 *   the split-BF16 tensor-core product (O(ns^2 N M) work, 24 ns P bytes per trajectory).
 * Returns OTVMC_ERR_INVALID for another mode or a Jastrow ansatz.  Not synchronised with
 * calls in flight on the same ansatz: set it before launching them. */
enum { OTVMC_RBM_T_FACTORED = 0, OTVMC_RBM_T_MATERIALISED = 1 };
OTVMC_API otvmc_status otvmc_ansatz_set_rbm_t_build(otvmc_ansatz* ansatz, int mode);

/* Bytes of work_d needed by any stage entry point below for this batch shape. */
OTVMC_API size_t otvmc_workspace_bytes(const otvmc_ansatz* ansatz, int ntraj, int ns, int precision);

/* Synchronises `stream`, returns the first device-side error recorded in work_d since
 * the last check (OTVMC_OK if none) and clears it. */
OTVMC_API otvmc_status otvmc_check(void* work_d, void* stream);

/* ------------------------------------------------------------------ A1: Wiener increments
 * dW_d[t][n] = sqrt(dt) z, z ~ N(0,1) from the counter (n/4, step, traj0+t, 2<<28)
 * (Eq. 2: independent increments of variance dt, one per jump operator; App. C uses the
 * same draw in predictor and corrector).  dW_d: [ntraj][N_L] double. */
OTVMC_API otvmc_status otvmc_draw_noise(const otvmc_model* model, int ntraj, int traj0, uint64_t seed,
                              int64_t step, double dt, double* dW_d, void* stream);

/* I.i.d. uniform chain states (exact samples of |psi|^2 at theta = 0, the coherent state
 * along +x).  spins_d: [ntraj][ns][W] uint64. */
OTVMC_API otvmc_status otvmc_init_chains(const otvmc_ansatz* ansatz, int ntraj, int traj0, int ns,
                               uint64_t seed, uint64_t* spins_d, void* stream);

/* ------------------------------------------------------------------- A2: Metropolis
 * Continues every chain for n_sweep * N single-spin-flip proposals targeting
 * |psi_theta(x)|^2 (otVMC procedure paragraph), in place on spins_d.  The acceptance
 * test u < exp(2 Re log r) is decided as in FP64 (FP32 fast path with a guard band, FP64
 * near the threshold).  accepted_d (optional, may be NULL): [ntraj] uint64 counts, added to. */
OTVMC_API otvmc_status otvmc_sample(const otvmc_ansatz* ansatz, const double* theta_d, int ntraj,
                          int traj0, int ns, int n_sweep, uint64_t seed, int64_t eval_index,
                          uint64_t* spins_d, uint64_t* accepted_d, void* work_d,
                          size_t work_bytes, void* stream);

/* ------------------------------------------------------------ A3 + A5: local estimators
 * For every sample x: flip ratios r_j(x), E_H(x) = sum_{i<j} J_ij s_i s_j + h sum_j r_j,
 * <L_n + L_n^+> (real part of the sample mean of its local estimator; per trajectory),
 * E_eff(x) = E_H - i/2 sum_n [(L^+L)_loc - 2 <L+L^+> B^n(x) + (L^2)_loc]  (Eq. 5, the
 * c-number terms dropped: they cancel in F and N^n), and
 * v(x) = -i dt E_eff(x) + sum_n dW_n B^n(x), so that D = Cov(O^*, v).
 * Outputs (any may be NULL except v_d): Eeff_d [ntraj][ns] double2, v_d [ntraj][ns]
 * double2, lpl_d [ntraj][N_L] double.  FP64: the fields are exact fixed-point sums and the
 * transcendentals FP64.  MIXED: the imaginary field (the ratio's phase) stays exact in fixed
 * point, the real and coupling fields carry FP32-level rounding (for the Jastrow ansatz with
 * 32 <= N <= 128 they come from a tensor-core product of sigma with FP16 pieces of the couplings
 * and exact integer digits of the phase), the transcendentals are FP32. */
OTVMC_API otvmc_status otvmc_local_estimators(const otvmc_ansatz* ansatz, const double* theta_d,
                                    const uint64_t* spins_d, int ntraj, int ns,
                                    const double* dW_d, double dt, int precision,
                                    double* Eeff_d, double* v_d, double* lpl_d,
                                    void* work_d, size_t work_bytes, void* stream);

/* Allocation-free variant of otvmc_local_estimators (the paper has no counterpart: this is
 * an interface for callers that cannot give the library scratch memory -- code whose device
 * memory belongs to a memory manager with a hard budget it may not allocate outside of, or a
 * latency-sensitive loop where an allocation, which can synchronise the device, is not
 * acceptable).  Jastrow ansatz only (an RBM ansatz returns OTVMC_ERR_UNSUPPORTED).  Same
 * inputs, outputs and results (bit for bit) as otvmc_local_estimators, but no work_d: the
 * scratch is a fixed 32 MiB array inside this library's device memory, held by every GPU
 * that loads the library until the process exits.  Nothing is allocated by this call.
 *   - Batches whose scratch would exceed 32 MiB are rejected with OTVMC_ERR_WORKSPACE before
 *     anything is launched.  The scratch of a batch is about
 *     ntraj * (16 ns (N + q) + 16 N^2 + 40 N ceil(ns / b) + 16384 q ceil(N / 64)) bytes,
 *     b = 8 floor(256 / N32), N32 = N rounded up to a multiple of 32, q = ceil(N / 16) for
 *     N <= 128, else q = 1 and no last term (flip ratios, E_H in q partials, the fixed-point
 *     parameter tables, the per-block site sums, the operand images of the tensor-core
 *     estimators): at N = 64 and 4096 samples, 6 trajectories fit.
 *   - status_d (optional, caller-cleared): device int[2].  Device-side errors are recorded
 *     there as in the workspace status word of the other entry points: word 0 the first error
 *     code (e.g. OTVMC_ERR_RANGE when a parameter field leaves the fixed-point range), word 1
 *     its detail (the trajectory index).  Both words may be written.
 *   - All calls share the one array: calls that overlap on the GPU (different streams or
 *     threads without ordering) race and give wrong results; order them on one stream.
 *     The array keeps the last call's contents; nothing in it needs to start at zero.
 *   - The first call on each device looks up the array's device address (once per device,
 *     with that device current); make that first call before any stream capture. */
OTVMC_API otvmc_status otvmc_local_estimators_noalloc(const otvmc_ansatz* ansatz, const double* theta_d,
                                                      const uint64_t* spins_d, int ntraj, int ns,
                                                      const double* dW_d, double dt, int precision,
                                                      double* Eeff_d, double* v_d, double* lpl_d,
                                                      int* status_d, void* stream);

/* --------------------------------------------------------------- A4 + A6: S and D
 * S = <O^* O> - <O^*><O>, D = <O^* v> - <O^*><v> over the ns samples (definitions after
 * Eq. 8; D = -i F dt + sum_n N^n dW_n by linearity).  Jastrow: O is real (+-1), S real
 * symmetric.
 *   FP64:  S_d [ntraj][P][P] double (full symmetric) from FP64 centred O.
 *   MIXED: G_d [ntraj][P][P] float, the uncentred Gram counts sum_x O_xi O_xj for j >= i
 *          (row-major upper triangle; lower part unspecified), from an FP8 (E4M3) tcgen05
 *          GEMM (exact: O = +-1, FP32 accumulation exact below 2^24 samples); obar_d [ntraj][P]
 *          double column means; S = G / ns - obar obar^T exactly.  S_d, if not NULL, is
 *          also filled (full FP64).
 * RBM (FP64 only; theta_d required): O is complex (O_a = s, O_b = tanh gamma, O_W = s tanh
 *          gamma), S_d is [ntraj][P][P] double2 (complex Hermitian, full), obar_d (optional)
 *          [ntraj][P] double2; built as R^T R / ns with R = [[Re O_c, -Im O_c], [Im O_c, Re O_c]]
 *          (the real embedding of S), G_d unused.
 * D_d: [ntraj][P] double2.  Inputs v_d from otvmc_local_estimators.  Jastrow: D and obar are
 *          exact integer sums of O against v quantised to 64-bit fixed point (one scale per
 *          trajectory), converted once to FP64; on the mixed path with ns <= 2^17 the sums come
 *          out of the same tensor-core pass as G (the digits of the quantised v as extra
 *          operand rows), with identical results. */
OTVMC_API otvmc_status otvmc_build_S_F(const otvmc_ansatz* ansatz, const double* theta_d,
                             const uint64_t* spins_d, const double* v_d, int ntraj, int ns,
                             int precision, double* S_d, float* G_d, double* obar_d,
                             double* D_d, void* work_d, size_t work_bytes, void* stream);

/* ----------------------------------------------------------------- A7: regularised solve
 * delta = (S + eps I)^{-1} D by Cholesky (diagonal shift; the SNR filter of the otVMC
 * procedure paragraph needs the samples and is otvmc_solve_snr).  If S + eps I is
 * not positive definite in the working precision (a pivot not above zero, or a solution that
 * is not finite) the shift is raised (x100, up to 3 times) and OTVMC_ERR_NOT_PD is
 * recorded only if all attempts fail (delta = 0 then).
 *   FP64:  S_d (full FP64), FP64 Cholesky.
 *   MIXED: G_d + obar_d; tensor-core Cholesky of (S + eps I) / 2^k (2^k the power of two
 *          that bounds the factor's entries by 1; the factor held as two FP16 pieces, 22
 *          significant bits, each 128 x 128 tile product taken as three FP16 tcgen05 products
 *          accumulated in FP32), then two steps of iterative refinement with the residual
 *          D - (S + eps I) x in FP64 from the exact G.  A trajectory whose diagonal blocks
 *          would leave FP16's range, or whose solution is not finite, is solved by an FP32
 *          fallback factorisation (with the shift retries above) instead.
 *   RBM (FP64 only): S_d the complex [ntraj][P][P] double2 of otvmc_build_S_F; the real
 *          embedding [[Re S, -Im S], [Im S, Re S]] + eps I (size 2P) is factored in FP64.
 * shift_used_d (optional): [ntraj] double, the shift that succeeded.
 * delta_d: [ntraj][P] double2. */
OTVMC_API otvmc_status otvmc_solve_step(const otvmc_ansatz* ansatz, int ntraj, int ns, int precision,
                              int reg, double eps, double snr_thresh, const double* S_d,
                              const float* G_d, const double* obar_d, const double* D_d,
                              double* delta_d, double* shift_used_d, void* work_d,
                              size_t work_bytes, void* stream);

/* SNR-filtered pseudo-inverse in the eigenbasis of S (otVMC procedure paragraph; the filter of
 * the signal-to-noise regularisation it cites, whose shape the paper does not print -- read
 * here as below).  S = V diag(lambda) V^T, rho = V^T D, and per sample
 * Q_k(x) = (V^T O_c(x))_k v_c(x) (O_c, v_c centred by their sample means), whose mean is rho_k:
 *   SNR_k = |rho_k| / sqrt(Var_x Q_k / ns),
 *   f_k = 1 / (1 + (snr_thresh / SNR_k)^6) * 1 / (1 + (eps_svd lambda_max / lambda_k)^6),
 *   delta = V diag(f_k / lambda_k) rho, eigenvalues lambda_k <= 0 dropped.
 * Jastrow and tied Jastrow ansaetze, one CTA per trajectory, FP64 throughout.  P <= 96: a
 * cyclic Jacobi eigen-decomposition in shared memory.  Larger P (up to what the shared memory
 * of one CTA holds for the tridiagonal and a chunk of samples, about 3000): Householder
 * tridiagonalisation of a copy of S in the workspace, the eigenvectors formed explicitly and
 * refined by the implicit QL iteration (shift from the leading 2 x 2 block), then one pass over
 * the samples; this costs O(P^3) FP64 work per trajectory for the decomposition and
 * O(ns P^2) for the pass.  Inputs: S_d [ntraj][P][P] full FP64 S (otvmc_build_S_F), obar_d
 * [ntraj][P], spins_d [ntraj][ns][W], v_d [ntraj][ns] double2 (otvmc_local_estimators), D_d
 * [ntraj][P] double2.  work_bytes >= otvmc_snr_workspace_bytes(ansatz, ntraj) (256 bytes of
 * status for P <= 96, plus 2 P^2 doubles per trajectory beyond).  Outputs: delta_d [ntraj][P]
 * double2; lambda_d (optional) [ntraj][P] eigenvalues, unordered.  A decomposition that has
 * not converged (40 Jacobi sweeps, or 60 QL iterations for one eigenvalue) records
 * OTVMC_ERR_NONFINITE in the status word (delta = 0 for the QL case). */
OTVMC_API size_t otvmc_snr_workspace_bytes(const otvmc_ansatz* ansatz, int ntraj);
OTVMC_API otvmc_status otvmc_solve_snr(const otvmc_ansatz* ansatz, int ntraj, int ns, const double* S_d,
                                       const double* obar_d, const uint64_t* spins_d, const double* v_d,
                                       const double* D_d, double snr_thresh, double eps_svd, double* delta_d,
                                       double* lambda_d, void* work_d, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------ A8: SDE combination
 * App. C on theta (all [ntraj][P] double2):
 *   stage 0: out = theta + c delta0 with c = 1 (Heun: X-bar) or 1/2 (midpoint:
 *            (X + X-bar)/2), the point of the corrector evaluation;
 *   stage 1: out = theta + (delta0 + delta1)/2 (Heun) or theta + delta1 (midpoint).
 * Non-finite results leave theta unchanged for that trajectory and record
 * OTVMC_ERR_NONFINITE; failed_d (optional) [ntraj] int is set to 1 for it. */
OTVMC_API otvmc_status otvmc_sde_combine(int ntraj, int64_t P, int scheme, int stage,
                               const double* theta_d, const double* delta0_d,
                               const double* delta1_d, double* out_d, int* failed_d,
                               void* work_d, size_t work_bytes, void* stream);

/* --------------------------------------------------------------------- A9: observables
 * Per-trajectory moments from the current samples (local estimators, LITF paragraph):
 * m_a = (1/N) sum_j <s^a_j>, q_ab = (1/N^2) sum_{jk} <(s^a_j s^b_k + s^b_k s^a_j)/2>.
 * moments_d: [ntraj][OTVMC_MOMENTS] double in the order m_x m_y m_z q_xx q_yy q_zz q_xy
 * q_xz q_yz.  MIXED: FP32 ratios and sums (for the Jastrow ansatz with 32 <= N <= 64 the pair
 * sums as tensor-core products of FP16 pieces), agreeing with FP64 to about 1e-5 relative. */
OTVMC_API otvmc_status otvmc_observables(const otvmc_ansatz* ansatz, const double* theta_d,
                               const uint64_t* spins_d, int ntraj, int ns, int precision,
                               double* moments_d, void* work_d, size_t work_bytes,
                               void* stream);

/* Host: trajectory average (Eq. 3) of per-trajectory moments [ntraj][9] -> M[3],
 * C[3][3] = <q> - M M^T, xi2 = N lambda_min(C on the plane perpendicular to M) / |M|^2,
 * dM[3] = standard error of M.  Any output may be NULL. */
OTVMC_API otvmc_status otvmc_ensemble(const double* moments_h, int ntraj, int n_sites, double* M_h,
                            double* C_h, double* xi2_h, double* dM_h);

/* ------------------------------------------------------------- whole trajectories (A1-A9)
 * Runs n_steps trajectory steps for ntraj trajectories, all on the device, launching
 * every stage above batched over the trajectories.  RBM (FP64): when P > ns the solve takes
 * the push-through form delta = O_c^+ (T + eps I)^-1 v_c / ns with T = O_c O_c^+ / ns (the
 * same delta as (S + eps I)^-1 D), factoring a system of size 2 ns instead of 2 P.  theta_d [ntraj][P] and spins_d
 * [ntraj][ns][W] are the state (in/out; start chains with otvmc_init_chains).
 * moments_d (may be NULL when measure_every = 0): [n_meas][ntraj][9] with one row per
 * measured step (steps i with i % measure_every == 0, from the predictor samples at
 * theta_i) plus, if measure_final, one row at the final time.  With OTVMC_REG_SNR the solve is
 * otvmc_solve_snr's filter; on the mixed path its pass over the samples (beyond P = 96) projects
 * in FP32 (the variances that set the filter to about 1e-6 relative).  Synchronises and returns
 * the device status at the end.  work_bytes >= otvmc_run_workspace_bytes(...). */
typedef struct otvmc_run_desc {
    int ntraj;
    int traj0;
    int ns;
    int n_steps;
    int64_t step0;       /* index of the first step (resume) */
    int n_sweep;         /* Metropolis sweeps per evaluation */
    double dt;
    int scheme;          /* OTVMC_HEUN or OTVMC_MIDPOINT */
    int precision;       /* OTVMC_PREC_FP64 or OTVMC_PREC_MIXED */
    int reg;             /* OTVMC_REG_SHIFT, or OTVMC_REG_SNR (Jastrow ansaetze, eps_svd = 1e-12) */
    double eps;          /* diagonal shift */
    double snr_thresh;
    uint64_t seed;
    int measure_every;   /* 0: never */
    int measure_final;   /* 1: add a row at the final time */
    int use_graph;       /* reserved, must be 0 (graph replay of a step is not built:
                            the step's counter-based draws change every step) */
} otvmc_run_desc;

OTVMC_API size_t otvmc_run_workspace_bytes(const otvmc_ansatz* ansatz, const otvmc_run_desc* desc);
OTVMC_API int otvmc_run_n_meas(const otvmc_run_desc* desc);
OTVMC_API otvmc_status otvmc_run_trajectories(const otvmc_ansatz* ansatz, const otvmc_run_desc* desc,
                                    double* theta_d, uint64_t* spins_d, double* moments_d,
                                    void* work_d, size_t work_bytes, void* stream);

/* Grouped run: ngroups (1 .. OTVMC_MAX_GROUPS) batches of trajectories of one ansatz, each with its
 * own descriptor (sample count, trajectory range, steps, precision may differ: e.g. one ensemble
 * spread over several N_s), run concurrently in one call, each group on its own stream forked
 * from `stream` and joined back into it.  Group g reads and writes theta_d[g], spins_d[g] and
 * moments_d[g] (moments_d itself may be NULL when no group measures) exactly as
 * otvmc_run_trajectories with descs[g] would: its results are bit-identical to that call.  The
 * group with the largest ns runs at the highest stream priority.  work_d holds each group's run
 * workspace in turn (otvmc_run_grouped_workspace_bytes, 0 for invalid arguments).  Synchronises;
 * returns the first error of any group. */
enum { OTVMC_MAX_GROUPS = 8 };
OTVMC_API size_t otvmc_run_grouped_workspace_bytes(const otvmc_ansatz* ansatz, const otvmc_run_desc* descs,
                                                   int ngroups);
OTVMC_API otvmc_status otvmc_run_trajectories_grouped(const otvmc_ansatz* ansatz, const otvmc_run_desc* descs,
                                                      int ngroups, double* const* theta_d,
                                                      uint64_t* const* spins_d, double* const* moments_d,
                                                      void* work_d, size_t work_bytes, void* stream);

/* Launch-shape autotuner.  A run's launches can be issued as 1, 2 or 4 sub-batches on forked
 * streams (each of at least 8 trajectories), and the mixed tensor-core solver's launches as 1, 2
 * or 4 trajectory groups on forked streams inside each; none of this changes any result.
 * otvmc_autotune_run times one step of every candidate shape for this batch (the fastest of three
 * repetitions, from copies of theta_d and spins_d, which are left untouched; with measurements
 * when desc measures),
 * records the fastest for the batch shape (ansatz kind and sizes, ns, ntraj, precision,
 * regulariser), and later runs of that shape in this process use it.  Without a record the
 * built-in shape applies (2 sub-batches for a Jastrow batch of 32 trajectories or more, else 1;
 * the solver's own group rule).  otvmc_run_workspace_bytes already covers every shape.
 * work_bytes >= otvmc_autotune_workspace_bytes (the run's workspace plus copies of the state).
 * Outputs (optional): the chosen sub-batch count, group count (0: the solver's rule) and the
 * step time in ms.  Synchronises.  otvmc_autotune_clear forgets every record. */
OTVMC_API size_t otvmc_autotune_workspace_bytes(const otvmc_ansatz* ansatz, const otvmc_run_desc* desc);
OTVMC_API otvmc_status otvmc_autotune_run(const otvmc_ansatz* ansatz, const otvmc_run_desc* desc,
                                          const double* theta_d, const uint64_t* spins_d, void* work_d,
                                          size_t work_bytes, void* stream, int* pipes_out, int* groups_out,
                                          double* ms_out);
OTVMC_API void otvmc_autotune_clear(void);

/* The linear stochastic Schroedinger equation (App. B) instead of the nonlinear one: the same
 * otVMC equations with E_eff replaced by E_eff^lin = <x|H - i/2 sum_n (L_n^+ L_n + L_n^2)|psi>/psi(x)
 * (so F^lin = F - i sum_n <L_n + L_n^+> N^n), and for every trajectory the normalisation Q of
 * its unnormalised state, d ln Q = 2 Im<E_eff^lin> dt + 2 sum_n Re<B^n> o dW_n (the
 * normalisation SDE, read in Stratonovich form for ln Q), integrated by the run's scheme
 * alongside theta.  lnQ_d [ntraj] (in/out, 0 for a normalised start) holds ln Q; lnQ_rows_d
 * (optional) [n_meas][ntraj] receives ln Q at each measured row.  Ensemble averages of the
 * linear SSE weight each trajectory's (normalised) moments by Q = exp(ln Q):
 * otvmc_ensemble_weighted.  Everything else as otvmc_run_trajectories.  Synchronises. */
OTVMC_API otvmc_status otvmc_run_trajectories_linear(const otvmc_ansatz* ansatz, const otvmc_run_desc* desc,
                                                     double* theta_d, uint64_t* spins_d, double* moments_d,
                                                     double* lnQ_d, double* lnQ_rows_d, void* work_d,
                                                     size_t work_bytes, void* stream);

/* Host: the trajectory average of the linear SSE (App. B, the weighted form of Eq. 3):
 * M = (1/N_T) sum_j w_j m_j and <q> likewise, with weights w_h[ntraj] = Q_j; then C, xi2 and dM
 * as otvmc_ensemble (dM the standard error of the weighted samples w_j m_j). */
OTVMC_API otvmc_status otvmc_ensemble_weighted(const double* moments_h, const double* w_h, int ntraj, int n_sites,
                                               double* M_h, double* C_h, double* xi2_h, double* dM_h);

/* Same with host buffers (pinned or pageable): copies theta_h / spins_h in, runs, copies
 * theta_h / spins_h / moments_h back; device copies live in work_d, which must hold
 * otvmc_run_host_workspace_bytes(...).  Synchronises. */
OTVMC_API size_t otvmc_run_host_workspace_bytes(const otvmc_ansatz* ansatz, const otvmc_run_desc* desc);
OTVMC_API otvmc_status otvmc_run_trajectories_host(const otvmc_ansatz* ansatz, const otvmc_run_desc* desc,
                                         double* theta_h, uint64_t* spins_h, double* moments_h,
                                         void* work_d, size_t work_bytes, void* stream);

/* ------------------------------------------------------------------ kernel timing
 * When enabled, every kernel launch of the library is bracketed by two CUDA events on
 * its own stream; otvmc_profile_read sums the elapsed times per kernel class.  Enabling
 * clears earlier records.  Not for use inside CUDA graph capture.
 * otvmc_profile_enable(OTVMC_PROFILE_ON) keeps the normal schedule, in which the Cholesky
 * solver's trajectory groups run concurrently on forked streams, so that a launch's elapsed
 * time includes the time it shares the GPU with the other groups' kernels.
 * OTVMC_PROFILE_SERIAL runs those groups one after another on the calling stream (the same
 * launches, no overlap), so that each elapsed time is the launch's own duration; results are
 * identical, only the schedule differs.  OTVMC_PROFILE_OFF (0) stops recording. */
enum { OTVMC_PROFILE_OFF = 0, OTVMC_PROFILE_ON = 1, OTVMC_PROFILE_SERIAL = 2 };
enum {
    OTVMC_K_SAMPLE = 0,  /* Metropolis sweeps */
    OTVMC_K_PREP = 1,    /* fixed-point parameter tables */
    OTVMC_K_EST1 = 2,    /* fields, flip ratios, E_H */
    OTVMC_K_EST2 = 3,    /* E_eff, v */
    OTVMC_K_REDUCE = 4,  /* site means, v reductions and quantisation */
    OTVMC_K_OBS = 5,     /* observables */
    OTVMC_K_D = 6,       /* D = Cov(O^*, v) and column means */
    OTVMC_K_OBUILD = 7,  /* O in E4M3 / FP64 */
    OTVMC_K_GRAM = 8,    /* Gram G = O^T O (tensor cores); the RBM T of the mixed T path */
    OTVMC_K_SYRK = 9,    /* FP64 S (plain path) */
    OTVMC_K_SOLVE = 10,  /* Cholesky solve (FP64 path) / triangular substitutions and refinement */
    OTVMC_K_SDE = 11,    /* predictor-corrector combination */
    OTVMC_K_NOISE = 12,  /* Wiener increments, chain initialisation */
    OTVMC_K_CHOLU = 13,  /* tensor-core block-column update of the Cholesky factorization */
    OTVMC_K_CHOLP = 14,  /* panel rows below the diagonal block (X = C L_dd^-T) */
    OTVMC_K_CHOLD = 15,  /* diagonal-block factor and inverse */
    OTVMC_K_RESID = 16,  /* refinement residual G x, tile-parallel */
    OTVMC_K_CLASSES = 17
};
OTVMC_API void otvmc_profile_enable(int on);
/* Synchronises the recorded events; total milliseconds and launch count of one class. */
OTVMC_API otvmc_status otvmc_profile_read(int kernel_class, double* total_ms, uint64_t* launches);

/* Test hook (the paper has no counterpart): bound, in nanoseconds, of the pipeline waits of
 * the tensor-core kernels (Gram, Cholesky update and panel) on the current device; 0 restores
 * the default of 2 s.  A wait that runs out makes its CTA stop issuing work, drain the copies
 * and products already in flight (those waits keep the 2 s bound), free its tensor memory and
 * return; OTVMC_ERR_TIMEOUT is then recorded in the status word and the call's results are
 * unspecified.  A tiny bound lets a test drive that path; it is not for production use.
 * Synchronous with respect to the device (a symbol copy); do not call while kernels of this
 * library run. */
OTVMC_API otvmc_status otvmc_debug_set_wait_limit(uint64_t ns);

/* Thread-local message describing the last error returned on this thread. */
OTVMC_API const char* otvmc_last_error(void);

/* Number of kernel launches this library has enqueued in this process (all threads). */
OTVMC_API uint64_t otvmc_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* OTVMC_H */
