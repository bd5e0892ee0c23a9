// Host-side internals of libotvmc: handle layouts and kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/otvmc.h"

struct otvmc_model {
    int n = 0;
    int nops = 0;
    double h = 0.0;
    std::vector<double> J, kappa, gamma;
    std::vector<int> op_kind, op_site;  // per jump operator: 0 decay, 1 dephasing
    // device copies
    double* J_d = nullptr;         // [n][n]
    long long* QJ_d = nullptr;     // [n][n] J in fixed point (2^-48 units)
    long long* baseJ_d = nullptr;  // [n] -sum_k QJ[j][k]
    double* site_d = nullptr;      // [4][n]: kappa, gamma, sqrt(kappa), sqrt(gamma)
    int* opidx_d = nullptr;        // [2][n]: decay / dephasing operator index, -1 if none
};

struct otvmc_ansatz {
    const otvmc_model* model = nullptr;
    int kind = 0;
    int n = 0;
    int m = 0;
    int64_t P = 0;
    int* pairs_d = nullptr;  // Jastrow: [P - n][2] sites (j, k), j < k
    int2* tiles_d = nullptr; // upper-triangle tiles of the tensor-core Gram kernel
    int ntiles = 0;
    int rbm_t_build = 0;     // OTVMC_RBM_T_FACTORED or OTVMC_RBM_T_MATERIALISED
    // Tied Jastrow (OTVMC_LJ): the full Jastrow of the same model, on which sampling, local
    // estimators, observables and the pair-level sums run with the expanded parameters, and the
    // groups of pairs that share a parameter (pairs by their full-Jastrow pair index).
    otvmc_ansatz* full = nullptr;
    int lj_d = 0, lj_pbc = 0, ngroups = 0;
    int* grp_off_d = nullptr;   // [ngroups + 1]
    int* grp_pair_d = nullptr;  // [N(N-1)/2], grouped
    int* pair_grp_d = nullptr;  // [N(N-1)/2] group of each pair
};

namespace otvmc {

void set_error(const std::string& msg);
otvmc_status cuda_status(cudaError_t e, const char* what);
void count_launch(int n = 1);

// Kernel timing (otvmc_profile_enable): records a CUDA event pair around a launch.
bool profiling();
bool profiling_serial();  // profiling with the solver's trajectory groups on the calling stream
void prof_record(int cls, cudaStream_t s, bool start);
struct ProfScope {
    int cls;
    cudaStream_t s;
    bool on;
    ProfScope(int c, cudaStream_t st) : cls(c), s(st), on(profiling()) {
        if (on) prof_record(cls, s, true);
    }
    ~ProfScope() {
        if (on) prof_record(cls, s, false);
    }
};

// Workspace carving: 256-byte aligned regions after the 256-byte status area.
struct Carver {
    char* base;
    size_t off;
    size_t cap;
    explicit Carver(void* b, size_t c) : base((char*)b), off(256), cap(c) {}
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
    bool ok() const { return off <= cap; }
};

constexpr int EST_SAMPLES_PER_THREAD = 8;
inline int est_threads_per_sample(int n) { return ((n + 31) / 32) * 32; }
inline int est_samples_per_block(int n) { return (256 / est_threads_per_sample(n)) * EST_SAMPLES_PER_THREAD; }
inline int est_blocks(int n, int ns) { int sb = est_samples_per_block(n); return (ns + sb - 1) / sb; }
inline int obs_samples_per_thread() { return 32; }
inline int obs_blocks(int n, int ns) {
    const int sb = (256 / est_threads_per_sample(n)) * obs_samples_per_thread();
    return (ns + sb - 1) / sb;
}
// Tensor-core local estimators (Jastrow, mixed path, ETC_MIN_N <= N <= ETC_MAX_N): CTAs of ETC_SITES sites
// by ETC_TILES tiles of 128 samples; E_H in one partial per site block, the per-site sums in
// one partial per CTA along the samples.
// Below ETC_MIN_N sites the SIMT kernel's N^2 work per sample is smaller than the tensor-core
// kernel's fixed costs (operand preparation, TMEM allocation, one more launch).
constexpr int ETC_SITES = 16, ETC_TILES = 4, ETC_MIN_N = 32, ETC_MAX_N = 128;
inline int est_tc_chunks(int ns) { return (ns + 128 * ETC_TILES - 1) / (128 * ETC_TILES); }
inline int est_tc_nq(int n) { return n <= ETC_MAX_N ? (n + ETC_SITES - 1) / ETC_SITES : 1; }
// Tensor-core observables (Jastrow, mixed path, OTC_MIN_N <= N <= OTC_MAX_N): one partial of
// the nine moments per 512 samples.
constexpr int OTC_MIN_N = 32, OTC_MAX_N = 64;
inline int obs_tc_chunks(int ns) { return (ns + 511) / 512; }
constexpr int VRED_BLOCK = 256;  // samples per block of the v reduction
inline int v_blocks(int ns) { return (ns + VRED_BLOCK - 1) / VRED_BLOCK; }

// Per-trajectory scratch of one evaluation (all device pointers).
struct EvalBufs {
    long long* Qre;      // [T][n][n]
    long long* Qim;      // [T][n][n]
    long long* base_re;  // [T][n]
    long long* base_im;  // [T][n]
    double2* r;          // [T][ns][n] flip ratios
    double2* EH;         // [T][ns]
    double2* part_r;     // [T][nblk][n]
    double2* part_sr;    // [T][nblk][n]
    double* part_s;      // [T][nblk][n]
    double2* mean_r;     // [T][n]
    double2* mean_sr;    // [T][n]
    double* mean_s;      // [T][n]
    double2* part_v;     // [T][vblk]
    double* part_vmax;   // [T][vblk]
    long long* qv;       // [T][ns][2] quantised centred v
    double* vinfo;       // [T][4]: mean re, mean im, 2^-e, qsum re/im as doubles? (see k_estim)
    long long* qsum;     // [T][2]
    double2* Epm;        // [T][2][n][n] exp(+-4 eta) for observables
    double* part_obs;    // [T][obs_blocks][9]
    long long* dsum;     // [T][P][3] exact sums behind D and obar
    float* dx;           // Jastrow only: [T][P][D_XROWS] sums of O_k against the extra rows of O
    float4* rtab;        // RBM only: the mixed kernels' FP32 tables (rbm_tab_bytes)
    char* etc;           // Jastrow, N <= ETC_MAX_N: operand images of the tensor-core estimators
    char* otc;           // Jastrow, OTC_MIN_N <= N <= OTC_MAX_N: operand images of the tensor-core observables
};
// EH is [T][ns][est_tc_nq(n)] for the Jastrow ansatz (partials per site block on the
// tensor-core path, the first entry alone otherwise), [T][ns] for the others.

// Extra rows of the E4M3 operand O on the mixed Jastrow path: the quantised centred v as
// sixteen balanced base-16 digits (in [-8, 7], exact in E4M3) of its real part and sixteen of
// its imaginary part, then a row of ones; the Gram kernel's tiles reach these columns, so the
// same tensor-core pass yields sum_x O_k(x) q(x) and sum_x O_k(x), exactly while 8 ns < 2^24.
constexpr int D_XROWS = 33;
constexpr int D_XROWS_MAX_NS = 1 << 17;

size_t eval_bufs_bytes(const otvmc_ansatz* a, int ntraj, int ns);
EvalBufs carve_eval_bufs(Carver& c, const otvmc_ansatz* a, int ntraj, int ns);
// Only the buffers of the Jastrow local estimators (prep, est1, site means, est2); the others
// are null.
EvalBufs carve_est_bufs(Carver& c, const otvmc_ansatz* a, int ntraj, int ns);

// ---- launchers (return cudaGetLastError of the launch)
cudaError_t launch_noise(const otvmc_model* m, int ntraj, int traj0, uint64_t seed, int64_t step,
                         double dt, double* dW, cudaStream_t s);
cudaError_t launch_init_chains(int n, int ntraj, int traj0, int ns, uint64_t seed, uint64_t* spins,
                               cudaStream_t s);
cudaError_t launch_sample_jastrow(const otvmc_ansatz* a, const double2* theta, int ntraj, int traj0,
                                  int ns, int n_sweep, uint64_t seed, int64_t eval, uint64_t* spins,
                                  unsigned long long* accepted, int* status, cudaStream_t s);
cudaError_t launch_jastrow_prep(const otvmc_ansatz* a, const double2* theta, int ntraj, const EvalBufs& b,
                                int* status, cudaStream_t s);
cudaError_t launch_est1_jastrow(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, bool fp32,
                                const EvalBufs& b, int* status, cudaStream_t s);
cudaError_t launch_site_means(const otvmc_ansatz* a, int ntraj, int ns, bool fp32, const EvalBufs& b, double* lpl,
                              cudaStream_t s);
cudaError_t launch_est2(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, bool fp32,
                        const double* dW, double dt, const double* lpl, const EvalBufs& b, double2* Eeff, double2* v,
                        cudaStream_t s);
cudaError_t launch_vpart(int ntraj, int ns, const double2* v, const EvalBufs& b, cudaStream_t s);
cudaError_t launch_vquant(int ntraj, int ns, const double2* v, const EvalBufs& b, cudaStream_t s);
cudaError_t launch_D_fixed_jastrow(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns,
                                   const EvalBufs& b, double* obar, double2* D, cudaStream_t s);
// Ot [ntraj][rows][o_pitch(ns)] E4M3 codes, samples from ns to the pitch zero: rows = P, or
// P + D_XROWS with the extra rows from qv when qv is given
constexpr int o_pitch(int ns) { return (ns + 15) / 16 * 16; }
cudaError_t launch_obuild_f8_jastrow(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns,
                                     const long long* qv, uint8_t* Ot, cudaStream_t s);
cudaError_t launch_obuild_f64_jastrow(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns,
                                      const double* obar, double* Oc, cudaStream_t s);
cudaError_t launch_syrk_f64(int ntraj, int P, int ns, const double* Oc, double* S, cudaStream_t s);
cudaError_t launch_gemv_D_f64(int ntraj, int P, int ns, const double* Oc, const double2* v, const EvalBufs& b,
                              double2* D, cudaStream_t s);
std::vector<int2> gram_tiles(int P);
std::vector<int2> gram_tiles_x(int P, int PC);
// G (P x P, upper) from the E4M3 operand Ot [ntraj][rows][pitch] (pitch a multiple of 16, the
// samples from ns on zero); with X, also X[t][k][c] = sum_x O_k O_{P+c} for k < P,
// c < rows - P (the extra rows; the tile list must reach column rows - 1).
cudaError_t launch_gram_tc(int ntraj, int P, int rows, int ns, int pitch, const uint8_t* Ot, const int2* tiles,
                           int ntiles, float* G, float* X, int* status, cudaStream_t s);
cudaError_t launch_D_from_gram(const otvmc_ansatz* a, int ntraj, int ns, const EvalBufs& b, double* obar, double2* D,
                               cudaStream_t s);
cudaError_t launch_expand_S(int ntraj, int P, int ns, const float* G, const double* obar, double* S,
                            cudaStream_t s);
// RBM ansatz, FP64 path (k_rbm.cu)
cudaError_t launch_sample_rbm(const otvmc_ansatz* an, const double2* theta, int ntraj, int traj0, int ns, int n_sweep,
                              uint64_t seed, int64_t eval, uint64_t* spins, double2* gam, double* lcr,
                              unsigned long long* accepted, cudaStream_t s);
cudaError_t launch_est_rbm(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int ntraj, int ns,
                           const EvalBufs& b, cudaStream_t s);
cudaError_t launch_obs_rbm(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int ntraj, int ns,
                           bool fp32, const EvalBufs& b, cudaStream_t s);
// RBM, FP32 sampling (decisions equal to FP64) and estimators (k_rbm_mixed.cu); M <= 256
constexpr int RBM_MIXED_MAX_M = 256;
cudaError_t launch_sample_rbm_mixed(const otvmc_ansatz* an, const double2* theta, int ntraj, int traj0, int ns,
                                    int n_sweep, uint64_t seed, int64_t eval, float4* tab, uint64_t* spins,
                                    unsigned long long* accepted, cudaStream_t s);
cudaError_t launch_est_rbm_mixed(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int ntraj,
                                 int ns, const EvalBufs& b, cudaStream_t s);
cudaError_t launch_obs_final(int n, int ns, int ntraj, const EvalBufs& b, double* moments, cudaStream_t s);
cudaError_t launch_obs_final_n(int n, int ns, int ntraj, int nblk, const EvalBufs& b, double* moments, cudaStream_t s);
size_t rbm_build_bytes(const otvmc_ansatz* a, int ntraj, int ns);
size_t rbm_solve_bytes(int ntraj, int P);
cudaError_t launch_rbm_build(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, const double2* v,
                             const double* vinfo, int T, int ns, void* ws, double2* S_out, double2* obar_out,
                             double2* D_out, cudaStream_t s);
cudaError_t launch_rbm_solve_S(const otvmc_ansatz* a, int T, int ns, double eps, const double2* S, const double2* D,
                               double2* delta, double* shift_used, void* ws, int* status, cudaStream_t s);
cudaError_t launch_rbm_build_solve(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, const double2* v,
                                   const double* vinfo, int T, int ns, double eps, void* ws, void* chol,
                                   double2* delta, int* status, cudaStream_t s);
size_t rbm_mixed_bytes(const otvmc_ansatz* a, int ntraj, int ns);
cudaError_t launch_rbm_build_solve_mixed(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins,
                                         const double2* v, const double* vinfo, int T, int ns, double eps, void* ws,
                                         double2* delta, int* status, cudaStream_t s);
cudaError_t launch_gram_split(int ntraj, int rows, int K, int kpad, const uint16_t* Xs, float* G, int* status,
                              cudaStream_t s);
// RBM T path of the mixed path without materialised O (k_rbm_factored.cu)
size_t rbm_factored_bytes(const otvmc_ansatz* a, int ntraj, int ns);
// Corrections of the mixed RBM solve against the exact operator (k_rbm_factored.cu)
// number of corrections: one after the factorised T (FP32 entries from exact integer and short
// FP32 sums), two after the materialised split-BF16 product (FP32 sums over K = 2P)
constexpr int RBM_REFINE_FACTORED = 1;
constexpr int RBM_REFINE_MATERIALISED = 2;
size_t rbm_tanh_obar_bytes(const otvmc_ansatz* a, int ntraj);
cudaError_t launch_rbm_tanh_obar(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int T, int ns,
                                 double2* Td, float2* Tf, unsigned long long* fmax, double2* obar, void* ws,
                                 cudaStream_t s);
size_t rbm_refine_bytes(const otvmc_ansatz* a, int ntraj, int ns);
cudaError_t launch_rbm_refine_push(const otvmc_ansatz* a, int T, int ns, double eps, int iters,
                                   const uint64_t* spins, const double2* Td, const unsigned long long* fmax,
                                   const double2* obar, const double2* rhs, double2* z, void* chol, void* ws,
                                   double2* delta, cudaStream_t s);
cudaError_t launch_rbm_refine_S(const otvmc_ansatz* a, int T, int ns, double eps, int iters, const uint64_t* spins,
                                const double2* Td, const unsigned long long* fmax, const double2* obar,
                                const double2* vemb, double2* xe, void* chol, void* ws, double2* delta,
                                cudaStream_t s);
cudaError_t launch_rbm_build_solve_factored(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins,
                                            const double2* v, const double* vinfo, int T, int ns, double eps,
                                            void* ws, double2* delta, int* status, cudaStream_t s);
// FP32 tables of the mixed RBM kernels, one buffer: flip factors [T][N][M] and [T][M][N]
// float4, then W [T][N][M] float2, then a [T][N] float2 (k_rbm_mixed.cu: rbm_flip_table_kernel)
inline size_t rbm_tab_bytes(const otvmc_ansatz* a, int ntraj) {
    return (size_t)ntraj * ((size_t)a->n * a->m * 40 + (size_t)a->n * 8) + 256;
}
// scratch of RBM sampling: the FP64 sampler's angles and Re lc [T][M][ns], then the FP32
// sampler's tables
inline size_t rbm_sample_bytes(const otvmc_ansatz* a, int ntraj, int ns) {
    return (size_t)ntraj * a->m * ns * (16 + 8) + rbm_tab_bytes(a, ntraj) + 1024;
}

// tied Jastrow (k_lj.cu)
cudaError_t launch_lj_expand(const otvmc_ansatz* a, int ntraj, const double2* theta, double2* theta_full,
                             cudaStream_t s);
// the tied log-derivatives O [ntraj][P][ns] int16 that launch_lj_build left in its workspace
const int16_t* lj_built_O(const otvmc_ansatz* a, int ntraj, const void* ws);
size_t lj_build_bytes(const otvmc_ansatz* a, int ntraj, int ns);
cudaError_t launch_lj_build(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, const EvalBufs& b,
                            void* ws, double* S, double* obar, double2* D, cudaStream_t s);

// SNR-filtered eigen pseudo-inverse (one CTA per trajectory, P <= SNR_PMAX)
constexpr int SNR_PMAX = 96;
constexpr double SNR_EPS_SVD = 1e-12;
size_t snr_smem_bytes(int P);
// the same filter for larger P: Householder tridiagonalisation, implicit QL, sample pass (k_snr_big.cu)
size_t snr_big_ws_bytes(int ntraj, int P);
bool snr_big_fits(int P);
cudaError_t launch_snr_big(const otvmc_ansatz* a, int ntraj, int ns, const uint64_t* spins, const double* S,
                           const double* obar, const double2* v, const double2* D, double thr, double eps_svd,
                           double2* delta, double* lam, void* ws, int* status, cudaStream_t s,
                           bool fp32_pass = false, const int16_t* Oint = nullptr);
cudaError_t launch_snr_solve(const otvmc_ansatz* a, int ntraj, int ns, const uint64_t* spins, const double* S,
                             const double* obar, const double2* v, const double2* D, double thr, double eps_svd,
                             double2* delta, double* lam, int* status, cudaStream_t s);
cudaError_t launch_chol_solve(int ntraj, int P, int ns, int precision, double eps, const double* S,
                              const float* G, const double* obar, const double2* D, double2* delta,
                              double* shift_used, void* ws, int refine_iters, int* status, cudaStream_t s);
size_t chol_ws_bytes(int ntraj, int P, int precision);
// bound of the pipeline waits of the tensor-core kernels of one translation unit (current device)
cudaError_t gram_set_wait_limit(unsigned long long ns);
cudaError_t est_tc_set_wait_limit(unsigned long long ns);
// Tensor-core local estimators (k_est_tc.cu): bytes of b.etc, and the launch (prep + fields,
// ratios, E_H partials, per-site sums) in place of the SIMT est1 kernel.
size_t est_tc_bytes(int ntraj, int n);
cudaError_t launch_est_tc(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, const EvalBufs& b,
                          int* status, cudaStream_t s);
// Tensor-core observables (k_obs_tc.cu): bytes of b.otc, and the launch (operand preparation,
// moments, final reduction) in place of observables_kernel + obs_final_kernel.
size_t obs_tc_bytes(int ntraj, int n);
cudaError_t obs_tc_set_wait_limit(unsigned long long ns);
cudaError_t launch_obs_tc(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, const EvalBufs& b,
                          double* moments, int* status, cudaStream_t s);
inline bool obs_tc_ok(const otvmc_ansatz* a, bool fp32) {
    return fp32 && a->kind == OTVMC_JASTROW && a->n >= OTC_MIN_N && a->n <= OTC_MAX_N;
}
inline bool est_tc_ok(const otvmc_ansatz* a, bool fp32) {
    return fp32 && a->kind == OTVMC_JASTROW && a->n >= ETC_MIN_N && a->n <= ETC_MAX_N;
}
cudaError_t chol_set_wait_limit(unsigned long long ns);
// number of trajectory groups of the mixed solver's launches issued by this host thread from now
// on (0: the built-in rule); returns the previous setting
int chol_set_groups(int groups);
constexpr int CHOL_MAX_GROUPS = 4;
// x += (L L^T)^-1 r with the factor left in ws by the last mixed (tensor-core) solve of this size
cudaError_t launch_chol_tc_resolve(int ntraj, int P, void* ws, const double2* r, double2* x, cudaStream_t s);
// linear SSE: ln Q of every trajectory from the mean of v^lin (k_misc.cu)
cudaError_t launch_lnq(int ntraj, int scheme, int stage, const double* vinfo, double* g0, double* lnQ,
                       cudaStream_t s);
cudaError_t launch_sde(int ntraj, int64_t P, int scheme, int stage, const double2* theta, const double2* d0,
                       const double2* d1, double2* out, int* failed, int* status, cudaStream_t s);
cudaError_t launch_obs_prep(const otvmc_ansatz* a, const double2* theta, int ntraj, bool fp32,
                            const EvalBufs& b, cudaStream_t s);
cudaError_t launch_observables(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, bool fp32,
                               const EvalBufs& b, double* moments, int* status, cudaStream_t s);

}  // namespace otvmc
