// C ABI of libotvmc: handles, argument checks, workspace carving, stage entry points and
// the batched trajectory driver (otVMC procedure paragraph, App. C).
#include <atomic>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace otvmc {

static thread_local std::string g_err;
static std::atomic<unsigned long long> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::atomic<bool> g_prof_on{false};
static std::atomic<bool> g_prof_serial{false};
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_prof_pool;

bool profiling() { return g_prof_on.load(std::memory_order_relaxed); }
bool profiling_serial() { return g_prof_serial.load(std::memory_order_relaxed); }

void prof_record(int cls, cudaStream_t s, bool start) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e;
    if (!g_prof_pool.empty()) {
        e = g_prof_pool.back();
        g_prof_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return;
    }
    cudaEventRecord(e, s);
    if (start) {
        g_prof.push_back({cls, e, nullptr});
    } else {
        for (auto it = g_prof.rbegin(); it != g_prof.rend(); ++it)
            if (it->cls == cls && it->b == nullptr) {
                it->b = e;
                return;
            }
        g_prof_pool.push_back(e);
    }
}
void count_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
otvmc_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return OTVMC_OK;
    std::string detail = g_err.rfind("cholesky:", 0) == 0 ? " (" + g_err + ")" : std::string();
    set_error(std::string(what) + ": " + cudaGetErrorString(e) + detail);
    return OTVMC_ERR_CUDA;
}

static otvmc_status fail(otvmc_status st, const std::string& msg) {
    set_error(msg);
    return st;
}

#define CK(expr, what)                                              \
    do {                                                            \
        cudaError_t e_ = (expr);                                    \
        if (e_ != cudaSuccess) return cuda_status(e_, what);        \
    } while (0)

size_t eval_bufs_bytes(const otvmc_ansatz* a, int ntraj, int ns) {
    Carver c(nullptr, (size_t)-1);
    carve_eval_bufs(c, a, ntraj, ns);
    return c.off;
}

EvalBufs carve_eval_bufs(Carver& c, const otvmc_ansatz* a, int T, int ns) {
    const int n = a->n;
    const size_t nblk = est_blocks(n, ns), vblk = v_blocks(ns);
    EvalBufs b;
    b.Qre = c.take<long long>((size_t)T * n * n);
    b.Qim = c.take<long long>((size_t)T * n * n);
    b.base_re = c.take<long long>((size_t)T * n);
    b.base_im = c.take<long long>((size_t)T * n);
    b.r = c.take<double2>((size_t)T * ns * n);
    b.EH = c.take<double2>((size_t)T * ns * (a->kind == OTVMC_JASTROW ? est_tc_nq(n) : 1));
    b.part_r = c.take<double2>((size_t)T * nblk * n);
    b.part_sr = c.take<double2>((size_t)T * nblk * n);
    b.part_s = c.take<double>((size_t)T * nblk * n);
    b.mean_r = c.take<double2>((size_t)T * n);
    b.mean_sr = c.take<double2>((size_t)T * n);
    b.mean_s = c.take<double>((size_t)T * n);
    b.part_v = c.take<double2>((size_t)T * vblk);
    b.part_vmax = c.take<double>((size_t)T * vblk);
    b.qv = c.take<long long>((size_t)T * ns * 2);
    b.vinfo = c.take<double>((size_t)T * 4);
    b.qsum = c.take<long long>((size_t)T * 2);
    b.Epm = c.take<double2>((size_t)T * 2 * n * n);
    b.rtab = a->kind == OTVMC_RBM ? (float4*)c.take<char>(rbm_tab_bytes(a, T)) : nullptr;
    b.part_obs = c.take<double>((size_t)T * (nblk > (size_t)obs_blocks(n, ns) ? nblk : obs_blocks(n, ns)) * 9);
    b.dsum = c.take<long long>((size_t)T * a->P * 3);
    b.dx = a->kind == OTVMC_JASTROW ? c.take<float>((size_t)T * a->P * D_XROWS) : nullptr;
    b.etc = (a->kind == OTVMC_JASTROW && n <= ETC_MAX_N) ? c.take<char>(est_tc_bytes(T, n)) : nullptr;
    b.otc = (a->kind == OTVMC_JASTROW && n >= OTC_MIN_N && n <= OTC_MAX_N) ? c.take<char>(obs_tc_bytes(T, n)) : nullptr;
    return b;
}

EvalBufs carve_est_bufs(Carver& c, const otvmc_ansatz* a, int T, int ns) {
    const int n = a->n;
    const size_t nblk = est_blocks(n, ns), vblk = v_blocks(ns);
    EvalBufs b{};
    b.Qre = c.take<long long>((size_t)T * n * n);
    b.Qim = c.take<long long>((size_t)T * n * n);
    b.base_re = c.take<long long>((size_t)T * n);
    b.base_im = c.take<long long>((size_t)T * n);
    b.r = c.take<double2>((size_t)T * ns * n);
    b.EH = c.take<double2>((size_t)T * ns * (a->kind == OTVMC_JASTROW ? est_tc_nq(n) : 1));
    b.part_r = c.take<double2>((size_t)T * nblk * n);
    b.part_sr = c.take<double2>((size_t)T * nblk * n);
    b.part_s = c.take<double>((size_t)T * nblk * n);
    b.mean_r = c.take<double2>((size_t)T * n);
    b.mean_sr = c.take<double2>((size_t)T * n);
    b.mean_s = c.take<double>((size_t)T * n);
    b.part_v = c.take<double2>((size_t)T * vblk);
    b.part_vmax = c.take<double>((size_t)T * vblk);
    b.etc = (a->kind == OTVMC_JASTROW && n <= ETC_MAX_N) ? c.take<char>(est_tc_bytes(T, n)) : nullptr;
    return b;
}

static size_t obuf_bytes(const otvmc_ansatz* a, int T, int ns, int precision) {
    if (precision == OTVMC_PREC_FP64) return (size_t)T * a->P * ns * 8 + 256;
    return (size_t)T * (a->P + D_XROWS) * o_pitch(ns) + 256;  // E4M3 O and its extra rows
}

static bool valid_ansatz(const otvmc_ansatz* a) { return a != nullptr && a->model != nullptr && a->P > 0; }

static otvmc_status check_batch(const otvmc_ansatz* a, int ntraj, int ns) {
    if (!valid_ansatz(a)) return fail(OTVMC_ERR_INVALID, "null or invalid ansatz");
    if (ntraj < 1 || ns < 1) return fail(OTVMC_ERR_INVALID, "ntraj and ns must be >= 1");
    return OTVMC_OK;
}
static otvmc_status rbm_precision(const otvmc_ansatz* a, int precision) {
    if (a->kind == OTVMC_RBM && precision == OTVMC_PREC_MIXED && a->m > RBM_MIXED_MAX_M)
        return fail(OTVMC_ERR_UNSUPPORTED, "the mixed RBM path is built for n_hidden <= 256");
    return OTVMC_OK;
}
// RBM sampling: the FP32 warp-per-chain sampler (its decisions equal the FP64 ones) when the
// hidden layer fits it, else the FP64 thread-per-chain sampler with its scratch.
static cudaError_t sample_rbm_any(const otvmc_ansatz* a, const double2* theta, int T, int traj0, int ns, int n_sweep,
                                  uint64_t seed, int64_t ev, uint64_t* spins, double2* gam, double* lcr, float4* tab,
                                  unsigned long long* accepted, cudaStream_t s) {
    if (a->m <= RBM_MIXED_MAX_M)
        return launch_sample_rbm_mixed(a, theta, T, traj0, ns, n_sweep, seed, ev, tab, spins, accepted, s);
    return launch_sample_rbm(a, theta, T, traj0, ns, n_sweep, seed, ev, spins, gam, lcr, accepted, s);
}

}  // namespace otvmc

using namespace otvmc;

extern "C" {

const char* otvmc_last_error(void) { return g_err.c_str(); }

void otvmc_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_prof) {
        if (r.a) g_prof_pool.push_back(r.a);
        if (r.b) g_prof_pool.push_back(r.b);
    }
    g_prof.clear();
    g_prof_on.store(on != 0);
    g_prof_serial.store(on == OTVMC_PROFILE_SERIAL);
}

otvmc_status otvmc_profile_read(int cls, double* total_ms, uint64_t* launches) {
    if (cls < 0 || cls >= OTVMC_K_CLASSES) return fail(OTVMC_ERR_INVALID, "unknown kernel class");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    double ms = 0.0;
    uint64_t cnt = 0;
    for (auto& r : g_prof) {
        if (r.cls != cls || !r.b) continue;
        CK(cudaEventSynchronize(r.b), "event synchronize");
        float f = 0.f;
        CK(cudaEventElapsedTime(&f, r.a, r.b), "event elapsed");
        ms += f;
        ++cnt;
    }
    if (total_ms) *total_ms = ms;
    if (launches) *launches = cnt;
    return OTVMC_OK;
}
uint64_t otvmc_launch_count(void) { return g_launches.load(); }

otvmc_status otvmc_debug_set_wait_limit(uint64_t ns) {
    const unsigned long long v = ns == 0 ? 2000000000ull : (unsigned long long)ns;
    CK(gram_set_wait_limit(v), "set wait limit (Gram kernel)");
    CK(chol_set_wait_limit(v), "set wait limit (Cholesky kernels)");
    CK(est_tc_set_wait_limit(v), "set wait limit (estimator kernels)");
    CK(obs_tc_set_wait_limit(v), "set wait limit (observables kernels)");
    return OTVMC_OK;
}

otvmc_status otvmc_lattice_couplings(int dim, const int* extent, double J, double alpha, int kac, int pbc,
                                     double* J_out_h) {
    if ((dim != 1 && dim != 2) || !extent || !J_out_h) return fail(OTVMC_ERR_INVALID, "dim must be 1 or 2");
    const int lx = extent[0], ly = dim == 2 ? extent[1] : 1;
    if (lx < 1 || ly < 1) return fail(OTVMC_ERR_INVALID, "bad extent");
    const int n = lx * ly;
    double ksum = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            if (i == j) {
                J_out_h[i * n + j] = 0.0;
                continue;
            }
            double dx = std::fabs((double)(i / ly - j / ly)), dy = std::fabs((double)(i % ly - j % ly));
            if (dim == 1) {
                dx = std::fabs((double)(i - j));
                dy = 0.0;
            }
            if (pbc) {
                dx = std::fmin(dx, (double)lx - dx);
                if (dim == 2) dy = std::fmin(dy, (double)ly - dy);
            }
            const double r = std::sqrt(dx * dx + dy * dy);
            J_out_h[i * n + j] = J * std::pow(r, -alpha);
            if (i < j) ksum += std::pow(r, -alpha);
        }
    if (kac && n > 1) {
        const double K = ksum / (n - 1);
        for (int i = 0; i < n * n; ++i) J_out_h[i] /= K;
    }
    return OTVMC_OK;
}

otvmc_status otvmc_model_create(const otvmc_model_desc* d, otvmc_model** out) {
    if (!d || !out || !d->J_h) return fail(OTVMC_ERR_INVALID, "null model description");
    const int n = d->n;
    if (n < 1 || n > OTVMC_MAX_SITES) return fail(OTVMC_ERR_INVALID, "n out of range");
    auto* m = new otvmc_model();
    m->n = n;
    m->h = d->h;
    m->J.assign(d->J_h, d->J_h + (size_t)n * n);
    m->kappa.assign(n, 0.0);
    m->gamma.assign(n, 0.0);
    if (d->kappa_h) m->kappa.assign(d->kappa_h, d->kappa_h + n);
    if (d->gamma_h) m->gamma.assign(d->gamma_h, d->gamma_h + n);
    for (int i = 0; i < n; ++i) {
        if (!(m->kappa[i] >= 0.0) || !(m->gamma[i] >= 0.0) || !std::isfinite(m->kappa[i]) ||
            !std::isfinite(m->gamma[i])) {
            delete m;
            return fail(OTVMC_ERR_INVALID, "rates must be finite and >= 0");
        }
        double rowsum = 0.0;
        for (int j = 0; j < n; ++j) {
            const double v = m->J[(size_t)i * n + j];
            if (!std::isfinite(v) || v != m->J[(size_t)j * n + i] || (i == j && v != 0.0)) {
                delete m;
                return fail(OTVMC_ERR_INVALID, "J must be finite, symmetric, zero diagonal");
            }
            rowsum += std::fabs(v);
        }
        if (!(rowsum < 8192.0)) {
            delete m;
            return fail(OTVMC_ERR_RANGE, "row sums of |J| must be < 8192 (fixed-point range)");
        }
    }
    std::vector<int> opidx(2 * n, -1);
    for (int i = 0; i < n; ++i)
        if (m->kappa[i] > 0) {
            opidx[i] = (int)m->op_kind.size();
            m->op_kind.push_back(0);
            m->op_site.push_back(i);
        }
    for (int i = 0; i < n; ++i)
        if (m->gamma[i] > 0) {
            opidx[n + i] = (int)m->op_kind.size();
            m->op_kind.push_back(1);
            m->op_site.push_back(i);
        }
    m->nops = (int)m->op_kind.size();
    std::vector<long long> QJ((size_t)n * n), baseJ(n);
    for (int i = 0; i < n; ++i) {
        long long s = 0;
        for (int j = 0; j < n; ++j) {
            QJ[(size_t)i * n + j] = std::llrint(m->J[(size_t)i * n + j] * 281474976710656.0);
            s += QJ[(size_t)i * n + j];
        }
        baseJ[i] = -s;
    }
    std::vector<double> site(4 * n);
    for (int i = 0; i < n; ++i) {
        site[i] = m->kappa[i];
        site[n + i] = m->gamma[i];
        site[2 * n + i] = std::sqrt(m->kappa[i]);
        site[3 * n + i] = std::sqrt(m->gamma[i]);
    }
    bool ok = cudaMalloc(&m->J_d, sizeof(double) * n * n) == cudaSuccess &&
              cudaMalloc(&m->QJ_d, sizeof(long long) * n * n) == cudaSuccess &&
              cudaMalloc(&m->baseJ_d, sizeof(long long) * n) == cudaSuccess &&
              cudaMalloc(&m->site_d, sizeof(double) * 4 * n) == cudaSuccess &&
              cudaMalloc(&m->opidx_d, sizeof(int) * 2 * n) == cudaSuccess;
    ok = ok && cudaMemcpy(m->J_d, m->J.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->QJ_d, QJ.data(), sizeof(long long) * n * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->baseJ_d, baseJ.data(), sizeof(long long) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->site_d, site.data(), sizeof(double) * 4 * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->opidx_d, opidx.data(), sizeof(int) * 2 * n, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        otvmc_model_destroy(m);
        return fail(OTVMC_ERR_OOM, "device allocation for the model failed");
    }
    *out = m;
    return OTVMC_OK;
}

void otvmc_model_destroy(otvmc_model* m) {
    if (!m) return;
    cudaFree(m->J_d);
    cudaFree(m->QJ_d);
    cudaFree(m->baseJ_d);
    cudaFree(m->site_d);
    cudaFree(m->opidx_d);
    delete m;
}

int otvmc_model_nops(const otvmc_model* m) { return m ? m->nops : 0; }

otvmc_status otvmc_ansatz_create(const otvmc_model* model, int kind, int n_hidden, otvmc_ansatz** out) {
    if (!model || !out) return fail(OTVMC_ERR_INVALID, "null model");
    if (kind != OTVMC_JASTROW && kind != OTVMC_RBM) return fail(OTVMC_ERR_INVALID, "unknown ansatz kind");
    const int n = model->n;
    if (kind == OTVMC_RBM) {
        if (n_hidden < 1 || n_hidden > 4096) return fail(OTVMC_ERR_INVALID, "RBM needs 1 <= n_hidden <= 4096");
        auto* a = new otvmc_ansatz();
        a->model = model;
        a->kind = kind;
        a->n = n;
        a->m = n_hidden;
        a->P = (int64_t)n + n_hidden + (int64_t)n * n_hidden;
        *out = a;
        return OTVMC_OK;
    }
    if (n > 200) return fail(OTVMC_ERR_UNSUPPORTED, "Jastrow kernels are built for n <= 200");
    auto* a = new otvmc_ansatz();
    a->model = model;
    a->kind = kind;
    a->n = n;
    a->P = (int64_t)n * (n + 1) / 2;
    std::vector<int> pairs;
    for (int j = 0; j < n; ++j)
        for (int k = j + 1; k < n; ++k) {
            pairs.push_back(j);
            pairs.push_back(k);
        }
    std::vector<int2> tiles = gram_tiles_x((int)a->P, (int)a->P + D_XROWS);
    a->ntiles = (int)tiles.size();
    bool ok = true;
    if (!pairs.empty())
        ok = cudaMalloc(&a->pairs_d, sizeof(int) * pairs.size()) == cudaSuccess &&
             cudaMemcpy(a->pairs_d, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMalloc(&a->tiles_d, sizeof(int2) * tiles.size()) == cudaSuccess &&
         cudaMemcpy(a->tiles_d, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        otvmc_ansatz_destroy(a);
        return fail(OTVMC_ERR_OOM, "device allocation for the ansatz failed");
    }
    *out = a;
    return OTVMC_OK;
}

void otvmc_ansatz_destroy(otvmc_ansatz* a) {
    if (!a) return;
    cudaFree(a->pairs_d);
    cudaFree(a->tiles_d);
    cudaFree(a->grp_off_d);
    cudaFree(a->grp_pair_d);
    cudaFree(a->pair_grp_d);
    otvmc_ansatz_destroy(a->full);
    delete a;
}

otvmc_status otvmc_ansatz_create_lj(const otvmc_model* model, int d, int pbc, otvmc_ansatz** out) {
    if (!model || !out || d < 0 || (pbc != 0 && pbc != 1)) return fail(OTVMC_ERR_INVALID, "create_lj: bad arguments");
    otvmc_ansatz* full = nullptr;
    otvmc_status st = otvmc_ansatz_create(model, OTVMC_JASTROW, 0, &full);
    if (st) return st;
    const int n = model->n;
    auto dist = [&](int j, int k) { return pbc ? std::min(k - j, n - (k - j)) : k - j; };
    auto pidx = [&](int j, int k) { return j * n - j * (j + 1) / 2 + (k - j - 1); };
    // groups: each pair at distance <= d on its own (row-major), then one group per larger distance
    std::vector<int> off{0}, gpair, pgrp((size_t)n * (n - 1) / 2, -1);
    for (int j = 0; j < n; ++j)
        for (int k = j + 1; k < n; ++k)
            if (dist(j, k) <= d) {
                pgrp[pidx(j, k)] = (int)off.size() - 1;
                gpair.push_back(pidx(j, k));
                off.push_back((int)gpair.size());
            }
    for (int D = d + 1; D < n; ++D) {
        const size_t before = gpair.size();
        for (int j = 0; j < n; ++j)
            for (int k = j + 1; k < n; ++k)
                if (dist(j, k) == D) {
                    pgrp[pidx(j, k)] = (int)off.size() - 1;
                    gpair.push_back(pidx(j, k));
                }
        if (gpair.size() > before) off.push_back((int)gpair.size());
    }
    auto* a = new otvmc_ansatz();
    a->model = model;
    a->kind = OTVMC_LJ;
    a->n = n;
    a->full = full;
    a->lj_d = d;
    a->lj_pbc = pbc;
    a->ngroups = (int)off.size() - 1;
    a->P = (int64_t)n + a->ngroups;
    bool ok = cudaMalloc(&a->grp_off_d, sizeof(int) * off.size()) == cudaSuccess &&
              cudaMemcpy(a->grp_off_d, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !gpair.empty())
        ok = cudaMalloc(&a->grp_pair_d, sizeof(int) * gpair.size()) == cudaSuccess &&
             cudaMemcpy(a->grp_pair_d, gpair.data(), sizeof(int) * gpair.size(), cudaMemcpyHostToDevice) ==
                 cudaSuccess &&
             cudaMalloc(&a->pair_grp_d, sizeof(int) * pgrp.size()) == cudaSuccess &&
             cudaMemcpy(a->pair_grp_d, pgrp.data(), sizeof(int) * pgrp.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        otvmc_ansatz_destroy(a);
        return fail(OTVMC_ERR_OOM, "device allocation for the ansatz failed");
    }
    *out = a;
    return OTVMC_OK;
}

// The ansatz whose kernels run the sampling, estimators and observables: the full Jastrow of a
// tied Jastrow (on the expanded parameters), else the ansatz itself.
static const otvmc_ansatz* eval_ansatz(const otvmc_ansatz* a) { return a->kind == OTVMC_LJ ? a->full : a; }

int64_t otvmc_ansatz_nparams(const otvmc_ansatz* a) { return a ? a->P : 0; }

otvmc_status otvmc_ansatz_set_rbm_t_build(otvmc_ansatz* a, int mode) {
    if (!a || a->kind != OTVMC_RBM) return fail(OTVMC_ERR_INVALID, "set_rbm_t_build: not an RBM ansatz");
    if (mode != OTVMC_RBM_T_FACTORED && mode != OTVMC_RBM_T_MATERIALISED)
        return fail(OTVMC_ERR_INVALID, "set_rbm_t_build: unknown mode");
    a->rbm_t_build = mode;
    return OTVMC_OK;
}

size_t otvmc_workspace_bytes(const otvmc_ansatz* a, int ntraj, int ns, int precision) {
    if (!valid_ansatz(a) || ntraj < 1 || ns < 1) return 0;
    const size_t ev = eval_bufs_bytes(a, ntraj, ns);
    if (a->kind == OTVMC_RBM) {
        // sample scratch, estimators + lpl, build (R, embedded S, obar), solve (embedded S + Cholesky)
        size_t m = rbm_sample_bytes(a, ntraj, ns) + 256;
        const size_t est = ev + (size_t)ntraj * (a->model->nops + 1) * 8 + 1024;
        const size_t build = ev + rbm_build_bytes(a, ntraj, ns) + 1024;
        const size_t solve = 256 + rbm_solve_bytes(ntraj, (int)a->P) + 1024;
        if (est > m) m = est;
        if (build > m) m = build;
        if (solve > m) m = solve;
        return m + 256;
    }
    if (a->kind == OTVMC_LJ) {
        // expanded parameters, then the full Jastrow's evaluation buffers and the tied build, or
        // the FP64 solve
        const size_t thf = (size_t)ntraj * a->full->P * 16 + 256;
        size_t m = thf + eval_bufs_bytes(a->full, ntraj, ns) + (size_t)ntraj * (a->model->nops + 1) * 8 +
                   lj_build_bytes(a, ntraj, ns) + (size_t)ntraj * a->P * 8 + 2048;
        const size_t solve = 256 + chol_ws_bytes(ntraj, (int)a->P, OTVMC_PREC_FP64);
        if (solve > m) m = solve;
        return m + 256;
    }
    const size_t build = ev + obuf_bytes(a, ntraj, ns, precision) + (size_t)ntraj * a->P * 8 + 1024;
    const size_t solve = 256 + chol_ws_bytes(ntraj, (int)a->P, precision);
    size_t m = ev;
    if (build > m) m = build;
    if (solve > m) m = solve;
    return m + 256;
}

otvmc_status otvmc_check(void* work_d, void* stream) {
    if (!work_d) return fail(OTVMC_ERR_INVALID, "null workspace");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(s), "stream synchronize");
    int st[2] = {0, 0};
    CK(cudaMemcpy(st, work_d, sizeof(st), cudaMemcpyDeviceToHost), "status read");
    if (st[0] != 0) {
        const int zero[2] = {0, 0};
        CK(cudaMemcpy(work_d, zero, sizeof(zero), cudaMemcpyHostToDevice), "status clear");
        char buf[128];
        std::snprintf(buf, sizeof(buf), "device status %d (trajectory/detail %d)", st[0], st[1]);
        set_error(buf);
        return (otvmc_status)st[0];
    }
    return OTVMC_OK;
}

otvmc_status otvmc_draw_noise(const otvmc_model* m, int ntraj, int traj0, uint64_t seed, int64_t step, double dt,
                              double* dW_d, void* stream) {
    if (!m || ntraj < 1 || traj0 < 0 || !(dt > 0.0) || (m->nops > 0 && !dW_d))
        return fail(OTVMC_ERR_INVALID, "draw_noise: bad arguments");
    CK(launch_noise(m, ntraj, traj0, seed, step, dt, dW_d, (cudaStream_t)stream), "noise launch");
    return OTVMC_OK;
}

otvmc_status otvmc_init_chains(const otvmc_ansatz* a, int ntraj, int traj0, int ns, uint64_t seed,
                               uint64_t* spins_d, void* stream) {
    if (!valid_ansatz(a) || ntraj < 1 || ns < 1 || traj0 < 0 || !spins_d)
        return fail(OTVMC_ERR_INVALID, "init_chains: bad arguments");
    CK(launch_init_chains(a->n, ntraj, traj0, ns, seed, spins_d, (cudaStream_t)stream), "init launch");
    return OTVMC_OK;
}

otvmc_status otvmc_sample(const otvmc_ansatz* a, const double* theta_d, int ntraj, int traj0, int ns, int n_sweep,
                          uint64_t seed, int64_t eval_index, uint64_t* spins_d, uint64_t* accepted_d, void* work_d,
                          size_t work_bytes, void* stream) {
    otvmc_status st = check_batch(a, ntraj, ns);
    if (st) return st;
    if (!theta_d || !spins_d || !work_d || n_sweep < 0 || traj0 < 0)
        return fail(OTVMC_ERR_INVALID, "sample: bad arguments");
    if (work_bytes < 256) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
    if (a->kind == OTVMC_RBM) {
        Carver c(work_d, work_bytes);
        double2* gam = c.take<double2>((size_t)ntraj * a->m * ns);
        double* lcr = c.take<double>((size_t)ntraj * a->m * ns);
        float4* tab = (float4*)c.take<char>(rbm_tab_bytes(a, ntraj));
        if (!c.ok()) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
        CK(sample_rbm_any(a, (const double2*)theta_d, ntraj, traj0, ns, n_sweep, seed, eval_index, spins_d, gam, lcr,
                             tab, (unsigned long long*)accepted_d, (cudaStream_t)stream),
           "sample launch");
        return OTVMC_OK;
    }
    const double2* th = (const double2*)theta_d;
    if (a->kind == OTVMC_LJ) {
        Carver c(work_d, work_bytes);
        double2* thf = c.take<double2>((size_t)ntraj * a->full->P);
        if (!c.ok()) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
        CK(launch_lj_expand(a, ntraj, th, thf, (cudaStream_t)stream), "expand launch");
        th = thf;
    }
    CK(launch_sample_jastrow(eval_ansatz(a), th, ntraj, traj0, ns, n_sweep, seed, eval_index, spins_d,
                             (unsigned long long*)accepted_d, (int*)work_d, (cudaStream_t)stream),
       "sample launch");
    return OTVMC_OK;
}

// est1 + site means + est2 on carved buffers; lpl may be internal.
// lpl_e (optional): the <L + L^+> that E_eff takes, in place of the estimated ones (zeros give the
// linear SSE's E_eff^lin = E_H - i/2 sum_n [(L^+L)_loc + (L^2)_loc]).
static otvmc_status run_estimators(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int T, int ns,
                                   const double* dW, double dt, bool fp32, const EvalBufs& b, double* lpl,
                                   double2* Eeff, double2* v, int* status, cudaStream_t s,
                                   const double* lpl_e = nullptr) {
    if (a->kind == OTVMC_RBM) {
        if (fp32) CK(launch_est_rbm_mixed(a, theta, spins, T, ns, b, s), "est rbm launch");
        else CK(launch_est_rbm(a, theta, spins, T, ns, b, s), "est rbm launch");
    } else {
        CK(launch_jastrow_prep(a, theta, T, b, status, s), "prep launch");
        CK(launch_est1_jastrow(a, spins, T, ns, fp32, b, status, s), "est1 launch");
    }
    CK(launch_site_means(a, T, ns, fp32, b, lpl, s), "site means launch");
    if (v) CK(launch_est2(a, spins, T, ns, fp32, dW, dt, lpl_e ? lpl_e : lpl, b, Eeff, v, s), "est2 launch");
    return OTVMC_OK;
}

otvmc_status otvmc_local_estimators(const otvmc_ansatz* a, const double* theta_d, const uint64_t* spins_d, int ntraj,
                                    int ns, const double* dW_d, double dt, int precision, double* Eeff_d,
                                    double* v_d, double* lpl_d, void* work_d, size_t work_bytes, void* stream) {
    otvmc_status st = check_batch(a, ntraj, ns);
    if (st) return st;
    if (!theta_d || !spins_d || !v_d || !work_d || (a->model->nops > 0 && !dW_d))
        return fail(OTVMC_ERR_INVALID, "local_estimators: bad arguments");
    if (precision != OTVMC_PREC_FP64 && precision != OTVMC_PREC_MIXED)
        return fail(OTVMC_ERR_INVALID, "unknown precision");
    if ((st = rbm_precision(a, precision))) return st;
    Carver c(work_d, work_bytes);
    double2* thf = a->kind == OTVMC_LJ ? c.take<double2>((size_t)ntraj * a->full->P) : nullptr;
    EvalBufs b = carve_eval_bufs(c, eval_ansatz(a), ntraj, ns);
    double* lpl = lpl_d ? lpl_d : c.take<double>((size_t)ntraj * (a->model->nops + 1));
    if (!c.ok()) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
    const double2* th = (const double2*)theta_d;
    if (thf) {
        CK(launch_lj_expand(a, ntraj, th, thf, (cudaStream_t)stream), "expand launch");
        th = thf;
    }
    return run_estimators(eval_ansatz(a), th, spins_d, ntraj, ns, dW_d, dt, precision == OTVMC_PREC_MIXED, b, lpl,
                          (double2*)Eeff_d, (double2*)v_d, (int*)work_d, (cudaStream_t)stream);
}

// D (and obar) from v; S or G by precision.
static otvmc_status run_build(const otvmc_ansatz* a, const uint64_t* spins, const double2* v, int T, int ns,
                              int precision, bool v_parts_ready, const EvalBufs& b, void* obuf, double* S, float* G,
                              double* obar, double2* D, int* status, cudaStream_t s) {
    const int P = (int)a->P;
    if (!v_parts_ready) CK(launch_vpart(T, ns, v, b, s), "vpart launch");
    CK(launch_vquant(T, ns, v, b, s), "vquant launch");
    if (precision == OTVMC_PREC_FP64) {
        CK(launch_D_fixed_jastrow(a, spins, T, ns, b, obar, D, s), "D launch");
        double* Oc = (double*)obuf;
        CK(launch_obuild_f64_jastrow(a, spins, T, ns, obar, Oc, s), "obuild f64 launch");
        CK(launch_syrk_f64(T, P, ns, Oc, S, s), "syrk launch");
        CK(launch_gemv_D_f64(T, P, ns, Oc, v, b, D, s), "gemv launch");
    } else {
        // D and obar from the Gram pass (the digits of q as extra rows of O) while the digit
        // sums stay exact in FP32; else by the integer sums
        const bool dx = b.dx != nullptr && ns <= D_XROWS_MAX_NS;
        if (!dx) CK(launch_D_fixed_jastrow(a, spins, T, ns, b, obar, D, s), "D launch");
        uint8_t* Ot = (uint8_t*)obuf;
        CK(launch_obuild_f8_jastrow(a, spins, T, ns, dx ? b.qv : nullptr, Ot, s), "obuild launch");
        CK(launch_gram_tc(T, P, dx ? P + D_XROWS : P, ns, o_pitch(ns), Ot, a->tiles_d, a->ntiles, G,
                          dx ? b.dx : nullptr, status, s),
           "gram launch");
        if (dx) CK(launch_D_from_gram(a, T, ns, b, obar, D, s), "D launch");
        if (S) CK(launch_expand_S(T, P, ns, G, obar, S, s), "expand launch");
    }
    return OTVMC_OK;
}

otvmc_status otvmc_build_S_F(const otvmc_ansatz* a, const double* theta_d, const uint64_t* spins_d,
                             const double* v_d, int ntraj, int ns, int precision, double* S_d, float* G_d,
                             double* obar_d, double* D_d, void* work_d, size_t work_bytes, void* stream) {
    otvmc_status st = check_batch(a, ntraj, ns);
    if (st) return st;
    if (!spins_d || !v_d || !D_d || !work_d) return fail(OTVMC_ERR_INVALID, "build_S_F: bad arguments");
    if (a->kind == OTVMC_RBM) {
        if ((st = rbm_precision(a, precision))) return st;
        if (!theta_d || !S_d) return fail(OTVMC_ERR_INVALID, "RBM build needs theta_d and S_d");
        Carver c(work_d, work_bytes);
        EvalBufs b = carve_eval_bufs(c, a, ntraj, ns);
        char* ws = c.take<char>(rbm_build_bytes(a, ntraj, ns));
        if (!c.ok()) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
        cudaStream_t s = (cudaStream_t)stream;
        CK(launch_vpart(ntraj, ns, (const double2*)v_d, b, s), "vpart launch");
        CK(launch_vquant(ntraj, ns, (const double2*)v_d, b, s), "vquant launch");
        CK(launch_rbm_build(a, (const double2*)theta_d, spins_d, (const double2*)v_d, b.vinfo, ntraj, ns, ws,
                            (double2*)S_d, (double2*)obar_d, (double2*)D_d, s),
           "rbm build launch");
        return OTVMC_OK;
    }
    if (a->kind == OTVMC_LJ) {
        if (precision != OTVMC_PREC_FP64 && precision != OTVMC_PREC_MIXED)
            return fail(OTVMC_ERR_INVALID, "unknown precision");
        if (!S_d) return fail(OTVMC_ERR_INVALID, "tied Jastrow build needs S_d (FP64 at either precision)");
        Carver c(work_d, work_bytes);
        c.take<double2>((size_t)ntraj * a->full->P);  // same layout as the other stages
        EvalBufs b = carve_eval_bufs(c, a->full, ntraj, ns);
        char* ws = c.take<char>(lj_build_bytes(a, ntraj, ns));
        double* obar = obar_d ? obar_d : c.take<double>((size_t)ntraj * a->P);
        if (!c.ok()) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
        cudaStream_t s = (cudaStream_t)stream;
        CK(launch_vpart(ntraj, ns, (const double2*)v_d, b, s), "vpart launch");
        CK(launch_vquant(ntraj, ns, (const double2*)v_d, b, s), "vquant launch");
        CK(launch_lj_build(a, spins_d, ntraj, ns, b, ws, S_d, obar, (double2*)D_d, s), "tied build launch");
        return OTVMC_OK;
    }
    if (precision == OTVMC_PREC_FP64 && !S_d) return fail(OTVMC_ERR_INVALID, "FP64 build needs S_d");
    if (precision == OTVMC_PREC_MIXED) {
        if (!G_d) return fail(OTVMC_ERR_INVALID, "mixed build needs G_d");
        if (ns % 8 != 0 || ns >= (1 << 24))
            return fail(OTVMC_ERR_INVALID, "mixed build needs ns % 8 == 0 and ns < 2^24");
    } else if (precision != OTVMC_PREC_FP64) {
        return fail(OTVMC_ERR_INVALID, "unknown precision");
    }
    Carver c(work_d, work_bytes);
    EvalBufs b = carve_eval_bufs(c, a, ntraj, ns);
    void* obuf = c.take<char>(obuf_bytes(a, ntraj, ns, precision));
    double* obar = obar_d ? obar_d : c.take<double>((size_t)ntraj * a->P);
    if (!c.ok()) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
    return run_build(a, spins_d, (const double2*)v_d, ntraj, ns, precision, false, b, obuf, S_d, G_d, obar,
                     (double2*)D_d, (int*)work_d, (cudaStream_t)stream);
}

otvmc_status otvmc_solve_step(const otvmc_ansatz* a, int ntraj, int ns, int precision, int reg, double eps,
                              double snr_thresh, const double* S_d, const float* G_d, const double* obar_d,
                              const double* D_d, double* delta_d, double* shift_used_d, void* work_d,
                              size_t work_bytes, void* stream) {
    (void)snr_thresh;
    otvmc_status st = check_batch(a, ntraj, ns);
    if (st) return st;
    if (reg != OTVMC_REG_SHIFT)
        return fail(OTVMC_ERR_UNSUPPORTED, "solve_step takes the diagonal shift; the SNR filter needs the samples: "
                                           "use otvmc_solve_snr");
    if (!D_d || !delta_d || !work_d || !(eps >= 0.0)) return fail(OTVMC_ERR_INVALID, "solve_step: bad arguments");
    if (a->kind == OTVMC_RBM) {
        if ((st = rbm_precision(a, precision))) return st;
        if (!S_d) return fail(OTVMC_ERR_INVALID, "RBM solve needs the complex S_d");
        if (work_bytes < 256 + rbm_solve_bytes(ntraj, (int)a->P)) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
        CK(launch_rbm_solve_S(a, ntraj, ns, eps, (const double2*)S_d, (const double2*)D_d, (double2*)delta_d,
                              shift_used_d, (char*)work_d + 256, (int*)work_d, (cudaStream_t)stream),
           "rbm solve launch");
        return OTVMC_OK;
    }
    if (a->kind == OTVMC_LJ) {
        // S of the tied parameters is built in FP64 at either precision: FP64 Cholesky
        if (!S_d) return fail(OTVMC_ERR_INVALID, "tied Jastrow solve needs S_d");
        precision = OTVMC_PREC_FP64;
    }
    if (precision == OTVMC_PREC_FP64 && !S_d) return fail(OTVMC_ERR_INVALID, "FP64 solve needs S_d");
    if (precision == OTVMC_PREC_MIXED && (!G_d || !obar_d))
        return fail(OTVMC_ERR_INVALID, "mixed solve needs G_d and obar_d");
    if (work_bytes < 256 + chol_ws_bytes(ntraj, (int)a->P, precision))
        return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
    CK(launch_chol_solve(ntraj, (int)a->P, ns, precision, eps, S_d, G_d, obar_d, (const double2*)D_d,
                         (double2*)delta_d, shift_used_d, (char*)work_d + 256, 1, (int*)work_d, (cudaStream_t)stream),
       "solve launch");
    return OTVMC_OK;
}

otvmc_status otvmc_solve_snr(const otvmc_ansatz* a, int ntraj, int ns, const double* S_d, const double* obar_d,
                             const uint64_t* spins_d, const double* v_d, const double* D_d, double snr_thresh,
                             double eps_svd, double* delta_d, double* lambda_d, void* work_d, size_t work_bytes,
                             void* stream) {
    otvmc_status st = check_batch(a, ntraj, ns);
    if (st) return st;
    if (a->kind == OTVMC_RBM) return fail(OTVMC_ERR_UNSUPPORTED, "solve_snr: built for the Jastrow ansaetze");
    if (!snr_big_fits((int)a->P))
        return fail(OTVMC_ERR_UNSUPPORTED, "solve_snr: P beyond the shared memory of one CTA");
    if (!S_d || !obar_d || !spins_d || !v_d || !D_d || !delta_d || !work_d || !(snr_thresh >= 0.0) ||
        !(eps_svd >= 0.0))
        return fail(OTVMC_ERR_INVALID, "solve_snr: bad arguments");
    if (work_bytes < otvmc_snr_workspace_bytes(a, ntraj)) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
    if (a->P > SNR_PMAX)
        CK(launch_snr_big(a, ntraj, ns, spins_d, S_d, obar_d, (const double2*)v_d, (const double2*)D_d, snr_thresh,
                          eps_svd, (double2*)delta_d, lambda_d, (char*)work_d + 256, (int*)work_d,
                          (cudaStream_t)stream),
           "snr solve launch");
    else
        CK(launch_snr_solve(a, ntraj, ns, spins_d, S_d, obar_d, (const double2*)v_d, (const double2*)D_d, snr_thresh,
                            eps_svd, (double2*)delta_d, lambda_d, (int*)work_d, (cudaStream_t)stream),
           "snr solve launch");
    return OTVMC_OK;
}

size_t otvmc_snr_workspace_bytes(const otvmc_ansatz* a, int ntraj) {
    if (!a || ntraj < 1) return 0;
    return a->P > SNR_PMAX ? 256 + snr_big_ws_bytes(ntraj, (int)a->P) : 256;
}

otvmc_status otvmc_sde_combine(int ntraj, int64_t P, int scheme, int stage, const double* theta_d,
                               const double* delta0_d, const double* delta1_d, double* out_d, int* failed_d,
                               void* work_d, size_t work_bytes, void* stream) {
    if (ntraj < 1 || P < 1 || !theta_d || !delta0_d || !out_d || !work_d || work_bytes < 256 ||
        (scheme != OTVMC_HEUN && scheme != OTVMC_MIDPOINT) || (stage != 0 && stage != 1) ||
        (stage == 1 && scheme == OTVMC_HEUN && !delta1_d) || (stage == 1 && scheme == OTVMC_MIDPOINT && !delta1_d))
        return fail(OTVMC_ERR_INVALID, "sde_combine: bad arguments");
    CK(launch_sde(ntraj, P, scheme, stage, (const double2*)theta_d, (const double2*)delta0_d,
                  (const double2*)delta1_d, (double2*)out_d, failed_d, (int*)work_d, (cudaStream_t)stream),
       "sde launch");
    return OTVMC_OK;
}

otvmc_status otvmc_observables(const otvmc_ansatz* a, const double* theta_d, const uint64_t* spins_d, int ntraj,
                               int ns, int precision, double* moments_d, void* work_d, size_t work_bytes,
                               void* stream) {
    otvmc_status st = check_batch(a, ntraj, ns);
    if (st) return st;
    if (!theta_d || !spins_d || !moments_d || !work_d) return fail(OTVMC_ERR_INVALID, "observables: bad arguments");
    Carver c(work_d, work_bytes);
    double2* thf = a->kind == OTVMC_LJ ? c.take<double2>((size_t)ntraj * a->full->P) : nullptr;
    const otvmc_ansatz* e = eval_ansatz(a);
    EvalBufs b = carve_eval_bufs(c, e, ntraj, ns);
    double* lpl = c.take<double>((size_t)ntraj * (a->model->nops + 1));
    if (!c.ok()) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    const bool fp32 = precision == OTVMC_PREC_MIXED;
    if ((st = rbm_precision(a, precision))) return st;
    const double2* th = (const double2*)theta_d;
    if (thf) {
        CK(launch_lj_expand(a, ntraj, th, thf, s), "expand launch");
        th = thf;
    }
    st = run_estimators(e, th, spins_d, ntraj, ns, nullptr, 0.0, fp32, b, lpl, nullptr, nullptr, (int*)work_d, s);
    if (st) return st;
    if (a->kind == OTVMC_RBM) {
        CK(launch_obs_rbm(a, th, spins_d, ntraj, ns, fp32, b, s), "observables launch");
        CK(launch_obs_final(a->n, ns, ntraj, b, moments_d, s), "observables launch");
        return OTVMC_OK;
    }
    CK(launch_obs_prep(e, th, ntraj, fp32, b, s), "obs prep launch");
    CK(launch_observables(e, spins_d, ntraj, ns, fp32, b, moments_d, (int*)work_d, s), "observables launch");
    return OTVMC_OK;
}

otvmc_status otvmc_ensemble(const double* mom, int ntraj, int n_sites, double* M_h, double* C_h, double* xi2_h,
                            double* dM_h) {
    if (!mom || ntraj < 1 || n_sites < 1) return fail(OTVMC_ERR_INVALID, "ensemble: bad arguments");
    double M[3] = {0, 0, 0}, Q[6] = {0, 0, 0, 0, 0, 0};
    for (int t = 0; t < ntraj; ++t) {
        for (int a = 0; a < 3; ++a) M[a] += mom[t * 9 + a];
        for (int a = 0; a < 6; ++a) Q[a] += mom[t * 9 + 3 + a];
    }
    for (int a = 0; a < 3; ++a) M[a] /= ntraj;
    for (int a = 0; a < 6; ++a) Q[a] /= ntraj;
    // q order: xx yy zz xy xz yz
    double C[3][3];
    C[0][0] = Q[0] - M[0] * M[0];
    C[1][1] = Q[1] - M[1] * M[1];
    C[2][2] = Q[2] - M[2] * M[2];
    C[0][1] = C[1][0] = Q[3] - M[0] * M[1];
    C[0][2] = C[2][0] = Q[4] - M[0] * M[2];
    C[1][2] = C[2][1] = Q[5] - M[1] * M[2];
    if (M_h)
        for (int a = 0; a < 3; ++a) M_h[a] = M[a];
    if (C_h)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) C_h[a * 3 + b] = C[a][b];
    if (dM_h) {
        for (int a = 0; a < 3; ++a) {
            double s2 = 0.0;
            for (int t = 0; t < ntraj; ++t) {
                const double d = mom[t * 9 + a] - M[a];
                s2 += d * d;
            }
            dM_h[a] = ntraj > 1 ? std::sqrt(s2 / (ntraj - 1) / ntraj) : 0.0;
        }
    }
    if (xi2_h) {
        const double nrm = std::sqrt(M[0] * M[0] + M[1] * M[1] + M[2] * M[2]);
        if (!(nrm > 0.0)) {
            *xi2_h = NAN;
        } else {
            const double u[3] = {M[0] / nrm, M[1] / nrm, M[2] / nrm};
            int amin = 0;
            for (int a = 1; a < 3; ++a)
                if (std::fabs(u[a]) < std::fabs(u[amin])) amin = a;
            double e1[3] = {0, 0, 0};
            e1[amin] = 1.0;
            const double dot = e1[0] * u[0] + e1[1] * u[1] + e1[2] * u[2];
            for (int a = 0; a < 3; ++a) e1[a] -= dot * u[a];
            const double n1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
            for (int a = 0; a < 3; ++a) e1[a] /= n1;
            const double e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
            auto quad = [&](const double* x, const double* y) {
                double s = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) s += x[a] * C[a][b] * y[b];
                return s;
            };
            const double a11 = quad(e1, e1), a22 = quad(e2, e2), a12 = quad(e1, e2);
            const double lmin = 0.5 * (a11 + a22) - std::sqrt(0.25 * (a11 - a22) * (a11 - a22) + a12 * a12);
            *xi2_h = n_sites * lmin / (nrm * nrm);
        }
    }
    return OTVMC_OK;
}

// ------------------------------------------------------------------------ trajectories
struct RunBufs {
    double2* theta_c;
    double2* d0;
    double2* d1;
    double* dW;
    double* lpl;
    double2* Eeff;
    double2* v;
    double* obar;
    double2* D;
    double* S;
    float* G;
    void* obuf;
    void* chol;
    double2* gam;  // RBM sampler scratch
    double* lcr;
    float4* tab;   // RBM flip table of the FP32 sampler
    void* rbm;     // RBM build scratch
    void* snr;     // SNR filter beyond the shared-memory size: the eigen-decomposition's matrices
    double2* thf;  // tied Jastrow: the expanded parameters of the full Jastrow
    double* lpl0;  // linear SSE: zeros in place of <L + L^+> in E_eff
    double* gq;    // linear SSE: the predictor's increment of ln Q
    EvalBufs eb;
};

// Linear SSE (App. B): ln Q per trajectory (in/out) and its values at the measured rows.
struct LinState {
    double* lnQ;
    double* rows;
};

static RunBufs carve_run(Carver& c, const otvmc_ansatz* a, const otvmc_run_desc* d) {
    const int T = d->ntraj, ns = d->ns;
    const size_t P = (size_t)a->P;
    RunBufs r;
    r.thf = a->kind == OTVMC_LJ ? c.take<double2>((size_t)T * a->full->P) : nullptr;
    r.eb = carve_eval_bufs(c, a->kind == OTVMC_LJ ? a->full : a, T, ns);
    r.theta_c = c.take<double2>(T * P);
    r.d0 = c.take<double2>(T * P);
    r.d1 = c.take<double2>(T * P);
    r.dW = c.take<double>((size_t)T * (a->model->nops + 1));
    r.lpl = c.take<double>((size_t)T * (a->model->nops + 1));
    r.lpl0 = c.take<double>((size_t)T * (a->model->nops + 1));
    r.gq = c.take<double>((size_t)T);
    r.Eeff = c.take<double2>((size_t)T * ns);
    r.v = c.take<double2>((size_t)T * ns);
    r.obar = c.take<double>(T * P);
    r.D = c.take<double2>(T * P);
    r.gam = nullptr;
    r.lcr = nullptr;
    r.tab = nullptr;
    r.rbm = nullptr;
    r.snr = (d->reg == OTVMC_REG_SNR && a->P > SNR_PMAX) ? c.take<char>(snr_big_ws_bytes(T, (int)P)) : nullptr;
    if (a->kind == OTVMC_RBM) {
        r.S = nullptr;
        r.G = nullptr;
        r.obuf = nullptr;
        r.gam = c.take<double2>((size_t)T * a->m * ns);
        r.lcr = c.take<double>((size_t)T * a->m * ns);
        r.tab = (float4*)c.take<char>(rbm_tab_bytes(a, T));
        if (d->precision == OTVMC_PREC_MIXED) {
            r.rbm = c.take<char>(rbm_mixed_bytes(a, T, ns));
            r.chol = nullptr;
        } else {
            r.rbm = c.take<char>(rbm_build_bytes(a, T, ns));
            r.chol = c.take<char>(chol_ws_bytes(T, 2 * (int)(P <= (size_t)ns ? P : (size_t)ns), OTVMC_PREC_FP64));
        }
        return r;
    }
    if (a->kind == OTVMC_LJ) {
        // S of the tied parameters in FP64 from exact integer counts, FP64 Cholesky
        r.S = c.take<double>(T * P * P);
        r.G = nullptr;
        r.obuf = c.take<char>(lj_build_bytes(a, T, ns));
        r.chol = c.take<char>(chol_ws_bytes(T, (int)P, OTVMC_PREC_FP64));
        return r;
    }
    if (d->precision == OTVMC_PREC_FP64) {
        r.S = c.take<double>(T * P * P);
        r.G = nullptr;
    } else {
        // the SNR filter works on the full FP64 S, expanded from the exact counts
        r.S = d->reg == OTVMC_REG_SNR ? c.take<double>(T * P * P) : nullptr;
        r.G = c.take<float>(T * P * P);
    }
    r.obuf = c.take<char>(obuf_bytes(a, T, ns, d->precision));
    r.chol = c.take<char>(chol_ws_bytes(T, (int)P, d->precision));
    return r;
}

static otvmc_status check_run(const otvmc_ansatz* a, const otvmc_run_desc* d) {
    otvmc_status st = check_batch(a, d ? d->ntraj : 0, d ? d->ns : 0);
    if (st) return st;
    if (d->n_steps < 0 || d->n_sweep < 0 || !(d->dt > 0.0) || d->traj0 < 0 || d->step0 < 0 ||
        (d->scheme != OTVMC_HEUN && d->scheme != OTVMC_MIDPOINT) || d->measure_every < 0 || !(d->eps >= 0.0))
        return fail(OTVMC_ERR_INVALID, "run: bad descriptor");
    if (d->precision != OTVMC_PREC_FP64 && d->precision != OTVMC_PREC_MIXED)
        return fail(OTVMC_ERR_INVALID, "unknown precision");
    if (d->precision == OTVMC_PREC_MIXED && (d->ns % 8 != 0 || d->ns >= (1 << 24)))
        return fail(OTVMC_ERR_INVALID, "mixed precision needs ns % 8 == 0 and ns < 2^24");
    if (d->reg != OTVMC_REG_SHIFT && d->reg != OTVMC_REG_SNR) return fail(OTVMC_ERR_INVALID, "unknown regulariser");
    if (d->use_graph != 0) return fail(OTVMC_ERR_UNSUPPORTED, "run: use_graph is reserved and must be 0");
    if ((st = rbm_precision(a, d->precision))) return st;
    if (a->kind == OTVMC_RBM && d->reg != OTVMC_REG_SHIFT)
        return fail(OTVMC_ERR_UNSUPPORTED, "the SNR regulariser is built for the Jastrow ansatz");
    if (d->reg == OTVMC_REG_SNR && a->kind != OTVMC_RBM && (!snr_big_fits((int)a->P) || !(d->snr_thresh >= 0.0)))
        return fail(OTVMC_ERR_UNSUPPORTED, "SNR regulariser: needs snr_thresh >= 0 and P within the shared "
                                           "memory of one CTA");
    return OTVMC_OK;
}

int otvmc_run_n_meas(const otvmc_run_desc* d) {
    if (!d) return 0;
    int n = 0;
    if (d->measure_every > 0)
        for (int i = 0; i < d->n_steps; ++i)
            if (i % d->measure_every == 0) ++n;
    if (d->measure_final) ++n;
    return n;
}

// Trajectory pipelines: a batch of at least RUN_PIPE_MIN trajectories runs as RUN_PIPES
// contiguous sub-batches, each advanced through all its steps on a stream of its own forked
// from the caller's, so that the sub-batches' launches overlap one another's tails and
// gaps (the sub-batches start together; a start staggered by one evaluation's sampling and
// Gram phase measured slower on the 64-spin benchmark).  Trajectories are independent
// and every random draw is keyed by the global trajectory id, so the split leaves every
// result unchanged.  Each sub-batch carves its own region of the workspace; all share the
// status word at its head.
constexpr int RUN_PIPES = 2;
constexpr int RUN_PIPE_MIN = 32;
constexpr int RUN_MAX_PIPES = 4;      // the most sub-batches a launch-shape setting may ask for
constexpr int RUN_PIPE_MIN_SIZE = 8;  // ... each of at least this many trajectories

// Launch shape of a run: sub-batches on forked streams, and trajectory groups of the mixed
// solver inside each (0: the solver's own rule).  Neither changes any result (trajectories are
// independent and every draw is keyed by the global trajectory id).  otvmc_autotune_run times
// the candidates on a batch and records the fastest per batch shape; runs of that shape use it.
struct LaunchShape {
    int pipes;
    int groups;
};
struct TuneKey {
    int kind, n, m, P, ns, ntraj, precision, reg;
    bool operator<(const TuneKey& o) const {
        const int a[8] = {kind, n, m, P, ns, ntraj, precision, reg};
        const int b[8] = {o.kind, o.n, o.m, o.P, o.ns, o.ntraj, o.precision, o.reg};
        for (int i = 0; i < 8; ++i)
            if (a[i] != b[i]) return a[i] < b[i];
        return false;
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, LaunchShape> g_tune;
static TuneKey tune_key(const otvmc_ansatz* a, const otvmc_run_desc* d) {
    return TuneKey{a->kind, a->n, a->m, (int)a->P, d->ns, d->ntraj, d->precision, d->reg};
}

// (Jastrow only by default: with the RBM's T path the solve of size 2 ns dominates, and
// sub-batches whose solves compete measured slower.)
static LaunchShape default_shape(const otvmc_ansatz* a, const otvmc_run_desc* d) {
    return LaunchShape{a->kind == OTVMC_JASTROW && d->ntraj >= RUN_PIPE_MIN ? RUN_PIPES : 1, 0};
}
static LaunchShape run_shape(const otvmc_ansatz* a, const otvmc_run_desc* d) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(a, d));
    return it != g_tune.end() ? it->second : default_shape(a, d);
}
// sub-batch counts a run of this batch may use (the workspace is sized for the largest need)
static int pipe_candidates(const otvmc_run_desc* d, int* out) {
    int n = 0;
    for (int np = 1; np <= RUN_MAX_PIPES; np *= 2)
        if (np == 1 || d->ntraj >= np * RUN_PIPE_MIN_SIZE) out[n++] = np;
    return n;
}

// Sub-batch p of np: its descriptor and the offset of its first trajectory in the batch.
static otvmc_run_desc pipe_desc(const otvmc_run_desc* d, int p, int np, int* first) {
    const int ta = (int)((long long)d->ntraj * p / np), tb = (int)((long long)d->ntraj * (p + 1) / np);
    otvmc_run_desc q = *d;
    q.ntraj = tb - ta;
    q.traj0 = d->traj0 + ta;
    *first = ta;
    return q;
}

// Workspace bytes of one sub-batch (256-byte head included, rounded to 256).
static size_t pipe_bytes(const otvmc_ansatz* a, const otvmc_run_desc* q) {
    Carver c(nullptr, (size_t)-1);
    carve_run(c, a, q);
    return (c.off + 255) & ~(size_t)255;
}

struct PipeStreams {
    cudaStream_t s[RUN_MAX_PIPES];
    cudaEvent_t fork;
    cudaEvent_t join[RUN_MAX_PIPES];
};
// One set per (device, calling stream), created on first use.
static PipeStreams& pipe_streams(cudaStream_t caller) {
    static std::mutex mu;
    static std::map<std::pair<int, uintptr_t>, PipeStreams> sets;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, (uintptr_t)caller);
    auto it = sets.find(key);
    if (it != sets.end()) return it->second;
    PipeStreams& g = sets[key];
    for (int i = 0; i < RUN_MAX_PIPES; ++i) {
        cudaStreamCreateWithFlags(&g.s[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&g.join[i], cudaEventDisableTiming);
    }
    cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming);
    return g;
}

static size_t run_bytes_pipes(const otvmc_ansatz* a, const otvmc_run_desc* d, int np) {
    size_t total = 0;
    for (int p = 0; p < np; ++p) {
        int first = 0;
        const otvmc_run_desc q = pipe_desc(d, p, np, &first);
        total += pipe_bytes(a, &q);
    }
    return total + 256;
}

// The largest need over the launch shapes a run of this batch may take (a shape recorded by
// the autotuner later must fit a workspace sized now).
size_t otvmc_run_workspace_bytes(const otvmc_ansatz* a, const otvmc_run_desc* d) {
    if (check_run(a, d)) return 0;
    int cand[4];
    const int nc = pipe_candidates(d, cand);
    size_t best = 0;
    for (int i = 0; i < nc; ++i) best = std::max(best, run_bytes_pipes(a, d, cand[i]));
    return best;
}

// One evaluation at theta (eval index ev): sample, estimators, [observables], S/D, solve.
static otvmc_status run_eval(const otvmc_ansatz* a, const otvmc_run_desc* d, const RunBufs& r, const double2* theta,
                             uint64_t* spins, int64_t ev, double* moments_row, double2* delta, int* status,
                             cudaStream_t s, const LinState* lin) {
    const int T = d->ntraj, ns = d->ns;
    const bool fp32 = d->precision == OTVMC_PREC_MIXED;
    const double* lpl_e = lin ? r.lpl0 : nullptr;
    const int stage = (int)(ev & 1);
    if (a->kind == OTVMC_RBM) {
        CK(sample_rbm_any(a, theta, T, d->traj0, ns, d->n_sweep, d->seed, ev, spins, r.gam, r.lcr, r.tab, nullptr, s),
           "sample launch");
        otvmc_status st =
            run_estimators(a, theta, spins, T, ns, r.dW, d->dt, fp32, r.eb, r.lpl, r.Eeff, r.v, status, s, lpl_e);
        if (st) return st;
        if (moments_row) {
            CK(launch_obs_rbm(a, theta, spins, T, ns, fp32, r.eb, s), "observables launch");
            CK(launch_obs_final(a->n, ns, T, r.eb, moments_row, s), "observables launch");
        }
        CK(launch_vquant(T, ns, r.v, r.eb, s), "vquant launch");
        if (lin) CK(launch_lnq(T, d->scheme, stage, r.eb.vinfo, r.gq, lin->lnQ, s), "lnq launch");
        if (fp32)
            CK(launch_rbm_build_solve_mixed(a, theta, spins, r.v, r.eb.vinfo, T, ns, d->eps, r.rbm, delta, status, s),
               "rbm build/solve launch");
        else
            CK(launch_rbm_build_solve(a, theta, spins, r.v, r.eb.vinfo, T, ns, d->eps, r.rbm, r.chol, delta, status,
                                      s),
               "rbm build/solve launch");
        return OTVMC_OK;
    }
    // the tied Jastrow samples, estimates and measures through the full Jastrow's kernels
    const otvmc_ansatz* e = eval_ansatz(a);
    const double2* th = theta;
    if (a->kind == OTVMC_LJ) {
        CK(launch_lj_expand(a, T, theta, r.thf, s), "expand launch");
        th = r.thf;
    }
    CK(launch_sample_jastrow(e, th, T, d->traj0, ns, d->n_sweep, d->seed, ev, spins, nullptr, status, s),
       "sample launch");
    otvmc_status st =
        run_estimators(e, th, spins, T, ns, r.dW, d->dt, fp32, r.eb, r.lpl, r.Eeff, r.v, status, s, lpl_e);
    if (st) return st;
    if (moments_row) {
        CK(launch_obs_prep(e, th, T, fp32, r.eb, s), "obs prep launch");
        CK(launch_observables(e, spins, T, ns, fp32, r.eb, moments_row, status, s), "observables launch");
    }
    if (a->kind == OTVMC_LJ) {
        CK(launch_vquant(T, ns, r.v, r.eb, s), "vquant launch");
        CK(launch_lj_build(a, spins, T, ns, r.eb, r.obuf, r.S, r.obar, r.D, s), "tied build launch");
    } else {
        st = run_build(a, spins, r.v, T, ns, d->precision, true, r.eb, r.obuf, r.S, r.G, r.obar, r.D, status, s);
        if (st) return st;
    }
    if (lin) CK(launch_lnq(T, d->scheme, stage, r.eb.vinfo, r.gq, lin->lnQ, s), "lnq launch");
    if (d->reg == OTVMC_REG_SNR) {
        if (a->P > SNR_PMAX)
            CK(launch_snr_big(a, T, ns, spins, r.S, r.obar, r.v, r.D, d->snr_thresh, SNR_EPS_SVD, delta, nullptr,
                              r.snr, status, s, d->precision == OTVMC_PREC_MIXED,
                              a->kind == OTVMC_LJ ? lj_built_O(a, T, r.obuf) : nullptr),
               "snr solve launch");
        else
            CK(launch_snr_solve(a, T, ns, spins, r.S, r.obar, r.v, r.D, d->snr_thresh, SNR_EPS_SVD, delta, nullptr,
                                status, s),
               "snr solve launch");
        return OTVMC_OK;
    }
    CK(launch_chol_solve(T, (int)a->P, ns, a->kind == OTVMC_LJ ? OTVMC_PREC_FP64 : d->precision, d->eps, r.S, r.G,
                         r.obar, r.D, delta, nullptr, r.chol, 1, status, s),
       "solve launch");
    return OTVMC_OK;
}

// All steps of one (sub-)batch on stream s; moments rows hold mstride trajectories, of which
// this batch's come first in moments_d.
static otvmc_status run_steps(const otvmc_ansatz* a, const otvmc_run_desc* d, double* theta_d, uint64_t* spins_d,
                              double* moments_d, int mstride, void* work_d, size_t work_bytes, int* status,
                              cudaStream_t s, const LinState* lin) {
    Carver c(work_d, work_bytes);
    RunBufs r = carve_run(c, a, d);
    if (!c.ok()) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
    if (lin)
        CK(cudaMemsetAsync(r.lpl0, 0, sizeof(double) * (size_t)d->ntraj * (a->model->nops + 1), s), "memset");
    // ln Q at a measured row (the value at the time of that row's samples)
    auto lnq_row = [&](int row) -> cudaError_t {
        if (!lin || !lin->rows) return cudaSuccess;
        return cudaMemcpyAsync(lin->rows + (size_t)row * mstride, lin->lnQ, sizeof(double) * d->ntraj,
                               cudaMemcpyDeviceToDevice, s);
    };
    const int T = d->ntraj;
    const int64_t P = a->P;
    double2* theta = (double2*)theta_d;
    int row = 0;
    for (int i = 0; i < d->n_steps; ++i) {
        const int64_t step = d->step0 + i;
        CK(launch_noise(a->model, T, d->traj0, d->seed, step, d->dt, r.dW, s), "noise launch");
        double* mrow = nullptr;
        if (d->measure_every > 0 && i % d->measure_every == 0 && moments_d) {
            CK(lnq_row(row), "lnq row copy");
            mrow = moments_d + (size_t)(row++) * mstride * OTVMC_MOMENTS;
        }
        otvmc_status st = run_eval(a, d, r, theta, spins_d, 2 * step, mrow, r.d0, status, s, lin);
        if (st) return st;
        CK(launch_sde(T, P, d->scheme, 0, theta, r.d0, nullptr, r.theta_c, nullptr, status, s), "sde launch");
        st = run_eval(a, d, r, r.theta_c, spins_d, 2 * step + 1, nullptr, r.d1, status, s, lin);
        if (st) return st;
        CK(launch_sde(T, P, d->scheme, 1, theta, r.d0, r.d1, theta, nullptr, status, s), "sde launch");
    }
    if (d->measure_final && moments_d) {
        const int64_t ev = 2 * (d->step0 + d->n_steps);
        const bool rbm = a->kind == OTVMC_RBM;
        if (rbm)
            CK(sample_rbm_any(a, theta, T, d->traj0, d->ns, d->n_sweep, d->seed, ev, spins_d, r.gam, r.lcr, r.tab, nullptr,
                                 s),
               "sample launch");
        const otvmc_ansatz* e = eval_ansatz(a);
        const double2* th = theta;
        if (a->kind == OTVMC_LJ) {
            CK(launch_lj_expand(a, T, theta, r.thf, s), "expand launch");
            th = r.thf;
        }
        if (!rbm)
            CK(launch_sample_jastrow(e, th, T, d->traj0, d->ns, d->n_sweep, d->seed, ev, spins_d, nullptr, status, s),
               "sample launch");
        const bool fp32 = d->precision == OTVMC_PREC_MIXED;
        otvmc_status st = run_estimators(e, th, spins_d, T, d->ns, nullptr, 0.0, fp32, r.eb, r.lpl, nullptr, nullptr,
                                         status, s);
        if (st) return st;
        CK(lnq_row(row), "lnq row copy");
        double* mrow = moments_d + (size_t)row * mstride * OTVMC_MOMENTS;
        if (rbm) {
            CK(launch_obs_rbm(a, theta, spins_d, T, d->ns, fp32, r.eb, s), "observables launch");
            CK(launch_obs_final(a->n, d->ns, T, r.eb, mrow, s), "observables launch");
        } else {
            CK(launch_obs_prep(e, th, T, fp32, r.eb, s), "obs prep launch");
            CK(launch_observables(e, spins_d, T, d->ns, fp32, r.eb, mrow, status, s), "observables launch");
        }
    }
    return OTVMC_OK;
}

// The batch as sub-batches on forked streams (one after another on s under serial profiling).
// Restores the issuing thread's solver-group setting when a run's launches have been issued.
struct GroupSetting {
    int old;
    explicit GroupSetting(int g) : old(chol_set_groups(g)) {}
    ~GroupSetting() { chol_set_groups(old); }
};

static otvmc_status run_pipelined_shape(const otvmc_ansatz* a, const otvmc_run_desc* d, double* theta_d,
                                        uint64_t* spins_d, double* moments_d, void* work_d, size_t work_bytes,
                                        cudaStream_t s, const LinState* lin, LaunchShape shape) {
    int* status = (int*)work_d;
    const int np = shape.pipes;
    const GroupSetting gs_(shape.groups);
    if (np == 1) return run_steps(a, d, theta_d, spins_d, moments_d, d->ntraj, work_d, work_bytes, status, s, lin);
    const bool forked = !profiling_serial();
    PipeStreams& ps = pipe_streams(s);
    if (forked) CK(cudaEventRecord(ps.fork, s), "pipeline fork");
    const size_t W = (size_t)((a->n + 63) / 64);
    char* w = (char*)work_d;
    size_t left = work_bytes;
    for (int p = 0; p < np; ++p) {
        int first = 0;
        const otvmc_run_desc q = pipe_desc(d, p, np, &first);
        const size_t need = pipe_bytes(a, &q);
        if (need > left) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
        cudaStream_t sp = forked ? ps.s[p] : s;
        if (forked) CK(cudaStreamWaitEvent(sp, ps.fork, 0), "pipeline fork");
        LinState lp{};
        if (lin) lp = LinState{lin->lnQ + first, lin->rows ? lin->rows + first : nullptr};
        otvmc_status st = run_steps(a, &q, theta_d + (size_t)first * a->P * 2, spins_d + (size_t)first * d->ns * W,
                                    moments_d ? moments_d + (size_t)first * OTVMC_MOMENTS : nullptr, d->ntraj, w, need,
                                    status, sp, lin ? &lp : nullptr);
        if (forked) {
            // joined also after an error, so that the caller's stream stays ordered after it
            CK(cudaEventRecord(ps.join[p], sp), "pipeline join");
            CK(cudaStreamWaitEvent(s, ps.join[p], 0), "pipeline join");
        }
        if (st) return st;
        w += need;
        left -= need;
    }
    return OTVMC_OK;
}

static otvmc_status run_pipelined(const otvmc_ansatz* a, const otvmc_run_desc* d, double* theta_d, uint64_t* spins_d,
                                  double* moments_d, void* work_d, size_t work_bytes, cudaStream_t s,
                                  const LinState* lin = nullptr) {
    return run_pipelined_shape(a, d, theta_d, spins_d, moments_d, work_d, work_bytes, s, lin, run_shape(a, d));
}

otvmc_status otvmc_run_trajectories(const otvmc_ansatz* a, const otvmc_run_desc* d, double* theta_d,
                                    uint64_t* spins_d, double* moments_d, void* work_d, size_t work_bytes,
                                    void* stream) {
    otvmc_status st = check_run(a, d);
    if (st) return st;
    if (!theta_d || !spins_d || !work_d) return fail(OTVMC_ERR_INVALID, "run: null buffer");
    if (otvmc_run_n_meas(d) > 0 && !moments_d) return fail(OTVMC_ERR_INVALID, "run: moments_d needed");
    cudaStream_t s = (cudaStream_t)stream;
    st = run_pipelined(a, d, theta_d, spins_d, moments_d, work_d, work_bytes, s);
    if (st) return st;
    return otvmc_check(work_d, stream);
}

// Grouped runs: up to OTVMC_MAX_GROUPS batches of one ansatz with their own descriptors, each on
// its own forked stream (one set per (device, calling stream)).  Streams take priorities by the
// groups' sample counts: the group with the most samples per trajectory, whose step is the
// longest chain of dependent launches, gets the highest priority, so that the others' launches
// fill the GPU around it rather than delay it.
struct GroupRunStreams {
    cudaStream_t s[OTVMC_MAX_GROUPS];
    cudaEvent_t fork;
    cudaEvent_t join[OTVMC_MAX_GROUPS];
};
static GroupRunStreams& group_run_streams(cudaStream_t caller) {
    static std::mutex mu;
    static std::map<std::pair<int, uintptr_t>, GroupRunStreams> sets;
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0;
    cudaGetDevice(&dev);
    auto key = std::make_pair(dev, (uintptr_t)caller);
    auto it = sets.find(key);
    if (it != sets.end()) return it->second;
    GroupRunStreams& g = sets[key];
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int i = 0; i < OTVMC_MAX_GROUPS; ++i) {
        // rank i (0 = most samples) gets priority greatest + i, clamped to the range
        const int pr = std::min(least, greatest + i);
        cudaStreamCreateWithPriority(&g.s[i], cudaStreamNonBlocking, pr);
        cudaEventCreateWithFlags(&g.join[i], cudaEventDisableTiming);
    }
    cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming);
    return g;
}

static size_t group_slice(size_t b) { return (b + 255) & ~(size_t)255; }

size_t otvmc_run_grouped_workspace_bytes(const otvmc_ansatz* a, const otvmc_run_desc* descs, int ngroups) {
    if (!a || !descs || ngroups < 1 || ngroups > OTVMC_MAX_GROUPS) return 0;
    size_t total = 0;
    for (int g = 0; g < ngroups; ++g) {
        const size_t b = otvmc_run_workspace_bytes(a, &descs[g]);
        if (!b) return 0;
        total += group_slice(b);
    }
    return total;
}

otvmc_status otvmc_run_trajectories_grouped(const otvmc_ansatz* a, const otvmc_run_desc* descs, int ngroups,
                                            double* const* theta_d, uint64_t* const* spins_d,
                                            double* const* moments_d, void* work_d, size_t work_bytes,
                                            void* stream) {
    if (!a || !descs || !theta_d || !spins_d || !work_d || ngroups < 1 || ngroups > OTVMC_MAX_GROUPS)
        return fail(OTVMC_ERR_INVALID, "run_grouped: bad arguments");
    size_t off[OTVMC_MAX_GROUPS], need[OTVMC_MAX_GROUPS], total = 0;
    for (int g = 0; g < ngroups; ++g) {
        otvmc_status st = check_run(a, &descs[g]);
        if (st) return st;
        if (!theta_d[g] || !spins_d[g]) return fail(OTVMC_ERR_INVALID, "run_grouped: null buffer");
        if (otvmc_run_n_meas(&descs[g]) > 0 && (!moments_d || !moments_d[g]))
            return fail(OTVMC_ERR_INVALID, "run_grouped: moments_d needed");
        need[g] = otvmc_run_workspace_bytes(a, &descs[g]);
        off[g] = total;
        total += group_slice(need[g]);
    }
    if (total > work_bytes) return fail(OTVMC_ERR_WORKSPACE, "run_grouped: workspace too small");
    // rank of each group by sample count (ties by position): rank 0 runs at the highest priority
    int rank[OTVMC_MAX_GROUPS];
    for (int g = 0; g < ngroups; ++g) {
        rank[g] = 0;
        for (int h = 0; h < ngroups; ++h)
            if (descs[h].ns > descs[g].ns || (descs[h].ns == descs[g].ns && h < g)) ++rank[g];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const bool forked = ngroups > 1 && !profiling_serial();
    GroupRunStreams& gs = group_run_streams(s);
    if (forked) CK(cudaEventRecord(gs.fork, s), "grouped fork");
    otvmc_status first_err = OTVMC_OK;
    // launched in rank order: the longest group's first launches go out first
    for (int r = 0; r < ngroups; ++r) {
        int g = 0;
        while (rank[g] != r) ++g;
        char* w = (char*)work_d + off[g];
        cudaStream_t sg = forked ? gs.s[r] : s;
        if (forked) CK(cudaStreamWaitEvent(sg, gs.fork, 0), "grouped fork");
        otvmc_status st = run_pipelined(a, &descs[g], theta_d[g], spins_d[g], moments_d ? moments_d[g] : nullptr, w,
                                        need[g], sg);
        if (forked) {
            CK(cudaEventRecord(gs.join[r], sg), "grouped join");
            CK(cudaStreamWaitEvent(s, gs.join[r], 0), "grouped join");
        }
        if (st && !first_err) first_err = st;
    }
    if (first_err) return first_err;
    // every group's device status lives at the head of its own workspace slice
    for (int g = 0; g < ngroups; ++g) {
        otvmc_status st = otvmc_check((char*)work_d + off[g], stream);
        if (st && !first_err) first_err = st;
    }
    return first_err;
}

// ------------------------------------------------------------------ launch-shape autotuner
// the tuning step: one step with the caller's measurement setting
static otvmc_run_desc tune_desc(const otvmc_run_desc* d) {
    otvmc_run_desc q = *d;
    q.n_steps = 1;
    q.measure_every = d->measure_every > 0 ? 1 : 0;
    return q;
}
static size_t tune_state_bytes(const otvmc_ansatz* a, const otvmc_run_desc* d) {
    const size_t T = (size_t)d->ntraj;
    const otvmc_run_desc q = tune_desc(d);
    return ((T * a->P * 16 + 255) & ~(size_t)255) + ((T * d->ns * ((a->n + 63) / 64) * 8 + 255) & ~(size_t)255) +
           (((size_t)otvmc_run_n_meas(&q) * T * OTVMC_MOMENTS * 8 + 255) & ~(size_t)255);
}

size_t otvmc_autotune_workspace_bytes(const otvmc_ansatz* a, const otvmc_run_desc* d) {
    const size_t b = otvmc_run_workspace_bytes(a, d);
    return b ? ((b + 255) & ~(size_t)255) + tune_state_bytes(a, d) : 0;
}

otvmc_status otvmc_autotune_run(const otvmc_ansatz* a, const otvmc_run_desc* d, const double* theta_d,
                                const uint64_t* spins_d, void* work_d, size_t work_bytes, void* stream,
                                int* pipes_out, int* groups_out, double* ms_out) {
    otvmc_status st = check_run(a, d);
    if (st) return st;
    if (!theta_d || !spins_d || !work_d) return fail(OTVMC_ERR_INVALID, "autotune: null buffer");
    const size_t need = otvmc_autotune_workspace_bytes(a, d);
    if (work_bytes < need) return fail(OTVMC_ERR_WORKSPACE, "autotune: workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    // one step with the caller's measurement setting, from copies of the caller's state (left
    // untouched)
    const otvmc_run_desc q = tune_desc(d);
    const size_t rb = (otvmc_run_workspace_bytes(a, d) + 255) & ~(size_t)255;
    const size_t T = (size_t)d->ntraj, W = (size_t)((a->n + 63) / 64);
    double* th = (double*)((char*)work_d + rb);
    uint64_t* sp = (uint64_t*)((char*)th + ((T * a->P * 16 + 255) & ~(size_t)255));
    double* mo = (double*)((char*)sp + ((T * d->ns * W * 8 + 255) & ~(size_t)255));
    int cand[4];
    const int nc = pipe_candidates(d, cand);
    const bool grouped = a->kind != OTVMC_LJ && d->precision == OTVMC_PREC_MIXED;  // the tensor-core solver
    const int gcand[4] = {0, 1, 2, CHOL_MAX_GROUPS};
    const int ngc = grouped ? 4 : 1;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "autotune event");
    CK(cudaEventCreate(&e1), "autotune event");
    LaunchShape best{1, 0};
    float best_ms = INFINITY;
    for (int i = 0; i < nc && !st; ++i)
        for (int j = 0; j < ngc && !st; ++j) {
            const LaunchShape sh{cand[i], gcand[j]};
            float ms = INFINITY;
            for (int rep = 0; rep < 3 && !st; ++rep) {  // the fastest of three (the first may be cold)
                cudaMemcpyAsync(th, theta_d, T * a->P * 16, cudaMemcpyDeviceToDevice, s);
                cudaMemcpyAsync(sp, spins_d, T * d->ns * W * 8, cudaMemcpyDeviceToDevice, s);
                cudaEventRecord(e0, s);
                st = run_pipelined_shape(a, &q, th, sp, otvmc_run_n_meas(&q) ? mo : nullptr, work_d, rb, s, nullptr,
                                         sh);
                cudaEventRecord(e1, s);
                if (!st) st = otvmc_check(work_d, stream);
                float m = 0.f;
                if (!st && cudaEventElapsedTime(&m, e0, e1) == cudaSuccess) ms = std::min(ms, m);
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = sh;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(a, d)] = best;
    }
    if (pipes_out) *pipes_out = best.pipes;
    if (groups_out) *groups_out = best.groups;
    if (ms_out) *ms_out = best_ms;
    return OTVMC_OK;
}

void otvmc_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

otvmc_status otvmc_run_trajectories_linear(const otvmc_ansatz* a, const otvmc_run_desc* d, double* theta_d,
                                           uint64_t* spins_d, double* moments_d, double* lnQ_d, double* lnQ_rows_d,
                                           void* work_d, size_t work_bytes, void* stream) {
    otvmc_status st = check_run(a, d);
    if (st) return st;
    if (!theta_d || !spins_d || !work_d || !lnQ_d) return fail(OTVMC_ERR_INVALID, "run_linear: null buffer");
    if (otvmc_run_n_meas(d) > 0 && !moments_d) return fail(OTVMC_ERR_INVALID, "run_linear: moments_d needed");
    cudaStream_t s = (cudaStream_t)stream;
    const LinState lin{lnQ_d, moments_d ? lnQ_rows_d : nullptr};
    st = run_pipelined(a, d, theta_d, spins_d, moments_d, work_d, work_bytes, s, &lin);
    if (st) return st;
    return otvmc_check(work_d, stream);
}

otvmc_status otvmc_ensemble_weighted(const double* mom, const double* w, int ntraj, int n_sites, double* M_h,
                                     double* C_h, double* xi2_h, double* dM_h) {
    if (!mom || !w || ntraj < 1 || n_sites < 1) return fail(OTVMC_ERR_INVALID, "ensemble_weighted: bad arguments");
    std::vector<double> wm((size_t)ntraj * OTVMC_MOMENTS);
    for (int t = 0; t < ntraj; ++t)
        for (int k = 0; k < OTVMC_MOMENTS; ++k) wm[(size_t)t * OTVMC_MOMENTS + k] = w[t] * mom[(size_t)t * OTVMC_MOMENTS + k];
    return otvmc_ensemble(wm.data(), ntraj, n_sites, M_h, C_h, xi2_h, dM_h);
}

size_t otvmc_run_host_workspace_bytes(const otvmc_ansatz* a, const otvmc_run_desc* d) {
    const size_t base = otvmc_run_workspace_bytes(a, d);
    if (!base) return 0;
    const size_t T = d->ntraj;
    const size_t io = T * a->P * 16 + T * d->ns * ((a->n + 63) / 64) * 8 +
                      (size_t)otvmc_run_n_meas(d) * T * OTVMC_MOMENTS * 8 + 3 * 256;
    return base + io;
}

otvmc_status otvmc_run_trajectories_host(const otvmc_ansatz* a, const otvmc_run_desc* d, double* theta_h,
                                         uint64_t* spins_h, double* moments_h, void* work_d, size_t work_bytes,
                                         void* stream) {
    otvmc_status st = check_run(a, d);
    if (st) return st;
    if (!theta_h || !spins_h || !work_d) return fail(OTVMC_ERR_INVALID, "run_host: null buffer");
    const int nmeas = otvmc_run_n_meas(d);
    if (nmeas > 0 && !moments_h) return fail(OTVMC_ERR_INVALID, "run_host: moments_h needed");
    const size_t base = otvmc_run_workspace_bytes(a, d);
    if (work_bytes < otvmc_run_host_workspace_bytes(a, d)) return fail(OTVMC_ERR_WORKSPACE, "workspace too small");
    const size_t T = d->ntraj;
    const size_t th_bytes = T * a->P * 16, sp_bytes = T * d->ns * ((a->n + 63) / 64) * 8,
                 mo_bytes = (size_t)nmeas * T * OTVMC_MOMENTS * 8;
    char* io = (char*)work_d + ((base + 255) & ~(size_t)255);
    double* th_d = (double*)io;
    uint64_t* sp_d = (uint64_t*)(io + ((th_bytes + 255) & ~(size_t)255));
    double* mo_d = (double*)((char*)sp_d + ((sp_bytes + 255) & ~(size_t)255));
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(th_d, theta_h, th_bytes, cudaMemcpyHostToDevice, s), "theta upload");
    CK(cudaMemcpyAsync(sp_d, spins_h, sp_bytes, cudaMemcpyHostToDevice, s), "spins upload");
    st = run_pipelined(a, d, th_d, sp_d, nmeas ? mo_d : nullptr, work_d, base, s);
    if (st) return st;
    CK(cudaMemcpyAsync(theta_h, th_d, th_bytes, cudaMemcpyDeviceToHost, s), "theta download");
    CK(cudaMemcpyAsync(spins_h, sp_d, sp_bytes, cudaMemcpyDeviceToHost, s), "spins download");
    if (nmeas) CK(cudaMemcpyAsync(moments_h, mo_d, mo_bytes, cudaMemcpyDeviceToHost, s), "moments download");
    return otvmc_check(work_d, stream);
}

}  // extern "C"
