// Allocation-free variant of otvmc_local_estimators.
//
// Some callers cannot hand the library a workspace: their device memory is owned by a
// memory manager with a hard budget that they may not allocate outside of, or they run in
// a latency-sensitive loop where an allocation (which may synchronise the device) is not
// acceptable.  This entry point takes only inputs and outputs; its scratch is a fixed
// array of this library in device memory, which every GPU that loads the library holds
// until the process exits.
#include <mutex>
#include <string>

#include "common.cuh"

namespace otvmc {

// Largest scratch the allocation-free entry point can use.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device, looked up once per device.
// (In host code the array's name is only a host-side stand-in, not a device address.)
static cudaError_t noalloc_scratch(void** out) {
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static void* addr[MAXDEV] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAXDEV) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = p;
    }
    *out = addr[dev];
    return cudaSuccess;
}

}  // namespace otvmc

using namespace otvmc;

extern "C" otvmc_status otvmc_local_estimators_noalloc(const otvmc_ansatz* a, const double* theta_d,
                                                       const uint64_t* spins_d, int ntraj, int ns,
                                                       const double* dW_d, double dt, int precision, double* Eeff_d,
                                                       double* v_d, double* lpl_d, int* status_d, void* stream) {
    if (a == nullptr || a->model == nullptr || a->P <= 0) {
        set_error("local_estimators_noalloc: null or invalid ansatz");
        return OTVMC_ERR_INVALID;
    }
    if (a->kind != OTVMC_JASTROW) {
        set_error("local_estimators_noalloc: only the Jastrow ansatz is built");
        return OTVMC_ERR_UNSUPPORTED;
    }
    if (ntraj < 1 || ns < 1 || !theta_d || !spins_d || !v_d || (a->model->nops > 0 && !dW_d) ||
        (precision != OTVMC_PREC_FP64 && precision != OTVMC_PREC_MIXED)) {
        set_error("local_estimators_noalloc: bad arguments");
        return OTVMC_ERR_INVALID;
    }
    // size of the scratch this call needs, before touching the device
    Carver sz(nullptr, (size_t)-1);
    carve_est_bufs(sz, a, ntraj, ns);
    if (!lpl_d) sz.take<double>((size_t)ntraj * (a->model->nops + 1));
    if (sz.off > NOALLOC_SCRATCH_BYTES) {
        set_error("local_estimators_noalloc: this batch needs " + std::to_string(sz.off) +
                  " bytes of scratch, more than the fixed " + std::to_string(NOALLOC_SCRATCH_BYTES) +
                  " bytes; use otvmc_local_estimators with a workspace, or fewer trajectories per call");
        return OTVMC_ERR_WORKSPACE;
    }
    void* base = nullptr;
    cudaError_t e = noalloc_scratch(&base);
    if (e != cudaSuccess) return cuda_status(e, "local_estimators_noalloc: scratch address");
    Carver c(base, NOALLOC_SCRATCH_BYTES);
    EvalBufs b = carve_est_bufs(c, a, ntraj, ns);
    double* lpl = lpl_d ? lpl_d : c.take<double>((size_t)ntraj * (a->model->nops + 1));
    // Every buffer the kernels read below is fully written earlier in this call, so nothing in
    // the shared scratch needs clearing between calls.
    cudaStream_t s = (cudaStream_t)stream;
    const bool fp32 = precision == OTVMC_PREC_MIXED;
    e = launch_jastrow_prep(a, (const double2*)theta_d, ntraj, b, status_d, s);
    if (e != cudaSuccess) return cuda_status(e, "local_estimators_noalloc: prep launch");
    e = launch_est1_jastrow(a, spins_d, ntraj, ns, fp32, b, status_d, s);
    if (e != cudaSuccess) return cuda_status(e, "local_estimators_noalloc: est1 launch");
    e = launch_site_means(a, ntraj, ns, fp32, b, lpl, s);
    if (e != cudaSuccess) return cuda_status(e, "local_estimators_noalloc: site means launch");
    e = launch_est2(a, spins_d, ntraj, ns, fp32, dW_d, dt, lpl, b, (double2*)Eeff_d, (double2*)v_d, s);
    if (e != cudaSuccess) return cuda_status(e, "local_estimators_noalloc: est2 launch");
    return OTVMC_OK;
}
