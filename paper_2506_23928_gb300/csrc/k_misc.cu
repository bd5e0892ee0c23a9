// Wiener increments (Eq. 2), initial chain states, and the predictor-corrector
// combination of App. C.
#include "common.cuh"

namespace otvmc {

// Delta W[t][n] = sqrt(dt) * z: four normals per Philox counter (two Box-Muller pairs).
__global__ void noise_kernel(int nops, int traj0, uint32_t k0, uint32_t k1, uint32_t step, double sdt,
                             double* __restrict__ dW) {
    const int t = blockIdx.x;
    const int nq = (nops + 3) / 4;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const u32x4 w = philox(u32x4{(uint32_t)q, step, (uint32_t)(traj0 + t), TAG_NOISE << 28}, k0, k1);
        double z[4], s, c;
        double rad = sqrt(-2.0 * log(u01(w.x)));
        sincospi(2.0 * u01(w.y), &s, &c);
        z[0] = rad * c;
        z[1] = rad * s;
        rad = sqrt(-2.0 * log(u01(w.z)));
        sincospi(2.0 * u01(w.w), &s, &c);
        z[2] = rad * c;
        z[3] = rad * s;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int n = 4 * q + i;
            if (n < nops) dW[(size_t)t * nops + n] = sdt * z[i];
        }
    }
}

cudaError_t launch_noise(const otvmc_model* m, int ntraj, int traj0, uint64_t seed, int64_t step, double dt,
                         double* dW, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_NOISE, s);
    if (m->nops == 0) return cudaSuccess;
    noise_kernel<<<ntraj, 64, 0, s>>>(m->nops, traj0, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)step,
                                      sqrt(dt), dW);
    count_launch();
    return cudaGetLastError();
}

// Uniform i.i.d. configurations; unused high bits of the last word are zero.
__global__ void init_chains_kernel(int n, int W, int ns, int traj0, uint32_t k0, uint32_t k1,
                                   uint64_t* __restrict__ spins) {
    const int chain = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (chain >= ns) return;
    uint64_t* out = spins + ((size_t)t * ns + chain) * W;
    for (int q = 0; 2 * q < W; ++q) {
        const u32x4 w = philox(u32x4{(uint32_t)q, (uint32_t)chain, (uint32_t)(traj0 + t), TAG_INIT << 28}, k0, k1);
        const uint64_t a = (uint64_t)w.x | ((uint64_t)w.y << 32);
        const uint64_t b = (uint64_t)w.z | ((uint64_t)w.w << 32);
        for (int h = 0; h < 2; ++h) {
            const int wi = 2 * q + h;
            if (wi >= W) break;
            uint64_t v = h ? b : a;
            const int bits = n - 64 * wi;
            if (bits < 64) v &= (1ull << bits) - 1ull;
            out[wi] = v;
        }
    }
}

cudaError_t launch_init_chains(int n, int ntraj, int traj0, int ns, uint64_t seed, uint64_t* spins,
                               cudaStream_t s) {
    ProfScope prof_(OTVMC_K_NOISE, s);
    const int W = (n + 63) / 64;
    dim3 grid((ns + 127) / 128, ntraj);
    init_chains_kernel<<<grid, 128, 0, s>>>(n, W, ns, traj0, (uint32_t)seed, (uint32_t)(seed >> 32), spins);
    count_launch();
    return cudaGetLastError();
}

// App. C on theta.  stage 0: out = theta + c * d0 (c = 1 Heun predictor point, 1/2
// midpoint point).  stage 1: Heun theta + (d0 + d1)/2, midpoint theta + d1.  A trajectory
// whose result is not finite keeps theta (out = theta) and is flagged.
__global__ void sde_kernel(int64_t P, int scheme, int stage, const double2* __restrict__ theta,
                           const double2* __restrict__ d0, const double2* __restrict__ d1,
                           double2* __restrict__ out, int* failed, int* status) {
    const int t = blockIdx.x;
    const double2* th = theta + (size_t)t * P;
    const double2* a = d0 + (size_t)t * P;
    const double2* b = d1 ? d1 + (size_t)t * P : nullptr;
    double2* o = out + (size_t)t * P;
    int bad = 0;
    for (int64_t k = threadIdx.x; k < P; k += blockDim.x) {
        double2 v;
        if (stage == 0) {
            const double c = (scheme == OTVMC_HEUN) ? 1.0 : 0.5;
            v = make_double2(th[k].x + c * a[k].x, th[k].y + c * a[k].y);
        } else if (scheme == OTVMC_HEUN) {
            v = make_double2(th[k].x + 0.5 * (a[k].x + b[k].x), th[k].y + 0.5 * (a[k].y + b[k].y));
        } else {
            v = make_double2(th[k].x + b[k].x, th[k].y + b[k].y);
        }
        bad |= !(isfinite(v.x) && isfinite(v.y));
    }
    bad = __syncthreads_or(bad);
    if (bad) {
        if (threadIdx.x == 0) {
            record_error(status, OTVMC_ERR_NONFINITE, t);
            if (failed) failed[t] = 1;
        }
    }
    for (int64_t k = threadIdx.x; k < P; k += blockDim.x) {
        double2 v = th[k];
        if (!bad) {
            if (stage == 0) {
                const double c = (scheme == OTVMC_HEUN) ? 1.0 : 0.5;
                v = make_double2(th[k].x + c * a[k].x, th[k].y + c * a[k].y);
            } else if (scheme == OTVMC_HEUN) {
                v = make_double2(th[k].x + 0.5 * (a[k].x + b[k].x), th[k].y + 0.5 * (a[k].y + b[k].y));
            } else {
                v = make_double2(th[k].x + b[k].x, th[k].y + b[k].y);
            }
        }
        o[k] = v;
    }
}

cudaError_t launch_sde(int ntraj, int64_t P, int scheme, int stage, const double2* theta, const double2* d0,
                       const double2* d1, double2* out, int* failed, int* status, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SDE, s);
    sde_kernel<<<ntraj, 256, 0, s>>>(P, scheme, stage, theta, d0, d1, out, failed, status);
    count_launch();
    return cudaGetLastError();
}

// Normalisation of the linear SSE (App. B): d ln Q = 2 Im<E_eff^lin> dt + 2 sum_n Re<B^n> o dW_n,
// which over one step is twice the real part of the sample mean of v^lin = -i dt E_eff^lin +
// sum_n dW_n B^n (vinfo[4 t] after the v reduction).  Stage 0 keeps the predictor's increment;
// stage 1 advances ln Q by the scheme of the parameters: the trapezoidal mean of the two
// increments (Heun) or the corrector's increment (midpoint).
__global__ void lnq_kernel(int ntraj, int scheme, int stage, const double* __restrict__ vinfo,
                           double* __restrict__ g0, double* __restrict__ lnQ) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntraj) return;
    const double g = 2.0 * vinfo[4 * t];
    if (stage == 0) {
        g0[t] = g;
    } else {
        lnQ[t] += scheme == OTVMC_HEUN ? 0.5 * (g0[t] + g) : g;
    }
}

cudaError_t launch_lnq(int ntraj, int scheme, int stage, const double* vinfo, double* g0, double* lnQ,
                       cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SDE, s);
    lnq_kernel<<<(ntraj + 127) / 128, 128, 0, s>>>(ntraj, scheme, stage, vinfo, g0, lnQ);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
