// RBM ansatz (Eq. 11), plain FP64 path: sampling, local estimators, log-derivatives, the
// complex S (or T when P > ns) through its real embedding, D, and the observables.
//
//   log psi(x) = sum_i a_i s_i + sum_m lc(gamma_m(x)),  gamma_m = b_m + sum_i W_im s_i,
//   lc(z) = log(2 cosh z);  theta = [a (N), b (M), W (N x M, row-major)], P = N + M + N M.
//   Flip ratio:  log r_j = -2 a_j s_j + sum_m [lc(gamma_m - 2 W_jm s_j) - lc(gamma_m)].
//   Log-derivatives (definitions after Eq. 8):  O_a_i = s_i, O_b_m = tanh gamma_m,
//   O_W_im = s_i tanh gamma_m  (complex).
//
// Complex Hermitian S = O_c^+ O_c / ns and T = O_c O_c^+ / ns are never formed as complex
// matrices on this path.  With O_c = Or + i Oi (ns x P) and the real (2 ns x 2 P) matrix
//     R = [[Or, -Oi], [Oi, Or]],
// R^T R / ns = [[Re S, -Im S], [Im S, Re S]] and R R^T / ns = [[Re T, -Im T], [Im T, Re T]]
// (the real embeddings, positive definite exactly when S and T are), R^T [vr; vi] / ns =
// [Re D; Im D] for D = O_c^+ v_c / ns, and R^T [yr; yi] / ns = [Re; Im] of O_c^+ y / ns.  So
// (S + eps I) delta = D is a real symmetric solve of size 2P, and the push-through form
// delta = O_c^+ (T + eps I)^-1 v_c / ns (same delta) one of size 2 ns.
#include <cuda_bf16.h>

#include "common.cuh"

namespace otvmc {

// log(2 cosh z) = s z + log1p(exp(-2 s z)), s = sign(Re z): no overflow.
__device__ __forceinline__ double2 lc2(double2 z) {
    const double s = z.x >= 0.0 ? 1.0 : -1.0;
    const double e = exp(-2.0 * s * z.x);
    double sn, cs;
    sincos(2.0 * z.y, &sn, &cs);
    const double wr = e * cs, wi = -s * e * sn;  // exp(-2 s z)
    return make_double2(s * z.x + 0.5 * log1p(2.0 * wr + wr * wr + wi * wi), s * z.y + atan2(wi, 1.0 + wr));
}
// Re lc(z) only (the Metropolis ratio |psi'/psi|^2 needs the real part).
__device__ __forceinline__ double lc2_re(double2 z) {
    const double ax = fabs(z.x);
    const double e = exp(-2.0 * ax);
    return ax + 0.5 * log1p(e * (2.0 * cos(2.0 * z.y) + e));
}
// tanh z = s (1 - w) / (1 + w), w = exp(-2 s z), s = sign(Re z).
__device__ __forceinline__ double2 ctanh(double2 z) {
    const double s = z.x >= 0.0 ? 1.0 : -1.0;
    const double e = exp(-2.0 * s * z.x);
    double sn, cs;
    sincos(2.0 * z.y, &sn, &cs);
    const double wr = e * cs, wi = -s * e * sn;
    const double nr = 1.0 - wr, ni = -wi, dr = 1.0 + wr, di = wi;
    const double den = dr * dr + di * di;
    return make_double2(s * (nr * dr + ni * di) / den, s * (ni * dr - nr * di) / den);
}
__device__ __forceinline__ double2 cexp2(double2 z) {
    double sn, cs;
    sincos(z.y, &sn, &cs);
    const double e = exp(z.x);
    return make_double2(e * cs, e * sn);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

struct RbmTheta {
    const double2* a;  // [N]
    const double2* b;  // [M]
    const double2* W;  // [N][M]
};
__device__ __forceinline__ RbmTheta rbm_split(const double2* theta, int P, int n, int M, int t) {
    const double2* th = theta + (size_t)t * P;
    return RbmTheta{th, th + n, th + n + M};
}

// ------------------------------------------------------------------------- sampling
// One thread per chain; the chain's angles gamma and Re lc(gamma) live in scratch laid out
// [t][m][chain] (coalesced across the chains of a warp).  Proposal draws as in the Jastrow
// sampler (same counters), accepted iff u < exp(2 Re log r_j), all in FP64.
__global__ void __launch_bounds__(128) sample_rbm_kernel(const double2* __restrict__ theta, int P, int n, int M,
                                                         int W, int ns, int n_sweep, uint32_t k0, uint32_t k1,
                                                         uint32_t evtag, int traj0, uint64_t* __restrict__ spins,
                                                         double2* __restrict__ gam, double* __restrict__ lcr,
                                                         unsigned long long* __restrict__ accepted) {
    const int t = blockIdx.y;
    const int chain = blockIdx.x * blockDim.x + threadIdx.x;
    if (chain >= ns) return;
    const RbmTheta th = rbm_split(theta, P, n, M, t);
    uint64_t* sp = spins + ((size_t)t * ns + chain) * W;
    uint64_t wd[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) wd[w] = w < W ? sp[w] : 0ull;
    double2* g = gam + (size_t)t * M * ns + chain;  // g[m * ns]
    double* l0 = lcr + (size_t)t * M * ns + chain;
    for (int m = 0; m < M; ++m) {
        double2 z = th.b[m];
        for (int i = 0; i < n; ++i) {
            const double si = ((wd[i >> 6] >> (i & 63)) & 1ull) ? 1.0 : -1.0;
            z.x += th.W[(size_t)i * M + m].x * si;
            z.y += th.W[(size_t)i * M + m].y * si;
        }
        g[(size_t)m * ns] = z;
        l0[(size_t)m * ns] = lc2_re(z);
    }
    const int nprop = n_sweep * n;
    int nacc = 0;
    u32x4 draw = {0u, 0u, 0u, 0u};
    for (int p = 0; p < nprop; ++p) {
        if ((p & 1) == 0) draw = philox(u32x4{(uint32_t)(p / 2), (uint32_t)chain, (uint32_t)(traj0 + t), evtag}, k0, k1);
        const uint32_t wsite = (p & 1) ? draw.z : draw.x;
        const uint32_t wu = (p & 1) ? draw.w : draw.y;
        const int j = (int)(((unsigned long long)wsite * (unsigned long long)n) >> 32);
        const double sj = ((wd[j >> 6] >> (j & 63)) & 1ull) ? 1.0 : -1.0;
        const double u = u01(wu);
        double lr = -2.0 * th.a[j].x * sj;
        const double2* Wj = th.W + (size_t)j * M;
        for (int m = 0; m < M; ++m) {
            const double2 z = g[(size_t)m * ns];
            lr += lc2_re(make_double2(z.x - 2.0 * Wj[m].x * sj, z.y - 2.0 * Wj[m].y * sj)) - l0[(size_t)m * ns];
        }
        if (u < exp(2.0 * lr)) {
            for (int m = 0; m < M; ++m) {
                const double2 z = g[(size_t)m * ns];
                const double2 z1 = make_double2(z.x - 2.0 * Wj[m].x * sj, z.y - 2.0 * Wj[m].y * sj);
                g[(size_t)m * ns] = z1;
                l0[(size_t)m * ns] = lc2_re(z1);
            }
            wd[j >> 6] ^= 1ull << (j & 63);
            ++nacc;
        }
    }
#pragma unroll
    for (int w = 0; w < 4; ++w)
        if (w < W) sp[w] = wd[w];
    if (accepted != nullptr && nacc) atomicAdd(accepted + t, (unsigned long long)nacc);
}

cudaError_t launch_sample_rbm(const otvmc_ansatz* an, const double2* theta, int ntraj, int traj0, int ns, int n_sweep,
                              uint64_t seed, int64_t eval, uint64_t* spins, double2* gam, double* lcr,
                              unsigned long long* accepted, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SAMPLE, s);
    const int n = an->n, W = (n + 63) / 64;
    const uint32_t evtag = (TAG_SAMPLE << 28) | ((uint32_t)eval & 0x0FFFFFFFu);
    dim3 grid((ns + 127) / 128, ntraj);
    sample_rbm_kernel<<<grid, 128, 0, s>>>(theta, (int)an->P, n, an->m, W, ns, n_sweep, (uint32_t)seed,
                                           (uint32_t)(seed >> 32), evtag, traj0, spins, gam, lcr, accepted);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------- local estimators
// Same blocking and outputs as the Jastrow est1 kernel (r, E_H, per-CTA site sums), so that
// the site means, <L+L^+>, E_eff and v kernels are shared: thread (g, j) owns site j of
// samples g, g + SPP, ..; each round first computes the SPP samples' angles and lc(gamma)
// in shared memory.
__global__ void __launch_bounds__(256) est_rbm_kernel(int n, int M, int W, int P, int ns, double h,
                                                      const double2* __restrict__ theta,
                                                      const uint64_t* __restrict__ spins,
                                                      const long long* __restrict__ QJ,
                                                      const long long* __restrict__ baseJ, double2* __restrict__ r_out,
                                                      double2* __restrict__ EH_out, double2* __restrict__ part_r,
                                                      double2* __restrict__ part_sr, double* __restrict__ part_s) {
    constexpr int SPT = EST_SAMPLES_PER_THREAD;
    const int NT = ((n + 31) / 32) * 32;
    const int SPP = 256 / NT;
    const int SB = SPP * SPT;
    const int t = blockIdx.y, blk = blockIdx.x;
    const int j = threadIdx.x % NT, g = threadIdx.x / NT;
    const bool active = (g < SPP) && (j < n);
    const int s0 = blk * SB;
    extern __shared__ __align__(16) unsigned char smraw[];
    double2* gs = (double2*)smraw;        // [SPP][M] gamma
    double2* ls = gs + SPP * M;           // [SPP][M] lc(gamma)
    double2* ered = ls + SPP * M;         // [SB][NT/32]
    uint64_t* sw = (uint64_t*)(ered + SB * (NT / 32));  // [SPP][W]
    __shared__ double2 red_r[256], red_sr[256];
    __shared__ double red_s[256];
    const RbmTheta th = rbm_split(theta, P, n, M, t);
    double2 pr = make_double2(0, 0), psr = make_double2(0, 0);
    double ps = 0.0;
    const int lane = threadIdx.x & 31, wis = j / 32;
    for (int q = 0; q < SPT; ++q) {
        __syncthreads();
        for (int i = threadIdx.x; i < SPP * W; i += blockDim.x) {
            const int gg = i / W, w = i - gg * W;
            const int s = s0 + gg + q * SPP;
            sw[i] = s < ns ? spins[((size_t)t * ns + s) * W + w] : 0ull;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < SPP * M; i += blockDim.x) {
            const int gg = i / M, m = i - gg * M;
            const uint64_t* w = sw + gg * W;
            double2 z = th.b[m];
            for (int k = 0; k < n; ++k) {
                const double sk = ((w[k >> 6] >> (k & 63)) & 1ull) ? 1.0 : -1.0;
                z.x += th.W[(size_t)k * M + m].x * sk;
                z.y += th.W[(size_t)k * M + m].y * sk;
            }
            gs[i] = z;
            ls[i] = lc2(z);
        }
        __syncthreads();
        const int sl = g + q * SPP;
        const int s = s0 + sl;
        double2 contrib = make_double2(0.0, 0.0);
        if (active && s < ns) {
            const uint64_t* w = sw + g * W;
            const double sj = ((w[j >> 6] >> (j & 63)) & 1ull) ? 1.0 : -1.0;
            double2 lr = make_double2(-2.0 * th.a[j].x * sj, -2.0 * th.a[j].y * sj);
            const double2* Wj = th.W + (size_t)j * M;
            for (int m = 0; m < M; ++m) {
                const double2 z = gs[g * M + m];
                const double2 l1 = lc2(make_double2(z.x - 2.0 * Wj[m].x * sj, z.y - 2.0 * Wj[m].y * sj));
                lr = cadd(lr, csub(l1, ls[g * M + m]));
            }
            const double2 r = cexp2(lr);
            r_out[((size_t)t * ns + s) * n + j] = r;
            // Ising part of E_H from the exact fixed-point field sum_k J_jk s_k
            long long aj = 0;
            for (int k = 0; k < n; ++k)
                if ((w[k >> 6] >> (k & 63)) & 1ull) aj += QJ[(size_t)j * n + k];
            const double fj = (double)(baseJ[j] + 2 * aj) * FX_INV;
            contrib = make_double2(0.5 * sj * fj + h * r.x, h * r.y);
            pr.x += r.x;
            pr.y += r.y;
            psr.x += sj * r.x;
            psr.y += sj * r.y;
            ps += sj;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            contrib.x += __shfl_xor_sync(0xffffffffu, contrib.x, off);
            contrib.y += __shfl_xor_sync(0xffffffffu, contrib.y, off);
        }
        if (lane == 0 && g < SPP) ered[sl * (NT / 32) + wis] = contrib;
    }
    __syncthreads();
    if (threadIdx.x < SB) {
        const int sl = threadIdx.x, s = s0 + sl;
        if (s < ns) {
            double2 e = make_double2(0.0, 0.0);
            for (int w = 0; w < NT / 32; ++w) e = cadd(e, ered[sl * (NT / 32) + w]);
            EH_out[(size_t)t * ns + s] = e;
        }
    }
    red_r[threadIdx.x] = pr;
    red_sr[threadIdx.x] = psr;
    red_s[threadIdx.x] = ps;
    __syncthreads();
    if (threadIdx.x < n) {
        const int jj = threadIdx.x;
        double2 a = make_double2(0, 0), b = make_double2(0, 0);
        double c = 0.0;
        for (int gg = 0; gg < SPP; ++gg) {
            a = cadd(a, red_r[gg * NT + jj]);
            b = cadd(b, red_sr[gg * NT + jj]);
            c += red_s[gg * NT + jj];
        }
        const size_t o = ((size_t)t * gridDim.x + blk) * n + jj;
        part_r[o] = a;
        part_sr[o] = b;
        part_s[o] = c;
    }
}

cudaError_t launch_est_rbm(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int ntraj, int ns,
                           const EvalBufs& b, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_EST1, s);
    const int n = a->n, M = a->m, W = (n + 63) / 64;
    const int NT = ((n + 31) / 32) * 32, SPP = 256 / NT, SB = SPP * EST_SAMPLES_PER_THREAD;
    const size_t smem = (size_t)2 * SPP * M * 16 + (size_t)SB * (NT / 32) * 16 + (size_t)SPP * W * 8 + 64;
    cudaError_t e = cudaFuncSetAttribute(est_rbm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const otvmc_model* m = a->model;
    dim3 grid(est_blocks(n, ns), ntraj);
    est_rbm_kernel<<<grid, 256, smem, s>>>(n, M, W, (int)a->P, ns, m->h, theta, spins, m->QJ_d, m->baseJ_d, b.r, b.EH,
                                           b.part_r, b.part_sr, b.part_s);
    count_launch();
    return cudaGetLastError();
}

// --------------------------------------------------------------- log-derivatives
// Th[t][m][x] = tanh gamma_m(x)
__global__ void __launch_bounds__(256) rbm_tanh_kernel(int n, int M, int W, int P, int ns,
                                                       const double2* __restrict__ theta,
                                                       const uint64_t* __restrict__ spins, double2* __restrict__ Th) {
    const int t = blockIdx.z, m = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ns) return;
    const RbmTheta th = rbm_split(theta, P, n, M, t);
    const uint64_t* w = spins + ((size_t)t * ns + x) * W;
    double2 z = th.b[m];
    for (int k = 0; k < n; ++k) {
        const double sk = ((w[k >> 6] >> (k & 63)) & 1ull) ? 1.0 : -1.0;
        z.x += th.W[(size_t)k * M + m].x * sk;
        z.y += th.W[(size_t)k * M + m].y * sk;
    }
    Th[((size_t)t * M + m) * ns + x] = ctanh(z);
}

__device__ __forceinline__ double2 rbm_O(const uint64_t* sp, int W, int n, int M, int ns, const double2* Tht, int k,
                                         int x) {
    if (k < n) return make_double2(((sp[(size_t)x * W + (k >> 6)] >> (k & 63)) & 1ull) ? 1.0 : -1.0, 0.0);
    if (k < n + M) return Tht[(size_t)(k - n) * ns + x];
    const int i = (k - n - M) / M, m = (k - n - M) - i * M;
    const double si = ((sp[(size_t)x * W + (i >> 6)] >> (i & 63)) & 1ull) ? 1.0 : -1.0;
    return cscale(Tht[(size_t)m * ns + x], si);
}

// obar_k = mean_x O_xk, one warp per parameter (fixed-order reduction)
__global__ void __launch_bounds__(256) rbm_obar_kernel(int n, int M, int W, int P, int ns,
                                                       const uint64_t* __restrict__ spins,
                                                       const double2* __restrict__ Th, double2* __restrict__ obar) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * 8 + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (k >= P) return;
    const uint64_t* sp = spins + (size_t)t * ns * W;
    const double2* Tht = Th + (size_t)t * M * ns;
    double2 a = make_double2(0.0, 0.0);
    for (int x = lane; x < ns; x += 32) a = cadd(a, rbm_O(sp, W, n, M, ns, Tht, k, x));
    for (int off = 16; off > 0; off >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, off);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, off);
    }
    if (lane == 0) obar[(size_t)t * P + k] = make_double2(a.x / ns, a.y / ns);
}

// R = [[Or, -Oi], [Oi, Or]] of the centred O, (2 ns) x (2 P); kmajor: R^T stored [2P][2ns]
// (rows = parameters), else R stored [2ns][2P] (rows = samples).
__global__ void __launch_bounds__(256) rbm_R_kernel(int n, int M, int W, int P, int ns, int kmajor,
                                                    const uint64_t* __restrict__ spins,
                                                    const double2* __restrict__ Th, const double2* __restrict__ obar,
                                                    double* __restrict__ R) {
    const int t = blockIdx.y;
    const uint64_t* sp = spins + (size_t)t * ns * W;
    const double2* Tht = Th + (size_t)t * M * ns;
    double* Rt = R + (size_t)t * 4 * P * ns;
    const size_t NS2 = 2 * (size_t)ns, P2 = 2 * (size_t)P;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)P * ns; e += (size_t)gridDim.x * blockDim.x) {
        int k, x;
        if (kmajor) {
            k = (int)(e / ns);
            x = (int)(e - (size_t)k * ns);
        } else {
            x = (int)(e / P);
            k = (int)(e - (size_t)x * P);
        }
        const double2 o = csub(rbm_O(sp, W, n, M, ns, Tht, k, x), obar[(size_t)t * P + k]);
        if (kmajor) {
            Rt[(size_t)k * NS2 + x] = o.x;
            Rt[(size_t)k * NS2 + ns + x] = o.y;
            Rt[(size_t)(P + k) * NS2 + x] = -o.y;
            Rt[(size_t)(P + k) * NS2 + ns + x] = o.x;
        } else {
            Rt[(size_t)x * P2 + k] = o.x;
            Rt[(size_t)x * P2 + P + k] = -o.y;
            Rt[(size_t)(ns + x) * P2 + k] = o.y;
            Rt[(size_t)(ns + x) * P2 + P + k] = o.x;
        }
    }
}

// u[x'] for x' < 2 ns: [Re v - Re vbar; Im v - Im vbar] (vbar from vinfo), stored as the real
// parts of double2 (the solver's right-hand side layout); also usable as a real vector.
__global__ void rbm_vtilde_kernel(int ns, const double2* __restrict__ v, const double* __restrict__ vinfo,
                                  double2* __restrict__ u) {
    const int t = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 2 * ns) return;
    const double2 vv = v[(size_t)t * ns + (x < ns ? x : x - ns)];
    const double val = x < ns ? vv.x - vinfo[4 * t] : vv.y - vinfo[4 * t + 1];
    u[(size_t)t * 2 * ns + x] = make_double2(val, 0.0);
}

// out[k'] = inv sum_x' R[x'][k'] u[x'].x  (k' < 2P), written as the real part of double2.
// kmajor: one warp per k' along the contiguous samples; else one thread per k'.
__global__ void __launch_bounds__(256) rbm_gemv_kernel(int P, int ns, int kmajor, double inv, const double* __restrict__ R,
                                                       const double2* __restrict__ u, double2* __restrict__ out) {
    const int t = blockIdx.y;
    const size_t NS2 = 2 * (size_t)ns, P2 = 2 * (size_t)P;
    const double* Rt = R + (size_t)t * 4 * P * ns;
    const double2* ut = u + (size_t)t * NS2;
    if (kmajor) {
        const int k = blockIdx.x * 8 + threadIdx.x / 32, lane = threadIdx.x & 31;
        if (k >= 2 * P) return;
        double a = 0.0;
        for (size_t x = lane; x < NS2; x += 32) a = fma(Rt[(size_t)k * NS2 + x], ut[x].x, a);
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) out[(size_t)t * P2 + k] = make_double2(a * inv, 0.0);
    } else {
        const int k = blockIdx.x * blockDim.x + threadIdx.x;
        if (k >= 2 * P) return;
        double a = 0.0;
        for (size_t x = 0; x < NS2; ++x) a = fma(Rt[x * P2 + k], ut[x].x, a);
        out[(size_t)t * P2 + k] = make_double2(a * inv, 0.0);
    }
}

// delta_k = x[k] + i x[P + k] from the real solution of the embedded system.
__global__ void rbm_unpack_kernel(int P, const double2* __restrict__ xe, double2* __restrict__ delta) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    delta[(size_t)t * P + k] = make_double2(xe[(size_t)t * 2 * P + k].x, xe[(size_t)t * 2 * P + P + k].x);
}

// Complex S from the embedding: S = E[0:P][0:P] + i E[P:2P][0:P]; and back.
__global__ void rbm_extract_S_kernel(int P, const double* __restrict__ E, double2* __restrict__ S) {
    const int t = blockIdx.y;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)P * P; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / P, j = e - i * P;
        const double* Et = E + (size_t)t * 4 * P * P;
        S[(size_t)t * P * P + e] = make_double2(Et[i * 2 * P + j], Et[(P + i) * 2 * P + j]);
    }
}
__global__ void rbm_embed_S_kernel(int P, const double2* __restrict__ S, double* __restrict__ E) {
    const int t = blockIdx.y;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)P * P; e += (size_t)gridDim.x * blockDim.x) {
        const size_t i = e / P, j = e - i * P;
        const double2 s = S[(size_t)t * P * P + e];
        double* Et = E + (size_t)t * 4 * P * P;
        Et[i * 2 * P + j] = s.x;
        Et[(P + i) * 2 * P + P + j] = s.x;
        Et[(P + i) * 2 * P + j] = s.y;
        Et[i * 2 * P + P + j] = -s.y;
    }
}
// [Re D; Im D] as the real parts of double2 (embedded right-hand side)
__global__ void rbm_embed_D_kernel(int P, const double2* __restrict__ D, double2* __restrict__ De) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const double2 d = D[(size_t)t * P + k];
    De[(size_t)t * 2 * P + k] = make_double2(d.x, 0.0);
    De[(size_t)t * 2 * P + P + k] = make_double2(d.y, 0.0);
}

// -------------------------------------------------------------------- observables
// The moments of the Jastrow observables kernel, with the two-flip ratios computed directly:
// log r_jk = -2 a_j s_j - 2 a_k s_k + sum_m [lc(gamma_m - 2 W_jm s_j - 2 W_km s_k) - lc(gamma_m)].
// Thread (g, j), samples blk * SB + g + q SPP, SB = SPP * spt.
template <typename R2>
__global__ void __launch_bounds__(256) obs_rbm_kernel(int n, int M, int W, int P, int ns, int spt,
                                                      const double2* __restrict__ theta,
                                                      const uint64_t* __restrict__ spins,
                                                      const R2* __restrict__ r, double* __restrict__ part_obs) {
    const int NT = ((n + 31) / 32) * 32;
    const int SPP = 256 / NT;
    const int SB = SPP * spt;
    const int t = blockIdx.y, blk = blockIdx.x;
    const int j = threadIdx.x % NT, g = threadIdx.x / NT;
    const bool active = (g < SPP) && (j < n);
    extern __shared__ __align__(16) unsigned char smraw[];
    double2* gs = (double2*)smraw;   // [SPP][M]
    double2* ls = gs + SPP * M;      // [SPP][M]
    uint64_t* sw = (uint64_t*)(ls + SPP * M);  // [SPP][W]
    __shared__ double red[256 * 9];
    const RbmTheta th = rbm_split(theta, P, n, M, t);
    double acc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = 0.0;
    for (int q = 0; q < spt; ++q) {
        __syncthreads();
        for (int i = threadIdx.x; i < SPP * W; i += blockDim.x) {
            const int gg = i / W, w = i - gg * W;
            const int s = blk * SB + gg + q * SPP;
            sw[i] = s < ns ? spins[((size_t)t * ns + s) * W + w] : 0ull;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < SPP * M; i += blockDim.x) {
            const int gg = i / M, m = i - gg * M;
            const uint64_t* w = sw + gg * W;
            double2 z = th.b[m];
            for (int k = 0; k < n; ++k) {
                const double sk = ((w[k >> 6] >> (k & 63)) & 1ull) ? 1.0 : -1.0;
                z.x += th.W[(size_t)k * M + m].x * sk;
                z.y += th.W[(size_t)k * M + m].y * sk;
            }
            gs[i] = z;
            ls[i] = lc2(z);
        }
        __syncthreads();
        const int s = blk * SB + g + q * SPP;
        if (!(active && s < ns)) continue;
        const uint64_t* w = sw + g * W;
        int S = 0;
        for (int ww = 0; ww < W; ++ww) S += 2 * __popcll(w[ww]);
        S -= n;
        const double sj = ((w[j >> 6] >> (j & 63)) & 1ull) ? 1.0 : -1.0;
        double2 A = make_double2(0.0, 0.0), B = make_double2(0.0, 0.0);
        for (int k = 0; k < n; ++k) {
            if (k == j) continue;
            const double sk = ((w[k >> 6] >> (k & 63)) & 1ull) ? 1.0 : -1.0;
            double2 lr = make_double2(-2.0 * (th.a[j].x * sj + th.a[k].x * sk), -2.0 * (th.a[j].y * sj + th.a[k].y * sk));
            for (int m = 0; m < M; ++m) {
                const double2 z = gs[g * M + m];
                const double2 wj = th.W[(size_t)j * M + m], wk = th.W[(size_t)k * M + m];
                const double2 z1 = make_double2(z.x - 2.0 * (wj.x * sj + wk.x * sk), z.y - 2.0 * (wj.y * sj + wk.y * sk));
                lr = cadd(lr, csub(lc2(z1), ls[g * M + m]));
            }
            const double2 rjk = cexp2(lr);
            A = cadd(A, rjk);
            B = cadd(B, cscale(rjk, sk));
        }
        const R2 rr = r[((size_t)t * ns + s) * n + j];
        const double2 rj = make_double2((double)rr.x, (double)rr.y);
        acc[0] += rj.x;
        acc[1] += sj * rj.y;
        acc[2] += sj;
        acc[3] += A.x;
        acc[4] += -sj * B.x;
        if (j == 0) acc[5] += (double)S * S - n;
        acc[6] += B.y;
        acc[7] += rj.x * (S - sj);
        acc[8] += sj * rj.y * (S - sj);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 9; ++i) red[threadIdx.x * 9 + i] = acc[i];
    __syncthreads();
    if (threadIdx.x < 9) {
        double sum = 0.0;
        for (int k = 0; k < 256; ++k) sum += red[k * 9 + threadIdx.x];
        part_obs[((size_t)t * gridDim.x + blk) * 9 + threadIdx.x] = sum;
    }
}

cudaError_t launch_obs_rbm(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int ntraj, int ns,
                           bool fp32, const EvalBufs& b, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_OBS, s);
    const int n = a->n, M = a->m, W = (n + 63) / 64;
    const int NT = ((n + 31) / 32) * 32, SPP = 256 / NT;
    const size_t smem = (size_t)2 * SPP * M * 16 + (size_t)SPP * W * 8 + 64;
    dim3 grid(obs_blocks(n, ns), ntraj);
    cudaError_t e;
    if (fp32) {
        e = cudaFuncSetAttribute(obs_rbm_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        obs_rbm_kernel<float2><<<grid, 256, smem, s>>>(n, M, W, (int)a->P, ns, obs_samples_per_thread(), theta, spins,
                                                       reinterpret_cast<const float2*>(b.r), b.part_obs);
    } else {
        e = cudaFuncSetAttribute(obs_rbm_kernel<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        obs_rbm_kernel<double2><<<grid, 256, smem, s>>>(n, M, W, (int)a->P, ns, obs_samples_per_thread(), theta,
                                                        spins, b.r, b.part_obs);
    }
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ build and solve
size_t rbm_build_bytes(const otvmc_ansatz* a, int ntraj, int ns) {
    const size_t P = (size_t)a->P, M = (size_t)a->m, T = (size_t)ntraj;
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t mx = P > (size_t)ns ? P : (size_t)ns;
    const size_t big = 4 * mx * mx;  // embedded S (2P x 2P, stage build) or T (2 ns x 2 ns)
    const size_t rhs = 2 * mx;
    return r(T * M * ns * 16) + r(T * 4 * P * ns * 8) + r(T * big * 8) + 2 * r(T * rhs * 16) + r(T * P * 16);
}

struct RbmBuild {
    double2* Th;
    double* R;
    double* E;      // embedded S (2P x 2P) or T (2ns x 2ns)
    double2* rhs;   // embedded right-hand side / solution
    double2* sol;
    double2* obar;  // complex column means
};
static RbmBuild carve_rbm(void* ws, const otvmc_ansatz* a, int ntraj, int ns) {
    const size_t P = (size_t)a->P, M = (size_t)a->m, T = (size_t)ntraj;
    char* p = (char*)ws;
    auto take = [&](size_t b) {
        char* q = p;
        p += (b + 255) & ~(size_t)255;
        return (void*)q;
    };
    const size_t mx = P > (size_t)ns ? P : (size_t)ns;
    const size_t big = 4 * mx * mx;
    const size_t rhs = 2 * mx;
    RbmBuild r;
    r.Th = (double2*)take(T * M * ns * 16);
    r.R = (double*)take(T * 4 * P * ns * 8);
    r.E = (double*)take(T * big * 8);
    r.rhs = (double2*)take(T * rhs * 16);
    r.sol = (double2*)take(T * rhs * 16);
    r.obar = (double2*)take(T * P * 16);
    return r;
}

cudaError_t launch_syrk_f64_scaled(int ntraj, int rows, int K, double inv, const double* O, double* S, cudaStream_t s);

// Common front part: tanh, column means, R in the layout the path needs.
static cudaError_t rbm_front(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int T, int ns,
                             const RbmBuild& rb, bool kmajor, cudaStream_t s) {
    const int n = a->n, M = a->m, W = (n + 63) / 64, P = (int)a->P;
    {
        ProfScope prof_(OTVMC_K_OBUILD, s);
        rbm_tanh_kernel<<<dim3((ns + 255) / 256, M, T), 256, 0, s>>>(n, M, W, P, ns, theta, spins, rb.Th);
        count_launch();
        rbm_obar_kernel<<<dim3((P + 7) / 8, T), 256, 0, s>>>(n, M, W, P, ns, spins, rb.Th, rb.obar);
        count_launch();
        rbm_R_kernel<<<dim3(512, T), 256, 0, s>>>(n, M, W, P, ns, kmajor ? 1 : 0, spins, rb.Th, rb.obar, rb.R);
        count_launch();
    }
    return cudaGetLastError();
}

// S path (build): embedded S and D; writes complex S (optional), obar (complex) and D.
cudaError_t launch_rbm_build(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, const double2* v,
                             const double* vinfo, int T, int ns, void* ws, double2* S_out, double2* obar_out,
                             double2* D_out, cudaStream_t s) {
    const int P = (int)a->P;
    RbmBuild rb = carve_rbm(ws, a, T, ns);
    cudaError_t e = rbm_front(a, theta, spins, T, ns, rb, true, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof_(OTVMC_K_D, s);
        rbm_vtilde_kernel<<<dim3((2 * ns + 255) / 256, T), 256, 0, s>>>(ns, v, vinfo, rb.rhs);
        rbm_gemv_kernel<<<dim3((2 * P + 7) / 8, T), 256, 0, s>>>(P, ns, 1, 1.0 / ns, rb.R, rb.rhs, rb.sol);
        rbm_unpack_kernel<<<dim3((P + 255) / 256, T), 256, 0, s>>>(P, rb.sol, D_out);
        count_launch(3);
    }
    if (S_out) {
        e = launch_syrk_f64_scaled(T, 2 * P, 2 * ns, 1.0 / ns, rb.R, rb.E, s);
        if (e != cudaSuccess) return e;
        rbm_extract_S_kernel<<<dim3(256, T), 256, 0, s>>>(P, rb.E, S_out);
        count_launch();
    }
    if (obar_out) {
        e = cudaMemcpyAsync(obar_out, rb.obar, (size_t)T * P * 16, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_chol_solve(int ntraj, int P, int ns, int precision, double eps, const double* S, const float* G,
                              const double* obar, const double2* D, double2* delta, double* shift_used, void* ws,
                              int refine_iters, int* status, cudaStream_t s);

size_t chol_ws_bytes(int ntraj, int P, int precision);

// Stage solve from a complex S: embed, real FP64 Cholesky of size 2P, unpack.
size_t rbm_solve_bytes(int ntraj, int P) {
    auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t T = (size_t)ntraj;
    return r(T * 4 * P * P * 8) + 2 * r(T * 2 * P * 16) + chol_ws_bytes(ntraj, 2 * P, OTVMC_PREC_FP64);
}
cudaError_t launch_rbm_solve_S(const otvmc_ansatz* a, int T, int ns, double eps, const double2* S, const double2* D,
                               double2* delta, double* shift_used, void* ws, int* status, cudaStream_t s) {
    const int P = (int)a->P;
    char* p = (char*)ws;
    auto take = [&](size_t b) {
        char* q = p;
        p += (b + 255) & ~(size_t)255;
        return (void*)q;
    };
    double* E = (double*)take((size_t)T * 4 * P * P * 8);
    double2* rhs = (double2*)take((size_t)T * 2 * P * 16);
    double2* sol = (double2*)take((size_t)T * 2 * P * 16);
    void* chol = p;
    rbm_embed_S_kernel<<<dim3(256, T), 256, 0, s>>>(P, S, E);
    rbm_embed_D_kernel<<<dim3((P + 255) / 256, T), 256, 0, s>>>(P, D, rhs);
    count_launch(2);
    cudaError_t e = launch_chol_solve(T, 2 * P, ns, OTVMC_PREC_FP64, eps, E, nullptr, nullptr, rhs, sol, shift_used,
                                      chol, 1, status, s);
    if (e != cudaSuccess) return e;
    rbm_unpack_kernel<<<dim3((P + 255) / 256, T), 256, 0, s>>>(P, sol, delta);
    count_launch();
    return cudaGetLastError();
}

// Whole evaluation's build + solve (run path): S path when P <= ns, else the T path.
cudaError_t launch_rbm_build_solve(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, const double2* v,
                                   const double* vinfo, int T, int ns, double eps, void* ws, void* chol,
                                   double2* delta, int* status, cudaStream_t s) {
    const int P = (int)a->P;
    RbmBuild rb = carve_rbm(ws, a, T, ns);
    const bool tpath = P > ns;
    cudaError_t e = rbm_front(a, theta, spins, T, ns, rb, !tpath, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof_(OTVMC_K_D, s);
        rbm_vtilde_kernel<<<dim3((2 * ns + 255) / 256, T), 256, 0, s>>>(ns, v, vinfo, rb.rhs);
        count_launch();
    }
    if (!tpath) {
        {
            ProfScope prof_(OTVMC_K_D, s);
            rbm_gemv_kernel<<<dim3((2 * P + 7) / 8, T), 256, 0, s>>>(P, ns, 1, 1.0 / ns, rb.R, rb.rhs, rb.sol);
            count_launch();
        }
        e = launch_syrk_f64_scaled(T, 2 * P, 2 * ns, 1.0 / ns, rb.R, rb.E, s);
        if (e != cudaSuccess) return e;
        // solve (E + eps I) x = [Re D; Im D]
        e = launch_chol_solve(T, 2 * P, ns, OTVMC_PREC_FP64, eps, rb.E, nullptr, nullptr, rb.sol, rb.rhs, nullptr, chol,
                              1, status, s);
        if (e != cudaSuccess) return e;
        rbm_unpack_kernel<<<dim3((P + 255) / 256, T), 256, 0, s>>>(P, rb.rhs, delta);
        count_launch();
        return cudaGetLastError();
    }
    // T path: (T~ + eps I) y = v~, then delta~ = R^T y / ns
    e = launch_syrk_f64_scaled(T, 2 * ns, 2 * P, 1.0 / ns, rb.R, rb.E, s);
    if (e != cudaSuccess) return e;
    e = launch_chol_solve(T, 2 * ns, ns, OTVMC_PREC_FP64, eps, rb.E, nullptr, nullptr, rb.rhs, rb.sol, nullptr, chol, 1,
                          status, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof_(OTVMC_K_D, s);
        rbm_gemv_kernel<<<dim3((2 * P + 255) / 256, T), 256, 0, s>>>(P, ns, 0, 1.0 / ns, rb.R, rb.sol, rb.rhs);
        rbm_unpack_kernel<<<dim3((P + 255) / 256, T), 256, 0, s>>>(P, rb.rhs, delta);
        count_launch(2);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------ mixed build and solve
// R (as above) in FP32, written as three BF16 pieces r = h + m + l stacked along the row:
// kmajor: Xs[t][k'][p * kpad + x'] (rows = 2P parameters, K = 2 ns samples), else
// Xs[t][x'][p * kpad + k'] (rows = 2 ns samples, K = 2P parameters); columns K .. kpad zero.
__device__ __forceinline__ void split3(float v, uint16_t& h, uint16_t& m, uint16_t& l) {
    const __nv_bfloat16 bh = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(bh);
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const __nv_bfloat16 bl = __float2bfloat16_rn(r1 - __bfloat162float(bm));
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}

__global__ void __launch_bounds__(256) rbm_Xsplit_kernel(int n, int M, int W, int P, int ns, int kmajor, int kpad,
                                                         const uint64_t* __restrict__ spins,
                                                         const double2* __restrict__ Th,
                                                         const double2* __restrict__ obar, uint16_t* __restrict__ Xs) {
    const int t = blockIdx.y;
    const uint64_t* sp = spins + (size_t)t * ns * W;
    const double2* Tht = Th + (size_t)t * M * ns;
    const int rows = kmajor ? 2 * P : 2 * ns, K = kmajor ? 2 * ns : 2 * P;
    uint16_t* X = Xs + (size_t)t * rows * 3 * kpad;
    const size_t rs = (size_t)3 * kpad;  // row stride
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)P * ns; e += (size_t)gridDim.x * blockDim.x) {
        int k, x;
        if (kmajor) {
            k = (int)(e / ns);
            x = (int)(e - (size_t)k * ns);
        } else {
            x = (int)(e / P);
            k = (int)(e - (size_t)x * P);
        }
        const double2 o = csub(rbm_O(sp, W, n, M, ns, Tht, k, x), obar[(size_t)t * P + k]);
        // the four entries of R for (x, k): (x, k) = Re, (x, P+k) = -Im, (ns+x, k) = Im, (ns+x, P+k) = Re
        const float vr = (float)o.x, vi = (float)o.y;
        uint16_t hr, mr, lr, hi, mi, li, hn, mn, ln;
        split3(vr, hr, mr, lr);
        split3(vi, hi, mi, li);
        split3(-vi, hn, mn, ln);
        size_t a0, a1, a2, a3;  // (row, column) of the four entries
        if (kmajor) {  // rows parameters, columns samples
            a0 = (size_t)k * rs + x;
            a1 = (size_t)(P + k) * rs + x;
            a2 = (size_t)k * rs + ns + x;
            a3 = (size_t)(P + k) * rs + ns + x;
        } else {
            a0 = (size_t)x * rs + k;
            a1 = (size_t)x * rs + P + k;
            a2 = (size_t)(ns + x) * rs + k;
            a3 = (size_t)(ns + x) * rs + P + k;
        }
        X[a0] = hr; X[a0 + kpad] = mr; X[a0 + 2 * kpad] = lr;
        X[a1] = hn; X[a1 + kpad] = mn; X[a1 + 2 * kpad] = ln;
        X[a2] = hi; X[a2 + kpad] = mi; X[a2 + 2 * kpad] = li;
        X[a3] = hr; X[a3 + kpad] = mr; X[a3 + 2 * kpad] = lr;
    }
    const int padc = kpad - K;
    if (padc > 0)
        for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)rows * 3 * padc;
             e += (size_t)gridDim.x * blockDim.x) {
            const size_t r = e / (3 * padc), q = e - r * 3 * padc, pc = q / padc, c = q - pc * padc;
            X[r * rs + pc * kpad + K + c] = 0;
        }
}

__device__ __forceinline__ float bf16v(uint16_t u) { return __bfloat162float(__ushort_as_bfloat16(u)); }

// out[k'] = inv sum_x' R[x'][k'] u[x'].x over the split pieces (k' < 2P); kmajor: one warp per
// k' along the contiguous samples, else one thread per k'.  Runs of FP32 products, FP64 sums.
__global__ void __launch_bounds__(256) rbm_split_gemv_kernel(int P, int ns, int kmajor, int kpad, double inv,
                                                             const uint16_t* __restrict__ Xs,
                                                             const double2* __restrict__ u, double2* __restrict__ out) {
    const int t = blockIdx.y;
    const size_t NS2 = 2 * (size_t)ns, P2 = 2 * (size_t)P, rs = (size_t)3 * kpad;
    const size_t rows = kmajor ? P2 : NS2;
    const uint16_t* X = Xs + (size_t)t * rows * rs;
    const double2* ut = u + (size_t)t * NS2;
    if (kmajor) {
        const int k = blockIdx.x * 8 + threadIdx.x / 32, lane = threadIdx.x & 31;
        if (k >= 2 * P) return;
        const uint16_t* row = X + (size_t)k * rs;
        double a = 0.0;
        for (size_t x = lane; x < NS2; x += 32) {
            const float r = bf16v(row[x]) + bf16v(row[kpad + x]) + bf16v(row[2 * kpad + x]);
            a = fma((double)r, ut[x].x, a);
        }
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) out[(size_t)t * P2 + k] = make_double2(a * inv, 0.0);
    } else {
        const int k = blockIdx.x * blockDim.x + threadIdx.x;
        if (k >= 2 * P) return;
        double a = 0.0;
        for (size_t x0 = 0; x0 < NS2; x0 += 64) {
            float f = 0.f;
            const size_t xe = x0 + 64 < NS2 ? x0 + 64 : NS2;
            for (size_t x = x0; x < xe; ++x) {
                const uint16_t* e = X + x * rs + k;
                const float r = bf16v(e[0]) + bf16v(e[kpad]) + bf16v(e[2 * kpad]);
                f = fmaf(r, (float)ut[x].x, f);
            }
            a += (double)f;
        }
        out[(size_t)t * P2 + k] = make_double2(a * inv, 0.0);
    }
}

static size_t rup(size_t b) { return (b + 255) & ~(size_t)255; }
static int kpad64(int k) { return (k + 63) / 64 * 64; }

size_t chol_ws_bytes(int ntraj, int P, int precision);

size_t rbm_mixed_bytes(const otvmc_ansatz* a, int ntraj, int ns) {
    const size_t P = (size_t)a->P, M = (size_t)a->m, T = (size_t)ntraj;
    const bool tpath = P > (size_t)ns;
    if (tpath && a->rbm_t_build == OTVMC_RBM_T_FACTORED) return rbm_factored_bytes(a, ntraj, ns);
    const size_t rows = tpath ? 2 * (size_t)ns : 2 * P, K = tpath ? 2 * P : 2 * (size_t)ns;
    const size_t kp = (size_t)kpad64((int)K);
    const size_t mx = P > (size_t)ns ? P : (size_t)ns;
    return rup(T * M * ns * 16) + rup(T * P * 16) + rup(T * rows * 3 * kp * 2) + rup(T * rows * rows * 4) +
           rup(T * rows * 8) + 2 * rup(T * 2 * mx * 16) + rbm_refine_bytes(a, ntraj, ns) +
           (tpath ? 0 : rup(T * 2 * P * 16)) + rup(T * 8) + rbm_tanh_obar_bytes(a, ntraj) +
           chol_ws_bytes(ntraj, (int)rows, OTVMC_PREC_MIXED) + 1024;
}

cudaError_t launch_gram_split(int ntraj, int rows, int K, int kpad, const uint16_t* Xs, float* G, int* status,
                              cudaStream_t s);

// Whole evaluation's build + solve on the tensor cores: R in three BF16 pieces, the split Gram
// R^T R or R R^T in FP32 (six piece products), the mixed Cholesky of size 2P or 2 ns with it as
// its matrix (obar = 0: R is centred), then corrections against the FP64 operator applied
// through the factorisation of O (k_rbm_factored.cu) and delta in FP64.
// On the T path the ansatz's default (OTVMC_RBM_T_FACTORED) forms T without R instead.
cudaError_t launch_rbm_build_solve_mixed(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins,
                                         const double2* v, const double* vinfo, int T, int ns, double eps, void* ws,
                                         double2* delta, int* status, cudaStream_t s) {
    const int P = (int)a->P, n = a->n, M = a->m, W = (n + 63) / 64;
    const bool tpath = P > ns;
    if (tpath && a->rbm_t_build == OTVMC_RBM_T_FACTORED)
        return launch_rbm_build_solve_factored(a, theta, spins, v, vinfo, T, ns, eps, ws, delta, status, s);
    const int rows = tpath ? 2 * ns : 2 * P, K = tpath ? 2 * P : 2 * ns, kp = kpad64(K);
    const size_t mx = (size_t)(P > ns ? P : ns);
    char* q = (char*)ws;
    auto take = [&](size_t b) {
        char* r = q;
        q += rup(b);
        return (void*)r;
    };
    double2* Th = (double2*)take((size_t)T * M * ns * 16);
    double2* obar = (double2*)take((size_t)T * P * 16);
    uint16_t* Xs = (uint16_t*)take((size_t)T * rows * 3 * kp * 2);
    float* Gs = (float*)take((size_t)T * rows * rows * 4);
    double* zero = (double*)take((size_t)T * rows * 8);
    double2* rhs = (double2*)take((size_t)T * 2 * mx * 16);
    double2* sol = (double2*)take((size_t)T * 2 * mx * 16);
    void* rws = take(rbm_refine_bytes(a, T, ns));
    double2* xe = tpath ? nullptr : (double2*)take((size_t)T * 2 * P * 16);
    unsigned long long* fmax = (unsigned long long*)take((size_t)T * 8);
    void* tws = take(rbm_tanh_obar_bytes(a, T));
    void* chol = q;
    cudaError_t e = launch_rbm_tanh_obar(a, theta, spins, T, ns, Th, nullptr, fmax, obar, tws, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof_(OTVMC_K_OBUILD, s);
        rbm_Xsplit_kernel<<<dim3(1024, T), 256, 0, s>>>(n, M, W, P, ns, tpath ? 0 : 1, kp, spins, Th, obar, Xs);
        rbm_vtilde_kernel<<<dim3((2 * ns + 255) / 256, T), 256, 0, s>>>(ns, v, vinfo, rhs);
        count_launch(2);
    }
    e = cudaMemsetAsync(zero, 0, (size_t)T * rows * 8, s);
    if (e != cudaSuccess) return e;
    e = launch_gram_split(T, rows, K, kp, Xs, Gs, status, s);
    if (e != cudaSuccess) return e;
    if (!tpath) {
        {
            ProfScope prof_(OTVMC_K_D, s);
            rbm_split_gemv_kernel<<<dim3((2 * P + 7) / 8, T), 256, 0, s>>>(P, ns, 1, kp, 1.0 / ns, Xs, rhs, sol);
            count_launch();
        }
        // (S~ + eps I) x = [Re D~; Im D~], S~ = Gs / ns, then corrections against the FP64 operator
        e = launch_chol_solve(T, rows, ns, OTVMC_PREC_MIXED, eps, nullptr, Gs, zero, sol, xe, nullptr, chol, 0,
                              status, s);
        if (e != cudaSuccess) return e;
        return launch_rbm_refine_S(a, T, ns, eps, RBM_REFINE_MATERIALISED, spins, Th, fmax, obar, rhs, xe, chol, rws,
                                   delta, s);
    }
    // (T~ + eps I) y = v~, T~ = Gs / ns, then corrections against the FP64 operator (through the
    // factorisation of O with the FP64 tanh gamma and obar) and delta = O_c^+ y / ns in FP64
    e = launch_chol_solve(T, rows, ns, OTVMC_PREC_MIXED, eps, nullptr, Gs, zero, rhs, sol, nullptr, chol, 0, status,
                          s);
    if (e != cudaSuccess) return e;
    return launch_rbm_refine_push(a, T, ns, eps, RBM_REFINE_MATERIALISED, spins, Th, fmax, obar, rhs, sol, chol, rws,
                                  delta, s);
}

}  // namespace otvmc
