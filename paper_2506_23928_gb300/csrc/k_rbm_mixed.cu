// RBM ansatz (Eq. 11), FP32 sampling and local estimators.
//
// Sampling: one warp per Markov chain, the lanes over the hidden units (lane l owns units
// l, l + 32, ...), the chain's angles gamma_m in FP32 registers, updated on accepted flips.
// A proposal at site j is accepted iff u < exp(2 Re log r_j) with
//     Re log r_j = -2 Re(a_j) s_j + sum_m [Re lc(gamma_m - 2 W_jm s_j) - Re lc(gamma_m)],
//     Re lc(x + iy) = log |2 cosh(x + iy)| = |x| + log1p(e (2 cos 2y + e)) / 2,  e = exp(-2|x|).
// Each term carries an error bound: rounding of |x|, of the transcendentals and of
// t = e (2 cos 2y + e) (amplified by 1 / (1 + t) near a zero of cosh), plus the error of the
// FP32 angles (a per-unit bound summed as the angle is formed and updated: 2^-24 of every
// rounded parameter and of every rounded sum) times |tanh gamma| (the derivative of Re lc).  When
// |Re log r_j - log u| is within twice the summed bound the proposal is decided in FP64 from
// the parameters, so every accept/reject equals the FP64 decision.
//
// Local estimators: the blocking of the Jastrow est1 kernel (thread (g, j) = site j of
// samples g, g + SPP, ...), angles and lc(gamma) per sample in shared memory, FP32 complex
// log 2cosh, flip ratios stored as float2.
#include "common.cuh"

namespace otvmc {

constexpr int RBM_MQ = 8;  // hidden units per lane: M <= 256

struct RelcF {
    float v;    // Re lc
    float err;  // bound of |computed - exact| for an exact input
    float dtn;  // |tanh z|, the derivative bound
};
__device__ __forceinline__ RelcF relc_f(float x, float y) {
    const float ax = fabsf(x);
    const float e = expf(-2.f * ax);
    const float c2 = cosf(2.f * y);
    const float t = e * (2.f * c2 + e);
    const float opt = 1.f + t;  // |2 cosh z|^2 e^{-2|x|} / 4 >= 0
    RelcF r;
    r.v = ax + 0.5f * log1pf(t);
    // near a zero of cosh the bound is not meaningful: force the FP64 decision
    const bool ok = opt > 1e-3f;
    r.err = ok ? 5.9604645e-8f * (ax + 8.f + 16.f / opt) : 1e30f;
    const float num = fmaxf(1.f + e * e - 2.f * e * c2, 0.f);
    r.dtn = ok ? sqrtf(num / opt) : 1e30f;
    return r;
}
__device__ __forceinline__ double relc_d(double x, double y) {
    const double ax = fabs(x);
    const double e = exp(-2.0 * ax);
    return ax + 0.5 * log1p(e * (2.0 * cos(2.0 * y) + e));
}

// WS: the weights W_jm as float2 in shared memory ([n][M], when they fit), else read from theta.
// MQ: hidden units per lane (M <= 32 MQ).
template <bool WS, int MQ>
__global__ void __launch_bounds__(256) sample_rbm_mixed_kernel(const double2* __restrict__ theta, int P, int n, int M,
                                                               int W, int ns, int n_sweep, uint32_t k0, uint32_t k1,
                                                               uint32_t evtag, int traj0, uint64_t* __restrict__ spins,
                                                               unsigned long long* __restrict__ accepted) {
    extern __shared__ float2 wsm[];
    const int t = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double2* th = theta + (size_t)t * P;
    const double2* a = th;
    const double2* b = th + n;
    const double2* Wt = th + n + M;
    if (WS)
        for (int e = threadIdx.x; e < n * M; e += blockDim.x) wsm[e] = make_float2((float)Wt[e].x, (float)Wt[e].y);
    if (WS) __syncthreads();
    const int chain = blockIdx.x * (blockDim.x >> 5) + warp;
    if (chain >= ns) return;
    uint64_t* sp = spins + ((size_t)t * ns + chain) * W;
    uint64_t wd[4];
#pragma unroll
    for (int w = 0; w < 4; ++w) wd[w] = w < W ? sp[w] : 0ull;
    auto spin = [&](int i) -> float {
        const int w = i >> 6;
        const uint64_t v = w == 0 ? wd[0] : w == 1 ? wd[1] : w == 2 ? wd[2] : wd[3];
        return ((v >> (i & 63)) & 1ull) ? 1.f : -1.f;
    };
    // angles, and Re lc with its error bound and |tanh| at the current angles (kept across
    // proposals, replaced on acceptance by the values of the accepted angles).  eb bounds the
    // error of either FP32 angle component against the exact angle: the rounding of b and of
    // every W_im taken (2^-24 of each), of every FP32 sum formed (2^-24 of the result), summed
    // as they happen.
    constexpr float U = 5.9604645e-8f * 1.001f;  // 2^-24, rounded up
    float gx[MQ], gy[MQ], l0[MQ], e0[MQ], d0[MQ], eb[MQ];
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
        const int m = lane + 32 * q;
        gx[q] = gy[q] = l0[q] = e0[q] = d0[q] = eb[q] = 0.f;
        if (m < M) {
            float zx = (float)b[m].x, zy = (float)b[m].y;
            float ex = U * fabsf(zx), ey = U * fabsf(zy);
            for (int i = 0; i < n; ++i) {
                const float si = spin(i);
                const double2 w = Wt[(size_t)i * M + m];
                const float wx = (float)w.x, wy = (float)w.y;
                zx = fmaf(wx, si, zx);
                zy = fmaf(wy, si, zy);
                ex += U * (fabsf(zx) + fabsf(wx));
                ey += U * (fabsf(zy) + fabsf(wy));
            }
            gx[q] = zx;
            gy[q] = zy;
            eb[q] = fmaxf(ex, ey) * 1.001f;
            const RelcF r0 = relc_f(zx, zy);
            l0[q] = r0.v;
            e0[q] = r0.err;
            d0[q] = r0.dtn;
        }
    }
    const int nprop = n_sweep * n;
    int nacc = 0;
    u32x4 draw = {0u, 0u, 0u, 0u};
    for (int p = 0; p < nprop; ++p) {
        if ((p & 1) == 0) draw = philox(u32x4{(uint32_t)(p / 2), (uint32_t)chain, (uint32_t)(traj0 + t), evtag}, k0, k1);
        const uint32_t wsite = (p & 1) ? draw.z : draw.x;
        const uint32_t wu = (p & 1) ? draw.w : draw.y;
        const int j = (int)(((unsigned long long)wsite * (unsigned long long)n) >> 32);
        const float sj = spin(j);
        float s = 0.f, err = 0.f;
        float nx[MQ], ny[MQ], l1[MQ], e1[MQ], d1[MQ], eb1[MQ];
#pragma unroll
        for (int q = 0; q < MQ; ++q) {
            const int m = lane + 32 * q;
            nx[q] = gx[q];
            ny[q] = gy[q];
            l1[q] = e1[q] = d1[q] = eb1[q] = 0.f;
            if (m < M) {
                float2 w;
                if (WS) {
                    w = wsm[j * M + m];
                } else {
                    const double2 wd2 = Wt[(size_t)j * M + m];
                    w = make_float2((float)wd2.x, (float)wd2.y);
                }
                // the angles after the flip: -2 s_j w is exact, so one rounding of the sum,
                // plus the rounding of W_jm to FP32 (twice, through the factor 2)
                nx[q] = fmaf(-2.f * sj, w.x, gx[q]);
                ny[q] = fmaf(-2.f * sj, w.y, gy[q]);
                eb1[q] = eb[q] + U * (fmaxf(fabsf(nx[q]), fabsf(ny[q])) + 2.f * fmaxf(fabsf(w.x), fabsf(w.y)));
                const RelcF r1 = relc_f(nx[q], ny[q]);
                l1[q] = r1.v;
                e1[q] = r1.err;
                d1[q] = r1.dtn;
                const float term = r1.v - l0[q];
                s += term;
                // evaluation and angle errors, plus the rounding of the term and of the
                // summation (at most MQ + 6 roundings on the way to the total)
                err += r1.err + e0[q] + 2.f * (eb1[q] * r1.dtn + eb[q] * d0[q]) +
                       5.9604645e-8f * (float)(MQ + 6) * (fabsf(term) + fabsf(r1.v) + fabsf(l0[q]));
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, off);
            err += __shfl_xor_sync(0xffffffffu, err, off);
        }
        // the butterfly leaves every lane with the same sums; take lane 0's all the same, so
        // that the decision is warp-uniform by construction
        s = __shfl_sync(0xffffffffu, s, 0);
        err = __shfl_sync(0xffffffffu, err, 0);
        const float aj = (float)a[j].x;
        const float lr = -2.f * aj * sj + s;  // Re log r_j; accept iff log u < 2 Re log r_j
        // u = (wu + 1/2) 2^-32 in FP32 (relative error <= 2^-24, inside the guard band below)
        const float lu = logf(fmaf((float)wu, 0x1.0p-32f, 0x1.0p-33f));
        const float guard = 4.f * (err + 1.2e-7f * fabsf(aj)) + 1e-6f + 4e-7f * fabsf(lu) + 2e-6f * fabsf(lr);
        const float d = 2.f * lr - lu;
        bool acc;
        if (d > guard) {
            acc = true;
        } else if (d < -guard) {
            acc = false;
        } else {
            // FP64 from the parameters
            double s64 = 0.0;
            for (int q = 0; q < MQ; ++q) {
                const int m = lane + 32 * q;
                if (m < M) {
                    double zx = b[m].x, zy = b[m].y;
                    for (int i = 0; i < n; ++i) {
                        const double si = spin(i);
                        zx += Wt[(size_t)i * M + m].x * si;
                        zy += Wt[(size_t)i * M + m].y * si;
                    }
                    const double2 w = Wt[(size_t)j * M + m];
                    s64 += relc_d(zx - 2.0 * w.x * sj, zy - 2.0 * w.y * sj) - relc_d(zx, zy);
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s64 += __shfl_xor_sync(0xffffffffu, s64, off);
            s64 = __shfl_sync(0xffffffffu, s64, 0);
            acc = u01(wu) < exp(2.0 * (-2.0 * a[j].x * sj + s64));
        }
        if (acc) {
#pragma unroll
            for (int q = 0; q < MQ; ++q) {
                gx[q] = nx[q];
                gy[q] = ny[q];
                l0[q] = l1[q];
                e0[q] = e1[q];
                d0[q] = d1[q];
                eb[q] = eb1[q];
            }
            const uint64_t bit = 1ull << (j & 63);
            const int w = j >> 6;
            if (w == 0) wd[0] ^= bit;
            if (w == 1) wd[1] ^= bit;
            if (w == 2) wd[2] ^= bit;
            if (w == 3) wd[3] ^= bit;
            ++nacc;
        }
    }
    if (lane < W) sp[lane] = lane == 0 ? wd[0] : lane == 1 ? wd[1] : lane == 2 ? wd[2] : wd[3];
    if (lane == 0 && accepted != nullptr && nacc) atomicAdd(accepted + t, (unsigned long long)nacc);
}

cudaError_t launch_sample_rbm_mixed(const otvmc_ansatz* an, const double2* theta, int ntraj, int traj0, int ns,
                                    int n_sweep, uint64_t seed, int64_t eval, uint64_t* spins,
                                    unsigned long long* accepted, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SAMPLE, s);
    if (an->m > 32 * RBM_MQ) return cudaErrorInvalidValue;
    const int n = an->n, W = (n + 63) / 64;
    const uint32_t evtag = (TAG_SAMPLE << 28) | ((uint32_t)eval & 0x0FFFFFFFu);
    const size_t wbytes = (size_t)n * an->m * sizeof(float2);
    const bool ws = wbytes <= 64 * 1024, small = an->m <= 128;
    // eight chains per CTA with four hidden units per lane; four with eight (more registers)
    const int cpb = small ? 8 : 4;
    dim3 grid((ns + cpb - 1) / cpb, ntraj);
    auto kern = ws ? (small ? sample_rbm_mixed_kernel<true, 4> : sample_rbm_mixed_kernel<true, RBM_MQ>)
                   : (small ? sample_rbm_mixed_kernel<false, 4> : sample_rbm_mixed_kernel<false, RBM_MQ>);
    const size_t smem = ws ? wbytes : 0;
    if (ws) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, 32 * cpb, smem, s>>>(theta, (int)an->P, n, an->m, W, ns, n_sweep, (uint32_t)seed, (uint32_t)(seed >> 32),
                                 evtag, traj0, spins, accepted);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------- local estimators
// log(2 cosh z) in FP32: s z + log1p(exp(-2 s z)), s = sign(Re z).
__device__ __forceinline__ float2 lc_f(float x, float y) {
    const float s = x >= 0.f ? 1.f : -1.f;
    const float e = expf(-2.f * s * x);
    float sn, cs;
    sincosf(2.f * y, &sn, &cs);
    const float wr = e * cs, wi = -s * e * sn;
    return make_float2(s * x + 0.5f * log1pf(2.f * wr + wr * wr + wi * wi), s * y + atan2f(wi, 1.f + wr));
}

template <bool WSMEM>
__global__ void __launch_bounds__(256) est_rbm_mixed_kernel(int n, int M, int W, int P, int ns, double h,
                                                            const double2* __restrict__ theta,
                                                            const uint64_t* __restrict__ spins,
                                                            const long long* __restrict__ QJ,
                                                            const long long* __restrict__ baseJ,
                                                            float2* __restrict__ r_out, double2* __restrict__ EH_out,
                                                            double2* __restrict__ part_r,
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
    float2* gs = (float2*)smraw;                  // [SPP][M] gamma
    float2* ls = gs + SPP * M;                    // [SPP][M] lc(gamma)
    double2* ered = (double2*)(ls + SPP * M);     // [SB][NT/32]
    uint64_t* sw = (uint64_t*)(ered + SB * (NT / 32));  // [SPP][W]
    float2* wf = (float2*)(sw + SPP * W);         // [n][M] W in FP32 (when it fits)
    __shared__ double2 red_r[256], red_sr[256];
    __shared__ double red_s[256];
    const double2* th = theta + (size_t)t * P;
    const double2* a = th;
    const double2* b = th + n;
    const double2* Wt = th + n + M;
    if (WSMEM)
        for (int i = threadIdx.x; i < n * M; i += blockDim.x) wf[i] = make_float2((float)Wt[i].x, (float)Wt[i].y);
    float2 pr = make_float2(0.f, 0.f), psr = make_float2(0.f, 0.f);
    int ps = 0;
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
            float zx = (float)b[m].x, zy = (float)b[m].y;
            for (int k = 0; k < n; ++k) {
                const float sk = ((w[k >> 6] >> (k & 63)) & 1ull) ? 1.f : -1.f;
                const float2 wk = WSMEM ? wf[k * M + m] : make_float2((float)Wt[(size_t)k * M + m].x,
                                                                      (float)Wt[(size_t)k * M + m].y);
                zx = fmaf(wk.x, sk, zx);
                zy = fmaf(wk.y, sk, zy);
            }
            gs[i] = make_float2(zx, zy);
            ls[i] = lc_f(zx, zy);
        }
        __syncthreads();
        const int sl = g + q * SPP;
        const int s = s0 + sl;
        float hrx = 0.f, hry = 0.f;
        long long isg = 0;
        if (active && s < ns) {
            const uint64_t* w = sw + g * W;
            const bool up = (w[j >> 6] >> (j & 63)) & 1ull;
            const float sj = up ? 1.f : -1.f;
            float lx = -2.f * (float)a[j].x * sj, ly = -2.f * (float)a[j].y * sj;
            for (int m = 0; m < M; ++m) {
                const float2 z = gs[g * M + m];
                const float2 wj = WSMEM ? wf[j * M + m] : make_float2((float)Wt[(size_t)j * M + m].x,
                                                                      (float)Wt[(size_t)j * M + m].y);
                const float2 l1 = lc_f(z.x - 2.f * wj.x * sj, z.y - 2.f * wj.y * sj);
                const float2 l0 = ls[g * M + m];
                lx += l1.x - l0.x;
                ly += l1.y - l0.y;
            }
            const float e = expf(lx);
            float sn, cs;
            sincosf(ly, &sn, &cs);
            const float2 r = make_float2(e * cs, e * sn);
            r_out[((size_t)t * ns + s) * n + j] = r;
            long long aj = 0;
            for (int k = 0; k < n; ++k)
                if ((w[k >> 6] >> (k & 63)) & 1ull) aj += QJ[(size_t)j * n + k];
            const long long fj = baseJ[j] + 2 * aj;
            isg = (up ? fj : -fj) >> 8;
            hrx = r.x;
            hry = r.y;
            pr.x += r.x;
            pr.y += r.y;
            psr.x += up ? r.x : -r.x;
            psr.y += up ? r.y : -r.y;
            ps += up ? 1 : -1;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            hrx += __shfl_xor_sync(0xffffffffu, hrx, off);
            hry += __shfl_xor_sync(0xffffffffu, hry, off);
            isg += __shfl_xor_sync(0xffffffffu, isg, off);
        }
        if (lane == 0 && g < SPP)
            ered[sl * (NT / 32) + wis] = make_double2(0.5 * (double)isg * 0x1.0p-40 + h * (double)hrx, h * (double)hry);
    }
    __syncthreads();
    if (threadIdx.x < SB) {
        const int sl = threadIdx.x, s = s0 + sl;
        if (s < ns) {
            double2 e = make_double2(0.0, 0.0);
            for (int w = 0; w < NT / 32; ++w) {
                e.x += ered[sl * (NT / 32) + w].x;
                e.y += ered[sl * (NT / 32) + w].y;
            }
            EH_out[(size_t)t * ns + s] = e;
        }
    }
    red_r[threadIdx.x] = make_double2((double)pr.x, (double)pr.y);
    red_sr[threadIdx.x] = make_double2((double)psr.x, (double)psr.y);
    red_s[threadIdx.x] = (double)ps;
    __syncthreads();
    if (threadIdx.x < n) {
        const int jj = threadIdx.x;
        double2 aa = make_double2(0, 0), bb = make_double2(0, 0);
        double c = 0.0;
        for (int gg = 0; gg < SPP; ++gg) {
            aa.x += red_r[gg * NT + jj].x;
            aa.y += red_r[gg * NT + jj].y;
            bb.x += red_sr[gg * NT + jj].x;
            bb.y += red_sr[gg * NT + jj].y;
            c += red_s[gg * NT + jj];
        }
        const size_t o = ((size_t)t * gridDim.x + blk) * n + jj;
        part_r[o] = aa;
        part_sr[o] = bb;
        part_s[o] = c;
    }
}

cudaError_t launch_est_rbm_mixed(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int ntraj,
                                 int ns, const EvalBufs& b, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_EST1, s);
    const int n = a->n, M = a->m, W = (n + 63) / 64;
    const int NT = ((n + 31) / 32) * 32, SPP = 256 / NT, SB = SPP * EST_SAMPLES_PER_THREAD;
    const size_t base = (size_t)2 * SPP * M * 8 + (size_t)SB * (NT / 32) * 16 + (size_t)SPP * W * 8 + 64;
    const size_t wbytes = (size_t)n * M * 8;
    const bool wsm = base + wbytes <= 160 * 1024;
    const size_t smem = base + (wsm ? wbytes : 0);
    const otvmc_model* m = a->model;
    dim3 grid(est_blocks(n, ns), ntraj);
    cudaError_t e;
    if (wsm) {
        e = cudaFuncSetAttribute(est_rbm_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        est_rbm_mixed_kernel<true><<<grid, 256, smem, s>>>(n, M, W, (int)a->P, ns, m->h, theta, spins, m->QJ_d,
                                                           m->baseJ_d, reinterpret_cast<float2*>(b.r), b.EH, b.part_r,
                                                           b.part_sr, b.part_s);
    } else {
        e = cudaFuncSetAttribute(est_rbm_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        est_rbm_mixed_kernel<false><<<grid, 256, smem, s>>>(n, M, W, (int)a->P, ns, m->h, theta, spins, m->QJ_d,
                                                            m->baseJ_d, reinterpret_cast<float2*>(b.r), b.EH,
                                                            b.part_r, b.part_sr, b.part_s);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
