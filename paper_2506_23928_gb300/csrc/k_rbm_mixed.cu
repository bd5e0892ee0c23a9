// RBM ansatz (Eq. 11), FP32 sampling and local estimators.
//
// Sampling: one warp per Markov chain, the lanes over the hidden units (lane l owns units
// l, l + 32, ...), the chain's angles gamma_m and tanh gamma_m in FP32 registers, updated on
// accepted flips.  A proposal at site j is accepted iff u < exp(2 Re log r_j) with
//     Re log r_j = -2 Re(a_j) s_j + sum_m Re log[cosh(gamma_m - 2 s_j W_jm) / cosh gamma_m],
//     cosh(g - 2 s W) / cosh g = cosh 2W - s tanh(g) sinh 2W = 1 + delta,
// so each term is (1/2) log1p(2 Re delta + |delta|^2) with delta small (of the order of
// |W tanh g|), from a per-trajectory table of cosh 2W - 1 and sinh 2W (FP64 rounded to FP32).
// Each term carries an error bound (of tanh g, itself bounded from the angle's accumulated
// rounding error, of the table and of the arithmetic).  When |2 Re log r_j - log u| is within
// four times the summed bound the proposal is decided in FP64 from the parameters, so every
// accept/reject equals the FP64 decision.
//
// Local estimators: the blocking of the Jastrow est1 kernel (thread (g, j) = site j of
// samples g, g + SPP, ...), angles and lc(gamma) per sample in shared memory, FP32 complex
// log 2cosh, flip ratios stored as float2.
#include "common.cuh"

namespace otvmc {

constexpr int RBM_MQ = 8;  // hidden units per lane: M <= 256

__device__ __forceinline__ double relc_d(double x, double y) {
    const double ax = fabs(x);
    const double e = exp(-2.0 * ax);
    return ax + 0.5 * log1p(e * (2.0 * cos(2.0 * y) + e));
}

// Flip factors of every weight, FP64 rounded to FP32: tab[t][i][m] = (cosh 2W_im - 1, sinh 2W_im),
// so that cosh(g - 2 s W) / cosh g = 1 + delta with delta = (cosh 2W - 1) - s tanh(g) sinh 2W.
// cosh(x + iy) - 1 = 2 sinh^2(x/2) cos y - 2 sin^2(y/2) + i sinh x sin y (no cancellation).
// Also W and a in FP32 (conversions from FP64 done once here, not in the samplers' loops).
struct RbmTabs {
    float4* flip;   // [T][n][M] (lanes over hidden units: the sampler)
    float4* flipT;  // [T][M][n] (lanes over sites: the estimators)
    float2* w;      // [T][n][M]
    float2* a;      // [T][n]
};
__host__ __device__ __forceinline__ RbmTabs rbm_tabs(float4* base, int T, int n, int M) {
    float4* ft = base + (size_t)T * n * M;
    float2* w = reinterpret_cast<float2*>(ft + (size_t)T * n * M);
    return RbmTabs{base, ft, w, w + (size_t)T * n * M};
}
__global__ void rbm_flip_table_kernel(const double2* __restrict__ theta, int P, int n, int M, float4* __restrict__ tab,
                                      float4* __restrict__ tabT, float2* __restrict__ wtab, float2* __restrict__ atab) {
    const int t = blockIdx.y;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        const double2 av = theta[(size_t)t * P + e];
        atab[(size_t)t * n + e] = make_float2((float)av.x, (float)av.y);
    }
    if (e >= n * M) return;
    const double2 w = theta[(size_t)t * P + n + M + e];
    wtab[(size_t)t * n * M + e] = make_float2((float)w.x, (float)w.y);
    const double x = 2.0 * w.x, y = 2.0 * w.y;
    double sy, cy, sh2, ch2;
    sincos(y, &sy, &cy);
    const double shx = sinh(x), chx = cosh(x), sx2 = sinh(0.5 * x), sy2 = sin(0.5 * y);
    ch2 = 2.0 * sx2 * sx2 * cy - 2.0 * sy2 * sy2;
    sh2 = shx * sy;
    const float4 f = make_float4((float)ch2, (float)sh2, (float)(shx * cy), (float)(chx * sy));
    tab[(size_t)t * n * M + e] = f;
    const int i = e / M, m = e - i * M;
    tabT[((size_t)t * M + m) * n + i] = f;
}

constexpr float UR = 5.9604645e-8f * 1.001f;  // 2^-24, rounded up

// tanh of an FP32 angle (error bound eb per component) and a bound of the error of the result:
// t = s (1 - w) / (1 + w), w = exp(-2 s g), s = sign(Re g).  |dw| <= 13 u (2 ulps of expf and of
// sincosf, the products; |w| <= 1) moves t by 2 |dw| / |1 + w|^2 (bounded with 30 u); the
// quotient adds about 10 u (1 + |t|); the
// angle error moves t by |1 - t^2| |dg| <= (1 + |t|^2) 2 eb.  Near a pole (|1 + w|^2 < 0.05) the
// bound is set huge, which sends every proposal touching the unit to the FP64 decision.
__device__ __forceinline__ void tanh_bound(float gx, float gy, float eb, float& tx, float& ty, float& et) {
    const float s = gx >= 0.f ? 1.f : -1.f;
    const float e = expf(-2.f * s * gx);
    float sn, cs;
    sincosf(2.f * gy, &sn, &cs);
    const float wr = e * cs, wi = -s * e * sn;
    const float dr = 1.f + wr, di = wi, nr = 1.f - wr, ni = -wi;
    const float den = dr * dr + di * di;
    const float inv = 1.f / den;
    tx = s * (nr * dr + ni * di) * inv;
    ty = s * (ni * dr - nr * di) * inv;
    const float at = fabsf(tx) + fabsf(ty);
    et = den > 0.05f ? UR * (30.f * inv + 10.f * (1.f + at)) + 2.f * eb * (1.f + at * at) : 1e30f;
}

// One warp per chain, lanes over the hidden units.  Per unit the lane keeps the FP32 angle g,
// the bound eb of its error (roundings of every parameter taken and every sum formed), t =
// tanh g and the bound et of its error.  The ratio term of a proposal is
//     Re lc(g - 2 s_j W_jm) - Re lc(g) = (1/2) log1p(2 Re delta + |delta|^2),
//     delta = (cosh 2W_jm - 1) - s_j t sinh 2W_jm  (from the flip table),
// a small number computed to a few ulps of itself; its bound adds the error of t, of the table
// entries and of the arithmetic.  WS: W_jm (needed on acceptance) as float2 in shared memory.
// MQ: hidden units per lane (M <= 32 MQ).
template <bool WS, int MQ>
__global__ void __launch_bounds__(MQ == 4 ? 256 : 128, MQ == 4 ? 3 : 4) sample_rbm_mixed_kernel(const double2* __restrict__ theta, int P, int n, int M,
                                                               int W, int ns, int n_sweep, uint32_t k0, uint32_t k1,
                                                               uint32_t evtag, int traj0, const float4* __restrict__ tab,
                                                               const float2* __restrict__ wtab,
                                                               const float2* __restrict__ atab,
                                                               uint64_t* __restrict__ spins,
                                                               unsigned long long* __restrict__ accepted) {
    extern __shared__ float2 wsm[];
    const int t = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double2* th = theta + (size_t)t * P;
    const double2* a = th;
    const double2* b = th + n;
    const double2* Wt = th + n + M;
    const float4* tb = tab + (size_t)t * n * M;
    const float2* wt32 = wtab + (size_t)t * n * M;
    const float2* at32 = atab + (size_t)t * n;
    if (WS) {
        for (int e = threadIdx.x; e < n * M; e += blockDim.x) wsm[e] = wt32[e];
        __syncthreads();
    }
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
    auto weight = [&](int i, int m) -> float2 { return WS ? wsm[i * M + m] : __ldg(wt32 + (size_t)i * M + m); };
    float gx[MQ], gy[MQ], eb[MQ], tx[MQ], ty[MQ], et[MQ];
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
        const int m = lane + 32 * q;
        gx[q] = gy[q] = eb[q] = tx[q] = ty[q] = et[q] = 0.f;
        if (m < M) {
            float zx = (float)b[m].x, zy = (float)b[m].y;
            float ex = UR * fabsf(zx), ey = UR * fabsf(zy);
            for (int i = 0; i < n; ++i) {
                const float si = spin(i);
                const float2 w = weight(i, m);
                zx = fmaf(w.x, si, zx);
                zy = fmaf(w.y, si, zy);
                ex += UR * (fabsf(zx) + fabsf(w.x));
                ey += UR * (fabsf(zy) + fabsf(w.y));
            }
            gx[q] = zx;
            gy[q] = zy;
            eb[q] = fmaxf(ex, ey) * 1.001f;
            tanh_bound(zx, zy, eb[q], tx[q], ty[q], et[q]);
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
#pragma unroll
        for (int q = 0; q < MQ; ++q) {
            const int m = lane + 32 * q;
            if (m < M) {
                const float4 f = __ldg(tb + (size_t)j * M + m);  // (cosh 2W - 1, sinh 2W)
                const float pr = tx[q] * f.z - ty[q] * f.w, pi = tx[q] * f.w + ty[q] * f.z;  // t sinh 2W
                const float dx = f.x - sj * pr, dy = f.y - sj * pi;
                const float ad = fabsf(dx) + fabsf(dy);                 // >= |delta|
                const float qv = fmaf(dx, dx, fmaf(dy, dy, 2.f * dx));  // |1 + delta|^2 - 1
                const float term = 0.5f * log1pf(qv);
                s += term;
                const float ash = fabsf(f.z) + fabsf(f.w), ac = fabsf(f.x) + fabsf(f.y);
                const float at = fabsf(tx[q]) + fabsf(ty[q]);
                // error of delta: t, the table's rounding (and its FP64 evaluation), the arithmetic
                const float ed = ash * et[q] + UR * (6.f * (ac + at * ash) + ad) + 1e-14f * ash * ash;
                const float eq = 2.f * (1.f + ad) * ed + ed * ed + 4.f * UR * (2.f * ad + ad * ad);
                const float om = 1.f - ad;
                // log1p's derivative 1 / |1 + delta|^2 <= 1 / (1 - |delta|)^2; 2 ulps of log1pf;
                // the rounding of the term on its way into the total (MQ + 6 roundings at most)
                err += ad < 0.5f ? 0.505f * eq / (om * om) + UR * (2.f + (float)(MQ + 6)) * fabsf(term) : 1e30f;
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
        const float aj = at32[j].x;
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
                const int m = lane + 32 * q;
                if (m < M) {
                    const float2 w = weight(j, m);
                    // -2 s_j w is exact: one rounding of the sum, plus W_jm's rounding (twice)
                    gx[q] = fmaf(-2.f * sj, w.x, gx[q]);
                    gy[q] = fmaf(-2.f * sj, w.y, gy[q]);
                    eb[q] += UR * (fmaxf(fabsf(gx[q]), fabsf(gy[q])) + 2.f * fmaxf(fabsf(w.x), fabsf(w.y)));
                    tanh_bound(gx[q], gy[q], eb[q], tx[q], ty[q], et[q]);
                }
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
                                    int n_sweep, uint64_t seed, int64_t eval, float4* tab, uint64_t* spins,
                                    unsigned long long* accepted, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SAMPLE, s);
    if (an->m > 32 * RBM_MQ) return cudaErrorInvalidValue;
    const int n = an->n, W = (n + 63) / 64, M = an->m;
    const uint32_t evtag = (TAG_SAMPLE << 28) | ((uint32_t)eval & 0x0FFFFFFFu);
    const RbmTabs tabs = rbm_tabs(tab, ntraj, n, M);
    rbm_flip_table_kernel<<<dim3((n * M + 255) / 256, ntraj), 256, 0, s>>>(theta, (int)an->P, n, M, tabs.flip, tabs.flipT, tabs.w,
                                                                          tabs.a);
    const size_t wbytes = (size_t)n * M * sizeof(float2);
    const bool ws = wbytes <= 64 * 1024, small = M <= 128;
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
    kern<<<grid, 32 * cpb, smem, s>>>(theta, (int)an->P, n, M, W, ns, n_sweep, (uint32_t)seed, (uint32_t)(seed >> 32),
                                      evtag, traj0, tabs.flip, tabs.w, tabs.a, spins, accepted);
    count_launch(2);
    return cudaGetLastError();
}

// ------------------------------------------------------------------- local estimators
// Flip ratio r_j = psi(x^(j)) / psi(x) = exp(-2 a_j s_j) prod_m cosh(g_m - 2 s_j W_jm) / cosh g_m
//               = exp(-2 a_j s_j) prod_m (1 + delta_jm),
// delta_jm = (cosh 2W_jm - 1) - s_j tanh(g_m) sinh 2W_jm (the flip table), in FP32: M complex
// multiply-adds per ratio and no transcendental beyond tanh g_m once per sample and unit.

__device__ __forceinline__ float2 rbmf_tanh(float gx, float gy) {
    float tx, ty, et;
    tanh_bound(gx, gy, 0.f, tx, ty, et);
    return make_float2(tx, ty);
}

template <bool WSMEM>
__global__ void __launch_bounds__(256) est_rbm_mixed_kernel(int n, int M, int W, int P, int ns, double h,
                                                            const double2* __restrict__ theta,
                                                            const uint64_t* __restrict__ spins,
                                                            const long long* __restrict__ QJ,
                                                            const long long* __restrict__ baseJ,
                                                            const float4* __restrict__ tab,  // [T][M][n]
                                                            const float2* __restrict__ wtab,
                                                            const float2* __restrict__ atab,
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
    float2* gs = (float2*)smraw;                  // [SPP][M] tanh gamma
    double2* ered = (double2*)(gs + 2 * SPP * M); // [SB][NT/32]
    uint64_t* sw = (uint64_t*)(ered + SB * (NT / 32));  // [SPP][W]
    float2* wf = (float2*)(sw + SPP * W);         // [n][M] W in FP32 (when it fits)
    __shared__ double2 red_r[256], red_sr[256];
    __shared__ double red_s[256];
    const double2* b = theta + (size_t)t * P + n;
    if (WSMEM)
        for (int i = threadIdx.x; i < n * M; i += blockDim.x) wf[i] = wtab[(size_t)t * n * M + i];
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
                const float2 wk = WSMEM ? wf[k * M + m] : __ldg(wtab + ((size_t)t * n + k) * M + m);
                zx = fmaf(wk.x, sk, zx);
                zy = fmaf(wk.y, sk, zy);
            }
            gs[i] = rbmf_tanh(zx, zy);
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
            const float4* tj = tab + (size_t)t * M * n + j;  // [m][j]: the lanes' loads coalesce
            float px = 1.f, py = 0.f;
#pragma unroll 4
            for (int m = 0; m < M; ++m) {
                const float2 tg = gs[g * M + m];
                const float4 f = __ldg(tj + (size_t)m * n);
                // 1 + delta = 1 + (cosh 2W - 1) - s_j tanh(g) sinh 2W
                const float ux = 1.f + f.x - sj * (tg.x * f.z - tg.y * f.w);
                const float uy = f.y - sj * (tg.x * f.w + tg.y * f.z);
                const float nx = px * ux - py * uy;
                py = px * uy + py * ux;
                px = nx;
            }
            const float2 a32 = atab[(size_t)t * n + j];
            const float e = expf(-2.f * a32.x * sj);
            float sn, cs;
            sincosf(-2.f * a32.y * sj, &sn, &cs);
            const float2 r = make_float2(e * (cs * px - sn * py), e * (cs * py + sn * px));
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
    const RbmTabs tabs = rbm_tabs(b.rtab, ntraj, n, M);
    rbm_flip_table_kernel<<<dim3((n * M + 255) / 256, ntraj), 256, 0, s>>>(theta, (int)a->P, n, M, tabs.flip, tabs.flipT, tabs.w,
                                                                          tabs.a);
    count_launch();
    cudaError_t e;
    if (wsm) {
        e = cudaFuncSetAttribute(est_rbm_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        est_rbm_mixed_kernel<true><<<grid, 256, smem, s>>>(n, M, W, (int)a->P, ns, m->h, theta, spins, m->QJ_d,
                                                           m->baseJ_d, tabs.flipT, tabs.w, tabs.a, reinterpret_cast<float2*>(b.r), b.EH, b.part_r,
                                                           b.part_sr, b.part_s);
    } else {
        e = cudaFuncSetAttribute(est_rbm_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        est_rbm_mixed_kernel<false><<<grid, 256, smem, s>>>(n, M, W, (int)a->P, ns, m->h, theta, spins, m->QJ_d,
                                                            m->baseJ_d, tabs.flipT, tabs.w, tabs.a, reinterpret_cast<float2*>(b.r), b.EH,
                                                            b.part_r, b.part_sr, b.part_s);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
