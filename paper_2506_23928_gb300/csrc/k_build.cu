// O_k, its column means, D = Cov(O^*, v) and (plain FP64 path) S by SIMT FP64, for the
// Jastrow ansatz (definitions after Eq. 8: S = <O^* O> - <O^*><O>, F and N^n likewise;
// D = -i F dt + sum_n N^n dW_n = Cov(O^*, v) with v = -i dt E_eff + sum_n dW_n B^n).
// Jastrow log-derivatives are real: O_{a_j} = sigma_j, O_{eta_jk} = sigma_j sigma_k (Eq. 12).
#include "common.cuh"

namespace otvmc {

// ------------------------------------------------------------------ D by exact int64 sums
// With q(x) the quantised centred v, sum_x O_xk q(x) = 2 sum_{x: O_xk = +1} q(x) - sum_x q(x)
// is exact; so is the count c_k = sum_x O_xk, whence obar_k = c_k / ns and
// D_k = (sum_x O_xk q(x) - c_k Q / ns) 2^-e / ns (Q = sum_x q(x)).
//
// The sums over {x: O_xk = +1} run as an outer-product tile: a CTA takes the 64-site blocks
// (JB, LB), JB <= LB, and a quarter of the samples; thread (tj, tl) owns sites
// j = 64 JB + 4 tj + a, l = 64 LB + 4 tl + b (a, b < 4), i.e. the pairs (j, l), j < l, and on
// the diagonal of a diagonal tile the singles O = sigma_j.  Partial sums are added into
// dsum with 64-bit integer atomics (exact, so the order does not matter).
constexpr int DT = 256;      // samples staged per pass
constexpr int DSPLIT = 4;    // sample ranges per trajectory

__host__ __device__ __forceinline__ int d_pair_idx(int lo, int hi, int n) {
    return lo * n - lo * (lo + 1) / 2 + (hi - lo - 1);
}

__global__ void __launch_bounds__(256) D_sums_jastrow_kernel(int n, int W, int P, int ns,
                                                             const uint64_t* __restrict__ spins,
                                                             const long long* __restrict__ qv,
                                                             unsigned long long* __restrict__ dsum) {
    __shared__ uint64_t swJ[DT], swL[DT];
    __shared__ longlong2 sq[DT];
    const int t = blockIdx.z, tid = threadIdx.x;
    int LB = 0;
    while ((LB + 1) * (LB + 2) / 2 <= (int)blockIdx.y) ++LB;
    const int JB = blockIdx.y - LB * (LB + 1) / 2;
    const int tj = tid >> 4, tl = tid & 15;
    const int j0 = 64 * JB + 4 * tj, l0 = 64 * LB + 4 * tl;
    const bool diag = (JB == LB) && (tj == tl);
    // this thread owns a useful entry iff some (j, l) with j <= l, both < n
    const bool work = j0 < n && l0 < n && j0 <= l0 + 3;
    const int xs = (int)(((long long)ns * blockIdx.x) / gridDim.x), xe = (int)(((long long)ns * (blockIdx.x + 1)) / gridDim.x);
    long long ar[16], ai[16];
    int cnt[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) ar[e] = ai[e] = 0, cnt[e] = 0;
    for (int x0 = xs; x0 < xe; x0 += DT) {
        const int nt = min(DT, xe - x0);
        __syncthreads();
        for (int i = tid; i < nt; i += blockDim.x) {
            const size_t xo = (size_t)t * ns + x0 + i;
            swJ[i] = spins[xo * W + JB];
            swL[i] = spins[xo * W + LB];
            sq[i] = make_longlong2(qv[xo * 2], qv[xo * 2 + 1]);
        }
        __syncthreads();
        if (work) {
            for (int x = 0; x < nt; ++x) {
                const uint32_t bj = (uint32_t)(swJ[x] >> (4 * tj)) & 0xFu;
                const uint32_t bl = (uint32_t)(swL[x] >> (4 * tl)) & 0xFu;
                const longlong2 q = sq[x];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t up = (diag && a == b) ? (bj >> a) & 1u : ~((bj >> a) ^ (bl >> b)) & 1u;
                        if (up) {
                            ar[4 * a + b] += q.x;
                            ai[4 * a + b] += q.y;
                            ++cnt[4 * a + b];
                        }
                    }
            }
        }
    }
    if (!work) return;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = j0 + a, l = l0 + b;
            if (j >= n || l >= n || j > l || (j == l && !diag)) continue;
            const int k = j == l ? j : n + d_pair_idx(j, l, n);
            unsigned long long* d = dsum + ((size_t)t * P + k) * 3;
            atomicAdd(d, (unsigned long long)ar[4 * a + b]);
            atomicAdd(d + 1, (unsigned long long)ai[4 * a + b]);
            atomicAdd(d + 2, (unsigned long long)(long long)cnt[4 * a + b]);
        }
}

__global__ void __launch_bounds__(256) D_final_kernel(int P, int ns, const long long* __restrict__ dsum,
                                                      const double* __restrict__ vinfo,
                                                      const long long* __restrict__ qsum, double* __restrict__ obar,
                                                      double2* __restrict__ D) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const long long* d = dsum + ((size_t)t * P + k) * 3;
    const long long ar = d[0], ai = d[1], cnt = d[2];
    const long long Qr = qsum[2 * t], Qi = qsum[2 * t + 1];
    const long long c = 2 * cnt - ns;
    const double inv = vinfo[4 * t + 2] / ns;
    const double dr = ((double)(2 * ar - Qr) - (double)c * (double)Qr / ns) * inv;
    const double di = ((double)(2 * ai - Qi) - (double)c * (double)Qi / ns) * inv;
    obar[(size_t)t * P + k] = (double)c / ns;
    D[(size_t)t * P + k] = make_double2(dr, di);
}

// D and obar from the Gram kernel's side output X[t][k][33] (the sums of O_k against the
// extra rows): sum_x O_k q = sum_p X[p] 16^p for the real (p < 16) and imaginary
// (16 <= p < 32) digits, in wrapping 64-bit arithmetic (the true sum fits in 64 bits), and
// c_k = X[32] = sum_x O_k; then the formula of D_final_kernel with 2 a_r - Q_r = sum_x O_k q_r.
__global__ void __launch_bounds__(256) D_from_gram_kernel(int P, int ns, const float* __restrict__ X,
                                                          const double* __restrict__ vinfo,
                                                          const long long* __restrict__ qsum, double* __restrict__ obar,
                                                          double2* __restrict__ D) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const float* x = X + ((size_t)t * P + k) * D_XROWS;
    unsigned long long sr = 0ull, si = 0ull;
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        sr += (unsigned long long)(long long)x[p] << (4 * p);
        si += (unsigned long long)(long long)x[16 + p] << (4 * p);
    }
    const long long c = (long long)x[32];
    const long long Qr = qsum[2 * t], Qi = qsum[2 * t + 1];
    const double inv = vinfo[4 * t + 2] / ns;
    const double dr = ((double)(long long)sr - (double)c * (double)Qr / ns) * inv;
    const double di = ((double)(long long)si - (double)c * (double)Qi / ns) * inv;
    obar[(size_t)t * P + k] = (double)c / ns;
    D[(size_t)t * P + k] = make_double2(dr, di);
}

cudaError_t launch_D_from_gram(const otvmc_ansatz* a, int ntraj, int ns, const EvalBufs& b, double* obar, double2* D,
                               cudaStream_t s) {
    ProfScope prof_(OTVMC_K_D, s);
    const int P = (int)a->P;
    D_from_gram_kernel<<<dim3((P + 255) / 256, ntraj), 256, 0, s>>>(P, ns, b.dx, b.vinfo, b.qsum, obar, D);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_D_fixed_jastrow(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns,
                                   const EvalBufs& b, double* obar, double2* D, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_D, s);
    const int n = a->n, W = (n + 63) / 64, P = (int)a->P;
    cudaError_t e = cudaMemsetAsync(b.dsum, 0, (size_t)ntraj * P * 3 * sizeof(long long), s);
    if (e != cudaSuccess) return e;
    dim3 grid(DSPLIT, W * (W + 1) / 2, ntraj);
    D_sums_jastrow_kernel<<<grid, 256, 0, s>>>(n, W, P, ns, spins, b.qv, (unsigned long long*)b.dsum);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    D_final_kernel<<<dim3((P + 255) / 256, ntraj), 256, 0, s>>>(P, ns, b.dsum, b.vinfo, b.qsum, obar, D);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ O in E4M3 (K-major)
// Ot[t][k][x] = O_xk as an E4M3 code (+1 = 0x38, -1 = 0xB8), rows k contiguous over the samples
// x with a pitch of o_pitch(ns) bytes (the samples from ns on hold 0), the operand layout of the
// tensor-core Gram kernel.  One thread = sixteen consecutive samples: it first transposes their
// spins into a 16-bit mask per site (bit s set: sigma_j of sample s is +1), then writes each
// parameter's sixteen codes as one 16-byte store, so a warp writes 512 contiguous bytes per
// parameter.  The parameters are split over gridDim.z blocks (each rebuilds the masks), so
// that small batches still fill the GPU.
constexpr int OB_SPT = 16;
constexpr int OB_THREADS = 128;

// Sixteen codes from a 16-bit mask: byte s is 0x38 (+1) if bit s is set, else 0xB8 (-1).  The
// multiply spreads the four bits of a nibble to bits 0, 8, 16, 24 (the shifted copies do not
// overlap, so no carries).
__device__ __forceinline__ uint4 e4m3_pm1x16(uint32_t e) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = 0xB8B8B8B8u ^ ((((e >> (4 * q)) & 0xFu) * 0x00204081u & 0x01010101u) << 7);
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// E4M3 code of an integer |d| <= 8, from the format's definition: sign bit, exponent biased by
// 7 (bits 3..6), three fraction bits; d = 2^e (1 + f / 8).
__device__ __forceinline__ uint32_t e4m3_small_int(int d) {
    if (d == 0) return 0u;
    const uint32_t sg = d < 0 ? 0x80u : 0u;
    const int a = d < 0 ? -d : d;
    const int e = 31 - __clz(a);
    return sg | ((uint32_t)(e + 7) << 3) | (uint32_t)((a << (3 - e)) - 8);
}

__global__ void __launch_bounds__(OB_THREADS) obuild_f8_jastrow_kernel(int n, int W, int P, int rows, int ns,
                                                                       int pitch, const uint64_t* __restrict__ spins,
                                                                       const int* __restrict__ pairs,
                                                                       const long long* __restrict__ qv,
                                                                       uint8_t* __restrict__ Ot) {
    extern __shared__ uint16_t msk[];  // [n][OB_THREADS]: site masks of each thread's samples
    const int t = blockIdx.y, tid = threadIdx.x;
    const int x0 = (blockIdx.x * OB_THREADS + tid) * OB_SPT;
    for (int w = 0; w < W; ++w) {
        uint64_t wd[OB_SPT];
#pragma unroll
        for (int q = 0; q < OB_SPT; ++q) wd[q] = (x0 + q < ns) ? spins[((size_t)t * ns + x0 + q) * W + w] : 0ull;
        const int bend = min(64, n - 64 * w);
        for (int b = 0; b < bend; ++b) {
            uint32_t m = 0;
#pragma unroll
            for (int q = 0; q < OB_SPT; ++q) m |= (uint32_t)((wd[q] >> b) & 1ull) << q;
            msk[(64 * w + b) * OB_THREADS + tid] = (uint16_t)m;
        }
    }
    __syncthreads();
    if (x0 >= pitch) return;  // x0 < pitch = o_pitch(ns) implies x0 < ns
    // byte masks of the valid samples (all ones except in the last group of a ragged ns)
    const int nv = min(OB_SPT, ns - x0);
    uint32_t vm[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c = min(4, max(0, nv - 4 * q));
        vm[q] = c >= 4 ? 0xFFFFFFFFu : ((1u << (8 * c)) - 1u);
    }
    uint8_t* base = Ot + (size_t)t * rows * pitch + x0;
    const int k0 = (int)(((long long)P * blockIdx.z) / gridDim.z);
    const int k1 = (int)(((long long)P * (blockIdx.z + 1)) / gridDim.z);
    for (int k = k0; k < k1; ++k) {
        uint32_t e;
        if (k < n) {
            e = msk[k * OB_THREADS + tid];
        } else {
            const int j = __ldg(pairs + 2 * (k - n)), l = __ldg(pairs + 2 * (k - n) + 1);
            e = ~(uint32_t)(msk[j * OB_THREADS + tid] ^ msk[l * OB_THREADS + tid]) & 0xFFFFu;
        }
        const uint4 v = e4m3_pm1x16(e);
        *reinterpret_cast<uint4*>(base + (size_t)k * pitch) = make_uint4(v.x & vm[0], v.y & vm[1], v.z & vm[2],
                                                                         v.w & vm[3]);
    }
    if (qv == nullptr || blockIdx.z != gridDim.z - 1) return;
    // extra rows P .. P + 32: the balanced base-16 digits d_p in [-8, 7] of q (real part, then
    // imaginary part; q = sum_p d_p 16^p), then ones; 0 for the samples from ns on
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        long long r[OB_SPT];
#pragma unroll
        for (int q = 0; q < OB_SPT; ++q) r[q] = (x0 + q < ns) ? qv[((size_t)t * ns + x0 + q) * 2 + h] : 0ll;
#pragma unroll 1
        for (int p = 0; p < 16; ++p) {
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int q = 0; q < OB_SPT; ++q) {
                const int d = (int)((r[q] & 0xF) ^ 0x8) - 0x8;
                r[q] = (r[q] - d) >> 4;  // exact: r - d is a multiple of 16
                w[q >> 2] |= e4m3_small_int(d) << (8 * (q & 3));
            }
            *reinterpret_cast<uint4*>(base + (size_t)(P + 16 * h + p) * pitch) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    *reinterpret_cast<uint4*>(base + (size_t)(P + 32) * pitch) =
        make_uint4(0x38383838u & vm[0], 0x38383838u & vm[1], 0x38383838u & vm[2], 0x38383838u & vm[3]);
}

cudaError_t launch_obuild_f8_jastrow(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns,
                                     const long long* qv, uint8_t* Ot, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_OBUILD, s);
    const int n = a->n, W = (n + 63) / 64, P = (int)a->P;
    const int pitch = o_pitch(ns);
    const int rows = qv != nullptr ? P + D_XROWS : P;
    const int per_block = OB_THREADS * OB_SPT;
    const int gx = (pitch + per_block - 1) / per_block;
    // parameter ranges: about eight blocks per SM over the batch, each range >= 64 parameters
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
        sms = 152;
    int kz = (8 * sms + gx * ntraj - 1) / (gx * ntraj);
    kz = max(1, min(kz, P / 64));
    dim3 grid(gx, ntraj, kz);
    const size_t smem = (size_t)n * OB_THREADS * sizeof(uint16_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(obuild_f8_jastrow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    obuild_f8_jastrow_kernel<<<grid, OB_THREADS, smem, s>>>(n, W, P, rows, ns, pitch, spins, a->pairs_d, qv, Ot);
    count_launch();
    return cudaGetLastError();
}

// --------------------------------------------------------------- plain FP64 path: O_c
__global__ void __launch_bounds__(256) obuild_f64_jastrow_kernel(int n, int W, int P, int ns,
                                                                 const uint64_t* __restrict__ spins,
                                                                 const int* __restrict__ pairs,
                                                                 const double* __restrict__ obar,
                                                                 double* __restrict__ Oc) {
    const int t = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ns) return;
    const uint64_t* w = spins + ((size_t)t * ns + x) * W;
    double* base = Oc + (size_t)t * P * ns + x;
    for (int k = 0; k < P; ++k) {
        double o;
        if (k < n) {
            o = ((w[k >> 6] >> (k & 63)) & 1ull) ? 1.0 : -1.0;
        } else {
            const int j = __ldg(pairs + 2 * (k - n)), l = __ldg(pairs + 2 * (k - n) + 1);
            const double sj = ((w[j >> 6] >> (j & 63)) & 1ull) ? 1.0 : -1.0;
            const double sl = ((w[l >> 6] >> (l & 63)) & 1ull) ? 1.0 : -1.0;
            o = sj * sl;
        }
        base[(size_t)k * ns] = o - obar[(size_t)t * P + k];
    }
}

cudaError_t launch_obuild_f64_jastrow(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns,
                                      const double* obar, double* Oc, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_OBUILD, s);
    const int n = a->n, W = (n + 63) / 64, P = (int)a->P;
    dim3 grid((ns + 255) / 256, ntraj);
    obuild_f64_jastrow_kernel<<<grid, 256, 0, s>>>(n, W, P, ns, spins, a->pairs_d, obar, Oc);
    count_launch();
    return cudaGetLastError();
}

// S[i][j] = inv sum_x Oc[i][x] Oc[j][x] over the K columns x of the rows i, j < P, FP64
// SIMT, 64x64 tiles of the upper triangle, mirrored into the lower triangle.
__global__ void __launch_bounds__(256) syrk_f64_kernel(int P, int ns, double inv, const double* __restrict__ Oc,
                                                       double* __restrict__ S) {
    constexpr int BT = 64, BK = 16;
    __shared__ double As[BK][BT + 1];
    __shared__ double Bs[BK][BT + 1];
    const int t = blockIdx.z;
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bj < bi) return;
    const double* O = Oc + (size_t)t * P * ns;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < ns; k0 += BK) {
        for (int i = threadIdx.x; i < BT * BK; i += 256) {
            const int r = i / BK, kk = i % BK;
            const int gi = bi * BT + r, gj = bj * BT + r, gk = k0 + kk;
            As[kk][r] = (gi < P && gk < ns) ? O[(size_t)gi * ns + gk] : 0.0;
            Bs[kk][r] = (gj < P && gk < ns) ? O[(size_t)gj * ns + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty * 4 + u];
                b[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
    double* St = S + (size_t)t * P * P;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gi = bi * BT + ty * 4 + u, gj = bj * BT + tx * 4 + v;
            if (gi < P && gj < P && gj >= gi) {
                const double val = acc[u][v] * inv;
                St[(size_t)gi * P + gj] = val;
                St[(size_t)gj * P + gi] = val;
            }
        }
}

cudaError_t launch_syrk_f64_scaled(int ntraj, int rows, int K, double inv, const double* O, double* S,
                                   cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SYRK, s);
    const int nb = (rows + 63) / 64;
    dim3 grid(nb, nb, ntraj);
    syrk_f64_kernel<<<grid, 256, 0, s>>>(rows, K, inv, O, S);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_syrk_f64(int ntraj, int P, int ns, const double* Oc, double* S, cudaStream_t s) {
    return launch_syrk_f64_scaled(ntraj, P, ns, 1.0 / ns, Oc, S, s);
}

// D_k = sum_x Oc[k][x] (v(x) - vbar) / ns, FP64: one warp per parameter.
__global__ void __launch_bounds__(256) gemv_D_f64_kernel(int P, int ns, const double* __restrict__ Oc,
                                                         const double2* __restrict__ v,
                                                         const double* __restrict__ vinfo, double2* __restrict__ D) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * 8 + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (k >= P) return;
    const double mr = vinfo[4 * t], mi = vinfo[4 * t + 1];
    const double* o = Oc + ((size_t)t * P + k) * ns;
    const double2* vv = v + (size_t)t * ns;
    double ar = 0.0, ai = 0.0;
    for (int x = lane; x < ns; x += 32) {
        const double c = o[x];
        ar = fma(c, vv[x].x - mr, ar);
        ai = fma(c, vv[x].y - mi, ai);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, off);
        ai += __shfl_xor_sync(0xffffffffu, ai, off);
    }
    if (lane == 0) D[(size_t)t * P + k] = make_double2(ar / ns, ai / ns);
}

cudaError_t launch_gemv_D_f64(int ntraj, int P, int ns, const double* Oc, const double2* v, const EvalBufs& b,
                              double2* D, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_D, s);
    dim3 grid((P + 7) / 8, ntraj);
    gemv_D_f64_kernel<<<grid, 256, 0, s>>>(P, ns, Oc, v, b.vinfo, D);
    count_launch();
    return cudaGetLastError();
}

// S = G / ns - obar obar^T (full, FP64) from the upper-triangle Gram counts.
__global__ void expand_S_kernel(int P, int ns, const float* __restrict__ G, const double* __restrict__ obar,
                                double* __restrict__ S) {
    const int t = blockIdx.y;
    const int i = blockIdx.x;
    const float* Gt = G + (size_t)t * P * P;
    const double* ob = obar + (size_t)t * P;
    double* St = S + (size_t)t * P * P;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        const float g = (j >= i) ? Gt[(size_t)i * P + j] : Gt[(size_t)j * P + i];
        St[(size_t)i * P + j] = (double)g / ns - ob[i] * ob[j];
    }
}

cudaError_t launch_expand_S(int ntraj, int P, int ns, const float* G, const double* obar, double* S,
                            cudaStream_t s) {
    ProfScope prof_(OTVMC_K_D, s);
    dim3 grid(P, ntraj);
    expand_S_kernel<<<grid, 256, 0, s>>>(P, ns, G, obar, S);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
