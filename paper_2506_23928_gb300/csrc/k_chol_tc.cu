// Regularised solve (S + eps I) delta = D of the otVMC equation (Eq. 8 with the
// diagonal-shift regulariser), batched over trajectories, with the O(P^3) part of the
// Cholesky factorization on the tensor cores.
//
// Left-looking blocked Cholesky, 128-wide block columns jb = 0, 128, ...:
//   update  (tcgen05)  C[i, jb:jb+128] = A[i, jb:jb+128] - sum_{k<jb} L[i,k] L[jb+c,k], i >= jb.
//           L is kept as three BF16 pieces (L = h + m + l to ~2^-24 relative); the six
//           products h.h + h.m + m.h + h.l + m.m + l.h accumulate in FP32 in TMEM, which
//           gives FP32-level accuracy.  One CTA = 128 rows x 128 columns of one trajectory;
//           32-column k slices (64-byte swizzle) in a 2-stage ring, two CTAs per SM.
//   diag    (SIMT)     factor the 128 x 128 diagonal block in shared memory (32-column
//           sub-blocks, shuffle-based leaf factor) and invert it;
//   trsm    (SIMT)     the rows below as a register-tiled GEMM X = C L_dd^-T, one 64-row tile
//           per CTA; both write L in FP32 (for the triangular solves) and as BF16 pieces
//           (for later updates), and the diagonal kernel writes L_dd^-1.
// solve     (SIMT)     forward/backward substitution by blocks through the stored inverses,
//           then one step of iterative refinement with the residual D - (S + eps I) x formed
//           in FP64 from the exact Gram counts (S = G/ns - obar obar^T).
// A trajectory whose pivot is not positive is marked and solved again by the single-CTA
// solver, which raises the shift (x100, at most three times).
#include <cuda_bf16.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "common.cuh"
#include "tc_common.cuh"

namespace otvmc {
namespace chol {

constexpr int NB = 128;                  // block column width
constexpr int BK = 32;                   // k extent of one TMA box (bf16: 64 bytes, 64-byte swizzle)
constexpr int NPC = 3;                   // bf16 pieces of L
constexpr int BOX = 128 * BK * 2;        // one 128-row box: 8 KB
constexpr int STAGE = 2 * NPC * BOX;     // A pieces + B pieces: 48 KB
constexpr int STAGES = 2;                // about 97 KB of shared memory: two CTAs per SM
constexpr int SMEM_U = STAGES * STAGE + 1024 + 256;
constexpr uint32_t TCOLS = 128;
constexpr int DS = NB + 1;               // shared-memory row stride of 128-wide blocks
constexpr int RT = 64;                   // panel rows per tile

__device__ __forceinline__ float a_orig(const float* Gt, const double* ob, int P, float inv_ns, int i, int j,
                                        float eps) {
    // (S + eps I)_ij for j <= i from the upper-triangle Gram counts, in FP32
    float v = Gt[(size_t)j * P + i] * inv_ns - (float)ob[i] * (float)ob[j];
    return i == j ? v + eps : v;
}

// ------------------------------------------------------------------------- update (tcgen05)
__global__ void __launch_bounds__(192, 2) chol_update_kernel(const __grid_constant__ CUtensorMap tmap, int t0, int P,
                                                             int ns, int NT, int jb, float eps,
                                                             const float* __restrict__ G,
                                                             const double* __restrict__ obar, float* __restrict__ Pn,
                                                             const int* __restrict__ fail, int* status) {
    using namespace tc;
    const int t = t0 + blockIdx.y;
    if (fail[t]) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int i0 = jb + blockIdx.x * 128;
    const int nk = jb / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (kb >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                uint8_t* st = smem + s * STAGE;
                mbar_expect_tx(&full[s], STAGE);
                // k slice kb covers columns [32 kb, 32 kb + 32) of the 64-column chunk kb / 2
                const int kx = (kb & 1) * BK, kc = kb >> 1;
                for (int p = 0; p < NPC; ++p) {
                    const int pl = (t * NPC + p) * NT;
                    tma_load_4d(st + p * BOX, &tmap, &full[s], kx, 0, kc, pl + (i0 >> 7));
                    tma_load_4d(st + (NPC + p) * BOX, &tmap, &full[s], kx, 0, kc, pl + (jb >> 7));
                }
                ++issued;
            }
            for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
                mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // piece products kept: (h,h) (h,m) (m,h) (h,l) (m,m) (l,h)
            const int pa[6] = {0, 0, 1, 0, 1, 2};
            const int pb[6] = {0, 1, 0, 2, 1, 0};
            constexpr uint32_t ID = idesc_bf16(128, NB);
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t st = su32(smem + s * STAGE);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
#pragma unroll
                    for (int q = 0; q < 6; ++q)
                        umma(tmem, smem_desc_sw64(st + pa[q] * BOX + k * 32),
                             smem_desc_sw64(st + (NPC + pb[q]) * BOX + k * 32), ID, (kb > 0 || k > 0 || q > 0) ? 1u : 0u);
                umma_commit(&empty[s]);
            }
            umma_commit(done);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        int ok = 0;
        if (lane == 0) ok = mbar_wait(done, 0, abort_flag) && !*abort_flag;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        fence_after();
        if (ok) {
            const int i = i0 + q * 32 + lane;
            const float* Gt = G + (size_t)t * P * P;
            const double* ob = obar + (size_t)t * P;
            const float inv_ns = 1.0f / (float)ns;
            float* prow = Pn + ((size_t)t * P + (i < P ? i : 0)) * NB;
#pragma unroll 1
            for (int c0 = 0; c0 < NB; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                if (i >= P) continue;
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    const int j = jb + c0 + u;
                    if (j < P && j <= i) prow[c0 + u] = a_orig(Gt, ob, P, inv_ns, i, j, eps) - __uint_as_float(v[u]);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) record_error(status, OTVMC_ERR_TIMEOUT, t);
    if (warp == 1) {
        if (lane == 0) mbar_wait(done, 0, nullptr);
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
    }
}

// --------------------------------------------------------------------------- panel (SIMT)
// BF16 pieces of L are stored tiled: for piece p of trajectory t, the 128-row tile i / 128
// and the 64-column block k / 64 form one contiguous 16 KB chunk [i % 128][k % 64], so
// that one TMA box of the update kernel is one contiguous read.
struct LbLayout {
    int NT;  // row tiles, ceil(P / 128)
    int KB;  // 64-column blocks, LD / 64
    __device__ __forceinline__ size_t plane() const { return (size_t)NT * KB * 128 * 64; }
    __device__ __forceinline__ size_t at(int i, int k) const {
        return (((size_t)(i >> 7) * KB + (k >> 6)) * 128 + (i & 127)) * 64 + (k & 63);
    }
};

__device__ __forceinline__ void store_L(float* Lf, __nv_bfloat16* Lbt, const LbLayout& lay, int LD, int i, int k,
                                        float x) {
    Lf[(size_t)i * LD + k] = x;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    const size_t idx = lay.at(i, k), pl = lay.plane();
    Lbt[idx] = h;
    Lbt[pl + idx] = m;
    Lbt[2 * pl + idx] = __float2bfloat16_rn(r2);
}

// Diagonal block of block column jb: Cholesky factor and its inverse (one CTA per trajectory).
// 32-column sub-blocks: warp 0 factors the 32 x 32 diagonal sub-block in registers with
// shuffles, all threads solve the sub-panel below and update the trailing part.  Rows and
// columns beyond nb are padded with the identity.
__global__ void __launch_bounds__(256) chol_diag_kernel(int t0, int P, int LD, int ns, int jb, float eps,
                                                           const float* __restrict__ G,
                                                           const double* __restrict__ obar,
                                                           const float* __restrict__ Pn, float* __restrict__ Lf,
                                                           __nv_bfloat16* __restrict__ Lb, float* __restrict__ Dinv,
                                                           int* __restrict__ fail) {
    const int t = t0 + blockIdx.x;
    if (fail[t]) return;
    extern __shared__ __align__(16) float dsm[];
    float* A = dsm;             // [NB][DS] block, then its factor (lower) and its inverse
                                // (strictly lower part of the inverse stored transposed above the diagonal)
    float* lid = A + NB * DS;   // [NB] diagonal of the inverse
    __shared__ int bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = min(NB, P - jb);
    const float* Gt = G + (size_t)t * P * P;
    const double* ob = obar + (size_t)t * P;
    const float inv_ns = 1.0f / (float)ns;
    if (tid == 0) bad = 0;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, c = e - i * NB;
        float v = 0.f;
        if (i < nb && c < nb) {
            if (c <= i) v = jb == 0 ? a_orig(Gt, ob, P, inv_ns, jb + i, jb + c, eps) : Pn[((size_t)t * P + jb + i) * NB + c];
        } else if (i == c) {
            v = 1.f;
        }
        A[i * DS + c] = v;
    }
    __syncthreads();
    for (int k0 = 0; k0 < NB; k0 += 32) {
        if (warp == 0) {
            float r[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) r[c] = A[(k0 + lane) * DS + k0 + c];
            bool ok = true;
#pragma unroll
            for (int p = 0; p < 32; ++p) {
                const float d = __shfl_sync(0xffffffffu, r[p], p);
                ok = ok && (d > 0.f) && isfinite(d);
                const float sd = sqrtf(fmaxf(d, 1e-30f));
                if (lane == p) r[p] = sd;
                if (lane > p) r[p] /= sd;
                const float colp = r[p];
#pragma unroll
                for (int c = p + 1; c < 32; ++c) {
                    const float lcp = __shfl_sync(0xffffffffu, colp, c);
                    if (lane >= c) r[c] = fmaf(-colp, lcp, r[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) A[(k0 + lane) * DS + k0 + c] = (c <= lane) ? r[c] : 0.f;
            if (lane == 0 && !ok) bad = 1;
        }
        __syncthreads();
        if (bad) break;
        // sub-panel rows below: X L_kk^T = A
        for (int i = k0 + 32 + tid; i < NB; i += blockDim.x) {
            float x[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                float a = A[i * DS + k0 + c];
#pragma unroll
                for (int k = 0; k < c; ++k) a = fmaf(-x[k], A[(k0 + c) * DS + k0 + k], a);
                x[c] = a / A[(k0 + c) * DS + k0 + c];
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) A[i * DS + k0 + c] = x[c];
        }
        __syncthreads();
        // trailing update A[i][j] -= X[i] . X[j] for k0+32 <= j <= i
        const int m = NB - k0 - 32;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = k0 + 32 + e / m, j = k0 + 32 + e % m;
            if (j > i) continue;
            float a = A[i * DS + j];
#pragma unroll 8
            for (int k = 0; k < 32; ++k) a = fmaf(-A[i * DS + k0 + k], A[j * DS + k0 + k], a);
            A[i * DS + j] = a;
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) fail[t] = 1;
        return;
    }
    // inverse of the lower-triangular factor, one column per thread, four partial sums;
    // column c of the inverse is kept in row c above the diagonal (Li[k][c] at A[c][k], k > c)
    if (tid < NB) {
        const int c = tid;
        const float dc = 1.f / A[c * DS + c];
        lid[c] = dc;
        for (int i = c + 1; i < NB; ++i) {
            float s0 = A[i * DS + c] * dc, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int k = c + 1;
            for (; k + 3 < i; k += 4) {
                s0 = fmaf(A[i * DS + k], A[c * DS + k], s0);
                s1 = fmaf(A[i * DS + k + 1], A[c * DS + k + 1], s1);
                s2 = fmaf(A[i * DS + k + 2], A[c * DS + k + 2], s2);
                s3 = fmaf(A[i * DS + k + 3], A[c * DS + k + 3], s3);
            }
            for (; k < i; ++k) s0 = fmaf(A[i * DS + k], A[c * DS + k], s0);
            A[c * DS + i] = -((s0 + s1) + (s2 + s3)) / A[i * DS + i];
        }
    }
    __syncthreads();
    const LbLayout lay{(P + NB - 1) / NB, LD / 64};
    float* Lft = Lf + (size_t)t * P * LD;
    __nv_bfloat16* Lbt = Lb + (size_t)t * NPC * lay.plane();
    float* Dv = Dinv + ((size_t)t * ((P + NB - 1) / NB) + jb / NB) * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, c = e - i * NB;
        float li = 0.f;
        if (i < nb && c < nb) li = (i == c) ? lid[c] : (i > c ? A[c * DS + i] : 0.f);
        Dv[e] = li;
        if (i < nb && c < nb) store_L(Lft, Lbt, lay, LD, jb + i, jb + c, c <= i ? A[i * DS + c] : 0.f);
    }
}

// Rows below the diagonal block: X = C L_dd^-T, one 64-row tile per CTA; each thread owns
// 4 rows x 8 columns (register tiling: 12 shared loads per 32 FMAs).
__global__ void __launch_bounds__(256) chol_trsm_kernel(int t0, int P, int LD, int ns, int jb, float eps,
                                                        const float* __restrict__ G, const double* __restrict__ obar,
                                                        const float* __restrict__ Pn, float* __restrict__ Lf,
                                                        __nv_bfloat16* __restrict__ Lb,
                                                        const float* __restrict__ Dinv, const int* __restrict__ fail) {
    const int t = t0 + blockIdx.y;
    if (fail[t]) return;
    extern __shared__ __align__(16) float tsm[];
    float* Li = tsm;            // [NB][DS]
    float* Ct = Li + NB * DS;   // [RT][DS]
    const int tid = threadIdx.x;
    const int nb = min(NB, P - jb);
    const int r0 = jb + nb + blockIdx.x * RT;
    const float* Gt = G + (size_t)t * P * P;
    const double* ob = obar + (size_t)t * P;
    const float inv_ns = 1.0f / (float)ns;
    const float* Dv = Dinv + ((size_t)t * ((P + NB - 1) / NB) + jb / NB) * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) Li[(e / NB) * DS + e % NB] = Dv[e];
    for (int e = tid; e < RT * nb; e += blockDim.x) {
        const int rr = e / nb, c = e - rr * nb;
        const int i = r0 + rr;
        float v = 0.f;
        if (i < P) v = jb == 0 ? a_orig(Gt, ob, P, inv_ns, i, jb + c, eps) : Pn[((size_t)t * P + i) * NB + c];
        Ct[rr * DS + c] = v;
    }
    __syncthreads();
    const int rg = tid % 16, cg = tid / 16;
    float acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[a][u] = 0.f;
    const int kend = min(nb, cg * 8 + 8);  // L_dd^-1 is lower triangular
    for (int k = 0; k < kend; ++k) {
        float cv[4], lv[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) cv[a] = Ct[(rg * 4 + a) * DS + k];
#pragma unroll
        for (int u = 0; u < 8; ++u) lv[u] = Li[(cg * 8 + u) * DS + k];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[a][u] = fmaf(cv[a], lv[u], acc[a][u]);
    }
    const LbLayout lay{(P + NB - 1) / NB, LD / 64};
    float* Lft = Lf + (size_t)t * P * LD;
    __nv_bfloat16* Lbt = Lb + (size_t)t * NPC * lay.plane();
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = r0 + rg * 4 + a;
        if (i < P)
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = cg * 8 + u;
                if (c < nb) store_L(Lft, Lbt, lay, LD, i, jb + c, acc[a][u]);
            }
    }
}

// ------------------------------------------------------------------------------ solves
// (s, c) += g * (xh + xl) with an error-free product and sum (Dekker/Knuth): the pair s + c
// carries about 48 bits, enough for an FP64-quality residual from FP32 arithmetic.
__device__ __forceinline__ void df_fma(float& s, float& c, float g, float xh, float xl) {
    const float p = g * xh;
    const float e = fmaf(g, xh, -p);
    const float t = s + p;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (p - bp);
    s = t;
    c += err + e;
    c = fmaf(g, xl, c);
}

// L L^T x = y for two right-hand sides held in shared memory (y[0..P), y[P..2P)).
__device__ void block_solve(int P, int LD, const float* Lft, const float* Dv, float* y, float* Db, float* tmp,
                            float* part) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nblk = (P + NB - 1) / NB;
    for (int b = 0; b < nblk; ++b) {
        const int jb = b * NB, nb = min(NB, P - jb);
        for (int e = tid; e < NB * NB; e += blockDim.x) Db[(e / NB) * DS + e % NB] = Dv[(size_t)b * NB * NB + e];
        __syncthreads();
        for (int e = tid; e < 2 * nb; e += blockDim.x) {
            const int c = e % nb, h = e / nb;
            float s = 0.f;
            for (int k = 0; k <= c; ++k) s = fmaf(Db[c * DS + k], y[h * P + jb + k], s);
            tmp[h * NB + c] = s;
        }
        __syncthreads();
        for (int e = tid; e < 2 * nb; e += blockDim.x) y[(e / nb) * P + jb + e % nb] = tmp[(e / nb) * NB + e % nb];
        __syncthreads();
        if (jb + nb < P) {
            // rows below: y_i -= L[i, jb:jb+128] . y_b; lane l owns columns 4l..4l+3, each warp
            // keeps four rows in flight
            float yb0[4], yb1[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                yb0[u] = y[jb + 4 * lane + u];
                yb1[u] = y[P + jb + 4 * lane + u];
            }
            const int nw = blockDim.x / 32;
            for (int i0 = jb + nb + 4 * warp; i0 < P; i0 += 4 * nw) {
                float4 l4[4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    l4[a] = (i0 + a < P) ? *reinterpret_cast<const float4*>(Lft + (size_t)(i0 + a) * LD + jb + 4 * lane)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                float s0[4], s1[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    s0[a] = l4[a].x * yb0[0] + l4[a].y * yb0[1] + l4[a].z * yb0[2] + l4[a].w * yb0[3];
                    s1[a] = l4[a].x * yb1[0] + l4[a].y * yb1[1] + l4[a].z * yb1[2] + l4[a].w * yb1[3];
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        s0[a] += __shfl_xor_sync(0xffffffffu, s0[a], off);
                        s1[a] += __shfl_xor_sync(0xffffffffu, s1[a], off);
                    }
                if (lane < 4 && i0 + lane < P) {
                    float v0 = s0[0], v1 = s1[0];
                    if (lane == 1) { v0 = s0[1]; v1 = s1[1]; }
                    if (lane == 2) { v0 = s0[2]; v1 = s1[2]; }
                    if (lane == 3) { v0 = s0[3]; v1 = s1[3]; }
                    y[i0 + lane] -= v0;
                    y[P + i0 + lane] -= v1;
                }
            }
        }
        __syncthreads();
    }
    for (int b = nblk - 1; b >= 0; --b) {
        const int jb = b * NB, nb = min(NB, P - jb);
        // partial sums over the solved rows below: warps stream rows, lane l owns columns 4l..4l+3
        float acc[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        {
            const int nw = blockDim.x / 32;
            for (int i0 = jb + nb + 4 * warp; i0 < P; i0 += 4 * nw) {
                float4 l4[4];
                float x0[4], x1[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const bool in = i0 + a < P;
                    l4[a] = in ? *reinterpret_cast<const float4*>(Lft + (size_t)(i0 + a) * LD + jb + 4 * lane)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
                    x0[a] = in ? y[i0 + a] : 0.f;
                    x1[a] = in ? y[P + i0 + a] : 0.f;
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    acc[0][0] = fmaf(l4[a].x, x0[a], acc[0][0]);
                    acc[1][0] = fmaf(l4[a].y, x0[a], acc[1][0]);
                    acc[2][0] = fmaf(l4[a].z, x0[a], acc[2][0]);
                    acc[3][0] = fmaf(l4[a].w, x0[a], acc[3][0]);
                    acc[0][1] = fmaf(l4[a].x, x1[a], acc[0][1]);
                    acc[1][1] = fmaf(l4[a].y, x1[a], acc[1][1]);
                    acc[2][1] = fmaf(l4[a].z, x1[a], acc[2][1]);
                    acc[3][1] = fmaf(l4[a].w, x1[a], acc[3][1]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            part[(warp * NB + 4 * lane + u) * 2] = acc[u][0];
            part[(warp * NB + 4 * lane + u) * 2 + 1] = acc[u][1];
        }
        for (int e = tid; e < NB * NB; e += blockDim.x) Db[(e / NB) * DS + e % NB] = Dv[(size_t)b * NB * NB + e];
        __syncthreads();
        for (int e = tid; e < 2 * nb; e += blockDim.x) {
            const int c = e % nb, h = e / nb;
            float sacc = 0.f;
            for (int w = 0; w < 8; ++w) sacc += part[(w * NB + c) * 2 + h];
            tmp[h * NB + c] = y[h * P + jb + c] - sacc;
        }
        __syncthreads();
        for (int e = tid; e < 2 * nb; e += blockDim.x) {
            const int c = e % nb, h = e / nb;
            float sacc = 0.f;
            for (int k = c; k < nb; ++k) sacc = fmaf(Db[k * DS + c], tmp[h * NB + k], sacc);
            y[h * P + jb + c] = sacc;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256, 1) chol_solve_tc_kernel(int t0, int P, int LD, int ns, double eps, int refine,
                                                               const float* __restrict__ G,
                                                               const double* __restrict__ obar,
                                                               const double2* __restrict__ D, const float* __restrict__ Lf,
                                                               const float* __restrict__ Dinv,
                                                               double* __restrict__ xws, double2* __restrict__ delta,
                                                               double* __restrict__ shift_used,
                                                               const int* __restrict__ fail) {
    const int t = t0 + blockIdx.x;
    if (fail[t]) return;
    extern __shared__ __align__(16) float ssm[];
    float* Db = ssm;              // [NB][DS]
    float* tmp = Db + NB * DS;    // [2][NB]
    float* y = tmp + 2 * NB;      // [2][P]
    float* xs = y + 2 * P;        // [4][P] x split into FP32 high and low parts (re h, re l, im h, im l)
    float* part = xs + 4 * P;     // [8][256][2][2] per-warp partial sums
    __shared__ double red[2][8];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float* Lft = Lf + (size_t)t * P * LD;
    const float* Dv = Dinv + (size_t)t * ((P + NB - 1) / NB) * NB * NB;
    const double2* Dt = D + (size_t)t * P;
    double* xr = xws + (size_t)t * 4 * P;
    double* xi = xr + P;
    double* rr = xi + P;
    double* ri = rr + P;
    for (int k = tid; k < P; k += blockDim.x) {
        y[k] = (float)Dt[k].x;
        y[P + k] = (float)Dt[k].y;
    }
    __syncthreads();
    block_solve(P, LD, Lft, Dv, y, Db, tmp, part);
    for (int k = tid; k < P; k += blockDim.x) {
        xr[k] = (double)y[k];
        xi[k] = (double)y[P + k];
    }
    __syncthreads();
    const float* Gt = G + (size_t)t * P * P;
    const double* ob = obar + (size_t)t * P;
    for (int it = 0; it < refine; ++it) {
        double a = 0.0, b = 0.0;
        for (int k = tid; k < P; k += blockDim.x) {
            a += ob[k] * xr[k];
            b += ob[k] * xi[k];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, off);
            b += __shfl_xor_sync(0xffffffffu, b, off);
        }
        if (lane == 0) {
            red[0][warp] = a;
            red[1][warp] = b;
        }
        __syncthreads();
        double oxr = 0.0, oxi = 0.0;
        for (int w = 0; w < 8; ++w) {
            oxr += red[0][w];
            oxi += red[1][w];
        }
        // x = xh + xl in FP32 pairs (48 significant bits)
        for (int k = tid; k < P; k += blockDim.x) {
            const float rh = (float)xr[k], ih = (float)xi[k];
            xs[k] = rh;
            xs[P + k] = (float)(xr[k] - (double)rh);
            xs[2 * P + k] = ih;
            xs[3 * P + k] = (float)(xi[k] - (double)ih);
        }
        __syncthreads();
        // z_j = sum_{i<j} G[i][j] x_i: column chunks of 256, warps stream rows, lane l owns 8 columns
        for (int c0 = 0; c0 < P; c0 += 256) {
            float sh[8][2], sc[8][2];
#pragma unroll
            for (int u = 0; u < 8; ++u) sh[u][0] = sh[u][1] = sc[u][0] = sc[u][1] = 0.f;
            const int iend = min(P, c0 + 256);
            for (int i = warp; i < iend; i += blockDim.x / 32) {
                const float* grow = Gt + (size_t)i * P;
                const float xh0 = xs[i], xl0 = xs[P + i], xh1 = xs[2 * P + i], xl1 = xs[3 * P + i];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int jcol = c0 + 8 * lane + u;
                    if (jcol < P && jcol > i) {
                        const float g = grow[jcol];
                        df_fma(sh[u][0], sc[u][0], g, xh0, xl0);
                        df_fma(sh[u][1], sc[u][1], g, xh1, xl1);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int cl = 8 * lane + u;
                part[((warp * 256 + cl) * 2) * 2] = sh[u][0];
                part[((warp * 256 + cl) * 2) * 2 + 1] = sc[u][0];
                part[((warp * 256 + cl) * 2 + 1) * 2] = sh[u][1];
                part[((warp * 256 + cl) * 2 + 1) * 2 + 1] = sc[u][1];
            }
            __syncthreads();
            for (int cl = tid; cl < 256 && c0 + cl < P; cl += blockDim.x) {
                double zr = 0.0, zi = 0.0;
                for (int w = 0; w < 8; ++w) {
                    zr += (double)part[((w * 256 + cl) * 2) * 2] + (double)part[((w * 256 + cl) * 2) * 2 + 1];
                    zi += (double)part[((w * 256 + cl) * 2 + 1) * 2] + (double)part[((w * 256 + cl) * 2 + 1) * 2 + 1];
                }
                rr[c0 + cl] = zr;
                ri[c0 + cl] = zi;
            }
            __syncthreads();
        }
        // y_i = sum_{j>=i} G[i][j] x_j, one warp per row; residual D - (S + eps I) x
        for (int i = warp; i < P; i += blockDim.x / 32) {
            const float* grow = Gt + (size_t)i * P;
            float h0 = 0.f, c0f = 0.f, h1 = 0.f, c1f = 0.f;
            for (int jj = i + lane; jj < P; jj += 32) {
                const float g = grow[jj];
                df_fma(h0, c0f, g, xs[jj], xs[P + jj]);
                df_fma(h1, c1f, g, xs[2 * P + jj], xs[3 * P + jj]);
            }
            double yr2 = (double)h0 + (double)c0f, yi2 = (double)h1 + (double)c1f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                yr2 += __shfl_xor_sync(0xffffffffu, yr2, off);
                yi2 += __shfl_xor_sync(0xffffffffu, yi2, off);
            }
            if (lane == 0) {
                const double sxr = (yr2 + rr[i]) / ns - ob[i] * oxr + eps * xr[i];
                const double sxi = (yi2 + ri[i]) / ns - ob[i] * oxi + eps * xi[i];
                y[i] = (float)(Dt[i].x - sxr);
                y[P + i] = (float)(Dt[i].y - sxi);
            }
        }
        __syncthreads();
        block_solve(P, LD, Lft, Dv, y, Db, tmp, part);
        for (int k = tid; k < P; k += blockDim.x) {
            xr[k] += (double)y[k];
            xi[k] += (double)y[P + k];
        }
        __syncthreads();
    }
    for (int k = tid; k < P; k += blockDim.x) delta[(size_t)t * P + k] = make_double2(xr[k], xi[k]);
    if (tid == 0 && shift_used) shift_used[t] = eps;
}

inline int ldim(int P) { return ((P + 63) / 64) * 64; }

constexpr int CHOL_GROUPS = 4;
struct GroupStreams {
    cudaStream_t s[CHOL_GROUPS];
    cudaEvent_t fork;
    cudaEvent_t join[CHOL_GROUPS];
};
// Streams of the current device for the trajectory groups, created once per device.
inline GroupStreams& group_streams() {
    static std::mutex mu;
    static GroupStreams per_dev[16];
    static bool made[16] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    GroupStreams& g = per_dev[dev & 15];
    if (!made[dev & 15]) {
        for (int i = 0; i < CHOL_GROUPS; ++i) {
            cudaStreamCreateWithFlags(&g.s[i], cudaStreamNonBlocking);
            cudaEventCreateWithFlags(&g.join[i], cudaEventDisableTiming);
        }
        cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming);
        made[dev & 15] = true;
    }
    return g;
}

}  // namespace chol

size_t chol_tc_ws_bytes(int ntraj, int P) {
    using namespace chol;
    const size_t LD = ldim(P), nblk = (P + NB - 1) / NB;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += (bytes + 255) & ~(size_t)255; };
    add((size_t)ntraj * NPC * ((P + NB - 1) / NB) * 128 * LD * 2);   // Lb (tiled)
    add((size_t)ntraj * P * LD * 4);         // Lf (also the fallback solver's factor)
    add((size_t)ntraj * P * NB * 4);         // Pn
    add((size_t)ntraj * nblk * NB * NB * 4); // Dinv
    add((size_t)ntraj * 4);                  // fail
    add((size_t)ntraj * 2 * P * 4);          // fallback y
    add((size_t)ntraj * 4 * P * 8);          // x, residual
    return b + 256;
}

// Fallback: the single-CTA solver of k_solve.cu restricted to the marked trajectories.
cudaError_t launch_chol_solve_masked(int ntraj, int P, int ns, double eps, const float* G, const double* obar,
                                     const double2* D, double2* delta, double* shift_used, float* L, float* y,
                                     double* x, int refine_iters, const int* only, int* status, cudaStream_t s);

static cudaError_t chol_fail(cudaError_t e, const char* what) {
    if (e != cudaSuccess) set_error(std::string("cholesky: ") + what + ": " + cudaGetErrorString(e));
    return e;
}

cudaError_t launch_chol_tc(int ntraj, int P, int ns, double eps, const float* G, const double* obar,
                           const double2* D, double2* delta, double* shift_used, void* ws, int refine_iters,
                           int* status, cudaStream_t s) {
    using namespace chol;
    set_error("");
    const int LD = ldim(P);
    const size_t nblk = (P + NB - 1) / NB;
    char* p = (char*)ws;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)r;
    };
    const int NT = (P + NB - 1) / NB, KB = LD / 64;
    __nv_bfloat16* Lb = (__nv_bfloat16*)take((size_t)ntraj * NPC * NT * 128 * LD * 2);
    float* Lf = (float*)take((size_t)ntraj * P * LD * 4);
    float* Pn = (float*)take((size_t)ntraj * P * NB * 4);
    float* Dv = (float*)take((size_t)ntraj * nblk * NB * NB * 4);
    int* fail = (int*)take((size_t)ntraj * 4);
    float* yf = (float*)take((size_t)ntraj * 2 * P * 4);
    double* x = (double*)take((size_t)ntraj * 4 * P * 8);

    auto encode = tc::get_encode();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[4] = {64u, 128u, (cuuint64_t)KB, (cuuint64_t)ntraj * NPC * NT};
    const cuuint64_t strides[3] = {128u, 128u * 128u, (cuuint64_t)KB * 128u * 128u};
    const cuuint32_t box[4] = {(cuuint32_t)BK, 128u, 1u, 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    const CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void*)Lb, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "cholesky: cuTensorMapEncodeTiled returned %d (addr %p dims %llu %llu %llu %llu strides %llu %llu "
                 "%llu box %u %u)",
                 (int)cr, (void*)Lb, (unsigned long long)dims[0], (unsigned long long)dims[1],
                 (unsigned long long)dims[2], (unsigned long long)dims[3], (unsigned long long)strides[0],
                 (unsigned long long)strides[1], (unsigned long long)strides[2], box[0], box[1]);
        set_error(buf);
        return cudaErrorInvalidValue;
    }

    cudaError_t e = cudaMemsetAsync(fail, 0, (size_t)ntraj * 4, s);
    if (e != cudaSuccess) return chol_fail(e, "memset");
    const int dsmem = (NB * DS + NB) * (int)sizeof(float);
    const int tsmem = (NB + RT) * DS * (int)sizeof(float);
    e = cudaFuncSetAttribute(chol_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem);
    if (e != cudaSuccess) return chol_fail(e, "diag attribute");
    e = cudaFuncSetAttribute(chol_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tsmem);
    if (e != cudaSuccess) return chol_fail(e, "trsm attribute");
    e = cudaFuncSetAttribute(chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_U);
    if (e != cudaSuccess) return chol_fail(e, "update attribute");
    const float feps = (float)eps;
    const int ssmem = (NB * DS + 2 * NB + 2 * P + 4 * P + 8 * 256 * 2 * 2) * (int)sizeof(float);
    e = cudaFuncSetAttribute(chol_solve_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ssmem);
    if (e != cudaSuccess) return chol_fail(e, "solve attribute");
    // trajectory groups on forked streams: one group's latency-bound kernels overlap the
    // others' (fork and join by events, so the call stays ordered on `s`)
    const int ng = ntraj >= 16 ? CHOL_GROUPS : 1;
    GroupStreams& gs = group_streams();
    if (ng > 1) {
        e = cudaEventRecord(gs.fork, s);
        if (e != cudaSuccess) return chol_fail(e, "fork record");
    }
    for (int g = 0; g < ng; ++g) {
        const int ta = (int)((long long)ntraj * g / ng), tb = (int)((long long)ntraj * (g + 1) / ng);
        const int nt = tb - ta;
        if (nt <= 0) continue;
        cudaStream_t gsm = ng > 1 ? gs.s[g] : s;
        if (ng > 1 && (e = cudaStreamWaitEvent(gsm, gs.fork, 0)) != cudaSuccess) return e;
        for (int jb = 0; jb < P; jb += NB) {
            if (jb > 0) {
                ProfScope pu(OTVMC_K_CHOLU, gsm);
                dim3 grid((P - jb + 127) / 128, nt);
                chol_update_kernel<<<grid, 192, SMEM_U, gsm>>>(map, ta, P, ns, NT, jb, feps, G, obar, Pn, fail, status);
                count_launch();
            }
            {
                ProfScope pd(OTVMC_K_CHOLD, gsm);
                chol_diag_kernel<<<nt, 256, dsmem, gsm>>>(ta, P, LD, ns, jb, feps, G, obar, Pn, Lf, Lb, Dv, fail);
                count_launch();
            }
            const int nrows = P - jb - min(NB, P - jb);
            if (nrows > 0) {
                ProfScope pp(OTVMC_K_CHOLP, gsm);
                dim3 grid((nrows + RT - 1) / RT, nt);
                chol_trsm_kernel<<<grid, 256, tsmem, gsm>>>(ta, P, LD, ns, jb, feps, G, obar, Pn, Lf, Lb, Dv, fail);
                count_launch();
            }
        }
        {
            ProfScope ps(OTVMC_K_SOLVE, gsm);
            chol_solve_tc_kernel<<<nt, 256, ssmem, gsm>>>(ta, P, LD, ns, eps, refine_iters, G, obar, D, Lf, Dv, x,
                                                           delta, shift_used, fail);
            count_launch();
        }
        if (ng > 1) {
            if ((e = cudaEventRecord(gs.join[g], gsm)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, gs.join[g], 0)) != cudaSuccess) return e;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return chol_fail(e, "kernel launch");
    // trajectories whose pivot failed: robust solver with shift retries (exits at once for the others)
    return launch_chol_solve_masked(ntraj, P, ns, eps, G, obar, D, delta, shift_used, Lf, yf, x, refine_iters, fail,
                                    status, s);
}

}  // namespace otvmc
