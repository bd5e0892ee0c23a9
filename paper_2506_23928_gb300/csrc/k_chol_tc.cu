// Regularised solve (S + eps I) delta = D of the otVMC equation (Eq. 8 with the
// diagonal-shift regulariser), batched over trajectories, with the O(P^3) part of the
// Cholesky factorization on the tensor cores.
//
// Left-looking blocked Cholesky, 128-wide block columns jb = 0, 128, ...:
//   update  (tcgen05)  C[i, jb:jb+128] = A[i, jb:jb+128] - sum_{k<jb} L[i,k] L[jb+c,k], i >= jb.
//           L is kept as three BF16 pieces (L = h + m + l to ~2^-24 relative); the six
//           products h.h + h.m + m.h + h.l + m.m + l.h accumulate in FP32 in TMEM, which
//           gives FP32-level accuracy.  One CTA = 128 rows x 128 columns of one trajectory.
//   panel   (SIMT)     factor the 128 x 128 diagonal block in shared memory, invert it, and
//           solve the rows below as a small GEMM X = C L_dd^-T; write L in FP32 (for the
//           triangular solves) and as BF16 pieces (for later updates), and L_dd^-1.
// solve     (SIMT)     forward/backward substitution by blocks through the stored inverses,
//           then one step of iterative refinement with the residual D - (S + eps I) x formed
//           in FP64 from the exact Gram counts (S = G/ns - obar obar^T).
// A trajectory whose pivot is not positive is marked and solved again by the single-CTA
// solver, which raises the shift (x100, at most three times).
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace otvmc {
namespace chol {

constexpr int NB = 128;                  // block column width
constexpr int BK = 64;                   // k extent of one TMA box (bf16: 128 bytes)
constexpr int NPC = 3;                   // bf16 pieces of L
constexpr int BOX = 128 * BK * 2;        // one 128-row box: 16 KB
constexpr int STAGE = 2 * NPC * BOX;     // A pieces + B pieces: 96 KB
constexpr int STAGES = 2;
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
__global__ void __launch_bounds__(192, 1) chol_update_kernel(const __grid_constant__ CUtensorMap tmap, int P, int ns,
                                                             int jb, float eps, const float* __restrict__ G,
                                                             const double* __restrict__ obar, float* __restrict__ Pn,
                                                             const int* __restrict__ fail, int* status) {
    using namespace tc;
    const int t = blockIdx.y;
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
                for (int p = 0; p < NPC; ++p) {
                    tma_load_3d(st + p * BOX, &tmap, &full[s], kb * BK, i0, t * NPC + p);
                    tma_load_3d(st + (NPC + p) * BOX, &tmap, &full[s], kb * BK, jb, t * NPC + p);
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
                        umma(tmem, smem_desc(st + pa[q] * BOX + k * 32), smem_desc(st + (NPC + pb[q]) * BOX + k * 32),
                             ID, (kb > 0 || k > 0 || q > 0) ? 1u : 0u);
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
__device__ __forceinline__ void store_L(float* Lf, __nv_bfloat16* Lb, size_t plane, size_t idx, float x) {
    Lf[idx] = x;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    Lb[idx] = h;
    Lb[plane + idx] = m;
    Lb[2 * plane + idx] = __float2bfloat16_rn(r2);
}

__global__ void __launch_bounds__(256, 1) chol_panel_kernel(int P, int LD, int ns, int jb, float eps,
                                                            const float* __restrict__ G,
                                                            const double* __restrict__ obar,
                                                            const float* __restrict__ Pn, float* __restrict__ Lf,
                                                            __nv_bfloat16* __restrict__ Lb, float* __restrict__ Dinv,
                                                            int* __restrict__ fail) {
    const int t = blockIdx.x;
    if (fail[t]) return;
    extern __shared__ __align__(16) float psm[];
    float* Dg = psm;             // [NB][DS] diagonal block, then its Cholesky factor
    float* Li = Dg + NB * DS;    // [NB][DS] inverse of the factor
    float* Ct = Li + NB * DS;    // [RT][DS] panel rows
    __shared__ int bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = min(NB, P - jb);
    const float* Gt = G + (size_t)t * P * P;
    const double* ob = obar + (size_t)t * P;
    const float inv_ns = 1.0f / (float)ns;
    const size_t LL = (size_t)P * LD;             // elements of one trajectory's L
    float* Lft = Lf + (size_t)t * LL;
    __nv_bfloat16* Lbt = Lb + (size_t)t * NPC * LL;
    auto C = [&](int i, int c) -> float {  // updated block column entry (i >= jb + c)
        return jb == 0 ? a_orig(Gt, ob, P, inv_ns, i, jb + c, eps) : Pn[((size_t)t * P + i) * NB + c];
    };
    if (tid == 0) bad = 0;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, c = e - i * nb;
        Dg[i * DS + c] = (c <= i) ? C(jb + i, c) : 0.f;
    }
    __syncthreads();
    for (int p = 0; p < nb; ++p) {
        if (tid == 0) {
            const float d = Dg[p * DS + p];
            if (!(d > 0.f) || !isfinite(d)) bad = 1;
            else Dg[p * DS + p] = sqrtf(d);
        }
        __syncthreads();
        if (bad) break;
        const float piv = Dg[p * DS + p];
        for (int i = p + 1 + tid; i < nb; i += blockDim.x) Dg[i * DS + p] /= piv;
        __syncthreads();
        for (int i = p + 1 + warp; i < nb; i += blockDim.x / 32) {
            const float lip = Dg[i * DS + p];
            for (int c = p + 1 + lane; c <= i; c += 32) Dg[i * DS + c] -= lip * Dg[c * DS + p];
        }
        __syncthreads();
    }
    if (bad) {
        if (tid == 0) fail[t] = 1;
        return;
    }
    // inverse of the lower-triangular factor, one column per thread
    if (tid < nb) {
        const int c = tid;
        for (int i = 0; i < nb; ++i) {
            float v = 0.f;
            if (i == c) {
                v = 1.f / Dg[i * DS + i];
            } else if (i > c) {
                float s = 0.f;
                for (int k = c; k < i; ++k) s = fmaf(Dg[i * DS + k], Li[k * DS + c], s);
                v = -s / Dg[i * DS + i];
            }
            Li[i * DS + c] = v;
        }
    }
    __syncthreads();
    const int bidx = jb / NB;
    float* Dv = Dinv + ((size_t)t * ((P + NB - 1) / NB) + bidx) * NB * NB;
    for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, c = e - i * NB;
        Dv[e] = (i < nb && c < nb) ? Li[i * DS + c] : 0.f;
        if (i < nb && c < nb) store_L(Lft, Lbt, LL, (size_t)(jb + i) * LD + jb + c, c <= i ? Dg[i * DS + c] : 0.f);
    }
    // rows below the diagonal block: X = C L_dd^-T in tiles of RT rows
    const int r = tid % RT, cc = tid / RT;  // row of the tile, chunk of 32 columns
    for (int r0 = jb + nb; r0 < P; r0 += RT) {
        __syncthreads();
        for (int e = tid; e < RT * nb; e += blockDim.x) {
            const int rr = e / nb, c = e - rr * nb;
            Ct[rr * DS + c] = (r0 + rr < P) ? C(r0 + rr, c) : 0.f;
        }
        __syncthreads();
        float acc[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) acc[u] = 0.f;
        const int kend = min(nb, cc * 32 + 32);
        for (int k = 0; k < kend; ++k) {
            const float a = Ct[r * DS + k];
#pragma unroll
            for (int u = 0; u < 32; ++u) acc[u] = fmaf(a, Li[(cc * 32 + u) * DS + k], acc[u]);
        }
        const int i = r0 + r;
        if (i < P)
#pragma unroll
            for (int u = 0; u < 32; ++u) {
                const int c = cc * 32 + u;
                if (c < nb) store_L(Lft, Lbt, LL, (size_t)i * LD + jb + c, acc[u]);
            }
    }
}

// ------------------------------------------------------------------------------ solves
// L L^T x = y for two right-hand sides held in shared memory (y[0..P), y[P..2P)).
__device__ void block_solve(int P, int LD, const float* Lft, const float* Dv, float* y, float* Db, float* tmp) {
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
        for (int i = jb + nb + warp; i < P; i += blockDim.x / 32) {
            const float* row = Lft + (size_t)i * LD + jb;
            float s0 = 0.f, s1 = 0.f;
            for (int c = lane; c < nb; c += 32) {
                const float l = row[c];
                s0 = fmaf(l, y[jb + c], s0);
                s1 = fmaf(l, y[P + jb + c], s1);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, off);
                s1 += __shfl_xor_sync(0xffffffffu, s1, off);
            }
            if (lane == 0) {
                y[i] -= s0;
                y[P + i] -= s1;
            }
        }
        __syncthreads();
    }
    for (int b = nblk - 1; b >= 0; --b) {
        const int jb = b * NB, nb = min(NB, P - jb);
        for (int e = tid; e < 2 * nb; e += blockDim.x) {
            const int c = e % nb, h = e / nb;
            float s = 0.f;
            for (int i = jb + nb; i < P; ++i) s = fmaf(Lft[(size_t)i * LD + jb + c], y[h * P + i], s);
            tmp[h * NB + c] = y[h * P + jb + c] - s;
        }
        for (int e = tid; e < NB * NB; e += blockDim.x) Db[(e / NB) * DS + e % NB] = Dv[(size_t)b * NB * NB + e];
        __syncthreads();
        for (int e = tid; e < 2 * nb; e += blockDim.x) {
            const int c = e % nb, h = e / nb;
            float s = 0.f;
            for (int k = c; k < nb; ++k) s = fmaf(Db[k * DS + c], tmp[h * NB + k], s);
            y[h * P + jb + c] = s;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256, 1) chol_solve_tc_kernel(int P, int LD, int ns, double eps, int refine,
                                                               const float* __restrict__ G,
                                                               const double* __restrict__ obar,
                                                               const double2* __restrict__ D, const float* __restrict__ Lf,
                                                               const float* __restrict__ Dinv,
                                                               double* __restrict__ xws, double2* __restrict__ delta,
                                                               double* __restrict__ shift_used,
                                                               const int* __restrict__ fail) {
    const int t = blockIdx.x;
    if (fail[t]) return;
    extern __shared__ __align__(16) float ssm[];
    float* Db = ssm;              // [NB][DS]
    float* tmp = Db + NB * DS;    // [2][NB]
    float* y = tmp + 2 * NB;      // [2][P]
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
    block_solve(P, LD, Lft, Dv, y, Db, tmp);
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
        for (int j = tid; j < P; j += blockDim.x) {
            double zr = 0.0, zi = 0.0;
            for (int i = 0; i < j; ++i) {
                const double g = (double)Gt[(size_t)i * P + j];
                zr = fma(g, xr[i], zr);
                zi = fma(g, xi[i], zi);
            }
            rr[j] = zr;
            ri[j] = zi;
        }
        __syncthreads();
        for (int i = warp; i < P; i += blockDim.x / 32) {
            double yr2 = 0.0, yi2 = 0.0;
            for (int j = i + lane; j < P; j += 32) {
                const double g = (double)Gt[(size_t)i * P + j];
                yr2 = fma(g, xr[j], yr2);
                yi2 = fma(g, xi[j], yi2);
            }
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
        block_solve(P, LD, Lft, Dv, y, Db, tmp);
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

}  // namespace chol

size_t chol_tc_ws_bytes(int ntraj, int P) {
    using namespace chol;
    const size_t LD = ldim(P), nblk = (P + NB - 1) / NB;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += (bytes + 255) & ~(size_t)255; };
    add((size_t)ntraj * NPC * P * LD * 2);   // Lb
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

cudaError_t launch_chol_tc(int ntraj, int P, int ns, double eps, const float* G, const double* obar,
                           const double2* D, double2* delta, double* shift_used, void* ws, int refine_iters,
                           int* status, cudaStream_t s) {
    using namespace chol;
    ProfScope prof_(OTVMC_K_SOLVE, s);
    const int LD = ldim(P);
    const size_t nblk = (P + NB - 1) / NB;
    char* p = (char*)ws;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)r;
    };
    __nv_bfloat16* Lb = (__nv_bfloat16*)take((size_t)ntraj * NPC * P * LD * 2);
    float* Lf = (float*)take((size_t)ntraj * P * LD * 4);
    float* Pn = (float*)take((size_t)ntraj * P * NB * 4);
    float* Dv = (float*)take((size_t)ntraj * nblk * NB * NB * 4);
    int* fail = (int*)take((size_t)ntraj * 4);
    float* yf = (float*)take((size_t)ntraj * 2 * P * 4);
    double* x = (double*)take((size_t)ntraj * 4 * P * 8);

    auto encode = tc::get_encode();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)LD, (cuuint64_t)P, (cuuint64_t)ntraj * NPC};
    const cuuint64_t strides[2] = {(cuuint64_t)LD * 2, (cuuint64_t)P * LD * 2};
    const cuuint32_t box[3] = {(cuuint32_t)BK, 128u, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)Lb, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;

    cudaError_t e = cudaMemsetAsync(fail, 0, (size_t)ntraj * 4, s);
    if (e != cudaSuccess) return e;
    const int psmem = (2 * NB + RT) * DS * (int)sizeof(float);
    e = cudaFuncSetAttribute(chol_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_U);
    if (e != cudaSuccess) return e;
    const float feps = (float)eps;
    for (int jb = 0; jb < P; jb += NB) {
        if (jb > 0) {
            dim3 grid((P - jb + 127) / 128, ntraj);
            chol_update_kernel<<<grid, 192, SMEM_U, s>>>(map, P, ns, jb, feps, G, obar, Pn, fail, status);
            count_launch();
        }
        chol_panel_kernel<<<ntraj, 256, psmem, s>>>(P, LD, ns, jb, feps, G, obar, Pn, Lf, Lb, Dv, fail);
        count_launch();
    }
    const int ssmem = (NB * DS + 2 * NB + 2 * P) * (int)sizeof(float);
    e = cudaFuncSetAttribute(chol_solve_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ssmem);
    if (e != cudaSuccess) return e;
    chol_solve_tc_kernel<<<ntraj, 256, ssmem, s>>>(P, LD, ns, eps, refine_iters, G, obar, D, Lf, Dv, x, delta,
                                                    shift_used, fail);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // trajectories whose pivot failed: robust solver with shift retries (exits at once for the others)
    return launch_chol_solve_masked(ntraj, P, ns, eps, G, obar, D, delta, shift_used, Lf, yf, x, refine_iters, fail,
                                    status, s);
}

}  // namespace otvmc
