// Regularised solve (S + eps I) delta = D of the otVMC equation (Eq. 8 with the
// diagonal-shift regulariser), batched over trajectories, with the O(P^3) part of the
// Cholesky factorization on the tensor cores.
//
// Left-looking blocked Cholesky, 128-wide block columns jb = 0, 128, ...:
//   update  (tcgen05)  C[i, jb:jb+128] = A[i, jb:jb+128] - sum_{k<jb} L[i,k] L[jb+c,k], i >= jb.
//           L is kept as two FP16 pieces (L = h + m to 22 significant bits; the entries of L
//           are bounded by the square roots of the matrix's diagonal, at most 1 + eps for the
//           Jastrow S, far inside FP16's range); the three products h.h + h.m + m.h accumulate
//           in FP32 in TMEM (the dropped m.m is below 2^-22 of the product).  One CTA = 128 rows x 128 columns of
//           one trajectory; 32-column k slices (64-byte swizzle) in a 3-stage ring, two CTAs
//           per SM.
//   diag    (SIMT)     factor the 128 x 128 diagonal block and invert its factor in one pass of
//           right-looking elimination over register-held 8 x 8 tiles;
//   panel   (tcgen05)  the rows below, X = C L_dd^-T, with C (written by the update kernel as
//           FP16 pieces) and L_dd^-1 (written by the diagonal kernel as FP16 pieces) through the
//           same three piece products over K = 128, one 128-row tile per CTA; diag and panel
//           write L in FP32 (for the triangular solves) and as FP16 pieces (for later updates).
//   The factor is accurate to a few 2^-22 of |S|; the refinement below, whose residual is exact,
//   brings the solution to the accuracy of the FP64 solve.  Every trajectory's system is
//   factored divided by a power of two s >= max_i (S + eps I)_ii (chol_scale_kernel), which
//   changes no rounding and bounds the entries of L by 1, inside FP16's range for any S; a
//   block inverse beyond FP16's range (a near-singular S) sends the trajectory to the fallback.
//   The forward substitution L y = D rides along: diag applies L_dd^-1 to its block of the
//   right-hand side, the panel kernel subtracts the block's contribution from the rows below.
// solve     (SIMT)     backward substitution x = L^-T y by blocks through the stored inverses,
//           then iterative refinement: the residual D - (S + eps I) x from the exact Gram
//           counts (S = G/ns - obar obar^T) in double-float arithmetic, tile-parallel over
//           many CTAs, and one more forward and backward substitution for the correction.
// A trajectory whose pivot is not positive is marked and solved again by the single-CTA
// solver, which raises the shift (x100, at most three times).
#include <cuda_fp16.h>

#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"
#include "tc_common.cuh"

namespace otvmc {
namespace chol {

using piece_t = __half;                   // operand pieces of the tensor-core products
constexpr int NB = 128;                  // block column width
constexpr int BK = 32;                   // k extent of one operand box (fp16: 64 bytes, 64-byte swizzle)
constexpr int NPC = 2;                   // fp16 pieces of L (h + m: 22 significant bits)
constexpr int NPROD = 3;                 // piece products kept: h.h, h.m, m.h
constexpr int BOX = 128 * BK * 2;        // one 128-row box: 8 KB
constexpr int STAGE = 2 * NPC * BOX;     // A pieces + B pieces: 32 KB
constexpr int STAGES = 3;                // about 97 KB of shared memory: two CTAs per SM
constexpr int SMEM_U = STAGES * STAGE + 1024 + 256;
constexpr uint32_t TCOLS = 128;

__device__ __forceinline__ float a_orig(const float* Gt, const double* ob, int P, float inv_ns, int i, int j,
                                        float eps) {
    // (S + eps I)_ij for j <= i from the upper-triangle Gram counts, in FP32
    float v = Gt[(size_t)j * P + i] * inv_ns - (float)ob[i] * (float)ob[j];
    return i == j ? v + eps : v;
}

// ------------------------------------------------------------------ piece layout
// FP16 pieces of L are stored tiled: for piece p of trajectory t, the 128-row tile i / 128
// and the 32-column chunk k / 32 form one contiguous 8 KB block [i % 128][k % 32] laid out
// exactly as the update kernel's shared-memory operand box: rows of 64 bytes with the
// 64-byte swizzle (16-byte unit u of row r stored at unit u ^ ((r / 2) mod 4)), so that one
// box is one contiguous bulk copy.
struct LbLayout {
    int NT;  // row tiles, ceil(P / 128)
    int KC;  // 32-column chunks, LD / 32
    __host__ __device__ __forceinline__ size_t plane() const { return (size_t)NT * KC * 128 * 32; }
    __device__ __forceinline__ size_t at(int i, int k) const {
        const int r = i & 127, u = (k & 31) >> 3;
        return (((size_t)(i >> 7) * KC + (k >> 5)) * 128 + r) * 32 + ((u ^ ((r >> 1) & 3)) << 3) + (k & 7);
    }
};

__device__ __forceinline__ uint32_t pack_h2(piece_t lo, piece_t hi) {
    return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}
// x = h + m with h = fp16(x), m = fp16(x - h): 22 significant bits for |x| in the normal range
// of m, an absolute error below 2^-25 for smaller |x| (subnormal m); |x| < 65504.
__device__ __forceinline__ void split2(float x, piece_t& h, piece_t& m) {
    h = __float2half_rn(x);
    m = __float2half_rn(x - __half2float(h));
}

// The two FP16 pieces of eight consecutive entries (a 16-byte unit of each piece's plane).
__device__ __forceinline__ void store_P8(piece_t* Bt, size_t pl, size_t idx, const float (&v)[8]) {
    uint32_t h[4], m[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        piece_t hp[2], mp[2];
#pragma unroll
        for (int w = 0; w < 2; ++w) split2(v[2 * u + w], hp[w], mp[w]);
        h[u] = pack_h2(hp[0], hp[1]);
        m[u] = pack_h2(mp[0], mp[1]);
    }
    *reinterpret_cast<uint4*>(Bt + idx) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(Bt + pl + idx) = make_uint4(m[0], m[1], m[2], m[3]);
}

// ------------------------------------------------------------------------- update (tcgen05)
__global__ void __launch_bounds__(192, 2) chol_update_kernel(const piece_t* __restrict__ Lb, size_t plane,
                                                             int KC, int t0, int P, int ns, int jb, float eps,
                                                             const float* __restrict__ inv_s,
                                                             const float* __restrict__ G,
                                                             const double* __restrict__ obar, float* __restrict__ Pn,
                                                             piece_t* __restrict__ Cb, size_t planeC,
                                                             const int* __restrict__ fail, int* status) {
    using namespace tc;
    const int t = t0 + blockIdx.y;
    if (fail[t]) return;
    extern __shared__ uint8_t smem_raw[];
    __shared__ float obj_s[NB];
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
                // k slice kb = chunk kb of the row tiles i0 / 128 (A) and jb / 128 (B): each an
                // 8 KB contiguous image of the swizzled shared-memory box
                for (int p = 0; p < NPC; ++p) {
                    const piece_t* pl = Lb + (size_t)(t * NPC + p) * plane;
                    bulk_load(st + p * BOX, pl + ((size_t)(i0 >> 7) * KC + kb) * (BOX / 2), BOX, &full[s]);
                    bulk_load(st + (NPC + p) * BOX, pl + ((size_t)(jb >> 7) * KC + kb) * (BOX / 2), BOX, &full[s]);
                }
                ++issued;
            }
            for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
                mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // piece products kept: (h,h) (h,m) (m,h)
            const int pa[NPROD] = {0, 0, 1};
            const int pb[NPROD] = {0, 1, 0};
            constexpr uint32_t ID = idesc_f16(128, NB);
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
                    for (int q = 0; q < NPROD; ++q)
                        umma(tmem, smem_desc_sw64(st + pa[q] * BOX + k * 32),
                             smem_desc_sw64(st + (NPC + pb[q]) * BOX + k * 32), ID, (kb > 0 || k > 0 || q > 0) ? 1u : 0u);
                umma_commit(&empty[s]);
            }
            umma_commit(done);
        }
        __syncwarp();
    } else {
        // epilogue: C = A - acc.  The diagonal tile (blockIdx.x = 0) goes to PnT[t][c][i]
        // (FP32, transposed, so that the lanes of a warp store consecutive addresses) for the
        // diagonal-block kernel; the tiles below go out as two FP16 pieces in the operand-box
        // layout of the panel kernel (one 16-byte unit of each piece per 8 columns of a row).
        const int q = warp & 3;
        const float* Gt = G + (size_t)t * P * P;
        const double* ob = obar + (size_t)t * P;
        for (int c = threadIdx.x - 64; c < NB; c += 128) obj_s[c] = jb + c < P ? (float)ob[jb + c] : 0.f;
        int ok = 0;
        if (lane == 0) {
            ok = mbar_wait(done, 0, abort_flag) && !*abort_flag;
            if (!ok) *abort_flag = 1;  // a wait that ran out here is reported as well
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        fence_after();
        asm volatile("bar.sync 1, 128;" ::: "memory");  // obj_s written by the four epilogue warps
        if (ok) {
            const int i = i0 + q * 32 + lane;
            const int ii = i < P ? i : P - 1;
            const float inv_ns = 1.0f / (float)ns, sc = inv_s[t];
            const float obi = (float)ob[ii];
            float* pcol = Pn + (size_t)t * NB * P + ii;
#pragma unroll 1
            for (int c0 = 0; c0 < NB; c0 += 32) {
                // the chunk's 32 Gram counts first, unconditionally (clamped index), so that the
                // loads are all in flight before any store
                float g[32];
#pragma unroll
                for (int u = 0; u < 32; ++u) g[u] = __ldg(Gt + (size_t)min(jb + c0 + u, P - 1) * P + ii);
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                if (i >= P) continue;
                if (blockIdx.x == 0) {
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const int j = jb + c0 + u;
                        if (j < P && j <= i) {
                            float a = g[u] * inv_ns - obi * obj_s[c0 + u];
                            if (i == j) a += eps;
                            pcol[(size_t)(c0 + u) * P] = a * sc - __uint_as_float(v[u]);
                        }
                    }
                } else {
                    // rows below the diagonal block: every column j = jb + c0 + u < i
                    const LbLayout layC{(P + NB - 1) / NB, NB / BK};
                    piece_t* Cbt = Cb + (size_t)t * NPC * planeC;
#pragma unroll
                    for (int u8 = 0; u8 < 4; ++u8) {
                        float c8[8];
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            const int u = 8 * u8 + w;
                            c8[w] = (g[u] * inv_ns - obi * obj_s[c0 + u]) * sc - __uint_as_float(v[u]);
                        }
                        store_P8(Cbt, planeC, layC.at(i, c0 + 8 * u8), c8);
                    }
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

// Eight consecutive entries L[i][k0 .. k0+8) (k0 a multiple of 8): FP32 copy for the
// triangular solves and the two FP16 pieces h + m for the tensor-core updates.
// Only the first nv entries are in the matrix.
__device__ __forceinline__ void store_L8(float* Lft, piece_t* Lbt, const LbLayout& lay, int LD, int i, int k0,
                                         const float (&v)[8], int nv) {
    piece_t hp[8], mp[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) split2(v[u], hp[u], mp[u]);
    const size_t idx = lay.at(i, k0), pl = lay.plane();
    float* dst = Lft + (size_t)i * LD + k0;
    if (nv >= 8) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
        *reinterpret_cast<uint4*>(Lbt + idx) = make_uint4(pack_h2(hp[0], hp[1]), pack_h2(hp[2], hp[3]),
                                                          pack_h2(hp[4], hp[5]), pack_h2(hp[6], hp[7]));
        *reinterpret_cast<uint4*>(Lbt + pl + idx) = make_uint4(pack_h2(mp[0], mp[1]), pack_h2(mp[2], mp[3]),
                                                               pack_h2(mp[4], mp[5]), pack_h2(mp[6], mp[7]));
    } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < nv) {
                dst[u] = v[u];
                Lbt[idx + u] = hp[u];
                Lbt[pl + idx + u] = mp[u];
            }
    }
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__device__ __forceinline__ float dot4(float4 a, float4 b, float s) {
    return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, s))));
}

// Sum over the 32 lanes of eight values per lane in 9 shuffles (each step halves the values a
// lane keeps).  Lane l ends with the total of value 4 b4 + 2 b3 + b2, where b4 b3 b2 are bits
// 4, 3, 2 of l; the four lanes that differ in bits 0 and 1 hold the same total.
__device__ __forceinline__ float reduce8(float (&v)[8], int lane) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const bool up = lane & 16;
        const float send = up ? v[u] : v[u + 4];
        const float keep = up ? v[u + 4] : v[u];
        v[u] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const bool up = lane & 8;
        const float send = up ? v[u] : v[u + 2];
        const float keep = up ? v[u + 2] : v[u];
        v[u] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const bool up = lane & 4;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}
__device__ __forceinline__ int reduce8_index(int lane) {
    return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// ----------------------------------------------------------------------- diagonal block
// Cholesky factor L_dd of the 128 x 128 diagonal block of block column jb and its inverse
// X = L_dd^-1, one CTA of eight warps per trajectory, by 4 x 4 tiles of 32 (right-looking):
//   for k = 0..3:
//     L_kk, X_kk <- factor32(A_kk)                      (one warp, registers, shared broadcasts)
//     L_ik = A_ik X_kk^T (i > k);   X_kj = X_kk W_kj (j < k)
//     A_ij -= L_ik L_jk^T (k < j <= i);   W_ij -= L_ik X_kj (i > k, j <= k)
// W starts as the identity, so that X is the block forward substitution of L X = I.  The tile
// products are warp-level SIMT GEMMs on float4 shared-memory operands.  Warp 0 updates A_k+1,k+1
// first and factors it at once, while the other warps finish the remaining updates of step k.
// The forward substitution of the solve is fused in: the block's right-hand sides (D for the
// first block, else the running residual that the panel kernels of earlier block columns left
// behind) are multiplied by X here.  Rows and columns beyond nb are padded with the identity.
constexpr int DIAG_THREADS = 256;
constexpr int HB = 64;                      // half block
constexpr int TB = 32;                      // tile of the block algorithm
constexpr int DSD = NB + 4;                 // shared row of the 128-wide block (16-byte aligned)
constexpr int DSX = HB + 4;                 // shared row of a 64-wide quarter of the inverse
// The inverse is kept as its three nonzero 64 x 64 quarters X11, X21, X22 (X12 = 0), so that the
// kernel's ~119 KB of shared memory leaves room for an update-kernel CTA on the same SM.
constexpr int DIAG_SMEM = (NB * DSD + 3 * HB * DSX + 2 * NB) * (int)sizeof(float) + 16;

// Factor the 32 x 32 tile at A (row stride lda; lower triangle read) into L (written in place,
// zeros above the diagonal) and write X = L^-1 to X (row stride ldx, zeros above the diagonal).
// One warp: lane i holds row i of both.  Step m: the pivot is broadcast, lanes i >= m scale
// their entry of column m, lane m scales its row of X; column m of L and row m of X go to the
// scratch (scr: 128 floats, two buffers alternating by step), and every lane i > m subtracts
// L_im times them, reading the scratch four entries at a time.
// Returns false (uniformly over the warp) on a pivot that is not finite or not above dmin.
__device__ __noinline__ bool factor32(float* A, int lda, float* X, int ldx, float* scr, float dmin) {
    const int lane = threadIdx.x & 31;
    float a[TB], x[TB];
#pragma unroll
    for (int q = 0; q < TB / 4; ++q) {
        const float4 v = ld4(A + lane * lda + 4 * q);
        a[4 * q] = v.x;
        a[4 * q + 1] = v.y;
        a[4 * q + 2] = v.z;
        a[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < TB; ++j) {
        if (j > lane) a[j] = 0.f;
        x[j] = j == lane ? 1.f : 0.f;
    }
    bool ok = true;
#pragma unroll
    for (int m = 0; m < TB; ++m) {
        float* col = scr + (m & 1) * 2 * TB;
        float* xrow = col + TB;
        const float d = __shfl_sync(0xffffffffu, a[m], m);
        ok = ok && d > dmin && isfinite(d);
        // a few ulps suffice here: the factor is refined against the exact matrix later
        const float isd = rsqrtf(ok ? d : 1.f);
        const float l = lane >= m ? a[m] * isd : 0.f;
        a[m] = l;
        col[lane] = l;
        if (lane == m) {
#pragma unroll
            for (int j = 0; j <= m; ++j) x[j] *= isd;
#pragma unroll
            for (int q = 0; q <= m / 4; ++q)
                *reinterpret_cast<float4*>(xrow + 4 * q) = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        }
        __syncwarp();
        const float lu = lane > m ? l : 0.f;
#pragma unroll
        for (int q = (m + 1) / 4; q < TB / 4; ++q) {
            const float4 c = ld4(col + 4 * q);
            if (4 * q + 0 > m) a[4 * q + 0] = fmaf(-lu, c.x, a[4 * q + 0]);
            if (4 * q + 1 > m) a[4 * q + 1] = fmaf(-lu, c.y, a[4 * q + 1]);
            if (4 * q + 2 > m) a[4 * q + 2] = fmaf(-lu, c.z, a[4 * q + 2]);
            if (4 * q + 3 > m) a[4 * q + 3] = fmaf(-lu, c.w, a[4 * q + 3]);
        }
#pragma unroll
        for (int q = 0; q <= m / 4; ++q) {
            const float4 r = ld4(xrow + 4 * q);
            if (4 * q + 0 <= m) x[4 * q + 0] = fmaf(-lu, r.x, x[4 * q + 0]);
            if (4 * q + 1 <= m) x[4 * q + 1] = fmaf(-lu, r.y, x[4 * q + 1]);
            if (4 * q + 2 <= m) x[4 * q + 2] = fmaf(-lu, r.z, x[4 * q + 2]);
            if (4 * q + 3 <= m) x[4 * q + 3] = fmaf(-lu, r.w, x[4 * q + 3]);
        }
    }
#pragma unroll
    for (int q = 0; q < TB / 4; ++q) {
        float4 v, w;
        v.x = 4 * q + 0 <= lane ? a[4 * q + 0] : 0.f;
        v.y = 4 * q + 1 <= lane ? a[4 * q + 1] : 0.f;
        v.z = 4 * q + 2 <= lane ? a[4 * q + 2] : 0.f;
        v.w = 4 * q + 3 <= lane ? a[4 * q + 3] : 0.f;
        w.x = x[4 * q];
        w.y = x[4 * q + 1];
        w.z = x[4 * q + 2];
        w.w = x[4 * q + 3];
        *reinterpret_cast<float4*>(A + lane * lda + 4 * q) = v;
        *reinterpret_cast<float4*>(X + lane * ldx + 4 * q) = w;
    }
    __syncwarp();
    return ok;
}

// 32 x 32 x 32 tile products of one warp on shared-memory operands (row strides lda, ldb
// multiples of 4 and = 4 mod 32: conflict-free float4 rows).  Lane (g, c) = (lane / 4, lane % 4)
// owns rows g + 8 a (a < 4).
// NT: acc[a][b] = sum_m A[g + 8a][m] B[c + 4b][m]   (columns c + 4 b)
__device__ __forceinline__ void tile_nt(const float* A, int lda, const float* B, int ldb, float (&acc)[4][8]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 2
    for (int m = 0; m < TB; m += 4) {
        float4 av[4], bv[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = ld4(A + (g + 8 * a) * lda + m);
#pragma unroll
        for (int b = 0; b < 8; ++b) bv[b] = ld4(B + (c + 4 * b) * ldb + m);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = dot4(av[a], bv[b], acc[a][b]);
    }
}
// NN: acc[a][b] = sum_m A[g + 8a][m] B[m][8c + b]   (columns 8 c + b)
__device__ __forceinline__ void tile_nn(const float* A, int lda, const float* B, int ldb, float (&acc)[4][8]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
#pragma unroll 2
    for (int m = 0; m < TB; m += 4) {
        float4 av[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = ld4(A + (g + 8 * a) * lda + m);
#pragma unroll
        for (int mm = 0; mm < 4; ++mm) {
            const float4 b0 = ld4(B + (m + mm) * ldb + 8 * c), b1 = ld4(B + (m + mm) * ldb + 8 * c + 4);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float s = mm == 0 ? av[a].x : mm == 1 ? av[a].y : mm == 2 ? av[a].z : av[a].w;
                acc[a][0] = fmaf(s, b0.x, acc[a][0]);
                acc[a][1] = fmaf(s, b0.y, acc[a][1]);
                acc[a][2] = fmaf(s, b0.z, acc[a][2]);
                acc[a][3] = fmaf(s, b0.w, acc[a][3]);
                acc[a][4] = fmaf(s, b1.x, acc[a][4]);
                acc[a][5] = fmaf(s, b1.y, acc[a][5]);
                acc[a][6] = fmaf(s, b1.z, acc[a][6]);
                acc[a][7] = fmaf(s, b1.w, acc[a][7]);
            }
        }
    }
}
// C = sgn * acc (set) or C -= acc (sub), in the column layout of tile_nt (nt) or tile_nn.
template <bool NT>
__device__ __forceinline__ void tile_store(float* C, int ldc, const float (&acc)[4][8], bool sub) {
    const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            float& dst = C[(g + 8 * a) * ldc + (NT ? c + 4 * b : 8 * c + b)];
            dst = sub ? dst - acc[a][b] : acc[a][b];
        }
}

struct DiagTiles {
    float* A;
    float* X11;
    float* X21;
    float* X22;
    // tile (i, j) of the block (i >= j) and of the inverse / identity remainder W
    __device__ float* a(int i, int j) const { return A + i * TB * DSD + j * TB; }
    __device__ float* x(int i, int j) const {
        if (i < 2) return X11 + i * TB * DSX + j * TB;
        return (j < 2 ? X21 + j * TB : X22 + (j - 2) * TB) + (i - 2) * TB * DSX;
    }
};

// Phase "panel" of step k: job q < 3 - k is L_ik = A_ik X_kk^T with i = k + 1 + q; the others
// X_kj = X_kk W_kj with j = q - (3 - k).  In place: each job owns its output tile.
__device__ void diag_panel_job(const DiagTiles& T, int k, int q) {
    float acc[4][8];
    if (q < 3 - k) {
        float* Aik = T.a(k + 1 + q, k);
        tile_nt(Aik, DSD, T.x(k, k), DSX, acc);
        __syncwarp();
        tile_store<true>(Aik, DSD, acc, false);
    } else {
        float* Wkj = T.x(k, q - (3 - k));
        tile_nn(T.x(k, k), DSX, Wkj, DSX, acc);
        __syncwarp();
        tile_store<false>(Wkj, DSX, acc, false);
    }
    __syncwarp();
}
// Phase "update" of step k: the (3-k)(4-k)/2 tiles A_ij -= L_ik L_jk^T (k < j <= i) and the
// (3-k)(k+1) tiles W_ij -= L_ik X_kj (i > k, j <= k), numbered A tiles first, row by row.
__device__ int diag_update_jobs(int k) { return (3 - k) * (4 - k) / 2 + (3 - k) * (k + 1); }
__device__ void diag_update_job(const DiagTiles& T, int k, int q) {
    float acc[4][8];
    const int nA = (3 - k) * (4 - k) / 2;
    if (q < nA) {
        int i = k + 1, r = q;
        while (r > i - k - 1) { r -= i - k; ++i; }
        const int j = k + 1 + r;
        tile_nt(T.a(i, k), DSD, T.a(j, k), DSD, acc);
        tile_store<true>(T.a(i, j), DSD, acc, true);
    } else {
        const int r = q - nA, i = k + 1 + r / (k + 1), j = r % (k + 1);
        tile_nn(T.a(i, k), DSD, T.x(k, j), DSX, acc);
        tile_store<false>(T.x(i, j), DSX, acc, true);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(DIAG_THREADS) chol_diag_kernel(int t0, int P, int LD, int ns, int jb, float eps,
                                                                    const float* __restrict__ inv_s,
                                                                    const float* __restrict__ G,
                                                                    const double* __restrict__ obar,
                                                                    const double2* __restrict__ D,
                                                                    const float* __restrict__ Pn, float* __restrict__ Lf,
                                                                    piece_t* __restrict__ Lb,
                                                                    float* __restrict__ Dinv,
                                                                    piece_t* __restrict__ Db,
                                                                    float* __restrict__ yv, int* __restrict__ fail) {
    const int t = t0 + blockIdx.x;
    if (fail[t]) return;
    extern __shared__ __align__(16) float dsm[];
    float* A = dsm;                 // [NB][DSD] the block, becoming L (lower)
    float* X11 = A + NB * DSD;      // [HB][DSX] quarters of the inverse (lower)
    float* X21 = X11 + HB * DSX;    // [HB][DSX]
    float* X22 = X21 + HB * DSX;    // [HB][DSX]
    float* rhs = X22 + HB * DSX;    // [2][NB]
    __shared__ int pivots_ok;
    __shared__ __align__(16) float fscr[4 * TB];  // factor32's broadcast buffers
    const DiagTiles T{A, X11, X21, X22};
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nb = min(NB, P - jb);
    float* yt = yv + (size_t)t * 2 * P;
    const double2* Dt = D + (size_t)t * P;
    const float sc = inv_s[t];
    // Every pivot of the Cholesky factor of (S + eps I) / s is at least eps / s (a pivot is a
    // diagonal entry of a Schur complement, bounded below by the smallest eigenvalue).  A pivot
    // below half of that means that rounding in this precision has overtaken the shift: the
    // trajectory goes to the fallback solver, which raises the shift.
    const float dmin = 0.5f * eps * sc;
    if (tid < 2 * NB) {
        const int h = tid >> 7, i = tid & (NB - 1);
        float v = 0.f;
        if (i < nb) v = jb == 0 ? (float)(h ? Dt[i].y : Dt[i].x) * sc : yt[h * P + jb + i];
        rhs[h * NB + i] = v;
    }
    if (jb == 0)
        for (int k = NB + tid; k < P; k += blockDim.x) {
            const double2 d = Dt[k];
            yt[k] = (float)d.x * sc;
            yt[P + k] = (float)d.y * sc;
        }
    // the lower block (with the diagonal), identity padding beyond nb; lanes along rows i.
    // Loads are issued in batches of 32 per thread before any of them is used.
    {
        const float* Gt = G + (size_t)t * P * P;
        const float inv_ns = 1.0f / (float)ns;
        float* obs = X11;  // the block's column means (first block column only), X not yet in use
        if (jb == 0 && tid < NB) obs[tid] = tid < nb ? (float)obar[(size_t)t * P + tid] : 0.f;
        __syncthreads();
#pragma unroll 1
        for (int base = 0; base < NB * NB; base += 32 * DIAG_THREADS) {
            float v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int e = base + tid + DIAG_THREADS * q, c = e >> 7, i = e & (NB - 1);
                float x = 0.f;
                if (i < nb && c < nb && c <= i)
                    x = jb == 0 ? Gt[(size_t)c * P + i] : Pn[((size_t)t * NB + c) * P + jb + i];
                v[q] = x;
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int e = base + tid + DIAG_THREADS * q, c = e >> 7, i = e & (NB - 1);
                float x = i == c ? 1.f : 0.f;
                if (i < nb && c < nb && c <= i) {
                    x = v[q];
                    if (jb == 0) {
                        x = x * inv_ns - obs[i] * obs[c];
                        if (i == c) x += eps;
                        x *= sc;
                    }
                }
                A[i * DSD + c] = x;
            }
        }
    }
    __syncthreads();
    // W: zero below the diagonal tiles (the diagonal tiles are written by factor32)
    if (warp == 0) {
        const bool ok = factor32(T.a(0, 0), DSD, T.x(0, 0), DSX, fscr, dmin);
        if (tid == 0) pivots_ok = ok;
    } else {
        for (int e = tid - 32; e < 6 * TB * TB / 4; e += DIAG_THREADS - 32) {
            const int q = e / (TB * TB / 4), r = (e >> 3) & (TB - 1), c4 = e & 7;
            const int i = q == 0 ? 1 : q < 3 ? 2 : 3;
            const int j = q == 0 ? 0 : q == 1 ? 0 : q == 2 ? 1 : q == 3 ? 0 : q == 4 ? 1 : 2;
            *reinterpret_cast<float4*>(T.x(i, j) + r * DSX + 4 * c4) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        if (!pivots_ok) {  // uniform: read after a barrier
            if (tid == 0) fail[t] = 1;
            return;
        }
        if (warp < 3) diag_panel_job(T, k, warp);
        __syncthreads();
        if (k == 3) break;
        // warp 0: the next diagonal tile's update (job 0), then its factor; the others the rest
        const int nj = diag_update_jobs(k);
        if (warp == 0) {
            diag_update_job(T, k, 0);
            const bool ok = factor32(T.a(k + 1, k + 1), DSD, T.x(k + 1, k + 1), DSX, fscr, dmin);
            if (tid == 0) pivots_ok = ok;
        } else {
            for (int q = warp; q < nj; q += DIAG_THREADS / 32 - 1) diag_update_job(T, k, q);
        }
        __syncthreads();
    }
    // outputs: L (FP32 and FP16 pieces), X (padded rows / columns zero), y_b = X rhs
    const LbLayout lay{(P + NB - 1) / NB, LD / 32};
    float* Lft = Lf + (size_t)t * P * LD;
    piece_t* Lbt = Lb + (size_t)t * NPC * lay.plane();
    for (int e = tid; e < NB * (NB / 8); e += blockDim.x) {
        const int i = e >> 4, c8 = e & 15;
        if (i >= nb || c8 * 8 > i) continue;
        const int nv = nb - c8 * 8;
        const float4 q0 = ld4(A + i * DSD + c8 * 8), q1 = ld4(A + i * DSD + c8 * 8 + 4);
        float v[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (c8 * 8 + u > i) v[u] = 0.f;
        store_L8(Lft, Lbt, lay, LD, jb + i, jb + c8 * 8, v, nv);
    }
    // L_dd^-1 in FP32 and as two FP16 pieces in the operand-box layout of the panel kernel.  The
    // pieces must fit FP16 (|x| < 65504): a larger inverse (a near-singular block) sends the
    // trajectory to the fallback solver, as a failed pivot does.
    float* Dv = Dinv + ((size_t)t * ((P + NB - 1) / NB) + jb / NB) * NB * NB;
    const LbLayout layD{1, NB / BK};
    const size_t pl = layD.plane();
    piece_t* Dbt = Db + (size_t)t * NPC * pl;
    int big = 0;
    for (int e = tid; e < NB * (NB / 8); e += blockDim.x) {
        const int i = e >> 4, c8 = e & 15;
        // the eight entries from the quarter that holds them (X12 = 0)
        const float* src = i < HB ? (c8 < HB / 8 ? X11 + i * DSX + 8 * c8 : nullptr)
                                  : (c8 < HB / 8 ? X21 + (i - HB) * DSX + 8 * c8 : X22 + (i - HB) * DSX + 8 * c8 - HB);
        float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
        if (src) {
            q0 = ld4(src);
            q1 = ld4(src + 4);
        }
        float v[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int c = 8 * c8 + u;
            if (!(i < nb && c < nb && c <= i)) v[u] = 0.f;
            big |= !(fabsf(v[u]) < 16384.f);
        }
        *reinterpret_cast<float4*>(Dv + (size_t)i * NB + 8 * c8) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(Dv + (size_t)i * NB + 8 * c8 + 4) = make_float4(v[4], v[5], v[6], v[7]);
        store_P8(Dbt, pl, layD.at(i, 8 * c8), v);
    }
    if (__syncthreads_or(big)) {
        if (tid == 0) fail[t] = 1;
        return;
    }
    if (tid < 2 * NB) {
        const int h = tid >> 7, i = tid & (NB - 1);
        const float* rh = rhs + h * NB;
        float s = 0.f;
        if (i < HB) {
            for (int k = 0; k <= i; ++k) s = fmaf(X11[i * DSX + k], rh[k], s);
        } else {
            const float* x21 = X21 + (i - HB) * DSX;
            const float* x22 = X22 + (i - HB) * DSX;
#pragma unroll 8
            for (int k = 0; k < HB; ++k) s = fmaf(x21[k], rh[k], s);
            for (int k = HB; k <= i; ++k) s = fmaf(x22[k - HB], rh[k], s);
        }
        if (i < nb) yt[h * P + jb + i] = s;
    }
}

// ---------------------------------------------------------------------------------- panel
// Rows below the diagonal block, X = C L_dd^-T, on the tensor cores: one CTA = 128 rows of one
// trajectory, A = the rows of C (two FP16 pieces written by the update kernel, or for the
// first block column by chol_cb0_kernel from the Gram counts), B = L_dd^-1 (two pieces
// written by the diagonal kernel), the three piece products of the update kernel over K = 128
// (four 32-column slices), FP32 accumulators in TMEM.  The epilogue (one row per thread)
// writes L (FP32 + pieces) and subtracts the row's component along the block from the
// forward-substitution vector, y_i -= X[i, :] . y_b.

// C of the first block column for the rows below it: (S + eps I)_ic = G[c][i]/ns - obar_i obar_c
// (i >= 128 > c), as FP16 pieces.  Thread: row r = tid % 128 of the tile, column groups
// tid / 128 + 2 g (g < 8) of eight columns; rows beyond P are written as zeros.
__global__ void __launch_bounds__(256) chol_cb0_kernel(int t0, int P, int ns, const float* __restrict__ inv_s,
                                                       const float* __restrict__ G,
                                                       const double* __restrict__ obar, piece_t* __restrict__ Cb,
                                                       size_t planeC, const int* __restrict__ fail) {
    const int t = t0 + blockIdx.y;
    if (fail[t]) return;
    const int r = threadIdx.x & (NB - 1), i = NB * (1 + blockIdx.x) + r;
    const float* Gt = G + (size_t)t * P * P;
    const double* ob = obar + (size_t)t * P;
    const LbLayout layC{(P + NB - 1) / NB, NB / BK};
    piece_t* Cbt = Cb + (size_t)t * NPC * planeC;
    const float inv_ns = 1.0f / (float)ns, sc = inv_s[t];
    const float obi = i < P ? (float)ob[i] : 0.f;
#pragma unroll 1
    for (int g = 0; g < 8; ++g) {
        const int c0 = 8 * ((threadIdx.x >> 7) + 2 * g);
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = i < P ? Gt[(size_t)(c0 + u) * P + i] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = i < P ? (v[u] * inv_ns - obi * (float)ob[c0 + u]) * sc : 0.f;
        store_P8(Cbt, planeC, layC.at(i, c0), v);
    }
}

__global__ void __launch_bounds__(192, 2) chol_panel_kernel(const piece_t* __restrict__ Cb, size_t planeC,
                                                            const piece_t* __restrict__ Db, int t0, int P,
                                                            int LD, int jb, float* __restrict__ Lf,
                                                            piece_t* __restrict__ Lb, float* __restrict__ yv,
                                                            const int* __restrict__ fail, int* status) {
    using namespace tc;
    const int t = t0 + blockIdx.y;
    if (fail[t]) return;
    extern __shared__ uint8_t smem_raw[];
    __shared__ float yb_s[2][NB];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int i0 = jb + NB * (1 + blockIdx.x);
    constexpr int nk = NB / BK;
    const size_t planeD = (size_t)NB * NB;

    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
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
                const int st = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (kb >= STAGES && !mbar_wait(&empty[st], ph ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                uint8_t* sb = smem + st * STAGE;
                mbar_expect_tx(&full[st], STAGE);
                for (int p = 0; p < NPC; ++p) {
                    const piece_t* pa = Cb + (size_t)(t * NPC + p) * planeC;
                    const piece_t* pb = Db + (size_t)(t * NPC + p) * planeD;
                    bulk_load(sb + p * BOX, pa + ((size_t)(i0 >> 7) * nk + kb) * (BOX / 2), BOX, &full[st]);
                    bulk_load(sb + (NPC + p) * BOX, pb + (size_t)kb * (BOX / 2), BOX, &full[st]);
                }
                ++issued;
            }
            for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
                mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const int pa[NPROD] = {0, 0, 1};
            const int pb[NPROD] = {0, 1, 0};
            constexpr uint32_t ID = idesc_f16(128, NB);
            for (int kb = 0; kb < nk; ++kb) {
                const int st = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait(&full[st], ph, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t sa = su32(smem + st * STAGE);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
#pragma unroll
                    for (int q = 0; q < NPROD; ++q)
                        umma(tmem, smem_desc_sw64(sa + pa[q] * BOX + k * 32),
                             smem_desc_sw64(sa + (NPC + pb[q]) * BOX + k * 32), ID, (kb > 0 || k > 0 || q > 0) ? 1u : 0u);
                umma_commit(&empty[st]);
            }
            umma_commit(done);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;
        float* yt = yv + (size_t)t * 2 * P;
        for (int c = threadIdx.x - 64; c < NB; c += 128) {
            yb_s[0][c] = yt[jb + c];
            yb_s[1][c] = yt[P + jb + c];
        }
        int ok = 0;
        if (lane == 0) {
            ok = mbar_wait(done, 0, abort_flag) && !*abort_flag;
            if (!ok) *abort_flag = 1;  // a wait that ran out here is reported as well
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        fence_after();
        asm volatile("bar.sync 1, 128;" ::: "memory");  // yb_s written by the four epilogue warps
        if (ok) {
            const int i = i0 + q * 32 + lane;
            const LbLayout lay{(P + NB - 1) / NB, LD / 32};
            float* Lft = Lf + (size_t)t * P * LD;
            piece_t* Lbt = Lb + (size_t)t * NPC * lay.plane();
            float s0 = 0.f, s1 = 0.f;
#pragma unroll 1
            for (int c0 = 0; c0 < NB; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
                if (i >= P) continue;
#pragma unroll
                for (int u8 = 0; u8 < 4; ++u8) {
                    float x8[8];
#pragma unroll
                    for (int w = 0; w < 8; ++w) {
                        x8[w] = __uint_as_float(v[8 * u8 + w]);
                        s0 = fmaf(x8[w], yb_s[0][c0 + 8 * u8 + w], s0);
                        s1 = fmaf(x8[w], yb_s[1][c0 + 8 * u8 + w], s1);
                    }
                    store_L8(Lft, Lbt, lay, LD, i, jb + c0 + 8 * u8, x8, 8);
                }
            }
            if (i < P) {
                yt[i] -= s0;
                yt[P + i] -= s1;
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

// ------------------------------------------------------------------------------ solves
// Double-float pair (s + c carries about 48 bits) and its error-free accumulation.
struct DF {
    float s, c;
};
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float t = a.s + b.s;
    const float bp = t - a.s;
    const float e = (a.s - (t - bp)) + (b.s - bp);
    return DF{t, a.c + b.c + e};
}
// acc += g * (xh + xl), with the product g xh split exactly (FMA) and the sum by two-sum
__device__ __forceinline__ void df_fma(DF& acc, float g, float xh, float xl) {
    const float p = g * xh;
    const float e = fmaf(g, xh, -p);
    const float t = acc.s + p;
    const float bp = t - acc.s;
    const float err = (acc.s - (t - bp)) + (p - bp);
    acc.s = t;
    acc.c = fmaf(g, xl, acc.c + (err + e));
}
__device__ __forceinline__ DF shfl_df(DF v, int off) {
    return DF{__shfl_xor_sync(0xffffffffu, v.s, off), __shfl_xor_sync(0xffffffffu, v.c, off)};
}
// reduce8 for double-float pairs (same lane-to-value map)
__device__ __forceinline__ DF reduce8_df(DF (&v)[8], int lane) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const bool up = lane & 16;
        const DF send = up ? v[u] : v[u + 4];
        const DF keep = up ? v[u + 4] : v[u];
        v[u] = df_add(keep, shfl_df(send, 16));
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const bool up = lane & 8;
        const DF send = up ? v[u] : v[u + 2];
        const DF keep = up ? v[u + 2] : v[u];
        v[u] = df_add(keep, shfl_df(send, 8));
    }
    {
        const bool up = lane & 4;
        const DF send = up ? v[0] : v[1];
        const DF keep = up ? v[1] : v[0];
        v[0] = df_add(keep, shfl_df(send, 4));
    }
    v[0] = df_add(v[0], shfl_df(v[0], 2));
    v[0] = df_add(v[0], shfl_df(v[0], 1));
    return v[0];
}

// Refinement residual, tile-parallel: the products G x of the symmetric Gram counts with
// the current solution, one 128 x 128 upper tile (I <= J) of one trajectory per CTA.  The
// tile's row sums belong to row block I and its column sums (strictly below the diagonal
// for I = J) to row block J; each is written to its own slot part[t][row block][other
// block][128][2] (FP64), and the solve kernel adds the slots in a fixed order, so the
// result does not depend on scheduling.  Products and sums in double-float arithmetic.
__global__ void __launch_bounds__(256) chol_resid_kernel(int t0, int P, const float* __restrict__ G,
                                                         const double* __restrict__ xw, double* __restrict__ part,
                                                         const int* __restrict__ fail) {
    const int t = t0 + blockIdx.y;
    if (fail[t]) return;
    const int nblk = (P + NB - 1) / NB;
    int J = (int)((sqrtf(8.f * (float)blockIdx.x + 1.f) - 1.f) * 0.5f);
    while ((J + 1) * (J + 2) / 2 <= (int)blockIdx.x) ++J;
    while (J * (J + 1) / 2 > (int)blockIdx.x) --J;
    const int I = blockIdx.x - J * (J + 1) / 2;
    __shared__ float2 xI[2][NB], xJ[2][NB];
    __shared__ DF cred[8][NB][2];
    __shared__ double rowacc[2][NB];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const double* xt = xw + (size_t)t * 2 * P;
    {
        const int c = tid & (NB - 1), h = tid >> 7;
        const int iI = I * NB + c, iJ = J * NB + c;
        const double vI = iI < P ? xt[h * P + iI] : 0.0, vJ = iJ < P ? xt[h * P + iJ] : 0.0;
        const float hI = (float)vI, hJ = (float)vJ;
        xI[h][c] = make_float2(hI, (float)(vI - (double)hI));
        xJ[h][c] = make_float2(hJ, (float)(vJ - (double)hJ));
    }
    __syncthreads();
    const float* Gt = G + (size_t)t * P * P;
    const int j0 = J * NB + 4 * lane;
    const bool vec = (P & 3) == 0 && j0 + 3 < P;
    float2 xj[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        xj[u][0] = xJ[0][4 * lane + u];
        xj[u][1] = xJ[1][4 * lane + u];
    }
    DF cs[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u) cs[u][0] = cs[u][1] = DF{0.f, 0.f};
    // the four rows of group g (rows warp*16 + 4g .. +3 of the tile, columns j0 .. j0+3)
    auto load_group = [&](int g, float (&dst)[4][4]) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = I * NB + warp * 16 + 4 * g + a;
            const float* row = Gt + (size_t)i * P;
            if (i < P && vec) {
                const float4 q = ld4(row + j0);
                dst[a][0] = q.x; dst[a][1] = q.y; dst[a][2] = q.z; dst[a][3] = q.w;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) dst[a][u] = (i < P && j0 + u < P) ? row[j0 + u] : 0.f;
            }
        }
    };
    // loads of group g + 1 are issued before the arithmetic of group g
    float gv[4][4], gn[4][4];
    load_group(0, gv);
#pragma unroll 1
    for (int g = 0; g < 4; ++g) {
        if (g + 1 < 4) load_group(g + 1, gn);
        DF rs[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int r = warp * 16 + 4 * g + a;
            rs[2 * a] = rs[2 * a + 1] = DF{0.f, 0.f};
            const float2 xi0 = xI[0][r], xi1 = xI[1][r];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = 4 * lane + u;
                const float g_row = (I < J || c >= r) ? gv[a][u] : 0.f;
                const float g_col = (I < J || c > r) ? gv[a][u] : 0.f;
                df_fma(rs[2 * a], g_row, xj[u][0].x, xj[u][0].y);
                df_fma(rs[2 * a + 1], g_row, xj[u][1].x, xj[u][1].y);
                df_fma(cs[u][0], g_col, xi0.x, xi0.y);
                df_fma(cs[u][1], g_col, xi1.x, xi1.y);
            }
        }
        const DF s = reduce8_df(rs, lane);
        if ((lane & 3) == 0) {
            const int idx = reduce8_index(lane);
            rowacc[idx & 1][warp * 16 + 4 * g + (idx >> 1)] = (double)s.s + (double)s.c;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int u = 0; u < 4; ++u) gv[a][u] = gn[a][u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        cred[warp][4 * lane + u][0] = cs[u][0];
        cred[warp][4 * lane + u][1] = cs[u][1];
    }
    __syncthreads();
    {
        const int c = tid >> 1, h = tid & 1;
        DF s = cred[0][c][h];
#pragma unroll
        for (int w = 1; w < 8; ++w) s = df_add(s, cred[w][c][h]);
        const double col = (double)s.s + (double)s.c;
        double* pt = part + (size_t)t * nblk * nblk * (2 * NB);
        if (I < J) {
            pt[((size_t)I * nblk + J) * (2 * NB) + 2 * c + h] = rowacc[h][c];
            pt[((size_t)J * nblk + I) * (2 * NB) + 2 * c + h] = col;
        } else {
            pt[((size_t)I * nblk + I) * (2 * NB) + 2 * c + h] = rowacc[h][c] + col;
        }
    }
}

// Triangular solves L L^T x = y for the two right-hand sides (real and imaginary parts) of
// one trajectory, held in shared memory as y[0..PY) and y[PY..2 PY); one CTA of SW_WARPS
// warps per trajectory.  Forward, block b (left-looking): the 128 rows of the block take
// their dot products with y[0 : jb) (lanes along the row, four rows per warp and four
// column steps in flight), then y_b = L_bb^-1 (.) from the stored inverse.  Backward,
// block b from the last: column sums of the rows below (lanes along the block's columns,
// warps along the rows, eight rows per warp in flight), then x_b = L_bb^-T (.).
constexpr int SW_WARPS = 16;
constexpr int SWEEP_THREADS = 32 * SW_WARPS;
constexpr int SW_ROWS = NB / SW_WARPS;   // rows of a block per warp

__device__ void sweep_forward(int P, int PY, int LD, const float* Lt, const float* Dv, float* y, float* tb) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nblk = (P + NB - 1) / NB;
    for (int b = 0; b < nblk; ++b) {
        const int jb = b * NB, nb = min(NB, P - jb);
#pragma unroll 1
        for (int g = 0; g < SW_ROWS / 4; ++g) {
            const int rl = warp * SW_ROWS + 4 * g;
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = 0.f;
#pragma unroll 4
            for (int q = 0; q < b; ++q) {
                const int c = q * NB + 4 * lane;
                const float4 y0 = ld4(y + c), y1 = ld4(y + PY + c);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = jb + rl + a;
                    const float4 l = i < P ? ld4(Lt + (size_t)i * LD + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                    v[2 * a] = dot4(l, y0, v[2 * a]);
                    v[2 * a + 1] = dot4(l, y1, v[2 * a + 1]);
                }
            }
            const float s = reduce8(v, lane);
            if ((lane & 3) == 0) {
                const int idx = reduce8_index(lane), h = idx & 1, r = rl + (idx >> 1);
                tb[h * NB + r] = r < nb ? y[h * PY + jb + r] - s : 0.f;
            }
        }
        __syncthreads();
        const float* Db = Dv + (size_t)b * NB * NB;
        const float4 t0 = ld4(tb + 4 * lane), t1 = ld4(tb + NB + 4 * lane);
#pragma unroll
        for (int g = 0; g < SW_ROWS / 4; ++g) {
            const int rl = warp * SW_ROWS + 4 * g;
            float v[8];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float4 l = ld4(Db + (size_t)(rl + a) * NB + 4 * lane);
                v[2 * a] = dot4(l, t0, 0.f);
                v[2 * a + 1] = dot4(l, t1, 0.f);
            }
            const float s = reduce8(v, lane);
            if ((lane & 3) == 0) {
                const int idx = reduce8_index(lane), h = idx & 1, r = rl + (idx >> 1);
                if (r < nb) y[h * PY + jb + r] = s;
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void acc_col4(float (&acc)[4][2], float4 l, float x0, float x1) {
    acc[0][0] = fmaf(l.x, x0, acc[0][0]);
    acc[1][0] = fmaf(l.y, x0, acc[1][0]);
    acc[2][0] = fmaf(l.z, x0, acc[2][0]);
    acc[3][0] = fmaf(l.w, x0, acc[3][0]);
    acc[0][1] = fmaf(l.x, x1, acc[0][1]);
    acc[1][1] = fmaf(l.y, x1, acc[1][1]);
    acc[2][1] = fmaf(l.z, x1, acc[2][1]);
    acc[3][1] = fmaf(l.w, x1, acc[3][1]);
}

// Sum of the warps' partial column sums (fixed order); red is [SW_WARPS][NB][2].
__device__ __forceinline__ void put_col4(float* red, int warp, int lane, const float (&acc)[4][2]) {
    reinterpret_cast<float4*>(red + (warp * NB + 4 * lane) * 2)[0] =
        make_float4(acc[0][0], acc[0][1], acc[1][0], acc[1][1]);
    reinterpret_cast<float4*>(red + (warp * NB + 4 * lane) * 2)[1] =
        make_float4(acc[2][0], acc[2][1], acc[3][0], acc[3][1]);
}

__device__ void sweep_backward(int P, int PY, int LD, const float* Lt, const float* Dv, float* y, float* tb,
                               float* red) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nblk = (P + NB - 1) / NB;
    for (int b = nblk - 1; b >= 0; --b) {
        const int jb = b * NB, nb = min(NB, P - jb);
        float acc[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = 0.f;
        int i = jb + NB + warp;
        // sixteen rows per warp in flight (the pass is bound by the loads' latency)
        for (; i + 15 * SW_WARPS < P; i += 16 * SW_WARPS) {
            float4 l[16];
#pragma unroll
            for (int a = 0; a < 16; ++a) l[a] = ld4(Lt + (size_t)(i + a * SW_WARPS) * LD + jb + 4 * lane);
#pragma unroll
            for (int a = 0; a < 16; ++a) acc_col4(acc, l[a], y[i + a * SW_WARPS], y[PY + i + a * SW_WARPS]);
        }
        for (; i < P; i += SW_WARPS) acc_col4(acc, ld4(Lt + (size_t)i * LD + jb + 4 * lane), y[i], y[PY + i]);
        put_col4(red, warp, lane, acc);
        __syncthreads();
        if (tid < 2 * NB) {
            const int c = tid >> 1, h = tid & 1;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < SW_WARPS; ++w) s += red[(w * NB + c) * 2 + h];
            tb[h * NB + c] = c < nb ? y[h * PY + jb + c] - s : 0.f;
        }
        __syncthreads();
        const float* Db = Dv + (size_t)b * NB * NB;
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u][0] = acc[u][1] = 0.f;
#pragma unroll
        for (int kk = 0; kk < NB / SW_WARPS; ++kk) {
            const int k = warp + kk * SW_WARPS;
            acc_col4(acc, ld4(Db + (size_t)k * NB + 4 * lane), tb[k], tb[NB + k]);
        }
        put_col4(red, warp, lane, acc);
        __syncthreads();
        if (tid < 2 * NB) {
            const int c = tid >> 1, h = tid & 1;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < SW_WARPS; ++w) s += red[(w * NB + c) * 2 + h];
            if (c < nb) y[h * PY + jb + c] = s;
        }
        __syncthreads();
    }
}

// Solve passes of one trajectory per CTA.
//   mode 0: x = L^-T y from the forward result y that the factorization left in yv;
//   mode 1: r = D - (S + eps I) x with S x = (G x) / ns - obar (obar . x), G x summed from the
//           residual kernel's slots in FP64; then dx = L^-T L^-1 r and x += dx.
//   mode 2: the right-hand side D is a residual formed by the caller; dx = L^-T L^-1 D is added
//           to delta (in place, FP64), with the factor left by an earlier call.
// The last pass writes delta (and the shift used), the others keep x in xw (FP64).
// true (for this thread's entries) if both right-hand sides of y are finite
__device__ __forceinline__ bool sweep_finite(int P, int PY, const float* y) {
    bool ok = true;
    for (int k = threadIdx.x; k < P; k += blockDim.x) ok = ok && isfinite(y[k]) && isfinite(y[PY + k]);
    return ok;
}

__global__ void __launch_bounds__(SWEEP_THREADS) chol_sweep_kernel(int t0, int P, int LD, int ns, double eps, int mode,
                                                                    int last, const double* __restrict__ obar,
                                                                    const double2* __restrict__ D,
                                                                    const float* __restrict__ Lf,
                                                                    const float* __restrict__ Dinv,
                                                                    const float* __restrict__ yv,
                                                                    const double* __restrict__ part,
                                                                    double* __restrict__ xw, double2* __restrict__ delta,
                                                                    double* __restrict__ shift_used,
                                                                    int* __restrict__ fail,
                                                                    const float* __restrict__ inv_s) {
    const int t = t0 + blockIdx.x;
    if (fail[t]) return;
    const int nblk = (P + NB - 1) / NB, PY = nblk * NB;
    const double sc = (double)inv_s[t];  // the factor is of (S + eps I) / s: right-hand sides / s
    extern __shared__ __align__(16) float wsm[];
    float* y = wsm;              // [2][PY]
    float* red = y + 2 * PY;              // [SW_WARPS][NB][2]
    float* tb = red + SW_WARPS * NB * 2;  // [2][NB]
    __shared__ double dred[2][SWEEP_THREADS / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float* Lt = Lf + (size_t)t * P * LD;
    const float* Dv = Dinv + (size_t)t * nblk * NB * NB;
    double* xt = xw + (size_t)t * 2 * P;
    const double2* Dt = D + (size_t)t * P;
    for (int k = P + tid; k < PY; k += blockDim.x) y[k] = y[PY + k] = 0.f;
    if (mode == 2) {
        for (int k = tid; k < P; k += blockDim.x) {
            y[k] = (float)(Dt[k].x * sc);
            y[PY + k] = (float)(Dt[k].y * sc);
        }
        __syncthreads();
        sweep_forward(P, PY, LD, Lt, Dv, y, tb);
        sweep_backward(P, PY, LD, Lt, Dv, y, tb, red);
        // a correction that is not finite (an FP32 factor of a system too ill-conditioned for
        // it) is not applied: x keeps its value
        if (__syncthreads_or(!sweep_finite(P, PY, y))) return;
        double2* dt = delta + (size_t)t * P;
        for (int k = tid; k < P; k += blockDim.x) {
            const double2 o = dt[k];
            dt[k] = make_double2(o.x + (double)y[k], o.y + (double)y[PY + k]);
        }
        return;
    }
    if (mode == 0) {
        const float* yt = yv + (size_t)t * 2 * P;
        for (int k = tid; k < P; k += blockDim.x) {
            y[k] = yt[k];
            y[PY + k] = yt[P + k];
        }
        __syncthreads();
    } else {
        const double* ob = obar + (size_t)t * P;
        double a0 = 0.0, a1 = 0.0;
        for (int k = tid; k < P; k += blockDim.x) {
            a0 += ob[k] * xt[k];
            a1 += ob[k] * xt[P + k];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, off);
            a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        }
        if (lane == 0) {
            dred[0][warp] = a0;
            dred[1][warp] = a1;
        }
        __syncthreads();
        double ox0 = 0.0, ox1 = 0.0;
        for (int w = 0; w < SWEEP_THREADS / 32; ++w) {
            ox0 += dred[0][w];
            ox1 += dred[1][w];
        }
        const double* pt = part + (size_t)t * nblk * nblk * (2 * NB);
        const double inv_ns = 1.0 / (double)ns;
        for (int k = tid; k < P; k += blockDim.x) {
            const double2* pp = reinterpret_cast<const double2*>(pt + (size_t)(k >> 7) * nblk * (2 * NB) + 2 * (k & 127));
            double s0 = 0.0, s1 = 0.0;
#pragma unroll 4
            for (int J = 0; J < nblk; ++J) {
                const double2 q = pp[(size_t)J * NB];
                s0 += q.x;
                s1 += q.y;
            }
            const double r0 = Dt[k].x - (s0 * inv_ns - ob[k] * ox0 + eps * xt[k]);
            const double r1 = Dt[k].y - (s1 * inv_ns - ob[k] * ox1 + eps * xt[P + k]);
            y[k] = (float)(r0 * sc);
            y[PY + k] = (float)(r1 * sc);
        }
        __syncthreads();
        sweep_forward(P, PY, LD, Lt, Dv, y, tb);
    }
    sweep_backward(P, PY, LD, Lt, Dv, y, tb, red);
    // a solution that is not finite (an FP32 factor of a system too ill-conditioned for it, with
    // no pivot below zero) sends the trajectory to the fallback solver, which runs after the sweeps
    if (__syncthreads_or(!sweep_finite(P, PY, y))) {
        if (tid == 0) fail[t] = 1;
        return;
    }
    for (int k = tid; k < P; k += blockDim.x) {
        double vr = (double)y[k], vi = (double)y[PY + k];
        if (mode == 1) {
            vr += xt[k];
            vi += xt[P + k];
        }
        if (last) {
            delta[(size_t)t * P + k] = make_double2(vr, vi);
        } else {
            xt[k] = vr;
            xt[P + k] = vi;
        }
    }
    if (last && tid == 0 && shift_used) shift_used[t] = eps;
}

// inv_s[t] = 2^-k with 2^(k-1) < max_i (S + eps I)_ii <= 2^k (1 if that maximum is not a positive
// finite number): the factored system is (S + eps I) / s, whose factor has entries at most 1.
__global__ void chol_scale_kernel(int P, int ns, double eps, const float* __restrict__ G,
                                  const double* __restrict__ obar, float* __restrict__ inv_s) {
    const int t = blockIdx.x, tid = threadIdx.x;
    __shared__ double red[256];
    const float* Gt = G + (size_t)t * P * P;
    const double* ob = obar + (size_t)t * P;
    double mx = 0.0;
    for (int i = tid; i < P; i += 256) mx = fmax(mx, (double)Gt[(size_t)i * P + i] / ns - ob[i] * ob[i] + eps);
    red[tid] = mx;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) red[tid] = fmax(red[tid], red[tid + h]);
        __syncthreads();
    }
    if (tid == 0) {
        float v = 1.f;
        if (red[0] > 0.0 && red[0] < 1e30) {
            int k;
            const double f = frexp(red[0], &k);  // red = f 2^k, f in [1/2, 1)
            v = (float)ldexp(1.0, f == 0.5 ? 1 - k : -k);
        }
        inv_s[t] = v;
    }
}

inline int ldim(int P) { return ((P + 63) / 64) * 64; }

constexpr int CHOL_GROUPS = 4;
// Trajectory groups of one call: groups of 64 once the call has 128 trajectories or more
// (each launch then fills the GPU by itself), else CHOL_GROUPS groups from 16 trajectories.
// A run's launch-shape setting (set around a run's launches on the issuing host thread) may fix
// the number of groups instead: 1 .. CHOL_GROUPS, at most one group per trajectory.
thread_local int t_chol_groups = 0;
inline int chol_groups(int ntraj) {
    if (t_chol_groups > 0) return t_chol_groups < ntraj ? t_chol_groups : ntraj;
    if (ntraj < 16) return 1;
    if (ntraj >= 128) return ntraj / 64 < CHOL_GROUPS ? ntraj / 64 : CHOL_GROUPS;
    return CHOL_GROUPS;
}
struct GroupStreams {
    cudaStream_t s[CHOL_GROUPS];
    cudaEvent_t fork;
    cudaEvent_t join[CHOL_GROUPS];
};
// Streams for the trajectory groups: one set per (device, calling stream), created on first
// use, so that solves issued from different streams (the run's pipelines) do not share them.
inline GroupStreams& group_streams(cudaStream_t caller) {
    static std::mutex mu;
    static std::map<std::pair<int, uintptr_t>, GroupStreams> sets;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dev, (uintptr_t)caller);
    auto it = sets.find(key);
    if (it != sets.end()) return it->second;
    GroupStreams& g = sets[key];
    for (int i = 0; i < CHOL_GROUPS; ++i) {
        cudaStreamCreateWithFlags(&g.s[i], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&g.join[i], cudaEventDisableTiming);
    }
    cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming);
    return g;
}

}  // namespace chol

cudaError_t chol_set_wait_limit(unsigned long long ns) { return tc::set_wait_limit_tu(ns); }

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
    add((size_t)ntraj * 4 * P * 8);          // x (and the fallback's residual)
    add((size_t)ntraj * 2 * P * 4);          // forward-substitution vector
    add((size_t)ntraj * nblk * nblk * 2 * NB * 8);  // residual slots
    add((size_t)ntraj * NPC * nblk * NB * NB * 2);  // C of the panel rows, FP16 pieces
    add((size_t)ntraj * NPC * NB * NB * 2);         // L_dd^-1, FP16 pieces
    add((size_t)ntraj * 4);                         // 1 / s per trajectory
    return b + 256;
}

// Fallback: the single-CTA solver of k_solve.cu restricted to the marked trajectories; its
// factor of trajectory t goes to L + t * lstride (here the trajectory's own region of Lf, so
// that the factors of the other trajectories, which later corrections reuse, stay intact).
cudaError_t launch_chol_solve_masked(int ntraj, int P, int ns, double eps, const float* G, const double* obar,
                                     const double2* D, double2* delta, double* shift_used, float* L, size_t lstride,
                                     float* y, double* x, int refine_iters, const int* only, int* status,
                                     cudaStream_t s);

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
    const int NT = (P + NB - 1) / NB;
    piece_t* Lb = (piece_t*)take((size_t)ntraj * NPC * NT * 128 * LD * 2);
    float* Lf = (float*)take((size_t)ntraj * P * LD * 4);
    float* Pn = (float*)take((size_t)ntraj * P * NB * 4);
    float* Dv = (float*)take((size_t)ntraj * nblk * NB * NB * 4);
    int* fail = (int*)take((size_t)ntraj * 4);
    float* yf = (float*)take((size_t)ntraj * 2 * P * 4);
    double* x = (double*)take((size_t)ntraj * 4 * P * 8);
    float* yv = (float*)take((size_t)ntraj * 2 * P * 4);
    double* part = (double*)take((size_t)ntraj * nblk * nblk * 2 * NB * 8);
    const size_t planeC = LbLayout{NT, NB / BK}.plane();
    piece_t* Cb = (piece_t*)take((size_t)ntraj * NPC * planeC * 2);
    piece_t* Db = (piece_t*)take((size_t)ntraj * NPC * NB * NB * 2);
    float* inv_s = (float*)take((size_t)ntraj * 4);

    const LbLayout lay{NT, LD / 32};
    const size_t plane = lay.plane();

    cudaError_t e = cudaMemsetAsync(fail, 0, (size_t)ntraj * 4, s);
    if (e != cudaSuccess) return chol_fail(e, "memset");
    {
        ProfScope pd(OTVMC_K_CHOLD, s);
        chol_scale_kernel<<<ntraj, 256, 0, s>>>(P, ns, eps, G, obar, inv_s);
        count_launch();
    }
    e = cudaFuncSetAttribute(chol_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, DIAG_SMEM);
    if (e != cudaSuccess) return chol_fail(e, "diag attribute");
    e = cudaFuncSetAttribute(chol_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_U);
    if (e != cudaSuccess) return chol_fail(e, "panel attribute");
    e = cudaFuncSetAttribute(chol_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_U);
    if (e != cudaSuccess) return chol_fail(e, "update attribute");
    const float feps = (float)eps;
    const int PY = (int)nblk * NB;
    const int wsmem = (2 * PY + SW_WARPS * NB * 2 + 2 * NB) * (int)sizeof(float);
    e = cudaFuncSetAttribute(chol_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem);
    if (e != cudaSuccess) return chol_fail(e, "sweep attribute");
    // trajectory groups on forked streams: one group's latency-bound kernels overlap the
    // others' (fork and join by events, so the call stays ordered on `s`)
    // (under serial profiling the groups keep their launches but run one after another on s)
    const int ng = chol_groups(ntraj);
    const bool forked = ng > 1 && !profiling_serial();
    GroupStreams& gs = group_streams(s);
    if (forked) {
        e = cudaEventRecord(gs.fork, s);
        if (e != cudaSuccess) return chol_fail(e, "fork record");
    }
    for (int g = 0; g < ng; ++g) {
        const int ta = (int)((long long)ntraj * g / ng), tb = (int)((long long)ntraj * (g + 1) / ng);
        const int nt = tb - ta;
        if (nt <= 0) continue;
        cudaStream_t gsm = forked ? gs.s[g] : s;
        if (forked && (e = cudaStreamWaitEvent(gsm, gs.fork, 0)) != cudaSuccess) return e;
        for (int jb = 0; jb < P; jb += NB) {
            if (jb > 0) {
                ProfScope pu(OTVMC_K_CHOLU, gsm);
                dim3 grid((P - jb + 127) / 128, nt);
                chol_update_kernel<<<grid, 192, SMEM_U, gsm>>>(Lb, plane, LD / 32, ta, P, ns, jb, feps, inv_s, G, obar, Pn,
                                                               Cb, planeC, fail, status);
                count_launch();
            }
            {
                ProfScope pd(OTVMC_K_CHOLD, gsm);
                chol_diag_kernel<<<nt, DIAG_THREADS, DIAG_SMEM, gsm>>>(ta, P, LD, ns, jb, feps, inv_s, G, obar, D, Pn, Lf, Lb, Dv,
                                                                       Db, yv, fail);
                count_launch();
            }
            const int nrows = P - jb - min(NB, P - jb);
            if (nrows > 0) {
                ProfScope pp(OTVMC_K_CHOLP, gsm);
                dim3 grid((nrows + NB - 1) / NB, nt);
                if (jb == 0) {
                    chol_cb0_kernel<<<grid, 256, 0, gsm>>>(ta, P, ns, inv_s, G, obar, Cb, planeC, fail);
                    count_launch();
                }
                chol_panel_kernel<<<grid, 192, SMEM_U, gsm>>>(Cb, planeC, Db, ta, P, LD, jb, Lf, Lb, yv, fail, status);
                count_launch();
            }
        }
        {
            ProfScope ps(OTVMC_K_SOLVE, gsm);
            chol_sweep_kernel<<<nt, SWEEP_THREADS, wsmem, gsm>>>(ta, P, LD, ns, eps, 0, refine_iters <= 0 ? 1 : 0, obar,
                                                                  D, Lf, Dv, yv, part, x, delta, shift_used, fail, inv_s);
            count_launch();
        }
        for (int it = 0; it < refine_iters; ++it) {
            {
                ProfScope pr(OTVMC_K_RESID, gsm);
                dim3 grid((unsigned)(nblk * (nblk + 1) / 2), nt);
                chol_resid_kernel<<<grid, 256, 0, gsm>>>(ta, P, G, x, part, fail);
                count_launch();
            }
            ProfScope ps(OTVMC_K_SOLVE, gsm);
            chol_sweep_kernel<<<nt, SWEEP_THREADS, wsmem, gsm>>>(ta, P, LD, ns, eps, 1, it == refine_iters - 1 ? 1 : 0,
                                                                  obar, D, Lf, Dv, yv, part, x, delta, shift_used, fail, inv_s);
            count_launch();
        }
        if (forked) {
            if ((e = cudaEventRecord(gs.join[g], gsm)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, gs.join[g], 0)) != cudaSuccess) return e;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return chol_fail(e, "kernel launch");
    // trajectories whose pivot failed: robust solver with shift retries (exits at once for the others)
    return launch_chol_solve_masked(ntraj, P, ns, eps, G, obar, D, delta, shift_used, Lf, (size_t)P * LD, yf, x,
                                    refine_iters, fail, status, s);
}

// One more correction with the factor that the last launch_chol_tc on this workspace left:
// x += (L L^T)^-1 r for every trajectory whose pivots did not fail (the others were solved by
// the fallback with a raised shift and keep x).  r, x: [ntraj][P] double2 (two right-hand sides).
int chol_set_groups(int groups) {
    const int old = chol::t_chol_groups;
    chol::t_chol_groups = groups < 0 ? 0 : (groups > chol::CHOL_GROUPS ? chol::CHOL_GROUPS : groups);
    return old;
}

cudaError_t launch_chol_tc_resolve(int ntraj, int P, void* ws, const double2* r, double2* x, cudaStream_t s) {
    using namespace chol;
    const int LD = ldim(P);
    const size_t nblk = (P + NB - 1) / NB;
    const int NT = (P + NB - 1) / NB;
    char* p = (char*)ws;
    auto take = [&](size_t bytes) {
        char* q = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)q;
    };
    take((size_t)ntraj * NPC * NT * 128 * LD * 2);
    float* Lf = (float*)take((size_t)ntraj * P * LD * 4);
    take((size_t)ntraj * P * NB * 4);
    float* Dv = (float*)take((size_t)ntraj * nblk * NB * NB * 4);
    int* fail = (int*)take((size_t)ntraj * 4);
    take((size_t)ntraj * 2 * P * 4);                       // fallback y
    take((size_t)ntraj * 4 * P * 8);                       // x
    take((size_t)ntraj * 2 * P * 4);                       // forward-substitution vector
    take((size_t)ntraj * nblk * nblk * 2 * NB * 8);        // residual slots
    take((size_t)ntraj * NPC * LbLayout{NT, NB / BK}.plane() * 2);  // C pieces
    take((size_t)ntraj * NPC * NB * NB * 2);               // L_dd^-1 pieces
    const float* inv_s = (const float*)take((size_t)ntraj * 4);
    const int PY = (int)nblk * NB;
    const int wsmem = (2 * PY + SW_WARPS * NB * 2 + 2 * NB) * (int)sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(chol_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, wsmem);
    if (e != cudaSuccess) return chol_fail(e, "sweep attribute");
    ProfScope ps(OTVMC_K_SOLVE, s);
    chol_sweep_kernel<<<ntraj, SWEEP_THREADS, wsmem, s>>>(0, P, LD, 0, 0.0, 2, 0, nullptr, r, Lf, Dv, nullptr, nullptr,
                                                           nullptr, x, nullptr, fail, inv_s);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
