// Local-estimator fields of the Jastrow ansatz on the tensor cores (mixed path, 32 <= N <= 128).
//
// The flip ratios r_j(x) = psi(x^j) / psi(x) = exp(-2 sigma_j f_j(x)) of the transverse-field
// term and the diagonal Ising energy (E_H of the effective Hamiltonian, Eq. 5; the ansatz of
// Eq. 12) need, for every sample x and site j, the fields
//     f_j(x) = a_j + sum_k eta_jk sigma_k(x)   (complex),   f^J_j(x) = sum_k J_jk sigma_k(x).
// Over a tile of samples that is a product of the +-1 matrix sigma (samples x sites) with the
// coupling rows: a dense contraction over k, done here by tcgen05.mma (kind::f16, FP16 in, FP32
// accumulate in TMEM) with sigma, exact in FP16, as the A operand.  The B operand holds, per
// site j of a block of 16, eight rows ("pieces"):
//   0, 1   Re eta_j. scaled by a power of two 2^e_j (largest entry in [2^13, 2^14)) as two
//          FP16 pieces h + m (22 significant bits of the FP32 value relative to that entry);
//   2, 3   J_j. likewise, with its own power of two;
//   4..7   Im eta_j. in fixed point, each entry reduced modulo pi (the ratio depends on Im f_j
//          only modulo pi, and sigma = +-1 keeps the reduction exact) and rounded from units
//          of 2^-48 to units of 2^-42 (below 2^43 in magnitude), then written as four balanced
//          base-2^11 digits in [-1024, 1023], exact in FP16.
// The digit sums over k (at most 128 x 1024 in magnitude) are exact in FP32, so Im f_j is
// rebuilt exactly from the rounded entries in 64-bit integers (an error of at most N 2^-43
// against the unrounded sum) and the phase is reduced modulo 2 pi in fixed point, as on the
// SIMT path.  The real fields carry FP32-level rounding.
//
// One CTA = 16 sites x 4 tiles of 128 samples of one trajectory, 128 threads (one per sample
// of a tile), 128 TMEM columns, so that four CTAs share an SM:
//   - the B image of the site block (8 x 16 rows of 64 k per 64-site block kb, pre-swizzled
//     by est_tc_prep_kernel) arrives by one bulk copy;
//   - per tile every thread writes its sample's row of the sigma tile into shared memory
//     (128-byte swizzle), one thread issues the MMAs (M = 128 samples, N = 128, K = 16 per
//     instruction) and commits to an mbarrier;
//   - epilogue: thread = sample (TMEM lane), in two passes of 8 sites: r_j to global memory
//     and the sample's E_H over the 16 sites; the ratios also go to shared memory, from which
//     the per-site sums over the tile's samples (r_j, sigma_j r_j, sigma_j) are taken by
//     eight threads per site and added in a fixed order.
// E_H leaves as one partial per site block, EHq[t][x][block], summed in order by est2; the
// per-site sums as one partial per CTA (part_r / part_sr / part_s with est_tc_chunks(ns)
// blocks), summed in order by the site-means kernel.  All sums are in a fixed order: the
// results do not depend on scheduling.
// Every mbarrier wait is bounded; on timeout the CTA records OTVMC_ERR_TIMEOUT, drains its
// bulk copy and MMAs (bounded), frees TMEM and returns.
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace otvmc {
namespace etc {

constexpr int SB = ETC_SITES;           // sites per CTA
constexpr int NPIECE = 8;
constexpr int NCOL = NPIECE * SB;       // 128 accumulator columns
constexpr int A_BYTES = 128 * 128;      // one 64-site block of the sigma tile: 128 rows of 128 bytes
constexpr int B_BYTES = NCOL * 128;     // one 64-site block of the B image: 128 rows of 128 bytes
constexpr int TILES = ETC_TILES;        // sample tiles of 128 per CTA
constexpr int IM_SHIFT = 6;             // Im entries in units of 2^-42 on the tensor cores
constexpr uint32_t TCOLS = 128;
constexpr long long FX_PI = FX_TWO_PI / 2;  // FX_TWO_PI is even: the reduction below is exact

// Im-field entries reduced modulo pi (in units of 2^-48) into [-pi/2, pi/2], then rounded to
// units of 2^-42.
__device__ __forceinline__ long long reduce_pi(long long q) {
    long long r = q % FX_PI;
    if (r > FX_PI / 2) r -= FX_PI;
    if (r < -FX_PI / 2) r += FX_PI;
    return (r + (1ll << (IM_SHIFT - 1))) >> IM_SHIFT;
}

// Byte offset of the 16-byte unit c (0..7) of row r in a 128-byte-swizzled operand block.
__host__ __device__ __forceinline__ int sw128(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }

// Power of two that brings the largest |x| of a row into [2^13, 2^14) (0 for an all-zero row).
__device__ __forceinline__ int row_exp(float mx) { return mx > 0.f ? 13 - ilogbf(mx) : 0; }

// Per-site constants of a site block: a_j terms (FP32 of the fixed-point sums), the inverse
// row scales 2^-e_j, and Im a_j reduced modulo pi in units of 2^-42.
struct SiteTabs {
    float* aRe;
    float* aJ;
    float* sRe;
    float* sJ;
    long long* aIm;
};

// B images and per-site constants of one trajectory and site block (grid: site blocks x T).
// img[t][sb][kb]: B_BYTES each.
__global__ void __launch_bounds__(256) est_tc_prep_kernel(int n, int KB, const long long* __restrict__ Qre,
                                                          const long long* __restrict__ Qim,
                                                          const long long* __restrict__ base_re,
                                                          const long long* __restrict__ base_im,
                                                          const long long* __restrict__ QJ,
                                                          const long long* __restrict__ baseJ, uint8_t* __restrict__ img,
                                                          SiteTabs tabs) {
    __shared__ int ex[2][SB];
    const int sb = blockIdx.x, t = blockIdx.y, nsb = gridDim.x;
    const long long* qr = Qre + (size_t)t * n * n;
    const long long* qi = Qim + (size_t)t * n * n;
    uint8_t* out = img + ((size_t)t * nsb + sb) * KB * B_BYTES;
    if (threadIdx.x < 2 * SB) {
        const int kind = threadIdx.x / SB, j = sb * SB + threadIdx.x % SB;
        float mx = 0.f;
        if (j < n)
            for (int k = 0; k < n; ++k) mx = fmaxf(mx, fabsf(fx_to_float(kind == 0 ? qr[j * n + k] : QJ[j * n + k])));
        ex[kind][threadIdx.x % SB] = row_exp(mx);
    }
    __syncthreads();
    const int units = KB * NCOL * 8;
    for (int q = threadIdx.x; q < units; q += blockDim.x) {
        const int kb = q / (NCOL * 8), rem = q - kb * NCOL * 8;
        const int r = rem >> 3, c = rem & 7;
        const int p = r / SB, j = sb * SB + (r % SB);
        uint16_t h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int k = 64 * kb + 8 * c + e;
            __half v = __float2half_rn(0.f);
            if (j < n && k < n && j != k) {
                if (p < 4) {
                    const float x = ldexpf(fx_to_float(p < 2 ? qr[j * n + k] : QJ[j * n + k]), ex[p >> 1][r % SB]);
                    const __half hi = __float2half_rn(x);
                    v = (p & 1) ? __float2half_rn(x - __half2float(hi)) : hi;
                } else {
                    long long z = reduce_pi(qi[j * n + k]);
                    int d = 0;
                    for (int i = 0; i <= p - 4; ++i) {
                        d = (int)((z & 0x7FF) ^ 0x400) - 0x400;
                        z = (z - d) >> 11;  // exact: z - d is a multiple of 2^11
                    }
                    v = __int2half_rn(d);
                }
            }
            h[e] = __half_as_ushort(v);
        }
        *reinterpret_cast<uint4*>(out + (size_t)kb * B_BYTES + sw128(r, c)) =
            make_uint4(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16), h[4] | ((uint32_t)h[5] << 16),
                       h[6] | ((uint32_t)h[7] << 16));
    }
    if (threadIdx.x < SB) {
        const int j = sb * SB + threadIdx.x;
        const size_t o = (size_t)t * nsb * SB + j;
        tabs.sRe[o] = ldexpf(1.f, -ex[0][threadIdx.x]);
        tabs.sJ[o] = ldexpf(1.f, -ex[1][threadIdx.x]);
        if (j < n) {
            long long sr = base_re[(size_t)t * n + j], si = base_im[(size_t)t * n + j], sj = baseJ[j];
            for (int k = 0; k < n; ++k) {
                sr += qr[j * n + k];
                si += qi[j * n + k];
                sj += QJ[j * n + k];
            }
            tabs.aRe[o] = fx_to_float(sr);
            tabs.aJ[o] = fx_to_float(sj);
            tabs.aIm[o] = reduce_pi(si);
        } else {
            tabs.aRe[o] = 0.f;
            tabs.aJ[o] = 0.f;
            tabs.aIm[o] = 0;
        }
    }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct Smem {
    uint64_t bfull, mma;
    uint32_t tmem_slot;
    int abort_flag;
    float2 rs[SB][128];       // the tile's ratios, site-major
    uint64_t sw[2][128];      // the tile's spin words (64-site blocks 0 and 1)
    float tab[4][SB];         // aRe, sRe, aJ, sJ of the block's sites
    long long aim[SB];
    double acc[SB][5];        // per site: sums of Re r, Im r, sigma Re r, sigma Im r, sigma
};

template <int KB>
__global__ void __launch_bounds__(128, 4) est_tc_kernel(int n, int ns, double h, const uint64_t* __restrict__ spins,
                                                        const uint8_t* __restrict__ img, SiteTabs tabs,
                                                        float2* __restrict__ r_out, double2* __restrict__ EHq,
                                                        double2* __restrict__ part_r, double2* __restrict__ part_sr,
                                                        double* __restrict__ part_s, int nblk, int* status) {
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sA = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = sA + KB * A_BYTES;
    Smem& S = *reinterpret_cast<Smem*>(sB + KB * B_BYTES);
    const int chunk = blockIdx.x, sb = blockIdx.y, t = blockIdx.z, nsb = gridDim.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = (n + 63) / 64;
    volatile int* abort_flag = &S.abort_flag;

    if (tid == 0) {
        mbar_init(&S.bfull, 1);
        mbar_init(&S.mma, 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < SB * 5) (&S.acc[0][0])[tid] = 0.0;
    if (tid < SB) {
        const size_t o = (size_t)t * nsb * SB + sb * SB + tid;
        S.tab[0][tid] = tabs.aRe[o];
        S.tab[1][tid] = tabs.sRe[o];
        S.tab[2][tid] = tabs.aJ[o];
        S.tab[3][tid] = tabs.sJ[o];
        S.aim[tid] = tabs.aIm[o];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_slot;
    if (tid == 0) {
        mbar_expect_tx(&S.bfull, KB * B_BYTES);
        bulk_load(sB, img + ((size_t)t * nsb + sb) * KB * B_BYTES, KB * B_BYTES, &S.bfull);
    }

    const int jb0 = sb * SB;                  // first site of the block
    const int kw = jb0 >> 6;                  // its 64-site word
    int issued = 0;
#pragma unroll 1
    for (int tile = 0; tile < TILES; ++tile) {
        const int s0 = (chunk * TILES + tile) * 128;
        if (s0 >= ns) break;
        const int s = s0 + tid;
        const bool sv = s < ns;
        // the sigma tile: this thread's sample is row tid
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) {
            const uint64_t word = sv ? spins[((size_t)t * ns + s) * W + kb] : 0ull;
            S.sw[kb][tid] = word;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                uint32_t w4[4];
#pragma unroll
                for (int e2 = 0; e2 < 4; ++e2) {
                    uint32_t v2 = 0;
#pragma unroll
                    for (int e1 = 0; e1 < 2; ++e1) {
                        const int e = 2 * e2 + e1, k = 64 * kb + 8 * c + e;
                        const uint32_t bit = (uint32_t)(word >> (8 * c + e)) & 1u;
                        const uint32_t code = (sv && k < n) ? (0xBC00u ^ (bit << 15)) : 0u;
                        v2 |= code << (16 * e1);
                    }
                    w4[e2] = v2;
                }
                *reinterpret_cast<uint4*>(sA + kb * A_BYTES + sw128(tid, c)) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
        __syncthreads();
        if (tid == 0) {
            bool ok = !*abort_flag;
            if (ok && tile == 0 && !mbar_wait(&S.bfull, 0, abort_flag)) ok = false;
            if (ok) {
                fence_after();
                constexpr uint32_t ID = idesc_f16(128, NCOL);
#pragma unroll
                for (int kb = 0; kb < KB; ++kb)
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        umma(tmem, smem_desc(su32(sA + kb * A_BYTES) + k * 32), smem_desc(su32(sB + kb * B_BYTES) + k * 32),
                             ID, (kb > 0 || k > 0) ? 1u : 0u);
                umma_commit(&S.mma);
                ++issued;
            } else {
                *abort_flag = 1;
            }
        }
        int ok = 0;
        if (lane == 0) ok = !*abort_flag && mbar_wait(&S.mma, (uint32_t)tile & 1u, abort_flag) && !*abort_flag;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) *abort_flag = 1;
        fence_after();
        if (ok) {
            const uint32_t tq = tmem + ((uint32_t)(32 * warp) << 16);
            const uint64_t word = S.sw[kw][tid] >> (jb0 & 63);
            float fsg = 0.f, hrx = 0.f, hry = 0.f;
#pragma unroll 1
            for (int g = 0; g < 2; ++g) {
                const uint32_t tg = tq + (uint32_t)(8 * g);
                uint32_t v[8];
                float fre[8], fJ[8];
                tmem_ld8(tg + 0 * SB, v);
#pragma unroll
                for (int u = 0; u < 8; ++u) fre[u] = __uint_as_float(v[u]);
                tmem_ld8(tg + 1 * SB, v);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    fre[u] = fmaf(fre[u] + __uint_as_float(v[u]), S.tab[1][8 * g + u], S.tab[0][8 * g + u]);
                tmem_ld8(tg + 2 * SB, v);
#pragma unroll
                for (int u = 0; u < 8; ++u) fJ[u] = __uint_as_float(v[u]);
                tmem_ld8(tg + 3 * SB, v);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    fJ[u] = fmaf(fJ[u] + __uint_as_float(v[u]), S.tab[3][8 * g + u], S.tab[2][8 * g + u]);
                unsigned long long acc[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[u] = (unsigned long long)S.aim[8 * g + u];
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    tmem_ld8(tg + (uint32_t)((4 + d) * SB), v);
                    // digit sums are exact integers of at most 2^17 in magnitude; wrapping
                    // 64-bit arithmetic (the true field fits in 64 bits)
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        acc[u] += (unsigned long long)(long long)__float2int_rn(__uint_as_float(v[u])) << (11 * d);
                }
                float2 rr[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int j = jb0 + 8 * g + u;
                    const bool valid = sv && j < n;
                    const bool up = (word >> (8 * g + u)) & 1ull;
                    const long long fim = (long long)(acc[u] << IM_SHIFT);  // units of 2^-48
                    const long long lim = up ? -2 * fim : 2 * fim;
                    const float e = expf(up ? -2.f * fre[u] : 2.f * fre[u]);
                    const int kq = __float2int_rn(fx_to_float(lim) * 0.15915494309189535f);
                    const long long red = lim - (long long)kq * FX_TWO_PI;
                    float sn, cs;
                    sincosf(fx_to_float(red), &sn, &cs);
                    rr[u] = valid ? make_float2(e * cs, e * sn) : make_float2(0.f, 0.f);
                    if (valid) {
                        fsg += up ? fJ[u] : -fJ[u];
                        hrx += rr[u].x;
                        hry += rr[u].y;
                    }
                    S.rs[8 * g + u][tid] = rr[u];
                }
                if (sv) {
                    const int j0 = jb0 + 8 * g;
                    float2* dst = r_out + ((size_t)t * ns + s) * n + j0;
                    if ((n & 1) == 0 && j0 + 8 <= n) {
                        float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            d4[u] = make_float4(rr[2 * u].x, rr[2 * u].y, rr[2 * u + 1].x, rr[2 * u + 1].y);
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (j0 + u < n) dst[u] = rr[u];
                    }
                }
            }
            if (sv) EHq[((size_t)t * ns + s) * nsb + sb] = make_double2(0.5 * (double)fsg + h * (double)hrx, h * (double)hry);
        }
        fence_before();
        __syncthreads();
        // per-site sums over the tile: site u = tid / 8 takes samples p, p + 8, ... (p = tid % 8),
        // then the eight partial sums of a site are combined in a fixed tree
        if (!*abort_flag) {
            const int u = tid >> 3, p = tid & 7;
            const int sh = (jb0 & 63) + u;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f;
#pragma unroll 4
            for (int i = p; i < 128; i += 8) {
                const float2 r = S.rs[u][i];
                const bool in = s0 + i < ns && jb0 + u < n;
                const float sg = in ? (((S.sw[kw][i] >> sh) & 1ull) ? 1.f : -1.f) : 0.f;
                a0 += r.x;
                a1 += r.y;
                a2 = fmaf(sg, r.x, a2);
                a3 = fmaf(sg, r.y, a3);
                a4 += sg;
            }
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, off);
                a1 += __shfl_xor_sync(0xffffffffu, a1, off);
                a2 += __shfl_xor_sync(0xffffffffu, a2, off);
                a3 += __shfl_xor_sync(0xffffffffu, a3, off);
                a4 += __shfl_xor_sync(0xffffffffu, a4, off);
            }
            if (p == 0) {
                S.acc[u][0] += (double)a0;
                S.acc[u][1] += (double)a1;
                S.acc[u][2] += (double)a2;
                S.acc[u][3] += (double)a3;
                S.acc[u][4] += (double)a4;
            }
        }
        __syncthreads();  // rs, sw, the sigma tile and TMEM are free again
    }
    if (!*abort_flag && tid < SB) {
        const int j = jb0 + tid;
        if (j < n) {
            const size_t o = ((size_t)t * nblk + chunk) * n + j;
            part_r[o] = make_double2(S.acc[tid][0], S.acc[tid][1]);
            part_sr[o] = make_double2(S.acc[tid][2], S.acc[tid][3]);
            part_s[o] = S.acc[tid][4];
        }
    }
    __syncthreads();
    if (tid == 0 && *abort_flag) {
        record_error(status, OTVMC_ERR_TIMEOUT, t);
        // drain: the bulk copy and the last committed MMAs must be complete before exit
        mbar_wait(&S.bfull, 0, nullptr);
        if (issued > 0) mbar_wait(&S.mma, (uint32_t)(issued - 1) & 1u, nullptr);
    }
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
    }
}

template <int KB>
constexpr int smem_bytes() {
    return KB * (A_BYTES + B_BYTES) + (int)sizeof(Smem) + 1024;
}

}  // namespace etc

cudaError_t est_tc_set_wait_limit(unsigned long long ns) { return tc::set_wait_limit_tu(ns); }

size_t est_tc_bytes(int ntraj, int n) {
    if (n > ETC_MAX_N) return 0;
    const int nsb = (n + ETC_SITES - 1) / ETC_SITES, KB = (n + 63) / 64;
    return (size_t)ntraj * nsb * KB * etc::B_BYTES + (size_t)ntraj * nsb * ETC_SITES * 24 + 1024;
}

cudaError_t launch_est_tc(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, const EvalBufs& b,
                          int* status, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_EST1, s);
    const int n = a->n;
    if (n > ETC_MAX_N || b.etc == nullptr) return cudaErrorInvalidValue;
    const int nsb = (n + ETC_SITES - 1) / ETC_SITES, KB = (n + 63) / 64;
    uint8_t* img = (uint8_t*)(((uintptr_t)b.etc + 1023) & ~(uintptr_t)1023);
    const size_t ns_sites = (size_t)ntraj * nsb * ETC_SITES;
    etc::SiteTabs tabs;
    tabs.aIm = (long long*)(img + (size_t)ntraj * nsb * KB * etc::B_BYTES);
    tabs.aRe = (float*)(tabs.aIm + ns_sites);
    tabs.aJ = tabs.aRe + ns_sites;
    tabs.sRe = tabs.aJ + ns_sites;
    tabs.sJ = tabs.sRe + ns_sites;
    const otvmc_model* m = a->model;
    etc::est_tc_prep_kernel<<<dim3(nsb, ntraj), 256, 0, s>>>(n, KB, b.Qre, b.Qim, b.base_re, b.base_im, m->QJ_d,
                                                             m->baseJ_d, img, tabs);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nblk = est_tc_chunks(ns);
    dim3 grid(nblk, nsb, ntraj);
    if (KB == 1) {
        constexpr int SM = etc::smem_bytes<1>();
        e = cudaFuncSetAttribute(etc::est_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
        if (e != cudaSuccess) return e;
        etc::est_tc_kernel<1><<<grid, 128, SM, s>>>(n, ns, m->h, spins, img, tabs,
                                                    reinterpret_cast<float2*>(b.r), b.EH, b.part_r, b.part_sr,
                                                    b.part_s, nblk, status);
    } else {
        constexpr int SM = etc::smem_bytes<2>();
        e = cudaFuncSetAttribute(etc::est_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
        if (e != cudaSuccess) return e;
        etc::est_tc_kernel<2><<<grid, 128, SM, s>>>(n, ns, m->h, spins, img, tabs,
                                                    reinterpret_cast<float2*>(b.r), b.EH, b.part_r, b.part_sr,
                                                    b.part_s, nblk, status);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
