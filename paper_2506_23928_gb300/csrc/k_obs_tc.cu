// Per-trajectory observables of the Jastrow ansatz with the two-flip sums on the tensor cores
// (mixed path, 32 <= N <= 64).
//
// The pair moments (LITF paragraph: the squeezing parameter needs <s^a_j s^b_k>) use the
// two-flip ratios r_jk = r_j r_k E^{s_j s_k}_jk, E^{+-}_jk = exp(+-4 eta_jk) (zero on the
// diagonal).  With u+ = r o [s = +1] and u- = r o [s = -1] (per sample), the three sums over
// j != k that the moments need are bilinear forms:
//   A1 = u+^T E+ u+,  A2 = u-^T E+ u-,  A3 = u+^T E- u-   (E+- symmetric),
//   sum r_jk = A1 + A2 + 2 A3,  sum s_j s_k r_jk = A1 + A2 - 2 A3,  sum s_k r_jk = A1 - A2,
// and over a tile of 128 samples the products Y1 = E+ u+, Y2 = E+ u-, Y3 = E- u- are three
// (128 x 2N) . (2N x 2N) real products (the complex matrices in their real embedding: row j of
// Re Y takes [Re E_j., -Im E_j.], row N + j of Im Y takes [Im E_j., Re E_j.], against
// [Re u, Im u]).  They run on tcgen05 (kind::f16, FP16 in, FP32 accumulate in TMEM): u+- and
// E+- each as two FP16 pieces h + m after a power-of-two scale (per sample for u, per row j for
// E), three piece products (h.h, h.m, m.h).  The epilogue takes the dot products with u+- and
// adds the single-site terms; one partial of the nine moments per CTA, in the layout of the
// SIMT kernel, so that obs_final_kernel reads either.
//
// One CTA = 4 tiles of 128 samples of one trajectory, 128 threads (one per sample of a tile),
// 384 of 512 TMEM columns, about 195 KB of shared memory: one CTA per SM.  Per tile and per
// half of K (Re u, then Im u): the threads write the A operands (u+, u- pieces) from the staged
// ratios, one bulk copy brings the B operands (E+, E- pieces), one thread issues the MMAs.
// Every mbarrier wait is bounded; on timeout the CTA records OTVMC_ERR_TIMEOUT, drains its
// copies and MMAs (bounded), frees TMEM and returns.
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace otvmc {
namespace otc {

constexpr int TILES = 4;
constexpr int BLK = 16384;              // one 128-row x 64-column FP16 operand block, 128-byte swizzle
constexpr int B_HALF = 4 * BLK;         // E+ h, E+ m, E- h, E- m of one half of K
constexpr int RS = 65;                  // row stride (float2) of the staged ratios
constexpr uint32_t TCOLS = 512;

__host__ __device__ __forceinline__ int sw128(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }
__device__ __forceinline__ int row_exp(float mx) { return mx > 0.f ? 13 - ilogbf(mx) : 0; }

// B images of one trajectory: img[t][kh][e][piece] (kh = half of K, e = E+ / E-), each a
// 128 x 64 block; rows j < 64 give Re Y_j, rows 64 + j give Im Y_j; escale[t][e][j] = 2^-ex.
__global__ void __launch_bounds__(256) obs_tc_prep_kernel(int n, const double2* __restrict__ Epm,
                                                          uint8_t* __restrict__ img, float* __restrict__ escale) {
    __shared__ int ex[2][64];
    const int t = blockIdx.x;
    const double2* E = Epm + (size_t)t * 2 * n * n;
    if (threadIdx.x < 128) {
        const int e = threadIdx.x >> 6, j = threadIdx.x & 63;
        float mx = 0.f;
        if (j < n)
            for (int k = 0; k < n; ++k)
                if (k != j) {
                    const double2 v = E[(size_t)e * n * n + (size_t)k * n + j];
                    mx = fmaxf(mx, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
                }
        ex[e][j] = row_exp(mx);
        escale[((size_t)t * 2 + e) * 64 + j] = ldexpf(1.f, -ex[e][j]);
    }
    __syncthreads();
    uint8_t* out = img + (size_t)t * 2 * B_HALF;
    // units: (kh, e, piece, row, 16-byte unit c)
    for (int q = threadIdx.x; q < 2 * 2 * 2 * 128 * 8; q += blockDim.x) {
        const int c = q & 7, row = (q >> 3) & 127, piece = (q >> 10) & 1, e = (q >> 11) & 1, kh = q >> 12;
        const int j = row & 63, im = row >> 6;
        uint16_t hv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = 8 * c + i;
            float x = 0.f;
            if (j < n && k < n && j != k) {
                // E^{+-}_jk stored at [e][k][j] by obs_prep_kernel
                const double2 v = E[(size_t)e * n * n + (size_t)k * n + j];
                const float re = (float)v.x, iv = (float)v.y;
                x = kh == 0 ? (im ? iv : re) : (im ? re : -iv);
                x = ldexpf(x, ex[e][j]);
            }
            const __half h = __float2half_rn(x);
            hv[i] = __half_as_ushort(piece ? __float2half_rn(x - __half2float(h)) : h);
        }
        *reinterpret_cast<uint4*>(out + (size_t)kh * B_HALF + (size_t)(e * 2 + piece) * BLK + sw128(row, c)) =
            make_uint4(hv[0] | ((uint32_t)hv[1] << 16), hv[2] | ((uint32_t)hv[3] << 16), hv[4] | ((uint32_t)hv[5] << 16),
                       hv[6] | ((uint32_t)hv[7] << 16));
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
    float esc[2][64];         // E+- row scales 2^-ex (the trajectory's)
    double red[4][9];         // per warp: the nine moments summed over its samples
};
constexpr int SMEM_BYTES = 4 * BLK + B_HALF + 128 * RS * 8 + (int)sizeof(Smem) + 1024;

// Moments of the tile's samples (grid: sample chunks x T).  part_obs[t][chunk][9] as
// observables_kernel writes it.
__global__ void __launch_bounds__(128, 1) obs_tc_kernel(int n, int ns, const uint64_t* __restrict__ spins,
                                                        const float2* __restrict__ r, const uint8_t* __restrict__ img,
                                                        const float* __restrict__ escale, double* __restrict__ part_obs,
                                                        int* status) {
    using namespace tc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sA = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);  // [u+-][piece] blocks
    uint8_t* sB = sA + 4 * BLK;                                                    // [E+-][piece] blocks
    float2* rs = (float2*)(sB + B_HALF);                                           // [128][RS] staged ratios
    Smem& S = *reinterpret_cast<Smem*>((uint8_t*)rs + 128 * RS * 8);
    const int chunk = blockIdx.x, t = blockIdx.y;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int* abort_flag = &S.abort_flag;

    if (tid == 0) {
        mbar_init(&S.bfull, 1);
        mbar_init(&S.mma, 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    S.esc[tid >> 6][tid & 63] = escale[(size_t)t * 128 + tid];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem_slot)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_slot;
    const uint8_t* bimg = img + (size_t)t * 2 * B_HALF;

    double acc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = 0.0;
    int nmma = 0, nb = 0;  // MMA groups committed, B copies issued
#pragma unroll 1
    for (int tile = 0; tile < TILES; ++tile) {
        const int s0 = (chunk * TILES + tile) * 128;
        if (s0 >= ns || *abort_flag) break;
        const int s = s0 + tid;
        const bool sv = s < ns;
        // stage the tile's ratios (contiguous in r), then this sample's spin word and scale
        {
            const int cnt = min(128, ns - s0) * n;
            const float2* src = r + ((size_t)t * ns + s0) * n;
            for (int i = tid; i < cnt; i += 128) rs[(i / n) * RS + (i % n)] = src[i];
        }
        const uint64_t word = sv ? spins[(size_t)t * ns + s] : 0ull;
        __syncthreads();
        const float2* rr = rs + tid * RS;
        float mx = 0.f;
        for (int k = 0; k < n; ++k) mx = fmaxf(mx, fmaxf(fabsf(rr[k].x), fabsf(rr[k].y)));
        const int xs = sv ? row_exp(mx) : 0;
#pragma unroll 1
        for (int kh = 0; kh < 2; ++kh) {
            if (tid == 0 && !*abort_flag) {
                mbar_expect_tx(&S.bfull, B_HALF);
                bulk_load(sB, bimg + (size_t)kh * B_HALF, B_HALF, &S.bfull);
                ++nb;
            }
            // A: [u+ h, u+ m, u- h, u- m], row tid, columns k < 64 (kh = 0: Re u_k, 1: Im u_k)
#pragma unroll 1
            for (int c = 0; c < 8; ++c) {
                uint32_t w[4][4];
#pragma unroll
                for (int i2 = 0; i2 < 4; ++i2) {
                    uint32_t pk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int e1 = 0; e1 < 2; ++e1) {
                        const int k = 8 * c + 2 * i2 + e1;
                        float x = 0.f;
                        if (sv && k < n) x = ldexpf(kh == 0 ? rr[k].x : rr[k].y, xs);
                        const __half h = __float2half_rn(x);
                        const __half m = __float2half_rn(x - __half2float(h));
                        const bool up = (word >> k) & 1ull;
                        const uint32_t hb = __half_as_ushort(h), mb = __half_as_ushort(m);
                        pk[0] |= (up ? hb : 0u) << (16 * e1);
                        pk[1] |= (up ? mb : 0u) << (16 * e1);
                        pk[2] |= (up ? 0u : hb) << (16 * e1);
                        pk[3] |= (up ? 0u : mb) << (16 * e1);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) w[b][i2] = pk[b];
                }
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    *reinterpret_cast<uint4*>(sA + b * BLK + sw128(tid, c)) = make_uint4(w[b][0], w[b][1], w[b][2], w[b][3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor core
            __syncthreads();
            if (tid == 0) {
                bool ok = !*abort_flag && mbar_wait(&S.bfull, (uint32_t)(nb - 1) & 1u, abort_flag);
                if (ok) {
                    fence_after();
                    constexpr uint32_t ID = idesc_f16(128, 128);
                    // outputs: Y1 = E+ u+ (cols 0..127), Y2 = E+ u- (128..255), Y3 = E- u- (256..383)
                    const int ua[3] = {0, 2, 2}, eb[3] = {0, 0, 2};
                    const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
#pragma unroll
                    for (int o = 0; o < 3; ++o)
#pragma unroll
                        for (int q = 0; q < 3; ++q)
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                umma(tmem + 128 * o, smem_desc(su32(sA + (ua[o] + pa[q]) * BLK) + k * 32),
                                     smem_desc(su32(sB + (eb[o] + pb[q]) * BLK) + k * 32), ID,
                                     (kh > 0 || q > 0 || k > 0) ? 1u : 0u);
                    umma_commit(&S.mma);
                    ++nmma;
                } else {
                    *abort_flag = 1;
                }
            }
            __syncthreads();  // nmma / abort seen by all (thread 0 wrote them before the barrier)
            int ok = 0;
            if (lane == 0) ok = !*abort_flag && mbar_wait(&S.mma, (uint32_t)(2 * tile + kh) & 1u, abort_flag);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) *abort_flag = 1;
            fence_after();
            __syncthreads();  // the operands may be overwritten: the products are complete
        }
        if (*abort_flag) break;
        // epilogue: this sample's dot products with u+- (true values from the staged ratios)
        const uint32_t tq = tmem + ((uint32_t)(32 * warp) << 16);
        const float inv_u = ldexpf(1.f, -xs);
        float a1x = 0.f, a1y = 0.f, a2x = 0.f, a2y = 0.f, a3x = 0.f, a3y = 0.f;
        float sre = 0.f, sim = 0.f, ssre = 0.f, ssim = 0.f;
#pragma unroll 1
        for (int j0 = 0; j0 < 64; j0 += 8) {
            uint32_t y1r[8], y1i[8], y2r[8], y2i[8], y3r[8], y3i[8];
            tmem_ld8(tq + j0, y1r);
            tmem_ld8(tq + 64 + j0, y1i);
            tmem_ld8(tq + 128 + j0, y2r);
            tmem_ld8(tq + 192 + j0, y2i);
            tmem_ld8(tq + 256 + j0, y3r);
            tmem_ld8(tq + 320 + j0, y3i);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u;
                if (!sv || j >= n) continue;
                const float2 rj = rr[j];
                const bool up = (word >> j) & 1ull;
                const float fp = inv_u * S.esc[0][j], fm = inv_u * S.esc[1][j];
                const float Y1r = __uint_as_float(y1r[u]) * fp, Y1i = __uint_as_float(y1i[u]) * fp;
                const float Y2r = __uint_as_float(y2r[u]) * fp, Y2i = __uint_as_float(y2i[u]) * fp;
                const float Y3r = __uint_as_float(y3r[u]) * fm, Y3i = __uint_as_float(y3i[u]) * fm;
                if (up) {
                    // u+_j (E+ u+)_j and u+_j (E- u-)_j
                    a1x += rj.x * Y1r - rj.y * Y1i;
                    a1y += rj.x * Y1i + rj.y * Y1r;
                    a3x += rj.x * Y3r - rj.y * Y3i;
                    a3y += rj.x * Y3i + rj.y * Y3r;
                    ssre += rj.x;
                    ssim += rj.y;
                } else {
                    a2x += rj.x * Y2r - rj.y * Y2i;
                    a2y += rj.x * Y2i + rj.y * Y2r;
                    ssre -= rj.x;
                    ssim -= rj.y;
                }
                sre += rj.x;
                sim += rj.y;
            }
        }
        if (sv) {
            const int Ssum = 2 * __popcll(word) - n;
            const double fS = (double)Ssum;
            acc[0] += (double)sre;                          // sum Re r_j
            acc[1] += (double)ssim;                         // sum s_j Im r_j
            acc[2] += fS;                                   // sum s_j
            acc[3] += (double)(a1x + a2x + 2.f * a3x);      // Re sum r_jk
            acc[4] -= (double)(a1x + a2x - 2.f * a3x);      // -Re sum s_j s_k r_jk
            acc[5] += fS * fS - (double)n;                  // S^2 - n
            acc[6] += (double)(a1y - a2y);                  // Im sum s_k r_jk
            acc[7] += fS * (double)sre - (double)ssre;      // sum Re r_j (S - s_j)
            acc[8] += fS * (double)ssim - (double)sim;      // sum s_j Im r_j (S - s_j)
        }
        fence_before();
        __syncthreads();  // TMEM and the staged ratios are free again
    }
    // the CTA's partial: warps in order
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        double v = acc[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) S.red[warp][i] = v;
    }
    __syncthreads();
    if (tid < 9 && !*abort_flag)
        part_obs[((size_t)t * gridDim.x + chunk) * 9 + tid] = S.red[0][tid] + S.red[1][tid] + S.red[2][tid] + S.red[3][tid];
    if (tid == 0 && *abort_flag) {
        record_error(status, OTVMC_ERR_TIMEOUT, t);
        // drain: every bulk copy and committed MMA group must be complete before exit
        if (nb > 0) mbar_wait(&S.bfull, (uint32_t)(nb - 1) & 1u, nullptr);
        if (nmma > 0) mbar_wait(&S.mma, (uint32_t)(nmma - 1) & 1u, nullptr);
    }
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
    }
}

}  // namespace otc

cudaError_t obs_tc_set_wait_limit(unsigned long long ns) { return tc::set_wait_limit_tu(ns); }

size_t obs_tc_bytes(int ntraj, int n) {
    if (n < OTC_MIN_N || n > OTC_MAX_N) return 0;
    return (size_t)ntraj * (2 * otc::B_HALF + 2 * 64 * sizeof(float)) + 1024;
}

cudaError_t launch_obs_tc(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, const EvalBufs& b,
                          double* moments, int* status, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_OBS, s);
    const int n = a->n;
    if (n < OTC_MIN_N || n > OTC_MAX_N || b.otc == nullptr) return cudaErrorInvalidValue;
    uint8_t* img = (uint8_t*)(((uintptr_t)b.otc + 1023) & ~(uintptr_t)1023);
    float* escale = (float*)(img + (size_t)ntraj * 2 * otc::B_HALF);
    otc::obs_tc_prep_kernel<<<ntraj, 256, 0, s>>>(n, b.Epm, img, escale);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nblk = obs_tc_chunks(ns);
    e = cudaFuncSetAttribute(otc::obs_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, otc::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    otc::obs_tc_kernel<<<dim3(nblk, ntraj), 128, otc::SMEM_BYTES, s>>>(n, ns, spins, reinterpret_cast<const float2*>(b.r),
                                                                      img, escale, b.part_obs, status);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_obs_final_n(n, ns, ntraj, nblk, b, moments, s);
}

}  // namespace otvmc
