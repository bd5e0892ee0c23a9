// Uncentred Gram matrix G = O^T O of the local operators on the 5th-generation tensor cores
// (tcgen05, sm_103a): the contraction behind the quantum geometric tensor
// S = <O^* O> - <O^*><O> (definitions after Eq. 8), S = G / ns - obar obar^T.
//
// For the Jastrow ansatz O = +-1 is exact in E4M3, the operands are FP8 (kind::f8f6f4, twice
// the BF16 rate, half the bytes) and FP32 accumulation of integer sums below 2^24 is exact, so
// G (and with the FP64 centring, S) is exact.  The same kernel in BF16 forms the Gram of the
// three-piece split operands of the RBM path.
//
// One CTA computes one 128 x 256 tile of the upper triangle of G for one trajectory:
//   warp 0      TMA producer: three 128-row boxes (A rows i, B rows j, j+128) of 128 bytes
//               per stage into a 2-stage ring, 128-byte swizzled, completing on mbarriers (two
//               CTAs per SM, so that one CTA's epilogue overlaps the other's MMAs);
//   warp 1      allocates 256 TMEM columns; one lane issues tcgen05.mma (M=128, N=256,
//               K = 32 E4M3 or 16 BF16, FP32 accumulate in TMEM) and commits each stage back;
//   warps 2..5  epilogue: tcgen05.ld of their 32 TMEM lanes, FP32 stores of the j >= i part;
//               operand rows from P on (the digits of the quantised v and a row of ones, on the
//               mixed Jastrow path) give the columns of a side output X instead.
// Every mbarrier wait is bounded (2 s of %globaltimer); on timeout the CTA records
// OTVMC_ERR_TIMEOUT, drains its own copies and MMAs (bounded), frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "tc_common.cuh"

namespace otvmc {
namespace tc {

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int STAGES = 2;  // two CTAs per SM: one's epilogue overlaps the other's MMAs
constexpr int BOX_BYTES = 128 * BK * 2;  // 16 KB: one 128-row box
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint32_t TMEM_COLS = 256;

// Split operands: X = [X_h | X_m | X_l] stacked along k (piece stride kpad); the k loop runs
// over the products (h,h) (h,m) (m,h) (h,l) (m,m) (l,h) of a piece of the A rows with a piece
// of the B rows, whose FP32 sum reproduces the product of the unsplit operand to ~2^-24.
__constant__ int c_pair_a[6] = {0, 0, 1, 0, 1, 2};
__constant__ int c_pair_b[6] = {0, 1, 0, 2, 1, 0};

// (mb, nb) of upper-triangle tile q, enumerated in the order of gram_tiles()
__device__ __forceinline__ int2 tile_of(int q, int P) {
    const int MT = (P + BM - 1) / BM, NT = (P + BN - 1) / BN;
    for (int mb = 0; mb < MT; ++mb) {
        const int first = (mb * BM) / BN;  // smallest nb with (nb + 1) BN > mb BM
        const int cnt = NT - first;
        if (q < cnt) return make_int2(mb, first + q);
        q -= cnt;
    }
    return make_int2(MT, NT);
}

// F8: operands in E4M3 (kind::f8f6f4, 128 samples per 128-byte stage row, K = 32 per MMA);
// else BF16 (kind::f16, 64 samples per row, K = 16).  The stage layout in bytes is the same.
template <bool F8>
__global__ void __launch_bounds__(192, 2) gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, int P, int ns,
                                                          int kpad, int npairs, const int2* __restrict__ tiles,
                                                          float* __restrict__ G, float* __restrict__ X, int nx,
                                                          int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * A_BYTES;
    uint64_t* full = (uint64_t*)(sB + STAGES * B_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* done = empty + STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int t = blockIdx.y;
    const int2 tl = tiles ? tiles[blockIdx.x] : tile_of(blockIdx.x, P);
    const int i0 = tl.x * BM, j0 = tl.y * BN;
    constexpr int BKE = F8 ? 2 * BK : BK;  // samples per stage
    const int nks = (ns + BKE - 1) / BKE;  // k slices of one piece
    const int nk = nks * npairs;

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
                     "r"(TMEM_COLS));
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
                mbar_expect_tx(&full[s], STAGE_BYTES);
                const int pr = kb / nks, kk = kb - pr * nks;
                const int ka = c_pair_a[pr] * kpad + kk * BKE, kbx = c_pair_b[pr] * kpad + kk * BKE;
                tma_load_3d(sA + s * A_BYTES, &tmap, &full[s], ka, i0, t);
                tma_load_3d(sB + s * B_BYTES, &tmap, &full[s], kbx, j0, t);
                tma_load_3d(sB + s * B_BYTES + BOX_BYTES, &tmap, &full[s], kbx, j0 + 128, t);
                ++issued;
            }
            // drain: every issued stage must have landed before the CTA may exit
            for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
                mbar_wait(&full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, nullptr);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % STAGES;
                const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                fence_after();
                const uint32_t a0 = su32(sA + s * A_BYTES), b0 = su32(sB + s * B_BYTES);
#pragma unroll
                for (int k = 0; k < BK / 16; ++k) {  // 32 bytes of each row per instruction
                    if (F8)
                        umma_f8(tmem, smem_desc(a0 + k * 32), smem_desc(b0 + k * 32), idesc_e4m3(BM, BN),
                                (kb > 0 || k > 0) ? 1u : 0u);
                    else
                        umma(tmem, smem_desc(a0 + k * 32), smem_desc(b0 + k * 32), idesc_bf16(BM, BN),
                             (kb > 0 || k > 0) ? 1u : 0u);
                }
                umma_commit(&empty[s]);
            }
            umma_commit(done);
        }
        __syncwarp();
    } else {
        const int q = warp & 3;  // TMEM lanes 32q..32q+31 belong to this warp
        int ok = 0;
        if (lane == 0) {
            ok = mbar_wait(done, 0, abort_flag) && !*abort_flag;
            if (!ok) *abort_flag = 1;  // a wait that ran out here is reported as well
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
        fence_after();
        if (ok) {
            const int row = q * 32 + lane;
            const int gi = i0 + row;
            float* Grow = G + ((size_t)t * P + (gi < P ? gi : 0)) * P;
            // columns P .. P + nx - 1 (extra rows of the operand) of the rows gi < P go to X
            float* Xrow = (X != nullptr && gi < P) ? X + ((size_t)t * P + gi) * nx : nullptr;
#pragma unroll 1
            for (int c = 0; c < BN; c += 32) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
                const int gj0 = j0 + c;
                if (Xrow != nullptr && gj0 + 31 >= P && gj0 < P + nx) {
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const int gj = gj0 + u;
                        if (gj >= P && gj < P + nx) Xrow[gj - P] = __uint_as_float(v[u]);
                    }
                }
                if (gi >= P || gj0 + 31 < gi || gj0 >= P) continue;
                if (gj0 >= gi && gj0 + 31 < P && ((reinterpret_cast<uintptr_t>(Grow + gj0) & 15u) == 0)) {
                    float4* dst = (float4*)(Grow + gj0);
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        dst[u] = make_float4(__uint_as_float(v[4 * u]), __uint_as_float(v[4 * u + 1]),
                                             __uint_as_float(v[4 * u + 2]), __uint_as_float(v[4 * u + 3]));
                } else {
#pragma unroll
                    for (int u = 0; u < 32; ++u) {
                        const int gj = gj0 + u;
                        if (gj >= gi && gj < P) Grow[gj] = __uint_as_float(v[u]);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) record_error(status, OTVMC_ERR_TIMEOUT, t);
    if (warp == 1) {
        // all MMAs of this CTA have completed once `done` fired; wait (bounded) before freeing
        if (lane == 0) mbar_wait(done, 0, nullptr);
        __syncwarp();
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

}  // namespace tc

cudaError_t gram_set_wait_limit(unsigned long long ns) { return tc::set_wait_limit_tu(ns); }

// Upper-triangle tiles (mb, nb) of 128 x 256 that contain some j >= i.
std::vector<int2> gram_tiles(int P) { return gram_tiles_x(P, P); }

// Tiles (mb, nb) of 128 rows < P by 256 columns < PC (PC >= P) that contain some column >= row.
std::vector<int2> gram_tiles_x(int P, int PC) {
    std::vector<int2> v;
    const int MT = (P + tc::BM - 1) / tc::BM, NT = (PC + tc::BN - 1) / tc::BN;
    for (int mb = 0; mb < MT; ++mb)
        for (int nb = 0; nb < NT; ++nb)
            if ((nb + 1) * tc::BN > mb * tc::BM) v.push_back(make_int2(mb, nb));
    return v;
}

cudaError_t launch_gram_tc(int ntraj, int P, int rows, int ns, int pitch, const uint8_t* Ot, const int2* tiles,
                           int ntiles, float* G, float* X, int* status, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_GRAM, s);
    if (rows < P || (X != nullptr && rows == P) || pitch < ns || pitch % 16 != 0) return cudaErrorInvalidValue;
    auto encode = tc::get_encode();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)rows, (cuuint64_t)ntraj};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch, (cuuint64_t)rows * pitch};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * tc::BK), 128u, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, (void*)Ot, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc::gram_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    dim3 grid(ntiles, ntraj);
    tc::gram_tc_kernel<true><<<grid, 192, tc::SMEM_BYTES, s>>>(map, P, pitch, pitch, 1, tiles, G, X,
                                                                X ? rows - P : 0, status);
    count_launch();
    return cudaGetLastError();
}

// G = X X^T (upper triangle, FP32) for X = X_h + X_m + X_l given as the three BF16 pieces
// stacked along k: Xs[t][row][piece * kpad + k], rows x K per piece (K <= kpad, kpad a multiple
// of 64, the columns K..kpad zero), six piece products.
cudaError_t launch_gram_split(int ntraj, int rows, int K, int kpad, const uint16_t* Xs, float* G, int* status,
                              cudaStream_t s) {
    ProfScope prof_(OTVMC_K_GRAM, s);
    if (kpad % tc::BK != 0 || K > kpad) return cudaErrorInvalidValue;
    auto encode = tc::get_encode();
    if (!encode) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)3 * kpad, (cuuint64_t)rows, (cuuint64_t)ntraj};
    const cuuint64_t strides[2] = {(cuuint64_t)3 * kpad * 2, (cuuint64_t)rows * 3 * kpad * 2};
    const cuuint32_t box[3] = {(cuuint32_t)tc::BK, 128u, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)Xs, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(tc::gram_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tc::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const int ntiles = (int)gram_tiles(rows).size();
    dim3 grid(ntiles, ntraj);
    tc::gram_tc_kernel<false><<<grid, 192, tc::SMEM_BYTES, s>>>(map, rows, kpad, kpad, 6, nullptr, G, nullptr, 0, status);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
