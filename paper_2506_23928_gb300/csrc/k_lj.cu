// Partially inhomogeneous long-range Jastrow LJPHd / LJH (Eq. 12 and the paragraph after it).
//
// The two-body parameters are shared within groups of pairs: eta_jk = eta_g(j,k), every pair at
// distance <= d in a group of its own, all pairs at one larger distance in one group.  So
//     log psi = sum_i a_i s_i + sum_g eta_g sum_{(j,k) in g} s_j s_k,
//     O_{a_i} = s_i,   O_{eta_g} = sum_{(j,k) in g} s_j s_k   (an integer, |O| <= group size).
// Sampling, local estimators and observables only need the pair parameters eta_jk, so they run
// the full-Jastrow kernels on the expanded parameters theta_full (expand kernel).  D and obar are
// the full Jastrow's exact sums folded over each group (fold kernel).  S = G / ns - obar obar^T
// from the integer Gram matrix G = sum_x O(x) O(x)^T, accumulated exactly in integers on the CUDA
// cores (the tied rows reach |O| = N, so their products exceed what an FP32 tensor-core
// accumulator holds exactly; P is N + a few N, small next to the full Jastrow's N(N+1)/2).
#include "common.cuh"

namespace otvmc {
namespace lj {

constexpr int GT = 64;  // Gram tile (rows x columns)
constexpr int GK = 64;  // samples per chunk of the Gram kernel

// theta_full[t] = [a, eta_jk for j < k row-major] from theta[t] = [a, eta_g]
__global__ void expand_kernel(int n, int P, int Pf, const int* __restrict__ pair_grp,
                              const double2* __restrict__ theta, double2* __restrict__ theta_full) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Pf) return;
    const double2* th = theta + (size_t)t * P;
    theta_full[(size_t)t * Pf + k] = k < n ? th[k] : th[n + pair_grp[k - n]];
}

// obar[t][k] (and D, if given) of the tied parameters: the biases copied, each group the sum of
// its pairs' full-Jastrow values (in the fixed group order of grp_off / grp_pair).
__global__ void fold_kernel(int n, int P, int Pf, const int* __restrict__ grp_off, const int* __restrict__ grp_pair,
                            const double* __restrict__ obar_full, const double2* __restrict__ D_full,
                            double* __restrict__ obar, double2* __restrict__ D) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const double* of = obar_full + (size_t)t * Pf;
    const double2* df = D_full + (size_t)t * Pf;
    double o;
    double2 v;
    if (k < n) {
        o = of[k];
        v = df[k];
    } else {
        o = 0.0;
        v = make_double2(0.0, 0.0);
        for (int e = grp_off[k - n]; e < grp_off[k - n + 1]; ++e) {
            const int q = n + grp_pair[e];
            o += of[q];
            v.x += df[q].x;
            v.y += df[q].y;
        }
    }
    obar[(size_t)t * P + k] = o;
    if (D) D[(size_t)t * P + k] = v;
}

// O[t][k][x] as int16: s_k for k < n, sum over the group's pairs of s_j s_l for the rest.
// One thread per sample (coalesced stores along x), 16 rows per CTA row block.
__global__ void __launch_bounds__(256) obuild_kernel(int n, int W, int P, int ns, const int* __restrict__ grp_off,
                                                     const int* __restrict__ grp_pair, const int* __restrict__ pairs,
                                                     const uint64_t* __restrict__ spins, int16_t* __restrict__ O) {
    const int t = blockIdx.z, k0 = blockIdx.y * 16;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ns) return;
    uint64_t w[4];
    const uint64_t* sp = spins + ((size_t)t * ns + x) * W;
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = q < W ? sp[q] : 0ull;
    for (int k = k0; k < k0 + 16 && k < P; ++k) {
        int v;
        if (k < n) {
            v = ((w[k >> 6] >> (k & 63)) & 1ull) ? 1 : -1;
        } else {
            // s_j s_l = +1 when the bits agree; sum = size - 2 (number of disagreeing pairs)
            const int e0 = __ldg(grp_off + k - n), e1 = __ldg(grp_off + k - n + 1);
            int dis = 0;
            for (int e = e0; e < e1; ++e) {
                const int p = __ldg(grp_pair + e);
                const int j = __ldg(pairs + 2 * p), l = __ldg(pairs + 2 * p + 1);
                dis += (int)(((w[j >> 6] >> (j & 63)) ^ (w[l >> 6] >> (l & 63))) & 1ull);
            }
            v = (e1 - e0) - 2 * dis;
        }
        O[((size_t)t * P + k) * ns + x] = (int16_t)v;
    }
}

// Upper tiles I <= J (64 x 64) of G[t] = sum_x O_k(x) O_l(x) in int64: per chunk of 64 samples
// the products (|O| <= 256) are summed exactly in int32, then added to int64.  Thread (ty, tx)
// owns rows 4 ty .. 4 ty + 3 and columns 4 tx .. 4 tx + 3; the chunks sit in shared memory
// transposed (sample-major), so that a thread's four rows are one 8-byte load.
__global__ void __launch_bounds__(256) gram_int_kernel(int P, int ns, const int16_t* __restrict__ O,
                                                       long long* __restrict__ G) {
    const int t = blockIdx.y;
    int J = (int)((sqrtf(8.f * (float)blockIdx.x + 1.f) - 1.f) * 0.5f);
    while ((J + 1) * (J + 2) / 2 <= (int)blockIdx.x) ++J;
    while (J * (J + 1) / 2 > (int)blockIdx.x) --J;
    const int I = blockIdx.x - J * (J + 1) / 2;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    __shared__ __align__(16) int16_t As[GK][GT + 4];
    __shared__ __align__(16) int16_t Bs[GK][GT + 4];
    const int16_t* Ot = O + (size_t)t * P * ns;
    const int r0 = I * GT, c0 = J * GT;
    long long acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    for (int x0 = 0; x0 < ns; x0 += GK) {
        __syncthreads();
        for (int e = tid; e < GT * GK; e += 256) {
            const int r = e / GK, xs = e - r * GK, x = x0 + xs;
            As[xs][r] = (r0 + r < P && x < ns) ? Ot[(size_t)(r0 + r) * ns + x] : (int16_t)0;
            Bs[xs][r] = (c0 + r < P && x < ns) ? Ot[(size_t)(c0 + r) * ns + x] : (int16_t)0;
        }
        __syncthreads();
        int s[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) s[a][b] = 0;
#pragma unroll 8
        for (int xs = 0; xs < GK; ++xs) {
            const short4 av = *reinterpret_cast<const short4*>(&As[xs][4 * ty]);
            const short4 bv = *reinterpret_cast<const short4*>(&Bs[xs][4 * tx]);
            const int ar[4] = {av.x, av.y, av.z, av.w}, bc[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) s[a][b] += ar[a] * bc[b];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] += s[a][b];
    }
    long long* Gt = G + (size_t)t * P * P;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = r0 + 4 * ty + a;
        if (i >= P) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int j = c0 + 4 * tx + b;
            if (j < P && j >= i) Gt[(size_t)i * P + j] = acc[a][b];
        }
    }
}

// S[t] full symmetric FP64: S_ij = G_ij / ns - obar_i obar_j (G upper triangle)
__global__ void S_kernel(int P, int ns, const long long* __restrict__ G, const double* __restrict__ obar,
                         double* __restrict__ S) {
    const int t = blockIdx.y;
    const double inv = 1.0 / ns;
    const long long* Gt = G + (size_t)t * P * P;
    const double* ob = obar + (size_t)t * P;
    double* St = S + (size_t)t * P * P;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)P * P;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / P), j = (int)(e - (size_t)i * P);
        const long long g = i <= j ? Gt[(size_t)i * P + j] : Gt[(size_t)j * P + i];
        St[e] = (double)g * inv - ob[i] * ob[j];
    }
}

static size_t rup(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace lj

cudaError_t launch_lj_expand(const otvmc_ansatz* a, int ntraj, const double2* theta, double2* theta_full,
                             cudaStream_t s) {
    const int Pf = (int)a->full->P;
    ProfScope prof_(OTVMC_K_PREP, s);
    lj::expand_kernel<<<dim3((Pf + 255) / 256, ntraj), 256, 0, s>>>(a->n, (int)a->P, Pf, a->pair_grp_d, theta,
                                                                     theta_full);
    count_launch();
    return cudaGetLastError();
}

size_t lj_build_bytes(const otvmc_ansatz* a, int ntraj, int ns) {
    using lj::rup;
    const size_t T = (size_t)ntraj, P = (size_t)a->P, Pf = (size_t)a->full->P;
    return rup(T * Pf * 8) + rup(T * Pf * 16) + rup(T * P * ns * 2) + rup(T * P * P * 8) + 256;
}

const int16_t* lj_built_O(const otvmc_ansatz* a, int ntraj, const void* ws) {
    using lj::rup;
    const size_t T = (size_t)ntraj, Pf = (size_t)a->full->P;
    return (const int16_t*)((const char*)ws + rup(T * Pf * 8) + rup(T * Pf * 16));
}

// S (full FP64), obar and D of the tied parameters from the samples and the quantised v in b
// (vpart / vquant already run on b): D and obar of the full Jastrow by the exact integer sums,
// folded over the groups; S from the exact integer Gram matrix of the tied O.
cudaError_t launch_lj_build(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, const EvalBufs& b,
                            void* ws, double* S, double* obar, double2* D, cudaStream_t s) {
    using lj::rup;
    const otvmc_ansatz* f = a->full;
    const int n = a->n, P = (int)a->P, Pf = (int)f->P, W = (n + 63) / 64;
    char* q = (char*)ws;
    auto take = [&](size_t bytes) {
        char* r = q;
        q += rup(bytes);
        return (void*)r;
    };
    double* obar_f = (double*)take((size_t)ntraj * Pf * 8);
    double2* D_f = (double2*)take((size_t)ntraj * Pf * 16);
    int16_t* O = (int16_t*)take((size_t)ntraj * P * ns * 2);
    long long* G = (long long*)take((size_t)ntraj * P * P * 8);
    cudaError_t e = launch_D_fixed_jastrow(f, spins, ntraj, ns, b, obar_f, D_f, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof_(OTVMC_K_D, s);
        lj::fold_kernel<<<dim3((P + 255) / 256, ntraj), 256, 0, s>>>(n, P, Pf, a->grp_off_d, a->grp_pair_d, obar_f,
                                                                     D_f, obar, D);
        count_launch();
    }
    {
        ProfScope prof_(OTVMC_K_OBUILD, s);
        lj::obuild_kernel<<<dim3((ns + 255) / 256, (P + 15) / 16, ntraj), 256, 0, s>>>(
            n, W, P, ns, a->grp_off_d, a->grp_pair_d, f->pairs_d, spins, O);
        count_launch();
    }
    {
        ProfScope prof_(OTVMC_K_GRAM, s);
        const int nt = (P + lj::GT - 1) / lj::GT;
        lj::gram_int_kernel<<<dim3(nt * (nt + 1) / 2, ntraj), 256, 0, s>>>(P, ns, O, G);
        lj::S_kernel<<<dim3(256, ntraj), 256, 0, s>>>(P, ns, G, obar, S);
        count_launch(2);
    }
    return cudaGetLastError();
}

}  // namespace otvmc
