// Metropolis sampling of |psi_theta(x)|^2 for the long-range Jastrow ansatz (Eq. 12),
// one group of G lanes per Markov chain (otVMC procedure paragraph: configurations are
// drawn by the Metropolis algorithm from the normalised |psi|^2).
//
// Proposal p of a chain flips the site drawn from Philox; it is accepted iff
// u < |psi(x')/psi(x)|^2 = exp(ell), ell = -4 sigma_j Re f_j, f_j = a_j + sum_k eta_jk sigma_k.
// The lanes keep Re f in FP32 registers (initialised from scratch every call, updated on
// accepted flips).  With u = 2^-24 the FP32 value differs from the exact field by at most
// (N + 2 + m) u R_j, R_j = |Re a_j| + sum_k |Re eta_jk|, m = flips accepted so far, so a
// guard band of four times that bound (plus the error of logf) decides every proposal as
// FP64 would; proposals inside the band recompute ell in FP64 from theta.
#include "common.cuh"

namespace otvmc {

__host__ __device__ __forceinline__ int pair_index(int lo, int hi, int n) {
    return lo * n - lo * (lo + 1) / 2 + (hi - lo - 1);
}

__device__ __forceinline__ uint64_t word_sel(const uint64_t (&wd)[4], int w) {
    uint64_t r = wd[0];
    if (w == 1) r = wd[1];
    if (w == 2) r = wd[2];
    if (w == 3) r = wd[3];
    return r;
}
__device__ __forceinline__ int spin_sel(const uint64_t (&wd)[4], int j) {
    return ((word_sel(wd, j >> 6) >> (j & 63)) & 1ull) ? 1 : -1;
}
__device__ __forceinline__ void flip_sel(uint64_t (&wd)[4], int j) {
    const uint64_t m = 1ull << (j & 63);
    const int w = j >> 6;
    if (w == 0) wd[0] ^= m;
    if (w == 1) wd[1] ^= m;
    if (w == 2) wd[2] ^= m;
    if (w == 3) wd[3] ^= m;
}

template <int G, int MAXS>
__global__ void __launch_bounds__(256) sample_jastrow_kernel(
    const double2* __restrict__ theta, int P, int n, int W, int ns, int n_sweep, int chains_per_group,
    uint32_t k0, uint32_t k1, uint32_t evtag, int traj0, uint64_t* __restrict__ spins,
    unsigned long long* __restrict__ accepted) {
    extern __shared__ float sm[];
    const int t = blockIdx.y;
    const double2* th = theta + (size_t)t * P;
    float* eta = sm;         // [n][n] Re eta, symmetric, zero diagonal
    float* a = eta + n * n;  // [n]   Re a
    float* R = a + n;        // [n]   |Re a_j| + sum_k |Re eta_jk| (rounded up)
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int j = idx / n, k = idx - j * n;
        float v = 0.f;
        if (j != k) v = (float)th[n + pair_index(min(j, k), max(j, k), n)].x;
        eta[idx] = v;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        a[j] = (float)th[j].x;
        double r = fabs(th[j].x);
        for (int k = 0; k < n; ++k)
            if (k != j) r += fabs(th[n + pair_index(min(j, k), max(j, k), n)].x);
        R[j] = (float)(r * (1.0 + 1e-6)) + 1e-30f;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((lane / G) * G));
    const int groups_per_block = blockDim.x / G;
    const int group = threadIdx.x / G;
    const int nslots = (n + G - 1) / G;
    const int nprop = n_sweep * n;
    const float ulp = 5.9604645e-8f;  // 2^-24
    unsigned long long acc_total = 0;

    for (int ci = 0; ci < chains_per_group; ++ci) {
        const int chain = (blockIdx.x * chains_per_group + ci) * groups_per_block + group;
        if (chain >= ns) continue;  // uniform over the group
        uint64_t wd[4];
        uint64_t* sp = spins + ((size_t)t * ns + chain) * W;
#pragma unroll
        for (int w = 0; w < 4; ++w) wd[w] = (w < W) ? sp[w] : 0ull;

        float f[MAXS];
#pragma unroll
        for (int s = 0; s < MAXS; ++s) {
            const int k = gl + s * G;
            f[s] = (s < nslots && k < n) ? a[k] : 0.f;
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            if (w >= W) break;
            const uint64_t word = wd[w];
            const int iend = min(64, n - 64 * w);
            for (int b = 0; b < iend; ++b) {
                const float sg = ((word >> b) & 1ull) ? 1.f : -1.f;
                const float* er = eta + (64 * w + b) * n;
#pragma unroll
                for (int s = 0; s < MAXS; ++s) {
                    const int k = gl + s * G;
                    if (s < nslots && k < n) f[s] = fmaf(sg, er[k], f[s]);
                }
            }
        }

        int m = 0;
        u32x4 cache = {0u, 0u, 0u, 0u};
        for (int p = 0; p < nprop; ++p) {
            if ((p % (2 * G)) == 0)
                cache = philox(u32x4{(uint32_t)(p / 2 + gl), (uint32_t)chain, (uint32_t)(traj0 + t), evtag}, k0, k1);
            const int srcl = (p / 2) % G;
            const bool hi = (p & 1) != 0;
            const uint32_t wsite = __shfl_sync(gmask, hi ? cache.z : cache.x, srcl, G);
            const uint32_t wu = __shfl_sync(gmask, hi ? cache.w : cache.y, srcl, G);
            const int j = (int)(((unsigned long long)wsite * (unsigned long long)n) >> 32);
            const int owner = j % G, slot = j / G;
            float mine = f[0];
#pragma unroll
            for (int s = 1; s < MAXS; ++s)
                if (s == slot) mine = f[s];
            const float fj = __shfl_sync(gmask, mine, owner, G);
            const int sj = spin_sel(wd, j);
            const double u = u01(wu);
            const float l32 = -4.f * (float)sj * fj;
            const float lu = logf((float)u);
            const float guard = 4.f * (float)(n + 3 + m) * ulp * R[j] * 1.01f + 1e-6f + 4e-7f * fabsf(lu);
            const float d = l32 - lu;
            bool acc;
            if (d > guard) {
                acc = true;
            } else if (d < -guard) {
                acc = false;
            } else {
                double part = 0.0;
                for (int k = gl; k < n; k += G)
                    if (k != j) part += th[n + pair_index(min(j, k), max(j, k), n)].x * (double)spin_sel(wd, k);
#pragma unroll
                for (int off = G / 2; off > 0; off >>= 1) part += __shfl_xor_sync(gmask, part, off, G);
                const double ell = -4.0 * (double)sj * (th[j].x + part);
                acc = u < exp(ell);
            }
            if (acc) {
                const float c = -2.f * (float)sj;
                const float* er = eta + j * n;
#pragma unroll
                for (int s = 0; s < MAXS; ++s) {
                    const int k = gl + s * G;
                    if (s < nslots && k < n) f[s] = fmaf(c, er[k], f[s]);
                }
                flip_sel(wd, j);
                ++m;
            }
        }
        if (gl == 0) {
#pragma unroll
            for (int w = 0; w < 4; ++w)
                if (w < W) sp[w] = wd[w];
            acc_total += (unsigned long long)m;
        }
    }
    if (accepted != nullptr && gl == 0 && acc_total) atomicAdd(accepted + t, acc_total);
}

template <int G, int MAXS>
static cudaError_t launch_sample_g(const otvmc_ansatz* an, const double2* theta, int ntraj, int traj0, int ns,
                                   int n_sweep, uint64_t seed, int64_t eval, uint64_t* spins,
                                   unsigned long long* accepted, cudaStream_t s) {
    const int n = an->n, W = (n + 63) / 64;
    const size_t smem = ((size_t)n * n + 2 * n) * sizeof(float);
    auto kern = sample_jastrow_kernel<G, MAXS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int cpg = 4;
    const int chains_per_block = cpg * (256 / G);
    dim3 grid((ns + chains_per_block - 1) / chains_per_block, ntraj);
    const uint32_t evtag = (TAG_SAMPLE << 28) | ((uint32_t)eval & 0x0FFFFFFFu);
    kern<<<grid, 256, smem, s>>>(theta, (int)an->P, n, W, ns, n_sweep, cpg, (uint32_t)seed, (uint32_t)(seed >> 32),
                                 evtag, traj0, spins, accepted);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sample_jastrow(const otvmc_ansatz* an, const double2* theta, int ntraj, int traj0, int ns,
                                  int n_sweep, uint64_t seed, int64_t eval, uint64_t* spins,
                                  unsigned long long* accepted, int* status, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SAMPLE, s);
    (void)status;
    const int n = an->n;
    if (n <= 8) return launch_sample_g<8, 1>(an, theta, ntraj, traj0, ns, n_sweep, seed, eval, spins, accepted, s);
    if (n <= 16) return launch_sample_g<16, 1>(an, theta, ntraj, traj0, ns, n_sweep, seed, eval, spins, accepted, s);
    return launch_sample_g<32, 8>(an, theta, ntraj, traj0, ns, n_sweep, seed, eval, spins, accepted, s);
}

}  // namespace otvmc
