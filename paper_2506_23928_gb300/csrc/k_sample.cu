// Metropolis sampling of |psi_theta(x)|^2 for the long-range Jastrow ansatz (Eq. 12),
// one thread per Markov chain (otVMC procedure paragraph: configurations are drawn by the
// Metropolis algorithm from the normalised |psi|^2).
//
// Proposal p of a chain flips the site drawn from Philox; it is accepted iff
// u < |psi(x')/psi(x)|^2 = exp(ell), ell = -4 sigma_j Re f_j, f_j = a_j + sum_k eta_jk sigma_k.
// Each thread keeps Re f of its chain in FP32 in shared memory (initialised from scratch
// every call, updated on accepted flips).  With u = 2^-24 the FP32 value differs from the exact field by at most
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

// One thread per chain.  Shared memory: fields f[k][thread] (k-major, so a thread's own
// entries fall in distinct banks), Re eta [j][k] with a row stride of 1 mod 32 words, Re a,
// and the row bounds R.
__global__ void __launch_bounds__(256) sample_jastrow_kernel(const double2* __restrict__ theta, int P, int n, int W,
                                                             int ns, int n_sweep, int stride, uint32_t k0, uint32_t k1,
                                                             uint32_t evtag, int traj0, uint64_t* __restrict__ spins,
                                                             unsigned long long* __restrict__ accepted) {
    extern __shared__ float sm[];
    const int t = blockIdx.y;
    const int TPB = blockDim.x;
    const double2* th = theta + (size_t)t * P;
    float* f = sm;                   // [n][TPB]
    float* eta = f + n * TPB;        // [n][stride]
    float* a = eta + n * stride;     // [n]
    float* R = a + n;                // [n]
    for (int idx = threadIdx.x; idx < n * n; idx += TPB) {
        const int j = idx / n, k = idx - j * n;
        float v = 0.f;
        if (j != k) v = (float)th[n + pair_index(min(j, k), max(j, k), n)].x;
        eta[j * stride + k] = v;
    }
    for (int j = threadIdx.x; j < n; j += TPB) {
        a[j] = (float)th[j].x;
        double r = fabs(th[j].x);
        for (int k = 0; k < n; ++k)
            if (k != j) r += fabs(th[n + pair_index(min(j, k), max(j, k), n)].x);
        R[j] = (float)(r * (1.0 + 1e-6)) + 1e-30f;
    }
    __syncthreads();

    const int chain = blockIdx.x * TPB + threadIdx.x;
    if (chain >= ns) return;
    float* fm = f + threadIdx.x;  // fm[k * TPB]
    uint64_t wd[4];
    uint64_t* sp = spins + ((size_t)t * ns + chain) * W;
#pragma unroll
    for (int w = 0; w < 4; ++w) wd[w] = (w < W) ? sp[w] : 0ull;

    // fields from scratch: f_k = a_k + sum_i eta_ki sigma_i (eta rows read in lockstep: broadcast)
    for (int k = 0; k < n; ++k) fm[k * TPB] = a[k];
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        if (w >= W) break;
        const uint64_t word = wd[w];
        const int iend = min(64, n - 64 * w);
        for (int b = 0; b < iend; ++b) {
            const float sg = ((word >> b) & 1ull) ? 1.f : -1.f;
            const float* er = eta + (64 * w + b) * stride;
            for (int k = 0; k < n; ++k) fm[k * TPB] = fmaf(sg, er[k], fm[k * TPB]);
        }
    }

    const int nprop = n_sweep * n;
    const float ulp = 5.9604645e-8f;  // 2^-24
    int m = 0;
    u32x4 draw = {0u, 0u, 0u, 0u};
    for (int p = 0; p < nprop; ++p) {
        if ((p & 1) == 0) draw = philox(u32x4{(uint32_t)(p / 2), (uint32_t)chain, (uint32_t)(traj0 + t), evtag}, k0, k1);
        const uint32_t wsite = (p & 1) ? draw.z : draw.x;
        const uint32_t wu = (p & 1) ? draw.w : draw.y;
        const int j = (int)(((unsigned long long)wsite * (unsigned long long)n) >> 32);
        const int sj = spin_sel(wd, j);
        const float fj = fm[j * TPB];
        // u = (wu + 1/2) 2^-32 in FP32 (relative error <= 2^-24, inside the guard band below)
        const float lu = logf(fmaf((float)wu, 0x1.0p-32f, 0x1.0p-33f));
        const float l32 = -4.f * (float)sj * fj;
        const float guard = 4.f * (float)(n + 3 + m) * ulp * R[j] * 1.01f + 1e-6f + 4e-7f * fabsf(lu);
        const float d = l32 - lu;
        bool acc;
        if (d > guard) {
            acc = true;
        } else if (d < -guard) {
            acc = false;
        } else {
            double part = 0.0;
            for (int k = 0; k < n; ++k)
                if (k != j) part += th[n + pair_index(min(j, k), max(j, k), n)].x * (double)spin_sel(wd, k);
            const double ell = -4.0 * (double)sj * (th[j].x + part);
            acc = u01(wu) < exp(ell);
        }
        if (acc) {
            const float c = -2.f * (float)sj;
            const float* er = eta + j * stride;
            for (int k = 0; k < n; ++k) fm[k * TPB] = fmaf(c, er[k], fm[k * TPB]);
            flip_sel(wd, j);
            ++m;
        }
    }
#pragma unroll
    for (int w = 0; w < 4; ++w)
        if (w < W) sp[w] = wd[w];
    if (accepted != nullptr && m) atomicAdd(accepted + t, (unsigned long long)m);
}

// Chains of at most NF <= 64 sites (one spin word): the same arithmetic as the kernel above
// (identical FMA order, so identical fields and decisions) with the chain's fields in
// registers.  The from-scratch sum reads each row of Re eta once for all threads (a
// broadcast); an accepted flip reads the flipped site's row (row stride NF + 1, so lanes on
// different rows meet at most two to a bank); the field of the proposed site is picked from
// the registers by a select tree on the bits of j.
template <int NF>
__device__ __forceinline__ float pick_field(const float (&f)[NF], int j) {
    float v[NF / 2];
#pragma unroll
    for (int i = 0; i < NF / 2; ++i) v[i] = (j & (NF / 2)) ? f[i + NF / 2] : f[i];
#pragma unroll
    for (int h = NF / 4; h >= 1; h >>= 1)
#pragma unroll
        for (int i = 0; i < h; ++i) v[i] = (j & h) ? v[i + h] : v[i];
    return v[0];
}

template <int NF>
__global__ void __launch_bounds__(256) sample_jastrow_reg_kernel(const double2* __restrict__ theta, int P, int n,
                                                                 int ns, int n_sweep, uint32_t k0, uint32_t k1,
                                                                 uint32_t evtag, int traj0,
                                                                 uint64_t* __restrict__ spins,
                                                                 unsigned long long* __restrict__ accepted) {
    constexpr int ST = NF + 1;
    __shared__ float eta[NF * ST];
    __shared__ float a[NF], R[NF];
    const int t = blockIdx.y;
    const double2* th = theta + (size_t)t * P;
    for (int idx = threadIdx.x; idx < NF * NF; idx += blockDim.x) {
        const int j = idx / NF, k = idx - j * NF;
        float v = 0.f;
        if (j < n && k < n && j != k) v = (float)th[n + pair_index(min(j, k), max(j, k), n)].x;
        eta[j * ST + k] = v;
    }
    for (int j = threadIdx.x; j < NF; j += blockDim.x) {
        if (j < n) {
            a[j] = (float)th[j].x;
            double r = fabs(th[j].x);
            for (int k = 0; k < n; ++k)
                if (k != j) r += fabs(th[n + pair_index(min(j, k), max(j, k), n)].x);
            R[j] = (float)(r * (1.0 + 1e-6)) + 1e-30f;
        } else {
            a[j] = 0.f;
            R[j] = 1e-30f;
        }
    }
    __syncthreads();

    const int chain = blockIdx.x * blockDim.x + threadIdx.x;
    if (chain >= ns) return;
    uint64_t* sp = spins + (size_t)t * ns + chain;
    uint64_t wd = *sp;
    float f[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) f[k] = a[k];
    for (int i = 0; i < n; ++i) {
        const float sg = ((wd >> i) & 1ull) ? 1.f : -1.f;
        const float* er = eta + i * ST;
#pragma unroll
        for (int k = 0; k < NF; ++k) f[k] = fmaf(sg, er[k], f[k]);
    }

    const int nprop = n_sweep * n;
    const float ulp = 5.9604645e-8f;  // 2^-24
    int m = 0;
    u32x4 draw = {0u, 0u, 0u, 0u};
    for (int p = 0; p < nprop; ++p) {
        if ((p & 1) == 0) draw = philox(u32x4{(uint32_t)(p / 2), (uint32_t)chain, (uint32_t)(traj0 + t), evtag}, k0, k1);
        const uint32_t wsite = (p & 1) ? draw.z : draw.x;
        const uint32_t wu = (p & 1) ? draw.w : draw.y;
        const int j = (int)(((unsigned long long)wsite * (unsigned long long)n) >> 32);
        const int sj = ((wd >> j) & 1ull) ? 1 : -1;
        const float fj = pick_field<NF>(f, j);
        // u = (wu + 1/2) 2^-32 in FP32 (relative error <= 2^-24, inside the guard band below)
        const float lu = logf(fmaf((float)wu, 0x1.0p-32f, 0x1.0p-33f));
        const float l32 = -4.f * (float)sj * fj;
        const float guard = 4.f * (float)(n + 3 + m) * ulp * R[j] * 1.01f + 1e-6f + 4e-7f * fabsf(lu);
        const float d = l32 - lu;
        bool acc;
        if (d > guard) {
            acc = true;
        } else if (d < -guard) {
            acc = false;
        } else {
            double part = 0.0;
            for (int k = 0; k < n; ++k)
                if (k != j) part += th[n + pair_index(min(j, k), max(j, k), n)].x * (((wd >> k) & 1ull) ? 1.0 : -1.0);
            const double ell = -4.0 * (double)sj * (th[j].x + part);
            acc = u01(wu) < exp(ell);
        }
        if (acc) {
            const float c = -2.f * (float)sj;
            const float* er = eta + j * ST;
#pragma unroll
            for (int k = 0; k < NF; ++k) f[k] = fmaf(c, er[k], f[k]);
            wd ^= 1ull << j;
            ++m;
        }
    }
    *sp = wd;
    if (accepted != nullptr && m) atomicAdd(accepted + t, (unsigned long long)m);
}

cudaError_t launch_sample_jastrow(const otvmc_ansatz* an, const double2* theta, int ntraj, int traj0, int ns,
                                  int n_sweep, uint64_t seed, int64_t eval, uint64_t* spins,
                                  unsigned long long* accepted, int* status, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SAMPLE, s);
    (void)status;
    const int n = an->n, W = (n + 63) / 64;
    const uint32_t evtag = (TAG_SAMPLE << 28) | ((uint32_t)eval & 0x0FFFFFFFu);
    if (n <= 64) {
        dim3 grid((ns + 255) / 256, ntraj);
        if (n <= 32)
            sample_jastrow_reg_kernel<32><<<grid, 256, 0, s>>>(theta, (int)an->P, n, ns, n_sweep, (uint32_t)seed,
                                                               (uint32_t)(seed >> 32), evtag, traj0, spins, accepted);
        else
            sample_jastrow_reg_kernel<64><<<grid, 256, 0, s>>>(theta, (int)an->P, n, ns, n_sweep, (uint32_t)seed,
                                                               (uint32_t)(seed >> 32), evtag, traj0, spins, accepted);
        count_launch();
        return cudaGetLastError();
    }
    const int stride = ((n + 31) / 32) * 32 + 1;
    const size_t fixed = ((size_t)n * stride + 2 * n) * sizeof(float);
    const size_t budget = 200 * 1024;
    int tpb = 256;
    while (tpb > 32 && fixed + (size_t)n * tpb * sizeof(float) > budget) tpb -= 32;
    const size_t smem = fixed + (size_t)n * tpb * sizeof(float);
    if (smem > budget) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(sample_jastrow_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((ns + tpb - 1) / tpb, ntraj);
    sample_jastrow_kernel<<<grid, tpb, smem, s>>>(theta, (int)an->P, n, W, ns, n_sweep, stride, (uint32_t)seed,
                                                  (uint32_t)(seed >> 32), evtag, traj0, spins, accepted);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
