// SNR-regularised solve in the eigenbasis of S (otVMC procedure paragraph, the
// regularisation of the cited signal-to-noise filter), for the Jastrow ansatz and small P.
//
// S = V diag(lambda) V^T (real symmetric for Jastrow), rho = V^T D.  The per-sample
// contributions Q_k(x) = (V^T O_c(x))_k v_c(x) average to rho_k; their spread gives
// SNR_k = |rho_k| / sqrt(Var_x Q_k / ns).  Each inverse eigenvalue is damped by
//     f_k = 1 / (1 + (thr / SNR_k)^6) * 1 / (1 + (eps_svd lambda_max / lambda_k)^6)
// and delta = V diag(f_k / lambda_k) rho (lambda_k <= 0 dropped).  The filter's shape is a
// reading of the cited regulariser; as the thresholds go to zero it is the plain
// pseudo-inverse.
//
// One CTA per trajectory, everything in FP64 in shared memory: cyclic Jacobi with the
// round-robin ordering (P/2 disjoint rotations per round, all applied at once), then two
// passes over the samples for the mean and the variance of Q.
#include "common.cuh"

namespace otvmc {

constexpr int SNR_THREADS = 256;
constexpr int SNR_SWEEPS = 40;  // bound on Jacobi sweeps (quadratic convergence: ~10 needed)

__device__ __forceinline__ void rr_pair(int m, int r, int k, int& p, int& q) {
    // circle method over m (even) indices: index m-1 fixed, the others rotate
    if (k == 0) {
        p = m - 1;
        q = r;
    } else {
        p = (r + k) % (m - 1);
        q = (r - k + (m - 1)) % (m - 1);
    }
}

// Jastrow O_k(x) - obar_k: k < n single sigma_j, else the pair (j, l) of pair index k - n, or
// (tied Jastrow, grp_off given) the sum of sigma_j sigma_l over the pairs of group k - n.
__device__ __forceinline__ double oc_val(const uint64_t* w, const int* pairs, const int* grp_off,
                                         const int* grp_pair, int n, int k, const double* ob) {
    if (k < n) return (double)spin_of(w, k) - ob[k];
    if (grp_off == nullptr) {
        const int j = pairs[2 * (k - n)], l = pairs[2 * (k - n) + 1];
        return (double)(spin_of(w, j) * spin_of(w, l)) - ob[k];
    }
    int sum = 0;
    for (int e = grp_off[k - n]; e < grp_off[k - n + 1]; ++e) {
        const int p = grp_pair[e];
        sum += spin_of(w, pairs[2 * p]) * spin_of(w, pairs[2 * p + 1]);
    }
    return (double)sum - ob[k];
}

__global__ void __launch_bounds__(SNR_THREADS) snr_solve_kernel(int n, int W, int P, int ns,
                                                                const uint64_t* __restrict__ spins,
                                                                const int* __restrict__ pairs,
                                                                const int* __restrict__ grp_off,
                                                                const int* __restrict__ grp_pair,
                                                                const double* __restrict__ S,
                                                                const double* __restrict__ obar,
                                                                const double2* __restrict__ v,
                                                                const double2* __restrict__ D, double thr,
                                                                double eps_svd, double2* __restrict__ delta,
                                                                double* __restrict__ lam_out, int* status) {
    extern __shared__ __align__(16) double snr_sm[];
    const int t = blockIdx.x, tid = threadIdx.x;
    const int LDA = P + 1;
    const int m = (P + 1) & ~1;          // even number of indices (one dummy when P is odd)
    double* A = snr_sm;                  // [P][P+1]
    double* V = A + P * LDA;             // [P][P+1]
    double* cs = V + P * LDA;            // [m/2][2] rotation (c, s)
    double2* rho = (double2*)(cs + m);   // [P]
    double2* qm = rho + P;               // [P] mean of Q
    double* var = (double*)(qm + P);     // [P]
    double* ob = var + P;                // [P]
    double2* part = (double2*)(ob + P);  // [SNR_THREADS] partial sums (samples split over groups)
    __shared__ double red[SNR_THREADS / 32];
    __shared__ double2 vbar_s;
    __shared__ int done_s;
    const double* St = S + (size_t)t * P * P;
    for (int e = tid; e < P * P; e += blockDim.x) {
        const int i = e / P, j = e - i * P;
        A[i * LDA + j] = St[e];
        V[i * LDA + j] = i == j ? 1.0 : 0.0;
    }
    for (int k = tid; k < P; k += blockDim.x) ob[k] = obar[(size_t)t * P + k];
    __syncthreads();

    // ---- Jacobi
    int sweep = 0;
    for (; sweep < SNR_SWEEPS; ++sweep) {
        // convergence: max |A_pq| (p != q) against max |A_pp|
        double off = 0.0, dg = 0.0;
        for (int e = tid; e < P * P; e += blockDim.x) {
            const int i = e / P, j = e - i * P;
            const double a = fabs(A[i * LDA + j]);
            if (i == j) dg = fmax(dg, a);
            else off = fmax(off, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
            off = fmax(off, __shfl_xor_sync(0xffffffffu, off, o));
            dg = fmax(dg, __shfl_xor_sync(0xffffffffu, dg, o));
        }
        if ((tid & 31) == 0) red[tid >> 5] = off;
        __syncthreads();
        if (tid == 0) {
            double mo = 0.0;
            for (int w = 0; w < SNR_THREADS / 32; ++w) mo = fmax(mo, red[w]);
            red[0] = mo;
        }
        __syncthreads();
        const double mo = red[0];
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = dg;
        __syncthreads();
        if (tid == 0) {
            double md = 0.0;
            for (int w = 0; w < SNR_THREADS / 32; ++w) md = fmax(md, red[w]);
            done_s = !(mo > 1e-15 * md);
        }
        __syncthreads();
        if (done_s) break;
        for (int r = 0; r < m - 1; ++r) {
            for (int k = tid; k < m / 2; k += blockDim.x) {
                int p, q;
                rr_pair(m, r, k, p, q);
                double c = 1.0, s = 0.0;
                if (p < P && q < P) {
                    const double apq = A[p * LDA + q];
                    if (apq != 0.0) {
                        const double tau = (A[q * LDA + q] - A[p * LDA + p]) / (2.0 * apq);
                        const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + tt * tt);
                        s = tt * c;
                    }
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = s;
            }
            __syncthreads();
            // rows: A <- J^T A (rows p, q of each pair)
            for (int e = tid; e < (m / 2) * P; e += blockDim.x) {
                const int k = e / P, j = e - k * P;
                int p, q;
                rr_pair(m, r, k, p, q);
                if (p >= P || q >= P) continue;
                const double c = cs[2 * k], s = cs[2 * k + 1];
                const double ap = A[p * LDA + j], aq = A[q * LDA + j];
                A[p * LDA + j] = c * ap - s * aq;
                A[q * LDA + j] = s * ap + c * aq;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = tid; e < (m / 2) * P; e += blockDim.x) {
                const int k = e / P, i = e - k * P;
                int p, q;
                rr_pair(m, r, k, p, q);
                if (p >= P || q >= P) continue;
                const double c = cs[2 * k], s = cs[2 * k + 1];
                const double ap = A[i * LDA + p], aq = A[i * LDA + q];
                A[i * LDA + p] = c * ap - s * aq;
                A[i * LDA + q] = s * ap + c * aq;
                const double vp = V[i * LDA + p], vq = V[i * LDA + q];
                V[i * LDA + p] = c * vp - s * vq;
                V[i * LDA + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    if (tid == 0 && sweep == SNR_SWEEPS) record_error(status, OTVMC_ERR_NONFINITE, t);

    // ---- rho = V^T D, vbar
    const double2* Dt = D + (size_t)t * P;
    for (int k = tid; k < P; k += blockDim.x) {
        double2 a = make_double2(0.0, 0.0);
        for (int i = 0; i < P; ++i) {
            const double vik = V[i * LDA + k];
            a.x += vik * Dt[i].x;
            a.y += vik * Dt[i].y;
        }
        rho[k] = a;
    }
    const double2* vt = v + (size_t)t * ns;
    {
        double2 a = make_double2(0.0, 0.0);
        for (int x = tid; x < ns; x += blockDim.x) {
            a.x += vt[x].x;
            a.y += vt[x].y;
        }
        part[tid] = a;
        __syncthreads();
        if (tid == 0) {
            double2 s = make_double2(0.0, 0.0);
            for (int i = 0; i < SNR_THREADS; ++i) {
                s.x += part[i].x;
                s.y += part[i].y;
            }
            vbar_s = make_double2(s.x / ns, s.y / ns);
        }
        __syncthreads();
    }
    const double2 vbar = vbar_s;

    // ---- two passes over the samples: thread (k, g) takes samples g, g + G, ...
    const int G = blockDim.x / P;  // sample groups (P <= blockDim.x)
    const int k = tid % P, g = tid / P;
    const uint64_t* sp = spins + (size_t)t * ns * W;
    for (int pass = 0; pass < 2; ++pass) {
        double2 acc = make_double2(0.0, 0.0);
        double accv = 0.0;
        if (g < G) {
            for (int x = g; x < ns; x += G) {
                const uint64_t* w = sp + (size_t)x * W;
                double y = 0.0;
                for (int i = 0; i < P; ++i) y += oc_val(w, pairs, grp_off, grp_pair, n, i, ob) * V[i * LDA + k];
                const double2 vc = make_double2(vt[x].x - vbar.x, vt[x].y - vbar.y);
                const double2 qv = make_double2(y * vc.x, y * vc.y);
                if (pass == 0) {
                    acc.x += qv.x;
                    acc.y += qv.y;
                } else {
                    const double dx = qv.x - qm[k].x, dy = qv.y - qm[k].y;
                    accv += dx * dx + dy * dy;
                }
            }
        }
        part[tid] = pass == 0 ? acc : make_double2(accv, 0.0);
        __syncthreads();
        if (tid < P) {
            double2 s = make_double2(0.0, 0.0);
            for (int gg = 0; gg < G; ++gg) {
                s.x += part[gg * P + tid].x;
                s.y += part[gg * P + tid].y;
            }
            if (pass == 0) qm[tid] = make_double2(s.x / ns, s.y / ns);
            else var[tid] = s.x / ns;
        }
        __syncthreads();
    }

    // ---- filter and back-transform
    if (tid == 0) {
        double lm = -INFINITY;
        for (int i = 0; i < P; ++i) lm = fmax(lm, A[i * LDA + i]);
        red[0] = lm;
    }
    __syncthreads();
    const double lam_max = red[0];
    for (int kk = tid; kk < P; kk += blockDim.x) {
        const double lam = A[kk * LDA + kk];
        const double snr = sqrt(rho[kk].x * rho[kk].x + rho[kk].y * rho[kk].y) / sqrt(var[kk] / ns + 1e-300);
        const double f_snr = 1.0 / (1.0 + pow(thr / snr, 6.0));
        const double f_svd = 1.0 / (1.0 + pow(eps_svd * lam_max / fmax(lam, 1e-300), 6.0));
        const double inv = lam > 0.0 ? f_snr * f_svd / fmax(lam, 1e-300) : 0.0;
        qm[kk] = make_double2(inv * rho[kk].x, inv * rho[kk].y);  // reuse: filtered coefficients
        if (lam_out) lam_out[(size_t)t * P + kk] = lam;
    }
    __syncthreads();
    for (int i = tid; i < P; i += blockDim.x) {
        double2 a = make_double2(0.0, 0.0);
        for (int kk = 0; kk < P; ++kk) {
            const double vik = V[i * LDA + kk];
            a.x += vik * qm[kk].x;
            a.y += vik * qm[kk].y;
        }
        delta[(size_t)t * P + i] = a;
    }
}

size_t snr_smem_bytes(int P) {
    const int m = (P + 1) & ~1;
    return (size_t)(2 * P * (P + 1) + m + 2 * P + 2 * P + 2 * P) * sizeof(double) + SNR_THREADS * 16 + 64;
}

cudaError_t launch_snr_solve(const otvmc_ansatz* a, int ntraj, int ns, const uint64_t* spins, const double* S,
                             const double* obar, const double2* v, const double2* D, double thr, double eps_svd,
                             double2* delta, double* lam, int* status, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_SOLVE, s);
    const int P = (int)a->P, n = a->n, W = (n + 63) / 64;
    const size_t smem = snr_smem_bytes(P);
    cudaError_t e = cudaFuncSetAttribute(snr_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const bool tied = a->kind == OTVMC_LJ;
    snr_solve_kernel<<<ntraj, SNR_THREADS, smem, s>>>(n, W, P, ns, spins, tied ? a->full->pairs_d : a->pairs_d,
                                                      tied ? a->grp_off_d : nullptr, tied ? a->grp_pair_d : nullptr,
                                                      S, obar, v, D, thr, eps_svd, delta, lam, status);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
