// SNR-regularised solve in the eigenbasis of S (otVMC procedure paragraph) for P beyond the
// shared-memory Jacobi of k_snr.cu: the same filter,
//     S = V diag(lambda) V^T,  rho = V^T D,  Q_k(x) = (V^T O_c(x))_k v_c(x),
//     SNR_k = |rho_k| / sqrt(Var_x Q_k / ns),
//     f_k = 1 / (1 + (thr / SNR_k)^6) * 1 / (1 + (eps_svd lambda_max / lambda_k)^6),
//     delta = V diag(f_k / lambda_k) rho   (lambda_k <= 0 dropped),
// with the eigen-decomposition done by
//   (1) Householder tridiagonalisation of a copy A of S: T = Q^T A Q, Q = H_0 H_1 ... H_{P-3},
//       H_k = I - tau_k v_k v_k^T acting on indices k+1 .. P-1 (v_k kept in column k of A);
//   (2) Q^T formed explicitly, as X = H_{P-3}, then X <- X H_k for k = P-4 .. 0, each step
//       touching only the trailing block that H_k acts on;
//   (3) the implicit QL iteration with the shift from the leading 2 x 2 block on T (d, e),
//       every plane rotation applied to the rows of X, so that at the end row k of X is the
//       eigenvector of eigenvalue d_k (X = V^T); eigenvalues to an absolute accuracy of a few
//       eps ||S||, as a dense symmetric eigensolver gives them;
// then (4) rho and one pass over the samples for the mean and the second moment of Q_k, and
// (5) the filter and the back-projection.  One CTA per trajectory, FP64 throughout; A and X
// live in the caller's workspace (2 P^2 doubles per trajectory), d, e, the reflector and the
// rotations of a QL sweep in shared memory.  The scalar recurrence of a QL sweep runs on one
// thread; the sweep's rotations are then applied to all columns of X at once.
#include "common.cuh"

namespace otvmc {

constexpr int SNRB_THREADS = 256;
constexpr int SNRB_WARPS = SNRB_THREADS / 32;
constexpr int SNRB_MAX_ITER = 60;        // QL iterations per eigenvalue before giving up
constexpr int SNRB_SMEM_BUDGET = 216 * 1024;  // + the signs of a chunk of samples
constexpr int SNRB_SGN_BYTES = 16 * 200;          // 16 samples x N <= 200 sites

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Sum over the CTA (every thread calls it; red holds SNRB_WARPS doubles).
__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < SNRB_WARPS; ++i) s += red[i];
    return s;
}

// Samples per chunk of the sample pass, chosen so that the shared memory fits the budget.
__host__ __device__ inline int snrb_chunk(int P) {
    const int c = (SNRB_SMEM_BUDGET / 8 - 7 * P - 33) / P;
    return c > 16 ? 16 : c;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// One pass over the samples in chunks of CH held in shared memory (och): per eigenvector k
// (row k of V), the sums over x of Q_k(x) = y_k(x) v_c(x), y_k(x) = sum_i V_ki O_c,i(x), and of
// |Q_k(x)|^2, added to qs[k] and q2[k].  One warp per k; y in T, Q and the sums in FP64.
template <typename T>
__device__ void snrb_sample_pass(int n, int W, int P, int ns, const uint64_t* sp, const int* pairs,
                                 const int* grp_off, const int* grp_pair, const int16_t* Oint, const double* ob,
                                 const T* V, T* och, signed char* sgn, int CH, const double2* vt, double vbx,
                                 double vby, double2* qs, double* q2) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int x0 = 0; x0 < ns; x0 += CH) {
        const int nc = min(CH, ns - x0);
        if (Oint != nullptr) {
            // the log-derivatives already built as integers ([P][ns] of this trajectory)
            for (int q = tid; q < nc * P; q += blockDim.x) {
                const int i = q / nc, c = q % nc;
                och[(size_t)c * P + i] = (T)((double)Oint[(size_t)i * ns + x0 + c] - ob[i]);
            }
        } else {
            // the chunk's spins as signs in shared memory, then O - obar from them
            for (int q = tid; q < nc * n; q += blockDim.x) {
                const int c = q / n, j = q % n;
                sgn[c * n + j] = (signed char)spin_of(sp + (size_t)(x0 + c) * W, j);
            }
            __syncthreads();
            for (int q = tid; q < nc * P; q += blockDim.x) {
                const int c = q / P, i = q % P;
                const signed char* sg = sgn + c * n;
                int o;
                if (i < n) {
                    o = sg[i];
                } else if (grp_off == nullptr) {
                    o = sg[pairs[2 * (i - n)]] * sg[pairs[2 * (i - n) + 1]];
                } else {
                    o = 0;
                    for (int e = grp_off[i - n]; e < grp_off[i - n + 1]; ++e) {
                        const int pp = grp_pair[e];
                        o += sg[pairs[2 * pp]] * sg[pairs[2 * pp + 1]];
                    }
                }
                och[(size_t)c * P + i] = (T)((double)o - ob[i]);
            }
        }
        __syncthreads();
        for (int k = warp; k < P; k += SNRB_WARPS) {
            const T* Vk = V + (size_t)k * P;
            T y[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) y[c] = (T)0;
            for (int i = lane; i < P; i += 32) {
                const T vk = Vk[i];
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    if (c < nc) y[c] += vk * och[(size_t)c * P + i];
            }
            double ax = 0.0, ay = 0.0, a2 = 0.0;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                if (c >= nc) break;
                const double yc = (double)warp_sum_t(y[c]);
                const double vx = vt[x0 + c].x - vbx, vy = vt[x0 + c].y - vby;
                const double qx = yc * vx, qy = yc * vy;
                ax += qx;
                ay += qy;
                a2 += qx * qx + qy * qy;
            }
            if (lane == 0) {
                qs[k].x += ax;
                qs[k].y += ay;
                q2[k] += a2;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SNRB_THREADS, 1) snr_big_kernel(
    int n, int W, int P, int ns, const uint64_t* __restrict__ spins, const int* __restrict__ pairs,
    const int* __restrict__ grp_off, const int* __restrict__ grp_pair, const double* __restrict__ S,
    const double* __restrict__ obar, const double2* __restrict__ v, const double2* __restrict__ D, double thr,
    double eps_svd, double* __restrict__ Aws, double* __restrict__ Xws, double2* __restrict__ delta,
    double* __restrict__ lam_out, int* status, int fp32_pass, const int16_t* __restrict__ Oint) {
    const int t = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    extern __shared__ __align__(16) double sm[];
    double* d = sm;            // [P] diagonal, then the eigenvalues
    double* e = d + P;         // [P] subdiagonal (e[i] couples i and i + 1)
    double* tau = e + P;       // [P]
    double* vb = tau + P;      // [P] reflector
    double* pb = vb + P;       // [P] p, then w
    double* cs = pb + P;       // [P] rotation cosines of a QL sweep
    double* ss = cs + P;       // [P] rotation sines
    double* red = ss + P;      // [32] (+1 for odd P: och stays 16-byte aligned)
    double* och = red + 32 + (P & 1);  // [CH][P] centred O of a chunk of samples
    signed char* sgn = reinterpret_cast<signed char*>(och + (size_t)snrb_chunk(P) * P);  // [CH][N] spins
    __shared__ int ql_l, ql_m, ql_lo, ql_done, ql_fail;
    const size_t PP = (size_t)P * P;
    double* A = Aws + (size_t)t * PP;
    double* X = Xws + (size_t)t * PP;
    const double* St = S + (size_t)t * PP;
    for (size_t i = tid; i < PP; i += blockDim.x) A[i] = St[i];
    __syncthreads();

    // ---- (1) tridiagonalisation
    for (int k = 0; k + 2 < P; ++k) {
        const int m = P - 1 - k;
        double s2 = 0.0;
        for (int i = tid; i < m; i += blockDim.x) {
            const double x = A[(size_t)(k + 1 + i) * P + k];
            vb[i] = x;
            s2 += x * x;
        }
        const double nrm2 = block_sum(s2, red);
        const double x0 = vb[0];
        const double alpha = nrm2 > 0.0 ? -copysign(sqrt(nrm2), x0) : 0.0;
        const double vtv = nrm2 - 2.0 * alpha * x0 + alpha * alpha;
        const double tk = vtv > 0.0 ? 2.0 / vtv : 0.0;
        __syncthreads();
        if (tid == 0) {
            vb[0] = x0 - alpha;
            d[k] = A[(size_t)k * P + k];
            e[k] = alpha;
            tau[k] = tk;
        }
        __syncthreads();
        if (tk != 0.0) {
            // p = tau B v (B the trailing block), one warp per row
            for (int i = warp; i < m; i += SNRB_WARPS) {
                const double* Bi = A + (size_t)(k + 1 + i) * P + k + 1;
                double s = 0.0;
                for (int j = lane; j < m; j += 32) s += Bi[j] * vb[j];
                s = warp_sum(s);
                if (lane == 0) pb[i] = tk * s;
            }
            __syncthreads();
            double pv = 0.0;
            for (int i = tid; i < m; i += blockDim.x) pv += pb[i] * vb[i];
            const double K = 0.5 * tk * block_sum(pv, red);
            for (int i = tid; i < m; i += blockDim.x) pb[i] -= K * vb[i];  // w = p - K v
            __syncthreads();
            // B -= v w^T + w v^T
            for (int i = warp; i < m; i += SNRB_WARPS) {
                double* Bi = A + (size_t)(k + 1 + i) * P + k + 1;
                const double vi = vb[i], wi = pb[i];
                for (int j = lane; j < m; j += 32) Bi[j] -= vi * pb[j] + wi * vb[j];
            }
        }
        __syncthreads();
        for (int i = tid; i < m; i += blockDim.x) A[(size_t)(k + 1 + i) * P + k] = vb[i];
        __syncthreads();
    }
    if (tid == 0) {
        if (P >= 2) {
            d[P - 2] = A[(size_t)(P - 2) * P + P - 2];
            e[P - 2] = A[(size_t)(P - 1) * P + P - 2];
            tau[P - 2] = 0.0;
        }
        d[P - 1] = A[(size_t)(P - 1) * P + P - 1];
        e[P - 1] = 0.0;
        tau[P - 1] = 0.0;
    }
    __syncthreads();

    // ---- (2) X = Q^T = H_{P-3} ... H_0, formed as X <- X H_k from the identity, k descending
    for (size_t i = tid; i < PP; i += blockDim.x) X[i] = (i / P == i % P) ? 1.0 : 0.0;
    __syncthreads();
    for (int k = P - 3; k >= 0; --k) {
        const double tk = tau[k];
        if (tk == 0.0) continue;  // uniform
        const int m = P - 1 - k;
        for (int i = tid; i < m; i += blockDim.x) vb[i] = A[(size_t)(k + 1 + i) * P + k];
        __syncthreads();
        // rows r >= k + 1 of X are the only ones with entries in columns k + 1 .. (X is the
        // identity elsewhere): u_r = (X v)_r, then X[r][k+1+b] -= tau u_r v_b
        for (int r = warp; r < m; r += SNRB_WARPS) {
            const double* Xr = X + (size_t)(k + 1 + r) * P + k + 1;
            double s = 0.0;
            for (int b = lane; b < m; b += 32) s += Xr[b] * vb[b];
            s = warp_sum(s);
            if (lane == 0) pb[r] = tk * s;
        }
        __syncthreads();
        for (int r = warp; r < m; r += SNRB_WARPS) {
            double* Xr = X + (size_t)(k + 1 + r) * P + k + 1;
            const double u = pb[r];
            for (int b = lane; b < m; b += 32) Xr[b] -= u * vb[b];
        }
        __syncthreads();
    }

    // ---- (3) implicit QL on (d, e); rotations applied to rows i, i + 1 of X
    if (tid == 0) {
        ql_l = 0;
        ql_done = 0;
        ql_fail = 0;
    }
    __syncthreads();
    int iter = 0;
    // deflation: |e_m| below eps of the neighbouring diagonal entries, or below eps of the norm of
    // T (the accuracy the decomposition has anyway; without it a block of eigenvalues at the
    // rounding level of a rank-deficient S, where e stays at that level, never deflates)
    double tol_abs = 0.0;
    if (tid == 0) {
        double tn = 0.0;
        for (int i = 0; i < P; ++i) tn = fmax(tn, fabs(d[i]) + fabs(e[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0));
        tol_abs = 2.220446049250313e-16 * tn;
    }
    while (true) {
        if (tid == 0) {
            // find the next unreduced block starting at l; run one QL sweep on it
            int l = ql_l, m = l, lo = -1;
            bool swept = false;
            while (l < P && !swept) {
                for (m = l; m < P - 1; ++m) {
                    const double dd = fabs(d[m]) + fabs(d[m + 1]);
                    if (fabs(e[m]) <= tol_abs || fabs(e[m]) <= 2.220446049250313e-16 * dd) break;
                }
                if (m == l) {  // d[l] converged
                    ++l;
                    iter = 0;
                    continue;
                }
                if (++iter > SNRB_MAX_ITER) {
                    ql_fail = 1;
                    l = P;
                    break;
                }
                double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                double r = hypot(g, 1.0);
                g = d[m] - d[l] + e[l] / (g + copysign(r, g));
                double s = 1.0, c = 1.0, p = 0.0;
                int i = m - 1;
                bool underflow = false;
                for (; i >= l; --i) {
                    double f = s * e[i];
                    const double b = c * e[i];
                    r = sqrt(f * f + g * g);
                    if (!(r > 1e-150)) r = hypot(f, g);  // squares below the normal range
                    e[i + 1] = r;
                    if (r == 0.0) {  // deflation inside the sweep
                        d[i + 1] -= p;
                        e[m] = 0.0;
                        underflow = true;
                        break;
                    }
                    const double ir = 1.0 / r;
                    s = f * ir;
                    c = g * ir;
                    g = d[i + 1] - p;
                    r = (d[i] - g) * s + 2.0 * c * b;
                    p = s * r;
                    d[i + 1] = g + p;
                    g = c * r - b;
                    cs[i] = c;
                    ss[i] = s;
                }
                lo = i + 1;  // rotations recorded for i = m - 1 .. lo
                if (!underflow) {
                    d[l] -= p;
                    e[l] = g;
                    e[m] = 0.0;
                }
                swept = true;
            }
            ql_l = l;
            ql_m = m;
            ql_lo = lo;
            ql_done = (l >= P) ? 1 : 0;
        }
        __syncthreads();
        if (ql_done) break;
        // apply rotations i = m - 1 down to lo to every column of X: rows i and i + 1
        {
            const int m = ql_m, lo = ql_lo;
            for (int col = tid; col < P; col += blockDim.x) {
                if (m - 1 < lo) break;
                double zi1 = X[(size_t)m * P + col];  // row i + 1 for i = m - 1
                // rows are loaded eight at a time ahead of the rotations that use them (each
                // row is stored only after it has been loaded)
                for (int i = m - 1; i >= lo; i -= 8) {
                    const int nb = min(8, i - lo + 1);
                    double z[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (u < nb) z[u] = X[(size_t)(i - u) * P + col];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if (u < nb) {
                            const double c = cs[i - u], s = ss[i - u];
                            X[(size_t)(i - u + 1) * P + col] = s * z[u] + c * zi1;
                            zi1 = c * z[u] - s * zi1;
                        }
                }
                X[(size_t)lo * P + col] = zi1;
            }
        }
        __syncthreads();
    }
    if (ql_fail) {
        if (tid == 0) record_error(status, OTVMC_ERR_NONFINITE, t);
        for (int i = tid; i < P; i += blockDim.x) delta[(size_t)t * P + i] = make_double2(0.0, 0.0);
        return;
    }

    // ---- (4) rho = V^T D (row k of X is eigenvector k), mean of v
    double2* rho = reinterpret_cast<double2*>(tau);  // tau and vb: P double2
    double2* qs = reinterpret_cast<double2*>(pb);    // pb and cs: sum of Q_k
    double* q2 = ss;                                 // sum of |Q_k|^2
    __syncthreads();
    const double2* Dt = D + (size_t)t * P;
    for (int k = warp; k < P; k += SNRB_WARPS) {
        const double* Xk = X + (size_t)k * P;
        double ax = 0.0, ay = 0.0;
        for (int i = lane; i < P; i += 32) {
            ax += Xk[i] * Dt[i].x;
            ay += Xk[i] * Dt[i].y;
        }
        ax = warp_sum(ax);
        ay = warp_sum(ay);
        if (lane == 0) {
            rho[k] = make_double2(ax, ay);
            qs[k] = make_double2(0.0, 0.0);
            q2[k] = 0.0;
        }
    }
    const double2* vt = v + (size_t)t * ns;
    double sx = 0.0, sy = 0.0;
    for (int x = tid; x < ns; x += blockDim.x) {
        sx += vt[x].x;
        sy += vt[x].y;
    }
    const double vbx = block_sum(sx, red) / ns;
    const double vby = block_sum(sy, red) / ns;
    __syncthreads();

    // one pass over the samples in chunks: y_k(x) = sum_i V_ik O_c,i(x), Q = y v_c
    const int CH = snrb_chunk(P);
    const uint64_t* sp = spins + (size_t)t * ns * W;
    const double* ob = obar + (size_t)t * P;
    const int16_t* Ot = Oint != nullptr ? Oint + (size_t)t * P * ns : nullptr;
    if (fp32_pass) {
        // y in FP32 from an FP32 copy of the eigenvectors (in A's place, no longer needed):
        // the variances only set the filter, to a relative accuracy of about 1e-6
        float* Xf = reinterpret_cast<float*>(A);
        for (size_t i = tid; i < PP; i += blockDim.x) Xf[i] = (float)X[i];
        __syncthreads();
        snrb_sample_pass<float>(n, W, P, ns, sp, pairs, grp_off, grp_pair, Ot, ob, Xf, reinterpret_cast<float*>(och),
                                sgn, CH, vt, vbx, vby, qs, q2);
    } else {
        snrb_sample_pass<double>(n, W, P, ns, sp, pairs, grp_off, grp_pair, Ot, ob, X, och, sgn, CH, vt, vbx, vby, qs,
                                 q2);
    }

    // ---- (5) filter and back-projection: delta_i = sum_k V_ik c_k, c_k = f_k rho_k / lambda_k
    double lm = -INFINITY;
    for (int k = tid; k < P; k += blockDim.x) lm = fmax(lm, d[k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) lm = fmax(lm, __shfl_xor_sync(0xffffffffu, lm, off));
    __syncthreads();
    if (lane == 0) red[warp] = lm;
    __syncthreads();
    lm = red[0];
    for (int i = 1; i < SNRB_WARPS; ++i) lm = fmax(lm, red[i]);
    // the filtered coefficients go to the chunk buffer (2 P doubles at least), clear of rho/qs/q2
    double2* cf = reinterpret_cast<double2*>(och);
    for (int k = tid; k < P; k += blockDim.x) {
        const double lam = d[k];
        const double mqx = qs[k].x / ns, mqy = qs[k].y / ns;
        const double var = fmax(q2[k] / ns - (mqx * mqx + mqy * mqy), 0.0);
        const double snr = sqrt(rho[k].x * rho[k].x + rho[k].y * rho[k].y) / sqrt(var / ns + 1e-300);
        const double f_snr = 1.0 / (1.0 + pow(thr / snr, 6.0));
        const double f_svd = 1.0 / (1.0 + pow(eps_svd * lm / fmax(lam, 1e-300), 6.0));
        const double inv = lam > 0.0 ? f_snr * f_svd / fmax(lam, 1e-300) : 0.0;
        cf[k] = make_double2(inv * rho[k].x, inv * rho[k].y);
        if (lam_out) lam_out[(size_t)t * P + k] = lam;
    }
    __syncthreads();
    for (int i = tid; i < P; i += blockDim.x) {
        double ax = 0.0, ay = 0.0;
        for (int k = 0; k < P; ++k) {
            const double xki = X[(size_t)k * P + i];
            ax += xki * cf[k].x;
            ay += xki * cf[k].y;
        }
        delta[(size_t)t * P + i] = make_double2(ax, ay);
    }
}

size_t snr_big_smem_bytes(int P) {
    return (size_t)(7 * P + 32 + (P & 1) + snrb_chunk(P) * P) * sizeof(double) + SNRB_SGN_BYTES;
}

size_t snr_big_ws_bytes(int ntraj, int P) { return (size_t)ntraj * 2 * (size_t)P * P * sizeof(double) + 256; }

bool snr_big_fits(int P) { return snrb_chunk(P) >= 2; }

cudaError_t launch_snr_big(const otvmc_ansatz* a, int ntraj, int ns, const uint64_t* spins, const double* S,
                           const double* obar, const double2* v, const double2* D, double thr, double eps_svd,
                           double2* delta, double* lam, void* ws, int* status, cudaStream_t s, bool fp32_pass,
                           const int16_t* Oint) {
    ProfScope prof_(OTVMC_K_SOLVE, s);
    const int P = (int)a->P, n = a->n, W = (n + 63) / 64;
    const size_t smem = snr_big_smem_bytes(P);
    cudaError_t e = cudaFuncSetAttribute(snr_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    double* Aws = (double*)ws;
    double* Xws = Aws + (size_t)ntraj * P * P;
    const bool tied = a->kind == OTVMC_LJ;
    snr_big_kernel<<<ntraj, SNRB_THREADS, smem, s>>>(n, W, P, ns, spins, tied ? a->full->pairs_d : a->pairs_d,
                                                     tied ? a->grp_off_d : nullptr, tied ? a->grp_pair_d : nullptr,
                                                     S, obar, v, D, thr, eps_svd, Aws, Xws, delta, lam, status,
                                                     fp32_pass ? 1 : 0, Oint);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
