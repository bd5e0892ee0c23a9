// Regularised solve (S + eps I) delta = D of the otVMC equation (Eq. 8 discretised with
// the diagonal-shift regulariser), batched: one CTA per trajectory.
//
// Left-looking blocked Cholesky with 64-wide block columns, stored column-major lower
// (L[i + j P], i >= j) in workspace.  For each block column: load A = S + eps I, subtract
// L[jb:, :jb] L[jb:jb+64, :jb]^T (register-tiled SIMT GEMM), factor the 64 x 64 diagonal
// block with one warp, and solve the panel below it.  The right-hand side is complex and
// S real (Jastrow), so the real and imaginary parts are two right-hand sides.
//
// precision FP64: S given in full FP64, FP64 factor and solves.
// precision MIXED: S = G / ns - obar obar^T from the exact Gram counts; FP32 factor and
// solves, then `refine` steps of iterative refinement x += solve(D - (S + eps I) x) with the
// residual formed in FP64 from G and obar.
// A pivot below eps / 2 (every pivot of the factor of S + eps I is at least eps: a smaller one
// means rounding in this precision has overtaken the shift), a pivot that is not finite, or a
// solution that is not finite restarts the factorization with eps * 100 (at most three
// restarts); if all fail delta = 0 and OTVMC_ERR_NOT_PD is recorded.
#include "common.cuh"

namespace otvmc {

constexpr int CB = 64;   // block column width
constexpr int MB = 128;  // GEMM row chunk
constexpr int KC = 16;   // GEMM k chunk

template <typename T>
struct SolveSmem {
    T As[KC][MB];
    T Bs[KC][CB];
    T Dg[CB][CB + 1];
};

template <typename T, bool GRAM>
__device__ __forceinline__ T load_A(int P, int ns, int i, int j, double eps, const double* S, const float* G,
                                    const double* ob) {
    // i >= j; returns (S + eps I)_ij
    double v;
    if (GRAM) v = (double)G[(size_t)j * P + i] / ns - ob[i] * ob[j];
    else v = S[(size_t)j * P + i];
    if (i == j) v += eps;
    return (T)v;
}

template <typename T, bool GRAM>
__device__ bool factor(int P, int ns, double eps, const double* S, const float* G, const double* ob, T* L,
                       SolveSmem<T>& sm) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int fail;
    if (tid == 0) fail = 0;
    for (int jb = 0; jb < P; jb += CB) {
        const int nb = min(CB, P - jb);
        const int M = P - jb;
        // (a) load the block column of A
        for (int c = 0; c < nb; ++c) {
            const int j = jb + c;
            for (int i = j + tid; i < P; i += blockDim.x) L[(size_t)j * P + i] = load_A<T, GRAM>(P, ns, i, j, eps, S, G, ob);
        }
        __syncthreads();
        // (b) C[jb:P, jb:jb+nb] -= L[jb:P, 0:jb] L[jb:jb+nb, 0:jb]^T
        if (jb > 0) {
            const int rg = tid / 16, cg = tid % 16;
            for (int r0 = jb; r0 < P; r0 += MB) {
                T acc[8][4];
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = (T)0;
                for (int k0 = 0; k0 < jb; k0 += KC) {
                    for (int e = tid; e < KC * MB; e += blockDim.x) {
                        const int kk = e / MB, i = e % MB;
                        const int gi = r0 + i;
                        sm.As[kk][i] = (gi < P) ? L[(size_t)(k0 + kk) * P + gi] : (T)0;
                    }
                    for (int e = tid; e < KC * CB; e += blockDim.x) {
                        const int kk = e / CB, c = e % CB;
                        sm.Bs[kk][c] = (c < nb) ? L[(size_t)(k0 + kk) * P + jb + c] : (T)0;
                    }
                    __syncthreads();
#pragma unroll 4
                    for (int kk = 0; kk < KC; ++kk) {
                        T a[8], b[4];
#pragma unroll
                        for (int u = 0; u < 8; ++u) a[u] = sm.As[kk][rg * 8 + u];
#pragma unroll
                        for (int v = 0; v < 4; ++v) b[v] = sm.Bs[kk][cg * 4 + v];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int gi = r0 + rg * 8 + u, c = cg * 4 + v, gj = jb + c;
                        if (gi < P && c < nb && gi >= gj) L[(size_t)gj * P + gi] -= acc[u][v];
                    }
            }
            __syncthreads();
        }
        (void)M;
        // (c) diagonal block: one warp, unblocked right-looking Cholesky in shared memory
        for (int e = tid; e < nb * nb; e += blockDim.x) {
            const int i = e / nb, c = e % nb;
            if (i >= c) sm.Dg[i][c] = L[(size_t)(jb + c) * P + jb + i];
        }
        __syncthreads();
        if (warp == 0) {
            for (int p = 0; p < nb; ++p) {
                const T d = sm.Dg[p][p];
                // every pivot of the factor of S + eps I is at least eps; one below eps / 2
                // means rounding has overtaken the shift (the caller raises it)
                const bool bad = !(d > (T)(0.5 * eps)) || !isfinite((double)d);
                if (bad) {
                    if (lane == 0) fail = 1;
                    break;
                }
                const T sd = sqrt(d);
                __syncwarp();
                for (int i = p + 1 + lane; i < nb; i += 32) sm.Dg[i][p] /= sd;
                if (lane == 0) sm.Dg[p][p] = sd;
                __syncwarp();
                for (int i = p + 1 + lane; i < nb; i += 32) {
                    const T lip = sm.Dg[i][p];
                    for (int c = p + 1; c <= i; ++c) sm.Dg[i][c] -= lip * sm.Dg[c][p];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (fail) return false;
        for (int e = tid; e < nb * nb; e += blockDim.x) {
            const int i = e / nb, c = e % nb;
            if (i >= c) L[(size_t)(jb + c) * P + jb + i] = sm.Dg[i][c];
        }
        // (d) panel: rows below the block, x L_dd^T = a
        for (int i = jb + nb + tid; i < P; i += blockDim.x) {
            T x[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                if (c < nb) {
                    T a = L[(size_t)(jb + c) * P + i];
                    for (int k = 0; k < c; ++k) a -= x[k] * sm.Dg[c][k];
                    x[c] = a / sm.Dg[c][c];
                }
            }
#pragma unroll
            for (int c = 0; c < CB; ++c)
                if (c < nb) L[(size_t)(jb + c) * P + i] = x[c];
        }
        __syncthreads();
    }
    return true;
}

// Solves L L^T x = y in place for two right-hand sides (yr, yi).
template <typename T>
__device__ void tri_solve(int P, const T* L, T* yr, T* yi) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // forward: L y = b
    for (int jb = 0; jb < P; jb += CB) {
        const int nb = min(CB, P - jb);
        if (warp == 0) {
            for (int c = 0; c < nb; ++c) {
                const int j = jb + c;
                const T d = L[(size_t)j * P + j];
                const T a = yr[j] / d, b = yi[j] / d;
                __syncwarp();
                for (int i = j + 1 + lane; i < jb + nb; i += 32) {
                    const T l = L[(size_t)j * P + i];
                    yr[i] -= l * a;
                    yi[i] -= l * b;
                }
                if (lane == 0) {
                    yr[j] = a;
                    yi[j] = b;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        for (int i = jb + nb + tid; i < P; i += blockDim.x) {
            T ar = yr[i], ai = yi[i];
            for (int c = 0; c < nb; ++c) {
                const T l = L[(size_t)(jb + c) * P + i];
                ar -= l * yr[jb + c];
                ai -= l * yi[jb + c];
            }
            yr[i] = ar;
            yi[i] = ai;
        }
        __syncthreads();
    }
    // backward: L^T x = y
    const int nblk = (P + CB - 1) / CB;
    for (int bk = nblk - 1; bk >= 0; --bk) {
        const int jb = bk * CB, nb = min(CB, P - jb);
        for (int c = warp; c < nb; c += blockDim.x / 32) {
            const int j = jb + c;
            T sr = (T)0, si = (T)0;
            for (int i = jb + nb + lane; i < P; i += 32) {
                const T l = L[(size_t)j * P + i];
                sr += l * yr[i];
                si += l * yi[i];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, off);
                si += __shfl_xor_sync(0xffffffffu, si, off);
            }
            if (lane == 0) {
                yr[j] -= sr;
                yi[j] -= si;
            }
        }
        __syncthreads();
        if (warp == 0) {
            for (int c = nb - 1; c >= 0; --c) {
                const int j = jb + c;
                const T d = L[(size_t)j * P + j];
                const T a = yr[j] / d, b = yi[j] / d;
                __syncwarp();
                for (int cc = lane; cc < c; cc += 32) {
                    const T l = L[(size_t)(jb + cc) * P + j];
                    yr[jb + cc] -= l * a;
                    yi[jb + cc] -= l * b;
                }
                if (lane == 0) {
                    yr[j] = a;
                    yi[j] = b;
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
}

template <typename T, bool GRAM>
__global__ void __launch_bounds__(256, 1) chol_solve_kernel(int P, int ns, double eps0, int refine,
                                                            const double* __restrict__ S, const float* __restrict__ G,
                                                            const double* __restrict__ obar,
                                                            const double2* __restrict__ D, double2* __restrict__ delta,
                                                            double* __restrict__ shift_used, T* __restrict__ Lws,
                                                            size_t lstride, T* __restrict__ yws,
                                                            double* __restrict__ xws, const int* __restrict__ only,
                                                            int* status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    SolveSmem<T>& sm = *reinterpret_cast<SolveSmem<T>*>(smraw);
    __shared__ double red[2][8];
    const int t = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (only != nullptr && only[t] == 0) return;
    const size_t PP = (size_t)P * P;
    T* L = Lws + (size_t)t * lstride;  // lstride >= P * P elements per trajectory
    const double* St = GRAM ? nullptr : S + (size_t)t * PP;
    const float* Gt = GRAM ? G + (size_t)t * PP : nullptr;
    const double* ob = GRAM ? obar + (size_t)t * P : nullptr;
    const double2* Dt = D + (size_t)t * P;
    T* yr = yws + (size_t)t * 2 * P;
    T* yi = yr + P;
    double* xr = xws + (size_t)t * 4 * P;
    double* xi = xr + P;
    double* rr = xi + P;
    double* ri = rr + P;

    double eps = eps0;
    bool ok = false;
    for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
        ok = factor<T, GRAM>(P, ns, eps, St, Gt, ob, L, sm);
        __syncthreads();
        if (ok) {
            for (int k = tid; k < P; k += blockDim.x) {
                yr[k] = (T)Dt[k].x;
                yi[k] = (T)Dt[k].y;
            }
            __syncthreads();
            tri_solve<T>(P, L, yr, yi);
            __syncthreads();
            // a solution that is not finite (a factor too ill-conditioned for this precision,
            // with no pivot below zero) counts as a failed attempt
            bool fin = true;
            for (int k = tid; k < P; k += blockDim.x) fin = fin && isfinite(yr[k]) && isfinite(yi[k]);
            ok = !__syncthreads_or(!fin);
        }
        if (!ok) eps *= 100.0;
    }
    if (!ok) {
        for (int k = tid; k < P; k += blockDim.x) delta[(size_t)t * P + k] = make_double2(0.0, 0.0);
        if (tid == 0) {
            record_error(status, OTVMC_ERR_NOT_PD, t);
            if (shift_used) shift_used[t] = eps;
        }
        return;
    }
    for (int k = tid; k < P; k += blockDim.x) {
        xr[k] = (double)yr[k];
        xi[k] = (double)yi[k];
    }
    __syncthreads();
    for (int it = 0; GRAM && it < refine; ++it) {
        // ox = obar^T x
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
        // z_j = sum_{i<j} G[i][j] x_i  (column sums of the strict upper triangle)
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
        // y_i = sum_{j>=i} G[i][j] x_j, one warp per row; residual
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
                yr[i] = (T)(Dt[i].x - sxr);
                yi[i] = (T)(Dt[i].y - sxi);
            }
        }
        __syncthreads();
        tri_solve<T>(P, L, yr, yi);
        for (int k = tid; k < P; k += blockDim.x) {
            xr[k] += (double)yr[k];
            xi[k] += (double)yi[k];
        }
        __syncthreads();
    }
    for (int k = tid; k < P; k += blockDim.x) delta[(size_t)t * P + k] = make_double2(xr[k], xi[k]);
    if (tid == 0 && shift_used) shift_used[t] = eps;
}

size_t chol_tc_ws_bytes(int ntraj, int P);
cudaError_t launch_chol_tc(int ntraj, int P, int ns, double eps, const float* G, const double* obar,
                           const double2* D, double2* delta, double* shift_used, void* ws, int refine_iters,
                           int* status, cudaStream_t s);

size_t chol_ws_bytes(int ntraj, int P, int precision) {
    if (precision != OTVMC_PREC_FP64) return chol_tc_ws_bytes(ntraj, P);
    return (size_t)ntraj * ((size_t)P * P * 8 + 2 * (size_t)P * 8 + 4 * (size_t)P * 8) + 3 * 256;
}

cudaError_t launch_chol_solve_masked(int ntraj, int P, int ns, double eps, const float* G, const double* obar,
                                     const double2* D, double2* delta, double* shift_used, float* L, size_t lstride,
                                     float* y, double* x, int refine_iters, const int* only, int* status,
                                     cudaStream_t s) {
    const int smem = (int)sizeof(SolveSmem<float>);
    cudaFuncSetAttribute(chol_solve_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    chol_solve_kernel<float, true><<<ntraj, 256, smem, s>>>(P, ns, eps, refine_iters, nullptr, G, obar, D, delta,
                                                            shift_used, L, lstride, y, x, only, status);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_chol_solve(int ntraj, int P, int ns, int precision, double eps, const double* S, const float* G,
                              const double* obar, const double2* D, double2* delta, double* shift_used, void* ws,
                              int refine_iters, int* status, cudaStream_t s) {
    if (precision != OTVMC_PREC_FP64)
        return launch_chol_tc(ntraj, P, ns, eps, G, obar, D, delta, shift_used, ws, refine_iters, status, s);
    ProfScope prof_(OTVMC_K_SOLVE, s);
    char* p = (char*)ws;
    auto take = [&](size_t bytes) {
        char* r = p;
        p += (bytes + 255) & ~(size_t)255;
        return (void*)r;
    };
    void* L = take((size_t)ntraj * P * P * 8);
    void* y = take((size_t)ntraj * 2 * P * 8);
    double* x = (double*)take((size_t)ntraj * 4 * P * 8);
    const int smem = (int)sizeof(SolveSmem<double>);
    cudaFuncSetAttribute(chol_solve_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    chol_solve_kernel<double, false><<<ntraj, 256, smem, s>>>(P, ns, eps, 0, S, G, obar, D, delta, shift_used,
                                                              (double*)L, (size_t)P * P, (double*)y, x, nullptr,
                                                              status);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
