// Local estimators of one evaluation (definitions after Eq. 8, effective Hamiltonian Eq. 5)
// for the Jastrow ansatz, the centred-v quantisation feeding D, and the per-trajectory
// observables (LITF paragraph).
//
// Fields f_j = a_j + sum_k eta_jk sigma_k (complex) and sum_k J_jk sigma_k are summed
// exactly in int64 fixed point (units of 2^-48): with sigma = +-1 the sum is
// base_j + 2 sum_{k: sigma_k = +1} Q_jk, base_j = Qa_j - sum_k Q_jk, so each term is one
// predicated 64-bit add and the result does not depend on the summation order.
#include "common.cuh"

namespace otvmc {

__host__ __device__ __forceinline__ int pair_idx(int lo, int hi, int n) {
    return lo * n - lo * (lo + 1) / 2 + (hi - lo - 1);
}

// ----------------------------------------------------------------- fixed-point tables
__global__ void jastrow_prep_kernel(const double2* __restrict__ theta, int P, int n, long long* __restrict__ Qre,
                                    long long* __restrict__ Qim, long long* __restrict__ base_re,
                                    long long* __restrict__ base_im, int* status) {
    const int t = blockIdx.x;
    const double2* th = theta + (size_t)t * P;
    long long* qr = Qre + (size_t)t * n * n;
    long long* qi = Qim + (size_t)t * n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int j = idx / n, k = idx - j * n;
        double2 v = make_double2(0.0, 0.0);
        if (j != k) v = th[n + pair_idx(min(j, k), max(j, k), n)];
        qr[idx] = fx_quant(v.x);
        qi[idx] = fx_quant(v.y);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double rr = fabs(th[j].x), ri = fabs(th[j].y);
        long long sr = 0, si = 0;
        for (int k = 0; k < n; ++k) {
            if (k == j) continue;
            const double2 v = th[n + pair_idx(min(j, k), max(j, k), n)];
            rr += fabs(v.x);
            ri += fabs(v.y);
            sr += qr[j * n + k];
            si += qi[j * n + k];
        }
        if (!(rr < 8192.0 && ri < 8192.0)) record_error(status, OTVMC_ERR_RANGE, t);
        base_re[(size_t)t * n + j] = (rr < 8192.0) ? fx_quant(th[j].x) - sr : 0;
        base_im[(size_t)t * n + j] = (ri < 8192.0) ? fx_quant(th[j].y) - si : 0;
    }
}

cudaError_t launch_jastrow_prep(const otvmc_ansatz* a, const double2* theta, int ntraj, const EvalBufs& b,
                                int* status, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_PREP, s);
    jastrow_prep_kernel<<<ntraj, 256, 0, s>>>(theta, (int)a->P, a->n, b.Qre, b.Qim, b.base_re, b.base_im, status);
    count_launch();
    return cudaGetLastError();
}

// --------------------------------------------------------------------------- est1
// One CTA: SB = (256/NT)*8 samples of one trajectory; thread (g, j) owns site j of the
// samples g, g + SPP, ... .  Produces r_j(x), E_H(x) and per-CTA site sums.
constexpr int EST_KC = 16;

template <bool FP32T>
__global__ void __launch_bounds__(256) est1_jastrow_kernel(
    int n, int W, int ns, double h, const uint64_t* __restrict__ spins, const long long* __restrict__ Qre,
    const long long* __restrict__ Qim, const long long* __restrict__ base_re, const long long* __restrict__ base_im,
    const long long* __restrict__ QJ, const long long* __restrict__ baseJ, void* __restrict__ r_out,
    double2* __restrict__ EH_out, double2* __restrict__ part_r, double2* __restrict__ part_sr,
    double* __restrict__ part_s) {
    constexpr int SPT = EST_SAMPLES_PER_THREAD;
    const int NT = ((n + 31) / 32) * 32;
    const int SPP = 256 / NT;
    const int SB = SPP * SPT;
    const int t = blockIdx.y, blk = blockIdx.x;
    const int j = threadIdx.x % NT, g = threadIdx.x / NT;
    const bool active = (g < SPP) && (j < n);
    const int s0 = blk * SB;

    extern __shared__ __align__(16) unsigned char smraw[];
    uint64_t* sw = (uint64_t*)smraw;                         // [SB][W]
    long long* qr_s = (long long*)(sw + SB * W);             // [KC][n]
    long long* qi_s = qr_s + EST_KC * n;
    long long* qj_s = qi_s + EST_KC * n;
    double2* ered = (double2*)(qj_s + EST_KC * n);           // [SPP*SPT][NT/32]

    for (int i = threadIdx.x; i < SB * W; i += blockDim.x) {
        const int sl = i / W, w = i - sl * W;
        const int s = s0 + sl;
        sw[i] = (s < ns) ? spins[((size_t)t * ns + s) * W + w] : 0ull;
    }

    // Real and J fields: exact int64 on the FP64 path, FP32 sums on the mixed path (staged as
    // FP32 in the same shared-memory rows).  The imaginary field stays exact int64 on both, for
    // the phase reduction modulo 2 pi.
    long long ar[SPT], ai[SPT], aj[SPT];
    float arf[SPT], ajf[SPT];
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
        ar[q] = ai[q] = aj[q] = 0;
        arf[q] = ajf[q] = 0.f;
    }
    float* qr_f = reinterpret_cast<float*>(qr_s);
    float* qj_f = reinterpret_cast<float*>(qj_s);

    const long long* QrT = Qre + (size_t)t * n * n;
    const long long* QiT = Qim + (size_t)t * n * n;
    for (int kc = 0; kc < n; kc += EST_KC) {
        __syncthreads();
        const int rows = min(EST_KC, n - kc);
        for (int i = threadIdx.x; i < rows * n; i += blockDim.x) {
            qi_s[i] = QiT[(size_t)kc * n + i];
            if constexpr (FP32T) {
                qr_f[i] = fx_to_float(QrT[(size_t)kc * n + i]);
                qj_f[i] = fx_to_float(QJ[(size_t)kc * n + i]);
            } else {
                qr_s[i] = QrT[(size_t)kc * n + i];
                qj_s[i] = QJ[(size_t)kc * n + i];
            }
        }
        __syncthreads();
        if (active) {
            uint64_t wq[SPT];
#pragma unroll
            for (int q = 0; q < SPT; ++q) wq[q] = sw[(g + q * SPP) * W + (kc >> 6)] >> (kc & 63);
            for (int kk = 0; kk < rows; ++kk) {
                const long long vi = qi_s[kk * n + j];
                if constexpr (FP32T) {
                    const float vr = qr_f[kk * n + j], vj = qj_f[kk * n + j];
#pragma unroll
                    for (int q = 0; q < SPT; ++q) {
                        if ((wq[q] >> kk) & 1ull) {
                            arf[q] += vr;
                            ai[q] += vi;
                            ajf[q] += vj;
                        }
                    }
                } else {
                    const long long vr = qr_s[kk * n + j], vj = qj_s[kk * n + j];
#pragma unroll
                    for (int q = 0; q < SPT; ++q) {
                        if ((wq[q] >> kk) & 1ull) {
                            ar[q] += vr;
                            ai[q] += vi;
                            aj[q] += vj;
                        }
                    }
                }
            }
        }
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, wis = j / 32;  // warp index within the sample's NT threads
    double2 pr = make_double2(0, 0), psr = make_double2(0, 0);
    double ps = 0.0;
    if constexpr (FP32T) {
        // MIXED: fields converted from the exact fixed-point sums straight to FP32, the phase
        // reduced modulo 2 pi in fixed point, ratios kept in FP32; per-thread sums in FP32.
        float2* rf = reinterpret_cast<float2*>(r_out);
        float2 prf = make_float2(0.f, 0.f), psrf = make_float2(0.f, 0.f);
        int psi = 0;
        const float bre = active ? fx_to_float(base_re[(size_t)t * n + j]) : 0.f;
        const float bj = active ? fx_to_float(baseJ[j]) : 0.f;
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
            const int sl = g + q * SPP;
            const int s = s0 + sl;
            float hrx = 0.f, hry = 0.f, fsg = 0.f;
            if (active && s < ns) {
                const bool up = (sw[sl * W + (j >> 6)] >> (j & 63)) & 1ull;
                const float fre = fmaf(2.f, arf[q], bre);
                const long long fim = base_im[(size_t)t * n + j] + 2 * ai[q];
                const float fj = fmaf(2.f, ajf[q], bj);
                // log r_j = -2 sigma_j f_j
                const long long lim = up ? -2 * fim : 2 * fim;
                const float e = expf(up ? -2.f * fre : 2.f * fre);
                const int kq = __float2int_rn(fx_to_float(lim) * 0.15915494309189535f);
                const long long red = lim - (long long)kq * FX_TWO_PI;
                float sn, cs;
                sincosf(fx_to_float(red), &sn, &cs);
                const float2 r = make_float2(e * cs, e * sn);
                rf[((size_t)t * ns + s) * n + j] = r;
                hrx = r.x;
                hry = r.y;
                fsg = up ? fj : -fj;  // sigma_j f^J_j
                prf.x += r.x;
                prf.y += r.y;
                psrf.x += up ? r.x : -r.x;
                psrf.y += up ? r.y : -r.y;
                psi += up ? 1 : -1;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                hrx += __shfl_xor_sync(0xffffffffu, hrx, off);
                hry += __shfl_xor_sync(0xffffffffu, hry, off);
                fsg += __shfl_xor_sync(0xffffffffu, fsg, off);
            }
            if (lane == 0 && g < SPP)
                ered[sl * (NT / 32) + wis] = make_double2(0.5 * (double)fsg + h * (double)hrx, h * (double)hry);
        }
        pr = make_double2((double)prf.x, (double)prf.y);
        psr = make_double2((double)psrf.x, (double)psrf.y);
        ps = (double)psi;
    } else {
        double2* rd = reinterpret_cast<double2*>(r_out);
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
            const int sl = g + q * SPP;
            const int s = s0 + sl;
            double2 contrib = make_double2(0.0, 0.0);
            if (active && s < ns) {
                const int sj = ((sw[sl * W + (j >> 6)] >> (j & 63)) & 1ull) ? 1 : -1;
                const double fre = (double)(base_re[(size_t)t * n + j] + 2 * ar[q]) * FX_INV;
                const double fim = (double)(base_im[(size_t)t * n + j] + 2 * ai[q]) * FX_INV;
                const double fj = (double)(baseJ[j] + 2 * aj[q]) * FX_INV;
                const double2 r = cexp_prec(-2.0 * sj * fre, -2.0 * sj * fim, false);
                rd[((size_t)t * ns + s) * n + j] = r;
                contrib = make_double2(0.5 * sj * fj + h * r.x, h * r.y);
                pr.x += r.x;
                pr.y += r.y;
                psr.x += sj * r.x;
                psr.y += sj * r.y;
                ps += sj;
            }
            // sum over the sample's sites: butterfly within each warp, then warps in order
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                contrib.x += __shfl_xor_sync(0xffffffffu, contrib.x, off);
                contrib.y += __shfl_xor_sync(0xffffffffu, contrib.y, off);
            }
            if (lane == 0 && g < SPP) ered[sl * (NT / 32) + wis] = contrib;
        }
    }
    __syncthreads();
    if (threadIdx.x < SB) {
        const int sl = threadIdx.x, s = s0 + sl;
        if (s < ns) {
            double2 e = make_double2(0.0, 0.0);
            for (int w = 0; w < NT / 32; ++w) {
                e.x += ered[sl * (NT / 32) + w].x;
                e.y += ered[sl * (NT / 32) + w].y;
            }
            EH_out[(size_t)t * ns + s] = e;
        }
    }
    // site sums over this CTA's samples: groups g in order
    __syncthreads();
    double2* red_r = (double2*)qr_s;  // reuse: [SPP][NT]
    double2* red_sr = red_r + SPP * NT;
    double* red_s = (double*)(red_sr + SPP * NT);
    if (g < SPP) {
        red_r[g * NT + j] = pr;
        red_sr[g * NT + j] = psr;
        red_s[g * NT + j] = ps;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        const int jj = threadIdx.x;
        double2 a = make_double2(0, 0), b = make_double2(0, 0);
        double c = 0.0;
        for (int gg = 0; gg < SPP; ++gg) {
            a.x += red_r[gg * NT + jj].x;
            a.y += red_r[gg * NT + jj].y;
            b.x += red_sr[gg * NT + jj].x;
            b.y += red_sr[gg * NT + jj].y;
            c += red_s[gg * NT + jj];
        }
        const size_t o = ((size_t)t * gridDim.x + blk) * n + jj;
        part_r[o] = a;
        part_sr[o] = b;
        part_s[o] = c;
    }
}

static size_t est1_smem(int n, int W) {
    const int NT = ((n + 31) / 32) * 32, SPP = 256 / NT, SB = SPP * EST_SAMPLES_PER_THREAD;
    size_t a = (size_t)SB * W * 8 + 3 * (size_t)EST_KC * n * 8 + (size_t)SB * (NT / 32) * 16 + 64;
    size_t b = (size_t)SB * W * 8 + (size_t)SPP * NT * 40 + 64;
    return a > b ? a : b;
}

cudaError_t launch_est1_jastrow(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, bool fp32,
                                const EvalBufs& b, int* status, cudaStream_t s) {
    if (est_tc_ok(a, fp32)) return launch_est_tc(a, spins, ntraj, ns, b, status, s);
    ProfScope prof_(OTVMC_K_EST1, s);
    (void)status;
    const int n = a->n, W = (n + 63) / 64;
    const size_t smem = est1_smem(n, W);
    dim3 grid(est_blocks(n, ns), ntraj);
    const otvmc_model* m = a->model;
    if (fp32) {
        cudaFuncSetAttribute(est1_jastrow_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        est1_jastrow_kernel<true><<<grid, 256, smem, s>>>(n, W, ns, m->h, spins, b.Qre, b.Qim, b.base_re, b.base_im,
                                                         m->QJ_d, m->baseJ_d, b.r, b.EH, b.part_r, b.part_sr,
                                                         b.part_s);
    } else {
        cudaFuncSetAttribute(est1_jastrow_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        est1_jastrow_kernel<false><<<grid, 256, smem, s>>>(n, W, ns, m->h, spins, b.Qre, b.Qim, b.base_re,
                                                          b.base_im, m->QJ_d, m->baseJ_d, b.r, b.EH, b.part_r,
                                                          b.part_sr, b.part_s);
    }
    count_launch();
    return cudaGetLastError();
}

// -------------------------------------------------------------------- site means, <L+L^+>
// mean_r_j = <r_j> (local sx_j), mean_sr_j = <sigma_j r_j>, mean_s_j = <sigma_j>; then
// <L + L^+> = sqrt(kappa_j) Re mean_r_j (decay), 2 sqrt(gamma_j) mean_s_j (dephasing).
__global__ void site_means_kernel(int n, int nblk, int ns, int nops, const double2* __restrict__ part_r,
                                  const double2* __restrict__ part_sr, const double* __restrict__ part_s,
                                  const double* __restrict__ site, const int* __restrict__ opidx,
                                  double2* __restrict__ mean_r, double2* __restrict__ mean_sr,
                                  double* __restrict__ mean_s, double* __restrict__ lpl) {
    const int t = blockIdx.x;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        double2 a = make_double2(0, 0), b = make_double2(0, 0);
        double c = 0.0;
        for (int k = 0; k < nblk; ++k) {
            const size_t o = ((size_t)t * nblk + k) * n + j;
            a.x += part_r[o].x;
            a.y += part_r[o].y;
            b.x += part_sr[o].x;
            b.y += part_sr[o].y;
            c += part_s[o];
        }
        const double inv = 1.0 / ns;
        a.x *= inv; a.y *= inv; b.x *= inv; b.y *= inv; c *= inv;
        mean_r[(size_t)t * n + j] = a;
        mean_sr[(size_t)t * n + j] = b;
        mean_s[(size_t)t * n + j] = c;
        if (lpl) {
            const int od = opidx[j], og = opidx[n + j];
            if (od >= 0) lpl[(size_t)t * nops + od] = site[2 * n + j] * a.x;
            if (og >= 0) lpl[(size_t)t * nops + og] = 2.0 * site[3 * n + j] * c;
        }
    }
}

cudaError_t launch_site_means(const otvmc_ansatz* a, int ntraj, int ns, bool fp32, const EvalBufs& b, double* lpl,
                              cudaStream_t s) {
    ProfScope prof_(OTVMC_K_REDUCE, s);
    const otvmc_model* m = a->model;
    // the per-site partials come from the tensor-core estimators (est_tc_chunks) or the SIMT ones
    site_means_kernel<<<ntraj, 256, 0, s>>>(a->n, est_tc_ok(a, fp32) ? est_tc_chunks(ns) : est_blocks(a->n, ns), ns,
                                            m->nops,
                                            b.part_r, b.part_sr, b.part_s,
                                            m->site_d, m->opidx_d, b.mean_r, b.mean_sr, b.mean_s, lpl);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- est2
// E_eff(x) = E_H(x) - i/2 sum_n [(L^+L)_loc - 2 <L+L^+>_n B^n(x) + (L^2)_loc]
// v(x) = -i dt E_eff(x) + sum_n dW_n B^n(x)
// decay site j:  B = sqrt(kappa_j) [sigma_j = -1] r_j, (L^+L)_loc = kappa_j (1 + sigma_j)/2, L^2 = 0
// dephasing j:   B = sqrt(gamma_j) sigma_j, (L^+L)_loc = (L^2)_loc = gamma_j
// One thread per sample, 256 samples per CTA.
template <typename R2>
__global__ void __launch_bounds__(VRED_BLOCK) est2_kernel(
    int n, int W, int ns, int nops, double dt, const uint64_t* __restrict__ spins, const R2* __restrict__ r,
    const double2* __restrict__ EH, const double* __restrict__ site, const int* __restrict__ opidx,
    const double* __restrict__ lpl, const double* __restrict__ dW, double2* __restrict__ Eeff_out,
    double2* __restrict__ v_out, double2* __restrict__ part_v, double* __restrict__ part_vmax) {
    extern __shared__ __align__(16) unsigned char smraw[];
    double* kap = (double*)smraw;  // [n]
    double* gam = kap + n;
    double* skap = gam + n;
    double* sgam = skap + n;
    double* lpl_d = sgam + n;  // per site, decay op
    double* lpl_g = lpl_d + n; // per site, dephasing op
    double* dw_d = lpl_g + n;
    double* dw_g = dw_d + n;
    double2* red = (double2*)(dw_g + n);  // [VRED_BLOCK]
    double* redm = (double*)(red + VRED_BLOCK);
    const int t = blockIdx.y;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        kap[j] = site[j];
        gam[j] = site[n + j];
        skap[j] = site[2 * n + j];
        sgam[j] = site[3 * n + j];
        const int od = opidx[j], og = opidx[n + j];
        lpl_d[j] = od >= 0 ? lpl[(size_t)t * nops + od] : 0.0;
        lpl_g[j] = og >= 0 ? lpl[(size_t)t * nops + og] : 0.0;
        dw_d[j] = od >= 0 ? dW[(size_t)t * nops + od] : 0.0;
        dw_g[j] = og >= 0 ? dW[(size_t)t * nops + og] : 0.0;
    }
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double2 v = make_double2(0, 0);
    if (s < ns) {
        const uint64_t* w = spins + ((size_t)t * ns + s) * W;
        const R2* rs = r + ((size_t)t * ns + s) * n;
        double br = 0.0, bi = 0.0;  // sum_n bracket_n
        double vr = 0.0, vi = 0.0;  // sum_n dW_n B^n
        for (int j = 0; j < n; ++j) {
            const int sj = ((w[j >> 6] >> (j & 63)) & 1ull) ? 1 : -1;
            if (kap[j] > 0.0) {
                double2 B = make_double2(0.0, 0.0);
                if (sj < 0) {
                    const double2 rj = make_double2((double)rs[j].x, (double)rs[j].y);
                    B = make_double2(skap[j] * rj.x, skap[j] * rj.y);
                }
                br += kap[j] * 0.5 * (1 + sj) - 2.0 * lpl_d[j] * B.x;
                bi += -2.0 * lpl_d[j] * B.y;
                vr += dw_d[j] * B.x;
                vi += dw_d[j] * B.y;
            }
            if (gam[j] > 0.0) {
                const double B = sgam[j] * sj;
                br += 2.0 * gam[j] - 2.0 * lpl_g[j] * B;
                vr += dw_g[j] * B;
            }
        }
        double2 E = EH[(size_t)t * ns + s];
        // -i/2 (br + i bi) = bi/2 - i br/2
        E.x += 0.5 * bi;
        E.y -= 0.5 * br;
        // -i dt E = dt E.y - i dt E.x
        v = make_double2(dt * E.y + vr, -dt * E.x + vi);
        if (Eeff_out) Eeff_out[(size_t)t * ns + s] = E;
        v_out[(size_t)t * ns + s] = v;
    }
    red[threadIdx.x] = v;
    redm[threadIdx.x] = fmax(fabs(v.x), fabs(v.y));
    __syncthreads();
    for (int st = VRED_BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            red[threadIdx.x].x += red[threadIdx.x + st].x;
            red[threadIdx.x].y += red[threadIdx.x + st].y;
            redm[threadIdx.x] = fmax(redm[threadIdx.x], redm[threadIdx.x + st]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_v[(size_t)t * gridDim.x + blockIdx.x] = red[0];
        part_vmax[(size_t)t * gridDim.x + blockIdx.x] = redm[0];
    }
}

// MIXED path of est2: the same sums regrouped per site,
//   sum_n bracket_n = C0 + sum_j c_j sigma_j + sum_{j down} alpha_j r_j,
//   sum_n dW_n B^n  =      sum_j d_j sigma_j + sum_{j down} beta_j r_j,
// with C0 = sum_j (kappa_j / 2 + 2 gamma_j), c_j = kappa_j / 2 - 2 <L+L^+>_deph sqrt(gamma_j),
// d_j = dW_deph sqrt(gamma_j), alpha_j = -2 <L+L^+>_decay sqrt(kappa_j), beta_j = dW_decay
// sqrt(kappa_j).  Products and runs of eight sites in FP32, the runs added in FP64.
__global__ void __launch_bounds__(VRED_BLOCK) est2_mixed_kernel(
    int n, int W, int ns, int nops, double dt, const uint64_t* __restrict__ spins, const float2* __restrict__ r,
    const double2* __restrict__ EH, int nq, const double* __restrict__ site, const int* __restrict__ opidx,
    const double* __restrict__ lpl, const double* __restrict__ dW, double2* __restrict__ Eeff_out,
    double2* __restrict__ v_out, double2* __restrict__ part_v, double* __restrict__ part_vmax) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float* al = (float*)smraw;  // [n]
    float* be = al + n;
    float* cc = be + n;
    float* dd = cc + n;
    double2* red = (double2*)(((uintptr_t)(dd + n) + 15) & ~(uintptr_t)15);  // [VRED_BLOCK]
    double* redm = (double*)(red + VRED_BLOCK);
    __shared__ double c0s;
    const int t = blockIdx.y;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int od = opidx[j], og = opidx[n + j];
        const double lpd = od >= 0 ? lpl[(size_t)t * nops + od] : 0.0, lpg = og >= 0 ? lpl[(size_t)t * nops + og] : 0.0;
        const double dwd = od >= 0 ? dW[(size_t)t * nops + od] : 0.0, dwg = og >= 0 ? dW[(size_t)t * nops + og] : 0.0;
        const double kap = site[j], skap = site[2 * n + j], sgam = site[3 * n + j];
        al[j] = (float)(-2.0 * lpd * skap);
        be[j] = (float)(dwd * skap);
        cc[j] = (float)(0.5 * kap - 2.0 * lpg * sgam);
        dd[j] = (float)(dwg * sgam);
    }
    if (threadIdx.x == 0) {
        double c0 = 0.0;
        for (int j = 0; j < n; ++j) c0 += 0.5 * site[j] + 2.0 * site[n + j];
        c0s = c0;
    }
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double2 v = make_double2(0, 0);
    if (s < ns) {
        const uint64_t* w = spins + ((size_t)t * ns + s) * W;
        const float2* rs = r + ((size_t)t * ns + s) * n;
        double Ar = 0.0, Ai = 0.0, Vr = 0.0, Vi = 0.0, Cs = 0.0, Ds = 0.0;
        for (int j0 = 0; j0 < n; j0 += 8) {
            const uint64_t word = w[j0 >> 6] >> (j0 & 63);
            float ar = 0.f, ai = 0.f, vr = 0.f, vi = 0.f, cs = 0.f, ds = 0.f;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int j = j0 + jj;
                if (j < n) {
                    const bool up = (word >> jj) & 1ull;
                    const float sg = up ? 1.f : -1.f;
                    cs = fmaf(cc[j], sg, cs);
                    ds = fmaf(dd[j], sg, ds);
                    if (!up) {
                        const float2 rj = rs[j];
                        ar = fmaf(al[j], rj.x, ar);
                        ai = fmaf(al[j], rj.y, ai);
                        vr = fmaf(be[j], rj.x, vr);
                        vi = fmaf(be[j], rj.y, vi);
                    }
                }
            }
            Ar += ar;
            Ai += ai;
            Vr += vr;
            Vi += vi;
            Cs += cs;
            Ds += ds;
        }
        const double br = c0s + Cs + Ar, bi = Ai;
        // E_H: the partials of the site blocks in order (one partial off the tensor-core path)
        double2 E = EH[((size_t)t * ns + s) * nq];
        for (int q = 1; q < nq; ++q) {
            const double2 e = EH[((size_t)t * ns + s) * nq + q];
            E.x += e.x;
            E.y += e.y;
        }
        E.x += 0.5 * bi;
        E.y -= 0.5 * br;
        v = make_double2(dt * E.y + Ds + Vr, -dt * E.x + Vi);
        if (Eeff_out) Eeff_out[(size_t)t * ns + s] = E;
        v_out[(size_t)t * ns + s] = v;
    }
    red[threadIdx.x] = v;
    redm[threadIdx.x] = fmax(fabs(v.x), fabs(v.y));
    __syncthreads();
    for (int st = VRED_BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            red[threadIdx.x].x += red[threadIdx.x + st].x;
            red[threadIdx.x].y += red[threadIdx.x + st].y;
            redm[threadIdx.x] = fmax(redm[threadIdx.x], redm[threadIdx.x + st]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_v[(size_t)t * gridDim.x + blockIdx.x] = red[0];
        part_vmax[(size_t)t * gridDim.x + blockIdx.x] = redm[0];
    }
}

cudaError_t launch_est2(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, bool fp32,
                        const double* dW, double dt, const double* lpl, const EvalBufs& b, double2* Eeff, double2* v,
                        cudaStream_t s) {
    ProfScope prof_(OTVMC_K_EST2, s);
    const otvmc_model* m = a->model;
    const int n = a->n, W = (n + 63) / 64;
    const size_t smem = (size_t)8 * n * 8 + VRED_BLOCK * 24 + 64;
    dim3 grid(v_blocks(ns), ntraj);
    if (fp32)
        est2_mixed_kernel<<<grid, VRED_BLOCK, (size_t)4 * n * 4 + 16 + VRED_BLOCK * 24, s>>>(
            n, W, ns, m->nops, dt, spins, reinterpret_cast<const float2*>(b.r), b.EH,
            est_tc_ok(a, fp32) ? est_tc_nq(n) : 1, m->site_d, m->opidx_d, lpl, dW, Eeff, v, b.part_v, b.part_vmax);
    else
        est2_kernel<double2><<<grid, VRED_BLOCK, smem, s>>>(n, W, ns, m->nops, dt, spins, b.r, b.EH, m->site_d,
                                                            m->opidx_d, lpl, dW, Eeff, v, b.part_v, b.part_vmax);
    count_launch();
    return cudaGetLastError();
}

// Per-CTA sums and max |component| of v (fixed-order tree), for callers that pass v.
__global__ void __launch_bounds__(VRED_BLOCK) vpart_kernel(int ns, const double2* __restrict__ v,
                                                           double2* __restrict__ part_v,
                                                           double* __restrict__ part_vmax) {
    __shared__ double2 red[VRED_BLOCK];
    __shared__ double redm[VRED_BLOCK];
    const int t = blockIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const double2 x = (s < ns) ? v[(size_t)t * ns + s] : make_double2(0.0, 0.0);
    red[threadIdx.x] = x;
    redm[threadIdx.x] = fmax(fabs(x.x), fabs(x.y));
    __syncthreads();
    for (int st = VRED_BLOCK / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) {
            red[threadIdx.x].x += red[threadIdx.x + st].x;
            red[threadIdx.x].y += red[threadIdx.x + st].y;
            redm[threadIdx.x] = fmax(redm[threadIdx.x], redm[threadIdx.x + st]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_v[(size_t)t * gridDim.x + blockIdx.x] = red[0];
        part_vmax[(size_t)t * gridDim.x + blockIdx.x] = redm[0];
    }
}

cudaError_t launch_vpart(int ntraj, int ns, const double2* v, const EvalBufs& b, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_REDUCE, s);
    dim3 grid(v_blocks(ns), ntraj);
    vpart_kernel<<<grid, VRED_BLOCK, 0, s>>>(ns, v, b.part_v, b.part_vmax);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------------ v quantisation
// q(x) = round((v(x) - vbar) 2^e) with e chosen so that |sum_x q| < 2^61; sums of q
// against O = +-1 are then exact int64.  vinfo[t] = {vbar.re, vbar.im, 2^-e, 0}.
__global__ void vquant_kernel(int ns, int vblk, const double2* __restrict__ v, const double2* __restrict__ part_v,
                              const double* __restrict__ part_vmax, long long* __restrict__ qv,
                              double* __restrict__ vinfo, long long* __restrict__ qsum) {
    __shared__ double sh[4];
    __shared__ unsigned long long acc[2];
    const int t = blockIdx.x;
    if (threadIdx.x == 0) {
        double2 m = make_double2(0, 0);
        double mx = 0.0;
        for (int k = 0; k < vblk; ++k) {
            m.x += part_v[(size_t)t * vblk + k].x;
            m.y += part_v[(size_t)t * vblk + k].y;
            mx = fmax(mx, part_vmax[(size_t)t * vblk + k]);
        }
        m.x /= ns;
        m.y /= ns;
        const double bound = mx + fmax(fabs(m.x), fabs(m.y));
        int E = 0;
        if (bound > 0.0) frexp(bound, &E);  // bound < 2^E
        int lg = 0;
        while ((1 << lg) < ns) ++lg;
        const int e = 60 - lg - E;
        sh[0] = m.x;
        sh[1] = m.y;
        sh[2] = ldexp(1.0, e);
        sh[3] = ldexp(1.0, -e);
        acc[0] = acc[1] = 0ull;
    }
    __syncthreads();
    const double mr = sh[0], mi = sh[1], sc = sh[2];
    long long lr = 0, li = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const double2 x = v[(size_t)t * ns + s];
        const long long a = __double2ll_rn((x.x - mr) * sc), b = __double2ll_rn((x.y - mi) * sc);
        qv[((size_t)t * ns + s) * 2] = a;
        qv[((size_t)t * ns + s) * 2 + 1] = b;
        lr += a;
        li += b;
    }
    atomicAdd(&acc[0], (unsigned long long)lr);
    atomicAdd(&acc[1], (unsigned long long)li);
    __syncthreads();
    if (threadIdx.x == 0) {
        qsum[2 * t] = (long long)acc[0];
        qsum[2 * t + 1] = (long long)acc[1];
        vinfo[4 * t] = mr;
        vinfo[4 * t + 1] = mi;
        vinfo[4 * t + 2] = sh[3];
        vinfo[4 * t + 3] = 0.0;
    }
}

cudaError_t launch_vquant(int ntraj, int ns, const double2* v, const EvalBufs& b, cudaStream_t s) {
    ProfScope prof_(OTVMC_K_REDUCE, s);
    vquant_kernel<<<ntraj, 256, 0, s>>>(ns, v_blocks(ns), v, b.part_v, b.part_vmax, b.qv, b.vinfo, b.qsum);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------- observables
// Epm[t][0][j][k] = exp(4 eta_jk), Epm[t][1][j][k] = exp(-4 eta_jk): the two-flip ratio is
// r_jk = r_j r_k exp(4 sigma_j sigma_k eta_jk).
__global__ void obs_prep_kernel(const double2* __restrict__ theta, int P, int n, double2* __restrict__ Epm) {
    const int t = blockIdx.x;
    const double2* th = theta + (size_t)t * P;
    double2* E = Epm + (size_t)t * 2 * n * n;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int j = idx / n, k = idx - j * n;
        double2 p = make_double2(1.0, 0.0), q = make_double2(1.0, 0.0);
        if (j != k) {
            const double2 e = th[n + pair_idx(min(j, k), max(j, k), n)];
            p = cexp_prec(4.0 * e.x, 4.0 * e.y, false);
            q = cexp_prec(-4.0 * e.x, -4.0 * e.y, false);
        }
        E[idx] = p;
        E[n * n + idx] = q;
    }
}

cudaError_t launch_obs_prep(const otvmc_ansatz* a, const double2* theta, int ntraj, bool fp32, const EvalBufs& b,
                            cudaStream_t s) {
    ProfScope prof_(OTVMC_K_OBS, s);
    (void)fp32;
    obs_prep_kernel<<<ntraj, 256, 0, s>>>(theta, (int)a->P, a->n, b.Epm);
    count_launch();
    return cudaGetLastError();
}

// Per sample x and site j: a_j = sum_{k != j} r_k E^{s_j s_k}_jk, b_j = sum_{k != j} s_k r_k E^{..}_jk.
// Then sum_{j != k} r_jk = sum_j r_j a_j, sum_{j != k} s_k r_jk = sum_j r_j b_j,
// sum_{j != k} s_j s_k r_jk = sum_j s_j r_j b_j.  Accumulated per thread:
//  [0] Re r_j              -> m_x      [1] Im s_j r_j        -> m_y   [2] s_j -> m_z
//  [3] Re r_j a_j          -> q_xx     [4] -Re s_j r_j b_j   -> q_yy  [5] (S^2 - n) -> q_zz
//  [6] Im r_j b_j          -> q_xy     [7] Re r_j (S - s_j)  -> q_xz  [8] Im s_j r_j (S - s_j) -> q_yz
template <typename R2>
__device__ __forceinline__ R2 to_r2(double2 v);
template <>
__device__ __forceinline__ double2 to_r2<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 to_r2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }

template <typename R2, typename R, bool SMEM_E>
__global__ void __launch_bounds__(256) observables_kernel(int n, int W, int ns, int spt, const uint64_t* __restrict__ spins,
                                                          const R2* __restrict__ r, const double2* __restrict__ Epm,
                                                          double* __restrict__ part_obs) {
    const int NT = ((n + 31) / 32) * 32;
    const int SPP = 256 / NT;
    const int SB = SPP * spt;
    const int t = blockIdx.y, blk = blockIdx.x;
    const int j = threadIdx.x % NT, g = threadIdx.x / NT;
    const bool active = (g < SPP) && (j < n);
    extern __shared__ __align__(16) unsigned char smraw[];
    const int nE = SMEM_E ? n * n : 0;
    R2* rs = (R2*)smraw;                     // [SPP][NT]
    unsigned char* un = smraw + (size_t)SPP * NT * sizeof(R2);
    R2* E0 = (R2*)un;                        // [n][n] exp(+4 eta) (shared-memory copy)
    R2* E1 = E0 + nE;                        // [n][n] exp(-4 eta)
    double* red = (double*)un;               // [256][9], over the tables once the samples are done
    const double2* G0 = Epm + (size_t)t * 2 * n * n;
    const double2* G1 = G0 + n * n;
    if (SMEM_E)
        for (int i = threadIdx.x; i < 2 * n * n; i += blockDim.x) E0[i] = to_r2<R2>(G0[i]);
    R acc[9];  // per-thread sums over its spt samples (FP32 on the MIXED path), then FP64
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = (R)0;
    for (int q = 0; q < spt; ++q) {
        const int s = blk * SB + g + q * SPP;
        __syncthreads();
        if (active && s < ns) rs[g * NT + j] = r[((size_t)t * ns + s) * n + j];
        __syncthreads();
        if (!(active && s < ns)) continue;
        const uint64_t* w = spins + ((size_t)t * ns + s) * W;
        int S = 0;
        for (int ww = 0; ww < W; ++ww) S += 2 * __popcll(w[ww]);
        S -= n;
        const uint64_t sjb = (w[j >> 6] >> (j & 63)) & 1ull;
        const int sj = sjb ? 1 : -1;
        R2 a2 = {0, 0}, b2 = {0, 0};
        const R2* rr = rs + g * NT;
        // all k, the diagonal included (E^{+}_jj = 1), whose term r_j (and sigma_j r_j) is
        // removed after the loop
        for (int k0 = 0; k0 < n; k0 += 64) {
            uint64_t word = w[k0 >> 6];
            const int kend = min(64, n - k0);
#pragma unroll 4
            for (int kk = 0; kk < kend; ++kk, word >>= 1) {
                const int k = k0 + kk;
                const uint64_t skb = word & 1ull;
                R2 e;
                if (SMEM_E) e = (skb == sjb ? E0 : E1)[k * n + j];
                else e = to_r2<R2>((skb == sjb ? G0 : G1)[k * n + j]);
                const R2 rk = rr[k];
                const R2 p = {rk.x * e.x - rk.y * e.y, rk.x * e.y + rk.y * e.x};
                const R sk = skb ? (R)1 : (R)-1;
                a2.x += p.x;
                a2.y += p.y;
                b2.x = fma(sk, p.x, b2.x);
                b2.y = fma(sk, p.y, b2.y);
            }
        }
        {
            const R2 rjj = rr[j];
            a2.x -= rjj.x;
            a2.y -= rjj.y;
            b2.x -= (R)sj * rjj.x;
            b2.y -= (R)sj * rjj.y;
        }
        const R2 rj = rr[j];
        const R rax = rj.x * a2.x - rj.y * a2.y;
        const R2 rb = {rj.x * b2.x - rj.y * b2.y, rj.x * b2.y + rj.y * b2.x};
        const R fs = (R)sj, fS = (R)(S - sj);
        acc[0] += rj.x;
        acc[1] += fs * rj.y;
        acc[2] += fs;
        acc[3] += rax;
        acc[4] -= fs * rb.x;
        if (j == 0) acc[5] += (R)(S * S - n);
        acc[6] += rb.y;
        acc[7] += rj.x * fS;
        acc[8] += fs * rj.y * fS;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 9; ++i) red[threadIdx.x * 9 + i] = (double)acc[i];
    __syncthreads();
    if (threadIdx.x < 9) {
        double sum = 0.0;
        for (int k = 0; k < 256; ++k) sum += red[k * 9 + threadIdx.x];
        part_obs[((size_t)t * gridDim.x + blk) * 9 + threadIdx.x] = sum;
    }
}

__global__ void obs_final_kernel(int n, int ns, int nblk, const double* __restrict__ part_obs,
                                 double* __restrict__ moments) {
    const int t = blockIdx.x;
    const int i = threadIdx.x;
    if (i >= 9) return;
    double sum = 0.0;
    for (int k = 0; k < nblk; ++k) sum += part_obs[((size_t)t * nblk + k) * 9 + i];
    sum /= ns;
    double out;
    if (i < 3) out = sum / n;
    else out = ((i < 6 ? (double)n : 0.0) + sum) / ((double)n * n);
    moments[(size_t)t * 9 + i] = out;
}

cudaError_t launch_obs_final_n(int n, int ns, int ntraj, int nblk, const EvalBufs& b, double* moments, cudaStream_t s) {
    obs_final_kernel<<<ntraj, 32, 0, s>>>(n, ns, nblk, b.part_obs, moments);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_obs_final(int n, int ns, int ntraj, const EvalBufs& b, double* moments, cudaStream_t s) {
    obs_final_kernel<<<ntraj, 32, 0, s>>>(n, ns, obs_blocks(n, ns), b.part_obs, moments);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_observables(const otvmc_ansatz* a, const uint64_t* spins, int ntraj, int ns, bool fp32,
                               const EvalBufs& b, double* moments, int* status, cudaStream_t s) {
    if (obs_tc_ok(a, fp32) && b.otc != nullptr) return launch_obs_tc(a, spins, ntraj, ns, b, moments, status, s);
    ProfScope prof_(OTVMC_K_OBS, s);
    const int n = a->n, W = (n + 63) / 64;
    const int NT = ((n + 31) / 32) * 32, SPP = 256 / NT;
    const int spt = obs_samples_per_thread();
    const int nblk = obs_blocks(n, ns);
    dim3 grid(nblk, ntraj);
    const size_t el = fp32 ? sizeof(float2) : sizeof(double2);
    // the sample staging, then one region for the exp(+-4 eta) tables and, after them, the
    // final reduction (at N = 64 in FP32: 66 KB, three CTAs per SM)
    const size_t red_b = 256 * 9 * 8, tab_b = 2 * (size_t)n * n * el;
    const size_t base = (size_t)SPP * NT * el + red_b + 64;
    const size_t full = (size_t)SPP * NT * el + (tab_b > red_b ? tab_b : red_b) + 64;
    const bool sm = full <= 200 * 1024;
    const size_t smem = sm ? full : base;
#define OTVMC_OBS_LAUNCH(R2, R, SM)                                                                          \
    do {                                                                                                     \
        cudaFuncSetAttribute(observables_kernel<R2, R, SM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        observables_kernel<R2, R, SM><<<grid, 256, smem, s>>>(n, W, ns, spt, spins,                           \
                                                             reinterpret_cast<const R2*>(b.r), b.Epm, b.part_obs);  \
    } while (0)
    if (fp32) {
        if (sm) OTVMC_OBS_LAUNCH(float2, float, true);
        else OTVMC_OBS_LAUNCH(float2, float, false);
    } else {
        if (sm) OTVMC_OBS_LAUNCH(double2, double, true);
        else OTVMC_OBS_LAUNCH(double2, double, false);
    }
#undef OTVMC_OBS_LAUNCH
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    obs_final_kernel<<<ntraj, 32, 0, s>>>(n, ns, nblk, b.part_obs, moments);
    count_launch();
    return cudaGetLastError();
}

}  // namespace otvmc
