// RBM (Eq. 11) push-through solve on the mixed path without materialising O.
//
// For the RBM the log-derivatives are O_a_i = s_i, O_b_m = t_m, O_W_im = s_i t_m (t = tanh
// gamma), so the uncentred kernel over samples factorises exactly:
//     sum_k O_k(x) O_k(x')^* = A + B + A B,
//     A(x, x') = sum_i s_i(x) s_i(x')  (an integer, n - 2 popcount(x xor x')),
//     B(x, x') = sum_m t_m(x) t_m(x')^*.
// Centring with obar (definitions after Eq. 8):
//     T_c(x, x') = sum_k (O_k(x) - obar_k)(O_k(x') - obar_k)^*
//                = A + B + A B - u(x) - u(x')^* + c,
//     u(x) = sum_k O_k(x) obar_k^*  =  s.abar^* + sum_m t_m (bbar_m^* + sum_i s_i Wbar_im^*),
//     c = sum_k |obar_k|^2.
// With u'(x) = u(x) - c/2 the last three terms are -u'(x) - u'(x')^*.  T_c costs
// O(ns^2 (N + M)) instead of the O(ns^2 N M) of the product of materialised rows, and the
// back-projection delta = O_c^+ z / ns of the push-through identity (z the complex solution of
// the size-2 ns system) is, per parameter,
//     a_i: sum_x s_i z - abar_i^* Z,   b_m: sum_x t_m^* z - bbar_m^* Z,
//     W_im: sum_x s_i t_m^* z - Wbar_im^* Z,   Z = sum_x z,   all divided by ns,
// an N x (M+1) product over the samples.  The column means obar are the same product with
// z = 1 and t unconjugated.  The real embedding written for the Cholesky is the one of
// k_rbm.cu: rows x and ns + x, [[Re T_c, -Im T_c], [Im T_c, Re T_c]], upper triangle.
#include "common.cuh"

namespace otvmc {
namespace rbmf {

constexpr int TB = 64;   // complex tile of T_c (samples x samples)
constexpr int MC = 32;   // hidden units per shared-memory chunk

__device__ __forceinline__ bool spin_up(const uint64_t* w, int i) { return (w[i >> 6] >> (i & 63)) & 1ull; }

// obar from the sums with z = 1 (conj = 0): a_i = Wsum[i][M], b_m = csum[m], W_im = Wsum[i][m]
// (delta_mode = 0), or delta from the sums with z the solution (conj = 1): the same entries
// minus obar_k^* Z, Z = csum[M] (delta_mode = 1).  Both divided by ns.
__global__ void finish_kernel(int n, int M, int P, int ns, int delta_mode, const double2* __restrict__ Wsum,
                              const double2* __restrict__ csum, const double2* __restrict__ obar,
                              double2* __restrict__ out) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const double2* Ws = Wsum + (size_t)t * n * (M + 1);
    const double2* cs = csum + (size_t)t * (M + 1);
    double2 v;
    if (k < n) v = Ws[(size_t)k * (M + 1) + M];
    else if (k < n + M) v = cs[k - n];
    else {
        const int q = k - n - M, i = q / M, m = q - i * M;
        v = Ws[(size_t)i * (M + 1) + m];
    }
    if (delta_mode) {
        const double2 Z = cs[M], o = obar[(size_t)t * P + k];
        // v - conj(o) Z
        v.x -= o.x * Z.x + o.y * Z.y;
        v.y -= o.x * Z.y - o.y * Z.x;
    }
    const double inv = 1.0 / ns;
    out[(size_t)t * P + k] = make_double2(v.x * inv, v.y * inv);
}

// u'(x) = sum_k O_k(x) obar_k^* - c/2 for 32 samples per CTA, thread = hidden unit m (M <= 256):
// h_m = bbar_m^* + sum_i s_i Wbar_im^*, then sum_m t_m h_m (warp shuffles, then over warps),
// plus s.abar^* and - c/2 (c summed in FP64 in a fixed order by every CTA alike).
__global__ void __launch_bounds__(256) center_kernel(int n, int M, int W, int P, int ns,
                                                     const uint64_t* __restrict__ spins,
                                                     const float2* __restrict__ Tf, const double2* __restrict__ obar,
                                                     float2* __restrict__ up) {
    const int t = blockIdx.y, x0 = blockIdx.x * 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ uint64_t sb[32][4];
    __shared__ double cred[256];
    __shared__ float2 red[8][32];
    const double2* ob = obar + (size_t)t * P;
    const uint64_t* sp = spins + (size_t)t * ns * W;
    double cp = 0.0;
    for (int k = tid; k < P; k += 256) cp += ob[k].x * ob[k].x + ob[k].y * ob[k].y;
    cred[tid] = cp;
    if (tid < 32 * W) {
        const int s = tid / W, w = tid - s * W;
        sb[s][w] = x0 + s < ns ? sp[(size_t)(x0 + s) * W + w] : 0ull;
    }
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) cred[tid] += cred[tid + h];
        __syncthreads();
    }
    const double c = cred[0];
    const int m = tid;
    float2 acc[32];
    if (m < M) {
        const double2 bb = ob[n + m];
#pragma unroll
        for (int s = 0; s < 32; ++s) acc[s] = make_float2((float)bb.x, -(float)bb.y);
        for (int i = 0; i < n; ++i) {
            const double2 wb = ob[n + M + (size_t)i * M + m];
            const float wr = (float)wb.x, wi = -(float)wb.y;
#pragma unroll
            for (int s = 0; s < 32; ++s) {
                const bool u = (sb[s][i >> 6] >> (i & 63)) & 1ull;
                acc[s].x += u ? wr : -wr;
                acc[s].y += u ? wi : -wi;
            }
        }
        const float2* Tm = Tf + ((size_t)t * M + m) * ns;
#pragma unroll
        for (int s = 0; s < 32; ++s) {
            const float2 tv = x0 + s < ns ? Tm[x0 + s] : make_float2(0.f, 0.f);
            acc[s] = make_float2(tv.x * acc[s].x - tv.y * acc[s].y, tv.x * acc[s].y + tv.y * acc[s].x);
        }
    } else {
#pragma unroll
        for (int s = 0; s < 32; ++s) acc[s] = make_float2(0.f, 0.f);
    }
    // reduce over the 32 hidden units of each warp: lane s ends with sample s's partial sum
#pragma unroll
    for (int s = 0; s < 32; ++s) {
        float vr = acc[s].x, vi = acc[s].y;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, off);
            vi += __shfl_xor_sync(0xffffffffu, vi, off);
        }
        if (lane == s) red[warp][s] = make_float2(vr, vi);
    }
    __syncthreads();
    if (tid < 32 && x0 + tid < ns) {
        float ur = 0.f, ui = 0.f;
        for (int w = 0; w < 8; ++w) {
            ur += red[w][tid].x;
            ui += red[w][tid].y;
        }
        float arr = 0.f, aii = 0.f;
        for (int i = 0; i < n; ++i) {
            const double2 ab = ob[i];
            const bool u = (sb[tid][i >> 6] >> (i & 63)) & 1ull;
            arr += u ? (float)ab.x : -(float)ab.x;
            aii += u ? -(float)ab.y : (float)ab.y;
        }
        up[(size_t)t * ns + x0 + tid] = make_float2((float)((double)(ur + arr) - 0.5 * c), ui + aii);
    }
}

// Upper tiles I <= J (64 x 64 samples) of the embedded T_c, one per CTA:
//   Re T_c at (x, x') and (ns + x, ns + x'); -Im T_c at (x, ns + x'); for I < J also
//   -Im T_c(x', x) = Im T_c(x, x') at (x', ns + x) (through a shared-memory transpose).
// Thread (ty, tx) owns rows 4 ty .. 4 ty + 3 and columns 4 tx .. 4 tx + 3 of the tile.
__global__ void __launch_bounds__(256) tc_kernel(int n, int M, int W, int ns, const uint64_t* __restrict__ spins,
                                                 const float2* __restrict__ Tf, const float2* __restrict__ up,
                                                 float* __restrict__ G) {
    const int t = blockIdx.y;
    int J = (int)((sqrtf(8.f * (float)blockIdx.x + 1.f) - 1.f) * 0.5f);
    while ((J + 1) * (J + 2) / 2 <= (int)blockIdx.x) ++J;
    while (J * (J + 1) / 2 > (int)blockIdx.x) --J;
    const int I = blockIdx.x - J * (J + 1) / 2;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    // the two t chunks, and after the products the transposed imaginary parts, share memory
    constexpr int RAW = 4 * MC * TB > TB * (TB + 1) ? 4 * MC * TB : TB * (TB + 1);
    __shared__ __align__(16) float raw[RAW];
    float2(*tr)[TB] = reinterpret_cast<float2(*)[TB]>(raw);
    float2(*tcl)[TB] = reinterpret_cast<float2(*)[TB]>(raw + 2 * MC * TB);
    float(*tim)[TB + 1] = reinterpret_cast<float(*)[TB + 1]>(raw);
    __shared__ uint64_t sbr[TB][4], sbc[TB][4];
    __shared__ float2 ur[TB], uc[TB];
    const float2* Tt = Tf + (size_t)t * M * ns;
    const uint64_t* sp = spins + (size_t)t * ns * W;
    const int xr0 = I * TB, xc0 = J * TB;
    for (int e = tid; e < TB * W; e += 256) {
        const int s = e / W, w = e - s * W;
        sbr[s][w] = xr0 + s < ns ? sp[(size_t)(xr0 + s) * W + w] : 0ull;
        sbc[s][w] = xc0 + s < ns ? sp[(size_t)(xc0 + s) * W + w] : 0ull;
    }
    if (tid < TB) {
        ur[tid] = xr0 + tid < ns ? up[(size_t)t * ns + xr0 + tid] : make_float2(0.f, 0.f);
        uc[tid] = xc0 + tid < ns ? up[(size_t)t * ns + xc0 + tid] : make_float2(0.f, 0.f);
    }
    float br[4][4], bi[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) br[a][b] = bi[a][b] = 0.f;
    for (int m0 = 0; m0 < M; m0 += MC) {
        __syncthreads();
        for (int e = tid; e < MC * TB; e += 256) {
            const int mm = e / TB, xs = e - mm * TB, m = m0 + mm;
            tr[mm][xs] = (m < M && xr0 + xs < ns) ? Tt[(size_t)m * ns + xr0 + xs] : make_float2(0.f, 0.f);
            tcl[mm][xs] = (m < M && xc0 + xs < ns) ? Tt[(size_t)m * ns + xc0 + xs] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int mm = 0; mm < MC; ++mm) {
            const float4 r01 = *reinterpret_cast<const float4*>(&tr[mm][4 * ty]);
            const float4 r23 = *reinterpret_cast<const float4*>(&tr[mm][4 * ty + 2]);
            const float4 c01 = *reinterpret_cast<const float4*>(&tcl[mm][4 * tx]);
            const float4 c23 = *reinterpret_cast<const float4*>(&tcl[mm][4 * tx + 2]);
            const float rx[4] = {r01.x, r01.z, r23.x, r23.z}, ry[4] = {r01.y, r01.w, r23.y, r23.w};
            const float cx[4] = {c01.x, c01.z, c23.x, c23.z}, cy[4] = {c01.y, c01.w, c23.y, c23.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    // t(x) t(x')^*
                    br[a][b] = fmaf(rx[a], cx[b], fmaf(ry[a], cy[b], br[a][b]));
                    bi[a][b] = fmaf(ry[a], cx[b], fmaf(-rx[a], cy[b], bi[a][b]));
                }
        }
    }
    const size_t ld = 2 * (size_t)ns;
    float* Gt = G + (size_t)t * ld * ld;
    float vre[4][4], vim[4][4];
    __syncthreads();  // the last chunk's reads are done before tim overwrites it
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = 4 * ty + a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int cc = 4 * tx + b;
            int pc = 0;
            for (int w = 0; w < W; ++w) {
                const int lo = 64 * w, valid = n - lo < 64 ? n - lo : 64;
                const uint64_t mask = valid == 64 ? ~0ull : ((1ull << valid) - 1ull);
                pc += __popcll((sbr[r][w] ^ sbc[cc][w]) & mask);
            }
            const float A = (float)(n - 2 * pc);
            vre[a][b] = fmaf(A, 1.f + br[a][b], br[a][b]) - ur[r].x - uc[cc].x;
            vim[a][b] = fmaf(A, bi[a][b], bi[a][b]) - ur[r].y + uc[cc].y;
            tim[cc][r] = vim[a][b];
        }
    }
    const bool vec = (ns & 3) == 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int x = xr0 + 4 * ty + a, xc = xc0 + 4 * tx;
        if (x >= ns) continue;
        float* row0 = Gt + (size_t)x * ld;
        float* row1 = Gt + (size_t)(ns + x) * ld + ns;
        float* row2 = Gt + (size_t)x * ld + ns;
        if (vec && xc + 3 < ns) {
            *reinterpret_cast<float4*>(row0 + xc) = make_float4(vre[a][0], vre[a][1], vre[a][2], vre[a][3]);
            *reinterpret_cast<float4*>(row1 + xc) = make_float4(vre[a][0], vre[a][1], vre[a][2], vre[a][3]);
            *reinterpret_cast<float4*>(row2 + xc) = make_float4(-vim[a][0], -vim[a][1], -vim[a][2], -vim[a][3]);
        } else {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (xc + b < ns) {
                    row0[xc + b] = vre[a][b];
                    row1[xc + b] = vre[a][b];
                    row2[xc + b] = -vim[a][b];
                }
        }
    }
    if (I == J) return;
    __syncthreads();
    // (x', ns + x) = Im T_c(x, x') for x' in tile J, x in tile I: rows along x'
    for (int e = tid; e < TB * TB; e += 256) {
        const int cc = e / TB, r = e - cc * TB;
        const int xp = xc0 + cc, x = xr0 + r;
        if (xp < ns && x < ns) Gt[(size_t)xp * ld + ns + x] = tim[cc][r];
    }
}

// [Re v_c; Im v_c] as real parts of double2 (the embedded right-hand side of the T system)
__global__ void rhs_kernel(int ns, const double2* __restrict__ v, const double* __restrict__ vinfo,
                           double2* __restrict__ u) {
    const int t = blockIdx.y;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= 2 * ns) return;
    const double2 vv = v[(size_t)t * ns + (x < ns ? x : x - ns)];
    const double val = x < ns ? vv.x - vinfo[4 * t] : vv.y - vinfo[4 * t + 1];
    u[(size_t)t * 2 * ns + x] = make_double2(val, 0.0);
}

// ------------------------------------------------------------------ refinement
// The FP32 T_c (and the FP32-level factor of T_c + eps I) carry errors of ~1e-7 of |T_c|, which
// the solve amplifies by up to |T_c| / eps.  The solution is therefore refined against the
// exact operator, applied through the same factorisation of O without forming T:
//     y = O_c^+ z / ns   (column sums, as for delta),
//     r = v_c - eps z - O_c y,   z += (L L^T)^-1 r.
// Every sum over sites or samples with a +-1 sign is taken exactly in 64-bit fixed point (one
// power-of-two scale per trajectory or column, chosen from a bound of the terms so that no sum
// can overflow), and only products and the final conversions are FP64: sums of the FP64 pipe's
// speed would cost more than the rest of the evaluation.

// tanh z = s (1 - w) / (1 + w), w = exp(-2 s z), s = sign(Re z), in FP64
__device__ __forceinline__ double2 ctanh_d(double2 z) {
    const double s = z.x >= 0.0 ? 1.0 : -1.0;
    const double e = exp(-2.0 * s * z.x);
    double sn, cs;
    sincos(2.0 * z.y, &sn, &cs);
    const double wr = e * cs, wi = -s * e * sn;
    const double nr = 1.0 - wr, ni = -wi, dr = 1.0 + wr, di = wi;
    const double inv = 1.0 / (dr * dr + di * di);
    return make_double2(s * (nr * dr + ni * di) * inv, s * (ni * dr - nr * di) * inv);
}

// Largest power of two 2^e with amax * cnt * 2^e < 2^62 (1 if amax is zero or not finite).
__device__ __forceinline__ double fx_scale(double amax, int cnt) {
    if (!(amax > 0.0) || !(amax < 1e300)) return 1.0;
    int ex;
    frexp(amax * (double)cnt, &ex);  // amax cnt < 2^ex
    return ldexp(1.0, 62 - ex);
}
__device__ __forceinline__ long long fxq(double v, double sc) { return __double2ll_rn(v * sc); }

struct ll2 {
    long long x, y;
};

// Per trajectory: the W block of a P-vector (theta for gamma, y for the residual) in fixed point,
// Wq[t][i][m] = round(W_im sc), Wqs[t][m] = sum_i Wq[t][i][m], with sc = 2^e and
// (|Re W| + |Im W|)_max N sc < 2^62.  One CTA per trajectory.
__global__ void __launch_bounds__(256) wquant_kernel(int n, int M, int P, const double2* __restrict__ src,
                                                     ll2* __restrict__ Wq, ll2* __restrict__ Wqs,
                                                     double* __restrict__ scale) {
    const int t = blockIdx.x, tid = threadIdx.x;
    __shared__ double red[256];
    const double2* Ws = src + (size_t)t * P + n + M;
    double mx = 0.0;
    for (int k = tid; k < n * M; k += 256) mx = fmax(mx, fabs(Ws[k].x) + fabs(Ws[k].y));
    red[tid] = mx;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) red[tid] = fmax(red[tid], red[tid + h]);
        __syncthreads();
    }
    const double sc = fx_scale(red[0], n);
    ll2* q = Wq + (size_t)t * n * M;
    for (int m = tid; m < M; m += 256) {
        long long sx = 0, sy = 0;
        for (int i = 0; i < n; ++i) {
            const double2 w = Ws[(size_t)i * M + m];
            const ll2 v{fxq(w.x, sc), fxq(w.y, sc)};
            q[(size_t)i * M + m] = v;
            sx += v.x;
            sy += v.y;
        }
        Wqs[(size_t)t * M + m] = ll2{sx, sy};
    }
    if (tid == 0) scale[t] = sc;
}

constexpr int AS = 16;  // samples per CTA of the per-sample kernels (thread = hidden unit)

// dn[q] = sum over the sites i with s_i(x_q) = -1 of Wq[i][m], for AS samples, so that
// sum_i s_i W_im = (Wqs_m - 2 dn) / sc exactly (the lanes of a warp share the sample: the test
// does not diverge).
__device__ __forceinline__ void down_sums(int n, int M, int m, const ll2* __restrict__ q, const uint64_t (*sb)[4],
                                          long long (&dx)[AS], long long (&dy)[AS]) {
#pragma unroll
    for (int k = 0; k < AS; ++k) dx[k] = dy[k] = 0;
    for (int i = 0; i < n; ++i) {
        const ll2 w = q[(size_t)i * M + m];
#pragma unroll
        for (int k = 0; k < AS; ++k)
            if (!((sb[k][i >> 6] >> (i & 63)) & 1ull)) {
                dx[k] += w.x;
                dy[k] += w.y;
            }
    }
}

// t_m(x) = tanh(b_m + sum_i W_im s_i(x)) with the site sum exact (fixed point) and tanh in FP64,
// laid out [t][m][x] in FP64 and (Tf not null) rounded to FP32; fmax[t] (the bits of a positive
// double, cleared by the caller) receives max(1, max_x,m |Re t| + |Im t|).  AS samples per CTA,
// thread = hidden unit.
__global__ void __launch_bounds__(256) tanh_fx_kernel(int n, int M, int W, int P, int ns,
                                                      const double2* __restrict__ theta,
                                                      const uint64_t* __restrict__ spins, const ll2* __restrict__ Wq,
                                                      const ll2* __restrict__ Wqs, const double* __restrict__ scale,
                                                      double2* __restrict__ Td, float2* __restrict__ Tf,
                                                      unsigned long long* __restrict__ fmax_bits) {
    const int t = blockIdx.y, x0 = blockIdx.x * AS, tid = threadIdx.x;
    __shared__ uint64_t sb[AS][4];
    __shared__ double red[256];
    const uint64_t* sp = spins + (size_t)t * ns * W;
    if (tid < AS * W) {
        const int k = tid / W, w = tid - k * W;
        sb[k][w] = x0 + k < ns ? sp[(size_t)(x0 + k) * W + w] : 0ull;
    }
    __syncthreads();
    const int m = tid;
    double mx = 1.0;
    if (m < M) {
        long long dx[AS], dy[AS];
        down_sums(n, M, m, Wq + (size_t)t * n * M, sb, dx, dy);
        const double inv = 1.0 / scale[t];
        const ll2 qs = Wqs[(size_t)t * M + m];
        const double2 b = theta[(size_t)t * P + n + m];
        double2* Tm = Td + ((size_t)t * M + m) * ns;
        float2* Fm = Tf ? Tf + ((size_t)t * M + m) * ns : nullptr;
#pragma unroll
        for (int k = 0; k < AS; ++k) {
            if (x0 + k >= ns) break;
            const double2 g = make_double2(b.x + (double)(qs.x - 2 * dx[k]) * inv, b.y + (double)(qs.y - 2 * dy[k]) * inv);
            const double2 tv = ctanh_d(g);
            Tm[x0 + k] = tv;
            if (Fm) Fm[x0 + k] = make_float2((float)tv.x, (float)tv.y);
            mx = fmax(mx, fabs(tv.x) + fabs(tv.y));
        }
    }
    red[tid] = mx;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (tid < h) red[tid] = fmax(red[tid], red[tid + h]);
        __syncthreads();
    }
    if (tid == 0) atomicMax(fmax_bits + t, (unsigned long long)__double_as_longlong(red[0]));
}

constexpr int XD = 32;  // samples per chunk of the column sums

// Column sums over the samples, for columns c = 0..M (c = M stands for the constant 1):
//     Wsum[t][i][c] = sum_x s_i(x) f_c(x) z(x),   csum[t][c] = sum_x f_c(x) z(x),
// with f_c = t_c^* (conj = 1) or t_c (conj = 0), and z = 1 when zr is null, else
// z(x) = zr[x].x + i zr[ns + x].x (real parts of the double2 solution of the embedded system).
// One CTA per (32 columns, 64 sites, trajectory); lane = column, warp = site residue mod 8.
// f z in FP64, then in fixed point with one scale per CTA from the bound fmax[t] zmax; per site
// the sum is taken as (sum over all samples) - 2 (sum over the samples where s_i = -1), exactly:
// the lanes of a warp share sample and site, so the test does not diverge.
__global__ void __launch_bounds__(256) colsum_fx_kernel(int n, int M, int W, int ns, int conj,
                                                        const uint64_t* __restrict__ spins,
                                                        const double2* __restrict__ Td,
                                                        const unsigned long long* __restrict__ fmax_bits,
                                                        const double2* __restrict__ zr, double2* __restrict__ Wsum,
                                                        double2* __restrict__ csum) {
    const int t = blockIdx.z, ib = blockIdx.y, c0 = blockIdx.x * 32;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ ll2 fz[XD][33];
    __shared__ uint64_t sb[XD];
    __shared__ double2 zs[XD];
    __shared__ double red[256];
    const double2* Tt = Td + (size_t)t * M * ns;
    const uint64_t* sp = spins + (size_t)t * ns * W;
    const double2* zt = zr ? zr + (size_t)t * 2 * ns : nullptr;
    double zm = 1.0;
    if (zt) {
        zm = 0.0;
        for (int x = tid; x < ns; x += 256) zm = fmax(zm, fabs(zt[x].x) + fabs(zt[ns + x].x));
    }
    red[tid] = zm;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) red[tid] = fmax(red[tid], red[tid + h]);
        __syncthreads();
    }
    const double sc = fx_scale(__longlong_as_double((long long)fmax_bits[t]) * red[0], ns);
    const int c = c0 + lane;
    long long tx = 0, ty = 0, dx[8], dy[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) dx[r] = dy[r] = 0;
    for (int x0 = 0; x0 < ns; x0 += XD) {
        __syncthreads();
        if (tid < XD) {
            const int x = x0 + tid;
            double2 z = make_double2(0.0, 0.0);
            uint64_t word = 0ull;
            if (x < ns) {
                z = zt ? make_double2(zt[x].x, zt[ns + x].x) : make_double2(1.0, 0.0);
                word = sp[(size_t)x * W + ib];
            }
            zs[tid] = z;
            sb[tid] = word;
        }
        __syncthreads();
        for (int e = tid; e < XD * 32; e += 256) {
            const int l = e / XD, xs = e - l * XD;
            const int cc = c0 + l, x = x0 + xs;
            double2 f = make_double2(0.0, 0.0);
            if (x < ns && cc <= M) {
                f = cc < M ? Tt[(size_t)cc * ns + x] : make_double2(1.0, 0.0);
                if (conj) f.y = -f.y;
            }
            const double2 w = cmul(f, zs[xs]);
            fz[xs][l] = ll2{fxq(w.x, sc), fxq(w.y, sc)};
        }
        __syncthreads();
        const int xe = ns - x0 < XD ? ns - x0 : XD;
        for (int xs = 0; xs < xe; ++xs) {
            const ll2 v = fz[xs][lane];
            const uint64_t word = sb[xs] >> warp;
            tx += v.x;
            ty += v.y;
#pragma unroll
            for (int r = 0; r < 8; ++r)
                if (!((word >> (8 * r)) & 1ull)) {
                    dx[r] += v.x;
                    dy[r] += v.y;
                }
        }
    }
    if (c > M) return;
    const double inv = 1.0 / sc;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int i = ib * 64 + warp + 8 * r;
        if (i < n)
            Wsum[((size_t)t * n + i) * (M + 1) + c] =
                make_double2((double)(tx - 2 * dx[r]) * inv, (double)(ty - 2 * dy[r]) * inv);
    }
    if (ib == 0 && warp == 0) csum[(size_t)t * (M + 1) + c] = make_double2((double)tx * inv, (double)ty * inv);
}

// r(x) = v_c(x) - eps z(x) - sum_k (O_k(x) - obar_k) y_k for AS samples per CTA, thread = hidden
// unit m (M <= 256):  sum_k O_k(x) y_k = s.y_a + sum_m t_m(x) (y_b_m + sum_i s_i y_W_im), the site
// sums exact in fixed point (Yq, Yqs, yscale from wquant_kernel on y), the products with t and
// the sum over m in FP64.  v_c, z and r are the embedded vectors: .x of [Re; Im] with ns entries each.
__global__ void __launch_bounds__(256) resid_fx_kernel(int n, int M, int W, int P, int ns, double eps,
                                                       const uint64_t* __restrict__ spins,
                                                       const double2* __restrict__ Td, const double2* __restrict__ obar,
                                                       const double2* __restrict__ y, const ll2* __restrict__ Yq,
                                                       const ll2* __restrict__ Yqs, const double* __restrict__ yscale,
                                                       const double2* __restrict__ rhs, const double2* __restrict__ z,
                                                       double2* __restrict__ r) {
    const int t = blockIdx.y, x0 = blockIdx.x * AS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    __shared__ uint64_t sb[AS][4];
    __shared__ double cr[256], ci[256];
    __shared__ double2 red[8][AS];
    const double2* yt = y + (size_t)t * P;
    const double2* ob = obar + (size_t)t * P;
    const uint64_t* sp = spins + (size_t)t * ns * W;
    double pr = 0.0, pi = 0.0;
    for (int k = tid; k < P; k += blockDim.x) {
        const double2 o = ob[k], v = yt[k];
        pr += o.x * v.x - o.y * v.y;
        pi += o.x * v.y + o.y * v.x;
    }
    cr[tid] = pr;
    ci[tid] = pi;
    if (tid < AS * W) {
        const int k = tid / W, w = tid - k * W;
        sb[k][w] = x0 + k < ns ? sp[(size_t)(x0 + k) * W + w] : 0ull;
    }
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (tid < h) {
            cr[tid] += cr[tid + h];
            ci[tid] += ci[tid + h];
        }
        __syncthreads();
    }
    const int m = tid;
    double2 acc[AS];
    if (m < M) {
        long long dx[AS], dy[AS];
        down_sums(n, M, m, Yq + (size_t)t * n * M, sb, dx, dy);
        const double inv = 1.0 / yscale[t];
        const ll2 qs = Yqs[(size_t)t * M + m];
        const double2 yb = yt[n + m];
        const double2* Tm = Td + ((size_t)t * M + m) * ns;
#pragma unroll
        for (int k = 0; k < AS; ++k) {
            const double2 tv = x0 + k < ns ? Tm[x0 + k] : make_double2(0.0, 0.0);
            acc[k] = cmul(tv, make_double2(yb.x + (double)(qs.x - 2 * dx[k]) * inv,
                                           yb.y + (double)(qs.y - 2 * dy[k]) * inv));
        }
    } else {
#pragma unroll
        for (int k = 0; k < AS; ++k) acc[k] = make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int k = 0; k < AS; ++k) {
        double vr = acc[k].x, vi = acc[k].y;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            vr += __shfl_xor_sync(0xffffffffu, vr, off);
            vi += __shfl_xor_sync(0xffffffffu, vi, off);
        }
        if (lane == k) red[warp][k] = make_double2(vr, vi);
    }
    __syncthreads();
    if (tid < AS && x0 + tid < ns) {
        const int x = x0 + tid;
        double orr = -cr[0], oi = -ci[0];
        for (int w = 0; w < nw; ++w) {
            orr += red[w][tid].x;
            oi += red[w][tid].y;
        }
        for (int i = 0; i < n; ++i) {
            const double2 ya = yt[i];
            if ((sb[tid][i >> 6] >> (i & 63)) & 1ull) {
                orr += ya.x;
                oi += ya.y;
            } else {
                orr -= ya.x;
                oi -= ya.y;
            }
        }
        const size_t b = (size_t)t * 2 * ns;
        r[b + x] = make_double2(rhs[b + x].x - eps * z[b + x].x - orr, 0.0);
        r[b + ns + x] = make_double2(rhs[b + ns + x].x - eps * z[b + ns + x].x - oi, 0.0);
    }
}

// S path (P <= ns): the embedded right-hand side of a correction, [Re; Im] of g - eps delta
// (g = O_c^+ w / ns with w = v_c - O_c delta), and the complex delta from the embedded solution.
__global__ void sres_kernel(int P, double eps, const double2* __restrict__ g, const double2* __restrict__ delta,
                            double2* __restrict__ r) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const double2 gv = g[(size_t)t * P + k], d = delta[(size_t)t * P + k];
    r[(size_t)t * 2 * P + k] = make_double2(gv.x - eps * d.x, 0.0);
    r[(size_t)t * 2 * P + P + k] = make_double2(gv.y - eps * d.y, 0.0);
}
__global__ void unembed_kernel(int P, const double2* __restrict__ xe, double2* __restrict__ delta) {
    const int t = blockIdx.y;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    delta[(size_t)t * P + k] = make_double2(xe[(size_t)t * 2 * P + k].x, xe[(size_t)t * 2 * P + P + k].x);
}

static size_t rup(size_t b) { return (b + 255) & ~(size_t)255; }
// threads of the per-sample kernels (thread = hidden unit): a power of two >= M
static int hid_threads(int M) { return M <= 128 ? 128 : 256; }

// fixed-point tables of one W block per trajectory (wquant_kernel)
struct FxTab {
    ll2* q;
    ll2* qs;
    double* scale;
};
static size_t fxtab_bytes(size_t n, size_t M, size_t T) { return rup(T * n * M * 16) + rup(T * M * 16) + rup(T * 8); }
template <typename Take>
static FxTab take_fxtab(Take& take, size_t n, size_t M, size_t T) {
    FxTab f;
    f.q = (ll2*)take(T * n * M * 16);
    f.qs = (ll2*)take(T * M * 16);
    f.scale = (double*)take(T * 8);
    return f;
}

}  // namespace rbmf

size_t rbm_tanh_obar_bytes(const otvmc_ansatz* a, int ntraj) {
    using namespace rbmf;
    const size_t M = (size_t)a->m, n = (size_t)a->n, T = (size_t)ntraj;
    return fxtab_bytes(n, M, T) + rup(T * n * (M + 1) * 16) + rup(T * (M + 1) * 16) + 256;
}

// t_m(x) = tanh gamma_m(x) in FP64 [T][M][ns] (Td) and FP32 (Tf, optional), the bound fmax [T]
// of |Re t| + |Im t| for the column sums, and obar [T][P] in FP64, with the site and sample sums
// exact in fixed point.
cudaError_t launch_rbm_tanh_obar(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins, int T, int ns,
                                 double2* Td, float2* Tf, unsigned long long* fmax, double2* obar, void* ws,
                                 cudaStream_t s) {
    using namespace rbmf;
    const int P = (int)a->P, n = a->n, M = a->m, W = (n + 63) / 64;
    char* q = (char*)ws;
    auto take = [&](size_t b) {
        char* r = q;
        q += rup(b);
        return (void*)r;
    };
    const FxTab wt = take_fxtab(take, n, M, T);
    double2* Wsum = (double2*)take((size_t)T * n * (M + 1) * 16);
    double2* csum = (double2*)take((size_t)T * (M + 1) * 16);
    cudaError_t e = cudaMemsetAsync(fmax, 0, (size_t)T * 8, s);
    if (e != cudaSuccess) return e;
    ProfScope prof_(OTVMC_K_OBUILD, s);
    wquant_kernel<<<T, 256, 0, s>>>(n, M, P, theta, wt.q, wt.qs, wt.scale);
    tanh_fx_kernel<<<dim3((ns + AS - 1) / AS, T), hid_threads(M), 0, s>>>(n, M, W, P, ns, theta, spins, wt.q, wt.qs,
                                                                          wt.scale, Td, Tf, fmax);
    colsum_fx_kernel<<<dim3((M + 1 + 31) / 32, W, T), 256, 0, s>>>(n, M, W, ns, 0, spins, Td, fmax, nullptr, Wsum,
                                                                   csum);
    finish_kernel<<<dim3((P + 255) / 256, T), 256, 0, s>>>(n, M, P, ns, 0, Wsum, csum, nullptr, obar);
    count_launch(4);
    return cudaGetLastError();
}

size_t rbm_refine_bytes(const otvmc_ansatz* a, int ntraj, int ns) {
    using namespace rbmf;
    const size_t P = (size_t)a->P, M = (size_t)a->m, n = (size_t)a->n, T = (size_t)ntraj, S = (size_t)ns;
    return rup(T * 2 * S * 16) + rup(T * P * 16) + rup(T * n * (M + 1) * 16) + rup(T * (M + 1) * 16) +
           rup(T * 2 * P * 16) + fxtab_bytes(n, M, T) + 256;
}

// Corrections of the push-through solve (see above) and delta = O_c^+ z / ns: z [T][2 ns] the
// embedded solution of the FP32 system (in/out), rhs the embedded v_c, Td the FP64 tanh gamma
// [T][M][ns] with its bound fmax, obar the FP64 column means, chol the workspace of the solve that
// produced z.
cudaError_t launch_rbm_refine_push(const otvmc_ansatz* a, int T, int ns, double eps, int iters,
                                   const uint64_t* spins, const double2* Td, const unsigned long long* fmax,
                                   const double2* obar, const double2* rhs, double2* z, void* chol, void* ws,
                                   double2* delta, cudaStream_t s) {
    using namespace rbmf;
    const int P = (int)a->P, n = a->n, M = a->m, W = (n + 63) / 64;
    char* q = (char*)ws;
    auto take = [&](size_t b) {
        char* r = q;
        q += rup(b);
        return (void*)r;
    };
    double2* r = (double2*)take((size_t)T * 2 * ns * 16);
    double2* y = (double2*)take((size_t)T * P * 16);
    double2* Wsum = (double2*)take((size_t)T * n * (M + 1) * 16);
    double2* csum = (double2*)take((size_t)T * (M + 1) * 16);
    take((size_t)T * 2 * P * 16);
    const FxTab yt = take_fxtab(take, n, M, T);
    const dim3 cs_grid((M + 1 + 31) / 32, W, T);
    for (int it = 0; it <= iters; ++it) {
        double2* out = it == iters ? delta : y;
        {
            ProfScope prof_(OTVMC_K_D, s);
            colsum_fx_kernel<<<cs_grid, 256, 0, s>>>(n, M, W, ns, 1, spins, Td, fmax, z, Wsum, csum);
            finish_kernel<<<dim3((P + 255) / 256, T), 256, 0, s>>>(n, M, P, ns, 1, Wsum, csum, obar, out);
            count_launch(2);
        }
        if (it == iters) break;
        {
            ProfScope prof_(OTVMC_K_RESID, s);
            wquant_kernel<<<T, 256, 0, s>>>(n, M, P, y, yt.q, yt.qs, yt.scale);
            resid_fx_kernel<<<dim3((ns + AS - 1) / AS, T), hid_threads(M), 0, s>>>(
                n, M, W, P, ns, eps, spins, Td, obar, y, yt.q, yt.qs, yt.scale, rhs, z, r);
            count_launch(2);
        }
        cudaError_t e = launch_chol_tc_resolve(T, 2 * ns, chol, r, z, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// The same corrections on the S path (P <= ns): the solve is (S + eps I) delta = D with
// S = O_c^+ O_c / ns, D = O_c^+ v_c / ns, so the residual D - (S + eps I) delta is
// O_c^+ (v_c - O_c delta) / ns - eps delta.  xe [T][2P] is the embedded solution of the FP32
// system (in/out), vemb [T][2 ns] the embedded v_c; delta receives the refined solution.
cudaError_t launch_rbm_refine_S(const otvmc_ansatz* a, int T, int ns, double eps, int iters, const uint64_t* spins,
                                const double2* Td, const unsigned long long* fmax, const double2* obar,
                                const double2* vemb, double2* xe, void* chol, void* ws, double2* delta,
                                cudaStream_t s) {
    using namespace rbmf;
    const int P = (int)a->P, n = a->n, M = a->m, W = (n + 63) / 64;
    char* q = (char*)ws;
    auto take = [&](size_t b) {
        char* r = q;
        q += rup(b);
        return (void*)r;
    };
    double2* w = (double2*)take((size_t)T * 2 * ns * 16);
    double2* g = (double2*)take((size_t)T * P * 16);
    double2* Wsum = (double2*)take((size_t)T * n * (M + 1) * 16);
    double2* csum = (double2*)take((size_t)T * (M + 1) * 16);
    double2* re = (double2*)take((size_t)T * 2 * P * 16);
    const FxTab dt = take_fxtab(take, n, M, T);
    const dim3 cs_grid((M + 1 + 31) / 32, W, T);
    const dim3 pg((P + 255) / 256, T);
    for (int it = 0; it <= iters; ++it) {
        unembed_kernel<<<pg, 256, 0, s>>>(P, xe, delta);
        count_launch();
        if (it == iters) break;
        {
            ProfScope prof_(OTVMC_K_RESID, s);
            // w = v_c - O_c delta (eps = 0: the z term vanishes)
            wquant_kernel<<<T, 256, 0, s>>>(n, M, P, delta, dt.q, dt.qs, dt.scale);
            resid_fx_kernel<<<dim3((ns + AS - 1) / AS, T), hid_threads(M), 0, s>>>(
                n, M, W, P, ns, 0.0, spins, Td, obar, delta, dt.q, dt.qs, dt.scale, vemb, vemb, w);
            colsum_fx_kernel<<<cs_grid, 256, 0, s>>>(n, M, W, ns, 1, spins, Td, fmax, w, Wsum, csum);
            finish_kernel<<<pg, 256, 0, s>>>(n, M, P, ns, 1, Wsum, csum, obar, g);
            sres_kernel<<<pg, 256, 0, s>>>(P, eps, g, delta, re);
            count_launch(5);
        }
        cudaError_t e = launch_chol_tc_resolve(T, 2 * P, chol, re, xe, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

size_t rbm_factored_bytes(const otvmc_ansatz* a, int ntraj, int ns) {
    using rbmf::rup;
    const size_t P = (size_t)a->P, M = (size_t)a->m, T = (size_t)ntraj, S = (size_t)ns;
    return rup(T * M * S * 8) + rup(T * M * S * 16) + rup(T * P * 16) + rup(T * S * 8) + rup(T * 4 * S * S * 4) +
           rup(T * 2 * S * 8) + 2 * rup(T * 2 * S * 16) + rup(T * 8) + rbm_tanh_obar_bytes(a, ntraj) +
           rbm_refine_bytes(a, ntraj, ns) + chol_ws_bytes(ntraj, (int)(2 * S), OTVMC_PREC_MIXED) + 1024;
}

// Build + solve of one evaluation on the T path (P > ns) of the mixed RBM path, factored:
// t in FP64 (and its FP32 rounding), obar, u', the embedded T_c in FP32, the tensor-core
// Cholesky of size 2 ns, then RBM_REFINE_FACTORED corrections against the exact operator and delta
// from the exact column sums of the solution.
cudaError_t launch_rbm_build_solve_factored(const otvmc_ansatz* a, const double2* theta, const uint64_t* spins,
                                            const double2* v, const double* vinfo, int T, int ns, double eps,
                                            void* ws, double2* delta, int* status, cudaStream_t s) {
    using namespace rbmf;
    const int P = (int)a->P, n = a->n, M = a->m, W = (n + 63) / 64;
    char* q = (char*)ws;
    auto take = [&](size_t b) {
        char* r = q;
        q += rup(b);
        return (void*)r;
    };
    float2* Tf = (float2*)take((size_t)T * M * ns * 8);
    double2* Td = (double2*)take((size_t)T * M * ns * 16);
    double2* obar = (double2*)take((size_t)T * P * 16);
    float2* up = (float2*)take((size_t)T * ns * 8);
    float* G = (float*)take((size_t)T * 4 * ns * ns * 4);
    double* zero = (double*)take((size_t)T * 2 * ns * 8);
    double2* rhs = (double2*)take((size_t)T * 2 * ns * 16);
    double2* sol = (double2*)take((size_t)T * 2 * ns * 16);
    unsigned long long* fmax = (unsigned long long*)take((size_t)T * 8);
    void* tws = take(rbm_tanh_obar_bytes(a, T));
    void* rws = take(rbm_refine_bytes(a, T, ns));
    void* chol = q;
    cudaError_t e = launch_rbm_tanh_obar(a, theta, spins, T, ns, Td, Tf, fmax, obar, tws, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope prof_(OTVMC_K_OBUILD, s);
        center_kernel<<<dim3((ns + 31) / 32, T), 256, 0, s>>>(n, M, W, P, ns, spins, Tf, obar, up);
        rhs_kernel<<<dim3((2 * ns + 255) / 256, T), 256, 0, s>>>(ns, v, vinfo, rhs);
        count_launch(2);
    }
    {
        ProfScope prof_(OTVMC_K_GRAM, s);
        const int nt = (ns + TB - 1) / TB;
        tc_kernel<<<dim3(nt * (nt + 1) / 2, T), 256, 0, s>>>(n, M, W, ns, spins, Tf, up, G);
        count_launch();
    }
    e = cudaMemsetAsync(zero, 0, (size_t)T * 2 * ns * 8, s);
    if (e != cudaSuccess) return e;
    // (T~ + eps I) y = v~ with T~ = G / ns (no refinement against the FP32 G: the corrections
    // below are taken against the exact operator)
    e = launch_chol_solve(T, 2 * ns, ns, OTVMC_PREC_MIXED, eps, nullptr, G, zero, rhs, sol, nullptr, chol, 0, status,
                          s);
    if (e != cudaSuccess) return e;
    return launch_rbm_refine_push(a, T, ns, eps, RBM_REFINE_FACTORED, spins, Td, fmax, obar, rhs, sol, chol, rws,
                                  delta, s);
}

}  // namespace otvmc
