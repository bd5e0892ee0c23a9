// Device-side helpers shared by the otVMC kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace otvmc {

// ------------------------------------------------------------------------ status word
// Status area at the start of every workspace: word 0 holds the first error code
// recorded on the device since the last otvmc_check; word 1 a detail (e.g. trajectory).
__device__ __forceinline__ void record_error(int* status, int code, int detail) {
    if (status == nullptr) return;
    if (atomicCAS(status, 0, code) == 0) atomicExch(status + 1, detail);
}

// --------------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of two 32x32->64 multiplications with
// the round keys bumped by the Weyl constants between rounds.
struct u32x4 { uint32_t x, y, z, w; };

__device__ __forceinline__ u32x4 philox(u32x4 c, uint32_t k0, uint32_t k1) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    }
    return c;
}

constexpr uint32_t TAG_SAMPLE = 1u, TAG_NOISE = 2u, TAG_INIT = 3u;

__device__ __forceinline__ double u01(uint32_t w) { return ((double)w + 0.5) * 0x1.0p-32; }

// --------------------------------------------------------------------- fixed point
// Real-valued fields sum_k c_k sigma_k with sigma = +-1 are accumulated exactly as int64
// multiples of 2^-FX_BITS, so their value does not depend on summation order.
constexpr int FX_BITS = 48;
constexpr double FX_SCALE = 281474976710656.0;      // 2^48
constexpr double FX_INV = 1.0 / 281474976710656.0;  // 2^-48
// |coefficient| * 2^48 must stay below this so that N of them cannot overflow int64.
__device__ __forceinline__ long long fx_quant(double x) { return __double2ll_rn(x * FX_SCALE); }
// 2 pi in units of 2^-48, rounded to the nearest integer
constexpr long long FX_TWO_PI = 1768559438007110LL;
// v 2^-48 in FP32 without FP64 arithmetic: high word (exact below 2^24) plus low word
__device__ __forceinline__ float fx_to_float(long long v) {
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)(v & 0xffffffffll);
    return fmaf((float)hi, 0x1.0p-16f, (float)lo * 0x1.0p-48f);
}

// ------------------------------------------------------------------------ misc
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int spin_of(const uint64_t* w, int j) {
    return ((w[j >> 6] >> (j & 63)) & 1ull) ? 1 : -1;
}

// exp(z) in FP64 (precision FP64) or with FP32 transcendentals after an FP64 reduction of
// the phase to [-pi, pi] (precision MIXED).
__device__ __forceinline__ double2 cexp_prec(double re, double im, bool fp32) {
    if (!fp32) {
        double s, c;
        sincos(im, &s, &c);
        const double e = exp(re);
        return make_double2(e * c, e * s);
    }
    const double k = rint(im * 0.15915494309189535);  // im / (2 pi)
    const double red = fma(-k, 6.283185307179586, im);
    float s, c;
    sincosf((float)red, &s, &c);
    const float e = expf((float)re);
    return make_double2((double)(e * c), (double)(e * s));
}

}  // namespace otvmc
