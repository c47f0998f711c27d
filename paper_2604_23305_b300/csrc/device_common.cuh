// Device helpers shared by the kernels: Philox4x32-10, Box-Muller, scan patterns.
#pragma once

#include <stdint.h>

#include "gateau_internal.h"

namespace gateau {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplies with the published multipliers, key bumped by the Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// ln(u) for u = (x + 1/2) 2^-32, accurate to a few ulp over the whole range:
// below 1/2, u is exact enough in float and logf is used; above, 1 - u =
// (~x + 1/2) 2^-32 is formed without cancellation and log1pf(-(1-u)) is used.
__device__ __forceinline__ float log_unit(uint32_t x) {
    if (x < 0x80000000u) {
        return logf(fmaf(static_cast<float>(x), 2.3283064365386963e-10f, 1.1641532182693481e-10f));
    }
    const float v = fmaf(static_cast<float>(~x), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    return log1pf(-v);
}

// cos and sin of 2 pi u_b, u_b = (x_b + 1/2) 2^-32: the angle is shifted by -pi into
// [-pi, pi), where the hardware sin/cos approximations are accurate (absolute error
// ~5e-7), and the results are negated back.
__device__ __forceinline__ float2 cos_sin_2pi_u(uint32_t xb) {
    const float ang = fmaf(static_cast<float>(xb), 1.4629180792671596e-09f, 7.314590396335798e-10f - 3.14159265358979f);
    float sn, cs;
    __sincosf(ang, &sn, &cs);
    return make_float2(-cs, -sn);
}

// Box-Muller pair from two words: r = sqrt(-2 ln u_a), angle 2 pi u_b.
__device__ __forceinline__ float2 box_muller(uint32_t xa, uint32_t xb) {
    const float r = sqrtf(-2.0f * log_unit(xa));
    const float2 cs = cos_sin_2pi_u(xb);
    return make_float2(r * cs.x, r * cs.y);
}

// Four white-noise normals for channels 4q..4q+3 of row (n, i).
__device__ __forceinline__ float4 white_normals4(long long n, int i, int q, uint32_t k0, uint32_t k1) {
    const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(n), static_cast<uint32_t>(n >> 32),
                                             static_cast<uint32_t>(i), static_cast<uint32_t>(q)),
                                  k0, k1);
    const float2 a = box_muller(x.x, x.y);
    const float2 b = box_muller(x.z, x.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

// The same four normals with the hardware approximations of log, sin and cos
// (absolute errors of order 1e-6 in z), used where sigma itself is only known to
// ~1e-3 (the split-BF16 path's noise contractions) and for the pink-noise normals
// (whose filtered output is compared at 1e-4 of its rms).  ln u is clamped at 0 so
// that u within an ulp of 1 gives z = 0, never the root of a negative number; the
// root is the special-function unit's (argument in [0, 44.4], never subnormal).
__device__ __forceinline__ float sqrt_approx(float x) {    // special-function unit, rel. error ~2^-22
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float2 box_muller_fast(uint32_t xa, uint32_t xb) {
    const float ua = fmaf(static_cast<float>(xa), 2.3283064365386963e-10f, 1.1641532182693481e-10f);
    const float r = sqrt_approx(-2.0f * fminf(__logf(ua), 0.f));
    const float2 cs = cos_sin_2pi_u(xb);
    return make_float2(r * cs.x, r * cs.y);
}

__device__ __forceinline__ float4 white_normals4_fast(long long n, int i, int q, uint32_t k0, uint32_t k1) {
    const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(n), static_cast<uint32_t>(n >> 32),
                                             static_cast<uint32_t>(i), static_cast<uint32_t>(q)),
                                  k0, k1);
    const float2 a = box_muller_fast(x.x, x.y);
    const float2 b = box_muller_fast(x.z, x.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Four pink-noise normals for samples 4m..4m+3 of sequence (i, ch).
__device__ __forceinline__ float4 pink_normals4(long long m, int i, int ch, uint32_t k0, uint32_t k1) {
    const uint4 x = philox4x32_10(make_uint4(static_cast<uint32_t>(m), static_cast<uint32_t>(m >> 32),
                                             static_cast<uint32_t>(i), 0x80000000u | static_cast<uint32_t>(ch)),
                                  k0, k1);
    const float2 a = box_muller_fast(x.x, x.y);
    const float2 b = box_muller_fast(x.z, x.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ float f4_get(const float4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

}  // namespace gateau
