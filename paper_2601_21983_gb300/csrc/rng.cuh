// Counter-based draws shared by the kernels: Philox4x32-10 (Salmon et al.,
// SC 2011) and the Box-Muller transform.  Normal e of a (seed, stream,
// iteration) sequence comes from block q = e / 4 with counter
// (q mod 2^32, q >> 32, iteration, stream) and key (seed mod 2^32, seed >> 32).
#pragma once

#include <stdint.h>

namespace smc {

// ------------------------------------------------------------ Philox4x32-10
// Salmon et al., SC 2011: ten rounds of two 32x32->64 multiplies, Weyl key bumps.
static __device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Box-Muller on (u1, u2) = ((x0 + 1) 2^-32, x1 2^-32).  ln u1 is taken through
// log1p of (u1 - 1) = -(~x0) 2^-32 when u1 > 1/2 so that u1 near 1 keeps its
// precision in float32.
static __device__ __forceinline__ float2 box_muller(uint32_t x0, uint32_t x1) {
    float lnu;
    if (x0 < 0x80000000u)
        lnu = logf(((float)x0 + 1.0f) * 2.3283064365386963e-10f);
    else
        lnu = log1pf(-(float)(~x0) * 2.3283064365386963e-10f);
    const float r = sqrtf(-2.0f * lnu);
    float s, co;
    sincospif((float)x1 * 4.656612873077393e-10f, &s, &co);
    return make_float2(r * co, r * s);
}

static __device__ __forceinline__ void normals4(uint64_t seed, uint32_t sid, uint32_t it, uint64_t q, float out[4]) {
    const uint4 x = philox10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), it, sid),
                             make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float2 a = box_muller(x.x, x.y), b = box_muller(x.z, x.w);
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

}  // namespace smc
