// Device-side random draws for EMPC breeding (Algorithm 1 cold start, parent
// draws, crossover, mutation gate and N(0, sigma) noise; Sec. V).
//
// Counter-based: every draw is Philox4x32-10 (Salmon et al., SC'11) of the
// counter (candidate, generation, purpose, block) under the key (seed lo,
// seed hi), so a candidate's draws do not depend on the launch shape.  All
// FP32 arithmetic uses round-to-nearest intrinsics, which the compiler never
// contracts or reorders, so the results are bit-reproducible on any host that
// performs the same IEEE operations in the same order.
#pragma once
#include <cstdint>

namespace empc {

enum : uint32_t { kDrawInit = 0, kDrawParents = 1, kDrawCross = 2, kDrawGate = 3, kDrawNoise = 4 };

struct Words4 {
    uint32_t w[4];
};

// Philox4x32-10: ten rounds of the 4-word Philox S-box with multipliers
// 0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ Words4 philox10(uint32_t c0, uint32_t c1, uint32_t c2,
                                           uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one widening multiply gives both halves of each 32 x 32 -> 64 product
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c0 = n0;
        c1 = (uint32_t)p1;
        c2 = n2;
        c3 = (uint32_t)p0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    Words4 o;
    o.w[0] = c0;
    o.w[1] = c1;
    o.w[2] = c2;
    o.w[3] = c3;
    return o;
}

__device__ __forceinline__ Words4 draw(uint64_t seed, uint32_t cand, uint32_t gen,
                                       uint32_t purpose, uint32_t block) {
    return philox10(cand, gen, purpose, block, (uint32_t)(seed & 0xFFFFFFFFull),
                    (uint32_t)(seed >> 32));
}

// [0, 1) with 24 random bits, and (0, 1].
__device__ __forceinline__ float unit_closed_open(uint32_t r) {
    return __fmul_rn((float)(r >> 8), 0x1p-24f);
}
__device__ __forceinline__ float unit_open_closed(uint32_t r) {
    return __fmul_rn((float)((r >> 8) + 1u), 0x1p-24f);
}

// ln(u), u in (0, 1] normal.  Split u = 2^e f with f folded into
// [sqrt(1/2), sqrt(2)], then ln f = 2 atanh(s), s = (f-1)/(f+1), from the
// odd power series of atanh through s^11 (|s| < 0.172).
__device__ __forceinline__ float ln_unit(float u) {
    const uint32_t bits = __float_as_uint(u);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    float f = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    if (f > 1.41421356f) {
        f = __fmul_rn(f, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float c = 1.0f / 11.0f;
    c = __fmaf_rn(c, s2, 1.0f / 9.0f);
    c = __fmaf_rn(c, s2, 1.0f / 7.0f);
    c = __fmaf_rn(c, s2, 1.0f / 5.0f);
    c = __fmaf_rn(c, s2, 1.0f / 3.0f);
    const float t = __fmul_rn(s2, c);
    const float s_twice = __fmul_rn(2.0f, s);
    const float lnf = __fmaf_rn(s_twice, t, s_twice);
    return __fmaf_rn((float)e, 0.693147180559945309f, lnf);
}

// sin and cos of 2 pi (r24 / 2^24).  The octant (top 3 of the 24 bits) and
// the in-octant fraction are exact; odd octants are reflected (1 - fraction,
// exact) so that the series argument stays in [0, pi/4], where the Taylor
// series of sin through phi^9 and cos through phi^10 suffice.
__device__ __forceinline__ void sincos_turn(uint32_t r24, float* sin_out, float* cos_out) {
    const uint32_t oct = (r24 >> 21) & 7u;
    float frac = __fmul_rn((float)(r24 & 0x1FFFFFu), 0x1p-21f);
    uint32_t quadrant;
    const bool reflect = (oct & 1u) != 0u;
    if (reflect) {
        frac = __fsub_rn(1.0f, frac);
        quadrant = ((oct + 1u) >> 1) & 3u;
    } else {
        quadrant = (oct >> 1) & 3u;
    }
    const float phi = __fmul_rn(frac, 0.785398163397448310f);
    const float p2 = __fmul_rn(phi, phi);
    float ks = 1.0f / 362880.0f;
    ks = __fmaf_rn(ks, p2, -1.0f / 5040.0f);
    ks = __fmaf_rn(ks, p2, 1.0f / 120.0f);
    ks = __fmaf_rn(ks, p2, -1.0f / 6.0f);
    const float p3 = __fmul_rn(p2, phi);
    float sv = __fmaf_rn(p3, ks, phi);
    float kc = -1.0f / 3628800.0f;
    kc = __fmaf_rn(kc, p2, 1.0f / 40320.0f);
    kc = __fmaf_rn(kc, p2, -1.0f / 720.0f);
    kc = __fmaf_rn(kc, p2, 1.0f / 24.0f);
    kc = __fmaf_rn(kc, p2, -0.5f);
    const float cv = __fmaf_rn(p2, kc, 1.0f);
    if (reflect) sv = -sv;
    float so, co;
    switch (quadrant) {
        case 0: so = sv; co = cv; break;
        case 1: so = cv; co = -sv; break;
        case 2: so = -sv; co = -cv; break;
        default: so = -cv; co = sv; break;
    }
    *sin_out = so;
    *cos_out = co;
}

// Box-Muller pair from two words: radius sqrt(-2 ln u1), u1 in (0, 1],
// angle 2 pi u2, u2 in [0, 1).
__device__ __forceinline__ void gauss_pair(uint32_t ra, uint32_t rb, float* z0, float* z1) {
    const float l = ln_unit(unit_open_closed(ra));
    const float rad = __fsqrt_rn(__fmul_rn(-2.0f, l));
    float s, c;
    sincos_turn(rb >> 8, &s, &c);
    *z0 = __fmul_rn(rad, c);
    *z1 = __fmul_rn(rad, s);
}

__device__ __forceinline__ float clamp_to(float v, float lo, float hi) {
    return fminf(fmaxf(v, lo), hi);
}

// Parent rank in [0, E) from one word: floor(r E / 2^32).
__device__ __forceinline__ int parent_rank(uint32_t r, int E) {
    return (int)(((uint64_t)r * (uint64_t)E) >> 32);
}

// Byte b of a decision stream (one Philox block per 16 bytes).
__device__ __forceinline__ uint32_t stream_byte(uint64_t seed, uint32_t cand, uint32_t gen,
                                                uint32_t purpose, uint32_t b) {
    const Words4 o = draw(seed, cand, gen, purpose, b >> 4);
    return (o.w[(b >> 2) & 3u] >> (8u * (b & 3u))) & 0xFFu;
}

}  // namespace empc
