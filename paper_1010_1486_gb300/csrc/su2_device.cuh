// su2_device.cuh -- device building blocks of the SU(2) heat bath (sm_103a).
//
// Quaternion algebra of SU(2) (Sec. 2 of Cardoso & Bicudo, LAT2010), the
// Philox4x32-10 counter generator (Salmon et al., SC'11), and log / exp /
// sin-cos(2 pi u) written from textbook series.  Every floating-point
// operation of the link path is an explicit round-to-nearest intrinsic
// (__fmul_rn, __fadd_rn, __fmaf_rn, __fdiv_rn, __fsqrt_rn), so the compiler
// can neither contract nor reassociate it: the results are a fixed function of
// the inputs, the same on every run and every launch shape.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace su2 {

// ---------------------------------------------------------------- Philox
// Philox4x32-10: ten rounds; each round multiplies words 0 and 2 by the two
// round constants (full 64-bit products), xors the high halves with words
// 1, 3 and the key, and the key advances by the two Weyl constants.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform in (0, 1]: the top 24 bits plus one, times 2^-24 (exact).
__device__ __forceinline__ float uniform01(uint32_t w)
{
    return __fmul_rn(__uint2float_rn((w >> 8) + 1u), 5.9604644775390625e-8f);
}

// Stream kinds of the counter word c2 = (kind << 3) | (parity << 2) | mu.
enum StreamKind : uint32_t { kCreutz = 0, kDirection = 1, kHotStart = 2, kLearned = 3 };

__device__ __forceinline__ uint4 draw(uint32_t k0, uint32_t k1, uint32_t eo, uint32_t sweep, uint32_t kind,
                                      uint32_t parity, uint32_t mu, uint32_t block)
{
    return philox4x32_10(make_uint4(eo, sweep, (kind << 3) | (parity << 2) | mu, block), k0, k1);
}

// ------------------------------------------------------ elementary functions
// ln 2 = kLn2Hi + kLn2Lo with kLn2Hi = 2839/4096 (12 significant bits, so
// n * kLn2Hi is exact for the exponents met here).
constexpr float kLn2Hi = 2839.0f / 4096.0f;
constexpr float kLn2Lo = 3.19461849e-05f;
constexpr float kInvLn2 = 1.44269502f;
constexpr float kSqrt2 = 1.41421354f;
constexpr float kHalfPi = 1.57079637f;

// log(x), x > 0 normal.  x = 2^k m, m in [1/sqrt2, sqrt2); with
// s = (m-1)/(m+1), log m = 2 atanh s = 2 (s + s^3/3 + ... + s^11/11).
__device__ __forceinline__ float log_series(float x)
{
    const uint32_t bits = __float_as_uint(x);
    int k = (int)((bits >> 23) & 0xffu) - 127;
    float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
    if (m > kSqrt2) {
        m = __fmul_rn(m, 0.5f);
        k += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float z = __fmul_rn(s, s);
    float q = __fmaf_rn(z, 1.0f / 11.0f, 1.0f / 9.0f);
    q = __fmaf_rn(q, z, 1.0f / 7.0f);
    q = __fmaf_rn(q, z, 1.0f / 5.0f);
    q = __fmaf_rn(q, z, 1.0f / 3.0f);
    const float s2 = __fmul_rn(2.0f, s);
    const float lm = __fmaf_rn(__fmul_rn(s2, z), q, s2);
    const float kf = (float)k;
    return __fmaf_rn(kf, kLn2Hi, __fmaf_rn(kf, kLn2Lo, lm));
}

// exp(y), y in [-87, 0]: y = n ln2 + r (Cody-Waite), e^r by its Taylor series
// to degree 7, times 2^n built in the exponent field.
__device__ __forceinline__ float exp_series(float y)
{
    const float n = floorf(__fadd_rn(__fmul_rn(y, kInvLn2), 0.5f));
    float r = __fmaf_rn(-n, kLn2Hi, y);
    r = __fmaf_rn(-n, kLn2Lo, r);
    float p = 1.0f / 5040.0f;
    p = __fmaf_rn(p, r, 1.0f / 720.0f);
    p = __fmaf_rn(p, r, 1.0f / 120.0f);
    p = __fmaf_rn(p, r, 1.0f / 24.0f);
    p = __fmaf_rn(p, r, 1.0f / 6.0f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    const int ni = (int)n;
    return __fmul_rn(p, __uint_as_float((uint32_t)(ni + 127) << 23));
}

// sin(2 pi u), cos(2 pi u) for u in [0, 1]: 4u = q + f with q the nearest
// integer (|f| <= 1/2, exact), x = f pi/2, Taylor series on |x| <= pi/4,
// then q quarter turns.
__device__ __forceinline__ void sincos_2pi(float u, float &sn, float &cs)
{
    const float w = __fmul_rn(4.0f, u);
    const float q = floorf(__fadd_rn(w, 0.5f));
    const float f = __fsub_rn(w, q);
    const float x = __fmul_rn(f, kHalfPi);
    const float z = __fmul_rn(x, x);
    float ps = __fmaf_rn(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = __fmaf_rn(ps, z, 1.0f / 120.0f);
    ps = __fmaf_rn(ps, z, -1.0f / 6.0f);
    const float s = __fmaf_rn(__fmul_rn(x, z), ps, x);
    float pc = __fmaf_rn(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = __fmaf_rn(pc, z, -1.0f / 720.0f);
    pc = __fmaf_rn(pc, z, 1.0f / 24.0f);
    pc = __fmaf_rn(pc, z, -0.5f);
    const float c = __fmaf_rn(z, pc, 1.0f);
    switch (((int)q) & 3) {
    case 0: sn = s; cs = c; break;
    case 1: sn = c; cs = -s; break;
    case 2: sn = -s; cs = -c; break;
    default: sn = -c; cs = s; break;
    }
}

// ------------------------------------------------------------- quaternions
// float4 (x, y, z, w) = (a0, a1, a2, a3) of U = a0 + i a.sigma.
// Four-term sums are the fixed chain p0 q0 + (p1 q1 + (p2 q2 + p3 q3)).
__device__ __forceinline__ float chain4(float p0, float q0, float p1, float q1, float p2, float q2, float p3,
                                        float q3)
{
    return __fmaf_rn(p0, q0, __fmaf_rn(p1, q1, __fmaf_rn(p2, q2, __fmul_rn(p3, q3))));
}

// (a b)_0 = a0 b0 - a.b ; (a b)_vec = a0 b + b0 a - a x b
__device__ __forceinline__ float4 qmul(float4 a, float4 b)
{
    return make_float4(chain4(a.x, b.x, -a.y, b.y, -a.z, b.z, -a.w, b.w),
                       chain4(a.x, b.y, a.y, b.x, -a.z, b.w, a.w, b.z),
                       chain4(a.x, b.z, a.z, b.x, -a.w, b.y, a.y, b.w),
                       chain4(a.x, b.w, a.w, b.x, -a.y, b.z, a.z, b.y));
}

// Real part only: (1/2) Tr(a b).
__device__ __forceinline__ float qmul_re(float4 a, float4 b)
{
    return chain4(a.x, b.x, -a.y, b.y, -a.z, b.z, -a.w, b.w);
}

__device__ __forceinline__ float4 qdag(float4 a) { return make_float4(a.x, -a.y, -a.z, -a.w); }

__device__ __forceinline__ float4 qadd(float4 a, float4 b)
{
    return make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
}

__device__ __forceinline__ float qnorm2(float4 a) { return chain4(a.x, a.x, a.y, a.y, a.z, a.z, a.w, a.w); }

// ------------------------------------------------------------ heat bath
constexpr int kMaxTrials = 4096;

// Heat-bath draw of one link from its staple v (Sec. 2).
//   k = |v| = sqrt(det V), U~^dag = v^dag / k
//   a0 ~ sqrt(1 - a0^2) exp(beta k a0): Creutz's method -- a0 = 1 + ln(x)/(beta k),
//     x uniform in [exp(-2 beta k), 1], kept iff r2^2 <= 1 - a0^2; trial t uses
//     words 2(t&1), 2(t&1)+1 of Creutz block t>>1.  beta k < 1e-6: a0 = 2 r1 - 1
//     with the same test (the Haar marginal); beta k > 43: exp(-2 beta k) -> 0.
//   direction: c = 2 u0 - 1, phi = 2 pi u1 from direction block 0;
//   a = (a0, r s cos phi, r s sin phi, r c), r = sqrt(1-a0^2), s = sqrt(1-c^2);
//   U' = a U~^dag.
// Returns the trial count (>= 1) or 0 if kMaxTrials trials were rejected.
__device__ __forceinline__ int heatbath_draw(float4 v, float beta, uint32_t k0, uint32_t k1, uint32_t eo,
                                             uint32_t sweep, uint32_t parity, uint32_t mu, float4 &out)
{
    const float k = __fsqrt_rn(qnorm2(v));
    float4 ut = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    if (k > 0.0f) {
        const float inv_k = __fdiv_rn(1.0f, k);
        ut = make_float4(__fmul_rn(v.x, inv_k), __fmul_rn(-v.y, inv_k), __fmul_rn(-v.z, inv_k),
                         __fmul_rn(-v.w, inv_k));
    }
    const float bk = __fmul_rn(beta, k);
    const bool haar = bk < 1e-6f;
    float e = 0.0f;
    if (!haar && bk <= 43.0f) e = exp_series(__fmul_rn(-2.0f, bk));
    const float one_minus_e = __fsub_rn(1.0f, e);

    float a0 = 0.0f;
    int trials = 0;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    for (int t = 0; t < kMaxTrials; ++t) {
        if ((t & 1) == 0) w = draw(k0, k1, eo, sweep, kCreutz, parity, mu, (uint32_t)(t >> 1));
        const float r1 = uniform01((t & 1) ? w.z : w.x);
        const float r2 = uniform01((t & 1) ? w.w : w.y);
        float cand;
        if (haar) {
            cand = __fsub_rn(__fmul_rn(2.0f, r1), 1.0f);
        } else {
            const float x = __fmaf_rn(r1, one_minus_e, e);
            cand = __fadd_rn(1.0f, __fdiv_rn(log_series(x), bk));
        }
        cand = cand < -1.0f ? -1.0f : (cand > 1.0f ? 1.0f : cand);
        if (__fmul_rn(r2, r2) <= __fmaf_rn(-cand, cand, 1.0f)) {
            a0 = cand;
            trials = t + 1;
            break;
        }
    }
    if (trials == 0) return 0;

    const uint4 d = draw(k0, k1, eo, sweep, kDirection, parity, mu, 0u);
    const float r = __fsqrt_rn(__fmaf_rn(-a0, a0, 1.0f));
    const float c = __fsub_rn(__fmul_rn(2.0f, uniform01(d.x)), 1.0f);
    const float st = __fsqrt_rn(__fmaf_rn(-c, c, 1.0f));
    float sn, cs;
    sincos_2pi(uniform01(d.y), sn, cs);
    const float rs = __fmul_rn(r, st);
    const float4 a = make_float4(a0, __fmul_rn(rs, cs), __fmul_rn(rs, sn), __fmul_rn(r, c));
    out = qmul(a, ut);
    return trials;
}

// --------------------------------------------------------------- geometry
// Lattice Ns^3 x Nt, lex = ((t Ns + z) Ns + y) Ns + x, parity (x+y+z+t)&1,
// even/odd index i = lex >> 1.  Links: float4 array, element (mu, parity, i)
// at (2 mu + parity) vh + i, vh = V/2.
struct Geom {
    int ns, nt;
    int vh;   // V / 2
    int vs;   // Ns^3
};

struct Coord {
    int c[4];
};

// Site of parity p with even/odd index i.
__device__ __forceinline__ Coord eo_to_coord(const Geom &g, int i, int p)
{
    const int lex0 = 2 * i;
    Coord r;
    int rest = lex0 / g.ns;
    const int x0 = lex0 - rest * g.ns;
    const int rest2 = rest / g.ns;
    r.c[1] = rest - rest2 * g.ns;
    r.c[3] = rest2 / g.ns;
    r.c[2] = rest2 - r.c[3] * g.ns;
    r.c[0] = x0 + ((r.c[1] + r.c[2] + r.c[3] + p) & 1);
    return r;
}

__device__ __forceinline__ int coord_to_eo(const Geom &g, const Coord &x)
{
    return (((x.c[3] * g.ns + x.c[2]) * g.ns + x.c[1]) * g.ns + x.c[0]) >> 1;
}

__device__ __forceinline__ int extent(const Geom &g, int mu) { return mu == 3 ? g.nt : g.ns; }

__device__ __forceinline__ Coord step(const Geom &g, Coord x, int mu, int s)
{
    const int L = extent(g, mu);
    int v = x.c[mu] + s;
    v = v < 0 ? v + L : (v >= L ? v - L : v);
    x.c[mu] = v;
    return x;
}

__device__ __forceinline__ size_t link_index(const Geom &g, int mu, int parity, int eo)
{
    return (size_t)(2 * mu + parity) * (size_t)g.vh + (size_t)eo;
}

}  // namespace su2
