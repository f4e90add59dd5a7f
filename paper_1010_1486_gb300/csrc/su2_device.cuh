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
// Philox4x32-10: ten rounds; each multiplies words 0 and 2 by the two round
// constants (full 64-bit products) and xors the high halves with words 1, 3
// and the round key; the key advances by the two Weyl constants per round.
// Round keys (k0 + r W0, k1 + r W1), r = 0..9, are computed once and passed
// by value, so in a kernel parameter they are read from the constant bank.
struct RoundKeys {
    uint32_t k0[10], k1[10];
};

__host__ __device__ inline RoundKeys make_round_keys(uint32_t a, uint32_t b)
{
    RoundKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k0[r] = a;
        rk.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return rk;
}

inline RoundKeys make_round_keys(uint64_t seed) { return make_round_keys((uint32_t)seed, (uint32_t)(seed >> 32)); }

__device__ __forceinline__ uint4 philox_rk(uint4 c, const RoundKeys &rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ rk.k0[round], lo1, hi0 ^ c.w ^ rk.k1[round], lo0);
    }
    return c;
}

// Two blocks under the same key, round by round: each round key is fetched
// once for both, and the two independent chains interleave.
__device__ __forceinline__ void philox2_rk(uint4 &a, uint4 &b, const RoundKeys &rk)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t k0 = rk.k0[round], k1 = rk.k1[round];
        const uint32_t alo0 = 0xD2511F53u * a.x, ahi0 = __umulhi(0xD2511F53u, a.x);
        const uint32_t alo1 = 0xCD9E8D57u * a.z, ahi1 = __umulhi(0xCD9E8D57u, a.z);
        const uint32_t blo0 = 0xD2511F53u * b.x, bhi0 = __umulhi(0xD2511F53u, b.x);
        const uint32_t blo1 = 0xCD9E8D57u * b.z, bhi1 = __umulhi(0xCD9E8D57u, b.z);
        a = make_uint4(ahi1 ^ a.y ^ k0, alo1, ahi0 ^ a.w ^ k1, alo0);
        b = make_uint4(bhi1 ^ b.y ^ k0, blo1, bhi0 ^ b.w ^ k1, blo0);
    }
}

// The same generator with the key schedule computed on the fly (for kernels
// whose key varies per work item, e.g. one seed per lattice of a batch).
__device__ __forceinline__ uint4 philox_key(uint4 c, uint32_t k0, uint32_t k1)
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

// Uniform in (0, 1]: the top 24 bits plus one, times 2^-24, formed as
// (w >> 8) 2^-24 + 2^-24 with one fused multiply-add (every step exact, so it
// is the same number as ((w >> 8) + 1) 2^-24).
__device__ __forceinline__ float uniform01(uint32_t w)
{
    return __fmaf_rn(__uint2float_rn(w >> 8), 5.9604644775390625e-8f, 5.9604644775390625e-8f);
}

// Uniform for the argument of a logarithm: w 2^-32 + 2^-33 from the whole
// word (w rounded to nearest, then one fused multiply-add), in [2^-33, 1].
// Creutz's x is uniform on [exp(-2 beta k), 1] (Sec. 2); from 24 bits -ln x
// would stop at 16.6 and cut away the law's tail beta k (1 - a0) > 16.6
// (2.8e-7 of its mass at large beta k, about +4e-7 on the plaquette at
// beta = 6); from the whole word the cut is at 22.9 (mass 6e-10).
__device__ __forceinline__ float uniform_log(uint32_t w)
{
    return __fmaf_rn(__uint2float_rn(w), 0x1p-32f, 0x1p-33f);
}

// Counter of a draw: (even/odd site index, sweep, (kind << 3) | (parity << 2) | mu, block).
enum StreamKind : uint32_t { kCreutz = 0, kDirection = 1, kHotStart = 2, kLearned = 3 };

__device__ __forceinline__ uint32_t stream_word(uint32_t kind, uint32_t parity, uint32_t mu)
{
    return (kind << 3) | (parity << 2) | mu;
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
    // q quarter turns: (s, c), (c, -s), (-s, -c), (-c, s) for q mod 4 = 0..3,
    // as selects (negation is exact)
    const int qi = (int)q;
    const float a = (qi & 1) ? c : s;
    const float b = (qi & 1) ? s : c;
    sn = (qi & 2) ? -a : a;
    cs = ((qi + 1) & 2) ? -b : b;
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

// a b + c: the chains of qmul with the innermost product fused with c's
// component (one rounding per component), as the staple accumulates its terms.
__device__ __forceinline__ float4 qmul_add(float4 a, float4 b, float4 c)
{
    return make_float4(__fmaf_rn(a.x, b.x, __fmaf_rn(-a.y, b.y, __fmaf_rn(-a.z, b.z, __fmaf_rn(-a.w, b.w, c.x)))),
                       __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(-a.z, b.w, __fmaf_rn(a.w, b.z, c.y)))),
                       __fmaf_rn(a.x, b.z, __fmaf_rn(a.z, b.x, __fmaf_rn(-a.w, b.y, __fmaf_rn(a.y, b.w, c.z)))),
                       __fmaf_rn(a.x, b.w, __fmaf_rn(a.w, b.x, __fmaf_rn(-a.y, b.z, __fmaf_rn(a.z, b.y, c.w)))));
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
constexpr float kHaarBelow = 1e-6f;  // beta k below this: a0 from the Haar marginal
// beta k above this: exp(-2 beta k) is not computed and taken as 0.  It
// changes no draw: for beta k > 21, e = exp(-2 beta k) < exp(-42) < 2^-60, so
// 1 - e rounds to 1 and x = r1 (1 - e) + e rounds to r1 for every log uniform
// r1 >= 2^-33 (uniform_log's smallest value), whose half ulp is at least
// 2^-57 > e.  The definition keeps e up to beta k = 43, where it leaves the
// binary32 normal range; between 21 and 43 it makes no difference to x.
// (A cutoff of 17 was wrong: there e ~ 2^-49 moves x = r1 for r1 below about
// 2^-26, i.e. for the smallest words.)
constexpr float kExpCutoff = 21.0f;

// Normalised staple (Sec. 2): k = |v| = sqrt(det V), U~^dag = v^dag / k
// (identity if k = 0), bk = beta k, e = exp(-2 beta k) (0 when beta k >
// kExpCutoff, where it changes no draw, or on the Haar branch).
struct DrawSetup {
    float4 ut;
    float bk;
    float e;
    float ibk;  // 1/(beta k), rounded once (0 on the Haar branch)
};

__device__ __forceinline__ DrawSetup prepare_draw(float4 v, float beta)
{
    DrawSetup d;
    const float k = __fsqrt_rn(qnorm2(v));
    d.ut = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    if (k > 0.0f) {
        const float inv_k = __frcp_rn(k);
        d.ut = make_float4(__fmul_rn(v.x, inv_k), __fmul_rn(-v.y, inv_k), __fmul_rn(-v.z, inv_k),
                           __fmul_rn(-v.w, inv_k));
    }
    d.bk = __fmul_rn(beta, k);
    d.e = 0.0f;
    if (!(d.bk < kHaarBelow) && d.bk <= kExpCutoff) d.e = exp_series(__fmul_rn(-2.0f, d.bk));
    d.ibk = d.bk < kHaarBelow ? 0.0f : __frcp_rn(d.bk);
    return d;
}

// One Creutz trial (Phys. Rev. D 21, 2308): candidate a0 = 1 + ln(x)/(beta k),
// evaluated as 1 + ln(x) ibk with ibk = 1/(beta k) rounded once per link,
// x = e + r1 (1 - e) uniform in [exp(-2 beta k), 1]; on the Haar branch
// a0 = 2 r1 - 1.  Clamped to [-1, 1]; accepted iff r2^2 <= 1 - a0^2.
__device__ __forceinline__ bool creutz_trial(float r1, float r2, float ibk, float e, float one_minus_e, bool haar,
                                             float &cand)
{
    float c;
    if (haar) {
        c = __fsub_rn(__fmul_rn(2.0f, r1), 1.0f);
    } else {
        c = __fadd_rn(1.0f, __fmul_rn(log_series(__fmaf_rn(r1, one_minus_e, e)), ibk));
    }
    c = c < -1.0f ? -1.0f : (c > 1.0f ? 1.0f : c);
    cand = c;
    return __fmul_rn(r2, r2) <= __fmaf_rn(-c, c, 1.0f);
}

// ------------------------------------------- screened Creutz trials
// The exact test above accepts iff A <= R, with A = r2^2, R = 1 - c^2,
// c = clamp(1 + L ibk, -1, 1), L = log_series(x).  With t = -L ibk, R lies
// within 2.4e-7 + 1.3e-7 t of g(t) = max(t (2 - t), 0): c = 1 - t up to two
// roundings of numbers bounded by 2, g is 2-Lipschitz, and c clamps to -1
// exactly where 1 - t < -1, i.e. where g vanishes.  The screen estimates
// t~ = -lg2(x) ln2 ibk with the hardware base-2 logarithm (__log2f: absolute
// error <= 2^-22 for x in [1/2, 1], relative <= 2.4e-7 below), and log_series
// has |L - ln x| <= 1e-6 |ln x| + 1e-7; both bounds hold for every float x in
// [2^-34, 1], the range x = e + r1 (1 - e) takes (r1 >= 2^-33).  So
// |t - t~| <= 2.7e-7 ibk + 1.4e-6 t~ and |R - g(t~)| <= 3e-7 + 5.4e-7 ibk +
// 3e-6 t~, and with the slack 2e-6 + 4e-6 ibk + 2e-5 t~ (more than six times
// that) a trial with A > g(t~) + slack is rejected and one with
// A < g(t~) - slack accepted by the exact test as well.  Only the trials in
// between (about one in 10^5 at beta k ~ 30) need the exact test, and an
// accepted trial needs its exact a0 only once, when the link gets its
// direction.  On the Haar branch (ibk = 0) the slack is infinite: every trial
// goes to the exact test.
enum : int { kScreenReject = 0, kScreenAccept = 1, kScreenUndecided = 2 };

struct CreutzScreen {
    float ln2_ibk;  // ln 2 / (beta k)
    float slack0;   // 2e-6 + 4e-6 ibk (infinite on the Haar branch)
};

__device__ __forceinline__ CreutzScreen make_screen(float ibk)
{
    CreutzScreen s;
    s.ln2_ibk = __fmul_rn(0.693147182f, ibk);
    s.slack0 = ibk == 0.0f ? __int_as_float(0x7f800000) : __fmaf_rn(4e-6f, ibk, 2e-6f);
    return s;
}

__device__ __forceinline__ int creutz_screen(float x, float r2, const CreutzScreen &s)
{
    const float tt = __fmul_rn(-__log2f(x), s.ln2_ibk);
    const float g = fmaxf(__fmaf_rn(-tt, tt, __fadd_rn(tt, tt)), 0.0f);
    const float slack = __fmaf_rn(2e-5f, tt, s.slack0);
    const float a = __fmul_rn(r2, r2);
    if (a > __fadd_rn(g, slack)) return kScreenReject;
    if (a < __fsub_rn(g, slack)) return kScreenAccept;
    return kScreenUndecided;
}

// The a0 of an accepted Creutz-branch trial from its x: the candidate that
// creutz_trial forms, operation for operation.
__device__ __forceinline__ float creutz_a0(float x, float ibk)
{
    const float c = __fadd_rn(1.0f, __fmul_rn(log_series(x), ibk));
    return c < -1.0f ? -1.0f : (c > 1.0f ? 1.0f : c);
}

// The value a link waiting for its direction carries: x of the accepted trial
// (ibk > 0), or a0 itself on the Haar branch (ibk = 0).
__device__ __forceinline__ float deferred_a0(float val, float ibk)
{
    const float a = creutz_a0(val, ibk);
    return ibk == 0.0f ? val : a;
}

// Both trials of one Creutz Philox block w (words 0, 1 then 2, 3), with the
// verdicts of creutz_trial.  Returns whether either accepts; `first` whether
// the first did, `val` what deferred_a0 turns into the accepted a0.  Every
// lane of the warp calls it together; lanes with live = false only keep the
// warp converged (their undecided trials do not force the exact branch).
__device__ __forceinline__ bool creutz_pair(uint4 w, float ibk, float e, bool live, bool &first, float &val)
{
    const CreutzScreen s = make_screen(ibk);
    const float ome = __fsub_rn(1.0f, e);
    const float r1a = uniform_log(w.x), r2a = uniform01(w.y);
    const float r1b = uniform_log(w.z), r2b = uniform01(w.w);
    float va = __fmaf_rn(r1a, ome, e), vb = __fmaf_rn(r1b, ome, e);
    int sa = creutz_screen(va, r2a, s);
    int sb = creutz_screen(vb, r2b, s);
    if (__any_sync(0xffffffffu, live && (sa == kScreenUndecided || sb == kScreenUndecided))) {
        const bool haar = ibk == 0.0f;
        float c;
        if (sa == kScreenUndecided) {
            sa = creutz_trial(r1a, r2a, ibk, e, ome, haar, c) ? kScreenAccept : kScreenReject;
            if (haar) va = c;
        }
        if (sb == kScreenUndecided) {
            sb = creutz_trial(r1b, r2b, ibk, e, ome, haar, c) ? kScreenAccept : kScreenReject;
            if (haar) vb = c;
        }
    }
    first = sa == kScreenAccept;
    val = first ? va : vb;
    return first || sb == kScreenAccept;
}

// Vector part uniform on the sphere of radius sqrt(1 - a0^2): c = 2 u0 - 1,
// phi = 2 pi u1 (direction block 0); returns U' = a U~^dag.
__device__ __forceinline__ float4 direction_from_uniforms(float a0, float4 ut, float uc, float uphi)
{
    const float r = __fsqrt_rn(__fmaf_rn(-a0, a0, 1.0f));
    const float c = __fsub_rn(__fmul_rn(2.0f, uc), 1.0f);
    const float st = __fsqrt_rn(__fmaf_rn(-c, c, 1.0f));
    float sn, cs;
    sincos_2pi(uphi, sn, cs);
    const float rs = __fmul_rn(r, st);
    const float4 a = make_float4(a0, __fmul_rn(rs, cs), __fmul_rn(rs, sn), __fmul_rn(r, c));
    return qmul(a, ut);
}

// The direction block of the link with (global) even/odd index eo is block 0
// of the direction stream at counter eo >> 1, shared by the pair of links
// eo = 2j, 2j + 1: the even one takes words 0, 1, the odd one words 2, 3.
__device__ __forceinline__ uint32_t direction_pair(uint32_t eo) { return eo >> 1; }

__device__ __forceinline__ float4 direction_update(float a0, float4 ut, uint4 d, uint32_t eo)
{
    const bool odd = (eo & 1u) != 0u;
    return direction_from_uniforms(a0, ut, uniform01(odd ? d.z : d.x), uniform01(odd ? d.w : d.y));
}

// The whole heat-bath draw of one link from its staple v (Sec. 2), trial by
// trial: trial t uses words 2(t&1), 2(t&1)+1 of Creutz block t>>1; the
// direction uses the link's two words of its pair's direction block.  Returns the number of
// trials, or 0 if kMaxTrials were all rejected (out untouched).  gen(counter)
// is the Philox generator under the lattice's key.
template <class Gen>
__device__ __forceinline__ int heatbath_draw_gen(float4 v, float beta, Gen gen, uint32_t eo, uint32_t sweep,
                                                 uint32_t parity, uint32_t mu, float4 &out)
{
    const DrawSetup s = prepare_draw(v, beta);
    const bool haar = s.bk < kHaarBelow;
    const float ome = __fsub_rn(1.0f, s.e);
    float a0 = 0.0f;
    int trials = 0;
    for (int b = 0; b < kMaxTrials / 2 && trials == 0; ++b) {
        const uint4 w = gen(make_uint4(eo, sweep, stream_word(kCreutz, parity, mu), (uint32_t)b));
        float cand;
        if (creutz_trial(uniform_log(w.x), uniform01(w.y), s.ibk, s.e, ome, haar, cand)) {
            a0 = cand;
            trials = 2 * b + 1;
        } else if (creutz_trial(uniform_log(w.z), uniform01(w.w), s.ibk, s.e, ome, haar, cand)) {
            a0 = cand;
            trials = 2 * b + 2;
        }
    }
    if (trials == 0) return 0;
    out = direction_update(a0, s.ut, gen(make_uint4(direction_pair(eo), sweep, stream_word(kDirection, parity, mu), 0u)),
                           eo);
    return trials;
}

__device__ __forceinline__ int heatbath_draw(float4 v, float beta, const RoundKeys &rk, uint32_t eo, uint32_t sweep,
                                             uint32_t parity, uint32_t mu, float4 &out)
{
    return heatbath_draw_gen(v, beta, [&](uint4 c) { return philox_rk(c, rk); }, eo, sweep, parity, mu, out);
}

// Two blocks under the key (k0, k1) with the key schedule computed on the fly,
// round by round (batched kernels: one key per lattice).
__device__ __forceinline__ void philox2_key(uint4 &a, uint4 &b, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t alo0 = 0xD2511F53u * a.x, ahi0 = __umulhi(0xD2511F53u, a.x);
        const uint32_t alo1 = 0xCD9E8D57u * a.z, ahi1 = __umulhi(0xCD9E8D57u, a.z);
        const uint32_t blo0 = 0xD2511F53u * b.x, bhi0 = __umulhi(0xD2511F53u, b.x);
        const uint32_t blo1 = 0xCD9E8D57u * b.z, bhi1 = __umulhi(0xCD9E8D57u, b.z);
        a = make_uint4(ahi1 ^ a.y ^ k0, alo1, ahi0 ^ a.w ^ k1, alo0);
        b = make_uint4(bhi1 ^ b.y ^ k0, blo1, bhi0 ^ b.w ^ k1, blo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Haar-random link (Marsaglia 1972), the hot start (Sec. 4.1): two points
// uniform in the unit disk, (x1,x2) with s1 and (x3,x4) with s2, give
// (x1, x2, x3 f, x4 f), f = sqrt((1-s1)/s2), uniform on S^3.  Candidate pair m
// uses words 2(m&1), 2(m&1)+1 of hot-start block m>>1 of the link's counter
// (even/odd index eo, sweep 0, parity, mu).  Returns false (out = identity)
// if 64 pairs gave no two points.
__device__ __forceinline__ bool hot_link(uint32_t eo, uint32_t parity, uint32_t mu, const RoundKeys &rk, float4 &out)
{
    float px[2] = {0.0f, 0.0f}, py[2] = {0.0f, 0.0f}, ps[2] = {1.0f, 1.0f};
    int found = 0;
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    for (int m = 0; m < 64 && found < 2; ++m) {
        if ((m & 1) == 0) w = philox_rk(make_uint4(eo, 0u, stream_word(kHotStart, parity, mu), (uint32_t)(m >> 1)), rk);
        const float x = __fsub_rn(__fmul_rn(2.0f, uniform01((m & 1) ? w.z : w.x)), 1.0f);
        const float y = __fsub_rn(__fmul_rn(2.0f, uniform01((m & 1) ? w.w : w.y)), 1.0f);
        const float s = __fmaf_rn(x, x, __fmul_rn(y, y));
        if (s < 1.0f && s > 0.0f) {
            px[found] = x;
            py[found] = y;
            ps[found] = s;
            ++found;
        }
    }
    out = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    if (found < 2) return false;
    const float f = __fsqrt_rn(__fdiv_rn(__fsub_rn(1.0f, ps[0]), ps[1]));
    out = make_float4(px[0], py[0], __fmul_rn(px[1], f), __fmul_rn(py[1], f));
    return true;
}

// Division by an invariant positive integer d < 2^31 with a multiply-high and
// shifts (Granlund & Montgomery, PLDI 1994, Fig. 4.1): with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> min(l,1))) >> max(l-1,0),
// t = mulhi(m, n), exact for every 32-bit n.
struct FastDiv {
    uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

__device__ __forceinline__ uint32_t fastdiv(uint32_t n, const FastDiv &f)
{
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// --------------------------------------------------------------- geometry
// Lattice Ns^3 x Nt, lex = ((t Ns + z) Ns + y) Ns + x, parity (x+y+z+t)&1,
// even/odd index i = lex >> 1.  Links: float4 array, element (mu, parity, i)
// at (2 mu + parity) vh + i, vh = V/2.
struct Geom {
    int ns, nt;
    int vh;         // V / 2
    int vs;         // Ns^3
    FastDiv div_ns;
    int ext[4];     // extent of direction mu
    int stride[4];  // lexicographic stride of direction mu: 1, Ns, Ns^2, Ns^3
    int wrap[4];    // (extent - 1) * stride: the jump across the periodic boundary
};

struct Coord {
    int c[4];
    int lex;
};

// Site of parity p with even/odd index i: lex = 2i or 2i + 1, whichever has
// parity p (Ns is even, so the two share y, z, t).
__device__ __forceinline__ Coord eo_to_coord(const Geom &g, int i, int p)
{
    const uint32_t lex0 = 2u * (uint32_t)i;
    Coord r;
    const uint32_t rest = fastdiv(lex0, g.div_ns);
    const uint32_t x0 = lex0 - rest * (uint32_t)g.ns;
    const uint32_t rest2 = fastdiv(rest, g.div_ns);
    r.c[1] = (int)(rest - rest2 * (uint32_t)g.ns);
    r.c[3] = (int)fastdiv(rest2, g.div_ns);
    r.c[2] = (int)rest2 - r.c[3] * g.ns;
    const int odd = (r.c[1] + r.c[2] + r.c[3] + p) & 1;
    r.c[0] = (int)x0 + odd;
    r.lex = (int)lex0 + odd;
    return r;
}

// Lexicographic index of the neighbour at +mu / -mu of a site with index lex
// and coordinate c_mu in direction mu (periodic).
__device__ __forceinline__ int lex_fwd(const Geom &g, int lex, int c_mu, int mu)
{
    return c_mu == g.ext[mu] - 1 ? lex - g.wrap[mu] : lex + g.stride[mu];
}

__device__ __forceinline__ int lex_bwd(const Geom &g, int lex, int c_mu, int mu)
{
    return c_mu == 0 ? lex + g.wrap[mu] : lex - g.stride[mu];
}

// 32-bit unsigned: a lattice holds fewer than 2^31 links (checked at
// creation), so the address is one wide multiply-add of the offset.
__device__ __forceinline__ uint32_t link_index(const Geom &g, int mu, int parity, int eo)
{
    return (uint32_t)(2 * mu + parity) * (uint32_t)g.vh + (uint32_t)eo;
}

}  // namespace su2
