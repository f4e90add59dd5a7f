// learned.cuh -- device side of the learned a0 proposal: the small MLP of
// beta k, the monotone rational-quadratic spline it parametrises (Durkan,
// Bekasov, Murray, Papamakarios, "Neural Spline Flows", NeurIPS 2019), and the
// independence-Metropolis link step that uses it as the proposal for the
// heat-bath law of a0 (Sec. 2 of Cardoso & Bicudo).  binary32 with explicit
// round-to-nearest intrinsics throughout.
//
// Weights (float[1947]): W1[32], b1[32], W2[32][32], b2[32], W3[25][32],
// b3[25], input mean, input scale; network input s = (beta k - mean) scale,
// h1 = relu(W1 s + b1), h2 = relu(W2 h1 + b2), o = W3 h2 + b3.
// Spline parameters (27 floats): knots x_0..x_8 and y_0..y_8 on [-1, 1] from
// widths / heights 2 (m + (1 - 8 m) softmax), m = 1e-3, and knot derivatives
// d_0..d_8 = 1e-3 + softplus.
#pragma once

#include "su2_device.cuh"

namespace su2 {
namespace learned {

constexpr int kBins = 8;
constexpr int kHidden = 32;
constexpr int kOut = 25;
constexpr int kParams = 27;
constexpr int kWeights = 1947;
constexpr int kTrainable = 1945;
constexpr int kOffW1 = 0, kOffB1 = 32, kOffW2 = 64, kOffB2 = 1088, kOffW3 = 1120, kOffB3 = 1920;
constexpr int kOffMean = 1945, kOffScale = 1946;
constexpr float kMinBin = 1e-3f;
constexpr float kMinDer = 1e-3f;

__device__ __forceinline__ float exp_neg(float y) { return y < -87.0f ? 0.0f : exp_series(y); }
__device__ __forceinline__ float relu(float x) { return x > 0.0f ? x : 0.0f; }

// Sums start at the bias and add w[i] x[i], i ascending, one fused multiply-add each.
__device__ __forceinline__ void mlp_forward(const float *__restrict__ w, float s, float (&o)[kOut])
{
    float h1[kHidden], h2[kHidden];
#pragma unroll
    for (int j = 0; j < kHidden; ++j) h1[j] = relu(__fmaf_rn(w[kOffW1 + j], s, w[kOffB1 + j]));
#pragma unroll 4
    for (int j = 0; j < kHidden; ++j) {
        float acc = w[kOffB2 + j];
#pragma unroll
        for (int i = 0; i < kHidden; ++i) acc = __fmaf_rn(w[kOffW2 + j * kHidden + i], h1[i], acc);
        h2[j] = relu(acc);
    }
#pragma unroll 5
    for (int j = 0; j < kOut; ++j) {
        float acc = w[kOffB3 + j];
#pragma unroll
        for (int i = 0; i < kHidden; ++i) acc = __fmaf_rn(w[kOffW3 + j * kHidden + i], h2[i], acc);
        o[j] = acc;
    }
}

// Knots -1 = k_0 < ... < k_8 = 1 from 8 unnormalised log-widths.
__device__ __forceinline__ void knots_from(const float *o8, float *k9)
{
    float mx = o8[0];
#pragma unroll
    for (int i = 1; i < kBins; ++i) mx = o8[i] > mx ? o8[i] : mx;
    float e[kBins], sum = 0.0f;
#pragma unroll
    for (int i = 0; i < kBins; ++i) {
        e[i] = exp_neg(__fsub_rn(o8[i], mx));
        sum = __fadd_rn(sum, e[i]);
    }
    k9[0] = -1.0f;
#pragma unroll
    for (int i = 0; i < kBins - 1; ++i) {
        const float width = __fmul_rn(2.0f, __fmaf_rn(1.0f - 8.0f * kMinBin, __fdiv_rn(e[i], sum), kMinBin));
        k9[i + 1] = __fadd_rn(k9[i], width);
    }
    k9[kBins] = 1.0f;
}

// softplus(t) = max(t, 0) + log(1 + exp(-|t|))
__device__ __forceinline__ float softplus(float t)
{
    const float at = t < 0.0f ? -t : t;
    return __fadd_rn(t > 0.0f ? t : 0.0f, log_series(__fadd_rn(1.0f, exp_neg(-at))));
}

__device__ __forceinline__ void spline_params(const float (&o)[kOut], float *p)
{
    knots_from(o, p);
    knots_from(o + kBins, p + kBins + 1);
#pragma unroll
    for (int i = 0; i <= kBins; ++i) p[2 * (kBins + 1) + i] = __fadd_rn(kMinDer, softplus(o[2 * kBins + i]));
}

// Parameter accessor: p(i) is spline parameter i (x_0..x_8, y_0..y_8, d_0..d_8).
// Linear interpolation between two table rows, element by element on demand:
// the rows are stored as pairs (r0_i, r1_i - r0_i), so p_i = r0_i + f (r1_i -
// r0_i) is one 8-byte load and one fused multiply-add, and no per-thread copy
// of the 27 parameters is needed.
struct PairParams {
    const float2 *row;
    float f;
    __device__ __forceinline__ float operator()(int i) const
    {
        const float2 q = row[i];
        return __fmaf_rn(f, q.y, q.x);
    }
};

// Largest k in 0..kBins-1 with knot p(base + k) <= v (knot 0 is the lower end,
// -1): the knots are non-decreasing, so three halvings find it.
template <class P>
__device__ __forceinline__ int bin_of(const P &p, int base, float v)
{
    static_assert(kBins == 8, "three halvings cover eight bins");
    int k = 0;
    if (p(base + 4) <= v) k = 4;
    if (p(base + k + 2) <= v) k += 2;
    if (p(base + k + 1) <= v) k += 1;
    return k;
}

// a = y_k + h (s xi^2 + d_k t)/den, den = s + (d_{k+1} + d_k - 2 s) t, t = xi (1 - xi),
// f' = s^2 (d_{k+1} xi^2 + 2 s t + d_k (1 - xi)^2) / den^2, evaluated with
// r = 1/den rounded once: a = y_k + num r, f' = (s^2 m) r^2; the caller gives s.
template <class P>
__device__ __forceinline__ float spline_eval(const P &p, int k, float xi, float s, float &fprime)
{
    constexpr int Y = kBins + 1, D = 2 * (kBins + 1);
    const float yk = p(Y + k);
    const float h = __fsub_rn(p(Y + k + 1), yk);
    const float dk = p(D + k), dk1 = p(D + k + 1);
    const float t = __fmul_rn(xi, __fsub_rn(1.0f, xi));
    const float sigma = __fsub_rn(__fadd_rn(dk1, dk), __fmul_rn(2.0f, s));
    const float den = __fmaf_rn(sigma, t, s);
    const float num = __fmul_rn(h, __fmaf_rn(__fmul_rn(s, xi), xi, __fmul_rn(dk, t)));
    const float omx = __fsub_rn(1.0f, xi);
    const float m = __fmaf_rn(__fmul_rn(dk1, xi), xi, __fmaf_rn(__fmul_rn(2.0f, s), t, __fmul_rn(__fmul_rn(dk, omx), omx)));
    const float r = __frcp_rn(den);  // correctly rounded 1/den, the same number as 1.0f / den
    fprime = __fmul_rn(__fmul_rn(__fmul_rn(s, s), m), __fmul_rn(r, r));
    return __fadd_rn(yk, __fmul_rn(num, r));
}

// xi = (z - x_k) iw and s = h iw with iw = 1/w rounded once.
template <class P>
__device__ __forceinline__ float spline_forward(const P &p, float z, float &fprime)
{
    constexpr int Y = kBins + 1;
    const int k = bin_of(p, 0, z);
    const float xk = p(k);
    const float iw = __frcp_rn(__fsub_rn(p(k + 1), xk));  // correctly rounded 1/w
    const float s = __fmul_rn(__fsub_rn(p(Y + k + 1), p(Y + k)), iw);
    float xi = __fmul_rn(__fsub_rn(z, xk), iw);
    xi = xi < 0.0f ? 0.0f : (xi > 1.0f ? 1.0f : xi);
    const float a = spline_eval(p, k, xi, s, fprime);
    return a < -1.0f ? -1.0f : (a > 1.0f ? 1.0f : a);
}

// Inverse on bin k of y: alpha xi^2 + beta xi + c = 0, xi = 2c / (-beta - sqrt(beta^2 - 4 alpha c)).
template <class P>
__device__ __forceinline__ float spline_inverse(const P &p, float a, float &fprime)
{
    constexpr int Y = kBins + 1, D = 2 * (kBins + 1);
    const int k = bin_of(p, Y, a);
    const float xk = p(k);
    const float w = __fsub_rn(p(k + 1), xk);
    const float yk = p(Y + k);
    const float h = __fsub_rn(p(Y + k + 1), yk);
    const float dk = p(D + k), dk1 = p(D + k + 1);
    const float s = __fdiv_rn(h, w);
    const float dy = __fsub_rn(a, yk);
    const float sigma = __fsub_rn(__fadd_rn(dk1, dk), __fmul_rn(2.0f, s));
    const float alpha = __fmaf_rn(dy, sigma, __fmul_rn(h, __fsub_rn(s, dk)));
    const float beta = __fmaf_rn(-dy, sigma, __fmul_rn(h, dk));
    const float c = __fmul_rn(-s, dy);
    float disc = __fmaf_rn(beta, beta, __fmul_rn(__fmul_rn(-4.0f, alpha), c));
    disc = disc > 0.0f ? disc : 0.0f;
    const float denom = __fsub_rn(-beta, __fsqrt_rn(disc));
    float xi = denom != 0.0f ? __fdiv_rn(__fmul_rn(2.0f, c), denom) : 0.0f;
    xi = xi < 0.0f ? 0.0f : (xi > 1.0f ? 1.0f : xi);
    spline_eval(p, k, xi, s, fprime);
    return __fmaf_rn(xi, w, xk);
}

// Row pair around network input s (clamped to the table's range) and the
// interpolation weight; pairs[j] holds rows j and j+1 as (r_j, r_{j+1} - r_j).
__device__ __forceinline__ PairParams pair_params(const float2 *pairs, int G, float s_lo, float inv_ds, float s)
{
    float u = __fmul_rn(__fsub_rn(s, s_lo), inv_ds);
    u = u < 0.0f ? 0.0f : (u > (float)(G - 1) ? (float)(G - 1) : u);
    int j = (int)floorf(u);
    if (j > G - 2) j = G - 2;
    PairParams pp;
    pp.row = pairs + j * kParams;
    pp.f = __fsub_rn(u, (float)j);
    return pp;
}

// inv_ds = (G - 1) / (s_hi - s_lo), the grid points per unit of s.
__device__ __forceinline__ float table_inv_ds(int G, float s_lo, float s_hi)
{
    return __fdiv_rn((float)(G - 1), __fsub_rn(s_hi, s_lo));
}

struct Proposal {
    const float2 *pairs;  // (G - 1) x 27 row pairs (shared memory)
    int G;
    float s_lo, inv_ds, mean, scale;
};

// Independence-Metropolis update of one link (staple v, current link old):
// proposal a0' = f(2 u0 - 1) with density 1/(2 f'), direction from u2, u3;
// accepted iff u1 <= exp(Delta) (or Delta >= 0) with
// Delta = beta k (a0' - a_cur) + log(sqrt((1 - a0'^2)/(1 - a_cur^2)) f'(z')/f'(z_cur)),
// a_cur = old U~.  All four uniforms from one Philox block of the learned
// stream.  In two parts, so a caller can place other work between them:
// learned_propose draws a0' and f'(z'); learned_accept decides (a rejected
// link keeps its value, an accepted one becomes a U~^dag with the direction).
struct LearnedDraw {
    DrawSetup d;
    PairParams ip;
    float a_new, fp_new;
};

__device__ __forceinline__ LearnedDraw learned_propose(const Proposal &pr, float beta, float4 v, float u0)
{
    LearnedDraw r;
    r.d = prepare_draw(v, beta);
    r.ip = pair_params(pr.pairs, pr.G, pr.s_lo, pr.inv_ds, __fmul_rn(__fsub_rn(r.d.bk, pr.mean), pr.scale));
    r.a_new = spline_forward(r.ip, __fsub_rn(__fmul_rn(2.0f, u0), 1.0f), r.fp_new);
    return r;
}

// The exact verdict from its parts: accept iff Delta >= 0 or u1 <= exp(Delta),
// Delta = beta k (a' - a) + log(ratio), ratio = sqrt((1 - a'^2) f'(z')^2 /
// ((1 - a^2) f'(z)^2)) as one square root of one quotient.
__device__ __forceinline__ bool metropolis_exact(float bk, float a_new, float acur, float fp_new, float fp_cur,
                                                 float u1)
{
    const float one_cur = __fmaf_rn(-acur, acur, 1.0f);
    if (!(one_cur > 0.0f)) return true;
    const float one_new = __fmaf_rn(-a_new, a_new, 1.0f);
    const float ratio = __fsqrt_rn(__fdiv_rn(__fmul_rn(one_new, __fmul_rn(fp_new, fp_new)),
                                             __fmul_rn(one_cur, __fmul_rn(fp_cur, fp_cur))));
    if (!(ratio > 0.0f)) return false;
    const float delta = __fmaf_rn(bk, __fsub_rn(a_new, acur), log_series(ratio));
    return delta >= 0.0f || u1 <= exp_neg(delta);
}

// The same verdict screened with the hardware base-2 logarithm (__log2f:
// absolute error <= 2^-22 on [1/2, 2], relative <= 2.4e-7 elsewhere; checked
// with the Creutz screen).  With N, D the ratio's numerator and denominator
// and l = (1/2) ln(N/D), the exact log(ratio) is within 2e-7 + 1e-6 |l| of l
// (a quotient, a square root, log_series), and the estimate
// d~ = beta k (a' - a) + (ln 2 / 2)(lg2 N - lg2 D) within
// 4e-7 + 6e-7 (|lg2 N| + |lg2 D|) + 6e-8 |d~| of the exact Delta; the slack
// 2e-4 + 4e-6 (|lg2 N| + |lg2 D|) is more than six times that.  For
// d~ < -slack, u1 <= exp_neg(Delta) is decided from ln u1 (estimated within
// 5e-6 for u1 >= 2^-24) against d~ with a further 1e-5 + 1e-6 |d~| (exp_neg
// is within 2 ulp of exp).  Returns kScreenAccept, kScreenReject or
// kScreenUndecided (tiny, huge or non-finite parts; inside a band).
__device__ __forceinline__ int metropolis_screen(float bk, float a_new, float acur, float fp_new, float fp_cur,
                                                 float u1)
{
    const float one_cur = __fmaf_rn(-acur, acur, 1.0f);
    if (!(one_cur > 0.0f)) return kScreenAccept;
    const float one_new = __fmaf_rn(-a_new, a_new, 1.0f);
    const float num = __fmul_rn(one_new, __fmul_rn(fp_new, fp_new));
    const float den = __fmul_rn(one_cur, __fmul_rn(fp_cur, fp_cur));
    if (!(num > 1e-30f && num < 1e30f && den > 1e-30f && den < 1e30f)) return kScreenUndecided;
    const float lg_n = __log2f(num), lg_d = __log2f(den);
    const float lr = __fmul_rn(0.346573591f, __fsub_rn(lg_n, lg_d));
    const float dt = __fmaf_rn(bk, __fsub_rn(a_new, acur), lr);
    const float slack = __fmaf_rn(4e-6f, __fadd_rn(fabsf(lg_n), fabsf(lg_d)), 2e-4f);
    if (dt > slack) return kScreenAccept;
    if (!(dt < -slack)) return kScreenUndecided;
    const float lu = __fmul_rn(0.693147182f, __log2f(u1));
    const float slack2 = __fmaf_rn(1e-6f, -dt, __fadd_rn(slack, 1e-5f));
    if (lu < __fsub_rn(dt, slack2)) return kScreenAccept;
    if (lu > __fadd_rn(dt, slack2)) return kScreenReject;
    return kScreenUndecided;
}

// The verdict of the step: screened, with the exact arithmetic for the lanes
// the screen leaves undecided.  Every lane of the warp calls it together;
// lanes with live = false only keep the warp converged.
__device__ __forceinline__ bool learned_accept(const LearnedDraw &r, float4 old, float u1, bool live)
{
    float acur = chain4(old.x, r.d.ut.x, old.y, r.d.ut.y, old.z, r.d.ut.z, old.w, r.d.ut.w);
    acur = acur < -1.0f ? -1.0f : (acur > 1.0f ? 1.0f : acur);
    float fp_cur;
    spline_inverse(r.ip, acur, fp_cur);
    int v = metropolis_screen(r.d.bk, r.a_new, acur, r.fp_new, fp_cur, u1);
    if (__any_sync(0xffffffffu, live && v == kScreenUndecided)) {
        if (v == kScreenUndecided)
            v = metropolis_exact(r.d.bk, r.a_new, acur, r.fp_new, fp_cur, u1) ? kScreenAccept : kScreenReject;
    }
    return v == kScreenAccept;
}

}  // namespace learned
}  // namespace su2
