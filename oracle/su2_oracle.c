/*
 * su2_oracle.c -- plain, slow CPU oracle for pure-gauge lattice SU(2)
 * (Cardoso & Bicudo, "Lattice SU(2) on GPU's", LAT2010).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, the smoke check of the entry module and the CPU-baseline leg
 * of the benchmark load it.  It shares no source with the CUDA library.
 *
 * What it computes, by section of the paper:
 *   - SU(2) elements as quaternions U = a0 + i a.sigma, |a| = 1      (Sec. 2)
 *   - staple V = sum of the six three-link products around U_mu(x)   (Sec. 2)
 *   - k = sqrt(det V), U~ = V/k, a0 drawn from sqrt(1-a0^2) e^{beta k a0}
 *     (Creutz rejection), uniform direction on S^2, U' = a U~^{-1}   (Sec. 2)
 *   - even/odd sites per direction mu, mu = 0..3 in order             (Sec. 4)
 *   - cold / hot start, mean plaquette, Polyakov loop                 (Sec. 4)
 * The random numbers the paper drew from a stored rand48 buffer (Sec. 4) are
 * replaced by the counter-based Philox4x32-10 generator (Salmon, Moraes, Dror,
 * Shaw, SC'11), implemented here from its published definition.
 *
 * Arithmetic contract (so that a GPU that follows the same contract gives the
 * same bits): link arithmetic is IEEE binary32 with round-to-nearest, no
 * contraction (compile with -ffp-contract=off), every fused operation written
 * as an explicit fmaf; sqrtf and '/' correctly rounded; log, exp and the
 * sine/cosine of 2*pi*u are the series defined below (never libm); global sums
 * are binary64.  The all-binary64 observables (suffix _f64) state the float
 * error of the plaquette and the Polyakov loop.
 *
 * Link storage here is the natural one: links[site][mu][c], site in
 * lexicographic order lex = ((t*Ns + z)*Ns + y)*Ns + x, c = a0..a3.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 bit     */
/* multiplications; the key is bumped by the Weyl constants between rounds.  */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* The top 24 bits of a 32-bit word, shifted into (0, 1]: ((x>>8)+1) 2^-24.
 * Exact in binary32; never 0. */
float orc_u01(uint32_t x)
{
    return (float)((x >> 8) + 1u) * (1.0f / 16777216.0f);
}

/* The uniform that feeds a logarithm: x 2^-32 + 2^-33 from the whole word,
 * (float)x rounded to nearest, then one fused multiply-add, so the value is
 * in [2^-33, 1] and exact ((2x + 1) 2^-33) for x < 2^23.  Creutz's method
 * takes x uniform on [exp(-2 beta k), 1] (Sec. 2): with the 24-bit uniform
 * above, -ln x would stop at 24 ln 2 = 16.6, cutting away the law's tail
 * beta k (1 - a0) > 16.6 (2.8e-7 of its mass at large beta k, enough to lift
 * the plaquette at beta = 6 by about 4e-7); from the whole word the cut is at
 * 33 ln 2 = 22.9 (mass 6e-10). */
float orc_u01_log(uint32_t x)
{
    return fmaf((float)x, 0x1p-32f, 0x1p-33f);
}

/* Counter layout: c0 = even/odd site index, c1 = sweep, c2 = (stream kind << 3)
 * | (parity << 2) | mu, c3 = block number within the stream.  Key = seed. */
enum { ORC_KIND_CREUTZ = 0, ORC_KIND_DIRECTION = 1, ORC_KIND_HOTSTART = 2, ORC_KIND_LEARNED = 3 };

static void draw_words(uint64_t seed, uint32_t eo, uint32_t sweep, int kind, int parity, int mu,
                       uint32_t block, uint32_t w[4])
{
    uint32_t ctr[4] = {eo, sweep, ((uint32_t)kind << 3) | ((uint32_t)parity << 2) | (uint32_t)mu, block};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

static void draw_block(uint64_t seed, uint32_t eo, uint32_t sweep, int kind, int parity, int mu,
                       uint32_t block, float u[4])
{
    uint32_t w[4];
    draw_words(seed, eo, sweep, kind, parity, mu, block, w);
    for (int i = 0; i < 4; ++i) u[i] = orc_u01(w[i]);
}

/* ------------------------------------------------------------------------ */
/* Elementary functions, written from textbook series (never libm).          */
/* ------------------------------------------------------------------------ */
static float bits_to_float(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static uint32_t float_to_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* ln 2 split so that n * LN2_HI is exact for |n| < 2^12:
 * LN2_HI = 2839 / 4096, LN2_LO = ln 2 - LN2_HI rounded to binary32. */
#define ORC_LN2_HI (2839.0f / 4096.0f)
#define ORC_LN2_LO 3.19461849e-05f
#define ORC_INV_LN2 1.44269502f
#define ORC_SQRT2 1.41421354f /* binary32 nearest to sqrt(2) */

/* Natural log of a positive normal float.  x = 2^k m with m in [sqrt(1/2),
 * sqrt(2)); log m = 2 atanh(s), s = (m-1)/(m+1), by the odd series
 * 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9 + s^11/11)  (|s| <= 0.1716). */
float orc_logf(float x)
{
    uint32_t b = float_to_bits(x);
    int k = (int)((b >> 23) & 0xffu) - 127;
    float m = bits_to_float((b & 0x007fffffu) | 0x3f800000u);
    if (m > ORC_SQRT2) {
        m = m * 0.5f;
        k = k + 1;
    }
    float f = m - 1.0f;
    float s = f / (m + 1.0f);
    float z = s * s;
    float q = fmaf(z, 1.0f / 11.0f, 1.0f / 9.0f);
    q = fmaf(q, z, 1.0f / 7.0f);
    q = fmaf(q, z, 1.0f / 5.0f);
    q = fmaf(q, z, 1.0f / 3.0f);
    float s2 = 2.0f * s;
    float r = s2 * z;
    float lm = fmaf(r, q, s2);
    float kf = (float)k;
    return fmaf(kf, ORC_LN2_HI, fmaf(kf, ORC_LN2_LO, lm));
}

/* exp(y) for y in [-87, 0]: Cody-Waite reduction y = n ln2 + r, |r| <= ln2/2,
 * then the Taylor series of e^r to degree 7 (truncation < 6e-9 relative),
 * then scaling by 2^n through the exponent bits. */
float orc_expf(float y)
{
    float t = y * ORC_INV_LN2;
    float n = floorf(t + 0.5f);
    float r = fmaf(-n, ORC_LN2_HI, y);
    r = fmaf(-n, ORC_LN2_LO, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int ni = (int)n;
    float scale = bits_to_float((uint32_t)(ni + 127) << 23);
    return p * scale;
}

/* sin(2 pi u), cos(2 pi u) for u in [0, 1].  w = 4u (exact), q = nearest
 * integer, f = w - q in [-1/2, 1/2] (exact), x = f pi/2; Taylor series of sin
 * to x^9 and cos to x^10 on |x| <= pi/4, then rotation by q quarter turns. */
void orc_sincos2pi(float u, float *sn_out, float *cs_out)
{
    float w = 4.0f * u;
    float q = floorf(w + 0.5f);
    float f = w - q;
    float x = f * 1.57079637f;
    float z = x * x;
    float ps = fmaf(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(ps, z, 1.0f / 120.0f);
    ps = fmaf(ps, z, -1.0f / 6.0f);
    float sn = fmaf(x * z, ps, x);
    float pc = fmaf(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = fmaf(pc, z, -1.0f / 720.0f);
    pc = fmaf(pc, z, 1.0f / 24.0f);
    pc = fmaf(pc, z, -0.5f);
    float cs = fmaf(z, pc, 1.0f);
    int quadrant = ((int)q) & 3;
    float s_out, c_out;
    if (quadrant == 0) { s_out = sn;  c_out = cs; }
    else if (quadrant == 1) { s_out = cs;  c_out = -sn; }
    else if (quadrant == 2) { s_out = -sn; c_out = -cs; }
    else { s_out = -cs; c_out = sn; }
    *sn_out = s_out;
    *cs_out = c_out;
}

void orc_logf_v(const float *x, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = orc_logf(x[i]); }
void orc_expf_v(const float *x, float *y, int64_t n) { for (int64_t i = 0; i < n; ++i) y[i] = orc_expf(x[i]); }
void orc_sincos2pi_v(const float *u, float *s, float *c, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) orc_sincos2pi(u[i], &s[i], &c[i]);
}

/* ------------------------------------------------------------------------ */
/* SU(2) as quaternions (Sec. 2): U = a0 1 + i a.sigma.                      */
/* (a b)_0 = a0 b0 - a.b ; (a b)_vec = a0 b + b0 a - a x b ; U^dagger = (a0,-a) */
/* Every 4-term sum is the chain fmaf(p0,q0, fmaf(p1,q1, fmaf(p2,q2, p3*q3))) */
/* with signs folded into the first factor of each pair (negation is exact). */
/* ------------------------------------------------------------------------ */
static float dot4(float p0, float q0, float p1, float q1, float p2, float q2, float p3, float q3)
{
    return fmaf(p0, q0, fmaf(p1, q1, fmaf(p2, q2, p3 * q3)));
}

void orc_quat_mul(const float a[4], const float b[4], float c[4])
{
    float r0 = dot4(a[0], b[0], -a[1], b[1], -a[2], b[2], -a[3], b[3]);
    float r1 = dot4(a[0], b[1], a[1], b[0], -a[2], b[3], a[3], b[2]);
    float r2 = dot4(a[0], b[2], a[2], b[0], -a[3], b[1], a[1], b[3]);
    float r3 = dot4(a[0], b[3], a[3], b[0], -a[1], b[2], a[2], b[1]);
    c[0] = r0; c[1] = r1; c[2] = r2; c[3] = r3;
}

/* c <- a b + c, each component the chain of orc_quat_mul with its innermost
 * product fused with the component of c: fmaf(p0,q0, fmaf(p1,q1, fmaf(p2,q2,
 * fmaf(p3,q3, c)))).  The staple accumulates its terms this way. */
static void quat_mul_add(const float a[4], const float b[4], float c[4])
{
    float r0 = fmaf(a[0], b[0], fmaf(-a[1], b[1], fmaf(-a[2], b[2], fmaf(-a[3], b[3], c[0]))));
    float r1 = fmaf(a[0], b[1], fmaf(a[1], b[0], fmaf(-a[2], b[3], fmaf(a[3], b[2], c[1]))));
    float r2 = fmaf(a[0], b[2], fmaf(a[2], b[0], fmaf(-a[3], b[1], fmaf(a[1], b[3], c[2]))));
    float r3 = fmaf(a[0], b[3], fmaf(a[3], b[0], fmaf(-a[1], b[2], fmaf(a[2], b[1], c[3]))));
    c[0] = r0; c[1] = r1; c[2] = r2; c[3] = r3;
}

static void quat_dag(const float a[4], float d[4])
{
    d[0] = a[0]; d[1] = -a[1]; d[2] = -a[2]; d[3] = -a[3];
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry: Ns^3 x Nt, periodic; mu = 0,1,2 spatial, mu = 3 time.   */
/* ------------------------------------------------------------------------ */
static int extent(int ns, int nt, int mu) { return mu == 3 ? nt : ns; }

static void site_coords(int64_t s, int ns, int c[4])
{
    c[0] = (int)(s % ns); s /= ns;
    c[1] = (int)(s % ns); s /= ns;
    c[2] = (int)(s % ns); s /= ns;
    c[3] = (int)s;
}

static int64_t site_index(const int c[4], int ns)
{
    return (((int64_t)c[3] * ns + c[2]) * ns + c[1]) * ns + c[0];
}

/* s shifted by `step` (+1 or -1) lattice units in direction mu, periodic. */
static int64_t site_shift(int64_t s, int mu, int step, int ns, int nt)
{
    int c[4];
    site_coords(s, ns, c);
    int L = extent(ns, nt, mu);
    c[mu] = (c[mu] + step + L) % L;
    return site_index(c, ns);
}

static int site_parity(int64_t s, int ns)
{
    int c[4];
    site_coords(s, ns, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

static const float *link_at(const float *links, int64_t s, int mu) { return links + (s * 4 + mu) * 4; }

/* ------------------------------------------------------------------------ */
/* Start configurations (Sec. 4: cold start and hot start kernels).          */
/* ------------------------------------------------------------------------ */
void orc_cold_start(int ns, int nt, float *links)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
    for (int64_t s = 0; s < vol; ++s)
        for (int mu = 0; mu < 4; ++mu) {
            float *l = links + (s * 4 + mu) * 4;
            l[0] = 1.0f; l[1] = 0.0f; l[2] = 0.0f; l[3] = 0.0f;
        }
}

/* Haar-random SU(2) link by Marsaglia's 4-D method (Ann. Math. Stat. 43,
 * 1972): two points uniform in the unit disk, (x1,x2) with s1 and (x3,x4)
 * with s2; the point (x1, x2, x3 f, x4 f), f = sqrt((1-s1)/s2), is uniform on
 * S^3.  Candidate pair m uses uniforms 2(m&1), 2(m&1)+1 of block m>>1 of the
 * hot-start stream.  Returns 0, or 1 if 64 pairs did not give two points. */
static int hot_link(uint64_t seed, uint32_t eo, int parity, int mu, float out[4])
{
    float pt[2][2];
    float sq[2];
    int found = 0;
    float u[4];
    for (int m = 0; m < 64 && found < 2; ++m) {
        if ((m & 1) == 0) draw_block(seed, eo, 0u, ORC_KIND_HOTSTART, parity, mu, (uint32_t)(m >> 1), u);
        float x = 2.0f * u[2 * (m & 1)] - 1.0f;
        float y = 2.0f * u[2 * (m & 1) + 1] - 1.0f;
        float s = fmaf(x, x, y * y);
        if (s < 1.0f && s > 0.0f) {
            pt[found][0] = x;
            pt[found][1] = y;
            sq[found] = s;
            ++found;
        }
    }
    if (found < 2) {
        out[0] = 1.0f; out[1] = 0.0f; out[2] = 0.0f; out[3] = 0.0f;
        return 1;
    }
    float f = sqrtf((1.0f - sq[0]) / sq[1]);
    out[0] = pt[0][0];
    out[1] = pt[0][1];
    out[2] = pt[1][0] * f;
    out[3] = pt[1][1] * f;
    return 0;
}

int orc_hot_start(int ns, int nt, uint64_t seed, float *links)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
    int errors = 0;
    for (int64_t s = 0; s < vol; ++s) {
        int p = site_parity(s, ns);
        for (int mu = 0; mu < 4; ++mu)
            errors += hot_link(seed, (uint32_t)(s >> 1), p, mu, links + (s * 4 + mu) * 4);
    }
    return errors;
}

/* ------------------------------------------------------------------------ */
/* Staple (Sec. 2): V = sum over nu != mu of                                  */
/*   U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag                                    */
/* + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu),                             */
/* so that (1/2) Tr(U_mu(x) V) is the sum of the six plaquettes holding it.   */
/* nu ascending, forward term then backward term, from 0; each term's second  */
/* product is fused with the running sum (quat_mul_add), one rounding per     */
/* component and term.                                                        */
/* ------------------------------------------------------------------------ */
void orc_staple(int ns, int nt, const float *links, int64_t s, int mu, float v[4])
{
    v[0] = 0.0f; v[1] = 0.0f; v[2] = 0.0f; v[3] = 0.0f;
    int64_t xp = site_shift(s, mu, +1, ns, nt);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        int64_t xn = site_shift(s, nu, +1, ns, nt);
        int64_t xm = site_shift(s, nu, -1, ns, nt);
        int64_t xpm = site_shift(xp, nu, -1, ns, nt);
        float d1[4], d2[4], t[4];
        /* forward: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
        quat_dag(link_at(links, xn, mu), d1);
        orc_quat_mul(link_at(links, xp, nu), d1, t);
        quat_dag(link_at(links, s, nu), d2);
        quat_mul_add(t, d2, v);
        /* backward: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) */
        quat_dag(link_at(links, xpm, nu), d1);
        quat_dag(link_at(links, xm, mu), d2);
        orc_quat_mul(d1, d2, t);
        quat_mul_add(t, link_at(links, xm, nu), v);
    }
}

/* ------------------------------------------------------------------------ */
/* Heat-bath update of one link (Sec. 2).                                    */
/*   k = sqrt(det V) = |v|, U~^dag = V^dag / k,                               */
/*   a0 ~ sqrt(1-a0^2) exp(beta k a0) by Creutz's rejection method            */
/*   (Phys. Rev. D 21, 2308 (1980)): a0 = 1 + ln(x)/(beta k) with x uniform   */
/*   in [exp(-2 beta k), 1], accepted iff r2^2 <= 1 - a0^2;                    */
/*   a = (a0, r sqrt(1-c^2) cos phi, r sqrt(1-c^2) sin phi, r c), r=sqrt(1-a0^2),*/
/*   c uniform in [-1,1], phi uniform in [0,2pi);  U' = a U~^dag.             */
/* Trial t uses uniforms 2(t&1), 2(t&1)+1 of block t>>1 of the Creutz stream; */
/* the direction uses uniforms 2(eo&1), 2(eo&1)+1 of direction block eo>>1.   */
/* beta k < 1e-6 (e.g. beta = 0): a0 = 2 r1 - 1, same acceptance test (Haar). */
/* beta k > 43: exp(-2 beta k) is taken as 0 (below the binary32 normal range).*/
/* Returns the number of trials, or -1 if 4096 trials were all rejected, in   */
/* which case out[] is left untouched.                                         */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_TRIALS 4096

/* The new link from its a0 (Sec. 2): the vector part uniform on the sphere of
 * radius r = sqrt(1 - a0^2), a = (a0, r sqrt(1-c^2) cos phi, r sqrt(1-c^2)
 * sin phi, r c) with c = 2 u - 1 and phi = 2 pi v, and U' = a U~^dag.  The
 * uniforms (u, v) of the link with even/odd index eo are words 0, 1 of
 * direction block eo/2 for even eo and words 2, 3 for odd eo: the two links
 * of a pair share one Philox block, each using words the other does not. */
static void heatbath_direction(float a0, const float ut[4], uint64_t seed, uint32_t eo, uint32_t sweep, int parity,
                               int mu, float out[4])
{
    float d[4];
    draw_block(seed, eo >> 1, sweep, ORC_KIND_DIRECTION, parity, mu, 0u, d);
    const float u = d[2 * (eo & 1u)], v = d[2 * (eo & 1u) + 1];
    float r = sqrtf(fmaf(-a0, a0, 1.0f));
    float c = 2.0f * u - 1.0f;
    float st = sqrtf(fmaf(-c, c, 1.0f));
    float sn, cs;
    orc_sincos2pi(v, &sn, &cs);
    float rs = r * st;
    float a[4] = {a0, rs * cs, rs * sn, r * c};
    orc_quat_mul(a, ut, out);
}

/* What a link's Creutz trials need from beta k (Sec. 2): e = exp(-2 beta k)
 * (0 on the Haar branch and above beta k = 43), 1 - e and 1/(beta k). */
struct creutz_setup {
    int haar;
    float e, one_minus_e, inv_bk;
};

static struct creutz_setup creutz_prepare(float bk)
{
    struct creutz_setup c;
    c.haar = bk < 1e-6f;
    c.e = 0.0f;
    if (!c.haar && bk <= 43.0f) c.e = orc_expf(-2.0f * bk);
    c.one_minus_e = 1.0f - c.e;
    /* a0 = 1 + ln(x)/(beta k) is evaluated as 1 + ln(x) * (1/(beta k)) with
     * the reciprocal rounded once per link (Sec. 2 fixes the formula, not its
     * rounding; one division per link instead of one per trial) */
    c.inv_bk = c.haar ? 0.0f : 1.0f / bk;
    return c;
}

/* The candidate a0 of one trial from its first uniform r1, clamped to
 * [-1, 1]; *x_out gets x = e + r1 (1 - e) (r1 itself on the Haar branch). */
static float creutz_candidate(const struct creutz_setup *c, float r1, float *x_out)
{
    float cand;
    if (c->haar) {
        *x_out = r1;
        cand = 2.0f * r1 - 1.0f;
    } else {
        float x = fmaf(r1, c->one_minus_e, c->e);
        *x_out = x;
        cand = 1.0f + orc_logf(x) * c->inv_bk;
    }
    if (cand < -1.0f) cand = -1.0f;
    if (cand > 1.0f) cand = 1.0f;
    return cand;
}

int orc_heatbath_link(float beta, const float v[4], uint64_t seed, uint32_t eo, uint32_t sweep,
                      int parity, int mu, float out[4])
{
    float k = sqrtf(dot4(v[0], v[0], v[1], v[1], v[2], v[2], v[3], v[3]));
    float ut[4];
    if (k > 0.0f) {
        float inv_k = 1.0f / k;
        ut[0] = v[0] * inv_k;
        ut[1] = -v[1] * inv_k;
        ut[2] = -v[2] * inv_k;
        ut[3] = -v[3] * inv_k;
    } else {
        ut[0] = 1.0f; ut[1] = 0.0f; ut[2] = 0.0f; ut[3] = 0.0f;
    }
    const struct creutz_setup setup = creutz_prepare(beta * k);

    float a0 = 0.0f;
    int trials = 0;
    int accepted = 0;
    uint32_t w[4];
    for (int t = 0; t < ORC_MAX_TRIALS; ++t) {
        if ((t & 1) == 0) draw_words(seed, eo, sweep, ORC_KIND_CREUTZ, parity, mu, (uint32_t)(t >> 1), w);
        float r1 = orc_u01_log(w[2 * (t & 1)]); /* the argument of the log */
        float r2 = orc_u01(w[2 * (t & 1) + 1]);
        float x;
        float cand = creutz_candidate(&setup, r1, &x);
        trials = t + 1;
        if (r2 * r2 <= fmaf(-cand, cand, 1.0f)) {
            a0 = cand;
            accepted = 1;
            break;
        }
    }
    if (!accepted) return -1;

    heatbath_direction(a0, ut, seed, eo, sweep, parity, mu, out);
    return trials;
}

/* a0 alone, as drawn for a link whose staple has beta k = bk (sampler tests).
 * Uses the Creutz stream of (seed, eo, sweep, parity, mu); *trials gets the
 * number of trials (or -1). */
float orc_creutz_a0(float bk, uint64_t seed, uint32_t eo, uint32_t sweep, int parity, int mu, int *trials)
{
    /* a staple along the identity with |V| = bk and beta = 1 gives exactly this bk */
    float v[4] = {bk, 0.0f, 0.0f, 0.0f};
    float out[4];
    int n = orc_heatbath_link(1.0f, v, seed, eo, sweep, parity, mu, out);
    *trials = n;
    return out[0];
}

/* x and the candidate a0 of single Creutz trials: trial i has beta k = bk[i]
 * (from a staple along the identity with |V| = bk[i], beta = 1, as in
 * orc_creutz_a0) and its first word w[i]; x = e + r1 (1 - e), r1 the log
 * uniform of w[i].  Lets a test compare the device's trial variable with the
 * definition for chosen words (the smallest included). */
void orc_creutz_x_a0_v(const float *bk, const uint32_t *w, int64_t n, float *x, float *a0)
{
    for (int64_t i = 0; i < n; ++i) {
        const float v[4] = {bk[i], 0.0f, 0.0f, 0.0f};
        const float k = sqrtf(dot4(v[0], v[0], v[1], v[1], v[2], v[2], v[3], v[3]));
        const struct creutz_setup setup = creutz_prepare(1.0f * k);
        a0[i] = creutz_candidate(&setup, orc_u01_log(w[i]), &x[i]);
    }
}

/* One heat-bath phase: every link U_mu(x) with parity(x) = p (Sec. 4).  The
 * checkerboard makes the order of sites irrelevant, so the loop may be split
 * across threads.  trials_out gets the number of trials; returns the number
 * of links whose sampler hit the trial cap. */
int64_t orc_heatbath_phase(int ns, int nt, double beta, uint64_t seed, uint32_t sweep, int mu, int p,
                           float *links, int64_t *trials_out, int nthreads)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
    float beta_f = (float)beta;
    int64_t trials = 0, errors = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) reduction(+ : trials, errors) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < vol; ++s) {
        if (site_parity(s, ns) != p) continue;
        float v[4];
        orc_staple(ns, nt, links, s, mu, v);
        float *l = links + (s * 4 + mu) * 4;
        int n = orc_heatbath_link(beta_f, v, seed, (uint32_t)(s >> 1), sweep, p, mu, l);
        if (n < 0) {
            errors += 1;
            trials += ORC_MAX_TRIALS;
        } else {
            trials += n;
        }
    }
    (void)nthreads;
    *trials_out = trials;
    return errors;
}

/* One sweep = for mu = 0..3: even sites, then odd sites (Sec. 4).
 * trials[2 mu + p] gets the trial count of each phase. */
int64_t orc_heatbath_sweep(int ns, int nt, double beta, uint64_t seed, uint32_t sweep, float *links,
                           int64_t trials[8], int nthreads)
{
    int64_t errors = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int p = 0; p < 2; ++p)
            errors += orc_heatbath_phase(ns, nt, beta, seed, sweep, mu, p, links, &trials[2 * mu + p], nthreads);
    return errors;
}

/* ------------------------------------------------------------------------ */
/* Observables (Sec. 4: plaquette per site, Polyakov loop per site, global   */
/* sum).  Per-site values in binary32 (same contract as the updates), summed */
/* in binary64; the _f64 variants do all arithmetic in binary64.             */
/* ------------------------------------------------------------------------ */
/* (1/2) Tr of U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag, summed over the
 * six planes mu < nu in the order (0,1),(0,2),(0,3),(1,2),(1,3),(2,3). */
float orc_site_plaquette(int ns, int nt, const float *links, int64_t s)
{
    float sum = 0.0f;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
            int64_t xmu = site_shift(s, mu, +1, ns, nt);
            int64_t xnu = site_shift(s, nu, +1, ns, nt);
            float t1[4], t2[4], d[4], full[4];
            orc_quat_mul(link_at(links, s, mu), link_at(links, xmu, nu), t1);
            quat_dag(link_at(links, xnu, mu), d);
            orc_quat_mul(t1, d, t2);
            quat_dag(link_at(links, s, nu), d);
            orc_quat_mul(t2, d, full);
            sum = sum + full[0];
        }
    return sum;
}

double orc_plaquette(int ns, int nt, const float *links)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
    double acc = 0.0;
    for (int64_t s = 0; s < vol; ++s) acc += (double)orc_site_plaquette(ns, nt, links, s);
    return acc / (6.0 * (double)vol);
}

void orc_site_plaquettes(int ns, int nt, const float *links, float *out)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
    for (int64_t s = 0; s < vol; ++s) out[s] = orc_site_plaquette(ns, nt, links, s);
}

static void qmul_d(const double a[4], const double b[4], double c[4])
{
    double r0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double r1 = a[0] * b[1] + a[1] * b[0] - a[2] * b[3] + a[3] * b[2];
    double r2 = a[0] * b[2] + a[2] * b[0] - a[3] * b[1] + a[1] * b[3];
    double r3 = a[0] * b[3] + a[3] * b[0] - a[1] * b[2] + a[2] * b[1];
    c[0] = r0; c[1] = r1; c[2] = r2; c[3] = r3;
}

static void load_d(const float *links, int64_t s, int mu, int dag, double q[4])
{
    const float *l = link_at(links, s, mu);
    q[0] = (double)l[0];
    for (int c = 1; c < 4; ++c) q[c] = dag ? -(double)l[c] : (double)l[c];
}

double orc_plaquette_f64(int ns, int nt, const float *links)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
    double acc = 0.0;
    for (int64_t s = 0; s < vol; ++s)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                double a[4], b[4], t1[4], t2[4], full[4];
                load_d(links, s, mu, 0, a);
                load_d(links, site_shift(s, mu, +1, ns, nt), nu, 0, b);
                qmul_d(a, b, t1);
                load_d(links, site_shift(s, nu, +1, ns, nt), mu, 1, a);
                qmul_d(t1, a, t2);
                load_d(links, s, nu, 1, a);
                qmul_d(t2, a, full);
                acc += full[0];
            }
    return acc / (6.0 * (double)vol);
}

/* Polyakov loop at spatial site xs: (1/2) Tr of U_3(xs,0) U_3(xs,1) ...
 * U_3(xs,Nt-1), multiplied left to right. */
float orc_site_polyakov(int ns, int nt, const float *links, int64_t xs)
{
    int64_t vs = (int64_t)ns * ns * ns;
    float p[4];
    memcpy(p, link_at(links, xs, 3), sizeof p);
    for (int t = 1; t < nt; ++t) {
        float q[4];
        orc_quat_mul(p, link_at(links, xs + (int64_t)t * vs, 3), q);
        memcpy(p, q, sizeof p);
    }
    return p[0];
}

double orc_polyakov(int ns, int nt, const float *links)
{
    int64_t vs = (int64_t)ns * ns * ns;
    double acc = 0.0;
    for (int64_t xs = 0; xs < vs; ++xs) acc += (double)orc_site_polyakov(ns, nt, links, xs);
    return acc / (double)vs;
}

double orc_polyakov_f64(int ns, int nt, const float *links)
{
    int64_t vs = (int64_t)ns * ns * ns;
    double acc = 0.0;
    for (int64_t xs = 0; xs < vs; ++xs) {
        double p[4], q[4], l[4];
        load_d(links, xs, 3, 0, p);
        for (int t = 1; t < nt; ++t) {
            load_d(links, xs + (int64_t)t * vs, 3, 0, l);
            qmul_d(p, l, q);
            memcpy(p, q, sizeof p);
        }
        acc += p[0];
    }
    return acc / (double)vs;
}

/* Projection back onto S^3: a <- a / sqrt(a.a). */
void orc_reunitarize(int ns, int nt, float *links)
{
    int64_t n = (int64_t)ns * ns * ns * nt * 4;
    for (int64_t i = 0; i < n; ++i) {
        float *a = links + i * 4;
        float nn = dot4(a[0], a[0], a[1], a[1], a[2], a[2], a[3], a[3]);
        float r = sqrtf(nn);
        a[0] = a[0] / r;
        a[1] = a[1] / r;
        a[2] = a[2] / r;
        a[3] = a[3] / r;
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Batch helpers for the statistical tests.                                  */
/* ------------------------------------------------------------------------ */
/* n draws of a0 at fixed beta k; draw i uses even/odd index eo0 + i. */
void orc_creutz_a0_v(float bk, uint64_t seed, uint32_t eo0, uint32_t sweep, int64_t n, float *a0, int32_t *trials)
{
    for (int64_t i = 0; i < n; ++i) {
        int t = 0;
        a0[i] = orc_creutz_a0(bk, seed, eo0 + (uint32_t)i, sweep, 0, 0, &t);
        trials[i] = t;
    }
}

/* n heat-bath updates of one link with a fixed staple v; update i uses sweep
 * number sweep0 + i (fresh draws each time).  out is float[n][4]. */
void orc_heatbath_link_v(float beta, const float v[4], uint64_t seed, uint32_t eo, uint32_t sweep0,
                         int parity, int mu, int64_t n, float *out, int32_t *trials)
{
    for (int64_t i = 0; i < n; ++i)
        trials[i] = orc_heatbath_link(beta, v, seed, eo, sweep0 + (uint32_t)i, parity, mu, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Kennedy-Pendleton a0 sampler (Phys. Lett. B 156 (1985) 393), the same    */
/* heat-bath law as Creutz's method with near-unit acceptance at large       */
/* beta k.  With a0 = 1 - 2u the law of u is u^{1/2} sqrt(1 - u) exp(-2 beta k u) */
/* on [0, 1]: u is drawn from the Gamma(3/2) part,                            */
/* u = -(ln r1 + cos^2(2 pi r2) ln r3) / (2 beta k) (an exponential plus half */
/* a squared Box-Muller normal), and accepted iff u <= 1 and r4^2 <= 1 - u.  */
/* Trial t uses the four uniforms of block t of the KP stream (kind 5).      */
/* Below beta k = 2 (where KP accepts poorly) the link is drawn by Creutz's  */
/* method exactly as orc_heatbath_link does.                                 */
/* ------------------------------------------------------------------------ */
#define ORC_KP_MIN_BK 2.0f
enum { ORC_KIND_KP = 5 };

int orc_heatbath_link_kp(float beta, const float v[4], uint64_t seed, uint32_t eo, uint32_t sweep, int parity, int mu,
                         float out[4])
{
    float k = sqrtf(dot4(v[0], v[0], v[1], v[1], v[2], v[2], v[3], v[3]));
    const float bk = beta * k;
    if (!(bk >= ORC_KP_MIN_BK)) return orc_heatbath_link(beta, v, seed, eo, sweep, parity, mu, out);
    const float inv_k = 1.0f / k;
    const float ut[4] = {v[0] * inv_k, -v[1] * inv_k, -v[2] * inv_k, -v[3] * inv_k};
    const float two_bk = 2.0f * bk;
    float a0 = 0.0f;
    int trials = 0;
    for (int t = 0; t < ORC_MAX_TRIALS; ++t) {
        uint32_t w[4];
        draw_words(seed, eo, sweep, ORC_KIND_KP, parity, mu, (uint32_t)t, w);
        /* words 0 and 2 feed logarithms */
        const float u[4] = {orc_u01_log(w[0]), orc_u01(w[1]), orc_u01_log(w[2]), orc_u01(w[3])};
        float sn, cs;
        orc_sincos2pi(u[1], &sn, &cs);
        const float num = fmaf(cs * cs, orc_logf(u[2]), orc_logf(u[0]));
        const float lam2 = -num / two_bk;
        if (lam2 <= 1.0f && u[3] * u[3] <= 1.0f - lam2) {
            a0 = fmaf(-2.0f, lam2, 1.0f);
            trials = t + 1;
            break;
        }
    }
    if (trials == 0) return -1;
    heatbath_direction(a0, ut, seed, eo, sweep, parity, mu, out);
    return trials;
}

int64_t orc_heatbath_phase_kp(int ns, int nt, double beta, uint64_t seed, uint32_t sweep, int mu, int p, float *links,
                              int64_t *trials_out, int nthreads)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
    float beta_f = (float)beta;
    int64_t trials = 0, errors = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) reduction(+ : trials, errors) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < vol; ++s) {
        if (site_parity(s, ns) != p) continue;
        float v[4];
        orc_staple(ns, nt, links, s, mu, v);
        float *l = links + (s * 4 + mu) * 4;
        int n = orc_heatbath_link_kp(beta_f, v, seed, (uint32_t)(s >> 1), sweep, p, mu, l);
        if (n < 0) {
            errors += 1;
            trials += ORC_MAX_TRIALS;
        } else {
            trials += n;
        }
    }
    (void)nthreads;
    *trials_out = trials;
    return errors;
}

int64_t orc_heatbath_sweep_kp(int ns, int nt, double beta, uint64_t seed, uint32_t sweep, float *links,
                              int64_t trials[8], int nthreads)
{
    int64_t errors = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int p = 0; p < 2; ++p)
            errors += orc_heatbath_phase_kp(ns, nt, beta, seed, sweep, mu, p, links, &trials[2 * mu + p], nthreads);
    return errors;
}

/* ------------------------------------------------------------------------ */
/* Time-slab decomposition (Sec. 4, multi-GPU part, Fig. 1): a rank holds     */
/* the Nt_local time slices t0 .. t0 + Nt_local - 1 of the Ns^3 x Nt lattice  */
/* plus one ghost slice on each side: an array of Ns^3 x (Nt_local + 2) sites */
/* in the natural layout, local slice tl = global slice (t0 - 1 + tl) mod Nt. */
/* A phase (mu, p) updates the interior links U_mu(x) with global parity p;   */
/* the staples read the ghosts for t +- 1 (no site of the interior wraps in  */
/* the local array), and the random numbers use the site's global even/odd   */
/* index and parity, so a slab phase is the lattice phase restricted to the   */
/* slab.  kp selects the Kennedy-Pendleton sampler.  Returns the cap hits.    */
/* ------------------------------------------------------------------------ */
int64_t orc_slab_phase(int ns, int nt, int t0, int nt_local, double beta, uint64_t seed, uint32_t sweep, int mu,
                       int p, int kp, float *slab, int64_t *trials_out, int nthreads)
{
    const int ntl = nt_local + 2;
    const int64_t vs = (int64_t)ns * ns * ns;
    const float beta_f = (float)beta;
    int64_t trials = 0, errors = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) reduction(+ : trials, errors) num_threads(nthreads)
#endif
    for (int64_t s = vs; s < (int64_t)(nt_local + 1) * vs; ++s) {
        int c[4];
        site_coords(s, ns, c);
        int g[4] = {c[0], c[1], c[2], (t0 - 1 + c[3] + nt) % nt};
        const int64_t sg = site_index(g, ns);
        if (site_parity(sg, ns) != p) continue;
        float v[4];
        orc_staple(ns, ntl, slab, s, mu, v);
        float *l = slab + (s * 4 + mu) * 4;
        int n = kp ? orc_heatbath_link_kp(beta_f, v, seed, (uint32_t)(sg >> 1), sweep, p, mu, l)
                   : orc_heatbath_link(beta_f, v, seed, (uint32_t)(sg >> 1), sweep, p, mu, l);
        if (n < 0) {
            errors += 1;
            trials += ORC_MAX_TRIALS;
        } else {
            trials += n;
        }
    }
    (void)nthreads;
    *trials_out = trials;
    return errors;
}

/* n draws of a0 at fixed beta k with the Kennedy-Pendleton sampler (draw i
 * uses even/odd index eo0 + i). */
void orc_kp_a0_v(float bk, uint64_t seed, uint32_t eo0, int64_t n, float *a0, int32_t *trials)
{
    const float v[4] = {bk, 0.0f, 0.0f, 0.0f};
    for (int64_t i = 0; i < n; ++i) {
        float out[4];
        trials[i] = orc_heatbath_link_kp(1.0f, v, seed, eo0 + (uint32_t)i, 0u, 0, 0, out);
        a0[i] = out[0];
    }
}

/* ------------------------------------------------------------------------ */
/* Over-relaxation: the microcanonical reflection of a link in its staple    */
/* (Adler, Phys. Rev. D 23 (1981) 2901; Creutz, Phys. Rev. D 36 (1987) 515;  */
/* Brown and Woch, Phys. Rev. Lett. 58 (1987) 2394).  It is not in the paper: */
/* it is the usual companion of the Sec. 2 heat bath.  With U~ = V/k,         */
/*   U' = U~^dag U^dag U~^dag,                                                */
/* so U' U~ = (U U~)^dag: the heat-bath variable a = U U~ is reflected to     */
/* a^dag, (1/2) Tr U'V = (1/2) Tr UV (the action is unchanged) and applying   */
/* the map twice gives U back.  No random numbers.  For k = 0 U~ is the       */
/* identity, as in the heat bath (the action does not depend on U then).      */
/* Products left to right: (U~^dag U^dag) U~^dag.                             */
/* ------------------------------------------------------------------------ */
void orc_overrelax_link(const float v[4], float u[4])
{
    float k = sqrtf(dot4(v[0], v[0], v[1], v[1], v[2], v[2], v[3], v[3]));
    float ut[4];
    if (k > 0.0f) {
        float inv_k = 1.0f / k;
        ut[0] = v[0] * inv_k;
        ut[1] = -v[1] * inv_k;
        ut[2] = -v[2] * inv_k;
        ut[3] = -v[3] * inv_k;
    } else {
        ut[0] = 1.0f; ut[1] = 0.0f; ut[2] = 0.0f; ut[3] = 0.0f;
    }
    float ud[4], t[4];
    quat_dag(u, ud);
    orc_quat_mul(ut, ud, t);
    orc_quat_mul(t, ut, u);
}

/* Every link U_mu(x) with parity(x) = p (links of one phase share no
 * plaquette, so the order of sites does not matter). */
void orc_overrelax_phase(int ns, int nt, int mu, int p, float *links, int nthreads)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < vol; ++s) {
        if (site_parity(s, ns) != p) continue;
        float v[4];
        orc_staple(ns, nt, links, s, mu, v);
        orc_overrelax_link(v, links + (s * 4 + mu) * 4);
    }
    (void)nthreads;
}

/* One over-relaxation sweep: mu = 0..3, even then odd, as the heat bath. */
void orc_overrelax_sweep(int ns, int nt, float *links, int nthreads)
{
    for (int mu = 0; mu < 4; ++mu)
        for (int p = 0; p < 2; ++p) orc_overrelax_phase(ns, nt, mu, p, links, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Wilson loops in the space-time planes, the next observables after the    */
/* plaquette and the Polyakov loop (not in the paper).  For a site x, a      */
/* spatial direction i and extents R (along i) and T (along t):              */
/*   S_R(y) = U_i(y) U_i(y+i) ... U_i(y+(R-1)i),                             */
/*   T_T(y) = U_t(y) U_t(y+t) ... U_t(y+(T-1)t)   (products left to right),  */
/*   A = S_R(x) T_T(x+R i),  B = T_T(x) S_R(x+T t),                          */
/*   W = (1/2) Tr A B^dag = A . B   (the four-component dot product),        */
/* which is the closed loop x -> x+Ri -> x+Ri+Tt -> x+Tt -> x.  Per loop in  */
/* binary32 with the link-arithmetic contract; the mean over x and i = 0..2  */
/* in binary64.  out[(R-1) tmax + (T-1)], R = 1..rmax, T = 1..tmax.          */
/* ------------------------------------------------------------------------ */
static int64_t site_step(int64_t s, int mu, int n, int ns, int nt)
{
    int c[4];
    site_coords(s, ns, c);
    int L = extent(ns, nt, mu);
    c[mu] = (int)(((int64_t)c[mu] + n) % L);
    return site_index(c, ns);
}

/* product of the n links U_mu(y) U_mu(y+mu) ... (n >= 1) */
static void line_product(const float *links, int64_t y, int mu, int n, int ns, int nt, float out[4])
{
    memcpy(out, link_at(links, y, mu), 4 * sizeof(float));
    for (int j = 1; j < n; ++j) {
        float t[4];
        orc_quat_mul(out, link_at(links, site_step(y, mu, j, ns, nt), mu), t);
        memcpy(out, t, sizeof t);
    }
}

float orc_wilson_loop_at(int ns, int nt, const float *links, int64_t s, int i, int R, int T)
{
    float sr_x[4], tt_xr[4], tt_x[4], sr_xt[4], a[4], b[4];
    line_product(links, s, i, R, ns, nt, sr_x);
    line_product(links, site_step(s, i, R, ns, nt), 3, T, ns, nt, tt_xr);
    line_product(links, s, 3, T, ns, nt, tt_x);
    line_product(links, site_step(s, 3, T, ns, nt), i, R, ns, nt, sr_xt);
    orc_quat_mul(sr_x, tt_xr, a);
    orc_quat_mul(tt_x, sr_xt, b);
    return dot4(a[0], b[0], a[1], b[1], a[2], b[2], a[3], b[3]);
}

void orc_wilson_loops(int ns, int nt, const float *links, int rmax, int tmax, double *out, int nthreads)
{
    int64_t vol = (int64_t)ns * ns * ns * nt;
    for (int R = 1; R <= rmax; ++R)
        for (int T = 1; T <= tmax; ++T) {
            double acc = 0.0;
#ifdef _OPENMP
            if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) reduction(+ : acc) num_threads(nthreads)
#endif
            for (int64_t s = 0; s < vol; ++s)
                for (int i = 0; i < 3; ++i) acc += (double)orc_wilson_loop_at(ns, nt, links, s, i, R, T);
            out[(R - 1) * tmax + (T - 1)] = acc / (3.0 * (double)vol);
        }
    (void)nthreads;
}
