/*
 * su2_oracle_learned.c -- CPU oracle of the learned a0 proposal.
 *
 * TEST INFRASTRUCTURE ONLY (see su2_oracle.c).  Shares no source with the
 * CUDA library.
 *
 * The heat-bath density of a0 given the staple (Sec. 2 of Cardoso & Bicudo),
 * p(a0) ~ sqrt(1 - a0^2) exp(beta k a0), is proposed by a monotone
 * rational-quadratic spline flow (Durkan, Bekasov, Murray, Papamakarios,
 * "Neural Spline Flows", NeurIPS 2019) whose 8 bins are set by a small MLP
 * of beta k; the proposal is used in an independence-Metropolis link step,
 * so the chain stays exact for any network.
 *
 * Network: s = (beta k - mean) * scale; h1 = relu(W1 s + b1) (32);
 * h2 = relu(W2 h1 + b2) (32); o = W3 h2 + b3 (25 = 8 widths, 8 heights,
 * 9 knot derivatives).  Weights as float[1947]: W1[32], b1[32], W2[32][32],
 * b2[32], W3[25][32], b3[25], mean, scale.
 * Spline on [-1,1]^2: widths 2 (m + (1 - 8m) softmax(o[0:8])), heights
 * likewise from o[8:16], m = 1e-3; derivatives 1e-3 + softplus(o[16:25]).
 * Knots x_0 = -1, x_{j+1} = x_j + w_j, x_8 = 1 (same for y).
 * Proposal: z uniform in (-1, 1], a0 = f(z), density q(a0) = 1 / (2 f'(z)).
 *
 * binary32 parts follow the same contract as su2_oracle.c (explicit fmaf,
 * no contraction, own exp/log series); the negative log-likelihood and its
 * gradient are binary64 (the training reference).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* from su2_oracle.c */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float orc_u01(uint32_t x);
float orc_u01_log(uint32_t x);
float orc_logf(float x);
float orc_expf(float y);
void orc_sincos2pi(float u, float *s, float *c);
void orc_quat_mul(const float a[4], const float b[4], float c[4]);
void orc_staple(int ns, int nt, const float *links, int64_t s, int mu, float v[4]);

#define LK 8           /* spline bins */
#define LH 32          /* hidden width */
#define LO 25          /* network outputs */
#define LP 27          /* spline parameters: x0..x8, y0..y8, d0..d8 */
#define LW 1945        /* trainable weights */
#define LW_ALL 1947    /* + input mean and scale */
#define MIN_BIN 1e-3f
#define MIN_DER 1e-3f
#define OFF_W1 0
#define OFF_B1 32
#define OFF_W2 64
#define OFF_B2 1088
#define OFF_W3 1120
#define OFF_B3 1920
#define OFF_MEAN 1945
#define OFF_SCALE 1946

enum { KIND_LEARNED = 3, KIND_COLLECT = 4 };

/* exp of y <= 0, 0 below the binary32 range of the series */
static float expf_neg(float y) { return y < -87.0f ? 0.0f : orc_expf(y); }

static float relu(float x) { return x > 0.0f ? x : 0.0f; }

/* ------------------------------------------------------------- network */
/* Each sum starts from the bias and adds w[i] * x[i] for i ascending, one
 * fmaf per term. */
void orc_mlp_forward(const float *w, float s, float o[LO])
{
    float h1[LH], h2[LH];
    for (int j = 0; j < LH; ++j) h1[j] = relu(fmaf(w[OFF_W1 + j], s, w[OFF_B1 + j]));
    for (int j = 0; j < LH; ++j) {
        float acc = w[OFF_B2 + j];
        for (int i = 0; i < LH; ++i) acc = fmaf(w[OFF_W2 + j * LH + i], h1[i], acc);
        h2[j] = relu(acc);
    }
    for (int j = 0; j < LO; ++j) {
        float acc = w[OFF_B3 + j];
        for (int i = 0; i < LH; ++i) acc = fmaf(w[OFF_W3 + j * LH + i], h2[i], acc);
        o[j] = acc;
    }
}

/* softmax of 8 values, then 2 (m + (1 - 8 m) p_i), accumulated into knots
 * starting at -1; the last knot is set to 1. */
static void knots_from(const float *o8, float *knots9)
{
    float mx = o8[0];
    for (int i = 1; i < LK; ++i) mx = o8[i] > mx ? o8[i] : mx;
    float e[LK], sum = 0.0f;
    for (int i = 0; i < LK; ++i) {
        e[i] = expf_neg(o8[i] - mx);
        sum = sum + e[i];
    }
    knots9[0] = -1.0f;
    for (int i = 0; i < LK - 1; ++i) {
        const float width = 2.0f * fmaf(1.0f - (float)LK * MIN_BIN, e[i] / sum, MIN_BIN);
        knots9[i + 1] = knots9[i] + width;
    }
    knots9[LK] = 1.0f;
}

/* softplus(t) = max(t, 0) + log(1 + exp(-|t|)) */
static float softplus(float t)
{
    const float at = t < 0.0f ? -t : t;
    return (t > 0.0f ? t : 0.0f) + orc_logf(1.0f + expf_neg(-at));
}

void orc_spline_params(const float o[LO], float p[LP])
{
    knots_from(o, p);
    knots_from(o + LK, p + LK + 1);
    for (int i = 0; i <= LK; ++i) p[2 * (LK + 1) + i] = MIN_DER + softplus(o[2 * LK + i]);
}

/* ----------------------------------------------------------- spline */
static int bin_of(const float *knots9, float v)
{
    int k = 0;
    for (int j = 1; j < LK; ++j)
        if (knots9[j] <= v) k = j;
    return k;
}

/* a = f(z) on bin k with xi = (z - x_k)/w, s = h/w, t = xi(1 - xi):
 * a = y_k + h (s xi^2 + d_k t) / (s + (d_{k+1} + d_k - 2 s) t),
 * f'(z) = s^2 (d_{k+1} xi^2 + 2 s t + d_k (1 - xi)^2) / den^2.
 * Rounding (ours, the formulas are Durkan et al.'s): with r = 1/den rounded
 * once, a = y_k + num r and f' = (s^2 m) r^2; the caller passes s. */
static float spline_eval(const float p[LP], int k, float xi, float s, float *fprime)
{
    const float *y = p + LK + 1, *d = p + 2 * (LK + 1);
    const float h = y[k + 1] - y[k];
    const float t = xi * (1.0f - xi);
    const float sigma = (d[k + 1] + d[k]) - 2.0f * s;
    const float den = fmaf(sigma, t, s);
    const float num = h * fmaf(s * xi, xi, d[k] * t);
    const float omx = 1.0f - xi;
    const float m = fmaf(d[k + 1] * xi, xi, fmaf(2.0f * s, t, d[k] * omx * omx));
    const float r = 1.0f / den;
    *fprime = (s * s * m) * (r * r);
    return y[k] + num * r;
}

/* xi = (z - x_k) iw and s = h iw with iw = 1/w rounded once. */
float orc_spline_forward(const float p[LP], float z, float *fprime)
{
    const float *y = p + LK + 1;
    const int k = bin_of(p, z);
    const float iw = 1.0f / (p[k + 1] - p[k]);
    const float s = (y[k + 1] - y[k]) * iw;
    float xi = (z - p[k]) * iw;
    xi = xi < 0.0f ? 0.0f : (xi > 1.0f ? 1.0f : xi);
    float a = spline_eval(p, k, xi, s, fprime);
    return a < -1.0f ? -1.0f : (a > 1.0f ? 1.0f : a);
}

/* Inverse on bin k of y: alpha xi^2 + beta xi + c = 0 with d = a - y_k,
 * alpha = h (s - d_k) + d sigma, beta = h d_k - d sigma, c = -s d,
 * xi = 2c / (-beta - sqrt(beta^2 - 4 alpha c)).  Returns xi's z and f'(z). */
float orc_spline_inverse(const float p[LP], float a, float *fprime)
{
    const float *x = p, *y = p + LK + 1, *d = p + 2 * (LK + 1);
    const int k = bin_of(y, a);
    const float w = x[k + 1] - x[k];
    const float h = y[k + 1] - y[k];
    const float s = h / w;
    const float dy = a - y[k];
    const float sigma = (d[k + 1] + d[k]) - 2.0f * s;
    const float alpha = fmaf(dy, sigma, h * (s - d[k]));
    const float beta = fmaf(-dy, sigma, h * d[k]);
    const float c = -s * dy;
    float disc = fmaf(beta, beta, -4.0f * alpha * c);
    disc = disc > 0.0f ? disc : 0.0f;
    const float denom = -beta - sqrtf(disc);
    float xi = denom != 0.0f ? (2.0f * c) / denom : 0.0f;
    xi = xi < 0.0f ? 0.0f : (xi > 1.0f ? 1.0f : xi);
    spline_eval(p, k, xi, s, fprime);
    return fmaf(xi, w, x[k]);
}

/* ------------------------------------------------------ proposal table */
/* Spline parameters of the network at G points s_j = s_lo + j (s_hi - s_lo)/(G-1). */
void orc_proposal_table(const float *w, float s_lo, float s_hi, int G, float *table)
{
    const float ds = (s_hi - s_lo) / (float)(G - 1);
    for (int j = 0; j < G; ++j) {
        float o[LO];
        orc_mlp_forward(w, fmaf((float)j, ds, s_lo), o);
        orc_spline_params(o, table + j * LP);
    }
}

/* Linear interpolation between the two grid rows around s (clamped to the grid). */
void orc_table_params(const float *table, int G, float s_lo, float s_hi, float s, float p[LP])
{
    const float inv_ds = (float)(G - 1) / (s_hi - s_lo);
    float u = (s - s_lo) * inv_ds;
    u = u < 0.0f ? 0.0f : (u > (float)(G - 1) ? (float)(G - 1) : u);
    int j = (int)floorf(u);
    if (j > G - 2) j = G - 2;
    const float f = u - (float)j;
    const float *r0 = table + j * LP, *r1 = table + (j + 1) * LP;
    for (int i = 0; i < LP; ++i) p[i] = fmaf(f, r1[i] - r0[i], r0[i]);
}

/* ------------------------------------------------- Metropolis link step */
/* Independence Metropolis for one link with staple v and current link old:
 * k = |v|, U~^dag = v^dag / k, a_cur = old U~ (the current heat-bath variable);
 * proposal a0' = f(z), z = 2 u0 - 1, direction from u2, u3 as in the heat
 * bath; accept with min(1, w(a0')/w(a_cur)), w(a) = sqrt(1 - a^2) e^{beta k a} f'(z(a))
 * (= target / proposal density up to constants), as u1 <= exp(Delta),
 * Delta = beta k (a0' - a_cur) + log(sqrt((1 - a0'^2)/(1 - a_cur^2)) f'(z')/f'(z_cur)).
 * All four uniforms come from one Philox block of the learned stream.
 *
 * The proposal's spline parameters are, by definition, the network's at
 * s = (beta k - mean) * scale (orc_learned_link_net).  orc_learned_link takes
 * them from the proposal table instead: the network at G grid points in s,
 * interpolated linearly, which is what the GPU kernel evaluates.  Both chains
 * are exact (acceptance and proposal use the same density); the tests bound
 * how far the table's density and acceptance are from the network's. */
static float staple_frame(const float v[4], float beta, float ut[4])
{
    const float k = sqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], fmaf(v[2], v[2], v[3] * v[3]))));
    ut[0] = 1.0f; ut[1] = 0.0f; ut[2] = 0.0f; ut[3] = 0.0f;
    if (k > 0.0f) {
        const float inv_k = 1.0f / k;
        ut[0] = v[0] * inv_k;
        ut[1] = -v[1] * inv_k;
        ut[2] = -v[2] * inv_k;
        ut[3] = -v[3] * inv_k;
    }
    return beta * k;
}

/* The step itself, given the link's spline parameters p; returns 1 if
 * accepted (out = new link), 0 if rejected (out = old). */
static int learned_step(const float p[LP], float bk, const float ut[4], const float old[4], uint64_t seed,
                        uint32_t eo, uint32_t sweep, int parity, int mu, float out[4])
{
    uint32_t ctr[4] = {eo, sweep, ((uint32_t)KIND_LEARNED << 3) | ((uint32_t)parity << 2) | (uint32_t)mu, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t wd[4];
    orc_philox4x32_10(ctr, key, wd);
    const float u0 = orc_u01(wd[0]), u1 = orc_u01(wd[1]), u2 = orc_u01(wd[2]), u3 = orc_u01(wd[3]);

    float fp_new, fp_cur;
    const float a_new = orc_spline_forward(p, 2.0f * u0 - 1.0f, &fp_new);
    /* current variable: a_cur = old U~, U~ = dag(ut): real part */
    float acur = fmaf(old[0], ut[0], fmaf(old[1], ut[1], fmaf(old[2], ut[2], old[3] * ut[3])));
    acur = acur < -1.0f ? -1.0f : (acur > 1.0f ? 1.0f : acur);
    orc_spline_inverse(p, acur, &fp_cur);

    const float one_cur = fmaf(-acur, acur, 1.0f);
    int accept;
    if (!(one_cur > 0.0f)) {
        accept = 1;
    } else {
        const float one_new = fmaf(-a_new, a_new, 1.0f);
        /* sqrt((1 - a'^2)/(1 - a^2)) f'(z')/f'(z) as one square root of one quotient */
        const float ratio = sqrtf((one_new * (fp_new * fp_new)) / (one_cur * (fp_cur * fp_cur)));
        if (!(ratio > 0.0f)) {
            accept = 0;
        } else {
            const float delta = fmaf(bk, a_new - acur, orc_logf(ratio));
            accept = delta >= 0.0f || u1 <= expf_neg(delta);
        }
    }
    if (!accept) {
        memcpy(out, old, 4 * sizeof(float));
        return 0;
    }
    const float r = sqrtf(fmaf(-a_new, a_new, 1.0f));
    const float c = 2.0f * u2 - 1.0f;
    const float st = sqrtf(fmaf(-c, c, 1.0f));
    float sn, cs;
    orc_sincos2pi(u3, &sn, &cs);
    const float rs = r * st;
    const float a[4] = {a_new, rs * cs, rs * sn, r * c};
    orc_quat_mul(a, ut, out);
    return 1;
}

/* The step with the table's interpolated spline parameters (the kernel's). */
int orc_learned_link(const float *table, int G, float s_lo, float s_hi, float mean, float scale, float beta,
                     const float v[4], const float old[4], uint64_t seed, uint32_t eo, uint32_t sweep, int parity,
                     int mu, float out[4])
{
    float ut[4];
    const float bk = staple_frame(v, beta, ut);
    float p[LP];
    orc_table_params(table, G, s_lo, s_hi, (bk - mean) * scale, p);
    return learned_step(p, bk, ut, old, seed, eo, sweep, parity, mu, out);
}

/* The step with the network evaluated at this link's beta k: the proposal
 * as defined (w holds the weights, then the input mean and scale). */
int orc_learned_link_net(const float *w, float beta, const float v[4], const float old[4], uint64_t seed,
                         uint32_t eo, uint32_t sweep, int parity, int mu, float out[4])
{
    float ut[4];
    const float bk = staple_frame(v, beta, ut);
    float o[LO], p[LP];
    orc_mlp_forward(w, (bk - w[OFF_MEAN]) * w[OFF_SCALE], o);
    orc_spline_params(o, p);
    return learned_step(p, bk, ut, old, seed, eo, sweep, parity, mu, out);
}

/* lattice helpers (same geometry as su2_oracle.c) */
static int lattice_parity(int64_t s, int ns)
{
    int c0 = (int)(s % ns);
    s /= ns;
    int c1 = (int)(s % ns);
    s /= ns;
    int c2 = (int)(s % ns);
    int c3 = (int)(s / ns);
    return (c0 + c1 + c2 + c3) & 1;
}

/* One learned phase (mu, parity); returns the number of accepted links. */
int64_t orc_learned_phase(int ns, int nt, double beta, uint64_t seed, uint32_t sweep, int mu, int p, float *links,
                          const float *table, int G, float s_lo, float s_hi, float mean, float scale)
{
    const int64_t vol = (int64_t)ns * ns * ns * nt;
    int64_t acc = 0;
    for (int64_t s = 0; s < vol; ++s) {
        if (lattice_parity(s, ns) != p) continue;
        float v[4], old[4], out[4];
        orc_staple(ns, nt, links, s, mu, v);
        float *l = links + (s * 4 + mu) * 4;
        memcpy(old, l, sizeof old);
        acc += orc_learned_link(table, G, s_lo, s_hi, mean, scale, (float)beta, v, old, seed, (uint32_t)(s >> 1), sweep,
                                p, mu, out);
        memcpy(l, out, sizeof out);
    }
    return acc;
}

int64_t orc_learned_sweep(int ns, int nt, double beta, uint64_t seed, uint32_t sweep, float *links, const float *table,
                          int G, float s_lo, float s_hi, float mean, float scale, int64_t accepted[8])
{
    int64_t total = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int p = 0; p < 2; ++p) {
            accepted[2 * mu + p] =
                orc_learned_phase(ns, nt, beta, seed, sweep, mu, p, links, table, G, s_lo, s_hi, mean, scale);
            total += accepted[2 * mu + p];
        }
    return total;
}

/* One sweep of the learned step with the network evaluated per link (the
 * definition); returns the number of accepted links, per phase in accepted[]. */
int64_t orc_learned_sweep_net(int ns, int nt, double beta, uint64_t seed, uint32_t sweep, float *links,
                              const float *w, int64_t accepted[8])
{
    const int64_t vol = (int64_t)ns * ns * ns * nt;
    int64_t total = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int p = 0; p < 2; ++p) {
            int64_t acc = 0;
            for (int64_t s = 0; s < vol; ++s) {
                if (lattice_parity(s, ns) != p) continue;
                float v[4], old[4], out[4];
                orc_staple(ns, nt, links, s, mu, v);
                float *l = links + (s * 4 + mu) * 4;
                memcpy(old, l, sizeof old);
                acc += orc_learned_link_net(w, (float)beta, v, old, seed, (uint32_t)(s >> 1), sweep, p, mu, out);
                memcpy(l, out, sizeof out);
            }
            accepted[2 * mu + p] = acc;
            total += acc;
        }
    return total;
}

/* ----------------------------------------------------- training pairs */
/* (beta k, a0) pairs for the links U_mu(x) of parity p whose even/odd index
 * is a multiple of `stride`: a0 is a fresh Creutz draw (the plain heat-bath
 * sampler, Sec. 2) on the collection stream, so the pair follows the exact
 * conditional law given the current staple.  Returns the number of pairs.
 * Trial t uses words 2(t&1), 2(t&1)+1 of collection block t>>1. */
int64_t orc_collect_pairs(int ns, int nt, double beta, uint64_t seed, uint32_t sweep, int mu, int p, int stride,
                          const float *links, float *pairs)
{
    const int64_t vol = (int64_t)ns * ns * ns * nt;
    const float beta_f = (float)beta;
    int64_t n = 0;
    for (int64_t s = 0; s < vol; ++s) {
        if (lattice_parity(s, ns) != p) continue;
        const uint32_t eo = (uint32_t)(s >> 1);
        if (eo % (uint32_t)stride != 0u) continue;
        float v[4];
        orc_staple(ns, nt, links, s, mu, v);
        const float k = sqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], fmaf(v[2], v[2], v[3] * v[3]))));
        const float bk = beta_f * k;
        const int haar = bk < 1e-6f;
        float e = 0.0f;
        if (!haar && bk <= 43.0f) e = orc_expf(-2.0f * bk);
        const float ome = 1.0f - e;
        const float inv_bk = haar ? 0.0f : 1.0f / bk; /* as in orc_heatbath_link */
        float a0 = 0.0f, u[4] = {0, 0, 0, 0};
        int got = 0;
        for (int t = 0; t < 4096 && !got; ++t) {
            if ((t & 1) == 0) {
                uint32_t ctr[4] = {eo, sweep, ((uint32_t)KIND_COLLECT << 3) | ((uint32_t)p << 2) | (uint32_t)mu,
                                   (uint32_t)(t >> 1)};
                uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
                uint32_t wd[4];
                orc_philox4x32_10(ctr, key, wd);
                /* words 0 and 2 feed the logarithm, as in orc_heatbath_link */
                u[0] = orc_u01_log(wd[0]);
                u[1] = orc_u01(wd[1]);
                u[2] = orc_u01_log(wd[2]);
                u[3] = orc_u01(wd[3]);
            }
            const float r1 = u[2 * (t & 1)], r2 = u[2 * (t & 1) + 1];
            float cand = haar ? 2.0f * r1 - 1.0f : 1.0f + orc_logf(fmaf(r1, ome, e)) * inv_bk;
            cand = cand < -1.0f ? -1.0f : (cand > 1.0f ? 1.0f : cand);
            if (r2 * r2 <= fmaf(-cand, cand, 1.0f)) {
                a0 = cand;
                got = 1;
            }
        }
        pairs[2 * n] = bk;
        pairs[2 * n + 1] = a0;
        ++n;
    }
    return n;
}

/* ================================================== binary64 training */
static double softplus_d(double t) { return (t > 0 ? t : 0) + log1p(exp(-fabs(t))); }
static double sigmoid_d(double t) { return t >= 0 ? 1.0 / (1.0 + exp(-t)) : exp(t) / (1.0 + exp(t)); }

typedef struct {
    double x[LK + 1], y[LK + 1], d[LK + 1];
    double pw[LK], ph[LK]; /* softmax probabilities */
} spline_d;

static void spline_from_outputs_d(const double o[LO], spline_d *sp)
{
    for (int part = 0; part < 2; ++part) {
        const double *oo = o + part * LK;
        double *prob = part ? sp->ph : sp->pw;
        double *kn = part ? sp->y : sp->x;
        double mx = oo[0];
        for (int i = 1; i < LK; ++i) mx = oo[i] > mx ? oo[i] : mx;
        double sum = 0;
        for (int i = 0; i < LK; ++i) {
            prob[i] = exp(oo[i] - mx);
            sum += prob[i];
        }
        kn[0] = -1.0;
        for (int i = 0; i < LK; ++i) {
            prob[i] /= sum;
            kn[i + 1] = kn[i] + 2.0 * ((double)MIN_BIN + (1.0 - LK * (double)MIN_BIN) * prob[i]);
        }
    }
    for (int i = 0; i <= LK; ++i) sp->d[i] = (double)MIN_DER + softplus_d(o[2 * LK + i]);
}

/* -log q(a) = log 2 + log f'(f^{-1}(a)) and, if g != NULL, its gradient
 * with respect to the 25 network outputs (implicit differentiation of
 * f(z) = a at fixed a, then through the knot sums, softmax and softplus). */
static double nll_outputs_d(const double o[LO], double a, double *g)
{
    spline_d sp;
    spline_from_outputs_d(o, &sp);
    int k = 0;
    for (int j = 1; j < LK; ++j)
        if (sp.y[j] <= a) k = j;
    const double W = sp.x[k + 1] - sp.x[k], H = sp.y[k + 1] - sp.y[k];
    const double D0 = sp.d[k], D1 = sp.d[k + 1];
    const double s = H / W, dy = a - sp.y[k];
    const double sig = D1 + D0 - 2 * s;
    const double al = H * (s - D0) + dy * sig, be = H * D0 - dy * sig, c = -s * dy;
    double disc = be * be - 4 * al * c;
    if (disc < 0) disc = 0;
    double xi = 2 * c / (-be - sqrt(disc));
    if (!(xi >= 0)) xi = 0;
    if (xi > 1) xi = 1;
    const double t = xi * (1 - xi);
    const double N = s * xi * xi + D0 * t, Dn = s + sig * t;
    const double M = D1 * xi * xi + 2 * s * t + D0 * (1 - xi) * (1 - xi);
    const double L = 2 * log(s) + log(M) - 2 * log(Dn);
    if (g) {
        const double Np = 2 * s * xi + D0 * (1 - 2 * xi), Dnp = sig * (1 - 2 * xi);
        const double Mp = 2 * D1 * xi + 2 * s * (1 - 2 * xi) - 2 * D0 * (1 - xi);
        const double F_xi = H * (Np * Dn - N * Dnp) / (Dn * Dn);
        const double L_xi = Mp / M - 2 * Dnp / Dn;
        const double F_Y = 1, F_H = N / Dn;
        const double F_s = H * (xi * xi * Dn - N * (1 - 2 * t)) / (Dn * Dn);
        const double F_D0 = H * t * (Dn - N) / (Dn * Dn);
        const double F_D1 = -H * N * t / (Dn * Dn);
        const double L_s = 2 / s + 2 * t / M - 2 * (1 - 2 * t) / Dn;
        const double L_D0 = (1 - xi) * (1 - xi) / M - 2 * t / Dn;
        const double L_D1 = xi * xi / M - 2 * t / Dn;
        const double dY = -L_xi * F_Y / F_xi;
        const double dHd = -L_xi * F_H / F_xi;
        const double ds = L_s - L_xi * F_s / F_xi;
        const double dD0 = L_D0 - L_xi * F_D0 / F_xi;
        const double dD1 = L_D1 - L_xi * F_D1 / F_xi;
        const double dH = dHd + ds / W, dW = -ds * H / (W * W);
        double gx[LK + 1] = {0}, gy[LK + 1] = {0}, gd[LK + 1] = {0};
        gy[k] += dY - dH;
        gy[k + 1] += dH;
        gx[k] -= dW;
        gx[k + 1] += dW;
        gd[k] += dD0;
        gd[k + 1] += dD1;
        for (int part = 0; part < 2; ++part) {
            const double *gk = part ? gy : gx;
            const double *prob = part ? sp.ph : sp.pw;
            double gw[LK];
            for (int i = 0; i < LK; ++i) {
                gw[i] = 0;
                for (int j = i + 1; j <= LK; ++j) gw[i] += gk[j];
                gw[i] *= 2.0 * (1.0 - LK * (double)MIN_BIN);
            }
            double dot = 0;
            for (int i = 0; i < LK; ++i) dot += gw[i] * prob[i];
            for (int m = 0; m < LK; ++m) g[part * LK + m] = prob[m] * (gw[m] - dot);
        }
        for (int i = 0; i <= LK; ++i) g[2 * LK + i] = gd[i] * sigmoid_d(o[2 * LK + i]);
    }
    return log(2.0) + L;
}

/* Mean NLL over n pairs (beta k, a0) and, if grad != NULL, its gradient with
 * respect to the 1945 trainable weights (w in the float[1947] layout, here
 * binary64; w[1945], w[1946] = input mean and scale, not trained). */
double orc_nll_grad(const double *w, const float *pairs, int64_t n, double *grad)
{
    if (grad) memset(grad, 0, sizeof(double) * LW);
    double total = 0;
    for (int64_t q = 0; q < n; ++q) {
        const double s = ((double)pairs[2 * q] - w[OFF_MEAN]) * w[OFF_SCALE];
        const double a = (double)pairs[2 * q + 1];
        double z1[LH], h1[LH], z2[LH], h2[LH], o[LO];
        for (int j = 0; j < LH; ++j) {
            z1[j] = w[OFF_W1 + j] * s + w[OFF_B1 + j];
            h1[j] = z1[j] > 0 ? z1[j] : 0;
        }
        for (int j = 0; j < LH; ++j) {
            double acc = w[OFF_B2 + j];
            for (int i = 0; i < LH; ++i) acc += w[OFF_W2 + j * LH + i] * h1[i];
            z2[j] = acc;
            h2[j] = acc > 0 ? acc : 0;
        }
        for (int j = 0; j < LO; ++j) {
            double acc = w[OFF_B3 + j];
            for (int i = 0; i < LH; ++i) acc += w[OFF_W3 + j * LH + i] * h2[i];
            o[j] = acc;
        }
        double go[LO];
        total += nll_outputs_d(o, a, grad ? go : NULL);
        if (!grad) continue;
        double gh2[LH] = {0}, gh1[LH] = {0};
        for (int j = 0; j < LO; ++j) {
            grad[OFF_B3 + j] += go[j];
            for (int i = 0; i < LH; ++i) {
                grad[OFF_W3 + j * LH + i] += go[j] * h2[i];
                gh2[i] += go[j] * w[OFF_W3 + j * LH + i];
            }
        }
        for (int j = 0; j < LH; ++j) {
            const double gz = z2[j] > 0 ? gh2[j] : 0;
            grad[OFF_B2 + j] += gz;
            for (int i = 0; i < LH; ++i) {
                grad[OFF_W2 + j * LH + i] += gz * h1[i];
                gh1[i] += gz * w[OFF_W2 + j * LH + i];
            }
        }
        for (int j = 0; j < LH; ++j) {
            const double gz = z1[j] > 0 ? gh1[j] : 0;
            grad[OFF_B1 + j] += gz;
            grad[OFF_W1 + j] += gz * s;
        }
    }
    if (grad)
        for (int i = 0; i < LW; ++i) grad[i] /= (double)n;
    return total / (double)n;
}

/* binary64 spline of given outputs for the pins: f(z), f'(z), f^{-1}(a) */
void orc_spline_d(const double o[LO], double z, double *a, double *fprime, double *zinv_of_a)
{
    spline_d sp;
    spline_from_outputs_d(o, &sp);
    int k = 0;
    for (int j = 1; j < LK; ++j)
        if (sp.x[j] <= z) k = j;
    const double W = sp.x[k + 1] - sp.x[k], H = sp.y[k + 1] - sp.y[k];
    const double s = H / W, xi = (z - sp.x[k]) / W, t = xi * (1 - xi);
    const double sig = sp.d[k + 1] + sp.d[k] - 2 * s, Dn = s + sig * t;
    *a = sp.y[k] + H * (s * xi * xi + sp.d[k] * t) / Dn;
    *fprime = s * s * (sp.d[k + 1] * xi * xi + 2 * s * t + sp.d[k] * (1 - xi) * (1 - xi)) / (Dn * Dn);
    /* inverse of the value *a */
    const double av = *a;
    int kk = 0;
    for (int j = 1; j < LK; ++j)
        if (sp.y[j] <= av) kk = j;
    const double W2 = sp.x[kk + 1] - sp.x[kk], H2 = sp.y[kk + 1] - sp.y[kk], s2 = H2 / W2, dy = av - sp.y[kk];
    const double sig2 = sp.d[kk + 1] + sp.d[kk] - 2 * s2;
    const double al = H2 * (s2 - sp.d[kk]) + dy * sig2, be = H2 * sp.d[kk] - dy * sig2, c = -s2 * dy;
    double disc = be * be - 4 * al * c;
    if (disc < 0) disc = 0;
    const double xi2 = 2 * c / (-be - sqrt(disc));
    *zinv_of_a = sp.x[kk] + xi2 * W2;
}

/* -log q for given outputs (pins: normalisation, finite differences) */
double orc_nll_outputs(const double o[LO], double a, double *g) { return nll_outputs_d(o, a, g); }

/* ------------------------------------------------------ batch helpers */
/* n successive learned updates of one link with a fixed staple (sweep
 * numbers 0..n-1); a0_out[i] = real part of U_i U~ after step i. */
int64_t orc_learned_chain(const float *table, int G, float s_lo, float s_hi, float mean, float scale, float beta,
                          const float v[4], const float old0[4], uint64_t seed, int64_t n, float *a0_out)
{
    float cur[4], nxt[4];
    memcpy(cur, old0, sizeof cur);
    const float k = sqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], fmaf(v[2], v[2], v[3] * v[3]))));
    const float inv_k = 1.0f / k;
    const float ut[4] = {v[0] * inv_k, -v[1] * inv_k, -v[2] * inv_k, -v[3] * inv_k};
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) {
        acc += orc_learned_link(table, G, s_lo, s_hi, mean, scale, beta, v, cur, seed, 7u, (uint32_t)i, 0, 0, nxt);
        memcpy(cur, nxt, sizeof cur);
        a0_out[i] = fmaf(cur[0], ut[0], fmaf(cur[1], ut[1], fmaf(cur[2], ut[2], cur[3] * ut[3])));
    }
    return acc;
}

/* orc_learned_chain with the network evaluated per step (the definition). */
int64_t orc_learned_chain_net(const float *w, float beta, const float v[4], const float old0[4], uint64_t seed,
                              int64_t n, float *a0_out)
{
    float cur[4], nxt[4], ut[4];
    memcpy(cur, old0, sizeof cur);
    staple_frame(v, beta, ut);
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) {
        acc += orc_learned_link_net(w, beta, v, cur, seed, 7u, (uint32_t)i, 0, 0, nxt);
        memcpy(cur, nxt, sizeof cur);
        a0_out[i] = fmaf(cur[0], ut[0], fmaf(cur[1], ut[1], fmaf(cur[2], ut[2], cur[3] * ut[3])));
    }
    return acc;
}

void orc_spline_forward_v(const float *p, const float *z, float *a, float *fp, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) a[i] = orc_spline_forward(p, z[i], &fp[i]);
}

void orc_spline_inverse_v(const float *p, const float *a, float *z, float *fp, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) z[i] = orc_spline_inverse(p, a[i], &fp[i]);
}
