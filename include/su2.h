/*
 * su2.h -- C ABI of the GB300 (sm_103a) lattice SU(2) heat-bath library.
 *
 * Pure-gauge SU(2) on an Ns^3 x Nt periodic lattice with the Wilson action,
 * updated by the checkerboard heat bath of Cardoso & Bicudo, "Lattice SU(2) on
 * GPU's" (LAT2010):
 *   Sec. 2  links are SU(2) elements U = a0 + i a.sigma stored as quaternions
 *           (a0, a1, a2, a3), |a| = 1; each link is redrawn from
 *           dP(U) ~ exp(beta/2 Tr(U V)) where V is the staple (sum of the six
 *           three-link products around U); with k = sqrt(det V) and
 *           U~ = V/k, a0 is drawn from sqrt(1-a0^2) exp(beta k a0), the vector
 *           part uniformly on the sphere of radius sqrt(1-a0^2), and the new
 *           link is U' = a U~^{-1}.
 *   Sec. 4  one iteration (sweep) updates, for mu = 0..3 in order, first the
 *           even then the odd sites; kernels for cold start, hot start,
 *           heat bath, plaquette, Polyakov loop and the global sum.
 *
 * Conventions common to every call:
 *   - Every call returns an su2_status; nothing is thrown across the ABI.
 *     On SU2_E_CUDA the text of the CUDA error is kept per thread and is
 *     returned by su2_last_error().
 *   - Host buffers are owned by the caller.  Device memory of a lattice is
 *     owned by the library (allocated through the hook of su2_set_allocator,
 *     else cudaMallocAsync on the lattice's stream) and freed by su2_destroy.
 *   - All device work of a lattice is ordered on the CUDA stream given to
 *     su2_create (NULL = the legacy default stream).  Calls that return host
 *     values (observables, links, statistics) synchronise that stream.
 *   - A handle is not thread-safe: one thread at a time per handle.
 *   - Directions: mu = 0,1,2 are x,y,z (extent Ns), mu = 3 is time (extent Nt).
 *     Sites are numbered lexicographically, lex = ((t*Ns + z)*Ns + y)*Ns + x;
 *     the parity of a site is (x+y+z+t) mod 2.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 *     counter (even/odd site index, sweep, stream kind/parity/mu, block), so a
 *     run is a pure function of (start, seed, beta, sweep count).  A 32-bit
 *     word w becomes the uniform ((w >> 8) + 1) 2^-24 in (0, 1], or, where the
 *     uniform is the argument of a logarithm (Creutz's x, the
 *     Kennedy-Pendleton exponentials), w 2^-32 + 2^-33 rounded once, in
 *     [2^-33, 1], so that -ln x is not cut at 24 ln 2.
 */
#ifndef SU2_H
#define SU2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SU2_ABI_VERSION 3

typedef struct su2_lattice su2_lattice;

typedef enum {
    SU2_COLD = 0, /* all links = identity (Sec. 4, cold start)            */
    SU2_HOT = 1   /* all links Haar-random on S^3 (Sec. 4, hot start)     */
} su2_start;

typedef enum {
    SU2_OK = 0,
    SU2_E_INVAL = 1,          /* bad argument (odd or < 2 extent, beta < 0 or not finite, NULL) */
    SU2_E_NOMEM = 2,          /* device or host allocation failed                                */
    SU2_E_CUDA = 3,           /* a CUDA call failed; see su2_last_error()                        */
    SU2_E_SAMPLER = 4,        /* a heat-bath draw hit its trial cap (link left unchanged)        */
    SU2_E_DEVICE_TIMEOUT = 5, /* a bounded device wait gave up                                   */
    SU2_E_NUMERIC = 6,        /* non-finite value met                                            */
    SU2_E_STATE = 7           /* call not valid in the handle's current state                    */
} su2_status;

/* Per-call statistics, filled by the sweep calls when the pointer is non-NULL. */
typedef struct {
    uint64_t sweeps;            /* sweeps performed by the call                               */
    uint64_t link_updates;      /* 4 V per sweep                                              */
    uint64_t trials[8];         /* heat-bath a0 trials of phase 2*mu + parity, summed over sweeps */
    uint64_t sampler_failures;  /* links whose draw hit the trial cap                         */
    uint32_t kernel_launches;   /* heat-bath phase launches (8 per sweep)                     */
    uint32_t timed;             /* 1 if kernel_ms / overrelax_ms are valid (su2_set_timing)   */
    double kernel_ms;           /* summed device time of the heat-bath phase kernels          */
    uint64_t overrelax_sweeps;  /* over-relaxation sweeps performed (see su2_set_overrelax)   */
    uint64_t overrelax_updates; /* 4 V per over-relaxation sweep                              */
    double overrelax_ms;        /* summed device time of the over-relaxation phase kernels    */
} su2_stats;

/* Resumable state: with the links (su2_get_links) it determines every later sweep. */
typedef struct {
    int32_t ns, nt;
    double beta;
    uint64_t seed;
    uint32_t sweep; /* sweeps done so far: the counter word of the next sweep */
} su2_state;

/* Device allocation hook (e.g. a framework's caching allocator).  alloc
 * returns device memory usable on `stream`, or NULL; free releases it. */
typedef void *(*su2_alloc_fn)(size_t bytes, int device, void *stream, void *ctx);
typedef void (*su2_free_fn)(void *ptr, size_t bytes, int device, void *stream, void *ctx);

/* Installs (or, with both NULL, removes) the process-wide allocation hook used
 * by lattices created afterwards.  Not thread-safe with concurrent su2_create. */
su2_status su2_set_allocator(su2_alloc_fn alloc, su2_free_fn free_fn, void *ctx);

/* Creates an Ns^3 x Nt lattice on the current CUDA device and initialises it
 * with a cold or hot start (Sec. 4).  ns, nt even and >= 2 (checkerboard with
 * periodic boundaries); beta finite and >= 0; 4 Ns^3 Nt < 2^31 links.
 * cuda_stream: a cudaStream_t or NULL.  *out receives the handle. */
su2_status su2_create(int ns, int nt, double beta, uint64_t seed, su2_start start, void *cuda_stream,
                      su2_lattice **out);

/* Frees the lattice's device memory (stream-ordered) and the handle.  NULL is a no-op. */
su2_status su2_destroy(su2_lattice *lat);

/* nsweeps >= 0 heat-bath sweeps (Sec. 2 update, Sec. 4 schedule: mu = 0..3,
 * even then odd).  Asynchronous unless stats != NULL, in which case the call
 * synchronises and fills *stats.  SU2_E_SAMPLER if any draw hit its cap. */
su2_status su2_heatbath_sweep(su2_lattice *lat, int nsweeps, su2_stats *stats);

/* One phase only: links U_mu(x) with parity(x) = parity, using the current
 * sweep counter (which is not advanced).  For tests and diagnostics. */
su2_status su2_heatbath_phase(su2_lattice *lat, int mu, int parity);

/* Generation loop: nsweeps sweeps; after every `measure_every`-th sweep
 * (0 = never) the plaquette and Polyakov loop are computed on the device and
 * kept; after every `reunit_every`-th sweep (0 = never) the links are
 * reunitarized.  plaq and poly (host, nullable) receive nsweeps/measure_every
 * values each.  Synchronises once at the end.  The plaquette of a measured
 * sweep is accumulated by the sweep itself (the odd phases of mu = 1, 2, 3
 * see every plaquette of the final links once, as (1/2) Tr U'S over the
 * staple terms S of the directions nu < mu); it equals su2_plaquette on the
 * same links up to binary32 rounding of the single plaquettes.  A sweep
 * reunitarized before its measurement uses the separate plaquette pass.
 * On a lattice created with a stream (not the legacy default stream) and
 * with timing off, each sweep is replayed from a CUDA graph captured on first
 * use (the sweep counter and the measurement slot are kept on the device;
 * the graph is captured again when the sampler, beta, seed, over-relaxation,
 * trial cap or the measurement buffer change); the chain is the same bit for
 * bit. */
su2_status su2_generate(su2_lattice *lat, int nsweeps, int measure_every, int reunit_every, double *plaq,
                        double *poly, su2_stats *stats);

/* a0 sampler of the plain heat bath.  SU2_SAMPLER_CREUTZ (default): Creutz's
 * rejection method (the method the paper cites).  SU2_SAMPLER_KP: the
 * Kennedy-Pendleton method (Phys. Lett. B 156 (1985) 393) for links with
 * beta k >= 2 -- same law, about one trial per link at large beta k, drawn
 * from its own Philox stream -- and Creutz's method below beta k = 2.  The
 * choice applies to the following sweeps (and to the learned fallback). */
#define SU2_SAMPLER_CREUTZ 0
#define SU2_SAMPLER_KP 1
su2_status su2_set_sampler(su2_lattice *lat, int sampler);

/* Over-relaxation (not in the paper; the usual companion of its heat bath:
 * Adler, Phys. Rev. D 23 (1981) 2901; Creutz, Phys. Rev. D 36 (1987) 515).
 * Each link U_mu(x) of a phase is replaced by its reflection in the staple,
 *   U' = U~^dag U^dag U~^dag,  U~ = V/k  (U~ = 1 if k = 0),
 * which keeps (1/2) Tr UV, so the action, and is its own inverse; no random
 * numbers.  Same phase order as the heat bath (mu = 0..3, even then odd).
 * Products (U~^dag U^dag) U~^dag in binary32 with the heat bath's rounding
 * contract.  Not ergodic alone: it is interleaved with heat-bath sweeps.
 *
 * su2_overrelax_sweep: nsweeps over-relaxation sweeps now (asynchronous; the
 *   heat-bath sweep counter is not advanced).
 * su2_overrelax_phase: one phase (tests, diagnostics).
 * su2_set_overrelax: every later heat-bath sweep of su2_heatbath_sweep and
 *   su2_generate is followed by n_or over-relaxation sweeps (0 = none, the
 *   default); su2_stats counts and times them separately.
 * All three return SU2_E_INVAL for a NULL handle, mu or parity out of range,
 * nsweeps < 0 or n_or outside 0 ... 64. */
su2_status su2_overrelax_sweep(su2_lattice *lat, int nsweeps);
su2_status su2_overrelax_phase(su2_lattice *lat, int mu, int parity);
su2_status su2_set_overrelax(su2_lattice *lat, int n_or);

/* a <- a / |a| for every link (the links drift from |a| = 1 by rounding). */
su2_status su2_reunitarize(su2_lattice *lat);

/* Mean plaquette (Sec. 4): (1/6V) sum_x sum_{mu<nu} (1/2) Tr U_mu(x) U_nu(x+mu)
 * U_mu(x+nu)^dag U_nu(x)^dag; per-site values in binary32, global sum in
 * binary64.  Synchronous. */
su2_status su2_plaquette(su2_lattice *lat, double *out);

/* Polyakov loop (Sec. 4): (1/Ns^3) sum over spatial sites of
 * (1/2) Tr prod_{t=0}^{Nt-1} U_3(x, t), signed; binary32 products (each
 * quarter of the time extent multiplied left to right, the quarters combined
 * in order as (P0 P1)(P2 P3)), binary64 sum.  Synchronous. */
su2_status su2_polyakov(su2_lattice *lat, double *out);

/* Space-time Wilson loops (not in the paper; the observables after the
 * plaquette and the Polyakov loop, from which the static potential follows).
 * For site x, spatial direction i = 0..2 and extents R, T:
 *   S_R(y) = U_i(y) U_i(y+i) ... U_i(y+(R-1)i),  T_T(y) = U_t(y) ... U_t(y+(T-1)t),
 *   W = (1/2) Tr [S_R(x) T_T(x+Ri)] [T_T(x) S_R(x+Tt)]^dag,
 * line products left to right in binary32, the mean over x and i in binary64.
 * out (host, rmax * tmax doubles) receives W at out[(R-1) tmax + (T-1)] for
 * R = 1..rmax, T = 1..tmax.  Requires 1 <= rmax <= min(16, Ns) and
 * 1 <= tmax <= min(64, Nt) (else SU2_E_INVAL).  Synchronous; allocates and
 * frees a small device buffer. */
su2_status su2_wilson_loops(su2_lattice *lat, int rmax, int tmax, double *out);

/* Copies all links to / from a host buffer of 16 V floats laid out
 * [lex site][mu][a0..a3].  Synchronous.  set_links does not reunitarize. */
su2_status su2_get_links(su2_lattice *lat, float *host);
su2_status su2_set_links(su2_lattice *lat, const float *host);

/* Asynchronous forms, for pipelines that keep several configurations in
 * flight (one lattice handle, with its own stream, per configuration): each
 * call only enqueues its work on the lattice's stream and returns.
 * - su2_set_links_async / su2_get_links_async: the host buffer as in
 *   su2_set_links / su2_get_links.  The links pass through the lattice's
 *   device staging buffer (16 V floats, allocated on first use) and the copy
 *   engines, so one lattice's transfers run beside another lattice's sweeps.
 *   The host buffer must stay valid (and, for set, unchanged) until su2_sync.
 *   Page-locked host memory makes the copies asynchronous; pageable memory
 *   works but the driver stages it synchronously.
 * - su2_generate_async: su2_generate without the statistics.  plaq / poly
 *   (host, nullable, nsweeps/measure_every values each, page-locked for an
 *   asynchronous copy) hold their values after su2_sync.
 * - su2_sync: waits for the lattice's stream.  Returns SU2_E_SAMPLER (and
 *   clears the flag) if a heat-bath draw hit its trial cap since the last
 *   synchronous statistics read, SU2_E_CUDA on a device error. */
su2_status su2_set_links_async(su2_lattice *lat, const float *host);
su2_status su2_get_links_async(su2_lattice *lat, float *host);
su2_status su2_generate_async(su2_lattice *lat, int nsweeps, int measure_every, int reunit_every, double *plaq,
                              double *poly);
su2_status su2_sync(su2_lattice *lat);

/* Link health (failure detection): counts the links with a non-finite
 * component (*nonfinite) and those with | |a| - 1 | > tol (*off_norm; both
 * pointers nullable).  Synchronous.  Returns SU2_E_NUMERIC if any link is
 * non-finite, SU2_E_INVAL for tol < 0 or NaN.  Heat-bath links stay within
 * about 3e-7 of unit norm; su2_reunitarize restores it. */
su2_status su2_check_links(su2_lattice *lat, double tol, uint64_t *nonfinite, uint64_t *off_norm);

/* Diagnostic cap on the a0 sampler's trials per link (Creutz and
 * Kennedy-Pendleton heat-bath sweeps of this lattice; even, 2..4096, default
 * 4096, where the chance of reaching it is below 0.8^4096).  A link that
 * reaches it keeps its old value, and the call that reads the statistics
 * (su2_generate, su2_heatbath_sweep with stats, su2_sync) returns
 * SU2_E_SAMPLER with stats->sampler_failures set.  Creutz draws of the
 * Kennedy-Pendleton sweep below beta k = 2 keep the default cap. */
su2_status su2_set_trial_cap(su2_lattice *lat, int max_trials);

/* Resumable state (sweep counter, seed, beta).  set_state requires matching extents. */
su2_status su2_get_state(const su2_lattice *lat, su2_state *out);
su2_status su2_set_state(su2_lattice *lat, const su2_state *in);
su2_status su2_set_beta(su2_lattice *lat, double beta);

/* Device view of the links: even/odd structure of arrays of float4,
 * element (mu, parity, i) at index (2 mu + parity) (V/2) + i, where i = lex/2
 * of a site of that parity.  The pointer stays owned by the lattice. */
su2_status su2_device_links(su2_lattice *lat, void **ptr, size_t *bytes);

/* When enabled, the sweep calls record CUDA events around each heat-bath
 * phase kernel on the lattice's stream and report the summed device time in
 * su2_stats.kernel_ms. */
su2_status su2_set_timing(su2_lattice *lat, int enable);

/* Self-tests of device building blocks (they launch kernels):
 * su2_selftest_philox: n rows of host input ck[6 n] = (key0, key1, c0, c1, c2,
 *   c3) -> out[4 n] Philox4x32-10 words.
 * su2_selftest_math: which = 0 log, 1 exp, 2 sin/cos of 2 pi x, 3 the
 *   hardware base-2 logarithm that screens Creutz trials; n inputs x[n] ->
 *   y[n] (and y2[n] = cos for which = 2).  which = 4: x holds n quadruples
 *   (r1, r2, 1/(beta k), exp(-2 beta k)); y[i] = the screen's verdict (0
 *   reject, 1 accept, 2 undecided), y2[i] = the exact test's (0 or 1).
 *   which = 5: x holds n octuples (beta k, a', a, f'(z'), f'(z), u1, unused,
 *   unused) of the learned step's Metropolis test; y[i] = the screened
 *   verdict, y2[i] = the exact one.  which = 6: x holds n pairs (beta k,
 *   w) with w a 32-bit Philox word stored in the float's bits; y[i] = the
 *   Creutz trial variable x = e + r1 (1 - e), r1 the log uniform of w,
 *   y2[i] = that trial's candidate a0 (Sec. 2), with e = exp(-2 beta k) as
 *   the heat-bath kernels set it up.  y2 may be NULL unless which is 2, 4, 5
 *   or 6. */
su2_status su2_selftest_philox(const uint32_t *ck, uint32_t *out, size_t n);
su2_status su2_selftest_math(int which, const float *x, float *y, float *y2, size_t n);

/* ---------------------------------------------------------------------------
 * Learned proposal (not in the paper).  A small network of beta k (MLP
 * 1 -> 32 -> 32 -> 25, ReLU) sets an 8-bin monotone rational-quadratic spline
 * (Durkan et al., NeurIPS 2019) that proposes a0 for the heat-bath law of
 * Sec. 2; an independence-Metropolis step accepts or rejects the proposed link
 * against that law, so the chain stays exact for any weights.  Weights as
 * float[1947]: W1[32], b1[32], W2[32][32], b2[32], W3[25][32], b3[25], input
 * mean, input scale (network input (beta k - mean) * scale).
 * ------------------------------------------------------------------------- */
typedef struct {
    uint64_t link_updates;     /* 4 V per sweep, learned or plain            */
    uint64_t accepted[8];      /* accepted learned proposals per phase 2 mu + parity */
    uint64_t plain_trials[8];  /* Creutz trials of the fallback sweeps       */
    uint32_t learned_sweeps;   /* sweeps done with the learned proposal      */
    uint32_t plain_sweeps;     /* fallback sweeps done with the heat bath    */
    uint32_t kernel_launches;  /* learned phase launches (8 per sweep)       */
    uint32_t timed;            /* 1 if kernel_ms is valid (su2_set_timing)   */
    double kernel_ms;          /* summed device time of the learned phase kernels */
} su2_learned_stats;

/* Installs the proposal: the network is evaluated (binary32, on the device)
 * at grid_points (2..400) equally spaced inputs s in [s_lo, s_hi]; a link's
 * spline parameters are interpolated linearly between the two grid points
 * around its clamped input.  Synchronous.
 * The proposal is defined by the network at each link's own s = (beta k -
 * mean) * scale; the kernel reads it from this table instead (one network
 * evaluation per grid point rather than about 1,900 multiply-adds per link),
 * which is why the call takes the grid: [s_lo, s_hi] should cover the s of
 * the lattice's links (inputs outside are clamped to the end rows), and 256
 * points keep the table's density within a few 1e-3 in total variation of
 * the network's.  The chain is exact for any table: proposal and acceptance
 * use the same interpolated density. */
su2_status su2_set_proposal(su2_lattice *lat, const float *weights, int n, double s_lo, double s_hi, int grid_points);

/* The grid_points x 27 spline parameters (knots x0..x8, y0..y8, derivatives
 * d0..d8) of the installed proposal. */
su2_status su2_get_proposal_table(su2_lattice *lat, float *host);

/* nsweeps sweeps with the learned Metropolis step; a sweep whose acceptance
 * is below min_acceptance (e.g. 0.7) is followed by one plain heat-bath sweep,
 * after which the learned step resumes.  Measurements as su2_generate.
 * Synchronises once at the end. */
su2_status su2_learned_generate(su2_lattice *lat, int nsweeps, int measure_every, double min_acceptance,
                                double *plaq, double *poly, su2_learned_stats *stats);

/* nsweeps learned sweeps without measurements and with the fallback at
 * acceptance 0.7: su2_learned_generate(lat, nsweeps, 0, 0.7, NULL, NULL,
 * stats).  stats may be NULL.  Synchronous. */
su2_status su2_learned_sweep(su2_lattice *lat, int nsweeps, su2_learned_stats *stats);

/* Training pairs (beta k, a0), float2 each, for the links U_mu(x) of the given
 * parity whose even/odd index is a multiple of stride (mu, parity and stride
 * choose the sample of links; one call per phase covers a sweep's links
 * with stride 1): a0 is a fresh Creutz
 * draw (own counter stream) given the current staple, so the pairs have the
 * exact heat-bath law and the lattice is not changed.  dev_pairs: device
 * buffer of cap pairs; *n receives ceil((V/2) / stride).  Asynchronous. */
su2_status su2_collect_pairs(su2_lattice *lat, int mu, int parity, int stride, float *dev_pairs, size_t cap,
                             size_t *n);

/* Training of the proposal by maximum likelihood on (beta k, a0) pairs: mean
 * -log q(a0 | beta k) over mini-batches, minimised with Adam (beta1 0.9,
 * beta2 0.999, eps 1e-8).  Per step, 128 samples per CTA: the two hidden
 * contractions of the forward pass and the two of the backward pass run on
 * the tensor cores (tcgen05, BF16 operands, FP32 accumulation in tensor
 * memory); the spline likelihood, its gradient and the weight-gradient sums
 * are FP32 on the CUDA cores.  The trainer owns its device memory; all calls
 * are ordered on its stream. */
typedef struct su2_trainer su2_trainer;

/* init_weights: float[1947] (host); seed keys the mini-batch sampling. */
su2_status su2_trainer_create(const float *init_weights, uint64_t seed, void *cuda_stream, su2_trainer **out);
su2_status su2_trainer_destroy(su2_trainer *tr);

/* Sets the input mean and scale (weights 1945, 1946) to the mean and
 * 1/standard deviation of beta k over n device pairs (float2). */
su2_status su2_trainer_set_input_scaling(su2_trainer *tr, const float *dev_pairs, size_t n);

/* `steps` Adam steps of `batch` (multiple of 128, <= 65536) pairs drawn with
 * replacement from the n device pairs; loss_per_step (host, nullable)
 * receives each step's mean loss.  Synchronises at the end. */
su2_status su2_trainer_fit(su2_trainer *tr, const float *dev_pairs, size_t n, int steps, int batch, double lr,
                           float *loss_per_step);

/* Mean loss and gradient (1945 floats, host) over exactly the n device pairs
 * (n a multiple of 128, <= 65536), without updating the weights. */
su2_status su2_trainer_gradient(su2_trainer *tr, const float *dev_pairs, size_t n, double *loss, float *grad);

/* Current weights (float[1947], host). */
su2_status su2_trainer_get_weights(su2_trainer *tr, float *host);

/* ---------------------------------------------------------------------------
 * Batches: many independent lattices (own Ns^3 x Nt, beta and seed each) swept
 * together.  Each lattice follows exactly the chain of su2_create +
 * su2_heatbath_sweep with its own arguments.  One sweep of the whole batch is
 * one persistent cooperative kernel launch: the eight even/odd phases of every
 * lattice with a grid-wide barrier between phases (each barrier wait bounded,
 * 2 s), then optionally the plaquette and Polyakov loop of every lattice.  On
 * a non-NULL stream the launch is captured into a CUDA graph once and replayed
 * per sweep.  The batch owns its device memory like a lattice.
 * ------------------------------------------------------------------------- */
typedef struct su2_batch su2_batch;

/* n >= 1 lattices; ns[i], nt[i] even >= 2 with 4 V_i < 2^31; beta[i] finite
 * >= 0; seed[i] any.  Cold or hot start for all.  Fails with SU2_E_CUDA on a
 * device without cooperative launches. */
su2_status su2_batch_create(int n, const int *ns, const int *nt, const double *beta, const uint64_t *seed,
                            su2_start start, void *cuda_stream, su2_batch **out);
su2_status su2_batch_destroy(su2_batch *b);

/* nsweeps sweeps of every lattice; synchronises; stats (nullable) sum the
 * trials over lattices.  SU2_E_DEVICE_TIMEOUT if a barrier wait gave up. */
su2_status su2_batch_sweep(su2_batch *b, int nsweeps, su2_stats *stats);

/* Sweeps with the plaquette and Polyakov loop of every lattice after every
 * measure_every-th sweep: plaq and poly (host, nullable) receive
 * (nsweeps / measure_every) x n values, row m = measurement m, column = lattice. */
su2_status su2_batch_generate(su2_batch *b, int nsweeps, int measure_every, double *plaq, double *poly,
                              su2_stats *stats);

/* Current plaquette / Polyakov loop of every lattice (out: n doubles). */
su2_status su2_batch_plaquette(su2_batch *b, double *out_n);
su2_status su2_batch_polyakov(su2_batch *b, double *out_n);

/* Links of lattice i in the layout of su2_get_links. */
su2_status su2_batch_get_links(su2_batch *b, int i, float *host);

/* Launch configuration: queue depth (1, 2, 4 or 8: the work is split into
 * chunks of 32 x depth sites, and each warp takes a contiguous range of chunks),
 * block size (64, 128 or 256 threads; the register budget is that of 768
 * threads per SM for every size) and grid (<= 0 or too large = all
 * co-resident blocks).  The default is depth 4, 128 threads, all co-resident
 * blocks.  su2_batch_set_config keeps the block size.  su2_batch_autotune
 * times all 60 combinations of depth, block size and grid (all co-resident
 * blocks, or 1/2, 1/4, 1/8, 1/16 of them) over `sweeps` sweeps each,
 * restores the links and sweep counter, and keeps the fastest (reported by
 * su2_batch_launch_info). */
su2_status su2_batch_set_launch(su2_batch *b, int queue_depth, int threads, int grid);
/* a0 sampler of every lattice of the batch: SU2_SAMPLER_CREUTZ (default) or
 * SU2_SAMPLER_KP, as su2_set_sampler for one lattice (each lattice's chain is
 * then that of su2_heatbath_sweep with the same sampler).  Keeps the launch
 * shape, clamped to the co-resident blocks of that sampler's kernel. */
su2_status su2_batch_set_sampler(su2_batch *b, int sampler);
su2_status su2_batch_set_config(su2_batch *b, int queue_depth, int grid);
su2_status su2_batch_launch_info(su2_batch *b, int *queue_depth, int *threads, int *grid);
su2_status su2_batch_autotune(su2_batch *b, int sweeps, int *queue_depth, int *grid);
su2_status su2_batch_info(su2_batch *b, int *n, uint32_t *sweep, int *queue_depth, int *grid, int *graphs);

/* Self-test of the bounded grid-barrier wait: `blocks` blocks wait for one
 * arrival more than there are blocks, so every wait must give up after
 * timeout_ns (<= 5 s); *timed_out receives the number of blocks that did. */
su2_status su2_selftest_barrier_timeout(int blocks, uint64_t timeout_ns, unsigned int *timed_out);

/* Self-test of the bounded mbarrier wait that the learned phase uses for its
 * proposal-table copy: in each of `blocks` blocks (1..1024) thread 0 sets up
 * an mbarrier that expects one arrival which never comes, and waits `polls`
 * polls (1..2^24); *timed_out receives the number of blocks whose wait gave
 * up (all of them). */
su2_status su2_selftest_mbar_timeout(int blocks, unsigned int polls, unsigned int *timed_out);

/* ------------------------------------------------------------------------
 * Time slabs: one lattice decomposed over ranks (Sec. 4, multi-GPU part, and
 * Fig. 1).  A slab holds the time slices t0 .. t0 + nt_local - 1 of the
 * Ns^3 x Nt lattice plus one ghost slice on each side (Ns^3 x (nt_local + 2)
 * sites; local slice tl is global slice (t0 - 1 + tl) mod Nt).  A phase
 * updates the slab's interior with the random numbers of the global sites, so
 * slabs that exchange their boundaries after every phase reproduce the single
 * lattice's chain bit for bit.  The paper exchanged the border cells through
 * host memory between the GPUs' threads; here the caller moves them (pack /
 * unpack through any buffer and transport) or, for slabs of one process,
 * su2_slab_exchange copies them directly.
 * ------------------------------------------------------------------------- */
typedef struct su2_slab su2_slab;

/* Ns, Nt, nt_local and t0 even, nt_local >= 2, t0 + nt_local <= Nt; the start
 * is that of the whole lattice (hot: the global sites' Haar links, ghosts
 * included).  Stream as su2_create.  SU2_E_INVAL on bad extents. */
su2_status su2_slab_create(int ns, int nt, int t0, int nt_local, double beta, uint64_t seed, su2_start start,
                           void *cuda_stream, su2_slab **out);
su2_status su2_slab_destroy(su2_slab *s);
/* SU2_SAMPLER_CREUTZ or SU2_SAMPLER_KP. */
su2_status su2_slab_set_sampler(su2_slab *s, int sampler);
/* Phase (mu, parity) of the slab's interior, parity of the global site; the
 * sweep counter advances after (3, 1).  Asynchronous.  Before the next phase
 * the boundaries of this one must be exchanged. */
su2_status su2_slab_phase(su2_slab *s, int mu, int parity);
/* Bytes of one boundary message: the Ns^3 / 2 links U_mu of one parity in one
 * time slice, float4 each (8 Ns^3). */
size_t su2_slab_boundary_bytes(const su2_slab *s);
/* After phase (mu, parity): pack side 0 (first interior slice) or 1 (last)
 * into dst; unpack src into side 0 (lower ghost) or 1 (upper ghost).  dst /
 * src: host (pinned or pageable) or device memory of su2_slab_boundary_bytes.
 * Asynchronous on the slab's stream (su2_slab_sync before reusing a host
 * buffer).  The first interior slice goes to the lower neighbour's upper
 * ghost, the last to the upper neighbour's lower ghost. */
su2_status su2_slab_pack(su2_slab *s, int mu, int parity, int side, void *dst);
su2_status su2_slab_unpack(su2_slab *s, int mu, int parity, int side, const void *src);
/* Both boundary copies of phase (mu, parity) between neighbouring slabs of
 * one process (lower's last slice -> upper's lower ghost, upper's first ->
 * lower's upper ghost), ordered after both slabs' work and before their next
 * phases (events when their streams differ).  lower == upper: a slab that
 * holds the whole lattice, its own neighbour. */
su2_status su2_slab_exchange(su2_slab *lower, su2_slab *upper, int mu, int parity);
su2_status su2_slab_sync(su2_slab *s);
/* Links of the whole local array, ghosts included, lexicographic in local
 * sites ([site][mu][a0..a3], 4 Ns^3 (nt_local + 2) float4).  Synchronous. */
su2_status su2_slab_get_links(su2_slab *s, float *host);
su2_status su2_slab_set_links(su2_slab *s, const float *host);
/* Trial counts per phase (2 mu + parity, parity of the global site) since the
 * last call (then cleared), and links that hit the trial cap (SU2_E_SAMPLER if
 * any).  Synchronous. */
su2_status su2_slab_stats(su2_slab *s, uint64_t trials[8], uint64_t *sampler_failures);
su2_status su2_slab_info(const su2_slab *s, int *t0, int *nt_local, uint32_t *sweep);

/* Mean plaquette of links that already sit in device memory, computed without
 * allocating anything (no cudaMalloc, cudaFree or allocating library call).
 * The paper has no counterpart: this is for callers that cannot allocate
 * device memory where they need the observable, e.g. a process whose
 * framework has claimed all device memory for its own pool, or code running
 * where an allocation would stall or is forbidden.
 *   links  device pointer to 8 (V/2) float4 in the even/odd layout described at
 *          su2_device_links (V = ns^3 nt), read only;
 *   out    device pointer to one double, written in stream order (same value as
 *          su2_plaquette up to the order of the fp64 sum);
 *   cuda_stream  cudaStream_t or NULL.  The call does not synchronise.
 * Limits: ns, nt even and >= 2; V <= 67,108,864 sites, else SU2_E_INVAL with
 * the limit in su2_last_error().  Scratch: a fixed 131,328-byte device array
 * inside libsu2 (held on every GPU that loads the library until exit).  The
 * first call on each device looks up that array's address
 * (cudaGetSymbolAddress), so make it before capturing a stream into a CUDA
 * graph.  All calls share the array and it keeps the last call's contents:
 * calls whose kernels may overlap on the GPU (unordered streams) race and
 * give wrong results -- order them.  The array's device address is looked up
 * once per device and kept for the life of the process; cudaDeviceReset
 * unloads the module and may move the array, so after a device reset this
 * entry point must not be called again in the same process. */
su2_status su2_plaquette_noalloc(const void *links, int ns, int nt, double *out, void *cuda_stream);

/* Self-test of the tensor-core path used by training: D (128 x 32, FP32,
 * row-major) = A (128 x K, BF16 bits, row-major) * B (32 x K, BF16 bits)^T,
 * K = 16 or 32, computed by tcgen05.mma with the accumulator in tensor memory. */
su2_status su2_selftest_mma(const uint16_t *A, const uint16_t *B, int K, float *D);

/* Human-readable status and the last CUDA error text of this thread. */
const char *su2_status_str(su2_status s);
const char *su2_last_error(void);
int su2_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SU2_H */
