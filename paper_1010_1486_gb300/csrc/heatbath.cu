// heatbath.cu -- the checkerboard heat-bath phase kernel and the sweep
// schedule (Sec. 2 update, Sec. 4 schedule of Cardoso & Bicudo, LAT2010).
//
// One phase (mu, parity) redraws every link U_mu(x) with parity(x) = parity.
// Its staple reads only links of the other three directions (both parities)
// and U_mu of the opposite parity, none of which the phase writes, so every
// thread works independently and the loads may use the read-only path.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "creutz_queue.cuh"
#include "observables.cuh"
#include "staple.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

// Staple of U_mu(x) (Sec. 2):
//   V = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//                    + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
// nu ascending, forward term first, accumulated from zero.
struct HbParams {
    float4 *links;
    Geom g;
    RoundKeys rk;
    int parity;
    float beta;
    uint32_t sweep;
    const uint32_t *sweep_dev;  // if non-NULL the sweep counter is read here (graph replays)
    int max_blocks;             // trial cap / 2: Philox blocks a link may use before it keeps its old value
    unsigned long long *trial_slots;
    unsigned int *flags;
    const unsigned int *gate;  // if non-NULL and *gate == 1 the phase is left to the learned kernel
    double *plaq;              // measuring phases: block partials of the plaquettes of planes (nu < mu, mu)
    SlabRange slab;            // SLAB kernels: the interior eo range and the global keys of its random numbers
    const float4 *same[4];     // links of direction d at the phase's parity
    const float4 *other[4];    // ... at the opposite parity
};

constexpr int kCrThreads = 256;
constexpr int kCrWarps = kCrThreads / 32;
#ifndef SU2_HB_MIN_BLOCKS
#define SU2_HB_MIN_BLOCKS 3
#endif
constexpr int kCrMinBlocks = SU2_HB_MIN_BLOCKS;  // blocks per SM the register budget is set for

// One heat-bath phase (mu = MU, sites of parity p.parity), Creutz's sampler.
//
// Warp w of the persistent grid takes the rounds of 32 consecutive links w,
// w + W, ... (W warps).  Each loop iteration (three per round) issues the six
// loads of one nu-group of the next round, does one third of the current
// round's work, then folds the loaded group into the next round's staple:
//   part 0  k, U~^dag, beta k, exp(-2 beta k); Philox block 0 (trials 0, 1);
//   part 1  trials 0 and 1, screened (creutz_pair); an accepted link goes to
//           the warp's direction queue, a link with both rejected to its
//           retry queue;
//   part 2  every 32 links in the direction queue: a0 (the one exact log of
//           the link), directions and stores.
// Whenever 32 links wait for a retry, the whole warp draws their next Philox
// block (two more trials each); accepted links move to the direction queue,
// the others go back to the retry queue.  At beta k ~ 30 two trials accept
// 41% of links, so the lanes stay busy instead of waiting for the slowest
// lane of a round.  Every draw depends only on the link's counters (trial t
// in words 2(t&1), 2(t&1)+1 of block t>>1; direction block 0), so the phase
// computes exactly the one-thread-per-link definition.  Lanes past the end
// work on a clamped index and drop their results.
//
// MEAS (odd phases of mu = 1, 2, 3 in a sweep that ends with a measurement):
// with S the staple terms of the directions nu < MU, (1/2) Tr U'S is the sum
// of the plaquettes of planes (nu, MU) at x and x - nu, so over the odd sites
// every such plaquette of the final configuration is counted once; the block
// partial goes to p.plaq[block].
template <int MU, bool MEAS, bool SLAB>
__global__ void __launch_bounds__(kCrThreads, kCrMinBlocks) hb_phase_kernel(const HbParams p)
{
    // a time slab updates its interior eo range; its random numbers are those
    // of the global site (even/odd index + rng_eo, global parity)
    const int eo_begin = SLAB ? p.slab.eo_begin : 0;
    const int eo_end = SLAB ? p.slab.eo_end : p.g.vh;
    const uint32_t rng_eo = SLAB ? p.slab.rng_eo : 0u;
    const uint32_t rng_parity = SLAB ? (uint32_t)p.slab.rng_parity : (uint32_t)p.parity;
    if (p.gate != nullptr && *(volatile const unsigned int *)p.gate == 1u) return;
    __shared__ CrQueues s_q[kCrWarps];
    const uint32_t sweep = p.sweep_dev ? *p.sweep_dev : p.sweep;
    const int lane = threadIdx.x & 31;
    CrQueues &Q = s_q[threadIdx.x >> 5];
    const unsigned int lanes_below = (1u << lane) - 1u;
    const int stride = gridDim.x * kCrThreads;
    const int last = eo_end - 1;
    const uint32_t sw_creutz = stream_word(kCreutz, rng_parity, MU);
    const uint32_t sw_dir = stream_word(kDirection, rng_parity, MU);
    unsigned int trials = 0;
    float plaq = 0.0f;  // per-thread partial in binary32; the block and grid sums are binary64
    int retry_n = 0, done_n = 0;  // warp-uniform queue lengths

    // Lanes that push nothing write to the last slot, which no live entry
    // reaches (at most 31 left over + 32 pushed = 63), so the stores need no
    // branch.
    auto push_done = [&](bool ok, float4 ut, float val, float ibk, int eo, float4 sp) {
        const unsigned int m = __ballot_sync(0xffffffffu, ok);
        const int q = ok ? done_n + __popc(m & lanes_below) : kCrQueue - 1;
        Q.d_ut[q] = ut;
        Q.d_val[q] = val;
        Q.d_ibk[q] = ibk;
        Q.d_eo[q] = eo;
        if (MEAS) Q.d_sp[q] = sp;
        done_n += __popc(m);
    };
    auto push_retry = [&](bool again, float4 ut, float ibk, float e, int eo, int blk, float4 sp) {
        const unsigned int m = __ballot_sync(0xffffffffu, again);
        const int q = again ? retry_n + __popc(m & lanes_below) : kCrQueue - 1;
        Q.r_ut[q] = ut;
        Q.r_ibk[q] = ibk;
        Q.r_e[q] = e;
        Q.r_eo[q] = eo;
        Q.r_blk[q] = blk;
        if (MEAS) Q.r_sp[q] = sp;
        retry_n += __popc(m);
    };
    // directions and stores of direction-queue entries [first, first + n)
    auto direction_pass = [&](int first, int n) {
        __syncwarp();
        if (lane < n) {
            const int q = first + lane;
            const int eo = Q.d_eo[q];
            const uint32_t eo_g = (uint32_t)eo + rng_eo;
            const uint4 wd = philox_rk(make_uint4(direction_pair(eo_g), sweep, sw_dir, 0u), p.rk);
            const float4 out = direction_update(deferred_a0(Q.d_val[q], Q.d_ibk[q]), Q.d_ut[q], wd, eo_g);
            p.links[link_index(p.g, MU, p.parity, eo)] = out;
            if (MEAS) plaq = __fadd_rn(plaq, qmul_re(out, Q.d_sp[q]));
        }
        __syncwarp();
    };
    auto flush_done = [&]() {
        while (done_n >= 32) {
            done_n -= 32;
            direction_pass(done_n, 32);
        }
    };
    // next Philox block of retry-queue entries [first, first + n)
    auto retry_pass = [&](int first, int n) {
        __syncwarp();
        const bool have = lane < n;
        float4 ut = make_float4(1.0f, 0.0f, 0.0f, 0.0f), sp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float ibk = 1.0f, e = 0.0f;
        int eo = 0, blk = 0;
        if (have) {
            const int q = first + lane;
            ut = Q.r_ut[q];
            ibk = Q.r_ibk[q];
            e = Q.r_e[q];
            eo = Q.r_eo[q];
            blk = Q.r_blk[q];
            if (MEAS) sp = Q.r_sp[q];
        }
        __syncwarp();
        const uint4 w = philox_rk(make_uint4((uint32_t)eo + rng_eo, sweep, sw_creutz, (uint32_t)blk), p.rk);
        bool first_ok;
        float val;
        const bool over = blk >= p.max_blocks;  // only with a cap of two trials
        const bool ok = creutz_pair(w, ibk, e, have, first_ok, val) && have && !over;
        bool again = false;
        if (ok) {
            trials += (unsigned int)(2 * blk + (first_ok ? 1 : 2));
        } else if (have) {
            if (!over && blk + 1 < p.max_blocks) {
                again = true;
            } else {
                atomicAdd(&p.flags[0], 1u);  // trial cap: the link keeps its old value
                trials += (unsigned int)(2 * p.max_blocks);
            }
        }
        push_retry(again, ut, ibk, e, eo, blk + 1, sp);
        push_done(ok, ut, val, ibk, eo, sp);
        flush_done();
    };

    int base = eo_begin + blockIdx.x * kCrThreads + (threadIdx.x & ~31);
    int cur = base + lane;
    float4 v_cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float4 sp_cur = v_cur;  // MEAS: staple terms of nu < MU (the first MU groups)
    if (base < eo_end) {
        const int e = min(cur, last);
        const Coord x = eo_to_coord(p.g, e, p.parity);
        const int e_p = eo_fwd<MU>(p.g, x, e);
        v_cur = add_nu_terms(v_cur, load_nu_bases<MU, OtherDir<MU, 0>::value>(p.same, p.other, p.g, x, e, e_p));
        if (MU == 1) sp_cur = v_cur;
        v_cur = add_nu_terms(v_cur, load_nu_bases<MU, OtherDir<MU, 1>::value>(p.same, p.other, p.g, x, e, e_p));
        if (MU == 2) sp_cur = v_cur;
        v_cur = add_nu_terms(v_cur, load_nu_bases<MU, OtherDir<MU, 2>::value>(p.same, p.other, p.g, x, e, e_p));
        if (MU == 3) sp_cur = v_cur;
    }
    while (base < eo_end) {  // warp-uniform
        const bool valid = cur <= last;
        const int nxt = cur + stride;
        const int en = min(nxt, last);
        const Coord xn = eo_to_coord(p.g, en, p.parity);
        const int en_p = eo_fwd<MU>(p.g, xn, en);
        // ---- part 0
        NuLinks nl = load_nu_bases<MU, OtherDir<MU, 0>::value>(p.same, p.other, p.g, xn, en, en_p);
        const DrawSetup d = prepare_draw(v_cur, p.beta);
        const uint4 w = philox_rk(make_uint4((uint32_t)cur + rng_eo, sweep, sw_creutz, 0u), p.rk);
        float4 v_next = add_nu_terms(make_float4(0.0f, 0.0f, 0.0f, 0.0f), nl);
        float4 sp_next = v_next;
        // ---- part 1
        nl = load_nu_bases<MU, OtherDir<MU, 1>::value>(p.same, p.other, p.g, xn, en, en_p);
        {
            bool first_ok;
            float val;
            const bool acc = creutz_pair(w, d.ibk, d.e, valid, first_ok, val);
            const bool ok = valid && acc;
            trials += ok ? (first_ok ? 1u : 2u) : 0u;
            push_done(ok, d.ut, val, d.ibk, cur, sp_cur);
            push_retry(valid && !acc, d.ut, d.ibk, d.e, cur, 1, sp_cur);
        }
        v_next = add_nu_terms(v_next, nl);
        if (MU == 2) sp_next = v_next;
        // ---- part 2
        nl = load_nu_bases<MU, OtherDir<MU, 2>::value>(p.same, p.other, p.g, xn, en, en_p);
        flush_done();
        v_next = add_nu_terms(v_next, nl);
        if (MU == 3) sp_next = v_next;
        while (retry_n >= 32) {
            retry_n -= 32;
            retry_pass(retry_n, 32);
        }
        base += stride;
        cur = nxt;
        v_cur = v_next;
        sp_cur = sp_next;
    }
    while (retry_n > 0) {
        const int n = min(retry_n, 32);
        retry_n -= n;
        retry_pass(retry_n, n);
    }
    if (done_n > 0) direction_pass(0, done_n);
    const unsigned int wsum = __reduce_add_sync(0xffffffffu, trials);
    if (lane == 0 && wsum)
        atomicAdd(&p.trial_slots[(2 * MU + p.parity) * kTrialSlots +
                                 ((blockIdx.x * kCrWarps + (threadIdx.x >> 5)) & (kTrialSlots - 1))],
                  (unsigned long long)wsum);
    if (MEAS) {
        const double total = block_sum((double)plaq);
        if (threadIdx.x == 0) p.plaq[blockIdx.x] = total;
    }
}

template <int MU, bool MEAS, bool SLAB = false>
static cudaError_t launch_hb(const HbParams &p, int device, cudaStream_t stream)
{
    static int blocks_per_sm[64] = {};
    static int num_sms[64] = {};
    if (device < 0 || device >= 64) device = 0;
    if (!blocks_per_sm[device]) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[device],
                                                                      hb_phase_kernel<MU, MEAS, SLAB>, kCrThreads, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&num_sms[device], cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm[device] < 1) blocks_per_sm[device] = 1;
    }
    const int n = SLAB ? p.slab.eo_end - p.slab.eo_begin : p.g.vh;
    const int want = (n + kCrThreads - 1) / kCrThreads;
    const int grid = std::max(1, std::min(std::min(want, blocks_per_sm[device] * num_sms[device]), kFusedSlots));
    hb_phase_kernel<MU, MEAS, SLAB><<<grid, kCrThreads, 0, stream>>>(p);
    return cudaGetLastError();
}

su2_status launch_hb_phase(su2_lattice *lat, int mu, int parity, uint32_t sweep, const unsigned int *gate)
{
    if (lat->sampler == SU2_SAMPLER_KP) return launch_kp_phase(lat, mu, parity, sweep, gate);
    HbParams p;
    p.gate = gate;
    p.links = lat->links;
    p.g = geom_of(lat);
    p.rk = make_round_keys(lat->seed);
    p.parity = parity;
    p.beta = (float)lat->beta;
    p.sweep = sweep;
    p.sweep_dev = lat->capturing ? lat->d_ctr : nullptr;
    p.max_blocks = lat->max_trials / 2;
    p.trial_slots = lat->scratch.trials;
    p.flags = lat->scratch.flags;
    p.plaq = fused_slot(lat, mu, parity, 0);
    set_bases(p.same, p.other, lat, parity);
    cudaError_t e;
    if (p.plaq) {
        switch (mu) {
        case 1: e = launch_hb<1, true>(p, lat->device, lat->stream); break;
        case 2: e = launch_hb<2, true>(p, lat->device, lat->stream); break;
        default: e = launch_hb<3, true>(p, lat->device, lat->stream); break;
        }
    } else {
        switch (mu) {
        case 0: e = launch_hb<0, false>(p, lat->device, lat->stream); break;
        case 1: e = launch_hb<1, false>(p, lat->device, lat->stream); break;
        case 2: e = launch_hb<2, false>(p, lat->device, lat->stream); break;
        default: e = launch_hb<3, false>(p, lat->device, lat->stream); break;
        }
    }
    SU2_CUDA(e);
    return SU2_OK;
}

su2_status launch_hb_phase_slab(su2_lattice *lat, int mu, int parity_local, uint32_t sweep, const SlabRange &r)
{
    if (lat->sampler == SU2_SAMPLER_KP) return launch_kp_phase_slab(lat, mu, parity_local, sweep, r);
    HbParams p;
    p.gate = nullptr;
    p.links = lat->links;
    p.g = geom_of(lat);
    p.rk = make_round_keys(lat->seed);
    p.parity = parity_local;
    p.beta = (float)lat->beta;
    p.sweep = sweep;
    p.sweep_dev = nullptr;
    p.max_blocks = lat->max_trials / 2;
    p.trial_slots = lat->scratch.trials;
    p.flags = lat->scratch.flags;
    p.plaq = nullptr;
    p.slab = r;
    set_bases(p.same, p.other, lat, parity_local);
    cudaError_t e;
    switch (mu) {
    case 0: e = launch_hb<0, false, true>(p, lat->device, lat->stream); break;
    case 1: e = launch_hb<1, false, true>(p, lat->device, lat->stream); break;
    case 2: e = launch_hb<2, false, true>(p, lat->device, lat->stream); break;
    default: e = launch_hb<3, false, true>(p, lat->device, lat->stream); break;
    }
    SU2_CUDA(e);
    return SU2_OK;
}

// ------------------------------------------------------------- timing
su2_status timing_begin(su2_lattice *lat, EventLog &log)
{
    if (!lat->timing) return SU2_OK;
    while (log.events.size() < log.used + 2) {
        cudaEvent_t e;
        SU2_CUDA(cudaEventCreate(&e));
        log.events.push_back(e);
    }
    SU2_CUDA(cudaEventRecord(log.events[log.used], lat->stream));
    return SU2_OK;
}

su2_status timing_end(su2_lattice *lat, EventLog &log)
{
    if (!lat->timing) return SU2_OK;
    SU2_CUDA(cudaEventRecord(log.events[log.used + 1], lat->stream));
    log.used += 2;
    return SU2_OK;
}

su2_status timing_read(su2_lattice *lat, EventLog &log, double *ms_out)
{
    double ms = 0.0;
    if (lat->timing && log.used) {
        SU2_CUDA(cudaEventSynchronize(log.events[log.used - 1]));
        for (size_t i = 0; i + 1 < log.used; i += 2) {
            float t = 0.0f;
            SU2_CUDA(cudaEventElapsedTime(&t, log.events[i], log.events[i + 1]));
            ms += t;
        }
    }
    *ms_out = ms;
    log.used = 0;
    return SU2_OK;
}

static su2_status timed_phase(su2_lattice *lat, int mu, int parity, uint32_t sweep)
{
    su2_status st = timing_begin(lat, lat->hb_log);
    if (st == SU2_OK) st = launch_hb_phase(lat, mu, parity, sweep);
    if (st == SU2_OK) st = timing_end(lat, lat->hb_log);
    return st;
}

static su2_status read_timing(su2_lattice *lat, su2_stats *stats)
{
    double ms = 0.0, or_ms = 0.0;
    su2_status st = timing_read(lat, lat->hb_log, &ms);
    su2_status st2 = timing_read(lat, lat->or_log, &or_ms);
    if (stats) {
        stats->kernel_ms = ms;
        stats->overrelax_ms = or_ms;
        stats->timed = lat->timing ? 1u : 0u;
    }
    return st != SU2_OK ? st : st2;
}

// One heat-bath sweep, then the lattice's over-relaxation sweeps; when the
// sweep is measured (lat->fused_part set), the last of these sweeps adds the
// plaquette.
static su2_status one_sweep(su2_lattice *lat)
{
    double *const fused = lat->fused_part;
    if (lat->overrelax > 0) lat->fused_part = nullptr;
    for (int mu = 0; mu < 4; ++mu)
        for (int parity = 0; parity < 2; ++parity) {
            su2_status st = timed_phase(lat, mu, parity, lat->sweep);
            if (st != SU2_OK) {
                lat->fused_part = fused;
                return st;
            }
        }
    lat->sweep += 1;
    lat->fused_part = fused;
    return lat->overrelax > 0 ? overrelax_sweeps(lat, lat->overrelax) : SU2_OK;
}

static su2_status ensure_history(su2_lattice *lat, int n)
{
    if (n <= lat->scratch.history_cap) return SU2_OK;
    device_free(lat->scratch.history, sizeof(double) * 2 * (size_t)lat->scratch.history_cap, lat->device,
                lat->stream);
    lat->scratch.history = (double *)device_alloc(sizeof(double) * 2 * (size_t)n, lat->device, lat->stream);
    lat->scratch.history_cap = lat->scratch.history ? n : 0;
    if (!lat->scratch.history) {
        set_last_error("device allocation of the measurement history failed");
        return SU2_E_NOMEM;
    }
    return SU2_OK;
}

// One sweep of su2_generate: the heat bath (and the lattice's over-relaxation
// sweeps), the reunitarization if due, and the measurement if due.  The
// plaquette comes out of the sweep itself unless the links are reunitarized
// before the measurement.  plaq_dst / poly_dst: the measurement slots (when
// capturing, the bases: the kernels add the device slot index).
static su2_status sweep_and_measure(su2_lattice *lat, bool measure, bool reunit, double *plaq_dst, double *poly_dst)
{
    su2_status st;
    const bool fused = measure && !reunit;
    if (fused && (st = fused_begin(lat)) != SU2_OK) return st;
    if ((st = one_sweep(lat)) != SU2_OK) {
        lat->fused_part = nullptr;
        return st;
    }
    if (reunit && (st = launch_reunitarize(lat)) != SU2_OK) return st;
    if (measure) {
        if (fused) return fused_finish_with_polyakov(lat, plaq_dst, poly_dst);
        if ((st = launch_plaquette(lat, plaq_dst)) != SU2_OK) return st;
        if ((st = launch_polyakov(lat, poly_dst)) != SU2_OK) return st;
    }
    return SU2_OK;
}

// Sets the device sweep counter and measurement slot from kernel parameters
// (no host memory is read when it runs, so enqueueing it never waits).
__global__ void set_counters_kernel(uint32_t *ctr, uint32_t sweep)
{
    ctr[0] = sweep;
    ctr[1] = 0u;
}

// Advances the device counters of graph replays: the sweep, and the
// measurement slot after a measured sweep.
__global__ void advance_kernel(uint32_t *ctr, int measured)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        ctr[0] += 1u;
        if (measured) ctr[1] += 1u;
    }
}

su2_status enqueue_set_counters(su2_lattice *lat)
{
    set_counters_kernel<<<1, 1, 0, lat->stream>>>(lat->d_ctr, lat->sweep);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status enqueue_advance(su2_lattice *lat, bool measured)
{
    advance_kernel<<<1, 32, 0, lat->stream>>>(lat->d_ctr, measured ? 1 : 0);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

uint64_t generation_signature(const su2_lattice *lat)
{
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the settings a captured sweep depends on
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    const float beta = (float)lat->beta;
    uint32_t bb;
    memcpy(&bb, &beta, sizeof bb);
    mix(bb);
    mix(lat->seed);
    mix((uint64_t)lat->sampler);
    mix((uint64_t)lat->overrelax);
    mix((uint64_t)lat->max_trials);
    mix((uint64_t)(uintptr_t)lat->scratch.history);
    mix((uint64_t)lat->scratch.history_cap);
    return h | 1ull;  // never 0 (0 marks an empty slot)
}

// The captured sweep of this variant (captured on first use or after a
// settings change); *exec = NULL if the stream refused the capture.
static su2_status generation_graph(su2_lattice *lat, bool measure, bool reunit, cudaGraphExec_t *exec)
{
    GenGraph &gg = lat->gen_graph[(measure ? 1 : 0) | (reunit ? 2 : 0)];
    const uint64_t sig = generation_signature(lat);
    if (gg.exec && gg.sig == sig) {
        *exec = gg.exec;
        return SU2_OK;
    }
    if (gg.exec) {
        cudaGraphExecDestroy(gg.exec);
        gg.exec = nullptr;
    }
    *exec = nullptr;
    if (cudaStreamBeginCapture(lat->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        lat->graphs_off = true;
        return SU2_OK;
    }
    const uint32_t sweep0 = lat->sweep;
    lat->capturing = true;
    su2_status st = sweep_and_measure(lat, measure, reunit, lat->scratch.history,
                                      lat->scratch.history + lat->scratch.history_cap);
    if (st == SU2_OK) {
        advance_kernel<<<1, 32, 0, lat->stream>>>(lat->d_ctr, measure ? 1 : 0);
        if (cudaGetLastError() != cudaSuccess) st = SU2_E_CUDA;
    }
    lat->capturing = false;
    lat->sweep = sweep0;  // the captured sweep advanced the host counter; the replay does it
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(lat->stream, &graph);
    if (st != SU2_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        lat->graphs_off = true;  // run this lattice eagerly from now on
        return SU2_OK;
    }
    const cudaError_t ei = cudaGraphInstantiate(&gg.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        gg.exec = nullptr;
        cudaGetLastError();
        lat->graphs_off = true;
        return SU2_OK;
    }
    gg.sig = sig;
    *exec = gg.exec;
    return SU2_OK;
}

// Enqueues nsweeps sweeps with their measurements and reunitarizations, and
// the copies of the measurement history to plaq / poly, on the lattice's
// stream.  clear_flags: start from cleared sampler flags (the synchronous
// call reads them back; the asynchronous one leaves them for su2_sync).
static su2_status generate_enqueue(su2_lattice *lat, int nsweeps, int measure_every, int reunit_every,
                                   double *plaq, double *poly, bool clear_flags)
{
    const int nmeas = measure_every > 0 ? nsweeps / measure_every : 0;
    su2_status st = ensure_history(lat, nmeas);
    if (st != SU2_OK) return st;
    if (clear_flags) {
        if ((st = launch_clear_counters(lat)) != SU2_OK) return st;
    } else {
        SU2_CUDA(cudaMemsetAsync(lat->scratch.trials, 0, sizeof(unsigned long long) * 8 * kTrialSlots,
                                 lat->stream));
    }
    lat->hb_log.used = 0;
    lat->or_log.used = 0;
    // Graph replays need a stream that can be captured and no per-launch events.
    bool graphs = lat->stream != nullptr && !lat->timing && !lat->graphs_off && nsweeps >= 1;
    if (graphs) {
        set_counters_kernel<<<1, 1, 0, lat->stream>>>(lat->d_ctr, lat->sweep);
        SU2_CUDA(cudaGetLastError());
    }
    int m = 0;
    for (int s = 1; s <= nsweeps; ++s) {
        const bool measure = measure_every > 0 && s % measure_every == 0;
        const bool reunit = reunit_every > 0 && s % reunit_every == 0;
        if (graphs) {
            cudaGraphExec_t exec = nullptr;
            if ((st = generation_graph(lat, measure, reunit, &exec)) != SU2_OK) return st;
            if (exec) {
                SU2_CUDA(cudaGraphLaunch(exec, lat->stream));
                lat->sweep += 1;
                if (measure) ++m;
                continue;
            }
            graphs = false;  // capture refused: run the rest eagerly
        }
        if ((st = sweep_and_measure(lat, measure, reunit, lat->scratch.history + m,
                                    lat->scratch.history + lat->scratch.history_cap + m)) != SU2_OK)
            return st;
        if (measure) ++m;
    }
    if (nmeas > 0 && plaq)
        SU2_CUDA(cudaMemcpyAsync(plaq, lat->scratch.history, sizeof(double) * nmeas, cudaMemcpyDeviceToHost,
                                 lat->stream));
    if (nmeas > 0 && poly)
        SU2_CUDA(cudaMemcpyAsync(poly, lat->scratch.history + lat->scratch.history_cap, sizeof(double) * nmeas,
                                 cudaMemcpyDeviceToHost, lat->stream));
    return SU2_OK;
}

}  // namespace su2

using namespace su2;

extern "C" {

su2_status su2_generate(su2_lattice *lat, int nsweeps, int measure_every, int reunit_every, double *plaq,
                        double *poly, su2_stats *stats)
{
    if (!lat || nsweeps < 0 || measure_every < 0 || reunit_every < 0) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    su2_status st = generate_enqueue(lat, nsweeps, measure_every, reunit_every, plaq, poly, true);
    if (st != SU2_OK) return st;
    if (stats) memset(stats, 0, sizeof *stats);
    st = collect_stats(lat, stats, (uint64_t)nsweeps);
    if (stats) {
        stats->kernel_launches = (uint32_t)(8 * nsweeps);
        stats->overrelax_sweeps = (uint64_t)nsweeps * (uint64_t)lat->overrelax;
        stats->overrelax_updates = stats->overrelax_sweeps * 4ull * (uint64_t)lat->vol;
    }
    su2_status st2 = read_timing(lat, stats);
    return st != SU2_OK ? st : st2;
}

su2_status su2_generate_async(su2_lattice *lat, int nsweeps, int measure_every, int reunit_every, double *plaq,
                              double *poly)
{
    if (!lat || nsweeps < 0 || measure_every < 0 || reunit_every < 0) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    return generate_enqueue(lat, nsweeps, measure_every, reunit_every, plaq, poly, false);
}

su2_status su2_heatbath_sweep(su2_lattice *lat, int nsweeps, su2_stats *stats)
{
    if (!lat || nsweeps < 0) return SU2_E_INVAL;
    if (stats) return su2_generate(lat, nsweeps, 0, 0, nullptr, nullptr, stats);
    DeviceGuard guard(lat->device);
    su2_status st;
    lat->hb_log.used = 0;
    lat->or_log.used = 0;
    for (int s = 0; s < nsweeps; ++s)
        if ((st = one_sweep(lat)) != SU2_OK) return st;
    lat->hb_log.used = 0;
    lat->or_log.used = 0;
    return SU2_OK;
}

su2_status su2_set_trial_cap(su2_lattice *lat, int max_trials)
{
    if (!lat || max_trials < 2 || max_trials > kMaxTrials || (max_trials & 1)) return SU2_E_INVAL;
    lat->max_trials = max_trials;
    return SU2_OK;
}

su2_status su2_heatbath_phase(su2_lattice *lat, int mu, int parity)
{
    if (!lat || mu < 0 || mu > 3 || (parity != 0 && parity != 1)) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    return launch_hb_phase(lat, mu, parity, lat->sweep);
}

}  // extern "C"
