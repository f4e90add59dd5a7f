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
    unsigned long long *trial_slots;
    unsigned int *flags;
    const unsigned int *gate;  // if non-NULL and *gate == 1 the phase is left to the learned kernel
};

constexpr int kHbWarps = kHbThreads / 32;

// One heat-bath phase (mu = MU, sites of parity p.parity).
//
// The V/2 sites are cut into rounds of 32 consecutive even/odd indices; warp
// w takes rounds w, w + W, w + 2W, ... (W warps in the grid), so all warps
// sweep the lattice together and neighbour links are re-read from L2.  Each
// warp runs one loop whose iterations interleave three kinds of work:
//   A  one third of the staple of its next round (the six links of one nu):
//      the loads are issued first and used at the end of the iteration, so
//      their latency hides behind B;  after the third part, U~^dag, beta k
//      and exp(-2 beta k) of the 32 sites go into the warp's ring of R rounds;
//   B  one Philox block (two Creutz trials) for the pending link each lane
//      holds; a lane whose link is accepted takes the next pending link of the
//      ring, so no lane idles while the slowest draw of its round finishes;
//   C  once every link of the oldest round is accepted, the 32 lanes draw the
//      directions and store U' = a U~^dag together (coalesced).
// A link's random numbers depend only on its counter, never on the lane or
// the iteration that handles it, so the phase computes exactly the
// one-thread-per-link definition.  Every iteration advances A, B or C, and B
// ends every link within kMaxTrials trials, so the loop terminates.
template <int MU, int R>
__global__ void __launch_bounds__(kHbThreads) hb_phase_kernel(const HbParams p)
{
    if (p.gate != nullptr && *(volatile const unsigned int *)p.gate == 1u) return;
    constexpr int Q = 32 * R;
    __shared__ float4 s_ut[kHbWarps][Q];
    __shared__ float s_bk[kHbWarps][Q];  // beta k; after acceptance a0 (NaN: trial cap hit)
    __shared__ float s_e[kHbWarps][Q];
    __shared__ int s_done[kHbWarps][R];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float4 *const ut_q = s_ut[wib];
    float *const bk_q = s_bk[wib];
    float *const e_q = s_e[wib];
    int *const done_q = s_done[wib];
    const unsigned int lanes_below = (1u << lane) - 1u;
    const int warp_global = blockIdx.x * kHbWarps + wib;
    const int nwarps = gridDim.x * kHbWarps;
    const int vh = p.g.vh;
    const int rounds_total = (vh + 31) >> 5;
    const int my_rounds = warp_global < rounds_total ? (rounds_total - warp_global + nwarps - 1) / nwarps : 0;
    const uint32_t sw_creutz = stream_word(kCreutz, (uint32_t)p.parity, MU);
    const uint32_t sw_dir = stream_word(kDirection, (uint32_t)p.parity, MU);

    if (lane < R) done_q[lane] = 0;
    unsigned int my_trials = 0;

    int a = 0, sub = 0;  // A: rounds produced, part (0..2) of the next one
    int f = 0;           // C: rounds finalised
    int produced = 0;    // valid links produced so far (their sequence numbers are 0 .. produced-1)
    int claim = 0;       // next sequence number to hand out
    int item = -1;       // B: sequence number of this lane's pending link
    int item_eo = 0;
    uint32_t blk = 0;
    float bk = 0.0f, e = 0.0f, ome = 1.0f;
    bool haar = false;
    Coord xa;            // A: site of this lane in round a
    int lex_pa = 0;
    float4 va = make_float4(0.0f, 0.0f, 0.0f, 0.0f);

    while (true) {
        __syncwarp();
        // ---- C: finalise every complete round, oldest first
        while (f < a) {
            const int k = warp_global + f * nwarps;
            const int rsize = min(32, vh - 32 * k);
            if (done_q[f % R] < rsize) break;
            if (lane < rsize) {
                const int slot = (f % R) * 32 + lane;
                const int eo = 32 * k + lane;
                const float a0 = bk_q[slot];
                if (a0 == a0) {
                    const uint4 d = philox_rk(make_uint4((uint32_t)eo, p.sweep, sw_dir, 0u), p.rk);
                    p.links[link_index(p.g, MU, p.parity, eo)] = direction_update(a0, ut_q[slot], d);
                } else {
                    atomicAdd(&p.flags[0], 1u);
                }
            }
            __syncwarp();
            if (lane == 0) done_q[f % R] = 0;
            __syncwarp();
            ++f;
        }
        if (f == my_rounds) break;

        // ---- hand pending links to idle lanes
        {
            const unsigned int need = __ballot_sync(0xffffffffu, item < 0);
            const int avail = produced - claim;
            if (item < 0) {
                const int rank = __popc(need & lanes_below);
                if (rank < avail) {
                    item = claim + rank;
                    const int slot = item % Q;
                    const int k = warp_global + (item >> 5) * nwarps;
                    item_eo = 32 * k + (item & 31);
                    blk = 0;
                    bk = bk_q[slot];
                    e = e_q[slot];
                    ome = __fsub_rn(1.0f, e);
                    haar = bk < kHaarBelow;
                }
            }
            claim += min(__popc(need), avail);
        }

        const bool do_a = a < my_rounds && a < f + R;
        const int a_k = warp_global + a * nwarps;
        const bool a_valid = do_a && 32 * a_k + lane < vh;
        NuLinks nl;
        // ---- A (issue): the six links of one nu for this lane's site of round a
        if (a_valid) {
            if (sub == 0) {
                xa = eo_to_coord(p.g, 32 * a_k + lane, p.parity);
                lex_pa = lex_fwd(p.g, xa.lex, xa.c[MU], MU);
                va = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
            // the three directions nu != MU, ascending
            if (sub == 0)
                nl = load_nu<MU, (MU == 0 ? 1 : 0)>(p.links, p.g, xa, lex_pa, p.parity);
            else if (sub == 1)
                nl = load_nu<MU, (MU <= 1 ? 2 : 1)>(p.links, p.g, xa, lex_pa, p.parity);
            else
                nl = load_nu<MU, (MU <= 2 ? 3 : 2)>(p.links, p.g, xa, lex_pa, p.parity);
        }

        // ---- B: one Philox block (two trials) for the pending link
        if (item >= 0) {
            const uint4 w = philox_rk(make_uint4((uint32_t)item_eo, p.sweep, sw_creutz, blk), p.rk);
            float cand;
            uint32_t t = 0;
            if (creutz_trial(uniform01(w.x), uniform01(w.y), bk, e, ome, haar, cand))
                t = 2 * blk + 1;
            else if (creutz_trial(uniform01(w.z), uniform01(w.w), bk, e, ome, haar, cand))
                t = 2 * blk + 2;
            bool finished = false;
            if (t) {
                my_trials += t;
                finished = true;
            } else if (++blk == (uint32_t)(kMaxTrials / 2)) {
                cand = __int_as_float(0x7fc00000);  // NaN: trial cap hit, the link keeps its value
                my_trials += kMaxTrials;
                finished = true;
            }
            if (finished) {
                bk_q[item % Q] = cand;
                atomicAdd(&done_q[(item >> 5) % R], 1);
                item = -1;
            }
        }

        // ---- A (use): add the two staple terms of nu; after the third part park the site
        if (do_a) {
            if (a_valid) {
                va = add_nu_terms(va, nl);
                if (sub == 2) {
                    const DrawSetup d = prepare_draw(va, p.beta);
                    const int slot = (a % R) * 32 + lane;
                    ut_q[slot] = d.ut;
                    bk_q[slot] = d.bk;
                    e_q[slot] = d.e;
                }
            }
            if (++sub == 3) {
                sub = 0;
                produced += min(32, vh - 32 * a_k);
                ++a;
            }
        }
    }
    const unsigned int wsum = __reduce_add_sync(0xffffffffu, my_trials);
    if (lane == 0 && wsum)
        atomicAdd(&p.trial_slots[(2 * MU + p.parity) * kTrialSlots + (warp_global & (kTrialSlots - 1))],
                  (unsigned long long)wsum);
}

// Depth R of each warp's ring (rounds of 32 links in flight).  SU2_HB_QUEUE
// = 2 | 4 | 8 overrides the default of 8 (tuning).
static int queue_depth()
{
    static const int depth = [] {
        const char *env = getenv("SU2_HB_QUEUE");
        const int d = env ? atoi(env) : 8;
        return (d == 2 || d == 4) ? d : 8;
    }();
    return depth;
}

template <int MU, int R>
static cudaError_t launch_hb(const HbParams &p, int device, cudaStream_t stream)
{
    static int blocks_per_sm[64] = {};
    static int num_sms[64] = {};
    if (device < 0 || device >= 64) device = 0;
    if (!blocks_per_sm[device]) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[device],
                                                                      hb_phase_kernel<MU, R>, kHbThreads, 0);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&num_sms[device], cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm[device] < 1) blocks_per_sm[device] = 1;
    }
    const int rounds = (p.g.vh + 31) / 32;
    const int want = (rounds + kHbWarps - 1) / kHbWarps;
    const int grid = std::max(1, std::min(want, blocks_per_sm[device] * num_sms[device]));
    hb_phase_kernel<MU, R><<<grid, kHbThreads, 0, stream>>>(p);
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
    p.trial_slots = lat->scratch.trials;
    p.flags = lat->scratch.flags;
    const int R = queue_depth();
    cudaError_t e;
    switch (R * 4 + mu) {
    case 8: e = launch_hb<0, 2>(p, lat->device, lat->stream); break;
    case 9: e = launch_hb<1, 2>(p, lat->device, lat->stream); break;
    case 10: e = launch_hb<2, 2>(p, lat->device, lat->stream); break;
    case 11: e = launch_hb<3, 2>(p, lat->device, lat->stream); break;
    case 16: e = launch_hb<0, 4>(p, lat->device, lat->stream); break;
    case 17: e = launch_hb<1, 4>(p, lat->device, lat->stream); break;
    case 18: e = launch_hb<2, 4>(p, lat->device, lat->stream); break;
    case 19: e = launch_hb<3, 4>(p, lat->device, lat->stream); break;
    case 32: e = launch_hb<0, 8>(p, lat->device, lat->stream); break;
    case 33: e = launch_hb<1, 8>(p, lat->device, lat->stream); break;
    case 34: e = launch_hb<2, 8>(p, lat->device, lat->stream); break;
    default: e = launch_hb<3, 8>(p, lat->device, lat->stream); break;
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

// One heat-bath sweep, then the lattice's over-relaxation sweeps.
static su2_status one_sweep(su2_lattice *lat)
{
    for (int mu = 0; mu < 4; ++mu)
        for (int parity = 0; parity < 2; ++parity) {
            su2_status st = timed_phase(lat, mu, parity, lat->sweep);
            if (st != SU2_OK) return st;
        }
    lat->sweep += 1;
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

}  // namespace su2

using namespace su2;

extern "C" {

su2_status su2_generate(su2_lattice *lat, int nsweeps, int measure_every, int reunit_every, double *plaq,
                        double *poly, su2_stats *stats)
{
    if (!lat || nsweeps < 0 || measure_every < 0 || reunit_every < 0) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    const int nmeas = measure_every > 0 ? nsweeps / measure_every : 0;
    su2_status st = ensure_history(lat, nmeas);
    if (st != SU2_OK) return st;
    if ((st = launch_clear_counters(lat)) != SU2_OK) return st;
    lat->hb_log.used = 0;
    lat->or_log.used = 0;
    int m = 0;
    for (int s = 1; s <= nsweeps; ++s) {
        if ((st = one_sweep(lat)) != SU2_OK) return st;
        if (reunit_every > 0 && s % reunit_every == 0 && (st = launch_reunitarize(lat)) != SU2_OK) return st;
        if (measure_every > 0 && s % measure_every == 0) {
            if ((st = launch_plaquette(lat, lat->scratch.history + m)) != SU2_OK) return st;
            if ((st = launch_polyakov(lat, lat->scratch.history + lat->scratch.history_cap + m)) != SU2_OK) return st;
            ++m;
        }
    }
    if (nmeas > 0 && plaq)
        SU2_CUDA(cudaMemcpyAsync(plaq, lat->scratch.history, sizeof(double) * nmeas, cudaMemcpyDeviceToHost,
                                 lat->stream));
    if (nmeas > 0 && poly)
        SU2_CUDA(cudaMemcpyAsync(poly, lat->scratch.history + lat->scratch.history_cap, sizeof(double) * nmeas,
                                 cudaMemcpyDeviceToHost, lat->stream));
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

su2_status su2_heatbath_phase(su2_lattice *lat, int mu, int parity)
{
    if (!lat || mu < 0 || mu > 3 || (parity != 0 && parity != 1)) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    return launch_hb_phase(lat, mu, parity, lat->sweep);
}

}  // extern "C"
