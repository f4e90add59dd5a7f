// kp.cu -- heat-bath phase with the Kennedy-Pendleton a0 sampler
// (Phys. Lett. B 156 (1985) 393).  Same law as Creutz's method (Sec. 2
// heat bath), but at large beta k nearly every trial is accepted: one thread
// per link, persistent grid, the staple of the next link loaded during the
// draw of the current one, and the few rejected links retried warp-wide.
//
// With a0 = 1 - 2u the law of u is u^{1/2} sqrt(1 - u) exp(-2 beta k u) on
// [0, 1]; a trial draws u = -(ln r1 + cos^2(2 pi r2) ln r3) / (2 beta k) and
// accepts iff u <= 1 and r4^2 <= 1 - u (block t of the KP stream).  Links with
// beta k < 2 are drawn by Creutz's method exactly as the plain kernel does.
#include <algorithm>

#include "kp_device.cuh"
#include "observables.cuh"
#include "staple.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

constexpr int kKpThreads = 128;
#ifndef SU2_KP_MIN_BLOCKS
#define SU2_KP_MIN_BLOCKS 6
#endif
constexpr int kKpMinBlocks = SU2_KP_MIN_BLOCKS;  // blocks per SM the register budget is set for

struct KpParams {
    float4 *links;
    Geom g;
    RoundKeys rk;
    int parity;
    float beta;
    uint32_t sweep;
    const uint32_t *sweep_dev;  // if non-NULL the sweep counter is read here (graph replays)
    int max_trials;             // trials a link may use before it keeps its old value
    unsigned long long *trial_slots;
    unsigned int *flags;
    const unsigned int *gate;  // skip the phase while *gate == 1 (learned sweeps)
    double *plaq;              // measuring phases: block partials of the plaquettes of planes (nu < mu, mu)
    SlabRange slab;            // SLAB kernels: the interior eo range and the global keys of its random numbers
    const float4 *same[4];     // links of direction d at the phase's parity
    const float4 *other[4];    // ... at the opposite parity
};

constexpr int kKpWarps = kKpThreads / 32;
constexpr int kRetryCap = 64;  // per warp: at most 31 left over + 32 pushed by one round

// Warp w of the grid takes the rounds of 32 consecutive links w, w + W, ...
// (W warps).  Each loop iteration (three per round) issues the six loads of
// one nu-group of the next round, does one third of the current round's
// draw, then folds the loaded group into the next round's staple, so 24
// registers of loads are in flight and the draw's arithmetic covers their
// latency:
//   part 0  k, beta k, U~^dag; the Philox blocks of the first trial and of
//           the direction;
//   part 1  the first trial;
//   part 2  the direction and the store of every accepted link.
// A link whose first trial is rejected is parked in the warp's retry queue
// in shared memory (U~^dag, beta k, index), and so is a link with beta k < 2
// (its staple in place of U~^dag), which the retry pass draws by Creutz's
// method exactly as the plain kernel does; keeping that rare draw out of the
// main loop leaves its registers to the pipeline (no spills).  Once 32 links wait, the whole
// warp runs their further trials 1, 2, ... together, so no warp spins on one
// lane's rejections.  Every draw depends only on the link's counters, so the
// phase computes exactly the one-thread-per-link definition.  Lanes past the
// end (last round, next round) work on a clamped index and drop their
// results, so the main path has no divergent branch.  MEAS: the plaquette
// contributions (1/2) Tr U'S, S the staple terms of nu < MU, as in the
// Creutz kernel.
template <int MU, bool MEAS, bool SLAB>
__global__ void __launch_bounds__(kKpThreads, kKpMinBlocks) kp_phase_kernel(const KpParams p)
{
    // a time slab: interior eo range, random numbers of the global site
    const int eo_begin = SLAB ? p.slab.eo_begin : 0;
    const int eo_end = SLAB ? p.slab.eo_end : p.g.vh;
    const uint32_t rng_eo = SLAB ? p.slab.rng_eo : 0u;
    const uint32_t rng_parity = SLAB ? (uint32_t)p.slab.rng_parity : (uint32_t)p.parity;
    if (p.gate != nullptr && *(volatile const unsigned int *)p.gate == 1u) return;
    __shared__ float4 s_ut[kKpWarps][kRetryCap];
    __shared__ float4 s_sp[MEAS ? kKpWarps : 1][kRetryCap];
    const uint32_t sweep = p.sweep_dev ? *p.sweep_dev : p.sweep;
    __shared__ float s_bk[kKpWarps][kRetryCap];
    __shared__ int s_eo[kKpWarps][kRetryCap];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const unsigned int lanes_below = (1u << lane) - 1u;
    const int stride = gridDim.x * kKpThreads;
    const int last = eo_end - 1;
    const uint32_t sw_kp = stream_word(kKennedyPendleton, rng_parity, MU);
    const uint32_t sw_dir = stream_word(kDirection, rng_parity, MU);
    unsigned int trials = 0;
    float plaq = 0.0f;  // per-thread partial in binary32; the block and grid sums are binary64
    int queued = 0;  // warp-uniform length of the retry queue

    // Trials 1, 2, ... of the queue entry of this lane (lane < n), then the
    // direction and the store.
    auto retry = [&](int first, int n) {
        if (lane < n) {
            const int q = first + lane;
            const float4 ut = s_ut[wib][q];
            const float bk_q = s_bk[wib][q];
            const float two_bk = __fmul_rn(2.0f, bk_q);
            const int eo = s_eo[wib][q];
            float a0 = 0.0f;
            int t = 1;
            if (!(bk_q >= kKpMinBk)) {  // beta k < 2: Creutz's method; the queue holds the staple
                float4 out;
                const int n = heatbath_draw(ut, p.beta, p.rk, (uint32_t)eo + rng_eo, sweep, rng_parity, MU, out);
                if (n > 0) {
                    p.links[link_index(p.g, MU, p.parity, eo)] = out;
                    if (MEAS) plaq = __fadd_rn(plaq, qmul_re(out, s_sp[MEAS ? wib : 0][q]));
                    trials += (unsigned int)n;
                } else {
                    atomicAdd(&p.flags[0], 1u);
                    trials += (unsigned int)kMaxTrials;
                }
                t = -1;
            } else {
                for (; t < p.max_trials; ++t)
                    if (kp_trial(philox_rk(make_uint4((uint32_t)eo + rng_eo, sweep, sw_kp, (uint32_t)t), p.rk), two_bk,
                                 a0))
                        break;
            }
            if (t < 0) {
            } else if (t < p.max_trials) {
                const float4 out =
                    direction_update(a0, ut,
                                     philox_rk(make_uint4(direction_pair((uint32_t)eo + rng_eo), sweep, sw_dir, 0u), p.rk),
                                     (uint32_t)eo + rng_eo);
                p.links[link_index(p.g, MU, p.parity, eo)] = out;
                if (MEAS) plaq = __fadd_rn(plaq, qmul_re(out, s_sp[MEAS ? wib : 0][q]));
                trials += (unsigned int)(t + 1);
            } else {
                atomicAdd(&p.flags[0], 1u);  // trial cap: the link keeps its old value
                trials += (unsigned int)p.max_trials;
            }
        }
        __syncwarp();
    };

    int base = eo_begin + blockIdx.x * kKpThreads + (wib << 5);
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
    // Direction blocks, one per pair of links (2j, 2j + 1) of a round: in an
    // even round of the warp, lanes 0..15 draw the blocks of this round's 16
    // pairs and lanes 16..31 those of the next round's (base + stride), so a
    // lane draws three Philox blocks per two links; each link takes its two
    // words from the lane that drew its pair's block.
    bool even_round = true;
    uint4 dblk = make_uint4(0u, 0u, 0u, 0u);
    while (base < eo_end) {  // warp-uniform
        const bool valid = cur <= last;
        const int nxt = cur + stride;
        const int en = min(nxt, last);
        const Coord xn = eo_to_coord(p.g, en, p.parity);
        const int en_p = eo_fwd<MU>(p.g, xn, en);
        // ---- part 0
        NuLinks nl = load_nu_bases<MU, OtherDir<MU, 0>::value>(p.same, p.other, p.g, xn, en, en_p);
        const float k = __fsqrt_rn(qnorm2(v_cur));
        const float bk = __fmul_rn(p.beta, k);
        const bool use_kp = bk >= kKpMinBk;
        const float inv_k = __frcp_rn(k);
        const float4 ut = make_float4(__fmul_rn(v_cur.x, inv_k), __fmul_rn(-v_cur.y, inv_k),
                                      __fmul_rn(-v_cur.z, inv_k), __fmul_rn(-v_cur.w, inv_k));
        uint4 w = make_uint4((uint32_t)cur + rng_eo, sweep, sw_kp, 0u);
        if (even_round) {  // warp-uniform
            const uint32_t pair0 = direction_pair((uint32_t)(lane < 16 ? base : base + stride) + rng_eo);
            dblk = make_uint4(pair0 + (uint32_t)(lane & 15), sweep, sw_dir, 0u);
            philox2_rk(w, dblk, p.rk);
        } else {
            w = philox_rk(w, p.rk);
        }
        float4 v_next = add_nu_terms(make_float4(0.0f, 0.0f, 0.0f, 0.0f), nl);
        float4 sp_next = v_next;
        // ---- part 1
        nl = load_nu_bases<MU, OtherDir<MU, 1>::value>(p.same, p.other, p.g, xn, en, en_p);
        float a0;
        const bool first_ok = kp_trial(w, __fmul_rn(2.0f, bk), a0);
        const bool accepted = valid && use_kp && first_ok;
        const bool park = valid && !(use_kp && first_ok);  // rejected, or beta k < 2 (Creutz, in the queue)
        const unsigned int parked = __ballot_sync(0xffffffffu, park);
        if (park) {  // rare at large beta k: a branch costs less than stores from every lane
            const int q = queued + __popc(parked & lanes_below);
            s_ut[wib][q] = use_kp ? ut : v_cur;
            s_bk[wib][q] = bk;
            s_eo[wib][q] = cur;
            if (MEAS) s_sp[MEAS ? wib : 0][q] = sp_cur;
        }
        queued += __popc(parked);
        v_next = add_nu_terms(v_next, nl);
        if (MU == 2) sp_next = v_next;
        // ---- part 2
        nl = load_nu_bases<MU, OtherDir<MU, 2>::value>(p.same, p.other, p.g, xn, en, en_p);
        const int src = (even_round ? 0 : 16) + (lane >> 1);
        const uint4 wd = make_uint4(__shfl_sync(0xffffffffu, dblk.x, src), __shfl_sync(0xffffffffu, dblk.y, src),
                                    __shfl_sync(0xffffffffu, dblk.z, src), __shfl_sync(0xffffffffu, dblk.w, src));
        const float4 out = direction_update(a0, ut, wd, (uint32_t)cur + rng_eo);
        if (accepted) p.links[link_index(p.g, MU, p.parity, cur)] = out;
        if (MEAS && accepted) plaq = __fadd_rn(plaq, qmul_re(out, sp_cur));
        trials += accepted ? 1u : 0u;
        v_next = add_nu_terms(v_next, nl);
        if (MU == 3) sp_next = v_next;
        __syncwarp();
        if (queued >= 32) {
            queued -= 32;
            retry(queued, 32);
        }
        base += stride;
        cur = nxt;
        v_cur = v_next;
        sp_cur = sp_next;
        even_round = !even_round;
    }
    if (queued > 0) retry(0, queued);
    const unsigned int wsum = __reduce_add_sync(0xffffffffu, trials);
    if (lane == 0 && wsum)
        atomicAdd(&p.trial_slots[(2 * MU + p.parity) * kTrialSlots + ((blockIdx.x * kKpWarps + wib) &
                                                                      (kTrialSlots - 1))],
                  (unsigned long long)wsum);
    if (MEAS) {
        const double total = block_sum((double)plaq);
        if (threadIdx.x == 0) p.plaq[blockIdx.x] = total;
    }
}

template <int MU, bool MEAS, bool SLAB = false>
static cudaError_t launch_kp(const KpParams &p, int device, cudaStream_t stream)
{
    static int per_sm[64] = {};
    static int sms[64] = {};
    if (device < 0 || device >= 64) device = 0;
    if (!per_sm[device]) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[device],
                                                                      kp_phase_kernel<MU, MEAS, SLAB>, kKpThreads, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms[device], cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        per_sm[device] = std::max(1, per_sm[device]);
    }
    const int n = SLAB ? p.slab.eo_end - p.slab.eo_begin : p.g.vh;
    const int want = (n + kKpThreads - 1) / kKpThreads;
    const int grid = std::max(1, std::min(std::min(want, per_sm[device] * sms[device]), kFusedSlots));
    kp_phase_kernel<MU, MEAS, SLAB><<<grid, kKpThreads, 0, stream>>>(p);
    return cudaGetLastError();
}

su2_status launch_kp_phase(su2_lattice *lat, int mu, int parity, uint32_t sweep, const unsigned int *gate)
{
    KpParams p;
    p.links = lat->links;
    p.g = geom_of(lat);
    p.rk = make_round_keys(lat->seed);
    p.parity = parity;
    p.beta = (float)lat->beta;
    p.sweep = sweep;
    p.sweep_dev = lat->capturing ? lat->d_ctr : nullptr;
    p.max_trials = lat->max_trials;
    p.trial_slots = lat->scratch.trials;
    p.flags = lat->scratch.flags;
    p.gate = gate;
    p.plaq = fused_slot(lat, mu, parity, 0);
    set_bases(p.same, p.other, lat, parity);
    cudaError_t e;
    if (p.plaq) {
        switch (mu) {
        case 1: e = launch_kp<1, true>(p, lat->device, lat->stream); break;
        case 2: e = launch_kp<2, true>(p, lat->device, lat->stream); break;
        default: e = launch_kp<3, true>(p, lat->device, lat->stream); break;
        }
    } else {
        switch (mu) {
        case 0: e = launch_kp<0, false>(p, lat->device, lat->stream); break;
        case 1: e = launch_kp<1, false>(p, lat->device, lat->stream); break;
        case 2: e = launch_kp<2, false>(p, lat->device, lat->stream); break;
        default: e = launch_kp<3, false>(p, lat->device, lat->stream); break;
        }
    }
    SU2_CUDA(e);
    return SU2_OK;
}

su2_status launch_kp_phase_slab(su2_lattice *lat, int mu, int parity_local, uint32_t sweep, const SlabRange &r)
{
    KpParams p;
    p.links = lat->links;
    p.g = geom_of(lat);
    p.rk = make_round_keys(lat->seed);
    p.parity = parity_local;
    p.beta = (float)lat->beta;
    p.sweep = sweep;
    p.sweep_dev = nullptr;
    p.max_trials = lat->max_trials;
    p.trial_slots = lat->scratch.trials;
    p.flags = lat->scratch.flags;
    p.gate = nullptr;
    p.plaq = nullptr;
    p.slab = r;
    set_bases(p.same, p.other, lat, parity_local);
    cudaError_t e;
    switch (mu) {
    case 0: e = launch_kp<0, false, true>(p, lat->device, lat->stream); break;
    case 1: e = launch_kp<1, false, true>(p, lat->device, lat->stream); break;
    case 2: e = launch_kp<2, false, true>(p, lat->device, lat->stream); break;
    default: e = launch_kp<3, false, true>(p, lat->device, lat->stream); break;
    }
    SU2_CUDA(e);
    return SU2_OK;
}

}  // namespace su2

extern "C" su2_status su2_set_sampler(su2_lattice *lat, int sampler)
{
    if (!lat || (sampler != SU2_SAMPLER_CREUTZ && sampler != SU2_SAMPLER_KP)) return SU2_E_INVAL;
    lat->sampler = sampler;
    return SU2_OK;
}
