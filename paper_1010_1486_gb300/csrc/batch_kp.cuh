// batch_kp.cuh -- the batched phase with the Kennedy-Pendleton a0 sampler:
// the phase of every lattice runs the single-lattice Kennedy-Pendleton
// pipeline (kp.cu) on the warp's segments, with the lattice's own Philox key,
// so each lattice's links equal those of su2_create + su2_set_sampler(KP) +
// su2_heatbath_sweep with the same arguments.  Included by the translation
// units that instantiate the Kennedy-Pendleton batch kernels.
#pragma once

#include "batch_device.cuh"
#include "kp_device.cuh"

namespace su2 {

// One phase (MU, parity) over every lattice.  Chunks and segments as in
// batch_phase: the warp's contiguous range of chunks of 32 R sites, each run
// of one lattice a segment with the lattice's descriptor staged in the warp's
// shared slot.  Per segment, rounds of 32 consecutive sites: the next round's
// staple is loaded one nu-group per stage while the current round is drawn
// (part 0: k, U~^dag, the first trial's and the direction's Philox blocks;
// part 1: the first trial; part 2: direction and store of accepted links).
// A link whose first trial is rejected, or with beta k < 2 (then drawn by
// Creutz's method, its staple queued in place of U~^dag), waits in the warp's
// queue; 32 waiting links are finished together, and the queue is emptied at
// the segment's end.  MEAS: the segment's (1/2) Tr U'S sum goes to the slot
// of its first chunk, as in batch_phase.
template <int MU, int R, bool MEAS>
__device__ void batch_phase_kp(const BatchParams &bp, int parity, uint32_t sweep, CrQueues &Q, LatDesc &sd,
                               unsigned int &my_trials)
{
    constexpr int C = 32 * R;
    const int lane = threadIdx.x & 31;
    const unsigned int lanes_below = (1u << lane) - 1u;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t sw_kp = stream_word(kKennedyPendleton, (uint32_t)parity, MU);
    const uint32_t sw_dir = stream_word(kDirection, (uint32_t)parity, MU);
    const int per = bp.total_chunks / nwarps, extra = bp.total_chunks % nwarps;
    const int c_end = warp_global * per + min(warp_global, extra) + per + (warp_global < extra ? 1 : 0);
    for (int chunk = warp_global * per + min(warp_global, extra); chunk < c_end;) {
        const int l = __ldg(bp.chunk_owner + chunk);
        const int lat_c0 = __ldg(bp.chunk_prefix + l);
        const int seg_end = min(c_end, __ldg(bp.chunk_prefix + l + 1));
        __syncwarp();
        {
            constexpr int kWords = (int)(sizeof(LatDesc) / sizeof(unsigned int));
            const unsigned int *src = (const unsigned int *)(bp.desc + l);
            unsigned int *dst = (unsigned int *)&sd;
            for (int i = lane; i < kWords; i += 32) dst[i] = __ldg(src + i);
        }
        __syncwarp();
        const Geom &g = sd.g;
        float4 *const links = sd.links;
        const uint32_t k0 = sd.k0, k1 = sd.k1;
        const float beta = sd.beta;
        const int base0 = (chunk - lat_c0) * C;
        const int last = min((seg_end - lat_c0) * C, g.vh) - 1;
        const int rounds = (last - base0 + 32) >> 5;
        int queued = 0;
        float plaq = 0.0f;  // per-thread partial in binary32; the block and grid sums are binary64
        auto gen = [&](uint4 c) { return philox_key(c, k0, k1); };

        // the queued links of lanes < n: further trials (or Creutz's method
        // below beta k = 2), then the direction and the store
        auto retry = [&](int first, int n) {
            if (lane < n) {
                const int q = first + lane;
                const float4 ut = Q.r_ut[q];
                const float bk_q = Q.r_ibk[q];
                const int eo = Q.r_eo[q];
                float a0 = 0.0f;
                int t = 1;
                if (!(bk_q >= kKpMinBk)) {  // the queue holds the staple
                    float4 out;
                    const int nt = heatbath_draw_gen(ut, beta, gen, (uint32_t)eo, sweep, (uint32_t)parity, MU, out);
                    if (nt > 0) {
                        links[link_index(g, MU, parity, eo)] = out;
                        if (MEAS) plaq = __fadd_rn(plaq, qmul_re(out, Q.r_sp[q]));
                        my_trials += (unsigned int)nt;
                    } else {
                        atomicAdd(&bp.flags[0], 1u);
                        my_trials += (unsigned int)kMaxTrials;
                    }
                    t = -1;
                } else {
                    const float two_bk = __fmul_rn(2.0f, bk_q);
                    for (; t < kMaxTrials; ++t)
                        if (kp_trial(gen(make_uint4((uint32_t)eo, sweep, sw_kp, (uint32_t)t)), two_bk, a0)) break;
                }
                if (t < 0) {
                } else if (t < kMaxTrials) {
                    const float4 out = direction_update(
                        a0, ut, gen(make_uint4(direction_pair((uint32_t)eo), sweep, sw_dir, 0u)), (uint32_t)eo);
                    links[link_index(g, MU, parity, eo)] = out;
                    if (MEAS) plaq = __fadd_rn(plaq, qmul_re(out, Q.r_sp[q]));
                    my_trials += (unsigned int)(t + 1);
                } else {
                    atomicAdd(&bp.flags[0], 1u);  // trial cap: the link keeps its old value
                    my_trials += (unsigned int)kMaxTrials;
                }
            }
            __syncwarp();
        };

        int cur = base0 + lane;
        float4 v_cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float4 sp_cur = v_cur;  // MEAS: staple terms of nu < MU (the first MU groups)
        {
            const int e = min(cur, last);
            const Coord x = eo_to_coord(g, e, parity);
            const int e_p = eo_fwd<MU>(g, x, e);
            v_cur = add_nu_terms(v_cur, load_nu_eo<MU, OtherDir<MU, 0>::value, false>(links, g, x, e, e_p, parity));
            if (MU == 1) sp_cur = v_cur;
            v_cur = add_nu_terms(v_cur, load_nu_eo<MU, OtherDir<MU, 1>::value, false>(links, g, x, e, e_p, parity));
            if (MU == 2) sp_cur = v_cur;
            v_cur = add_nu_terms(v_cur, load_nu_eo<MU, OtherDir<MU, 2>::value, false>(links, g, x, e, e_p, parity));
            if (MU == 3) sp_cur = v_cur;
        }
        // one direction block per pair of links, as in kp_phase_kernel: in even
        // rounds lanes 0..15 draw this round's pairs, lanes 16..31 the next's
        uint4 dblk = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
        for (int r = 0; r < rounds; ++r) {
            const bool valid = cur <= last;
            const bool even_round = (r & 1) == 0;
            const int nxt = cur + 32;
            const int en = min(nxt, last);  // the last round reloads its own links: harmless
            const Coord xn = eo_to_coord(g, en, parity);
            const int en_p = eo_fwd<MU>(g, xn, en);
            // ---- part 0
            NuLinks nl = load_nu_eo<MU, OtherDir<MU, 0>::value, false>(links, g, xn, en, en_p, parity);
            const float k = __fsqrt_rn(qnorm2(v_cur));
            const float bk = __fmul_rn(beta, k);
            const bool use_kp = bk >= kKpMinBk;
            const float inv_k = __frcp_rn(k);
            const float4 ut = make_float4(__fmul_rn(v_cur.x, inv_k), __fmul_rn(-v_cur.y, inv_k),
                                          __fmul_rn(-v_cur.z, inv_k), __fmul_rn(-v_cur.w, inv_k));
            uint4 w = make_uint4((uint32_t)cur, sweep, sw_kp, 0u);
            if (even_round) {  // warp-uniform
                const int rb = base0 + 32 * r + (lane < 16 ? 0 : 32);
                dblk = make_uint4(direction_pair((uint32_t)rb) + (uint32_t)(lane & 15), sweep, sw_dir, 0u);
                philox2_key(w, dblk, k0, k1);
            } else {
                w = gen(w);
            }
            float4 v_next = add_nu_terms(make_float4(0.0f, 0.0f, 0.0f, 0.0f), nl);
            float4 sp_next = v_next;
            // ---- part 1
            nl = load_nu_eo<MU, OtherDir<MU, 1>::value, false>(links, g, xn, en, en_p, parity);
            float a0;
            const bool first_ok = kp_trial(w, __fmul_rn(2.0f, bk), a0);
            const bool accepted = valid && use_kp && first_ok;
            const bool park = valid && !(use_kp && first_ok);
            const unsigned int parked = __ballot_sync(0xffffffffu, park);
            if (park) {  // rare at large beta k: a branch costs less than stores from every lane
                const int q = queued + __popc(parked & lanes_below);
                Q.r_ut[q] = use_kp ? ut : v_cur;
                Q.r_ibk[q] = bk;
                Q.r_eo[q] = cur;
                if (MEAS) Q.r_sp[q] = sp_cur;
            }
            queued += __popc(parked);
            v_next = add_nu_terms(v_next, nl);
            if (MU == 2) sp_next = v_next;
            // ---- part 2
            nl = load_nu_eo<MU, OtherDir<MU, 2>::value, false>(links, g, xn, en, en_p, parity);
            const int src = (even_round ? 0 : 16) + (lane >> 1);
            const uint4 wd = make_uint4(__shfl_sync(0xffffffffu, dblk.x, src), __shfl_sync(0xffffffffu, dblk.y, src),
                                        __shfl_sync(0xffffffffu, dblk.z, src), __shfl_sync(0xffffffffu, dblk.w, src));
            const float4 out = direction_update(a0, ut, wd, (uint32_t)cur);
            if (accepted) links[link_index(g, MU, parity, cur)] = out;
            if (MEAS && accepted) plaq = __fadd_rn(plaq, qmul_re(out, sp_cur));
            my_trials += accepted ? 1u : 0u;
            v_next = add_nu_terms(v_next, nl);
            if (MU == 3) sp_next = v_next;
            __syncwarp();
            if (queued >= 32) {
                queued -= 32;
                retry(queued, 32);
            }
            cur = nxt;
            v_cur = v_next;
            sp_cur = sp_next;
        }
        if (queued > 0) retry(0, queued);
        if (MEAS) {
            const double total = warp_sum((double)plaq);
            for (int c = chunk + lane; c < seg_end; c += 32)
                bp.chunk_partials[(MU - 1) * bp.total_chunks + c] = c == chunk ? total : 0.0;
        }
        chunk = seg_end;
    }
}

}  // namespace su2
