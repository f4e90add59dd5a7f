// batch_device.cuh -- device side of the batched sweep (batch.cu): one
// persistent cooperative launch per sweep runs the eight even/odd phases of
// many independent lattices with a bounded grid barrier between phases, then
// their measurements.  Shared by the translation units that instantiate the
// kernel for each a0 sampler (batch.cu: Creutz, batch_kp.cu:
// Kennedy-Pendleton).
#pragma once

#include <cuda_runtime.h>

#include "creutz_queue.cuh"
#include "observables.cuh"
#include "staple.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

// Threads per SM the register budget is set for (six blocks of 128): every
// block size T keeps it, with 768 / T blocks per SM.
constexpr int kBatchThreadsPerSm = 768;
constexpr int kBatchBlockSizes[3] = {64, 128, 256};

struct LatDesc {
    Geom g;
    float4 *links;
    uint32_t k0, k1;  // Philox key = seed
    float beta;
    int nplaq_rounds;  // ceil(V / 32) rounds of plaquette sites
    int npoly_rounds;  // ceil(Ns^3 / 32) rounds of Polyakov lines
};

struct BarrierState {
    unsigned int count;
    unsigned int gen;
    unsigned int error;  // bit 0: a barrier wait timed out
    unsigned int pad;
};

struct BatchParams {
    const LatDesc *desc;        // [n]
    const int *chunk_prefix;    // [n + 1]: first heat-bath chunk of each lattice
    const int *mround_prefix;   // [n + 1]: first measurement round of each lattice
    const int *chunk_owner;     // [total_chunks]: lattice of each chunk
    const int *mround_owner;    // [total_mrounds]: lattice of each measurement round
    const int2 *poly_rounds;    // [total_poly_rounds]: (measurement round, lattice) of the Polyakov rounds
    int n;
    int total_chunks;
    int total_mrounds;
    int total_poly_rounds;
    int do_sweep;               // run the eight phases
    int measure;                // then the plaquette and Polyakov loop
    int fused;                  // do_sweep && measure: the plaquette comes from the sweep
    double *chunk_partials;     // [3][total_chunks]: fused plaquette partials of phases (mu, odd), mu = 1, 2, 3
    unsigned int *sweep;        // sweep counter: read at start, advanced at the end
    unsigned int *meas_index;   // next history slot
    double *round_partials;     // [total_mrounds]
    double *history;            // [history_cap][2][n]
    int history_cap;
    BarrierState *bar;
    unsigned long long timeout_ns;
    unsigned long long *trial_slots;  // [8][kTrialSlots]
    unsigned int *flags;              // [0] sampler cap hits
};

__device__ __forceinline__ unsigned long long global_time_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  Every
// wait is bounded by timeout_ns: on expiry the block sets bar->error and all
// blocks stop waiting; the function then returns false everywhere and the
// caller abandons the sweep.
static __device__ bool grid_barrier(BarrierState *bar, unsigned long long timeout_ns)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &bar->gen;
        volatile unsigned int *verr = &bar->error;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == gridDim.x) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const unsigned long long t0 = global_time_ns();
            while (*vgen == g) {
                if (*verr & 1u) break;
                if (global_time_ns() - t0 > timeout_ns) {
                    atomicOr(&bar->error, 1u);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = (*verr & 1u) == 0u;
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// One phase (MU, parity) over every lattice: chunks of 32 R consecutive
// even/odd sites of one lattice; each warp takes a contiguous range of
// chunks and sweeps each lattice's part of it as in the single-lattice
// kernel: the staple of the next round of 32 sites is loaded one nu-group per
// stage while the current round is drawn; the first Philox block (trials 0,
// 1, screened) inline, links with both rejected retried 32 at a time from the
// warp's retry queue, accepted links given their a0, direction and store 32
// at a time; both queues are emptied at the end of the lattice's part.  MEAS
// (odd phases of mu = 1, 2, 3 in a measuring sweep): the part's sum of
// (1/2) Tr U'S, S the staple terms of nu < MU, goes to the slot of its first
// chunk in bp.chunk_partials (its other chunks get zeros); over the three
// phases every plaquette of the final configuration is counted once.
template <int MU, int R, bool MEAS>
__device__ void batch_phase(const BatchParams &bp, int parity, uint32_t sweep, CrQueues &Q, LatDesc &sd,
                            unsigned int &my_trials)
{
    constexpr int C = 32 * R;
    const int lane = threadIdx.x & 31;
    const unsigned int lanes_below = (1u << lane) - 1u;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t sw_creutz = stream_word(kCreutz, (uint32_t)parity, MU);
    const uint32_t sw_dir = stream_word(kDirection, (uint32_t)parity, MU);
    // the warp's contiguous range of chunks (sizes differ by at most one);
    // each run of chunks of one lattice is one segment: one pipeline start and
    // one queue drain per segment
    const int per = bp.total_chunks / nwarps, extra = bp.total_chunks % nwarps;
    const int c_end = warp_global * per + min(warp_global, extra) + per + (warp_global < extra ? 1 : 0);
    for (int chunk = warp_global * per + min(warp_global, extra); chunk < c_end;) {
        const int l = __ldg(bp.chunk_owner + chunk);
        const int lat_c0 = __ldg(bp.chunk_prefix + l);
        const int seg_end = min(c_end, __ldg(bp.chunk_prefix + l + 1));
        // the lattice's descriptor, staged in the warp's shared slot and read
        // from there (holding it in registers would crowd out the pipeline)
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
        int retry_n = 0, done_n = 0;
        float plaq = 0.0f;  // per-thread partial in binary32; the block and grid sums are binary64

        // lanes that push nothing write to the last slot, which no live entry
        // reaches (at most 31 left over + 32 pushed), so the stores need no branch
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
        auto direction_pass = [&](int first, int n) {
            __syncwarp();
            if (lane < n) {
                const int q = first + lane;
                const int eo = Q.d_eo[q];
                const uint4 wd = philox_key(make_uint4(direction_pair((uint32_t)eo), sweep, sw_dir, 0u), k0, k1);
                const float4 out = direction_update(deferred_a0(Q.d_val[q], Q.d_ibk[q]), Q.d_ut[q], wd, (uint32_t)eo);
                links[link_index(g, MU, parity, eo)] = out;
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
            const uint4 w = philox_key(make_uint4((uint32_t)eo, sweep, sw_creutz, (uint32_t)blk), k0, k1);
            bool first_ok;
            float val;
            const bool ok = creutz_pair(w, ibk, e, have, first_ok, val) && have;
            bool again = false;
            if (ok) {
                my_trials += (unsigned int)(2 * blk + (first_ok ? 1 : 2));
            } else if (have) {
                if (blk + 1 < kMaxTrials / 2) {
                    again = true;
                } else {
                    atomicAdd(&bp.flags[0], 1u);  // trial cap: the link keeps its old value
                    my_trials += (unsigned int)kMaxTrials;
                }
            }
            push_retry(again, ut, ibk, e, eo, blk + 1, sp);
            push_done(ok, ut, val, ibk, eo, sp);
            flush_done();
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
#pragma unroll 1
        for (int r = 0; r < rounds; ++r) {
            const bool valid = cur <= last;
            const int nxt = cur + 32;
            const int en = min(nxt, last);  // the last round reloads its own links: harmless
            const Coord xn = eo_to_coord(g, en, parity);
            const int en_p = eo_fwd<MU>(g, xn, en);
            // ---- part 0
            NuLinks nl = load_nu_eo<MU, OtherDir<MU, 0>::value, false>(links, g, xn, en, en_p, parity);
            const DrawSetup ds = prepare_draw(v_cur, beta);
            const uint4 w = philox_key(make_uint4((uint32_t)cur, sweep, sw_creutz, 0u), k0, k1);
            float4 v_next = add_nu_terms(make_float4(0.0f, 0.0f, 0.0f, 0.0f), nl);
            float4 sp_next = v_next;
            // ---- part 1
            nl = load_nu_eo<MU, OtherDir<MU, 1>::value, false>(links, g, xn, en, en_p, parity);
            {
                bool first_ok;
                float val;
                const bool acc = creutz_pair(w, ds.ibk, ds.e, valid, first_ok, val);
                const bool ok = valid && acc;
                my_trials += ok ? (first_ok ? 1u : 2u) : 0u;
                push_done(ok, ds.ut, val, ds.ibk, cur, sp_cur);
                push_retry(valid && !acc, ds.ut, ds.ibk, ds.e, cur, 1, sp_cur);
            }
            v_next = add_nu_terms(v_next, nl);
            if (MU == 2) sp_next = v_next;
            // ---- part 2
            nl = load_nu_eo<MU, OtherDir<MU, 2>::value, false>(links, g, xn, en, en_p, parity);
            flush_done();
            v_next = add_nu_terms(v_next, nl);
            if (MU == 3) sp_next = v_next;
            while (retry_n >= 32) {
                retry_n -= 32;
                retry_pass(retry_n, 32);
            }
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
        if (MEAS) {
            // the segment's sum in the slot of its first chunk, zeros in the others
            const double total = warp_sum((double)plaq);
            for (int c = chunk + lane; c < seg_end; c += 32)
                bp.chunk_partials[(MU - 1) * bp.total_chunks + c] = c == chunk ? total : 0.0;
        }
        chunk = seg_end;
    }
}

// Per round of 32 sites (or 32 Polyakov lines) of one lattice: the warp's
// fp64 sum of the binary32 per-site values, in a fixed order.  After a fused
// sweep only the Polyakov rounds run.
static __device__ void batch_measure_rounds(const BatchParams &bp)
{
    const int lane = threadIdx.x & 31;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int items = bp.fused ? bp.total_poly_rounds : bp.total_mrounds;
    for (int it = warp_global; it < items; it += nwarps) {
        int mr, l;
        if (bp.fused) {
            const int2 pr = __ldg(bp.poly_rounds + it);
            mr = pr.x;
            l = pr.y;
        } else {
            mr = it;
            l = __ldg(bp.mround_owner + it);
        }
        const LatDesc *d = bp.desc + l;
        const int local = mr - __ldg(bp.mround_prefix + l);
        const Geom g = d->g;
        double val = 0.0;
        if (local < d->nplaq_rounds) {
            const int s = local * 32 + lane;
            if (s < 2 * g.vh) {
                const int parity = s >= g.vh;
                const int eo = s - (parity ? g.vh : 0);
                val = (double)site_plaquette<false>(d->links, g, eo_to_coord(g, eo, parity), eo, parity);
            }
        } else {
            const int xs = (local - d->nplaq_rounds) * 32 + lane;
            if (xs < g.vs) val = (double)site_polyakov<false>(d->links, g, xs);
        }
        val = warp_sum(val);
        if (lane == 0) bp.round_partials[mr] = val;
    }
}

// Per lattice: sums of its round partials (after a fused sweep, of its chunk
// partials of the three measuring phases) in index order -> history slot.
static __device__ void batch_measure_final(const BatchParams &bp, unsigned int slot)
{
    const int lane = threadIdx.x & 31;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int l = warp_global; l < bp.n; l += nwarps) {
        const LatDesc *d = bp.desc + l;
        const int r0 = __ldg(bp.mround_prefix + l);
        const int np = d->nplaq_rounds, nl = d->npoly_rounds;
        double sp = 0.0, sl = 0.0;
        // the partials were written by other blocks before the grid barrier and
        // not read by this one: loads through L2 (__ldcg) see them
        if (bp.fused) {
            const int c0 = __ldg(bp.chunk_prefix + l), c1 = __ldg(bp.chunk_prefix + l + 1);
            for (int k = 0; k < 3; ++k)
                for (int c = c0 + lane; c < c1; c += 32) sp += __ldcg(bp.chunk_partials + k * bp.total_chunks + c);
        } else {
            for (int r = lane; r < np; r += 32) sp += __ldcg(bp.round_partials + r0 + r);
        }
        for (int r = lane; r < nl; r += 32) sl += __ldcg(bp.round_partials + r0 + np + r);
        sp = warp_sum(sp);
        sl = warp_sum(sl);
        if (lane == 0) {
            const double vol = 2.0 * (double)d->g.vh;
            bp.history[((size_t)slot * 2 + 0) * bp.n + l] = sp / (6.0 * vol);
            bp.history[((size_t)slot * 2 + 1) * bp.n + l] = sl / (double)d->g.vs;
        }
    }
}

// The a0 sampler of a batched phase.
enum BatchSampler : int { kBatchCreutz = 0, kBatchKP = 1 };

template <int MU, int R, bool MEAS>
__device__ void batch_phase_kp(const BatchParams &bp, int parity, uint32_t sweep, CrQueues &Q, LatDesc &sd,
                               unsigned int &my_trials);

// The phase with sampler S (the other sampler's template is not instantiated).
template <int S, int MU, int R, bool MEAS>
__device__ __forceinline__ void batch_phase_s(const BatchParams &bp, int parity, uint32_t sweep, CrQueues &Q,
                                              LatDesc &sd, unsigned int &my_trials)
{
    if constexpr (S == kBatchKP)
        batch_phase_kp<MU, R, MEAS>(bp, parity, sweep, Q, sd, my_trials);
    else
        batch_phase<MU, R, MEAS>(bp, parity, sweep, Q, sd, my_trials);
}

template <int R, int T, int S>
__global__ void __launch_bounds__(T, kBatchThreadsPerSm / T) batch_sweep_kernel(const BatchParams bp)
{
    __shared__ CrQueues s_q[T / 32];
    __shared__ LatDesc s_desc[T / 32];
    const int wib = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t sweep = *(volatile unsigned int *)bp.sweep;
    const unsigned int slot = *(volatile unsigned int *)bp.meas_index;
    const bool fused = bp.fused && (int)slot < bp.history_cap;
    bool ok = true;
    if (bp.do_sweep) {
        for (int ph = 0; ph < 8 && ok; ++ph) {
            const int parity = ph & 1;
            unsigned int my_trials = 0;
            const bool meas = fused && parity == 1;
            switch (ph >> 1) {
            case 0: batch_phase_s<S, 0, R, false>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials); break;
            case 1:
                if (meas) batch_phase_s<S, 1, R, true>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                else batch_phase_s<S, 1, R, false>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                break;
            case 2:
                if (meas) batch_phase_s<S, 2, R, true>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                else batch_phase_s<S, 2, R, false>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                break;
            default:
                if (meas) batch_phase_s<S, 3, R, true>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                else batch_phase_s<S, 3, R, false>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                break;
            }
            const unsigned int wsum = __reduce_add_sync(0xffffffffu, my_trials);
            if (lane == 0 && wsum)
                atomicAdd(&bp.trial_slots[ph * kTrialSlots + (warp_global & (kTrialSlots - 1))],
                          (unsigned long long)wsum);
            ok = grid_barrier(bp.bar, bp.timeout_ns);
        }
    }
    if (ok && bp.measure && (int)slot < bp.history_cap) {
        batch_measure_rounds(bp);
        ok = grid_barrier(bp.bar, bp.timeout_ns);
        if (ok) batch_measure_final(bp, slot);
    }
    if (ok && blockIdx.x == 0 && threadIdx.x == 0) {
        if (bp.do_sweep) *bp.sweep = sweep + 1u;
        if (bp.measure) *bp.meas_index = slot + 1u;
    }
}


// Kernel entry points for the host code: the address of batch_sweep_kernel
// for sampler S, queue depth R and block size T (64, 128, 256), taken in the
// translation unit that instantiates it.  The kernels are spread over four
// units (batch_k_<sampler><depths>.cu) that compile in parallel.
template <int R, int S>
void *batch_kernel_t(int T)
{
    if (T == 64) return (void *)batch_sweep_kernel<R, 64, S>;
    if (T == 256) return (void *)batch_sweep_kernel<R, 256, S>;
    return (void *)batch_sweep_kernel<R, 128, S>;
}
void *batch_kernel_creutz_12(int R, int T);  // R = 1, 2
void *batch_kernel_creutz_48(int R, int T);  // R = 4, 8
void *batch_kernel_kp_12(int R, int T);
void *batch_kernel_kp_48(int R, int T);

}  // namespace su2
