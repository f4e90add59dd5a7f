// batch.cu -- many independent lattices (uneven Ns^3 x Nt, own beta and seed)
// swept together: one persistent cooperative launch per sweep runs the eight
// even/odd phases of every lattice (Sec. 2 update, Sec. 4 schedule) with a
// grid-wide barrier between phases, then the plaquette and Polyakov loop of
// every lattice (Sec. 4), each reduced in a fixed order.  In a measuring
// sweep the plaquette comes from the odd phases of mu = 1, 2, 3 (as in the
// single-lattice sweep) and only the Polyakov loop reads the links again.  With a user stream
// the launch is captured once into a CUDA graph and replayed per sweep.
//
// Each lattice follows exactly the single-lattice chain: same Philox
// counters (its own seed as key), same arithmetic, so its links equal those
// of su2_create + su2_heatbath_sweep with the same arguments.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

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
__device__ bool grid_barrier(BarrierState *bar, unsigned long long timeout_ns)
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
        double plaq = 0.0;

        auto push_done = [&](bool ok, float4 ut, float val, float ibk, int eo, float4 sp) {
            const unsigned int m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int q = done_n + __popc(m & lanes_below);
                Q.d_ut[q] = ut;
                Q.d_val[q] = val;
                Q.d_ibk[q] = ibk;
                Q.d_eo[q] = eo;
                if (MEAS) Q.d_sp[q] = sp;
            }
            done_n += __popc(m);
        };
        auto push_retry = [&](bool again, float4 ut, float ibk, float e, int eo, int blk, float4 sp) {
            const unsigned int m = __ballot_sync(0xffffffffu, again);
            if (again) {
                const int q = retry_n + __popc(m & lanes_below);
                Q.r_ut[q] = ut;
                Q.r_ibk[q] = ibk;
                Q.r_e[q] = e;
                Q.r_eo[q] = eo;
                Q.r_blk[q] = blk;
                if (MEAS) Q.r_sp[q] = sp;
            }
            retry_n += __popc(m);
        };
        auto direction_pass = [&](int first, int n) {
            __syncwarp();
            if (lane < n) {
                const int q = first + lane;
                const int eo = Q.d_eo[q];
                const uint4 wd = philox_key(make_uint4((uint32_t)eo, sweep, sw_dir, 0u), k0, k1);
                const float4 out = direction_update(deferred_a0(Q.d_val[q], Q.d_ibk[q]), Q.d_ut[q], wd);
                links[link_index(g, MU, parity, eo)] = out;
                if (MEAS) plaq += (double)qmul_re(out, Q.d_sp[q]);
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
            const double total = warp_sum(plaq);
            for (int c = chunk + lane; c < seg_end; c += 32)
                bp.chunk_partials[(MU - 1) * bp.total_chunks + c] = c == chunk ? total : 0.0;
        }
        chunk = seg_end;
    }
}

// Per round of 32 sites (or 32 Polyakov lines) of one lattice: the warp's
// fp64 sum of the binary32 per-site values, in a fixed order.  After a fused
// sweep only the Polyakov rounds run.
__device__ void batch_measure_rounds(const BatchParams &bp)
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
__device__ void batch_measure_final(const BatchParams &bp, unsigned int slot)
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

template <int R, int T>
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
            case 0: batch_phase<0, R, false>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials); break;
            case 1:
                if (meas) batch_phase<1, R, true>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                else batch_phase<1, R, false>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                break;
            case 2:
                if (meas) batch_phase<2, R, true>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                else batch_phase<2, R, false>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                break;
            default:
                if (meas) batch_phase<3, R, true>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
                else batch_phase<3, R, false>(bp, parity, sweep, s_q[wib], s_desc[wib], my_trials);
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

// Self-test of the barrier's timeout: `expect` arrivals are awaited but only
// gridDim.x blocks exist, so with expect > gridDim.x every wait must give up
// after timeout_ns and report it.  The arrival count is reset for the next use.
__global__ void barrier_timeout_kernel(BarrierState *bar, unsigned int expect, unsigned long long timeout_ns,
                                       unsigned int *timed_out)
{
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &bar->gen;
        const unsigned int g = *vgen;
        const unsigned int arrived = atomicAdd(&bar->count, 1u) + 1u;
        if (arrived == expect) {
            atomicAdd(&bar->gen, 1u);
        } else {
            const unsigned long long t0 = global_time_ns();
            while (*vgen == g) {
                if (global_time_ns() - t0 > timeout_ns) {
                    atomicAdd(timed_out, 1u);
                    break;
                }
                __nanosleep(1000);
            }
        }
    }
}

}  // namespace su2

using namespace su2;

struct su2_batch {
    int n = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<int> ns, nt;
    std::vector<double> beta;
    std::vector<uint64_t> seed;
    std::vector<Geom> geom;
    std::vector<size_t> link_offset;  // in float4 units
    void *block = nullptr;
    size_t block_bytes = 0;
    float4 *links = nullptr;
    size_t links_count = 0;  // float4
    LatDesc *d_desc = nullptr;
    int *d_chunk_prefix = nullptr;
    int *d_mround_prefix = nullptr;
    double *d_partials = nullptr;
    double *d_chunk_partials = nullptr;  // [3][chunks at queue depth 2, the most]
    int *d_chunk_owner = nullptr;        // [chunks at queue depth 2]
    int *d_mround_owner = nullptr;       // [total_mrounds]
    int2 *d_poly_rounds = nullptr;       // [total_poly_rounds]
    int total_poly_rounds = 0;
    BarrierState *d_bar = nullptr;
    unsigned int *d_counters = nullptr;  // [0] sweep, [1] measurement index, [2..] flags
    unsigned long long *d_trials = nullptr;
    double *d_history = nullptr;
    int history_cap = 0;
    int total_mrounds = 0;
    int total_chunks = 0;
    int R = 4;
    int threads = 128;  // block size: 64, 128 or 256
    int grid = 0;
    int max_grid[3][3] = {};  // co-resident blocks for R = 2, 4, 8 x block sizes 64, 128, 256
    uint32_t sweep = 0;
    unsigned long long timeout_ns = 2000000000ull;
    bool use_graph = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [measure]
    void *staging = nullptr;
    size_t staging_bytes = 0;
};

namespace su2 {
namespace {

int r_index(int R) { return R == 2 ? 0 : (R == 4 ? 1 : 2); }
int t_index(int T) { return T == 64 ? 0 : (T == 128 ? 1 : 2); }

template <int R>
void *kernel_for_t(int T)
{
    if (T == 64) return (void *)batch_sweep_kernel<R, 64>;
    if (T == 256) return (void *)batch_sweep_kernel<R, 256>;
    return (void *)batch_sweep_kernel<R, 128>;
}

void *kernel_for(int R, int T)
{
    if (R == 2) return kernel_for_t<2>(T);
    if (R == 8) return kernel_for_t<8>(T);
    return kernel_for_t<4>(T);
}

void drop_graphs(su2_batch *b)
{
    for (auto &g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Recomputes the heat-bath chunk table for queue depth R; block size T.
su2_status set_depth(su2_batch *b, int R, int T, int grid)
{
    std::vector<int> prefix(b->n + 1, 0);
    for (int l = 0; l < b->n; ++l) prefix[l + 1] = prefix[l] + (b->geom[l].vh + 32 * R - 1) / (32 * R);
    std::vector<int> owner(prefix[b->n]);
    for (int l = 0; l < b->n; ++l)
        for (int c = prefix[l]; c < prefix[l + 1]; ++c) owner[c] = l;
    SU2_CUDA(cudaMemcpyAsync(b->d_chunk_prefix, prefix.data(), sizeof(int) * (b->n + 1), cudaMemcpyHostToDevice,
                             b->stream));
    SU2_CUDA(cudaMemcpyAsync(b->d_chunk_owner, owner.data(), sizeof(int) * owner.size(), cudaMemcpyHostToDevice,
                             b->stream));
    SU2_CUDA(cudaStreamSynchronize(b->stream));
    b->total_chunks = prefix[b->n];
    b->R = R;
    b->threads = T;
    b->grid = grid;
    drop_graphs(b);
    return SU2_OK;
}

BatchParams params_of(const su2_batch *b, int do_sweep, int measure)
{
    BatchParams p;
    p.desc = b->d_desc;
    p.chunk_prefix = b->d_chunk_prefix;
    p.mround_prefix = b->d_mround_prefix;
    p.chunk_owner = b->d_chunk_owner;
    p.mround_owner = b->d_mround_owner;
    p.poly_rounds = b->d_poly_rounds;
    p.n = b->n;
    p.total_chunks = b->total_chunks;
    p.total_mrounds = b->total_mrounds;
    p.total_poly_rounds = b->total_poly_rounds;
    p.do_sweep = do_sweep;
    p.measure = measure;
    p.sweep = b->d_counters;
    p.meas_index = b->d_counters + 1;
    p.round_partials = b->d_partials;
    p.fused = do_sweep && measure;
    p.chunk_partials = b->d_chunk_partials;
    p.history = b->d_history;
    p.history_cap = b->history_cap;
    p.bar = b->d_bar;
    p.timeout_ns = b->timeout_ns;
    p.trial_slots = b->d_trials;
    p.flags = b->d_counters + 2;
    return p;
}

// Enqueues one launch: reset of the barrier state, then the cooperative kernel.
cudaError_t enqueue_launch(su2_batch *b, int do_sweep, int measure)
{
    cudaError_t e = cudaMemsetAsync(b->d_bar, 0, sizeof(BarrierState), b->stream);
    if (e != cudaSuccess) return e;
    BatchParams p = params_of(b, do_sweep, measure);
    void *args[] = {&p};
    return cudaLaunchCooperativeKernel(kernel_for(b->R, b->threads), dim3(b->grid), dim3(b->threads), args, 0,
                                       b->stream);
}

su2_status launch_sweep(su2_batch *b, int measure)
{
    if (b->use_graph && b->stream) {
        cudaGraphExec_t &ge = b->graph[measure];
        if (!ge) {
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t le = enqueue_launch(b, 1, measure);
                e = cudaStreamEndCapture(b->stream, &graph);
                if (le != cudaSuccess) e = le;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                // capture of cooperative launches unavailable: launch directly from now on
                cudaGetLastError();
                ge = nullptr;
                b->use_graph = false;
            }
        }
        if (ge) {
            SU2_CUDA(cudaGraphLaunch(ge, b->stream));
            return SU2_OK;
        }
    }
    SU2_CUDA(enqueue_launch(b, 1, measure));
    return SU2_OK;
}

su2_status check_flags(su2_batch *b, su2_stats *stats, uint64_t sweeps, int launches)
{
    unsigned long long slots[8 * kTrialSlots];
    unsigned int counters[4];
    BarrierState bar;
    SU2_CUDA(cudaMemcpyAsync(slots, b->d_trials, sizeof slots, cudaMemcpyDeviceToHost, b->stream));
    SU2_CUDA(cudaMemcpyAsync(counters, b->d_counters, sizeof counters, cudaMemcpyDeviceToHost, b->stream));
    SU2_CUDA(cudaMemcpyAsync(&bar, b->d_bar, sizeof bar, cudaMemcpyDeviceToHost, b->stream));
    SU2_CUDA(cudaStreamSynchronize(b->stream));
    uint64_t sites = 0;
    for (const Geom &g : b->geom) sites += 2ull * (uint64_t)g.vh;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        for (int ph = 0; ph < 8; ++ph) {
            uint64_t s = 0;
            for (int j = 0; j < kTrialSlots; ++j) s += slots[ph * kTrialSlots + j];
            stats->trials[ph] = s;
        }
        stats->sampler_failures = counters[2];
        stats->sweeps = sweeps;
        stats->link_updates = sweeps * 4ull * sites;
        stats->kernel_launches = (uint32_t)launches;
    }
    b->sweep = counters[0];
    if (bar.error & 1u) {
        set_last_error("batch sweep: a grid barrier wait timed out");
        return SU2_E_DEVICE_TIMEOUT;
    }
    if (counters[2]) {
        set_last_error("heat-bath sampler hit its trial cap");
        return SU2_E_SAMPLER;
    }
    return SU2_OK;
}

su2_status clear_stats(su2_batch *b)
{
    SU2_CUDA(cudaMemsetAsync(b->d_trials, 0, sizeof(unsigned long long) * 8 * kTrialSlots, b->stream));
    SU2_CUDA(cudaMemsetAsync(b->d_counters + 2, 0, sizeof(unsigned int) * 2, b->stream));
    return SU2_OK;
}

su2_status ensure_history(su2_batch *b, int n)
{
    if (n <= b->history_cap) return SU2_OK;
    device_free(b->d_history, sizeof(double) * 2 * b->n * (size_t)b->history_cap, b->device, b->stream);
    b->d_history = (double *)device_alloc(sizeof(double) * 2 * b->n * (size_t)n, b->device, b->stream);
    b->history_cap = b->d_history ? n : 0;
    drop_graphs(b);  // the graphs hold the old history pointer
    if (!b->d_history) {
        set_last_error("device allocation of the batch history failed");
        return SU2_E_NOMEM;
    }
    return SU2_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace su2

extern "C" {

su2_status su2_batch_create(int n, const int *ns, const int *nt, const double *beta, const uint64_t *seed,
                            su2_start start, void *cuda_stream, su2_batch **out)
{
    if (!out || !ns || !nt || !beta || !seed || n < 1) {
        set_last_error("su2_batch_create: n >= 1 and non-NULL arrays required");
        return SU2_E_INVAL;
    }
    *out = nullptr;
    if (start != SU2_COLD && start != SU2_HOT) return SU2_E_INVAL;
    for (int l = 0; l < n; ++l) {
        if (ns[l] < 2 || nt[l] < 2 || (ns[l] & 1) || (nt[l] & 1) ||
            4.0 * (double)ns[l] * ns[l] * ns[l] * nt[l] >= 2147483648.0) {
            set_last_error("su2_batch_create: extents must be even, >= 2, 4V < 2^31 (lattice " + std::to_string(l) +
                           ")");
            return SU2_E_INVAL;
        }
        if (!std::isfinite(beta[l]) || beta[l] < 0.0) {
            set_last_error("su2_batch_create: beta must be finite and >= 0 (lattice " + std::to_string(l) + ")");
            return SU2_E_INVAL;
        }
    }
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));
    int coop = 0;
    SU2_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) {
        set_last_error("device does not support cooperative launches");
        return SU2_E_CUDA;
    }
    su2_batch *b = new (std::nothrow) su2_batch();
    if (!b) return SU2_E_NOMEM;
    b->n = n;
    b->device = dev;
    b->stream = (cudaStream_t)cuda_stream;
    b->ns.assign(ns, ns + n);
    b->nt.assign(nt, nt + n);
    b->beta.assign(beta, beta + n);
    b->seed.assign(seed, seed + n);
    size_t off = 0;
    size_t max_chunks = 0;  // chunks of 64 sites (queue depth 2)
    std::vector<int> mprefix(n + 1, 0);
    for (int l = 0; l < n; ++l) {
        const Geom g = make_geom(ns[l], nt[l]);
        max_chunks += ((size_t)g.vh + 63) / 64;
        b->geom.push_back(g);
        b->link_offset.push_back(off);
        off += (8 * (size_t)g.vh + 15) & ~(size_t)15;  // keep each lattice 256-byte aligned
        const int np = (2 * g.vh + 31) / 32, nl = (g.vs + 31) / 32;
        mprefix[l + 1] = mprefix[l] + np + nl;
    }
    b->links_count = off;
    b->total_mrounds = mprefix[n];
    const size_t links_bytes = align256(sizeof(float4) * off);
    const size_t desc_bytes = align256(sizeof(LatDesc) * n);
    const size_t prefix_bytes = align256(sizeof(int) * (n + 1));
    const size_t partial_bytes = align256(sizeof(double) * b->total_mrounds);
    const size_t chunk_bytes = align256(sizeof(double) * 3 * max_chunks);
    std::vector<int> mowner(b->total_mrounds);
    std::vector<int2> poly_rounds;
    for (int l = 0; l < n; ++l) {
        const int np = (2 * b->geom[l].vh + 31) / 32;
        for (int r = mprefix[l]; r < mprefix[l + 1]; ++r) {
            mowner[r] = l;
            if (r - mprefix[l] >= np) poly_rounds.push_back(make_int2(r, l));
        }
    }
    b->total_poly_rounds = (int)poly_rounds.size();
    const size_t owner_bytes = align256(sizeof(int) * max_chunks) + align256(sizeof(int) * b->total_mrounds) +
                               align256(sizeof(int2) * poly_rounds.size());
    const size_t bar_bytes = align256(sizeof(BarrierState));
    const size_t counter_bytes = align256(sizeof(unsigned int) * 8);
    const size_t trial_bytes = align256(sizeof(unsigned long long) * 8 * kTrialSlots);
    b->block_bytes = links_bytes + desc_bytes + 2 * prefix_bytes + partial_bytes + chunk_bytes + owner_bytes +
                     bar_bytes + counter_bytes + trial_bytes;
    b->block = device_alloc(b->block_bytes, dev, b->stream);
    if (!b->block) {
        delete b;
        set_last_error("device allocation of the batch failed");
        return SU2_E_NOMEM;
    }
    char *p = (char *)b->block;
    b->links = (float4 *)p;
    p += links_bytes;
    b->d_desc = (LatDesc *)p;
    p += desc_bytes;
    b->d_chunk_prefix = (int *)p;
    p += prefix_bytes;
    b->d_mround_prefix = (int *)p;
    p += prefix_bytes;
    b->d_partials = (double *)p;
    p += partial_bytes;
    b->d_chunk_partials = (double *)p;
    p += chunk_bytes;
    b->d_chunk_owner = (int *)p;
    p += align256(sizeof(int) * max_chunks);
    b->d_mround_owner = (int *)p;
    p += align256(sizeof(int) * b->total_mrounds);
    b->d_poly_rounds = (int2 *)p;
    p += align256(sizeof(int2) * poly_rounds.size());
    b->d_bar = (BarrierState *)p;
    p += bar_bytes;
    b->d_counters = (unsigned int *)p;
    p += counter_bytes;
    b->d_trials = (unsigned long long *)p;

    std::vector<LatDesc> desc(n);
    for (int l = 0; l < n; ++l) {
        desc[l].g = b->geom[l];
        desc[l].links = b->links + b->link_offset[l];
        desc[l].k0 = (uint32_t)seed[l];
        desc[l].k1 = (uint32_t)(seed[l] >> 32);
        desc[l].beta = (float)beta[l];
        desc[l].nplaq_rounds = (2 * b->geom[l].vh + 31) / 32;
        desc[l].npoly_rounds = (b->geom[l].vs + 31) / 32;
    }
    su2_status st = SU2_OK;
    cudaError_t e = cudaMemcpyAsync(b->d_desc, desc.data(), sizeof(LatDesc) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_mround_prefix, mprefix.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_mround_owner, mowner.data(), sizeof(int) * mowner.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess && !poly_rounds.empty())
        e = cudaMemcpyAsync(b->d_poly_rounds, poly_rounds.data(), sizeof(int2) * poly_rounds.size(),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_bar, 0, bar_bytes + counter_bytes + trial_bytes, b->stream);
    for (int l = 0; l < n && e == cudaSuccess; ++l)
        e = start_links(b->links + b->link_offset[l], b->geom[l], start == SU2_HOT, seed[l], b->d_counters + 2,
                        b->stream);  // the hot-start kernel counts failures in flags[1] = counter 3
    if (e == cudaSuccess) {
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        for (int i = 0; i < 3 && e == cudaSuccess; ++i)
            for (int j = 0; j < 3 && e == cudaSuccess; ++j) {
                const int R = i == 0 ? 2 : (i == 1 ? 4 : 8);
                int per_sm = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(R, kBatchBlockSizes[j]),
                                                                  kBatchBlockSizes[j], 0);
                b->max_grid[i][j] = std::max(1, per_sm * sms);
            }
    }
    if (e != cudaSuccess) st = cuda_fail(e, "su2_batch_create");
    if (st == SU2_OK) st = set_depth(b, 4, 128, b->max_grid[r_index(4)][t_index(128)]);
    if (st == SU2_OK) {
        unsigned int c[4];
        if (cudaMemcpyAsync(c, b->d_counters, sizeof c, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "su2_batch_create");
        else if (c[3]) {
            set_last_error("hot start: a link found no two disk points in 64 pairs");
            st = SU2_E_SAMPLER;
        }
    }
    if (st != SU2_OK) {
        su2_batch_destroy(b);
        return st;
    }
    *out = b;
    return SU2_OK;
}

su2_status su2_batch_destroy(su2_batch *b)
{
    if (!b) return SU2_OK;
    DeviceGuard guard(b->device);
    drop_graphs(b);
    device_free(b->staging, b->staging_bytes, b->device, b->stream);
    device_free(b->d_history, sizeof(double) * 2 * b->n * (size_t)b->history_cap, b->device, b->stream);
    device_free(b->block, b->block_bytes, b->device, b->stream);
    const cudaError_t e = cudaStreamSynchronize(b->stream);
    delete b;
    if (e != cudaSuccess) return cuda_fail(e, "su2_batch_destroy");
    return SU2_OK;
}

su2_status su2_batch_generate(su2_batch *b, int nsweeps, int measure_every, double *plaq, double *poly,
                              su2_stats *stats)
{
    if (!b || nsweeps < 0 || measure_every < 0) return SU2_E_INVAL;
    DeviceGuard guard(b->device);
    const int nmeas = measure_every > 0 ? nsweeps / measure_every : 0;
    su2_status st = ensure_history(b, std::max(nmeas, 1));
    if (st != SU2_OK) return st;
    if ((st = clear_stats(b)) != SU2_OK) return st;
    SU2_CUDA(cudaMemsetAsync(b->d_counters + 1, 0, sizeof(unsigned int), b->stream));
    for (int s = 1; s <= nsweeps; ++s) {
        const int measure = (measure_every > 0 && s % measure_every == 0) ? 1 : 0;
        if ((st = launch_sweep(b, measure)) != SU2_OK) return st;
    }
    st = check_flags(b, stats, (uint64_t)nsweeps, nsweeps);
    if (nmeas > 0 && (plaq || poly)) {
        std::vector<double> h((size_t)nmeas * 2 * b->n);
        SU2_CUDA(cudaMemcpyAsync(h.data(), b->d_history, sizeof(double) * h.size(), cudaMemcpyDeviceToHost,
                                 b->stream));
        SU2_CUDA(cudaStreamSynchronize(b->stream));
        for (int m = 0; m < nmeas; ++m)
            for (int l = 0; l < b->n; ++l) {
                if (plaq) plaq[(size_t)m * b->n + l] = h[((size_t)m * 2 + 0) * b->n + l];
                if (poly) poly[(size_t)m * b->n + l] = h[((size_t)m * 2 + 1) * b->n + l];
            }
    }
    return st;
}

su2_status su2_batch_sweep(su2_batch *b, int nsweeps, su2_stats *stats)
{
    return su2_batch_generate(b, nsweeps, 0, nullptr, nullptr, stats);
}

su2_status su2_batch_measure(su2_batch *b, double *plaq, double *poly)
{
    if (!b || (!plaq && !poly)) return SU2_E_INVAL;
    DeviceGuard guard(b->device);
    su2_status st = ensure_history(b, 1);
    if (st != SU2_OK) return st;
    SU2_CUDA(cudaMemsetAsync(b->d_counters + 1, 0, sizeof(unsigned int), b->stream));
    SU2_CUDA(enqueue_launch(b, 0, 1));
    std::vector<double> h(2 * (size_t)b->n);
    SU2_CUDA(cudaMemcpyAsync(h.data(), b->d_history, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, b->stream));
    BarrierState bar;
    SU2_CUDA(cudaMemcpyAsync(&bar, b->d_bar, sizeof bar, cudaMemcpyDeviceToHost, b->stream));
    SU2_CUDA(cudaStreamSynchronize(b->stream));
    if (bar.error & 1u) {
        set_last_error("batch measurement: a grid barrier wait timed out");
        return SU2_E_DEVICE_TIMEOUT;
    }
    for (int l = 0; l < b->n; ++l) {
        if (plaq) plaq[l] = h[l];
        if (poly) poly[l] = h[b->n + l];
    }
    return SU2_OK;
}

su2_status su2_batch_plaquette(su2_batch *b, double *out_n) { return su2_batch_measure(b, out_n, nullptr); }

su2_status su2_batch_polyakov(su2_batch *b, double *out_n) { return su2_batch_measure(b, nullptr, out_n); }

su2_status su2_batch_get_links(su2_batch *b, int i, float *host)
{
    if (!b || !host || i < 0 || i >= b->n) return SU2_E_INVAL;
    DeviceGuard guard(b->device);
    const Geom &g = b->geom[i];
    const size_t need = sizeof(float4) * 8 * (size_t)g.vh;
    if (!b->staging || b->staging_bytes < need) {
        device_free(b->staging, b->staging_bytes, b->device, b->stream);
        size_t most = 0;
        for (const Geom &x : b->geom) most = std::max(most, sizeof(float4) * 8 * (size_t)x.vh);
        b->staging = device_alloc(most, b->device, b->stream);
        b->staging_bytes = b->staging ? most : 0;
        if (!b->staging) return SU2_E_NOMEM;
    }
    SU2_CUDA(convert_links(b->links + b->link_offset[i], (float4 *)b->staging, g, true, b->stream));
    SU2_CUDA(cudaMemcpyAsync(host, b->staging, need, cudaMemcpyDeviceToHost, b->stream));
    SU2_CUDA(cudaStreamSynchronize(b->stream));
    return SU2_OK;
}

su2_status su2_batch_info(su2_batch *b, int *n, uint32_t *sweep, int *queue_depth, int *grid, int *graphs)
{
    if (!b) return SU2_E_INVAL;
    if (n) *n = b->n;
    if (sweep) *sweep = b->sweep;
    if (queue_depth) *queue_depth = b->R;
    if (grid) *grid = b->grid;
    if (graphs) *graphs = (b->use_graph && b->stream) ? 1 : 0;
    return SU2_OK;
}

su2_status su2_batch_set_launch(su2_batch *b, int queue_depth, int threads, int grid)
{
    if (!b || (queue_depth != 2 && queue_depth != 4 && queue_depth != 8) ||
        (threads != 64 && threads != 128 && threads != 256))
        return SU2_E_INVAL;
    const int most = b->max_grid[r_index(queue_depth)][t_index(threads)];
    if (grid <= 0 || grid > most) grid = most;
    DeviceGuard guard(b->device);
    return set_depth(b, queue_depth, threads, grid);
}

su2_status su2_batch_set_config(su2_batch *b, int queue_depth, int grid)
{
    if (!b) return SU2_E_INVAL;
    return su2_batch_set_launch(b, queue_depth, b->threads, grid);
}

su2_status su2_batch_launch_info(su2_batch *b, int *queue_depth, int *threads, int *grid)
{
    if (!b) return SU2_E_INVAL;
    if (queue_depth) *queue_depth = b->R;
    if (threads) *threads = b->threads;
    if (grid) *grid = b->grid;
    return SU2_OK;
}

// Times each candidate (queue depth 2/4/8 x block size 64/128/256 x full or
// half of the co-resident grid) over `sweeps` sweeps of the batch, then
// restores the links and the sweep counter, and keeps the fastest.
su2_status su2_batch_autotune(su2_batch *b, int sweeps, int *queue_depth, int *grid)
{
    if (!b || sweeps < 1) return SU2_E_INVAL;
    DeviceGuard guard(b->device);
    const size_t bytes = sizeof(float4) * b->links_count;
    void *saved = device_alloc(bytes, b->device, b->stream);
    if (!saved) return SU2_E_NOMEM;
    su2_status st = SU2_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float best = 1e30f;
    int best_r = b->R, best_t = b->threads, best_grid = b->grid;
    const uint32_t sweep0 = b->sweep;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMemcpyAsync(saved, b->links, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "su2_batch_autotune");
    const int depths[3] = {2, 4, 8};
    for (int c = 0; c < 18 && st == SU2_OK; ++c) {
            const int i = c / 6, j = (c / 2) % 3, half = c % 2;
            const int R = depths[i], T = kBatchBlockSizes[j];
            const int grid = half ? std::max(1, b->max_grid[i][j] / 2) : b->max_grid[i][j];
            if ((st = set_depth(b, R, T, grid)) != SU2_OK) break;
            if ((st = launch_sweep(b, 0)) != SU2_OK) break;  // warm-up (and graph capture)
            cudaEventRecord(e0, b->stream);
            for (int s = 0; s < sweeps && st == SU2_OK; ++s) st = launch_sweep(b, 0);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = cuda_fail(cudaGetLastError(), "su2_batch_autotune");
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_r = R;
                best_t = T;
                best_grid = grid;
            }
            // restore the configuration the candidates started from
            if (cudaMemcpyAsync(b->links, saved, bytes, cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess ||
                cudaMemcpyAsync(b->d_counters, &sweep0, sizeof sweep0, cudaMemcpyHostToDevice, b->stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(b->stream) != cudaSuccess) {
                st = cuda_fail(cudaGetLastError(), "su2_batch_autotune");
                break;
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    device_free(saved, bytes, b->device, b->stream);
    cudaStreamSynchronize(b->stream);
    b->sweep = sweep0;
    if (st == SU2_OK) st = set_depth(b, best_r, best_t, best_grid);
    if (st == SU2_OK) st = clear_stats(b);
    if (queue_depth) *queue_depth = b->R;
    if (grid) *grid = b->grid;
    return st;
}

su2_status su2_selftest_barrier_timeout(int blocks, uint64_t timeout_ns, unsigned int *timed_out)
{
    if (blocks < 1 || blocks > 1024 || !timed_out || timeout_ns > 5000000000ull) return SU2_E_INVAL;
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));
    const size_t bytes = 256 + sizeof(unsigned int);
    char *buf = (char *)device_alloc(bytes, dev, nullptr);
    if (!buf) return SU2_E_NOMEM;
    su2_status st = SU2_OK;
    BarrierState *bar = (BarrierState *)buf;
    unsigned int *count = (unsigned int *)(buf + 256);
    if (cudaMemsetAsync(buf, 0, bytes, nullptr) != cudaSuccess) st = cuda_fail(cudaGetLastError(), "memset");
    if (st == SU2_OK) {
        // one more arrival is expected than there are blocks: nothing completes the barrier
        barrier_timeout_kernel<<<blocks, 32>>>(bar, (unsigned int)blocks + 1u, timeout_ns, count);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(timed_out, count, sizeof(unsigned int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "barrier self-test");
    }
    device_free(buf, bytes, dev, nullptr);
    cudaStreamSynchronize(nullptr);
    return st;
}

}  // extern "C"
