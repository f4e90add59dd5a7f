// learned.cu -- the learned a0 proposal on the lattice: the proposal table
// (the network evaluated in binary32 registers at grid points of beta k),
// the independence-Metropolis phase kernel, the plain heat bath as fallback
// (a sweep whose acceptance falls below a threshold is followed by a plain
// sweep), and the collection of (beta k, a0) training pairs from fresh
// Creutz draws (Sec. 2 sampler) on the current configuration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "learned.cuh"
#include "observables.cuh"
#include "staple.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"
#include "tc05.cuh"

namespace su2 {

// One block of 768 threads per SM: the proposal table's row pairs (55 KB at
// 256 rows) are staged in shared memory once per SM rather than once per
// block, which leaves the rest to L1 (three 256-thread blocks: 93.7 us per
// phase at 48^4; one of 768: 87.0 us).
constexpr int kLearnThreads = 768;
#ifndef SU2_LEARN_MIN_BLOCKS
#define SU2_LEARN_MIN_BLOCKS 1
#endif
constexpr int kLearnMinBlocks = SU2_LEARN_MIN_BLOCKS;  // blocks per SM the register budget is set for
constexpr int kAcceptSlots = 64;
constexpr uint32_t kTableWaitPolls = 1u << 24;  // polls of the table copy's mbarrier before a block gives up

// Row pairs (r_j, r_{j+1} - r_j) of the table, the form the phase kernel
// interpolates from (one 8-byte load and one fused multiply-add per
// parameter); the tail up to a multiple of 16 bytes is zero.
__global__ void proposal_pairs_kernel(const float *__restrict__ table, int n_pairs, int n_padded,
                                      float2 *__restrict__ pairs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_padded) return;
    if (i < n_pairs) {
        const float r0 = table[i];
        pairs[i] = make_float2(r0, __fsub_rn(table[i + learned::kParams], r0));
    } else {
        pairs[i] = make_float2(0.0f, 0.0f);
    }
}

__global__ void proposal_table_kernel(const float *__restrict__ w, float s_lo, float s_hi, int G,
                                      float *__restrict__ table)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= G) return;
    const float ds = __fdiv_rn(__fsub_rn(s_hi, s_lo), (float)(G - 1));
    float o[learned::kOut];
    learned::mlp_forward(w, __fmaf_rn((float)j, ds, s_lo), o);
    learned::spline_params(o, table + j * learned::kParams);
}

struct LearnedParams {
    float4 *links;
    const float2 *pairs;               // the proposal table's row pairs (global, 16-byte aligned)
    unsigned int pair_bytes;           // their size, a multiple of 16 bytes
    unsigned int *flags;               // [2]: a block gave up waiting for the table copy
    const uint32_t *sweep_dev;         // if non-NULL the sweep counter is read here (graph replays)
    Geom g;
    RoundKeys rk;
    int parity;
    float beta;
    uint32_t sweep;
    const float *table;
    int G;
    float s_lo, s_hi, mean, scale;
    const unsigned int *gate;          // runs only while *gate == 1
    unsigned long long *acc_slots;     // [8][64]: accepted links per phase (call total)
    unsigned long long *sweep_slots;   // [64]: accepted links of this sweep
    double *plaq;                      // measuring phases: block partials of the plaquettes of planes (nu < mu, mu)
    const float4 *same[4];             // links of direction d at the phase's parity
    const float4 *other[4];            // ... at the opposite parity
};

__device__ __forceinline__ unsigned int block_sum_u32(unsigned int v)
{
    __shared__ unsigned int warp_sums[32];
    const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    v = __reduce_add_sync(0xffffffffu, v);
    if (lane == 0) warp_sums[warp] = v;
    __syncthreads();
    unsigned int total = 0;
    if (warp == 0) {
        total = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0u;
        total = __reduce_add_sync(0xffffffffu, total);
    }
    return total;
}

// One learned phase (MU, parity).  Persistent grid: each thread walks the
// links i, i + T, i + 2T, ... (T threads in the grid).  Each loop iteration
// (three per link) issues the six loads of one nu-group of the next link, does
// one third of the current link's step, then folds the loaded group into the
// next link's staple:
//   part 0  the Philox block, k, U~^dag, the table row, a0' = f(2 u0 - 1);
//   part 1  a_cur, f^-1(a_cur), the Metropolis test;
//   part 2  the direction and the store.
// MEAS: the plaquette contributions (1/2) Tr U'S of the final link (new or
// kept), S the staple terms of nu < MU, as in the heat-bath kernels.
template <int MU, bool MEAS>
__global__ void __launch_bounds__(kLearnThreads, kLearnMinBlocks) learned_phase_kernel(const LearnedParams p)
{
    extern __shared__ __align__(16) float2 s_pairs[];
    __shared__ __align__(8) uint64_t s_bar;
    if (*(volatile const unsigned int *)p.gate != 1u) return;
    // The table's row pairs come in by one bulk copy (the TMA engine) that
    // completes on an mbarrier, while the threads load their first staple.
    if (threadIdx.x == 0) {
        tc::mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(&s_bar)),
                     "r"(p.pair_bytes)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         tc::smem_addr(s_pairs)),
                     "l"(p.pairs), "r"(p.pair_bytes), "r"(tc::smem_addr(&s_bar))
                     : "memory");
    }
    __syncthreads();  // the barrier is initialised before anyone waits on it
    const learned::Proposal pr{s_pairs, p.G, p.s_lo, learned::table_inv_ds(p.G, p.s_lo, p.s_hi), p.mean, p.scale};
    const int stride = gridDim.x * blockDim.x;
    const uint32_t sweep = p.sweep_dev ? *p.sweep_dev : p.sweep;
    const uint32_t sw = stream_word(kLearned, (uint32_t)p.parity, MU);
    const int last = p.g.vh - 1;
    // Lanes past the end work on a clamped index and drop their results, so
    // the loop body has no divergent branch.
    int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    int cur = base + (threadIdx.x & 31);
    unsigned int acc = 0;
    float plaq = 0.0f;  // per-thread partial in binary32; the block and grid sums are binary64
    float4 v_cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float4 sp_cur = v_cur;  // MEAS: staple terms of nu < MU (the first MU groups)
    if (base < p.g.vh) {
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
    // Thread 0 waits for the table (bounded); a block whose wait gives up
    // flags it, waits once more (bounded) for its copy still in flight, and
    // leaves its links unchanged.  The others then observe the completed
    // phase themselves, which makes the copied bytes visible to them.
    __shared__ int s_table_ok;
    if (threadIdx.x == 0) {
        const bool ok = tc::mbar_wait(&s_bar, 0, kTableWaitPolls);
        if (!ok) {
            atomicAdd(&p.flags[2], 1u);
            tc::mbar_wait(&s_bar, 0, kTableWaitPolls);
        }
        s_table_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_table_ok) return;  // block-uniform
    tc::mbar_wait(&s_bar, 0, kTableWaitPolls);
    while (base < p.g.vh) {  // warp-uniform
        const bool valid = cur <= last;
        const int nxt = cur + stride;
        const int en = min(nxt, last);
        const Coord xn = eo_to_coord(p.g, en, p.parity);
        const int en_p = eo_fwd<MU>(p.g, xn, en);
        // ---- part 0
        NuLinks nl = load_nu_bases<MU, OtherDir<MU, 0>::value>(p.same, p.other, p.g, xn, en, en_p);
        const uint32_t li = link_index(p.g, MU, p.parity, min(cur, last));
        const float4 old = p.links[li];
        const uint4 w = philox_rk(make_uint4((uint32_t)cur, sweep, sw, 0u), p.rk);
        const learned::LearnedDraw r = learned::learned_propose(pr, p.beta, v_cur, uniform01(w.x));
        float4 v_next = add_nu_terms(make_float4(0.0f, 0.0f, 0.0f, 0.0f), nl);
        float4 sp_next = v_next;
        // ---- part 1
        nl = load_nu_bases<MU, OtherDir<MU, 1>::value>(p.same, p.other, p.g, xn, en, en_p);
        const bool ok = learned::learned_accept(r, old, uniform01(w.y), valid);
        const bool accept = valid && ok;
        v_next = add_nu_terms(v_next, nl);
        if (MU == 2) sp_next = v_next;
        // ---- part 2
        nl = load_nu_bases<MU, OtherDir<MU, 2>::value>(p.same, p.other, p.g, xn, en, en_p);
        const float4 out = direction_from_uniforms(r.a_new, r.d.ut, uniform01(w.z), uniform01(w.w));
        if (accept) p.links[li] = out;
        if (MEAS && valid) plaq = __fadd_rn(plaq, qmul_re(accept ? out : old, sp_cur));
        acc += accept ? 1u : 0u;
        v_next = add_nu_terms(v_next, nl);
        if (MU == 3) sp_next = v_next;
        base += stride;
        cur = nxt;
        v_cur = v_next;
        sp_cur = sp_next;
    }
    const unsigned int total = block_sum_u32(acc);
    if (threadIdx.x == 0 && total) {
        atomicAdd(&p.acc_slots[(2 * MU + p.parity) * kAcceptSlots + (blockIdx.x & (kAcceptSlots - 1))],
                  (unsigned long long)total);
        atomicAdd(&p.sweep_slots[blockIdx.x & (kAcceptSlots - 1)], (unsigned long long)total);
    }
    if (MEAS) {
        __syncthreads();
        const double ptotal = block_sum((double)plaq);
        if (threadIdx.x == 0) p.plaq[blockIdx.x] = ptotal;
    }
}

// End of a sweep: after a learned sweep whose acceptance is below the
// threshold, the next sweep is plain; after a plain sweep, learned again.
__global__ void learned_decide_kernel(unsigned int *ctl, unsigned long long *sweep_slots, double links,
                                      double min_acceptance)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    unsigned long long acc = 0;
    for (int j = 0; j < kAcceptSlots; ++j) {
        acc += sweep_slots[j];
        sweep_slots[j] = 0ull;
    }
    if (ctl[0] == 1u) {
        ctl[2] += 1u;
        ctl[0] = ((double)acc < min_acceptance * links) ? 0u : 1u;
    } else {
        ctl[1] += 1u;
        ctl[0] = 1u;
    }
}

// One (beta k, a0) pair per link U_mu(x) of parity p with even/odd index a
// multiple of `stride`: a0 is a Creutz draw on the collection stream (trial t
// uses words 2(t&1), 2(t&1)+1 of block t>>1), so the pair has the exact
// conditional law without touching the chain.
template <int MU>
__global__ void __launch_bounds__(kLearnThreads) collect_kernel(const float4 *__restrict__ links, Geom g, int parity,
                                                                 RoundKeys rk, float beta, uint32_t sweep, int stride,
                                                                 float2 *__restrict__ pairs, int n_pairs)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_pairs) return;
    const int eo = q * stride;
    const Coord x = eo_to_coord(g, eo, parity);
    const DrawSetup d = prepare_draw(staple_at<MU>(links, g, x, parity), beta);
    const bool haar = d.bk < kHaarBelow;
    const float ome = __fsub_rn(1.0f, d.e);
    float a0 = 0.0f;
    const uint32_t sw = stream_word(4u, (uint32_t)parity, MU);
    for (int b = 0; b < kMaxTrials / 2; ++b) {
        const uint4 w = philox_rk(make_uint4((uint32_t)eo, sweep, sw, (uint32_t)b), rk);
        float cand;
        if (creutz_trial(uniform_log(w.x), uniform01(w.y), d.ibk, d.e, ome, haar, cand)) {
            a0 = cand;
            break;
        }
        if (creutz_trial(uniform_log(w.z), uniform01(w.w), d.ibk, d.e, ome, haar, cand)) {
            a0 = cand;
            break;
        }
    }
    pairs[q] = make_float2(d.bk, a0);
}

// Grid of all co-resident blocks (at most `want`), for the kernels that walk
// their links in a loop.
template <typename Kernel>
static cudaError_t launch_persistent(Kernel kernel, const LearnedParams &p, int want, size_t smem, su2_lattice *lat)
{
    int per_sm = 0, sms = 0;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kLearnThreads, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, lat->device);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(std::min(want, std::max(1, per_sm) * sms), kFusedSlots));
    kernel<<<grid, kLearnThreads, smem, lat->stream>>>(p);
    return cudaGetLastError();
}

// Bytes of the row pairs of a G-row table, rounded up to 16 (a bulk copy
// moves a multiple of 16 bytes).
static size_t pair_bytes_of(int G) { return (sizeof(float2) * (size_t)(G - 1) * learned::kParams + 15) & ~(size_t)15; }

static su2_status launch_learned_phase(su2_lattice *lat, int mu, int parity)
{
    LearnedParams p;
    p.links = lat->links;
    p.g = geom_of(lat);
    p.rk = make_round_keys(lat->seed);
    p.parity = parity;
    p.beta = (float)lat->beta;
    p.sweep = lat->sweep;
    p.sweep_dev = lat->capturing ? lat->d_ctr : nullptr;
    p.table = lat->proposal;
    p.pairs = lat->proposal_pairs;
    p.flags = lat->scratch.flags;
    p.G = lat->proposal_g;
    p.s_lo = lat->prop_s_lo;
    p.s_hi = lat->prop_s_hi;
    p.mean = lat->prop_mean;
    p.scale = lat->prop_scale;
    p.gate = lat->learned_ctl;
    p.acc_slots = lat->accept_slots;
    p.sweep_slots = lat->accept_slots + 8 * kAcceptSlots;
    p.plaq = fused_slot(lat, mu, parity, 1);
    set_bases(p.same, p.other, lat, parity);
    p.pair_bytes = (unsigned int)pair_bytes_of(p.G);
    const size_t smem = p.pair_bytes;
    const int want = (p.g.vh + kLearnThreads - 1) / kLearnThreads;
    cudaError_t e;
    if (p.plaq) {
        switch (mu) {
        case 1: e = launch_persistent(learned_phase_kernel<1, true>, p, want, smem, lat); break;
        case 2: e = launch_persistent(learned_phase_kernel<2, true>, p, want, smem, lat); break;
        default: e = launch_persistent(learned_phase_kernel<3, true>, p, want, smem, lat); break;
        }
    } else {
        switch (mu) {
        case 0: e = launch_persistent(learned_phase_kernel<0, false>, p, want, smem, lat); break;
        case 1: e = launch_persistent(learned_phase_kernel<1, false>, p, want, smem, lat); break;
        case 2: e = launch_persistent(learned_phase_kernel<2, false>, p, want, smem, lat); break;
        default: e = launch_persistent(learned_phase_kernel<3, false>, p, want, smem, lat); break;
        }
    }
    SU2_CUDA(e);
    return SU2_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// An mbarrier that expects one arrival which never comes: the bounded wait
// must give up (the table wait of learned_phase_kernel, made to run out).
__global__ void mbar_timeout_kernel(uint32_t polls, unsigned int *timed_out)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!tc::mbar_wait(&bar, 0, polls)) atomicAdd(timed_out, 1u);
}

// One learned sweep: the eight learned phases, each followed by the plain
// phase gated off while the sweep is learned (it runs when the previous
// sweep's acceptance fell below min_acceptance), the fallback decision, and
// the measurement if due (plaq_dst / poly_dst: the slots, or when capturing
// the bases to which the kernels add the device slot index).
static su2_status learned_sweep_body(su2_lattice *lat, bool measure, double min_acceptance, double *plaq_dst,
                                     double *poly_dst)
{
    su2_status st;
    if (measure && (st = fused_begin(lat)) != SU2_OK) return st;
    for (int mu = 0; mu < 4; ++mu)
        for (int parity = 0; parity < 2; ++parity) {
            if ((st = timing_begin(lat, lat->hb_log)) == SU2_OK) st = launch_learned_phase(lat, mu, parity);
            if (st == SU2_OK) st = timing_end(lat, lat->hb_log);
            if (st == SU2_OK) st = launch_hb_phase(lat, mu, parity, lat->sweep, lat->learned_ctl);
            if (st != SU2_OK) {
                lat->fused_part = nullptr;
                return st;
            }
        }
    learned_decide_kernel<<<1, 32, 0, lat->stream>>>(lat->learned_ctl, lat->accept_slots + 8 * kAcceptSlots,
                                                     4.0 * (double)lat->vol, min_acceptance);
    SU2_CUDA(cudaGetLastError());
    if (measure) return fused_finish_with_polyakov(lat, plaq_dst, poly_dst);
    return SU2_OK;
}

// The captured learned sweep of this variant (captured on first use or after
// a settings change); *exec = NULL if the stream refused the capture.
static su2_status learned_graph(su2_lattice *lat, bool measure, double min_acceptance, cudaGraphExec_t *exec)
{
    GenGraph &gg = lat->learned_graph[measure ? 1 : 0];
    uint64_t sig = generation_signature(lat);
    auto mix = [&](uint64_t v) {
        for (int i = 0; i < 8; ++i) {
            sig ^= (v >> (8 * i)) & 0xffu;
            sig *= 1099511628211ull;
        }
    };
    uint32_t b[5];
    memcpy(&b[0], &lat->prop_s_lo, 4);
    memcpy(&b[1], &lat->prop_s_hi, 4);
    memcpy(&b[2], &lat->prop_mean, 4);
    memcpy(&b[3], &lat->prop_scale, 4);
    b[4] = (uint32_t)lat->proposal_g;
    for (uint32_t x : b) mix(x);
    uint64_t ma;
    memcpy(&ma, &min_acceptance, 8);
    mix(ma);
    sig |= 1ull;
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
    lat->capturing = true;
    su2_status st = learned_sweep_body(lat, measure, min_acceptance, lat->scratch.history,
                                       lat->scratch.history + lat->scratch.history_cap);
    if (st == SU2_OK) st = enqueue_advance(lat, measure);
    lat->capturing = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(lat->stream, &graph);
    if (st != SU2_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        lat->graphs_off = true;
        return st == SU2_E_CUDA ? SU2_OK : st;
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

}  // namespace su2

using namespace su2;

extern "C" {

su2_status su2_set_proposal(su2_lattice *lat, const float *weights, int n, double s_lo, double s_hi, int grid_points)
{
    if (!lat || !weights || n != learned::kWeights || grid_points < 2 || grid_points > 400 || !(s_hi > s_lo) ||
        !std::isfinite(s_lo) || !std::isfinite(s_hi)) {
        set_last_error("su2_set_proposal: 1947 weights, 2 <= grid_points <= 400, finite s_lo < s_hi");
        return SU2_E_INVAL;
    }
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(weights[i])) {
            set_last_error("su2_set_proposal: non-finite weight");
            return SU2_E_NUMERIC;
        }
    DeviceGuard guard(lat->device);
    const size_t table_bytes = align256(sizeof(float) * learned::kParams * 400);
    const size_t w_bytes = align256(sizeof(float) * learned::kWeights);
    const size_t ctl_bytes = align256(sizeof(unsigned int) * 4);
    const size_t slot_bytes = align256(sizeof(unsigned long long) * 9 * kAcceptSlots);
    const size_t pairs_bytes = align256(pair_bytes_of(400));
    if (!lat->learned_block) {
        lat->learned_bytes = table_bytes + w_bytes + ctl_bytes + slot_bytes + pairs_bytes;
        lat->learned_block = device_alloc(lat->learned_bytes, lat->device, lat->stream);
        if (!lat->learned_block) {
            set_last_error("device allocation of the learned proposal failed");
            return SU2_E_NOMEM;
        }
        char *q = (char *)lat->learned_block;
        lat->proposal = (float *)q;
        lat->learned_ctl = (unsigned int *)(q + table_bytes + w_bytes);
        lat->accept_slots = (unsigned long long *)(q + table_bytes + w_bytes + ctl_bytes);
        lat->proposal_pairs = (float2 *)(q + table_bytes + w_bytes + ctl_bytes + slot_bytes);
        SU2_CUDA(cudaMemsetAsync(lat->learned_ctl, 0, ctl_bytes + slot_bytes, lat->stream));
    }
    float *d_w = (float *)((char *)lat->learned_block + table_bytes);
    SU2_CUDA(cudaMemcpyAsync(d_w, weights, sizeof(float) * learned::kWeights, cudaMemcpyHostToDevice, lat->stream));
    proposal_table_kernel<<<(grid_points + 63) / 64, 64, 0, lat->stream>>>(d_w, (float)s_lo, (float)s_hi, grid_points,
                                                                         lat->proposal);
    SU2_CUDA(cudaGetLastError());
    const int n_pairs = (grid_points - 1) * learned::kParams;
    const int n_padded = (int)(pair_bytes_of(grid_points) / sizeof(float2));
    proposal_pairs_kernel<<<(n_padded + 255) / 256, 256, 0, lat->stream>>>(lat->proposal, n_pairs, n_padded,
                                                                          lat->proposal_pairs);
    SU2_CUDA(cudaGetLastError());
    SU2_CUDA(cudaStreamSynchronize(lat->stream));
    lat->proposal_g = grid_points;
    lat->prop_s_lo = (float)s_lo;
    lat->prop_s_hi = (float)s_hi;
    lat->prop_mean = weights[learned::kOffMean];
    lat->prop_scale = weights[learned::kOffScale];
    return SU2_OK;
}

su2_status su2_selftest_mbar_timeout(int blocks, unsigned int polls, unsigned int *timed_out)
{
    if (blocks < 1 || blocks > 1024 || polls < 1 || polls > (1u << 24) || !timed_out) return SU2_E_INVAL;
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));
    unsigned int *d = (unsigned int *)device_alloc(sizeof(unsigned int), dev, nullptr);
    if (!d) return SU2_E_NOMEM;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned int), nullptr);
    if (e == cudaSuccess) {
        mbar_timeout_kernel<<<blocks, 32>>>(polls, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(timed_out, d, sizeof(unsigned int), cudaMemcpyDeviceToHost);
    device_free(d, sizeof(unsigned int), dev, nullptr);
    cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "su2_selftest_mbar_timeout");
    return SU2_OK;
}

su2_status su2_get_proposal_table(su2_lattice *lat, float *host)
{
    if (!lat || !host) return SU2_E_INVAL;
    if (!lat->proposal_g) return SU2_E_STATE;
    DeviceGuard guard(lat->device);
    SU2_CUDA(cudaMemcpyAsync(host, lat->proposal, sizeof(float) * learned::kParams * lat->proposal_g,
                             cudaMemcpyDeviceToHost, lat->stream));
    SU2_CUDA(cudaStreamSynchronize(lat->stream));
    return SU2_OK;
}

su2_status su2_learned_generate(su2_lattice *lat, int nsweeps, int measure_every, double min_acceptance,
                                double *plaq, double *poly, su2_learned_stats *stats)
{
    if (!lat || nsweeps < 0 || measure_every < 0 || !(min_acceptance >= 0.0) || min_acceptance > 1.0)
        return SU2_E_INVAL;
    if (!lat->proposal_g) {
        set_last_error("su2_learned_generate: no proposal set (su2_set_proposal)");
        return SU2_E_STATE;
    }
    DeviceGuard guard(lat->device);
    const int nmeas = measure_every > 0 ? nsweeps / measure_every : 0;
    if (nmeas > 0) {
        // reuse the history buffer of su2_generate
        if (nmeas > lat->scratch.history_cap) {
            device_free(lat->scratch.history, sizeof(double) * 2 * (size_t)lat->scratch.history_cap, lat->device,
                        lat->stream);
            lat->scratch.history = (double *)device_alloc(sizeof(double) * 2 * (size_t)nmeas, lat->device, lat->stream);
            lat->scratch.history_cap = lat->scratch.history ? nmeas : 0;
            if (!lat->scratch.history) return SU2_E_NOMEM;
        }
    }
    su2_status st = launch_clear_counters(lat);
    if (st != SU2_OK) return st;
    const unsigned int ctl0[4] = {1u, 0u, 0u, 0u};
    SU2_CUDA(cudaMemcpyAsync(lat->learned_ctl, ctl0, sizeof ctl0, cudaMemcpyHostToDevice, lat->stream));
    SU2_CUDA(cudaMemsetAsync(lat->accept_slots, 0, sizeof(unsigned long long) * 9 * kAcceptSlots, lat->stream));
    lat->hb_log.used = 0;
    int m = 0;
    // Graph replays need a stream that can be captured and no per-launch events.
    bool graphs = lat->stream != nullptr && !lat->timing && !lat->graphs_off && nsweeps >= 1;
    if (graphs && (st = enqueue_set_counters(lat)) != SU2_OK) return st;
    for (int s = 1; s <= nsweeps; ++s) {
        // a measured sweep adds the plaquette through whichever kernel runs
        // each phase (learned, or the plain fallback)
        const bool measure = measure_every > 0 && s % measure_every == 0;
        if (graphs) {
            cudaGraphExec_t exec = nullptr;
            if ((st = learned_graph(lat, measure, min_acceptance, &exec)) != SU2_OK) return st;
            if (exec) {
                SU2_CUDA(cudaGraphLaunch(exec, lat->stream));
                lat->sweep += 1;
                if (measure) ++m;
                continue;
            }
            graphs = false;  // capture refused: run the rest eagerly
        }
        if ((st = learned_sweep_body(lat, measure, min_acceptance, lat->scratch.history + m,
                                     lat->scratch.history + lat->scratch.history_cap + m)) != SU2_OK)
            return st;
        lat->sweep += 1;
        if (measure) ++m;
    }
    if (nmeas > 0 && plaq)
        SU2_CUDA(cudaMemcpyAsync(plaq, lat->scratch.history, sizeof(double) * nmeas, cudaMemcpyDeviceToHost,
                                 lat->stream));
    if (nmeas > 0 && poly)
        SU2_CUDA(cudaMemcpyAsync(poly, lat->scratch.history + lat->scratch.history_cap, sizeof(double) * nmeas,
                                 cudaMemcpyDeviceToHost, lat->stream));
    unsigned long long slots[8 * kAcceptSlots];
    unsigned int ctl[4];
    SU2_CUDA(cudaMemcpyAsync(slots, lat->accept_slots, sizeof slots, cudaMemcpyDeviceToHost, lat->stream));
    SU2_CUDA(cudaMemcpyAsync(ctl, lat->learned_ctl, sizeof ctl, cudaMemcpyDeviceToHost, lat->stream));
    su2_stats plain;
    memset(&plain, 0, sizeof plain);
    st = collect_stats(lat, &plain, (uint64_t)nsweeps);
    double kms = 0.0;
    su2_status st_t = timing_read(lat, lat->hb_log, &kms);
    if (st == SU2_OK) st = st_t;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        for (int ph = 0; ph < 8; ++ph) {
            uint64_t a = 0;
            for (int j = 0; j < kAcceptSlots; ++j) a += slots[ph * kAcceptSlots + j];
            stats->accepted[ph] = a;
            stats->plain_trials[ph] = plain.trials[ph];
        }
        stats->plain_sweeps = ctl[1];
        stats->learned_sweeps = ctl[2];
        stats->link_updates = (uint64_t)nsweeps * 4ull * (uint64_t)lat->vol;
        stats->kernel_launches = (uint32_t)(8 * nsweeps);
        stats->timed = lat->timing ? 1u : 0u;
        stats->kernel_ms = kms;
    }
    return st;
}

su2_status su2_learned_sweep(su2_lattice *lat, int nsweeps, su2_learned_stats *stats)
{
    return su2_learned_generate(lat, nsweeps, 0, 0.7, nullptr, nullptr, stats);
}

su2_status su2_collect_pairs(su2_lattice *lat, int mu, int parity, int stride, float *dev_pairs, size_t cap,
                             size_t *n)
{
    if (!lat || !dev_pairs || !n || mu < 0 || mu > 3 || (parity != 0 && parity != 1) || stride < 1) return SU2_E_INVAL;
    const int n_pairs = (lat->vh + stride - 1) / stride;
    if ((size_t)n_pairs > cap) {
        set_last_error("su2_collect_pairs: buffer too small");
        return SU2_E_INVAL;
    }
    DeviceGuard guard(lat->device);
    const Geom g = geom_of(lat);
    const RoundKeys rk = make_round_keys(lat->seed);
    const int grid = (n_pairs + kLearnThreads - 1) / kLearnThreads;
    float2 *out = (float2 *)dev_pairs;
    const float beta = (float)lat->beta;
    switch (mu) {
    case 0: collect_kernel<0><<<grid, kLearnThreads, 0, lat->stream>>>(lat->links, g, parity, rk, beta, lat->sweep, stride, out, n_pairs); break;
    case 1: collect_kernel<1><<<grid, kLearnThreads, 0, lat->stream>>>(lat->links, g, parity, rk, beta, lat->sweep, stride, out, n_pairs); break;
    case 2: collect_kernel<2><<<grid, kLearnThreads, 0, lat->stream>>>(lat->links, g, parity, rk, beta, lat->sweep, stride, out, n_pairs); break;
    default: collect_kernel<3><<<grid, kLearnThreads, 0, lat->stream>>>(lat->links, g, parity, rk, beta, lat->sweep, stride, out, n_pairs); break;
    }
    SU2_CUDA(cudaGetLastError());
    *n = (size_t)n_pairs;
    return SU2_OK;
}

}  // extern "C"
