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

#include "batch_device.cuh"

namespace su2 {

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
    double *d_chunk_partials = nullptr;  // [3][chunks at queue depth 1, the most]
    int *d_chunk_owner = nullptr;        // [chunks at queue depth 1]
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
    int sampler = SU2_SAMPLER_CREUTZ;
    int max_grid[2][4][3] = {};  // co-resident blocks: sampler x R = 1, 2, 4, 8 x block sizes 64, 128, 256
    uint32_t sweep = 0;
    unsigned long long timeout_ns = 2000000000ull;
    bool use_graph = true;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // [measure]
    void *staging = nullptr;
    size_t staging_bytes = 0;
};

namespace su2 {
namespace {

int r_index(int R) { return R == 1 ? 0 : (R == 2 ? 1 : (R == 4 ? 2 : 3)); }
int t_index(int T) { return T == 64 ? 0 : (T == 128 ? 1 : 2); }

void *kernel_for(int sampler, int R, int T)
{
    if (sampler == SU2_SAMPLER_KP) return R <= 2 ? batch_kernel_kp_12(R, T) : batch_kernel_kp_48(R, T);
    return R <= 2 ? batch_kernel_creutz_12(R, T) : batch_kernel_creutz_48(R, T);
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
    return cudaLaunchCooperativeKernel(kernel_for(b->sampler, b->R, b->threads), dim3(b->grid), dim3(b->threads),
                                       args, 0,
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
    size_t max_chunks = 0;  // chunks of 32 sites (queue depth 1)
    std::vector<int> mprefix(n + 1, 0);
    for (int l = 0; l < n; ++l) {
        const Geom g = make_geom(ns[l], nt[l]);
        max_chunks += ((size_t)g.vh + 31) / 32;
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
        for (int sm = 0; sm < 2 && e == cudaSuccess; ++sm)
            for (int i = 0; i < 4 && e == cudaSuccess; ++i)
                for (int j = 0; j < 3 && e == cudaSuccess; ++j) {
                    const int R = 1 << i;
                    int per_sm = 0;
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_for(sm, R, kBatchBlockSizes[j]),
                                                                      kBatchBlockSizes[j], 0);
                    b->max_grid[sm][i][j] = std::max(1, per_sm * sms);
                }
    }
    if (e != cudaSuccess) st = cuda_fail(e, "su2_batch_create");
    if (st == SU2_OK) st = set_depth(b, 4, 128, b->max_grid[0][r_index(4)][t_index(128)]);
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
    if (!b || (queue_depth != 1 && queue_depth != 2 && queue_depth != 4 && queue_depth != 8) ||
        (threads != 64 && threads != 128 && threads != 256))
        return SU2_E_INVAL;
    const int most = b->max_grid[b->sampler][r_index(queue_depth)][t_index(threads)];
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

su2_status su2_batch_set_sampler(su2_batch *b, int sampler)
{
    if (!b || (sampler != SU2_SAMPLER_CREUTZ && sampler != SU2_SAMPLER_KP)) return SU2_E_INVAL;
    if (sampler == b->sampler) return SU2_OK;
    DeviceGuard guard(b->device);
    b->sampler = sampler;
    // the same launch shape, clamped to what this sampler's kernel holds co-resident
    return su2_batch_set_launch(b, b->R, b->threads, b->grid);
}

// Times each candidate (queue depth 1/2/4/8 x block size 64/128/256 x the
// co-resident grid or 1/2, 1/4, 1/8, 1/16 of it: small batches run faster on
// fewer blocks, whose grid barriers cost less) over `sweeps` sweeps of the
// batch, then restores the links and the sweep counter, and keeps the fastest.
constexpr int kGridFractions = 5;
constexpr int kAutotuneCandidates = 4 * 3 * kGridFractions;

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
    const int depths[4] = {1, 2, 4, 8};
    for (int c = 0; c < kAutotuneCandidates && st == SU2_OK; ++c) {
            const int i = c / (3 * kGridFractions), j = (c / kGridFractions) % 3, f = c % kGridFractions;
            const int R = depths[i], T = kBatchBlockSizes[j];
            const int most = b->max_grid[b->sampler][i][j];
            const int grid = std::max(1, most >> f);  // the co-resident grid, 1/2, 1/4, 1/8 or 1/16 of it
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
