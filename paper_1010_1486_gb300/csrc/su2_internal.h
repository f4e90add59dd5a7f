// su2_internal.h -- host-side state of a lattice handle and the launchers
// shared between the translation units of libsu2.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/su2.h"
#include "su2_device.cuh"

namespace su2 {

constexpr int kTrialSlots = 64;      // trial counters are spread over 64 slots per phase
constexpr int kReduceThreads = 256;  // block size of the observable kernels
constexpr int kHbThreads = 128;      // block size of the heat-bath phase kernel (4 warps)
// Plaquette measured during a sweep: the odd phases of mu = 1, 2, 3 each add
// the plaquettes of planes (nu, mu), nu < mu, through the new links; block
// partials go to slots [(mu - 1) * 2 + kind] * kFusedSlots + block (kind 0:
// heat bath / over-relaxation, 1: learned), zero-filled first.
constexpr int kFusedSlots = 1024;
constexpr int kFusedRegion = 6 * kFusedSlots;

// Device scratch of a lattice, carved from one allocation.
struct DeviceScratch {
    double *partials = nullptr;             // per-block partial sums of a reduction
    unsigned int *ticket = nullptr;         // last-block counter of a reduction
    double *result = nullptr;               // [0] plaquette, [1] Polyakov (latest)
    unsigned long long *trials = nullptr;   // [8][kTrialSlots]
    unsigned int *flags = nullptr;          // [0] sampler cap hits, [1] other errors
    double *history = nullptr;              // measurements of su2_generate: [2][history_cap]
    int partials_cap = 0;
    int history_cap = 0;
};

}  // namespace su2

namespace su2 {
// CUDA events recorded in pairs around timed kernel launches.
struct EventLog {
    std::vector<cudaEvent_t> events;
    size_t used = 0;
};

// One sweep of su2_generate captured as a CUDA graph; `sig` identifies the
// settings it was captured with (sampler, beta, seed, over-relaxation, buffers).
struct GenGraph {
    cudaGraphExec_t exec = nullptr;
    uint64_t sig = 0;
};
}  // namespace su2

struct su2_lattice {
    int ns = 0, nt = 0;
    int64_t vol = 0;  // Ns^3 Nt
    int vh = 0;       // vol / 2
    double beta = 0.0;
    uint64_t seed = 0;
    uint32_t sweep = 0;
    int sampler = 0;  // SU2_SAMPLER_CREUTZ or SU2_SAMPLER_KP
    int max_trials = 4096;  // sampler trials per link before it keeps its old value (su2_set_trial_cap)
    int device = 0;
    cudaStream_t stream = nullptr;

    void *block = nullptr;  // the single device allocation
    size_t block_bytes = 0;
    float4 *links = nullptr;  // 8 vh float4 (even/odd structure of arrays)
    su2::DeviceScratch scratch;

    void *staging = nullptr;  // lex-ordered copy for get/set_links (allocated on demand)
    size_t staging_bytes = 0;

    int overrelax = 0;  // over-relaxation sweeps after each heat-bath sweep
    double *fused_part = nullptr;  // slot region of the plaquette measured in the current sweep, or NULL
    bool capturing = false;        // launches are being captured into a generation graph
    bool graphs_off = false;       // a capture failed once: generate eagerly
    uint32_t *d_ctr = nullptr;     // device: [0] sweep counter, [1] measurement slot (graph replays)
    su2::GenGraph gen_graph[4];    // captured sweeps, variant = (measured) | (reunitarized) << 1
    su2::GenGraph learned_graph[2];  // captured learned sweeps, [measured]

    bool timing = false;
    su2::EventLog hb_log;  // heat-bath (and learned) phase launches
    su2::EventLog or_log;  // over-relaxation phase launches

    // learned proposal (allocated by su2_set_proposal)
    void *learned_block = nullptr;
    size_t learned_bytes = 0;
    float *proposal = nullptr;                 // G x 27 spline parameters
    float2 *proposal_pairs = nullptr;          // (G - 1) x 27 row pairs (r_j, r_{j+1} - r_j), padded to 16 bytes
    int proposal_g = 0;
    float prop_s_lo = 0, prop_s_hi = 1, prop_mean = 0, prop_scale = 1;
    unsigned int *learned_ctl = nullptr;       // [0] gate (1 = learned sweep), [1] plain sweeps, [2] learned sweeps
    unsigned long long *accept_slots = nullptr;  // [8][64] per call, then [64] per sweep
};

namespace su2 {

// The part of a phase that a time slab runs (Sec. 4, multi-GPU part): the
// even/odd indices [eo_begin, eo_end) of its interior slices, and the keys of
// their random numbers in the whole lattice -- even/odd index + rng_eo and the
// global parity rng_parity.  A whole lattice is [0, vh), 0, its own parity.
struct SlabRange {
    int eo_begin = 0, eo_end = 0;
    uint32_t rng_eo = 0;
    int rng_parity = 0;
};

// Error bookkeeping (per thread).
void set_last_error(const std::string &msg);
su2_status cuda_fail(cudaError_t e, const char *what);

#define SU2_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return ::su2::cuda_fail(e_, #call);             \
    } while (0)

// Keeps the lattice's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

inline Geom make_geom(int ns, int nt)
{
    Geom g;
    g.ns = ns;
    g.nt = nt;
    g.vh = (int)((int64_t)ns * ns * ns * nt / 2);
    g.vs = ns * ns * ns;
    g.div_ns = make_fastdiv((uint32_t)ns);
    int stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.ext[mu] = mu == 3 ? nt : ns;
        g.stride[mu] = stride;
        g.wrap[mu] = (g.ext[mu] - 1) * stride;
        stride *= g.ext[mu];
    }
    return g;
}

inline Geom geom_of(const su2_lattice *lat) { return make_geom(lat->ns, lat->nt); }

// The link arrays a phase of the given parity reads, by direction: same[d] at
// that parity, other[d] at the opposite one (kernel parameters, so the
// kernels address them from the constant bank instead of recomputing them).
inline void set_bases(const float4 **same, const float4 **other, const su2_lattice *lat, int parity)
{
    for (int d = 0; d < 4; ++d) {
        same[d] = lat->links + (size_t)(2 * d + parity) * (size_t)lat->vh;
        other[d] = lat->links + (size_t)(2 * d + (parity ^ 1)) * (size_t)lat->vh;
    }
}

inline int grid_for(int64_t n, int threads, int64_t cap = 152 * 64)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// Allocation through the installed hook (or cudaMallocAsync).
void *device_alloc(size_t bytes, int device, cudaStream_t stream);
void device_free(void *ptr, size_t bytes, int device, cudaStream_t stream);

// Start configurations and layout conversion of one lattice's links
// (8 vh float4 at `links`), enqueued on `stream`.
cudaError_t start_links(float4 *links, const Geom &g, bool hot, uint64_t seed, unsigned int *flags,
                        cudaStream_t stream);
cudaError_t convert_links(float4 *eo_links, float4 *lex_links, const Geom &g, bool to_lex, cudaStream_t stream);

// Block-partial slots of the fused plaquette for phase (mu, parity) and kernel
// kind, or NULL when that phase does not measure.
inline double *fused_slot(const su2_lattice *lat, int mu, int parity, int kind)
{
    if (!lat->fused_part || parity != 1 || mu < 1) return nullptr;
    return lat->fused_part + ((mu - 1) * 2 + kind) * kFusedSlots;
}
// Zero-fills the slot region and points the lattice at it (the next sweep
// measures); fused_finish_with_polyakov detaches it and, in one launch, sums
// the region (block shares in index order, then the shares in block order)
// into *plaq_dst (device) scaled to the mean plaquette, and writes the
// Polyakov loop to *poly_dst.
su2_status fused_begin(su2_lattice *lat);
// Graph replays of generation loops: the device sweep counter and measurement
// slot set from the host state (one-thread kernel), advanced at the end of a
// captured sweep; and the hash of the settings a captured sweep depends on.
su2_status enqueue_set_counters(su2_lattice *lat);
su2_status enqueue_advance(su2_lattice *lat, bool measured);
uint64_t generation_signature(const su2_lattice *lat);
su2_status fused_finish_with_polyakov(su2_lattice *lat, double *plaq_dst, double *poly_dst);

// Launchers (each enqueues on lat->stream and returns a status of the launch).
su2_status launch_cold_start(su2_lattice *lat);
su2_status launch_hot_start(su2_lattice *lat);
su2_status launch_hb_phase(su2_lattice *lat, int mu, int parity, uint32_t sweep,
                           const unsigned int *gate = nullptr);
su2_status launch_kp_phase(su2_lattice *lat, int mu, int parity, uint32_t sweep, const unsigned int *gate);
// A phase on the interior of a time slab: parity_local selects the slab's
// even/odd arrays, r the eo range and the random-number keys (sampler as set).
su2_status launch_hb_phase_slab(su2_lattice *lat, int mu, int parity_local, uint32_t sweep, const SlabRange &r);
su2_status launch_kp_phase_slab(su2_lattice *lat, int mu, int parity_local, uint32_t sweep, const SlabRange &r);
su2_status launch_reunitarize(su2_lattice *lat);
// Observables: write the value into *dst (device memory) without synchronising.
su2_status launch_plaquette(su2_lattice *lat, double *dst);
su2_status launch_polyakov(su2_lattice *lat, double *dst);
su2_status launch_clear_counters(su2_lattice *lat);
// CUDA events around a kernel on the lattice's stream (when timing is on),
// and the summed duration of the recorded pairs (synchronises, then resets).
su2_status timing_begin(su2_lattice *lat, EventLog &log);
su2_status timing_end(su2_lattice *lat, EventLog &log);
su2_status timing_read(su2_lattice *lat, EventLog &log, double *ms);
// Over-relaxation: one phase, and `n` sweeps (8 phases each, timed into or_log).
su2_status launch_or_phase(su2_lattice *lat, int mu, int parity);
su2_status overrelax_sweeps(su2_lattice *lat, int n);
// Reads and clears the trial counters and flags (synchronises).
su2_status collect_stats(su2_lattice *lat, su2_stats *stats, uint64_t sweeps);

}  // namespace su2
