// lattice.cu -- lattice handles: creation, device memory, cold/hot start
// (Sec. 4 of Cardoso & Bicudo), link layout conversion, reunitarization,
// resumable state, status strings.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

// ------------------------------------------------------------ error text
static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

su2_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return SU2_E_CUDA;
}

// ------------------------------------------------------ allocation hook
static std::mutex g_alloc_mutex;
static su2_alloc_fn g_alloc = nullptr;
static su2_free_fn g_free = nullptr;
static void *g_alloc_ctx = nullptr;

void *device_alloc(size_t bytes, int device, cudaStream_t stream)
{
    su2_alloc_fn fn;
    void *ctx;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        fn = g_alloc;
        ctx = g_alloc_ctx;
    }
    if (fn) return fn(bytes, device, (void *)stream, ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void device_free(void *ptr, size_t bytes, int device, cudaStream_t stream)
{
    if (!ptr) return;
    su2_free_fn fn;
    void *ctx;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        fn = g_free;
        ctx = g_alloc_ctx;
    }
    if (fn) {
        fn(ptr, bytes, device, (void *)stream, ctx);
        return;
    }
    cudaFreeAsync(ptr, stream);
}

// ------------------------------------------------------------- kernels
__global__ void cold_start_kernel(float4 *__restrict__ links, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        links[i] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
}

// Haar-random links (hot_link in su2_device.cuh), link (mu, parity, eo).
__global__ void hot_start_kernel(float4 *__restrict__ links, Geom g, const RoundKeys rk,
                                 unsigned int *__restrict__ flags)
{
    const int64_t n = 8 * (int64_t)g.vh;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int group = (int)(idx / g.vh);
        const int eo = (int)(idx - (int64_t)group * g.vh);
        float4 out;
        if (!hot_link((uint32_t)eo, (uint32_t)(group & 1), (uint32_t)(group >> 1), rk, out)) atomicAdd(&flags[1], 1u);
        links[idx] = out;
    }
}

// even/odd structure of arrays  <->  [lex site][mu][4].  Thread q takes
// float4 q of the lexicographic array (site q / 4, direction q % 4), so the
// lexicographic side -- a staging buffer or, for mapped pinned host memory,
// the caller's buffer itself read over the host link -- is accessed
// contiguously.
template <bool kToLex>
__global__ void convert_kernel(float4 *__restrict__ eo_links, float4 *__restrict__ lex_links, Geom g)
{
    const int64_t n = 8 * (int64_t)g.vh;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t site = (uint32_t)(q >> 2);
        const int mu = (int)(q & 3);
        const uint32_t r1 = fastdiv(site, g.div_ns);
        const uint32_t r2 = fastdiv(r1, g.div_ns);
        const uint32_t t = fastdiv(r2, g.div_ns);
        const uint32_t ns = (uint32_t)g.ns;
        const uint32_t coord_sum = (site - r1 * ns) + (r1 - r2 * ns) + (r2 - t * ns) + t;
        const uint32_t e = link_index(g, mu, (int)(coord_sum & 1u), (int)(site >> 1));
        if (kToLex)
            lex_links[q] = eo_links[e];
        else
            eo_links[e] = lex_links[q];
    }
}

// a <- a / |a|
__global__ void reunitarize_kernel(float4 *__restrict__ links, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = links[i];
        const float r = __fsqrt_rn(qnorm2(a));
        links[i] = make_float4(__fdiv_rn(a.x, r), __fdiv_rn(a.y, r), __fdiv_rn(a.z, r), __fdiv_rn(a.w, r));
    }
}

cudaError_t start_links(float4 *links, const Geom &g, bool hot, uint64_t seed, unsigned int *flags,
                        cudaStream_t stream)
{
    const int64_t n = 8 * (int64_t)g.vh;
    if (hot)
        hot_start_kernel<<<grid_for(n, 256), 256, 0, stream>>>(links, g, make_round_keys(seed), flags);
    else
        cold_start_kernel<<<grid_for(n, 256), 256, 0, stream>>>(links, n);
    return cudaGetLastError();
}

cudaError_t convert_links(float4 *eo_links, float4 *lex_links, const Geom &g, bool to_lex, cudaStream_t stream)
{
    const int64_t vol = 2 * (int64_t)g.vh;
    if (to_lex)
        convert_kernel<true><<<grid_for(vol, 256), 256, 0, stream>>>(eo_links, lex_links, g);
    else
        convert_kernel<false><<<grid_for(vol, 256), 256, 0, stream>>>(eo_links, lex_links, g);
    return cudaGetLastError();
}

su2_status launch_cold_start(su2_lattice *lat)
{
    const int64_t n = 8 * (int64_t)lat->vh;
    cold_start_kernel<<<grid_for(n, 256), 256, 0, lat->stream>>>(lat->links, n);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status launch_hot_start(su2_lattice *lat)
{
    const int64_t n = 8 * (int64_t)lat->vh;
    hot_start_kernel<<<grid_for(n, 256), 256, 0, lat->stream>>>(lat->links, geom_of(lat),
                                                                make_round_keys(lat->seed), lat->scratch.flags);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status launch_reunitarize(su2_lattice *lat)
{
    const int64_t n = 8 * (int64_t)lat->vh;
    reunitarize_kernel<<<grid_for(n, 256), 256, 0, lat->stream>>>(lat->links, n);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status launch_clear_counters(su2_lattice *lat)
{
    SU2_CUDA(cudaMemsetAsync(lat->scratch.trials, 0, sizeof(unsigned long long) * 8 * kTrialSlots, lat->stream));
    SU2_CUDA(cudaMemsetAsync(lat->scratch.flags, 0, sizeof(unsigned int) * 4, lat->stream));
    return SU2_OK;
}

su2_status collect_stats(su2_lattice *lat, su2_stats *stats, uint64_t sweeps)
{
    unsigned long long slots[8 * kTrialSlots];
    unsigned int flags[4];
    SU2_CUDA(cudaMemcpyAsync(slots, lat->scratch.trials, sizeof slots, cudaMemcpyDeviceToHost, lat->stream));
    SU2_CUDA(cudaMemcpyAsync(flags, lat->scratch.flags, sizeof flags, cudaMemcpyDeviceToHost, lat->stream));
    SU2_CUDA(cudaStreamSynchronize(lat->stream));
    if (stats) {
        for (int ph = 0; ph < 8; ++ph) {
            uint64_t s = 0;
            for (int j = 0; j < kTrialSlots; ++j) s += slots[ph * kTrialSlots + j];
            stats->trials[ph] = s;
        }
        stats->sampler_failures = flags[0];
        stats->sweeps = sweeps;
        stats->link_updates = sweeps * 4ull * (uint64_t)lat->vol;
    }
    if (flags[0] != 0) {
        set_last_error("heat-bath sampler hit its trial cap");
        return SU2_E_SAMPLER;
    }
    if (flags[2] != 0) {
        set_last_error("a learned phase gave up waiting for its proposal-table copy");
        return SU2_E_DEVICE_TIMEOUT;
    }
    return SU2_OK;
}

// Counts links with a non-finite component, and links with | |a| - 1 | > tol
// (|a|^2 summed as the fixed chain of the quaternion norm, in binary32).
__global__ void check_links_kernel(const float4 *__restrict__ L, int64_t n, float tol,
                                   unsigned long long *__restrict__ counts)
{
    unsigned long long bad = 0, off = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = __ldg(L + i);
        if (!(isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w))) {
            ++bad;
        } else {
            const float r = __fsqrt_rn(qnorm2(a));
            if (fabsf(__fsub_rn(r, 1.0f)) > tol) ++off;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad += __shfl_down_sync(0xffffffffu, bad, o);
        off += __shfl_down_sync(0xffffffffu, off, o);
    }
    if ((threadIdx.x & 31) == 0 && (bad | off)) {
        atomicAdd(counts, bad);
        atomicAdd(counts + 1, off);
    }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace su2

using namespace su2;

// ====================================================================== C ABI
extern "C" {

int su2_abi_version(void) { return SU2_ABI_VERSION; }

const char *su2_last_error(void) { return g_last_error.c_str(); }

const char *su2_status_str(su2_status s)
{
    switch (s) {
    case SU2_OK: return "ok";
    case SU2_E_INVAL: return "invalid argument";
    case SU2_E_NOMEM: return "out of memory";
    case SU2_E_CUDA: return "CUDA error";
    case SU2_E_SAMPLER: return "heat-bath sampler hit its trial cap";
    case SU2_E_DEVICE_TIMEOUT: return "device wait timed out";
    case SU2_E_NUMERIC: return "non-finite value";
    case SU2_E_STATE: return "invalid state for this call";
    }
    return "unknown status";
}

su2_status su2_set_allocator(su2_alloc_fn alloc, su2_free_fn free_fn, void *ctx)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_last_error("su2_set_allocator: alloc and free must both be set or both NULL");
        return SU2_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_ctx = alloc ? ctx : nullptr;
    return SU2_OK;
}

static su2_status validate_extents(int ns, int nt)
{
    if (ns < 2 || nt < 2 || (ns & 1) || (nt & 1)) {
        set_last_error("extents must be even and >= 2");
        return SU2_E_INVAL;
    }
    const double links = 4.0 * (double)ns * ns * ns * nt;
    if (links >= 2147483648.0) {
        set_last_error("lattice too large (4 V must be below 2^31)");
        return SU2_E_INVAL;
    }
    return SU2_OK;
}

static su2_status validate_beta(double beta)
{
    if (!std::isfinite(beta) || beta < 0.0) {
        set_last_error("beta must be finite and >= 0");
        return SU2_E_INVAL;
    }
    return SU2_OK;
}

su2_status su2_create(int ns, int nt, double beta, uint64_t seed, su2_start start, void *cuda_stream,
                      su2_lattice **out)
{
    if (!out) {
        set_last_error("su2_create: out is NULL");
        return SU2_E_INVAL;
    }
    *out = nullptr;
    su2_status st = validate_extents(ns, nt);
    if (st != SU2_OK) return st;
    if ((st = validate_beta(beta)) != SU2_OK) return st;
    if (start != SU2_COLD && start != SU2_HOT) {
        set_last_error("start must be SU2_COLD or SU2_HOT");
        return SU2_E_INVAL;
    }
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));

    su2_lattice *lat = new (std::nothrow) su2_lattice();
    if (!lat) return SU2_E_NOMEM;
    lat->ns = ns;
    lat->nt = nt;
    lat->vol = (int64_t)ns * ns * ns * nt;
    lat->vh = (int)(lat->vol / 2);
    lat->beta = beta;
    lat->seed = seed;
    lat->sweep = 0;
    lat->device = dev;
    lat->stream = (cudaStream_t)cuda_stream;

    // one allocation: links | partials | ticket | result | trials | flags
    const size_t links_bytes = align256(sizeof(float4) * 8 * (size_t)lat->vh);
    // one partial per block of the observable kernels (one site per thread)
    const int partials_cap = (int)std::max<int64_t>(152 * 64, (lat->vol + kReduceThreads - 1) / kReduceThreads);
    const size_t partials_bytes = align256(sizeof(double) * partials_cap);
    const size_t ticket_bytes = align256(sizeof(unsigned int) * 4);
    const size_t result_bytes = align256(sizeof(double) * 4);
    const size_t trials_bytes = align256(sizeof(unsigned long long) * 8 * kTrialSlots);
    const size_t flags_bytes = align256(sizeof(unsigned int) * 4);
    const size_t ctr_bytes = align256(sizeof(uint32_t) * 2);
    lat->block_bytes =
        links_bytes + partials_bytes + ticket_bytes + result_bytes + trials_bytes + flags_bytes + ctr_bytes;
    lat->block = device_alloc(lat->block_bytes, dev, lat->stream);
    if (!lat->block) {
        delete lat;
        set_last_error("device allocation of the lattice failed");
        return SU2_E_NOMEM;
    }
    char *p = (char *)lat->block;
    lat->links = (float4 *)p;
    p += links_bytes;
    lat->scratch.partials = (double *)p;
    lat->scratch.partials_cap = partials_cap;
    p += partials_bytes;
    lat->scratch.ticket = (unsigned int *)p;
    p += ticket_bytes;
    lat->scratch.result = (double *)p;
    p += result_bytes;
    lat->scratch.trials = (unsigned long long *)p;
    p += trials_bytes;
    lat->scratch.flags = (unsigned int *)p;
    p += flags_bytes;
    lat->d_ctr = (uint32_t *)p;

    st = SU2_OK;
    if (cudaMemsetAsync(lat->scratch.ticket, 0, ticket_bytes + result_bytes + trials_bytes + flags_bytes + ctr_bytes,
                        lat->stream) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "cudaMemsetAsync");
    if (st == SU2_OK) st = (start == SU2_HOT) ? launch_hot_start(lat) : launch_cold_start(lat);
    if (st == SU2_OK && start == SU2_HOT) {
        unsigned int flags[4];
        if (cudaMemcpyAsync(flags, lat->scratch.flags, sizeof flags, cudaMemcpyDeviceToHost, lat->stream) != cudaSuccess ||
            cudaStreamSynchronize(lat->stream) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "hot start");
        else if (flags[1] != 0) {
            set_last_error("hot start: a link found no two disk points in 64 pairs");
            st = SU2_E_SAMPLER;
        }
    }
    if (st != SU2_OK) {
        su2_destroy(lat);
        return st;
    }
    *out = lat;
    return SU2_OK;
}

su2_status su2_destroy(su2_lattice *lat)
{
    if (!lat) return SU2_OK;
    DeviceGuard guard(lat->device);
    for (cudaEvent_t e : lat->hb_log.events) cudaEventDestroy(e);
    for (cudaEvent_t e : lat->or_log.events) cudaEventDestroy(e);
    for (GenGraph &gg : lat->learned_graph)
        if (gg.exec) cudaGraphExecDestroy(gg.exec);
    for (GenGraph &gg : lat->gen_graph)
        if (gg.exec) cudaGraphExecDestroy(gg.exec);
    device_free(lat->staging, lat->staging_bytes, lat->device, lat->stream);
    device_free(lat->learned_block, lat->learned_bytes, lat->device, lat->stream);
    device_free(lat->scratch.history, sizeof(double) * 2 * (size_t)lat->scratch.history_cap, lat->device,
                lat->stream);
    device_free(lat->block, lat->block_bytes, lat->device, lat->stream);
    cudaError_t e = cudaStreamSynchronize(lat->stream);
    delete lat;
    if (e != cudaSuccess) return cuda_fail(e, "su2_destroy");
    return SU2_OK;
}

static su2_status ensure_staging(su2_lattice *lat)
{
    const size_t need = sizeof(float4) * 4 * (size_t)lat->vol;
    if (lat->staging && lat->staging_bytes >= need) return SU2_OK;
    device_free(lat->staging, lat->staging_bytes, lat->device, lat->stream);
    lat->staging = device_alloc(need, lat->device, lat->stream);
    lat->staging_bytes = lat->staging ? need : 0;
    if (!lat->staging) {
        set_last_error("device allocation of the staging buffer failed");
        return SU2_E_NOMEM;
    }
    return SU2_OK;
}

// Device address of a host buffer that is page-locked and mapped (e.g.
// cudaHostAlloc), else NULL.
static float4 *mapped_host(const void *host)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? (float4 *)a.devicePointer : nullptr;
}

su2_status su2_get_links(su2_lattice *lat, float *host)
{
    if (!lat || !host) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    const int grid = grid_for(4 * lat->vol, 256, 152 * 16);
    if (float4 *direct = mapped_host(host)) {
        convert_kernel<true><<<grid, 256, 0, lat->stream>>>(lat->links, direct, geom_of(lat));
        SU2_CUDA(cudaGetLastError());
    } else {
        su2_status st = ensure_staging(lat);
        if (st != SU2_OK) return st;
        convert_kernel<true><<<grid, 256, 0, lat->stream>>>(lat->links, (float4 *)lat->staging, geom_of(lat));
        SU2_CUDA(cudaGetLastError());
        SU2_CUDA(cudaMemcpyAsync(host, lat->staging, sizeof(float4) * 4 * (size_t)lat->vol, cudaMemcpyDeviceToHost,
                                 lat->stream));
    }
    SU2_CUDA(cudaStreamSynchronize(lat->stream));
    return SU2_OK;
}

su2_status su2_set_links(su2_lattice *lat, const float *host)
{
    if (!lat || !host) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    const int grid = grid_for(4 * lat->vol, 256, 152 * 16);
    if (float4 *direct = mapped_host(host)) {
        convert_kernel<false><<<grid, 256, 0, lat->stream>>>(lat->links, direct, geom_of(lat));
        SU2_CUDA(cudaGetLastError());
    } else {
        su2_status st = ensure_staging(lat);
        if (st != SU2_OK) return st;
        SU2_CUDA(cudaMemcpyAsync(lat->staging, host, sizeof(float4) * 4 * (size_t)lat->vol, cudaMemcpyHostToDevice,
                                 lat->stream));
        convert_kernel<false><<<grid, 256, 0, lat->stream>>>(lat->links, (float4 *)lat->staging, geom_of(lat));
        SU2_CUDA(cudaGetLastError());
    }
    SU2_CUDA(cudaStreamSynchronize(lat->stream));
    return SU2_OK;
}

// Asynchronous forms: the links always go through the staging buffer and the
// copy engines, so a transfer of one lattice runs beside the sweep kernels of
// another lattice on its own stream (a conversion kernel reading mapped host
// memory would need SMs that a persistent sweep holds).
su2_status su2_set_links_async(su2_lattice *lat, const float *host)
{
    if (!lat || !host) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    su2_status st = ensure_staging(lat);
    if (st != SU2_OK) return st;
    SU2_CUDA(cudaMemcpyAsync(lat->staging, host, sizeof(float4) * 4 * (size_t)lat->vol, cudaMemcpyHostToDevice,
                             lat->stream));
    convert_kernel<false><<<grid_for(4 * lat->vol, 256, 152 * 16), 256, 0, lat->stream>>>(
        lat->links, (float4 *)lat->staging, geom_of(lat));
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status su2_get_links_async(su2_lattice *lat, float *host)
{
    if (!lat || !host) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    su2_status st = ensure_staging(lat);
    if (st != SU2_OK) return st;
    convert_kernel<true><<<grid_for(4 * lat->vol, 256, 152 * 16), 256, 0, lat->stream>>>(
        lat->links, (float4 *)lat->staging, geom_of(lat));
    SU2_CUDA(cudaGetLastError());
    SU2_CUDA(cudaMemcpyAsync(host, lat->staging, sizeof(float4) * 4 * (size_t)lat->vol, cudaMemcpyDeviceToHost,
                             lat->stream));
    return SU2_OK;
}

su2_status su2_sync(su2_lattice *lat)
{
    if (!lat) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    unsigned int flags[4];
    SU2_CUDA(cudaMemcpyAsync(flags, lat->scratch.flags, sizeof flags, cudaMemcpyDeviceToHost, lat->stream));
    SU2_CUDA(cudaStreamSynchronize(lat->stream));
    if (flags[0] != 0) {
        SU2_CUDA(cudaMemsetAsync(lat->scratch.flags, 0, sizeof(unsigned int), lat->stream));
        SU2_CUDA(cudaStreamSynchronize(lat->stream));
        set_last_error("heat-bath sampler hit its trial cap");
        return SU2_E_SAMPLER;
    }
    return SU2_OK;
}

su2_status su2_check_links(su2_lattice *lat, double tol, uint64_t *nonfinite, uint64_t *off_norm)
{
    if (!lat || !(tol >= 0.0)) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    unsigned long long *d = (unsigned long long *)device_alloc(2 * sizeof(unsigned long long), lat->device,
                                                               lat->stream);
    if (!d) return SU2_E_NOMEM;
    unsigned long long h[2] = {0ull, 0ull};
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof h, lat->stream);
    if (e == cudaSuccess) {
        check_links_kernel<<<grid_for(4 * lat->vol, 256, 152 * 8), 256, 0, lat->stream>>>(lat->links, 4 * lat->vol,
                                                                                          (float)tol, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, lat->stream);
    device_free(d, 2 * sizeof(unsigned long long), lat->device, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    if (e != cudaSuccess) return cuda_fail(e, "su2_check_links");
    if (nonfinite) *nonfinite = h[0];
    if (off_norm) *off_norm = h[1];
    if (h[0]) {
        set_last_error("non-finite link components");
        return SU2_E_NUMERIC;
    }
    return SU2_OK;
}

su2_status su2_reunitarize(su2_lattice *lat)
{
    if (!lat) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    return launch_reunitarize(lat);
}

su2_status su2_get_state(const su2_lattice *lat, su2_state *out)
{
    if (!lat || !out) return SU2_E_INVAL;
    out->ns = lat->ns;
    out->nt = lat->nt;
    out->beta = lat->beta;
    out->seed = lat->seed;
    out->sweep = lat->sweep;
    return SU2_OK;
}

su2_status su2_set_state(su2_lattice *lat, const su2_state *in)
{
    if (!lat || !in) return SU2_E_INVAL;
    if (in->ns != lat->ns || in->nt != lat->nt) {
        set_last_error("su2_set_state: extents differ from the lattice's");
        return SU2_E_INVAL;
    }
    su2_status st = validate_beta(in->beta);
    if (st != SU2_OK) return st;
    lat->beta = in->beta;
    lat->seed = in->seed;
    lat->sweep = in->sweep;
    return SU2_OK;
}

su2_status su2_set_beta(su2_lattice *lat, double beta)
{
    if (!lat) return SU2_E_INVAL;
    su2_status st = validate_beta(beta);
    if (st != SU2_OK) return st;
    lat->beta = beta;
    return SU2_OK;
}

su2_status su2_device_links(su2_lattice *lat, void **ptr, size_t *bytes)
{
    if (!lat || !ptr) return SU2_E_INVAL;
    *ptr = lat->links;
    if (bytes) *bytes = sizeof(float4) * 8 * (size_t)lat->vh;
    return SU2_OK;
}

su2_status su2_set_timing(su2_lattice *lat, int enable)
{
    if (!lat) return SU2_E_INVAL;
    lat->timing = enable != 0;
    return SU2_OK;
}

}  // extern "C"
