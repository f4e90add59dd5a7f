// noalloc.cu -- mean plaquette of links that already sit in device memory,
// computed without allocating anything.
//
// Some callers cannot allocate device memory at the point where they want an
// observable: a host program that hands every byte of the GPU to its own
// memory pool up front and forbids outside allocations (a serving process or
// another framework's runtime), or code that runs where an allocation would
// stall or is not allowed.  For them this entry point takes the links and the
// output location from the caller and keeps its reduction scratch in a fixed
// array compiled into the library (every GPU that loads libsu2 holds it until
// the process exits).  The paper has no counterpart.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "observables.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

// Scratch of su2_plaquette_noalloc: [0, 256) reduction ticket, then one fp64
// partial per block of 4096 sites (16384 blocks).  Host code must not use
// the name as an address; scratch_address() looks the address up per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[256 + 8 * 16384];

namespace su2 {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaSitesPerBlock = 4096;  // block b sums sites [4096 b, 4096 b + 4096)
constexpr int kNaMaxBlocks = 16384;     // so at most 67,108,864 sites
constexpr long long kNaMaxSites = (long long)kNaSitesPerBlock * kNaMaxBlocks;
static_assert(sizeof(g_noalloc_scratch) == 256 + sizeof(double) * kNaMaxBlocks, "scratch layout");

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// The device address of g_noalloc_scratch on the current device, looked up
// once per device (host code may not use the symbol itself as an address).
su2_status scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) {
        set_last_error("su2_plaquette_noalloc: device ordinal out of range");
        return SU2_E_INVAL;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[device] = (unsigned char *)p;
    }
    *out = g_scratch_addr[device];
    return SU2_OK;
}

}  // namespace

// Same per-site values as plaquette_kernel; the partition of sites into
// blocks is fixed (4096 sites each) instead of grid-strided.
__global__ void __launch_bounds__(kNaThreads) plaquette_noalloc_kernel(const float4 *__restrict__ L, Geom g,
                                                                       unsigned char *__restrict__ scratch,
                                                                       double *__restrict__ out)
{
    unsigned int *ticket = (unsigned int *)scratch;
    double *partials = (double *)(scratch + 256);
    const int64_t vol = 2 * (int64_t)g.vh;
    const int64_t begin = (int64_t)blockIdx.x * kNaSitesPerBlock;
    const int64_t end = begin + kNaSitesPerBlock < vol ? begin + kNaSitesPerBlock : vol;
    double acc = 0.0;
    for (int64_t s = begin + threadIdx.x; s < end; s += blockDim.x) {
        const int parity = s >= g.vh;
        const int eo = (int)(s - (parity ? g.vh : 0));
        const Coord x = eo_to_coord(g, eo, parity);
        acc += (double)site_plaquette(L, g, x, eo, parity);
    }
    const double total = block_sum(acc);
    finish_reduction(total, partials, ticket, out, 1.0 / (6.0 * (double)vol));
}

}  // namespace su2

using namespace su2;

extern "C" su2_status su2_plaquette_noalloc(const void *links, int ns, int nt, double *out, void *cuda_stream)
{
    if (!links || !out) {
        set_last_error("su2_plaquette_noalloc: links and out must be device pointers");
        return SU2_E_INVAL;
    }
    if (ns < 2 || nt < 2 || (ns & 1) || (nt & 1)) {
        set_last_error("su2_plaquette_noalloc: extents must be even and >= 2");
        return SU2_E_INVAL;
    }
    const long long vol = (long long)ns * ns * ns * nt;
    if (vol > kNaMaxSites) {
        set_last_error("su2_plaquette_noalloc: " + std::to_string(vol) + " sites exceed the limit of " +
                       std::to_string(kNaMaxSites) + " sites of the fixed scratch array");
        return SU2_E_INVAL;
    }
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));
    unsigned char *scratch = nullptr;
    su2_status st = scratch_address(dev, &scratch);
    if (st != SU2_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // the ticket must start at zero; the partials are overwritten by every block
    SU2_CUDA(cudaMemsetAsync(scratch, 0, sizeof(unsigned int), stream));
    Geom g;
    g.ns = ns;
    g.nt = nt;
    g.vh = (int)(vol / 2);
    g.vs = ns * ns * ns;
    g.div_ns = make_fastdiv((uint32_t)ns);
    int stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
        g.ext[mu] = mu == 3 ? nt : ns;
        g.stride[mu] = stride;
        g.wrap[mu] = (g.ext[mu] - 1) * stride;
        stride *= g.ext[mu];
    }
    const int blocks = (int)((vol + kNaSitesPerBlock - 1) / kNaSitesPerBlock);
    plaquette_noalloc_kernel<<<blocks, kNaThreads, 0, stream>>>((const float4 *)links, g, scratch, out);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}
