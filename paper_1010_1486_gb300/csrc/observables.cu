// observables.cu -- mean plaquette and Polyakov loop with their global sums
// (Sec. 4 of Cardoso & Bicudo: per-site plaquette and Polyakov kernels and a
// kernel summing over all sites, here fused into one kernel each).
//
// Per-site values are binary32 (same operation order as the updates); the
// sum is binary64: warp shuffles, then one partial per block, then the last
// block to finish adds the partials in block order, so the result does not
// depend on the order in which blocks run.
#include <algorithm>

#include "observables.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

// dst (+ *idx when idx is given: the measurement slot of a graph replay)
__global__ void __launch_bounds__(kReduceThreads, 4) plaquette_kernel(const float4 *__restrict__ L, Geom g,
                                                                   double *__restrict__ partials,
                                                                   unsigned int *__restrict__ ticket,
                                                                   double *__restrict__ dst,
                                                                   const uint32_t *__restrict__ idx)
{
    float acc = 0.0f;  // per-thread partial in binary32; the block and grid sums are binary64
    const int64_t vol = 2 * (int64_t)g.vh;
    // sites in lexicographic order (both parities interleaved), so the
    // neighbour links a block reads were just read by its neighbours (L2)
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < vol; s += (int64_t)gridDim.x * blockDim.x) {
        const int eo = (int)(s >> 1);
        const int parity = (int)(s & 1) ^ (eo_to_coord(g, eo, 0).lex != 2 * eo);
        const Coord x = eo_to_coord(g, eo, parity);
        acc = __fadd_rn(acc, site_plaquette(L, g, x, eo, parity));
    }
    const double total = block_sum((double)acc);
    finish_reduction(total, partials, ticket, idx ? dst + *idx : dst, 1.0 / (6.0 * (double)vol));
}

// (1/2) Tr of U_3(x,0) U_3(x,1) ... U_3(x,Nt-1), multiplied left to right.
__global__ void __launch_bounds__(kReduceThreads) polyakov_kernel(const float4 *__restrict__ L, Geom g,
                                                                  double *__restrict__ partials,
                                                                  unsigned int *__restrict__ ticket,
                                                                  double *__restrict__ dst,
                                                                  const uint32_t *__restrict__ idx)
{
    float acc = 0.0f;  // per-thread partial in binary32; the block and grid sums are binary64
    for (int xs = blockIdx.x * blockDim.x + threadIdx.x; xs < g.vs; xs += gridDim.x * blockDim.x)
        acc = __fadd_rn(acc, site_polyakov(L, g, xs));
    const double total = block_sum((double)acc);
    finish_reduction(total, partials, ticket, idx ? dst + *idx : dst, 1.0 / (double)g.vs);
}

su2_status launch_plaquette(su2_lattice *lat, double *dst)
{
    const Geom g = geom_of(lat);
    // persistent grid (4 blocks of 256 per SM): each thread sums several
    // sites, one block reduction per block
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, lat->device);
    const int grid = grid_for(lat->vol, kReduceThreads, std::min(lat->scratch.partials_cap, 4 * sms));
    plaquette_kernel<<<grid, kReduceThreads, 0, lat->stream>>>(lat->links, g, lat->scratch.partials,
                                                               lat->scratch.ticket, dst,
                                                               lat->capturing ? lat->d_ctr + 1 : nullptr);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

// Ordered sum of the fused-plaquette slot region (one block).
__global__ void __launch_bounds__(kReduceThreads) fused_plaquette_kernel(const double *__restrict__ part, int n,
                                                                        double scale, double *__restrict__ dst,
                                                                        const uint32_t *__restrict__ idx)
{
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
    v = block_sum(v);
    if (threadIdx.x == 0) *(idx ? dst + *idx : dst) = v * scale;
}

su2_status fused_begin(su2_lattice *lat)
{
    if (lat->scratch.partials_cap < kFusedRegion) {
        set_last_error("reduction scratch too small for the fused plaquette");
        return SU2_E_INVAL;
    }
    SU2_CUDA(cudaMemsetAsync(lat->scratch.partials, 0, sizeof(double) * kFusedRegion, lat->stream));
    lat->fused_part = lat->scratch.partials;
    return SU2_OK;
}

su2_status fused_finish(su2_lattice *lat, double *dst)
{
    lat->fused_part = nullptr;
    fused_plaquette_kernel<<<1, kReduceThreads, 0, lat->stream>>>(lat->scratch.partials, kFusedRegion,
                                                                 1.0 / (6.0 * (double)lat->vol), dst,
                                                                 lat->capturing ? lat->d_ctr + 1 : nullptr);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status launch_polyakov(su2_lattice *lat, double *dst)
{
    const Geom g = geom_of(lat);
    const int grid = grid_for(g.vs, kReduceThreads, 152 * 8);
    polyakov_kernel<<<grid, kReduceThreads, 0, lat->stream>>>(lat->links, g, lat->scratch.partials,
                                                              lat->scratch.ticket + 1, dst,
                                                              lat->capturing ? lat->d_ctr + 1 : nullptr);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

}  // namespace su2

using namespace su2;

extern "C" {

su2_status su2_plaquette(su2_lattice *lat, double *out)
{
    if (!lat || !out) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    su2_status st = launch_plaquette(lat, lat->scratch.result);
    if (st != SU2_OK) return st;
    SU2_CUDA(cudaMemcpyAsync(out, lat->scratch.result, sizeof(double), cudaMemcpyDeviceToHost, lat->stream));
    SU2_CUDA(cudaStreamSynchronize(lat->stream));
    return SU2_OK;
}

su2_status su2_polyakov(su2_lattice *lat, double *out)
{
    if (!lat || !out) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    su2_status st = launch_polyakov(lat, lat->scratch.result + 1);
    if (st != SU2_OK) return st;
    SU2_CUDA(cudaMemcpyAsync(out, lat->scratch.result + 1, sizeof(double), cudaMemcpyDeviceToHost, lat->stream));
    SU2_CUDA(cudaStreamSynchronize(lat->stream));
    return SU2_OK;
}

}  // extern "C"
