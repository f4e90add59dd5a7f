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

// (1/2) Tr of U_3(x,0) U_3(x,1) ... U_3(x,Nt-1).  A block of kPolySeg warps
// takes 32 consecutive spatial sites at a time; warp s multiplies, left to
// right, the links of the s-th quarter of the time extent for each of the 32
// sites (each load instruction reads one time slice: 32 consecutive sites,
// two runs of 256 B), with all of a quarter's loads (up to kPolyBatch) in
// flight at once.  Warp 0 then combines the quarters through shared memory
// as (P0 P1)(P2 P3).  Short quarters are padded with the identity, which
// multiplies exactly.
constexpr int kPolySeg = 4;                  // warps per block: quarters of the time extent
constexpr int kPolyThreads = 32 * kPolySeg;  // block size
constexpr int kPolyBatch = 12;               // loads in flight per lane (Nt = 48: one batch)

// PLAQ: the kernel of a measuring sweep also sums the fused-plaquette slot
// region `fused` (kFusedRegion doubles): block b adds its contiguous share in
// index order, and the last block adds the block sums in block order into
// plaq_dst (scaled by plaq_scale), beside the Polyakov loop; `partials` then
// holds 2 gridDim.x doubles and must not overlap the slot region.
template <bool PLAQ>
__global__ void __launch_bounds__(kPolyThreads) polyakov_kernel(const float4 *__restrict__ L, Geom g,
                                                               double *__restrict__ partials,
                                                               unsigned int *__restrict__ ticket,
                                                               double *__restrict__ dst,
                                                               const uint32_t *__restrict__ idx,
                                                               const double *__restrict__ fused,
                                                               double *__restrict__ plaq_dst, double plaq_scale)
{
    __shared__ float4 s_part[kPolySeg][32];
    float acc = 0.0f;  // per-thread partial in binary32; the block and grid sums are binary64
    const int lane = threadIdx.x & 31;
    const int seg = threadIdx.x >> 5;
    const int len = (g.nt + kPolySeg - 1) / kPolySeg;
    const int t_begin = min(seg * len, g.nt);
    const int t_end = min(t_begin + len, g.nt);
    const float4 one = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    // block-uniform loop over groups of 32 sites
    for (int base = blockIdx.x * 32; base < g.vs; base += gridDim.x * 32) {
        const int xs = min(base + lane, g.vs - 1);
        const int rest = xs / g.ns;
        const int x = xs - rest * g.ns;
        const int y = rest % g.ns;
        const int z = rest / g.ns;
        const int p0 = (x + y + z) & 1;
        // a quarter of up to kPolyBatch links (Nt <= 4 kPolyBatch) is one
        // batch of unconditional loads (the index clamped to the quarter),
        // all issued before the first product; longer quarters loop
        auto batch = [&](float4 p, int t) {
            float4 q[kPolyBatch];
#pragma unroll
            for (int j = 0; j < kPolyBatch; ++j) {
                const int tj = min(t + j, t_end - 1);
                const int64_t lex = (int64_t)tj * g.vs + xs;
                q[j] = __ldg(L + link_index(g, 3, (p0 + tj) & 1, (int)(lex >> 1)));
            }
#pragma unroll
            for (int j = 0; j < kPolyBatch; ++j) p = qmul(p, t + j < t_end ? q[j] : one);
            return p;
        };
        float4 p = t_begin < t_end ? batch(one, t_begin) : one;
        for (int t = t_begin + kPolyBatch; t < t_end; t += kPolyBatch) p = batch(p, t);
        s_part[seg][lane] = p;
        __syncthreads();
        if (seg == 0) {
            const float4 p01 = qmul(s_part[0][lane], s_part[1][lane]);
            const float4 p23 = qmul(s_part[2][lane], s_part[3][lane]);
            if (base + lane < g.vs) acc = __fadd_rn(acc, qmul(p01, p23).x);
        }
        __syncthreads();
    }
    const double total_sum = block_sum((double)acc);
    if (!PLAQ) {
        finish_reduction(total_sum, partials, ticket, idx ? dst + *idx : dst, 1.0 / (double)g.vs);
        return;
    }
    const int per = (kFusedRegion + (int)gridDim.x - 1) / (int)gridDim.x;
    const int f0 = min((int)blockIdx.x * per, kFusedRegion);
    const int f1 = min(f0 + per, kFusedRegion);
    double fv = 0.0;
    for (int i = f0 + (int)threadIdx.x; i < f1; i += kPolyThreads) fv += fused[i];
    const double fused_sum = block_sum(fv);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = total_sum;
        partials[gridDim.x + blockIdx.x] = fused_sum;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double vp = 0.0, vq = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        vp += ((volatile double *)partials)[b];
        vq += ((volatile double *)partials)[gridDim.x + b];
    }
    vp = block_sum(vp);
    vq = block_sum(vq);
    if (threadIdx.x == 0) {
        const uint32_t slot = idx ? *idx : 0u;
        dst[slot] = vp * (1.0 / (double)g.vs);
        plaq_dst[slot] = vq * plaq_scale;
        *ticket = 0u;
    }
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

su2_status launch_polyakov(su2_lattice *lat, double *dst)
{
    const Geom g = geom_of(lat);
    const int grid = grid_for(g.vs, 32, std::min(lat->scratch.partials_cap, 152 * 8));
    polyakov_kernel<false><<<grid, kPolyThreads, 0, lat->stream>>>(lat->links, g, lat->scratch.partials,
                                                                     lat->scratch.ticket + 1, dst,
                                                                     lat->capturing ? lat->d_ctr + 1 : nullptr,
                                                                     nullptr, nullptr, 0.0);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status fused_finish_with_polyakov(su2_lattice *lat, double *plaq_dst, double *poly_dst)
{
    const Geom g = geom_of(lat);
    const int grid = grid_for(g.vs, 32, 152 * 8);
    if (lat->scratch.partials_cap < kFusedRegion + 2 * grid) {
        set_last_error("reduction scratch too small for the fused plaquette");
        return SU2_E_INVAL;
    }
    lat->fused_part = nullptr;
    polyakov_kernel<true><<<grid, kPolyThreads, 0, lat->stream>>>(
        lat->links, g, lat->scratch.partials + kFusedRegion, lat->scratch.ticket + 1, poly_dst,
        lat->capturing ? lat->d_ctr + 1 : nullptr, lat->scratch.partials, plaq_dst, 1.0 / (6.0 * (double)lat->vol));
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
