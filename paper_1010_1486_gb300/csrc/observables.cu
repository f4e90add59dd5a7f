// observables.cu -- mean plaquette and Polyakov loop with their global sums
// (Sec. 4 of Cardoso & Bicudo: per-site plaquette and Polyakov kernels and a
// kernel summing over all sites, here fused into one kernel each).
//
// Per-site values are binary32 (same operation order as the updates); the
// sum is binary64: warp shuffles, then one partial per block, then the last
// block to finish adds the partials in block order, so the result does not
// depend on the order in which blocks run.
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

// Block-wide sum of a double; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double warp_sums[32];
    const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) warp_sums[warp] = v;
    __syncthreads();
    v = 0.0;
    if (warp == 0) {
        const unsigned int nwarps = blockDim.x >> 5;
        v = lane < nwarps ? warp_sums[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    }
    __syncthreads();
    return v;
}

// Block partial -> partials[blockIdx]; the last block sums the partials in
// index order and writes scale * total to *dst, then re-arms the ticket.
__device__ __forceinline__ void finish_reduction(double block_total, double *__restrict__ partials,
                                                 unsigned int *__restrict__ ticket, double *__restrict__ dst,
                                                 double scale)
{
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = block_total;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += blockDim.x) v += ((volatile double *)partials)[b];
    v = block_sum(v);
    if (threadIdx.x == 0) {
        *dst = v * scale;
        *ticket = 0u;
    }
}

// Sum over the six planes mu < nu, in the order (0,1),(0,2),(0,3),(1,2),(1,3),
// (2,3), of (1/2) Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag.
__device__ __forceinline__ float site_plaquette(const float4 *__restrict__ L, const Geom &g, const Coord &x,
                                                int eo, int parity)
{
    const int op = parity ^ 1;
    float4 u[4];
    int e_fwd[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        u[mu] = __ldg(L + link_index(g, mu, parity, eo));
        e_fwd[mu] = lex_fwd(g, x.lex, x.c[mu], mu) >> 1;
    }
    float sum = 0.0f;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int nu = mu + 1; nu < 4; ++nu) {
            const float4 b = __ldg(L + link_index(g, nu, op, e_fwd[mu]));
            const float4 c = __ldg(L + link_index(g, mu, op, e_fwd[nu]));
            const float4 t = qmul(qmul(u[mu], b), qdag(c));
            sum = __fadd_rn(sum, qmul_re(t, qdag(u[nu])));
        }
    return sum;
}

__global__ void __launch_bounds__(kReduceThreads) plaquette_kernel(const float4 *__restrict__ L, Geom g,
                                                                   double *__restrict__ partials,
                                                                   unsigned int *__restrict__ ticket,
                                                                   double *__restrict__ dst)
{
    double acc = 0.0;
    const int64_t vol = 2 * (int64_t)g.vh;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < vol; s += (int64_t)gridDim.x * blockDim.x) {
        const int parity = s >= g.vh;
        const int eo = (int)(s - (parity ? g.vh : 0));
        const Coord x = eo_to_coord(g, eo, parity);
        acc += (double)site_plaquette(L, g, x, eo, parity);
    }
    const double total = block_sum(acc);
    finish_reduction(total, partials, ticket, dst, 1.0 / (6.0 * (double)vol));
}

// (1/2) Tr of U_3(x,0) U_3(x,1) ... U_3(x,Nt-1), multiplied left to right.
__global__ void __launch_bounds__(kReduceThreads) polyakov_kernel(const float4 *__restrict__ L, Geom g,
                                                                  double *__restrict__ partials,
                                                                  unsigned int *__restrict__ ticket,
                                                                  double *__restrict__ dst)
{
    double acc = 0.0;
    for (int xs = blockIdx.x * blockDim.x + threadIdx.x; xs < g.vs; xs += gridDim.x * blockDim.x) {
        int rest = xs / g.ns;
        const int x = xs - rest * g.ns;
        const int y = rest % g.ns;
        const int z = rest / g.ns;
        const int p0 = (x + y + z) & 1;
        float4 p = __ldg(L + link_index(g, 3, p0, xs >> 1));
        for (int t = 1; t < g.nt; ++t) {
            const int64_t lex = (int64_t)t * g.vs + xs;
            p = qmul(p, __ldg(L + link_index(g, 3, (p0 + t) & 1, (int)(lex >> 1))));
        }
        acc += (double)p.x;
    }
    const double total = block_sum(acc);
    finish_reduction(total, partials, ticket, dst, 1.0 / (double)g.vs);
}

su2_status launch_plaquette(su2_lattice *lat, double *dst)
{
    const Geom g = geom_of(lat);
    const int grid = grid_for(lat->vol, kReduceThreads, 152 * 8);
    plaquette_kernel<<<grid, kReduceThreads, 0, lat->stream>>>(lat->links, g, lat->scratch.partials,
                                                               lat->scratch.ticket, dst);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status launch_polyakov(su2_lattice *lat, double *dst)
{
    const Geom g = geom_of(lat);
    const int grid = grid_for(g.vs, kReduceThreads, 152 * 8);
    polyakov_kernel<<<grid, kReduceThreads, 0, lat->stream>>>(lat->links, g, lat->scratch.partials,
                                                              lat->scratch.ticket + 1, dst);
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
