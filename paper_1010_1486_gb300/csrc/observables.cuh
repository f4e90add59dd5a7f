// observables.cuh -- per-site plaquette and block-wide fp64 sum, shared by
// the reduction kernels.
#pragma once

#include "link_load.cuh"
#include "su2_device.cuh"

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

// Sum over the six planes mu < nu, in the order (0,1),(0,2),(0,3),(1,2),(1,3),
// (2,3), of (1/2) Tr U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag.
template <bool NC = true>
__device__ __forceinline__ float site_plaquette(const float4 *__restrict__ L, const Geom &g, const Coord &x,
                                                int eo, int parity)
{
    const int op = parity ^ 1;
    float4 u[4];
    int e_fwd[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        u[mu] = load_link<NC>(L + link_index(g, mu, parity, eo));
        e_fwd[mu] = lex_fwd(g, x.lex, x.c[mu], mu) >> 1;
    }
    float sum = 0.0f;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int nu = mu + 1; nu < 4; ++nu) {
            const float4 b = load_link<NC>(L + link_index(g, nu, op, e_fwd[mu]));
            const float4 c = load_link<NC>(L + link_index(g, mu, op, e_fwd[nu]));
            const float4 t = qmul(qmul(u[mu], b), qdag(c));
            sum = __fadd_rn(sum, qmul_re(t, qdag(u[nu])));
        }
    return sum;
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

// (1/2) Tr of U_3(x,0) U_3(x,1) ... U_3(x,Nt-1), multiplied left to right,
// for spatial site xs (lexicographic in x, y, z).
template <bool NC = true>
__device__ __forceinline__ float site_polyakov(const float4 *__restrict__ L, const Geom &g, int xs)
{
    const int rest = xs / g.ns;
    const int x = xs - rest * g.ns;
    const int y = rest % g.ns;
    const int z = rest / g.ns;
    const int p0 = (x + y + z) & 1;
    float4 p = load_link<NC>(L + link_index(g, 3, p0, xs >> 1));
    int t = 1;
    // eight loads in flight, then the eight products in t order
    for (; t + 8 <= g.nt; t += 8) {
        float4 q[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t lex = (int64_t)(t + j) * g.vs + xs;
            q[j] = load_link<NC>(L + link_index(g, 3, (p0 + t + j) & 1, (int)(lex >> 1)));
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) p = qmul(p, q[j]);
    }
    for (; t < g.nt; ++t) {
        const int64_t lex = (int64_t)t * g.vs + xs;
        p = qmul(p, load_link<NC>(L + link_index(g, 3, (p0 + t) & 1, (int)(lex >> 1))));
    }
    return p.x;
}

}  // namespace su2
