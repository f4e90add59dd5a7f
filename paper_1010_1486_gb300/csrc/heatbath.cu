// heatbath.cu -- the checkerboard heat-bath phase kernel and the sweep
// schedule (Sec. 2 update, Sec. 4 schedule of Cardoso & Bicudo, LAT2010).
//
// One phase (mu, parity) redraws every link U_mu(x) with parity(x) = parity.
// Its staple reads only links of the other three directions (both parities)
// and U_mu of the opposite parity, none of which the phase writes, so every
// thread works independently and the loads may use the read-only path.
#include <cstdio>

#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

// Sums `value` over the block and adds it to one of kTrialSlots counters.
__device__ __forceinline__ void block_add_trials(unsigned int value, unsigned long long *slot)
{
    __shared__ unsigned int warp_sums[32];
    const unsigned int lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const unsigned int w = __reduce_add_sync(0xffffffffu, value);
    if (lane == 0) warp_sums[warp] = w;
    __syncthreads();
    if (warp == 0) {
        const unsigned int nwarps = blockDim.x >> 5;
        unsigned int v = lane < nwarps ? warp_sums[lane] : 0u;
        v = __reduce_add_sync(0xffffffffu, v);
        if (lane == 0 && v) atomicAdd(slot, (unsigned long long)v);
    }
}

// Staple of U_mu(x) (Sec. 2):
//   V = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
//                    + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)
// nu ascending, forward term first, accumulated from zero.
template <int MU>
__device__ __forceinline__ float4 staple(const float4 *__restrict__ L, const Geom &g, const Coord &x, int eo,
                                         int parity)
{
    const int op = parity ^ 1;
    const Coord xp = step(g, x, MU, +1);
    const int e_xp = coord_to_eo(g, xp);
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == MU) continue;
        const int e_xn = coord_to_eo(g, step(g, x, nu, +1));
        const Coord xm = step(g, x, nu, -1);
        const int e_xm = coord_to_eo(g, xm);
        const int e_xpm = coord_to_eo(g, step(g, xp, nu, -1));
        const float4 u_nu_xp = __ldg(L + link_index(g, nu, op, e_xp));
        const float4 u_mu_xn = __ldg(L + link_index(g, MU, op, e_xn));
        const float4 u_nu_x = __ldg(L + link_index(g, nu, parity, eo));
        const float4 u_nu_xpm = __ldg(L + link_index(g, nu, parity, e_xpm));
        const float4 u_mu_xm = __ldg(L + link_index(g, MU, op, e_xm));
        const float4 u_nu_xm = __ldg(L + link_index(g, nu, op, e_xm));
        const float4 fwd = qmul(qmul(u_nu_xp, qdag(u_mu_xn)), qdag(u_nu_x));
        const float4 bwd = qmul(qmul(qdag(u_nu_xpm), qdag(u_mu_xm)), u_nu_xm);
        v = qadd(v, fwd);
        v = qadd(v, bwd);
    }
    return v;
}

template <int MU>
__global__ void __launch_bounds__(kHbThreads) hb_phase_kernel(float4 *__restrict__ links, Geom g, int parity,
                                                               float beta, uint32_t k0, uint32_t k1,
                                                               uint32_t sweep,
                                                               unsigned long long *__restrict__ trial_slots,
                                                               unsigned int *__restrict__ flags)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int trials = 0;
    if (i < g.vh) {
        const Coord x = eo_to_coord(g, i, parity);
        const float4 v = staple<MU>(links, g, x, i, parity);
        float4 out;
        const int n = heatbath_draw(v, beta, k0, k1, (uint32_t)i, sweep, (uint32_t)parity, (uint32_t)MU, out);
        if (n > 0) {
            links[link_index(g, MU, parity, i)] = out;
            trials = (unsigned int)n;
        } else {
            atomicAdd(&flags[0], 1u);  // trial cap: the link keeps its old value
            trials = (unsigned int)kMaxTrials;
        }
    }
    block_add_trials(trials, &trial_slots[(2 * MU + parity) * kTrialSlots + (blockIdx.x & (kTrialSlots - 1))]);
}

su2_status launch_hb_phase(su2_lattice *lat, int mu, int parity, uint32_t sweep)
{
    const Geom g = geom_of(lat);
    const int grid = (g.vh + kHbThreads - 1) / kHbThreads;
    const float beta = (float)lat->beta;
    const uint32_t k0 = (uint32_t)lat->seed, k1 = (uint32_t)(lat->seed >> 32);
    unsigned long long *slots = lat->scratch.trials;
    unsigned int *flags = lat->scratch.flags;
    switch (mu) {
    case 0: hb_phase_kernel<0><<<grid, kHbThreads, 0, lat->stream>>>(lat->links, g, parity, beta, k0, k1, sweep, slots, flags); break;
    case 1: hb_phase_kernel<1><<<grid, kHbThreads, 0, lat->stream>>>(lat->links, g, parity, beta, k0, k1, sweep, slots, flags); break;
    case 2: hb_phase_kernel<2><<<grid, kHbThreads, 0, lat->stream>>>(lat->links, g, parity, beta, k0, k1, sweep, slots, flags); break;
    default: hb_phase_kernel<3><<<grid, kHbThreads, 0, lat->stream>>>(lat->links, g, parity, beta, k0, k1, sweep, slots, flags); break;
    }
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

// ------------------------------------------------------------- timing
static su2_status timed_phase(su2_lattice *lat, int mu, int parity, uint32_t sweep)
{
    if (!lat->timing) return launch_hb_phase(lat, mu, parity, sweep);
    while (lat->events.size() < lat->events_used + 2) {
        cudaEvent_t e;
        SU2_CUDA(cudaEventCreate(&e));
        lat->events.push_back(e);
    }
    cudaEvent_t b = lat->events[lat->events_used], e = lat->events[lat->events_used + 1];
    lat->events_used += 2;
    SU2_CUDA(cudaEventRecord(b, lat->stream));
    su2_status st = launch_hb_phase(lat, mu, parity, sweep);
    if (st != SU2_OK) return st;
    SU2_CUDA(cudaEventRecord(e, lat->stream));
    return SU2_OK;
}

static su2_status read_timing(su2_lattice *lat, su2_stats *stats)
{
    double ms = 0.0;
    if (lat->timing && lat->events_used) {
        SU2_CUDA(cudaEventSynchronize(lat->events[lat->events_used - 1]));
        for (size_t i = 0; i + 1 < lat->events_used; i += 2) {
            float t = 0.0f;
            SU2_CUDA(cudaEventElapsedTime(&t, lat->events[i], lat->events[i + 1]));
            ms += t;
        }
    }
    if (stats) {
        stats->kernel_ms = ms;
        stats->timed = lat->timing ? 1u : 0u;
    }
    lat->events_used = 0;
    return SU2_OK;
}

static su2_status one_sweep(su2_lattice *lat)
{
    for (int mu = 0; mu < 4; ++mu)
        for (int parity = 0; parity < 2; ++parity) {
            su2_status st = timed_phase(lat, mu, parity, lat->sweep);
            if (st != SU2_OK) return st;
        }
    lat->sweep += 1;
    return SU2_OK;
}

static su2_status ensure_history(su2_lattice *lat, int n)
{
    if (n <= lat->scratch.history_cap) return SU2_OK;
    device_free(lat->scratch.history, sizeof(double) * 2 * (size_t)lat->scratch.history_cap, lat->device,
                lat->stream);
    lat->scratch.history = (double *)device_alloc(sizeof(double) * 2 * (size_t)n, lat->device, lat->stream);
    lat->scratch.history_cap = lat->scratch.history ? n : 0;
    if (!lat->scratch.history) {
        set_last_error("device allocation of the measurement history failed");
        return SU2_E_NOMEM;
    }
    return SU2_OK;
}

}  // namespace su2

using namespace su2;

extern "C" {

su2_status su2_generate(su2_lattice *lat, int nsweeps, int measure_every, int reunit_every, double *plaq,
                        double *poly, su2_stats *stats)
{
    if (!lat || nsweeps < 0 || measure_every < 0 || reunit_every < 0) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    const int nmeas = measure_every > 0 ? nsweeps / measure_every : 0;
    su2_status st = ensure_history(lat, nmeas);
    if (st != SU2_OK) return st;
    if ((st = launch_clear_counters(lat)) != SU2_OK) return st;
    lat->events_used = 0;
    int m = 0;
    for (int s = 1; s <= nsweeps; ++s) {
        if ((st = one_sweep(lat)) != SU2_OK) return st;
        if (reunit_every > 0 && s % reunit_every == 0 && (st = launch_reunitarize(lat)) != SU2_OK) return st;
        if (measure_every > 0 && s % measure_every == 0) {
            if ((st = launch_plaquette(lat, lat->scratch.history + m)) != SU2_OK) return st;
            if ((st = launch_polyakov(lat, lat->scratch.history + lat->scratch.history_cap + m)) != SU2_OK) return st;
            ++m;
        }
    }
    if (nmeas > 0 && plaq)
        SU2_CUDA(cudaMemcpyAsync(plaq, lat->scratch.history, sizeof(double) * nmeas, cudaMemcpyDeviceToHost,
                                 lat->stream));
    if (nmeas > 0 && poly)
        SU2_CUDA(cudaMemcpyAsync(poly, lat->scratch.history + lat->scratch.history_cap, sizeof(double) * nmeas,
                                 cudaMemcpyDeviceToHost, lat->stream));
    if (stats) memset(stats, 0, sizeof *stats);
    st = collect_stats(lat, stats, (uint64_t)nsweeps);
    if (stats) stats->kernel_launches = (uint32_t)(8 * nsweeps);
    su2_status st2 = read_timing(lat, stats);
    return st != SU2_OK ? st : st2;
}

su2_status su2_heatbath_sweep(su2_lattice *lat, int nsweeps, su2_stats *stats)
{
    if (!lat || nsweeps < 0) return SU2_E_INVAL;
    if (stats) return su2_generate(lat, nsweeps, 0, 0, nullptr, nullptr, stats);
    DeviceGuard guard(lat->device);
    su2_status st;
    lat->events_used = 0;
    for (int s = 0; s < nsweeps; ++s)
        if ((st = one_sweep(lat)) != SU2_OK) return st;
    if (lat->timing) lat->events_used = 0;
    return SU2_OK;
}

su2_status su2_heatbath_phase(su2_lattice *lat, int mu, int parity)
{
    if (!lat || mu < 0 || mu > 3 || (parity != 0 && parity != 1)) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    return launch_hb_phase(lat, mu, parity, lat->sweep);
}

}  // extern "C"
