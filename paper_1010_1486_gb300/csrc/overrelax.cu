// overrelax.cu -- over-relaxation phases: every link U_mu(x) of one phase is
// replaced by its reflection in the staple, U' = U~^dag U^dag U~^dag with
// U~ = V/k (Adler 1981; Creutz 1987), which keeps (1/2) Tr UV.  The usual
// companion of the Sec. 2 heat bath; not in the paper.  No random numbers:
// the phase reads the staple (as the heat bath) plus the old link and writes
// the new one, 144 bytes per link update.
#include <algorithm>

#include "observables.cuh"
#include "staple.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

constexpr int kOrThreads = 256;
#ifndef SU2_OR_MIN_BLOCKS
#define SU2_OR_MIN_BLOCKS 4
#endif
constexpr int kOrMinBlocks = SU2_OR_MIN_BLOCKS;  // blocks per SM the register budget is set for

struct OrParams {
    float4 *links;
    Geom g;
    int parity;
    double *plaq;  // measuring phases: block partials of the plaquettes of planes (nu < mu, mu)
    const float4 *same[4];   // links of direction d at the phase's parity
    const float4 *other[4];  // ... at the opposite parity
};

// U~^dag from the staple (identity if k = 0), as the heat bath's setup.
__device__ __forceinline__ float4 staple_direction(float4 v)
{
    const float k = __fsqrt_rn(qnorm2(v));
    if (!(k > 0.0f)) return make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    const float inv_k = __frcp_rn(k);
    return make_float4(__fmul_rn(v.x, inv_k), __fmul_rn(-v.y, inv_k), __fmul_rn(-v.z, inv_k),
                       __fmul_rn(-v.w, inv_k));
}

// Persistent grid: warp w takes the rounds of 32 consecutive links w, w + W,
// ... (W warps).  Each loop iteration (three per round) issues the six loads
// of one nu-group of the next round, does one third of the current round's
// update, then folds the loaded group into the next round's staple:
//   part 0  the old link, U~^dag;  part 1  U~^dag U^dag;  part 2  (...) U~^dag
//   and the store.  Lanes past the end work on a clamped index and drop their
// results, so the loop body has no divergent branch.  MEAS: the plaquette
// contributions (1/2) Tr U'S, S the staple terms of nu < MU, as in the
// heat-bath kernels.
template <int MU, bool MEAS>
__global__ void __launch_bounds__(kOrThreads, kOrMinBlocks) or_phase_kernel(const OrParams p)
{
    const int stride = gridDim.x * kOrThreads;
    const int last = p.g.vh - 1;
    int base = blockIdx.x * kOrThreads + (threadIdx.x & ~31);
    int cur = base + (threadIdx.x & 31);
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
        const float4 ut = staple_direction(v_cur);
        float4 v_next = add_nu_terms(make_float4(0.0f, 0.0f, 0.0f, 0.0f), nl);
        float4 sp_next = v_next;
        // ---- part 1
        nl = load_nu_bases<MU, OtherDir<MU, 1>::value>(p.same, p.other, p.g, xn, en, en_p);
        const float4 t = qmul(ut, qdag(old));
        v_next = add_nu_terms(v_next, nl);
        if (MU == 2) sp_next = v_next;
        // ---- part 2
        nl = load_nu_bases<MU, OtherDir<MU, 2>::value>(p.same, p.other, p.g, xn, en, en_p);
        const float4 out = qmul(t, ut);
        if (valid) p.links[li] = out;
        if (MEAS && valid) plaq = __fadd_rn(plaq, qmul_re(out, sp_cur));
        v_next = add_nu_terms(v_next, nl);
        if (MU == 3) sp_next = v_next;
        base += stride;
        cur = nxt;
        v_cur = v_next;
        sp_cur = sp_next;
    }
    if (MEAS) {
        const double total = block_sum((double)plaq);
        if (threadIdx.x == 0) p.plaq[blockIdx.x] = total;
    }
}

template <int MU, bool MEAS>
static cudaError_t launch_or(const OrParams &p, int device, cudaStream_t stream)
{
    static int per_sm[64] = {};
    static int sms[64] = {};
    if (device < 0 || device >= 64) device = 0;
    if (!per_sm[device]) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[device], or_phase_kernel<MU, MEAS>,
                                                                      kOrThreads, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms[device], cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        per_sm[device] = std::max(1, per_sm[device]);
    }
    const int want = (p.g.vh + kOrThreads - 1) / kOrThreads;
    const int grid = std::max(1, std::min(std::min(want, per_sm[device] * sms[device]), kFusedSlots));
    or_phase_kernel<MU, MEAS><<<grid, kOrThreads, 0, stream>>>(p);
    return cudaGetLastError();
}

su2_status launch_or_phase(su2_lattice *lat, int mu, int parity)
{
    OrParams p;
    p.links = lat->links;
    p.g = geom_of(lat);
    p.parity = parity;
    p.plaq = fused_slot(lat, mu, parity, 0);
    set_bases(p.same, p.other, lat, parity);
    cudaError_t e;
    if (p.plaq) {
        switch (mu) {
        case 1: e = launch_or<1, true>(p, lat->device, lat->stream); break;
        case 2: e = launch_or<2, true>(p, lat->device, lat->stream); break;
        default: e = launch_or<3, true>(p, lat->device, lat->stream); break;
        }
    } else {
        switch (mu) {
        case 0: e = launch_or<0, false>(p, lat->device, lat->stream); break;
        case 1: e = launch_or<1, false>(p, lat->device, lat->stream); break;
        case 2: e = launch_or<2, false>(p, lat->device, lat->stream); break;
        default: e = launch_or<3, false>(p, lat->device, lat->stream); break;
        }
    }
    SU2_CUDA(e);
    return SU2_OK;
}

su2_status overrelax_sweeps(su2_lattice *lat, int n)
{
    double *const fused = lat->fused_part;  // only the last sweep measures
    for (int s = 0; s < n; ++s) {
        lat->fused_part = s == n - 1 ? fused : nullptr;
        for (int mu = 0; mu < 4; ++mu)
            for (int parity = 0; parity < 2; ++parity) {
                su2_status st = timing_begin(lat, lat->or_log);
                if (st == SU2_OK) st = launch_or_phase(lat, mu, parity);
                if (st == SU2_OK) st = timing_end(lat, lat->or_log);
                if (st != SU2_OK) {
                    lat->fused_part = fused;
                    return st;
                }
            }
    }
    lat->fused_part = fused;
    return SU2_OK;
}

}  // namespace su2

using namespace su2;

extern "C" {

su2_status su2_overrelax_sweep(su2_lattice *lat, int nsweeps)
{
    if (!lat || nsweeps < 0) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    lat->or_log.used = 0;
    su2_status st = overrelax_sweeps(lat, nsweeps);
    lat->or_log.used = 0;
    return st;
}

su2_status su2_overrelax_phase(su2_lattice *lat, int mu, int parity)
{
    if (!lat || mu < 0 || mu > 3 || (parity != 0 && parity != 1)) return SU2_E_INVAL;
    DeviceGuard guard(lat->device);
    return launch_or_phase(lat, mu, parity);
}

su2_status su2_set_overrelax(su2_lattice *lat, int n_or)
{
    if (!lat || n_or < 0 || n_or > 64) return SU2_E_INVAL;
    lat->overrelax = n_or;
    return SU2_OK;
}

}  // extern "C"
