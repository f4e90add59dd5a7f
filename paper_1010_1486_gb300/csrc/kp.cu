// kp.cu -- heat-bath phase with the Kennedy-Pendleton a0 sampler
// (Phys. Lett. B 156 (1985) 393).  Same law as Creutz's method (Sec. 2
// heat bath), but at large beta k nearly every trial is accepted, so there
// is no rejection loop to balance: one thread per link, persistent grid, the
// 18 staple links of the next link loaded before the draw of the current one.
//
// With a0 = 1 - 2u the law of u is u^{1/2} sqrt(1 - u) exp(-2 beta k u) on
// [0, 1]; a trial draws u = -(ln r1 + cos^2(2 pi r2) ln r3) / (2 beta k) and
// accepts iff u <= 1 and r4^2 <= 1 - u (block t of the KP stream).  Links with
// beta k < 2 are drawn by Creutz's method exactly as the plain kernel does.
#include <algorithm>

#include "staple.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

constexpr int kKpThreads = 256;
constexpr float kKpMinBk = 2.0f;
constexpr uint32_t kKennedyPendleton = 5u;

struct KpParams {
    float4 *links;
    Geom g;
    RoundKeys rk;
    int parity;
    float beta;
    uint32_t sweep;
    unsigned long long *trial_slots;
    unsigned int *flags;
    const unsigned int *gate;  // skip the phase while *gate == 1 (learned sweeps)
};

// Returns the number of trials (0: cap hit, out unchanged).
template <int MU>
__device__ __forceinline__ int kp_draw(float4 v, float beta, const RoundKeys &rk, uint32_t eo, uint32_t sweep,
                                       uint32_t parity, float4 &out)
{
    const float k = __fsqrt_rn(qnorm2(v));
    const float bk = __fmul_rn(beta, k);
    if (!(bk >= kKpMinBk)) return heatbath_draw(v, beta, rk, eo, sweep, parity, MU, out);
    const float inv_k = __fdiv_rn(1.0f, k);
    const float4 ut = make_float4(__fmul_rn(v.x, inv_k), __fmul_rn(-v.y, inv_k), __fmul_rn(-v.z, inv_k),
                                  __fmul_rn(-v.w, inv_k));
    const float two_bk = __fmul_rn(2.0f, bk);
    const uint32_t sw = stream_word(kKennedyPendleton, parity, MU);
    float a0 = 0.0f;
    int trials = 0;
    for (int t = 0; t < kMaxTrials; ++t) {
        const uint4 w = philox_rk(make_uint4(eo, sweep, sw, (uint32_t)t), rk);
        float sn, cs;
        sincos_2pi(uniform01(w.y), sn, cs);
        const float num = __fmaf_rn(__fmul_rn(cs, cs), log_series(uniform01(w.z)), log_series(uniform01(w.x)));
        const float lam2 = __fdiv_rn(-num, two_bk);
        const float r4 = uniform01(w.w);
        if (lam2 <= 1.0f && __fmul_rn(r4, r4) <= __fsub_rn(1.0f, lam2)) {
            a0 = __fmaf_rn(-2.0f, lam2, 1.0f);
            trials = t + 1;
            break;
        }
    }
    if (trials == 0) return 0;
    out = direction_update(a0, ut, philox_rk(make_uint4(eo, sweep, stream_word(kDirection, parity, MU), 0u), rk));
    return trials;
}

template <int MU>
__global__ void __launch_bounds__(kKpThreads) kp_phase_kernel(const KpParams p)
{
    if (p.gate != nullptr && *(volatile const unsigned int *)p.gate == 1u) return;
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int trials = 0;
    NuLinks n0, n1, n2;
    if (i < p.g.vh) {
        const Coord x = eo_to_coord(p.g, i, p.parity);
        const int lex_p = lex_fwd(p.g, x.lex, x.c[MU], MU);
        n0 = load_nu<MU, OtherDir<MU, 0>::value>(p.links, p.g, x, lex_p, p.parity);
        n1 = load_nu<MU, OtherDir<MU, 1>::value>(p.links, p.g, x, lex_p, p.parity);
        n2 = load_nu<MU, OtherDir<MU, 2>::value>(p.links, p.g, x, lex_p, p.parity);
    }
    while (i < p.g.vh) {
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        v = add_nu_terms(v, n0);
        v = add_nu_terms(v, n1);
        v = add_nu_terms(v, n2);
        const int inext = i + stride;
        if (inext < p.g.vh) {
            const Coord x = eo_to_coord(p.g, inext, p.parity);
            const int lex_p = lex_fwd(p.g, x.lex, x.c[MU], MU);
            n0 = load_nu<MU, OtherDir<MU, 0>::value>(p.links, p.g, x, lex_p, p.parity);
            n1 = load_nu<MU, OtherDir<MU, 1>::value>(p.links, p.g, x, lex_p, p.parity);
            n2 = load_nu<MU, OtherDir<MU, 2>::value>(p.links, p.g, x, lex_p, p.parity);
        }
        float4 out;
        const int n = kp_draw<MU>(v, p.beta, p.rk, (uint32_t)i, p.sweep, (uint32_t)p.parity, out);
        if (n > 0) {
            p.links[link_index(p.g, MU, p.parity, i)] = out;
            trials += (unsigned int)n;
        } else {
            atomicAdd(&p.flags[0], 1u);  // trial cap: the link keeps its old value
            trials += (unsigned int)kMaxTrials;
        }
        i = inext;
    }
    const unsigned int wsum = __reduce_add_sync(0xffffffffu, trials);
    if ((threadIdx.x & 31) == 0 && wsum)
        atomicAdd(&p.trial_slots[(2 * MU + p.parity) * kTrialSlots + ((blockIdx.x * (kKpThreads / 32) + (threadIdx.x >> 5)) &
                                                                      (kTrialSlots - 1))],
                  (unsigned long long)wsum);
}

template <int MU>
static cudaError_t launch_kp(const KpParams &p, int device, cudaStream_t stream)
{
    static int per_sm[64] = {};
    static int sms[64] = {};
    if (device < 0 || device >= 64) device = 0;
    if (!per_sm[device]) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[device], kp_phase_kernel<MU>,
                                                                      kKpThreads, 0);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms[device], cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        per_sm[device] = std::max(1, per_sm[device]);
    }
    const int want = (p.g.vh + kKpThreads - 1) / kKpThreads;
    const int grid = std::max(1, std::min(want, per_sm[device] * sms[device]));
    kp_phase_kernel<MU><<<grid, kKpThreads, 0, stream>>>(p);
    return cudaGetLastError();
}

su2_status launch_kp_phase(su2_lattice *lat, int mu, int parity, uint32_t sweep, const unsigned int *gate)
{
    KpParams p;
    p.links = lat->links;
    p.g = geom_of(lat);
    p.rk = make_round_keys(lat->seed);
    p.parity = parity;
    p.beta = (float)lat->beta;
    p.sweep = sweep;
    p.trial_slots = lat->scratch.trials;
    p.flags = lat->scratch.flags;
    p.gate = gate;
    cudaError_t e;
    switch (mu) {
    case 0: e = launch_kp<0>(p, lat->device, lat->stream); break;
    case 1: e = launch_kp<1>(p, lat->device, lat->stream); break;
    case 2: e = launch_kp<2>(p, lat->device, lat->stream); break;
    default: e = launch_kp<3>(p, lat->device, lat->stream); break;
    }
    SU2_CUDA(e);
    return SU2_OK;
}

}  // namespace su2

extern "C" su2_status su2_set_sampler(su2_lattice *lat, int sampler)
{
    if (!lat || (sampler != SU2_SAMPLER_CREUTZ && sampler != SU2_SAMPLER_KP)) return SU2_E_INVAL;
    lat->sampler = sampler;
    return SU2_OK;
}
