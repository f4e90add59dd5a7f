// kp_device.cuh -- the Kennedy-Pendleton a0 trial (Phys. Lett. B 156 (1985)
// 393), shared by the single-lattice and the batched phase kernels.
//
// With a0 = 1 - 2u the heat-bath law of Sec. 2 becomes u^{1/2} sqrt(1 - u)
// exp(-2 beta k u) on [0, 1]; a trial draws u = -(ln r1 + cos^2(2 pi r2) ln r3)
// / (2 beta k) and accepts iff u <= 1 and r4^2 <= 1 - u.  Trial t uses block t
// of the Kennedy-Pendleton stream; links with beta k < 2 are drawn by
// Creutz's method instead.
#pragma once

#include "su2_device.cuh"

namespace su2 {

constexpr float kKpMinBk = 2.0f;
constexpr uint32_t kKennedyPendleton = 5u;  // stream kind of the trials

// One trial (block t of the KP stream): a0 = 1 - 2 u, and whether it is
// accepted.
__device__ __forceinline__ bool kp_trial(uint4 w, float two_bk, float &a0)
{
    float sn, cs;
    sincos_2pi(uniform01(w.y), sn, cs);
    const float num = __fmaf_rn(__fmul_rn(cs, cs), log_series(uniform_log(w.z)), log_series(uniform_log(w.x)));
    const float lam2 = __fdiv_rn(-num, two_bk);
    const float r4 = uniform01(w.w);
    a0 = __fmaf_rn(-2.0f, lam2, 1.0f);
    return lam2 <= 1.0f && __fmul_rn(r4, r4) <= __fsub_rn(1.0f, lam2);
}

}  // namespace su2
