// staple.cuh -- the staple of one link read straight from global memory
// (one thread per link), shared by the batched and learned kernels.
#pragma once

#include "link_load.cuh"
#include "su2_device.cuh"

namespace su2 {

// Staple of U_mu(x) (Sec. 2), nu ascending, forward then backward term, each
// term's second product fused with the running sum (qmul_add).
template <int MU>
__device__ __forceinline__ float4 staple_at(const float4 *__restrict__ L, const Geom &g, const Coord &x, int parity)
{
    const int op = parity ^ 1;
    const int lex_p = lex_fwd(g, x.lex, x.c[MU], MU);
    float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == MU) continue;
        const int e_xn = lex_fwd(g, x.lex, x.c[nu], nu) >> 1;
        const int e_xm = lex_bwd(g, x.lex, x.c[nu], nu) >> 1;
        const int e_xpm = lex_bwd(g, lex_p, x.c[nu], nu) >> 1;
        const float4 a = __ldg(L + link_index(g, nu, op, lex_p >> 1));
        const float4 b = __ldg(L + link_index(g, MU, op, e_xn));
        const float4 c = __ldg(L + link_index(g, nu, parity, x.lex >> 1));
        const float4 d = __ldg(L + link_index(g, nu, parity, e_xpm));
        const float4 e = __ldg(L + link_index(g, MU, op, e_xm));
        const float4 f = __ldg(L + link_index(g, nu, op, e_xm));
        v = qmul_add(qmul(a, qdag(b)), qdag(c), v);
        v = qmul_add(qmul(qdag(d), qdag(e)), f, v);
    }
    return v;
}

// Forward and backward staple terms of direction nu (Sec. 2), from the six
// links they need: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag and
// U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) (loaded by load_nu_eo below).
struct NuLinks {
    float4 nu_xp, mu_xn, nu_x, nu_xpm, mu_xm, nu_xm;
};

__device__ __forceinline__ float4 add_nu_terms(float4 v, const NuLinks &n)
{
    v = qmul_add(qmul(n.nu_xp, qdag(n.mu_xn)), qdag(n.nu_x), v);
    return qmul_add(qmul(qdag(n.nu_xpm), qdag(n.mu_xm)), n.nu_xm, v);
}

// Even/odd neighbour indices straight from the coordinates.  The strides of
// y, z, t are even, so (lex +- stride) >> 1 = eo +- stride/2 (and the
// periodic jump is even too); in x the step depends on the parity of x0.
// Index of x + nu:
template <int NU>
__device__ __forceinline__ int eo_fwd(const Geom &g, const Coord &x, int eo)
{
    if (NU == 0) return eo + (x.c[0] & 1) - (x.c[0] == g.ns - 1 ? (g.ns >> 1) : 0);
    return eo + (x.c[NU] == g.ext[NU] - 1 ? -(g.wrap[NU] >> 1) : (g.stride[NU] >> 1));
}

// eo(x - nu) - eo(x); the same for x + mu - nu against x + mu (mu != nu:
// the step to x + mu keeps x0 and its parity, or is in x itself).
template <int NU>
__device__ __forceinline__ int eo_bwd_offset(const Geom &g, const Coord &x)
{
    if (NU == 0) return (x.c[0] & 1) - 1 + (x.c[0] == 0 ? (g.ns >> 1) : 0);
    return x.c[NU] == 0 ? (g.wrap[NU] >> 1) : -(g.stride[NU] >> 1);
}

// The six links of direction nu with the indices above; eo = index of x,
// e_p = index of x + mu.  NC: read-only path (see load_link).
template <int MU, int NU, bool NC = true>
__device__ __forceinline__ NuLinks load_nu_eo(const float4 *__restrict__ L, const Geom &g, const Coord &x, int eo,
                                              int e_p, int parity)
{
    const int op = parity ^ 1;
    const float4 *__restrict__ nu_same = L + (uint32_t)(2 * NU + parity) * (uint32_t)g.vh;
    const float4 *__restrict__ nu_other = L + (uint32_t)(2 * NU + op) * (uint32_t)g.vh;
    const float4 *__restrict__ mu_other = L + (uint32_t)(2 * MU + op) * (uint32_t)g.vh;
    const int off_m = eo_bwd_offset<NU>(g, x);
    NuLinks n;
    n.nu_xp = load_link<NC>(nu_other + (uint32_t)e_p);
    n.mu_xn = load_link<NC>(mu_other + (uint32_t)eo_fwd<NU>(g, x, eo));
    n.nu_x = load_link<NC>(nu_same + (uint32_t)eo);
    n.nu_xpm = load_link<NC>(nu_same + (uint32_t)(e_p + off_m));
    n.mu_xm = load_link<NC>(mu_other + (uint32_t)(eo + off_m));
    n.nu_xm = load_link<NC>(nu_other + (uint32_t)(eo + off_m));
    return n;
}

// As load_nu_eo with the launch's array bases precomputed: same[d] = links of
// direction d at the phase's parity, other[d] = at the opposite parity.
template <int MU, int NU>
__device__ __forceinline__ NuLinks load_nu_bases(const float4 *const *same, const float4 *const *other, const Geom &g,
                                                 const Coord &x, int eo, int e_p)
{
    const int off_m = eo_bwd_offset<NU>(g, x);
    NuLinks n;
    n.nu_xp = __ldg(other[NU] + (uint32_t)e_p);
    n.mu_xn = __ldg(other[MU] + (uint32_t)eo_fwd<NU>(g, x, eo));
    n.nu_x = __ldg(same[NU] + (uint32_t)eo);
    n.nu_xpm = __ldg(same[NU] + (uint32_t)(e_p + off_m));
    n.mu_xm = __ldg(other[MU] + (uint32_t)(eo + off_m));
    n.nu_xm = __ldg(other[NU] + (uint32_t)(eo + off_m));
    return n;
}

// The three directions nu != MU in ascending order.
template <int MU, int J>
struct OtherDir {
    static constexpr int value = J < MU ? J : J + 1;
};

}  // namespace su2
