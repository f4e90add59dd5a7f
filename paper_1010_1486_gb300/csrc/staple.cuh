// staple.cuh -- the staple of one link read straight from global memory
// (one thread per link), shared by the batched and learned kernels.
#pragma once

#include "su2_device.cuh"

namespace su2 {

// Staple of U_mu(x) (Sec. 2), nu ascending, forward then backward term.
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
        v = qadd(v, qmul(qmul(a, qdag(b)), qdag(c)));
        v = qadd(v, qmul(qmul(qdag(d), qdag(e)), f));
    }
    return v;
}

// Forward and backward staple terms of direction nu (Sec. 2), from the six
// links they need: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag and
// U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu).
struct NuLinks {
    float4 nu_xp, mu_xn, nu_x, nu_xpm, mu_xm, nu_xm;
};

template <int MU, int NU>
__device__ __forceinline__ NuLinks load_nu(const float4 *__restrict__ L, const Geom &g, const Coord &x, int lex_p,
                                           int parity)
{
    constexpr int nu = NU;
    const int op = parity ^ 1;
    NuLinks n;
    const int e_xn = lex_fwd(g, x.lex, x.c[nu], nu) >> 1;
    const int e_xm = lex_bwd(g, x.lex, x.c[nu], nu) >> 1;
    const int e_xpm = lex_bwd(g, lex_p, x.c[nu], nu) >> 1;  // x + mu - nu keeps the nu coordinate of x
    n.nu_xp = __ldg(L + link_index(g, nu, op, lex_p >> 1));
    n.mu_xn = __ldg(L + link_index(g, MU, op, e_xn));
    n.nu_x = __ldg(L + link_index(g, nu, parity, x.lex >> 1));
    n.nu_xpm = __ldg(L + link_index(g, nu, parity, e_xpm));
    n.mu_xm = __ldg(L + link_index(g, MU, op, e_xm));
    n.nu_xm = __ldg(L + link_index(g, nu, op, e_xm));
    return n;
}

__device__ __forceinline__ float4 add_nu_terms(float4 v, const NuLinks &n)
{
    const float4 fwd = qmul(qmul(n.nu_xp, qdag(n.mu_xn)), qdag(n.nu_x));
    const float4 bwd = qmul(qmul(qdag(n.nu_xpm), qdag(n.mu_xm)), n.nu_xm);
    return qadd(qadd(v, fwd), bwd);
}

// The three directions nu != MU in ascending order.
template <int MU, int J>
struct OtherDir {
    static constexpr int value = J < MU ? J : J + 1;
};

}  // namespace su2
