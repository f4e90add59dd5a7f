// wilson.cu -- space-time Wilson loops W(R, T) (the observables that come
// after the Sec. 4 plaquette and Polyakov loop; not in the paper).
//
// For a site x, a spatial direction i and extents R (along i), T (along t):
//   S_R(y) = U_i(y) U_i(y+i) ... U_i(y+(R-1)i),  T_T(y) = U_t(y) ... U_t(y+(T-1)t),
//   A = S_R(x) T_T(x+Ri),  B = T_T(x) S_R(x+Tt),  loop = (1/2) Tr A B^dag = A . B,
// line products left to right, binary32 per loop (the link-arithmetic
// contract), binary64 mean over x and i = 0, 1, 2.  One launch per T: each
// thread takes (site, direction) items and, for R = 1 .. rmax, extends S_R
// and the line at height T by one link and walks T_T(x+Ri); per-R sums in
// registers, block partials in a fixed order, so the result is reproducible.
#include <algorithm>

#include "observables.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

constexpr int kWilsonThreads = 256;
constexpr int kWilsonMaxR = 16;
constexpr int kWilsonMaxT = 64;

struct Site {
    int c[4];
};

__device__ __forceinline__ float4 link_at_site(const float4 *__restrict__ L, const Geom &g, const Site &s, int mu)
{
    const int lex = ((s.c[3] * g.ns + s.c[2]) * g.ns + s.c[1]) * g.ns + s.c[0];
    const int parity = (s.c[0] + s.c[1] + s.c[2] + s.c[3]) & 1;
    return __ldg(L + link_index(g, mu, parity, lex >> 1));
}

__device__ __forceinline__ void step(const Geom &g, Site &s, int mu)
{
    const int c = s.c[mu] + 1;
    s.c[mu] = c == g.ext[mu] ? 0 : c;
}

template <int RM>
__global__ void __launch_bounds__(kWilsonThreads) wilson_kernel(const float4 *__restrict__ L, Geom g, int rmax, int T,
                                                                double *__restrict__ partials)
{
    double acc[RM];
#pragma unroll
    for (int r = 0; r < RM; ++r) acc[r] = 0.0;
    const int64_t items = 6 * (int64_t)g.vh;  // 3 V
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < items;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int site = (int)(q / 3);
        const int i = (int)(q - 3 * (int64_t)site);
        Site x;
        {
            const uint32_t rest = fastdiv((uint32_t)site, g.div_ns);
            x.c[0] = site - (int)rest * g.ns;
            const uint32_t rest2 = fastdiv(rest, g.div_ns);
            x.c[1] = (int)rest - (int)rest2 * g.ns;
            x.c[3] = (int)fastdiv(rest2, g.div_ns);
            x.c[2] = (int)rest2 - x.c[3] * g.ns;
        }
        // T_T(x) and the corner x + T t
        Site xt = x;
        float4 tt0 = link_at_site(L, g, xt, 3);
        step(g, xt, 3);
        for (int j = 1; j < T; ++j) {
            tt0 = qmul(tt0, link_at_site(L, g, xt, 3));
            step(g, xt, 3);
        }
        Site xs = x;  // x + (R-1) i along the bottom, then x + R i
        Site ys = xt; // x + T t + (R-1) i along the top
        float4 s_bot = make_float4(1.0f, 0.0f, 0.0f, 0.0f), s_top = s_bot;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            if (r < rmax) {
                const float4 ub = link_at_site(L, g, xs, i);
                const float4 ut = link_at_site(L, g, ys, i);
                s_bot = r == 0 ? ub : qmul(s_bot, ub);
                s_top = r == 0 ? ut : qmul(s_top, ut);
                step(g, xs, i);
                step(g, ys, i);
                // T_T(x + (r+1) i)
                Site z = xs;
                float4 tt = link_at_site(L, g, z, 3);
                step(g, z, 3);
                for (int j = 1; j < T; ++j) {
                    tt = qmul(tt, link_at_site(L, g, z, 3));
                    step(g, z, 3);
                }
                const float4 a = qmul(s_bot, tt);
                const float4 b = qmul(tt0, s_top);
                acc[r] += (double)chain4(a.x, b.x, a.y, b.y, a.z, b.z, a.w, b.w);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        const double v = block_sum(acc[r]);
        if (threadIdx.x == 0 && r < rmax) partials[(size_t)blockIdx.x * rmax + r] = v;
    }
}

// out[(R-1) tmax + (T-1)] = (sum over blocks, in order) / (3 V) for R = 1 .. rmax.
__global__ void wilson_finish_kernel(const double *__restrict__ partials, int nblocks, int rmax, int T, int tmax,
                                     double scale, double *__restrict__ out)
{
    for (int r = 0; r < rmax; ++r) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partials[(size_t)b * rmax + r];
        v = block_sum(v);
        if (threadIdx.x == 0) out[r * tmax + (T - 1)] = v * scale;
    }
}

template <int RM>
static cudaError_t launch_wilson(su2_lattice *lat, int rmax, int tmax, double *d_out)
{
    const Geom g = geom_of(lat);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, lat->device);
    const int grid = grid_for(6 * (int64_t)g.vh, kWilsonThreads, std::min(4 * sms, lat->scratch.partials_cap / rmax));
    const double scale = 1.0 / (6.0 * (double)g.vh);
    for (int T = 1; T <= tmax; ++T) {
        wilson_kernel<RM><<<grid, kWilsonThreads, 0, lat->stream>>>(lat->links, g, rmax, T, lat->scratch.partials);
        wilson_finish_kernel<<<1, kWilsonThreads, 0, lat->stream>>>(lat->scratch.partials, grid, rmax, T, tmax,
                                                                   scale, d_out);
    }
    return cudaGetLastError();
}

}  // namespace su2

using namespace su2;

extern "C" su2_status su2_wilson_loops(su2_lattice *lat, int rmax, int tmax, double *out)
{
    if (!lat || !out || rmax < 1 || tmax < 1 || rmax > kWilsonMaxR || tmax > kWilsonMaxT || rmax > lat->ns ||
        tmax > lat->nt) {
        set_last_error("su2_wilson_loops: 1 <= rmax <= min(16, Ns), 1 <= tmax <= min(64, Nt), out != NULL");
        return SU2_E_INVAL;
    }
    DeviceGuard guard(lat->device);
    const size_t bytes = sizeof(double) * (size_t)rmax * (size_t)tmax;
    double *d_out = (double *)device_alloc(bytes, lat->device, lat->stream);
    if (!d_out) {
        set_last_error("device allocation for the Wilson loops failed");
        return SU2_E_NOMEM;
    }
    cudaError_t e = rmax <= 4 ? launch_wilson<4>(lat, rmax, tmax, d_out)
                   : rmax <= 8 ? launch_wilson<8>(lat, rmax, tmax, d_out)
                               : launch_wilson<16>(lat, rmax, tmax, d_out);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, bytes, cudaMemcpyDeviceToHost, lat->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(lat->stream);
    device_free(d_out, bytes, lat->device, lat->stream);
    SU2_CUDA(e);
    return SU2_OK;
}
