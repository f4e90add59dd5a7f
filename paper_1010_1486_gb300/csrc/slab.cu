// slab.cu -- one time slab of a lattice, for the decomposition of a single
// lattice over several ranks (Sec. 4, multi-GPU part, and Fig. 1 of Cardoso &
// Bicudo, LAT2010).
//
// A slab holds the time slices t0 .. t0 + nt_local - 1 of an Ns^3 x Nt lattice
// plus one ghost slice on each side, as an Ns^3 x (nt_local + 2) lattice in the
// library's even/odd layout: local slice tl is global slice (t0 - 1 + tl) mod
// Nt.  A phase updates the interior slices only; the ghosts supply the t +- 1
// neighbours, so no interior site wraps around in the local array.  The random
// numbers of a link are those of its global site: with t0 and nt_local even,
// the local even/odd index is the global one minus (t0 - 1) Ns^3 / 2 and the
// local parity is the global one flipped (t0 - 1 is odd).  A decomposed chain
// is therefore the single lattice's chain bit for bit.
//
// After the phase (mu, parity) the links U_mu of that parity in the first and
// the last interior slice have changed, and the neighbours' ghost copies must
// follow before the next phase: su2_slab_pack / su2_slab_unpack move those
// Ns^3 / 2 links (8 Ns^3 bytes) to and from a caller buffer (host or device),
// and su2_slab_exchange does both directions between two slabs of one process.
#include <cuda_runtime.h>

#include <new>
#include <string>

#include "su2_device.cuh"
#include "su2_internal.h"

struct su2_slab {
    su2_lattice *lat = nullptr;  // the local array (ghosts included)
    int nt = 0, t0 = 0, nt_local = 0;
    cudaEvent_t ev = nullptr;  // orders exchanges between the streams of two slabs
};

namespace su2 {
namespace {

// Hot start of the local array: every link, ghosts included, is the link of
// its global site (hot_link keyed by the global even/odd index and parity).
__global__ void slab_hot_start_kernel(float4 *__restrict__ links, Geom g, int t_first, int nt_global,
                                      const RoundKeys rk, unsigned int *__restrict__ flags)
{
    const int64_t n = 8 * (int64_t)g.vh;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int group = (int)(idx / g.vh);
        const int eo = (int)(idx - (int64_t)group * g.vh);
        const int mu = group >> 1, parity = group & 1;
        const Coord x = eo_to_coord(g, eo, parity);
        const int tg = (x.c[3] + t_first + nt_global) % nt_global;
        const int lex_g = x.lex + (tg - x.c[3]) * g.vs;
        const uint32_t parity_g = (uint32_t)((x.c[0] + x.c[1] + x.c[2] + tg) & 1);
        float4 out;
        if (!hot_link((uint32_t)(lex_g >> 1), parity_g, (uint32_t)mu, rk, out)) atomicAdd(&flags[1], 1u);
        links[idx] = out;
    }
}

SlabRange slab_range(const su2_slab *s, int parity_global)
{
    const int half_slice = s->lat->ns * s->lat->ns * s->lat->ns / 2;
    SlabRange r;
    r.eo_begin = half_slice;                        // local slice 1
    r.eo_end = (s->nt_local + 1) * half_slice;      // .. local slice nt_local
    r.rng_eo = (uint32_t)((s->t0 - 1) * half_slice);  // global eo = local eo + (t0 - 1) Ns^3 / 2 (mod 2^32)
    r.rng_parity = parity_global;
    return r;
}

// Local parity of the links with global parity p: t0 - 1 is odd.
int local_parity(int parity_global) { return parity_global ^ 1; }

// Device address of local slice tl of the (mu, global parity) array.
float4 *slice_links(su2_slab *s, int mu, int parity_global, int tl)
{
    const int half_slice = s->lat->ns * s->lat->ns * s->lat->ns / 2;
    return s->lat->links + (size_t)(2 * mu + local_parity(parity_global)) * (size_t)s->lat->vh +
           (size_t)tl * (size_t)half_slice;
}

size_t slice_bytes(const su2_slab *s)
{
    return sizeof(float4) * (size_t)(s->lat->ns * s->lat->ns * s->lat->ns / 2);
}

su2_status check_phase_args(const su2_slab *s, int mu, int parity)
{
    if (!s || mu < 0 || mu > 3 || (parity != 0 && parity != 1)) {
        set_last_error("slab: bad handle, mu or parity");
        return SU2_E_INVAL;
    }
    return SU2_OK;
}

}  // namespace
}  // namespace su2

using namespace su2;

extern "C" {

su2_status su2_slab_create(int ns, int nt, int t0, int nt_local, double beta, uint64_t seed, su2_start start,
                           void *cuda_stream, su2_slab **out)
{
    if (!out) return SU2_E_INVAL;
    *out = nullptr;
    if (ns < 2 || (ns & 1) || nt < 2 || (nt & 1) || nt_local < 2 || (nt_local & 1) || (t0 & 1) || t0 < 0 ||
        t0 + nt_local > nt) {
        set_last_error("su2_slab_create: Ns, Nt and the slab's slice count must be even (>= 2), t0 even, and the "
                       "slab inside [0, Nt)");
        return SU2_E_INVAL;
    }
    if (start != SU2_COLD && start != SU2_HOT) return SU2_E_INVAL;
    su2_slab *s = new (std::nothrow) su2_slab();
    if (!s) return SU2_E_NOMEM;
    s->nt = nt;
    s->t0 = t0;
    s->nt_local = nt_local;
    su2_status st = su2_create(ns, nt_local + 2, beta, seed, SU2_COLD, cuda_stream, &s->lat);
    if (st != SU2_OK) {
        delete s;
        return st;
    }
    DeviceGuard guard(s->lat->device);
    if (cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) {
        su2_slab_destroy(s);
        return cuda_fail(cudaGetLastError(), "su2_slab_create: event");
    }
    if (start == SU2_HOT) {
        su2_lattice *lat = s->lat;
        const int64_t n = 8 * (int64_t)lat->vh;
        slab_hot_start_kernel<<<grid_for(n, 256), 256, 0, lat->stream>>>(lat->links, geom_of(lat), t0 - 1, nt,
                                                                          make_round_keys(seed), lat->scratch.flags);
        unsigned int flags[4];
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(flags, lat->scratch.flags, sizeof flags, cudaMemcpyDeviceToHost, lat->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(lat->stream) != cudaSuccess) {
            st = cuda_fail(cudaGetLastError(), "slab hot start");
        } else if (flags[1] != 0) {
            set_last_error("slab hot start: a link found no two disk points in 64 pairs");
            st = SU2_E_SAMPLER;
        }
        if (st != SU2_OK) {
            su2_slab_destroy(s);
            return st;
        }
    }
    *out = s;
    return SU2_OK;
}

su2_status su2_slab_destroy(su2_slab *s)
{
    if (!s) return SU2_OK;
    su2_status st = SU2_OK;
    if (s->lat) {
        DeviceGuard guard(s->lat->device);
        if (s->ev) cudaEventDestroy(s->ev);
        st = su2_destroy(s->lat);
    }
    delete s;
    return st;
}

su2_status su2_slab_set_sampler(su2_slab *s, int sampler)
{
    if (!s) return SU2_E_INVAL;
    return su2_set_sampler(s->lat, sampler);
}

su2_status su2_slab_phase(su2_slab *s, int mu, int parity)
{
    su2_status st = check_phase_args(s, mu, parity);
    if (st != SU2_OK) return st;
    DeviceGuard guard(s->lat->device);
    st = launch_hb_phase_slab(s->lat, mu, local_parity(parity), s->lat->sweep, slab_range(s, parity));
    if (st == SU2_OK && mu == 3 && parity == 1) s->lat->sweep += 1;
    return st;
}

size_t su2_slab_boundary_bytes(const su2_slab *s) { return s ? slice_bytes(s) : 0; }

su2_status su2_slab_pack(su2_slab *s, int mu, int parity, int side, void *dst)
{
    su2_status st = check_phase_args(s, mu, parity);
    if (st != SU2_OK) return st;
    if (!dst || (side != 0 && side != 1)) return SU2_E_INVAL;
    DeviceGuard guard(s->lat->device);
    const int tl = side == 0 ? 1 : s->nt_local;
    SU2_CUDA(cudaMemcpyAsync(dst, slice_links(s, mu, parity, tl), slice_bytes(s), cudaMemcpyDefault, s->lat->stream));
    return SU2_OK;
}

su2_status su2_slab_unpack(su2_slab *s, int mu, int parity, int side, const void *src)
{
    su2_status st = check_phase_args(s, mu, parity);
    if (st != SU2_OK) return st;
    if (!src || (side != 0 && side != 1)) return SU2_E_INVAL;
    DeviceGuard guard(s->lat->device);
    const int tl = side == 0 ? 0 : s->nt_local + 1;
    SU2_CUDA(cudaMemcpyAsync(slice_links(s, mu, parity, tl), src, slice_bytes(s), cudaMemcpyDefault, s->lat->stream));
    return SU2_OK;
}

su2_status su2_slab_exchange(su2_slab *lower, su2_slab *upper, int mu, int parity)
{
    su2_status st = check_phase_args(lower, mu, parity);
    if (st == SU2_OK) st = check_phase_args(upper, mu, parity);
    if (st != SU2_OK) return st;
    if (lower->lat->ns != upper->lat->ns || lower->nt != upper->nt ||
        (lower != upper && (lower->t0 + lower->nt_local) % lower->nt != upper->t0)) {
        set_last_error("su2_slab_exchange: the slabs are not neighbours of one lattice (lower then upper)");
        return SU2_E_INVAL;
    }
    cudaStream_t sl = lower->lat->stream, su = upper->lat->stream;
    const bool two_streams = lower != upper && sl != su;
    // the copies run on the lower slab's stream after both slabs' phases; the
    // upper slab's stream waits for them before its next phase
    if (two_streams) {
        DeviceGuard g(upper->lat->device);
        SU2_CUDA(cudaEventRecord(upper->ev, su));
    }
    DeviceGuard guard(lower->lat->device);
    if (two_streams) SU2_CUDA(cudaStreamWaitEvent(sl, upper->ev, 0));
    const size_t bytes = slice_bytes(lower);
    SU2_CUDA(cudaMemcpyAsync(slice_links(upper, mu, parity, 0), slice_links(lower, mu, parity, lower->nt_local), bytes,
                             cudaMemcpyDefault, sl));
    SU2_CUDA(cudaMemcpyAsync(slice_links(lower, mu, parity, lower->nt_local + 1), slice_links(upper, mu, parity, 1),
                             bytes, cudaMemcpyDefault, sl));
    if (two_streams) {
        SU2_CUDA(cudaEventRecord(lower->ev, sl));
        DeviceGuard g(upper->lat->device);
        SU2_CUDA(cudaStreamWaitEvent(su, lower->ev, 0));
    }
    return SU2_OK;
}

su2_status su2_slab_sync(su2_slab *s)
{
    if (!s) return SU2_E_INVAL;
    DeviceGuard guard(s->lat->device);
    SU2_CUDA(cudaStreamSynchronize(s->lat->stream));
    return SU2_OK;
}

su2_status su2_slab_get_links(su2_slab *s, float *host)
{
    if (!s) return SU2_E_INVAL;
    return su2_get_links(s->lat, host);
}

su2_status su2_slab_set_links(su2_slab *s, const float *host)
{
    if (!s) return SU2_E_INVAL;
    return su2_set_links(s->lat, host);
}

su2_status su2_slab_stats(su2_slab *s, uint64_t trials[8], uint64_t *sampler_failures)
{
    if (!s || !trials) return SU2_E_INVAL;
    DeviceGuard guard(s->lat->device);
    su2_stats st;
    su2_status r = collect_stats(s->lat, &st, 0);
    // the kernels count by local parity; report by the global one
    for (int mu = 0; mu < 4; ++mu)
        for (int p = 0; p < 2; ++p) trials[2 * mu + p] = st.trials[2 * mu + local_parity(p)];
    if (sampler_failures) *sampler_failures = st.sampler_failures;
    su2_status c = launch_clear_counters(s->lat);
    return r != SU2_OK ? r : c;
}

su2_status su2_slab_info(const su2_slab *s, int *t0, int *nt_local, uint32_t *sweep)
{
    if (!s) return SU2_E_INVAL;
    if (t0) *t0 = s->t0;
    if (nt_local) *nt_local = s->nt_local;
    if (sweep) *sweep = s->lat->sweep;
    return SU2_OK;
}

}  // extern "C"
