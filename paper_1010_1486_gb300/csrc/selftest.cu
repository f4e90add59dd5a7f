// selftest.cu -- device self-tests of the building blocks: the Philox
// counter generator and the series log / exp / sin-cos used by the heat bath.
// They let the tests compare the device arithmetic with independent
// implementations word for word.
#include "learned.cuh"
#include "su2_device.cuh"
#include "su2_internal.h"

namespace su2 {

__global__ void philox_selftest_kernel(const uint32_t *__restrict__ ck, uint32_t *__restrict__ out, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint32_t *r = ck + 6 * i;
        const uint4 w = philox_rk(make_uint4(r[2], r[3], r[4], r[5]), make_round_keys(r[0], r[1]));
        out[4 * i + 0] = w.x;
        out[4 * i + 1] = w.y;
        out[4 * i + 2] = w.z;
        out[4 * i + 3] = w.w;
    }
}

__global__ void math_selftest_kernel(int which, const float *__restrict__ x, float *__restrict__ y,
                                     float *__restrict__ y2, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (which == 0) {
            y[i] = log_series(x[i]);
        } else if (which == 1) {
            y[i] = exp_series(x[i]);
        } else if (which == 3) {
            y[i] = __log2f(x[i]);
        } else if (which == 4) {
            // quadruple (r1, r2, 1/(beta k), exp(-2 beta k)): the screen's
            // verdict and the exact test's
            const float r1 = x[4 * i], r2 = x[4 * i + 1], ibk = x[4 * i + 2], e = x[4 * i + 3];
            const float ome = __fsub_rn(1.0f, e);
            y[i] = (float)creutz_screen(__fmaf_rn(r1, ome, e), r2, make_screen(ibk));
            float c;
            y2[i] = creutz_trial(r1, r2, ibk, e, ome, ibk == 0.0f, c) ? 1.0f : 0.0f;
        } else if (which == 5) {
            // octuple (beta k, a', a, f'(z'), f'(z), u1, -, -): the screened and
            // the exact Metropolis verdicts of the learned step
            const float *q = x + 8 * i;
            y[i] = (float)learned::metropolis_screen(q[0], q[1], q[2], q[3], q[4], q[5]);
            y2[i] = learned::metropolis_exact(q[0], q[1], q[2], q[3], q[4], q[5]) ? 1.0f : 0.0f;
        } else if (which == 6) {
            // pair (beta k, first Philox word as bits): x = e + r1 (1 - e) and
            // the candidate a0 of that Creutz trial, with e from the draw setup
            // of a staple along the identity with |V| = beta k, beta = 1
            const DrawSetup d = prepare_draw(make_float4(x[2 * i], 0.0f, 0.0f, 0.0f), 1.0f);
            const float xv = __fmaf_rn(uniform_log(__float_as_uint(x[2 * i + 1])), __fsub_rn(1.0f, d.e), d.e);
            y[i] = xv;
            y2[i] = creutz_a0(xv, d.ibk);
        } else {
            float s, c;
            sincos_2pi(x[i], s, c);
            y[i] = s;
            y2[i] = c;
        }
    }
}

// Copies host input to a temporary device buffer, runs `launch`, copies back.
template <typename Launch>
static su2_status run_with_buffers(const void *in, size_t in_bytes, void *out, size_t out_bytes, void *out2,
                                   size_t out2_bytes, Launch launch)
{
    cudaStream_t s = nullptr;
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));
    const size_t total = in_bytes + out_bytes + out2_bytes + 512;
    char *buf = (char *)device_alloc(total, dev, s);
    if (!buf) return SU2_E_NOMEM;
    char *d_in = buf;
    char *d_out = buf + ((in_bytes + 255) & ~(size_t)255);
    char *d_out2 = d_out + ((out_bytes + 255) & ~(size_t)255);
    su2_status st = SU2_OK;
    if (cudaMemcpyAsync(d_in, in, in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        st = cuda_fail(cudaGetLastError(), "selftest upload");
    } else {
        launch(d_in, d_out, d_out2, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "selftest launch");
        if (st == SU2_OK && cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "selftest download");
        if (st == SU2_OK && out2 &&
            cudaMemcpyAsync(out2, d_out2, out2_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "selftest download");
    }
    device_free(buf, total, dev, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (st == SU2_OK && e != cudaSuccess) st = cuda_fail(e, "selftest");
    return st;
}

}  // namespace su2

using namespace su2;

extern "C" {

su2_status su2_selftest_philox(const uint32_t *ck, uint32_t *out, size_t n)
{
    if (!ck || !out) return SU2_E_INVAL;
    if (n == 0) return SU2_OK;
    return run_with_buffers(ck, 24 * n, out, 16 * n, nullptr, 0, [n](char *in, char *o, char *, cudaStream_t s) {
        philox_selftest_kernel<<<grid_for((int64_t)n, 256), 256, 0, s>>>((const uint32_t *)in, (uint32_t *)o, n);
    });
}

su2_status su2_selftest_math(int which, const float *x, float *y, float *y2, size_t n)
{
    const bool two = which == 2 || which == 4 || which == 5 || which == 6;
    if (!x || !y || which < 0 || which > 6 || (two && !y2)) return SU2_E_INVAL;
    if (n == 0) return SU2_OK;
    const size_t in_bytes = (which == 4 ? 16 : which == 5 ? 32 : which == 6 ? 8 : 4) * n;
    return run_with_buffers(x, in_bytes, y, 4 * n, two ? y2 : nullptr, two ? 4 * n : 0,
                            [which, n](char *in, char *o, char *o2, cudaStream_t s) {
                                math_selftest_kernel<<<grid_for((int64_t)n, 256), 256, 0, s>>>(
                                    which, (const float *)in, (float *)o, (float *)o2, n);
                            });
}

}  // extern "C"
