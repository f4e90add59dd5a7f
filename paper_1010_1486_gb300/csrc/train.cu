// train.cu -- training of the learned a0 proposal on the GPU: forward and
// backward passes of the MLP + rational-quadratic spline negative
// log-likelihood, with the two hidden-layer contractions of each pass on the
// 5th-generation tensor cores (BF16 operands, FP32 accumulation in tensor
// memory), and an Adam update.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "su2_device.cuh"
#include "su2_internal.h"
#include "tc05.cuh"

namespace su2 {

constexpr uint32_t kMbarPolls = 1u << 26;

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Self-test: D (128 x 32, FP32) = A (128 x K, BF16) * B (32 x K, BF16)^T on the
// tensor cores, K = 16 or 32, for comparison with a host reference.
__global__ void __launch_bounds__(128) mma_selftest_kernel(const uint16_t *__restrict__ A,
                                                           const uint16_t *__restrict__ B, int K,
                                                           float *__restrict__ D, unsigned int *__restrict__ err)
{
    __shared__ __align__(128) unsigned char sA[128 * 32 * 2];
    __shared__ __align__(128) unsigned char sB[32 * 32 * 2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x, warp = t >> 5;
    for (int k = 0; k < K; ++k) *(uint16_t *)(sA + tc::tile_offset(t, k, K)) = A[t * K + k];
    if (t < 32)
        for (int k = 0; k < K; ++k) *(uint16_t *)(sB + tc::tile_offset(t, k, K)) = B[t * K + k];
    tc::fence_smem_to_async();
    if (warp == 0) tc::tmem_alloc(&tmem_base, 32);
    if (t == 0) {
        tc::mbar_init(&mbar, 1);
        mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tmem_base;
    if (t == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, 32);
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        for (int j = 0; j < K / 16; ++j) {
            const uint64_t ad = tc::smem_desc(tc::smem_addr(sA) + 256u * j, 128u, sbo);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(sB) + 256u * j, 128u, sbo);
            tc::mma_bf16(taddr, ad, bd, idesc, j > 0 ? 1u : 0u);
        }
        tc::mma_commit(&mbar);
    }
    bool ok = tc::mbar_wait(&mbar, 0, kMbarPolls);
    if (!ok) ok = tc::mbar_wait(&mbar, 0, kMbarPolls);  // second bounded wait before giving up
    tc::fence_after_sync();
    if (ok) {
        float v[32];
        tc::tmem_load32(taddr + ((uint32_t)(warp * 32) << 16), v);
#pragma unroll
        for (int n = 0; n < 32; ++n) D[t * 32 + n] = v[n];
    } else if ((t & 31) == 0) {
        atomicAdd(err, 1u);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

}  // namespace su2

using namespace su2;

extern "C" su2_status su2_selftest_mma(const uint16_t *A, const uint16_t *B, int K, float *D)
{
    if (!A || !B || !D || (K != 16 && K != 32)) return SU2_E_INVAL;
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));
    const size_t bytesA = 128 * (size_t)K * 2, bytesB = 32 * (size_t)K * 2, bytesD = 128 * 32 * 4;
    char *buf = (char *)device_alloc(bytesA + bytesB + bytesD + 512, dev, nullptr);
    if (!buf) return SU2_E_NOMEM;
    uint16_t *dA = (uint16_t *)buf;
    uint16_t *dB = (uint16_t *)(buf + ((bytesA + 255) & ~(size_t)255));
    float *dD = (float *)((char *)dB + ((bytesB + 255) & ~(size_t)255));
    unsigned int *dErr = (unsigned int *)((char *)dD + bytesD);
    su2_status st = SU2_OK;
    cudaError_t e = cudaMemcpy(dA, A, bytesA, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dB, B, bytesB, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dErr, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        mma_selftest_kernel<<<1, 128>>>(dA, dB, K, dD, dErr);
        e = cudaGetLastError();
    }
    unsigned int err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, bytesD, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&err, dErr, sizeof err, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) st = cuda_fail(e, "su2_selftest_mma");
    else if (err) {
        set_last_error("tensor-core self-test: completion wait gave up");
        st = SU2_E_DEVICE_TIMEOUT;
    }
    device_free(buf, bytesA + bytesB + bytesD + 512, dev, nullptr);
    cudaDeviceSynchronize();
    return st;
}

// ============================================================== training
#include "learned.cuh"

namespace su2 {
namespace train {

constexpr int kRows = 128;      // samples per CTA (the MMA M dimension)
constexpr int kPad = 33;        // row stride of the fp32 stashes (bank-conflict free)
constexpr int kGradSlots = learned::kTrainable + 1;  // 1945 gradients + loss sum

// -log q(a | o) = log 2 + log f'(f^{-1}(a)) for the spline of outputs o, and
// its gradient with respect to o: implicit differentiation of f(z) = a at
// fixed a through the bin's knots, then the knot sums, the softmax and the
// softplus (binary32; the same formulas as the binary64 reference).
__device__ float nll_and_grad(const float (&o)[learned::kOut], float a, float (&g)[learned::kOut])
{
    constexpr int K = learned::kBins;
    float prob[2][K], kn[2][K + 1], d[K + 1];
    for (int part = 0; part < 2; ++part) {
        const float *oo = o + part * K;
        float mx = oo[0];
        for (int i = 1; i < K; ++i) mx = fmaxf(mx, oo[i]);
        float sum = 0.0f;
        for (int i = 0; i < K; ++i) {
            prob[part][i] = learned::exp_neg(oo[i] - mx);
            sum += prob[part][i];
        }
        kn[part][0] = -1.0f;
        for (int i = 0; i < K; ++i) {
            prob[part][i] = prob[part][i] / sum;
            kn[part][i + 1] = kn[part][i] + 2.0f * (learned::kMinBin + (1.0f - K * learned::kMinBin) * prob[part][i]);
        }
    }
    for (int i = 0; i <= K; ++i) d[i] = learned::kMinDer + learned::softplus(o[2 * K + i]);
    const float *x = kn[0], *y = kn[1];
    int k = 0;
    for (int j = 1; j < K; ++j)
        if (y[j] <= a) k = j;
    const float W = x[k + 1] - x[k], H = y[k + 1] - y[k], D0 = d[k], D1 = d[k + 1];
    const float s = H / W, dy = a - y[k], sig = D1 + D0 - 2.0f * s;
    const float al = H * (s - D0) + dy * sig, be = H * D0 - dy * sig, c = -s * dy;
    const float disc = fmaxf(be * be - 4.0f * al * c, 0.0f);
    const float den_q = -be - sqrtf(disc);
    float xi = den_q != 0.0f ? 2.0f * c / den_q : 0.0f;
    xi = fminf(fmaxf(xi, 0.0f), 1.0f);
    const float t = xi * (1.0f - xi);
    const float N = s * xi * xi + D0 * t, Dn = s + sig * t;
    const float M = D1 * xi * xi + 2.0f * s * t + D0 * (1.0f - xi) * (1.0f - xi);
    const float L = 2.0f * log_series(s) + log_series(M) - 2.0f * log_series(Dn);
    const float Np = 2.0f * s * xi + D0 * (1.0f - 2.0f * xi), Dnp = sig * (1.0f - 2.0f * xi);
    const float Mp = 2.0f * D1 * xi + 2.0f * s * (1.0f - 2.0f * xi) - 2.0f * D0 * (1.0f - xi);
    const float F_xi = H * (Np * Dn - N * Dnp) / (Dn * Dn);
    const float L_xi = Mp / M - 2.0f * Dnp / Dn;
    const float r = L_xi / F_xi;
    const float F_s = H * (xi * xi * Dn - N * (1.0f - 2.0f * t)) / (Dn * Dn);
    const float F_D0 = H * t * (Dn - N) / (Dn * Dn);
    const float F_D1 = -H * N * t / (Dn * Dn);
    const float dY = -r;
    const float dHd = -r * (N / Dn);
    const float ds = (2.0f / s + 2.0f * t / M - 2.0f * (1.0f - 2.0f * t) / Dn) - r * F_s;
    const float dD0 = ((1.0f - xi) * (1.0f - xi) / M - 2.0f * t / Dn) - r * F_D0;
    const float dD1 = (xi * xi / M - 2.0f * t / Dn) - r * F_D1;
    const float dH = dHd + ds / W, dW = -ds * H / (W * W);
    float gk[2][K + 1];
    for (int i = 0; i <= K; ++i) gk[0][i] = gk[1][i] = 0.0f;
    gk[1][k] += dY - dH;
    gk[1][k + 1] += dH;
    gk[0][k] -= dW;
    gk[0][k + 1] += dW;
    for (int part = 0; part < 2; ++part) {
        float gw[K], dot = 0.0f, tail = 0.0f;
        for (int i = K - 1; i >= 0; --i) {
            tail += gk[part][i + 1];
            gw[i] = tail * 2.0f * (1.0f - K * learned::kMinBin);
        }
        for (int i = 0; i < K; ++i) dot += gw[i] * prob[part][i];
        for (int m = 0; m < K; ++m) g[part * K + m] = prob[part][m] * (gw[m] - dot);
    }
    for (int i = 0; i <= K; ++i) {
        const float ti = o[2 * K + i];
        const float sg = ti >= 0.0f ? 1.0f / (1.0f + learned::exp_neg(-ti)) : learned::exp_neg(ti) / (1.0f + learned::exp_neg(ti));
        g[2 * K + i] = (i == k ? dD0 : (i == k + 1 ? dD1 : 0.0f)) * sg;
    }
    return 0.69314718f + L;
}

struct StepParams {
    const float *w;            // 1947 master weights (fp32)
    const float2 *pairs;       // (beta k, a0)
    long long n_pairs;
    int explicit_rows;         // 1: row r of CTA b is pair b*128 + r; 0: random pairs
    uint32_t step, k0, k1;     // Philox key and counter for random pairs
    float *partials;           // [gridDim.x][kGradSlots]
    unsigned int *err;
};

__device__ __forceinline__ uint16_t to_bf16(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

struct Smem {
    unsigned char A[kRows * 32 * 2];     // activation tile (A operand)
    unsigned char W2[32 * 32 * 2];       // B: W2 (n = output j, k = input i)
    unsigned char W3[32 * 32 * 2];       // B: W3 (n = output o, padded to 32)
    unsigned char W3T[32 * 32 * 2];      // B: W3^T (n = j, k = o padded)
    unsigned char W2T[32 * 32 * 2];      // B: W2^T (n = i, k = j)
    float h1[kRows][kPad], h2[kRows][kPad], go[kRows][kPad], dz2[kRows][kPad], dz1[kRows][kPad];
    float s_in[kRows];
    float loss[kRows];
    uint64_t mbar;
    uint32_t tmem_base;
};

// One MMA pass: D (tmem) = A (smem tile, 128 x 32) * B^T (32 x 32), then this
// thread's row of D into v.  Every thread must call it (barriers inside).
__device__ bool mma_pass(Smem &sm, const unsigned char *B, uint32_t taddr, uint32_t &phase, float (&v)[32])
{
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, 32);
        for (int j = 0; j < 2; ++j) {
            const uint64_t ad = tc::smem_desc(tc::smem_addr(sm.A) + 256u * j, 128u, 512u);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(B) + 256u * j, 128u, 512u);
            tc::mma_bf16(taddr, ad, bd, idesc, j > 0 ? 1u : 0u);
        }
        tc::mma_commit(&sm.mbar);
    }
    bool ok = tc::mbar_wait(&sm.mbar, phase, kMbarPolls);
    if (!ok) ok = tc::mbar_wait(&sm.mbar, phase, kMbarPolls);
    phase ^= 1u;
    tc::fence_after_sync();
    if (ok) {
        tc::tmem_load32(taddr + ((uint32_t)((threadIdx.x >> 5) * 32) << 16), v);
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.0f;
    }
    tc::fence_before_sync();
    __syncthreads();  // every thread has read D and A before either is overwritten
    return ok;
}

__device__ __forceinline__ void put_row_bf16(Smem &sm, int row, const float *vals, int n)
{
    for (int k = 0; k < 32; ++k) *(uint16_t *)(sm.A + tc::tile_offset(row, k, 32)) = k < n ? to_bf16(vals[k]) : (uint16_t)0;
}

// Forward + backward of kRows samples per CTA; per-CTA sums of the 1945
// gradients and of the loss go to partials[blockIdx.x].
__global__ void __launch_bounds__(kRows) train_step_kernel(const StepParams p)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    const int t = threadIdx.x, warp = t >> 5;
    const float *w = p.w;

    // B operands (bf16, core-matrix layout)
    for (int q = t; q < 32 * 32; q += blockDim.x) {
        const int r = q >> 5, c = q & 31;
        *(uint16_t *)(sm.W2 + tc::tile_offset(r, c, 32)) = to_bf16(w[learned::kOffW2 + r * 32 + c]);
        *(uint16_t *)(sm.W2T + tc::tile_offset(r, c, 32)) = to_bf16(w[learned::kOffW2 + c * 32 + r]);
        *(uint16_t *)(sm.W3 + tc::tile_offset(r, c, 32)) = r < learned::kOut ? to_bf16(w[learned::kOffW3 + r * 32 + c]) : (uint16_t)0;
        *(uint16_t *)(sm.W3T + tc::tile_offset(r, c, 32)) = c < learned::kOut ? to_bf16(w[learned::kOffW3 + c * 32 + r]) : (uint16_t)0;
    }
    if (warp == 0) tc::tmem_alloc(&sm.tmem_base, 32);
    if (t == 0) {
        tc::mbar_init(&sm.mbar, 1);
        mbar_init_fence();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = sm.tmem_base;
    uint32_t phase = 0;
    bool ok = true;

    // sample of this row
    long long idx;
    if (p.explicit_rows) {
        idx = (long long)blockIdx.x * kRows + t;
    } else {
        const uint4 r = philox_key(make_uint4((uint32_t)(blockIdx.x * kRows + t), p.step, 5u << 3, 0u), p.k0, p.k1);
        idx = (long long)(((unsigned long long)r.x * (unsigned long long)p.n_pairs) >> 32);
    }
    const float2 pr = p.pairs[idx];
    const float s = (pr.x - w[learned::kOffMean]) * w[learned::kOffScale];
    const float a = fminf(fmaxf(pr.y, -1.0f), 1.0f);
    sm.s_in[t] = s;

    // layer 1 (fp32), layer 2 (tensor cores)
    float v[32];
    for (int j = 0; j < 32; ++j) v[j] = learned::relu(w[learned::kOffW1 + j] * s + w[learned::kOffB1 + j]);
    for (int j = 0; j < 32; ++j) sm.h1[t][j] = v[j];
    put_row_bf16(sm, t, v, 32);
    ok &= mma_pass(sm, sm.W2, taddr, phase, v);
    for (int j = 0; j < 32; ++j) v[j] = learned::relu(v[j] + w[learned::kOffB2 + j]);
    for (int j = 0; j < 32; ++j) sm.h2[t][j] = v[j];
    put_row_bf16(sm, t, v, 32);
    // layer 3 (tensor cores)
    ok &= mma_pass(sm, sm.W3, taddr, phase, v);
    float o[learned::kOut], go[learned::kOut];
    for (int j = 0; j < learned::kOut; ++j) o[j] = v[j] + w[learned::kOffB3 + j];
    sm.loss[t] = nll_and_grad(o, a, go);
    for (int j = 0; j < 32; ++j) sm.go[t][j] = j < learned::kOut ? go[j] : 0.0f;
    put_row_bf16(sm, t, go, learned::kOut);
    // dh2 = go W3 (tensor cores), through the ReLU
    ok &= mma_pass(sm, sm.W3T, taddr, phase, v);
    for (int j = 0; j < 32; ++j) v[j] = sm.h2[t][j] > 0.0f ? v[j] : 0.0f;
    for (int j = 0; j < 32; ++j) sm.dz2[t][j] = v[j];
    put_row_bf16(sm, t, v, 32);
    // dh1 = dz2 W2 (tensor cores), through the ReLU
    ok &= mma_pass(sm, sm.W2T, taddr, phase, v);
    for (int j = 0; j < 32; ++j) sm.dz1[t][j] = sm.h1[t][j] > 0.0f ? v[j] : 0.0f;
    if (!ok && t == 0) atomicAdd(p.err, 1u);
    __syncthreads();

    // per-CTA gradient sums (fp32, rows in order)
    float *out = p.partials + (size_t)blockIdx.x * kGradSlots;
    for (int q = t; q < kGradSlots; q += blockDim.x) {
        float acc = 0.0f;
        if (q < 32) {  // W1
            for (int r = 0; r < kRows; ++r) acc += sm.dz1[r][q] * sm.s_in[r];
        } else if (q < 64) {  // b1
            for (int r = 0; r < kRows; ++r) acc += sm.dz1[r][q - 32];
        } else if (q < 1088) {  // W2[j][i]
            const int j = (q - 64) >> 5, i = (q - 64) & 31;
            for (int r = 0; r < kRows; ++r) acc += sm.dz2[r][j] * sm.h1[r][i];
        } else if (q < 1120) {  // b2
            for (int r = 0; r < kRows; ++r) acc += sm.dz2[r][q - 1088];
        } else if (q < 1920) {  // W3[o][j]
            const int oo = (q - 1120) >> 5, j = (q - 1120) & 31;
            for (int r = 0; r < kRows; ++r) acc += sm.go[r][oo] * sm.h2[r][j];
        } else if (q < 1945) {  // b3
            for (int r = 0; r < kRows; ++r) acc += sm.go[r][q - 1920];
        } else {  // loss
            for (int r = 0; r < kRows; ++r) acc += sm.loss[r];
        }
        out[q] = acc;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

// Sums the per-CTA partials (in CTA order) into the mean gradient and loss;
// with lr > 0 also applies one Adam step to the master weights.
__global__ void adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ partials, int nblocks, float inv_batch, float lr, float b1,
                            float b2, float eps, float bias1, float bias2, float *__restrict__ grad_out,
                            float *__restrict__ loss_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kGradSlots) return;
    float gsum = 0.0f;
    for (int b = 0; b < nblocks; ++b) gsum += partials[(size_t)b * kGradSlots + i];
    const float g = gsum * inv_batch;
    if (i == learned::kTrainable) {
        if (loss_out) *loss_out = g;
        return;
    }
    if (grad_out) grad_out[i] = g;
    if (lr > 0.0f) {
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / bias1) / (sqrtf(vi / bias2) + eps);
    }
}

// mean and 1 / standard deviation of beta k over the pairs -> w[1945], w[1946]
__global__ void input_scaling_kernel(const float2 *__restrict__ pairs, long long n, float *__restrict__ w)
{
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double x = (double)pairs[i].x;
        a += x;
        b += x * x;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            s1[threadIdx.x] += s1[threadIdx.x + off];
            s2[threadIdx.x] += s2[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)n;
        const double var = s2[0] / (double)n - mean * mean;
        w[learned::kOffMean] = (float)mean;
        w[learned::kOffScale] = (float)(1.0 / sqrt(var > 1e-12 ? var : 1e-12));
    }
}

}  // namespace train
}  // namespace su2

struct su2_trainer {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint64_t seed = 0;
    uint32_t step = 0;  // Adam steps taken
    void *block = nullptr;
    size_t block_bytes = 0;
    float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    unsigned int *err = nullptr;
    float *partials = nullptr;
    int partial_blocks = 0;
    float *losses = nullptr;  // per step of the last fit
    int losses_cap = 0;
};

namespace su2 {
namespace {

constexpr int kMaxBatch = 65536;

su2_status trainer_launch(su2_trainer *tr, const float *pairs, long long n, int batch, int explicit_rows, float lr,
                          float *loss_dst)
{
    const int nblocks = batch / train::kRows;
    train::StepParams p;
    p.w = tr->w;
    p.pairs = (const float2 *)pairs;
    p.n_pairs = n;
    p.explicit_rows = explicit_rows;
    p.step = tr->step;
    p.k0 = (uint32_t)tr->seed;
    p.k1 = (uint32_t)(tr->seed >> 32);
    p.partials = tr->partials;
    p.err = tr->err;
    train::train_step_kernel<<<nblocks, train::kRows, sizeof(train::Smem), tr->stream>>>(p);
    SU2_CUDA(cudaGetLastError());
    float bias1 = 1.0f, bias2 = 1.0f;
    if (lr > 0.0f) {
        tr->step += 1;
        bias1 = 1.0f - powf(0.9f, (float)tr->step);
        bias2 = 1.0f - powf(0.999f, (float)tr->step);
    }
    train::adam_kernel<<<(train::kGradSlots + 255) / 256, 256, 0, tr->stream>>>(
        tr->w, tr->m, tr->v, tr->partials, nblocks, 1.0f / (float)batch, lr, 0.9f, 0.999f, 1e-8f, bias1, bias2,
        tr->grad, loss_dst);
    SU2_CUDA(cudaGetLastError());
    return SU2_OK;
}

su2_status trainer_check(su2_trainer *tr)
{
    unsigned int err = 0;
    SU2_CUDA(cudaMemcpyAsync(&err, tr->err, sizeof err, cudaMemcpyDeviceToHost, tr->stream));
    SU2_CUDA(cudaStreamSynchronize(tr->stream));
    if (err) {
        set_last_error("training: a tensor-core completion wait gave up");
        return SU2_E_DEVICE_TIMEOUT;
    }
    return SU2_OK;
}

}  // namespace
}  // namespace su2

extern "C" {

su2_status su2_trainer_create(const float *init_weights, uint64_t seed, void *cuda_stream, su2_trainer **out)
{
    if (!init_weights || !out) return SU2_E_INVAL;
    *out = nullptr;
    int dev = 0;
    SU2_CUDA(cudaGetDevice(&dev));
    static bool attr_set[64] = {};
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        SU2_CUDA(cudaFuncSetAttribute(train::train_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(train::Smem)));
        attr_set[dev] = true;
    }
    su2_trainer *tr = new (std::nothrow) su2_trainer();
    if (!tr) return SU2_E_NOMEM;
    tr->device = dev;
    tr->stream = (cudaStream_t)cuda_stream;
    tr->seed = seed;
    tr->partial_blocks = kMaxBatch / train::kRows;
    const size_t wb = 2048 * sizeof(float);
    tr->block_bytes = 5 * wb + 256 + sizeof(float) * (size_t)tr->partial_blocks * train::kGradSlots;
    tr->block = device_alloc(tr->block_bytes, dev, tr->stream);
    if (!tr->block) {
        delete tr;
        return SU2_E_NOMEM;
    }
    char *q = (char *)tr->block;
    tr->w = (float *)q;
    tr->m = (float *)(q + wb);
    tr->v = (float *)(q + 2 * wb);
    tr->grad = (float *)(q + 3 * wb);
    tr->loss = (float *)(q + 4 * wb);
    tr->err = (unsigned int *)(q + 5 * wb);
    tr->partials = (float *)(q + 5 * wb + 256);
    su2_status st = SU2_OK;
    cudaError_t e = cudaMemsetAsync(tr->block, 0, 5 * wb + 256, tr->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tr->w, init_weights, sizeof(float) * learned::kWeights, cudaMemcpyHostToDevice, tr->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(tr->stream);
    if (e != cudaSuccess) st = cuda_fail(e, "su2_trainer_create");
    if (st != SU2_OK) {
        su2_trainer_destroy(tr);
        return st;
    }
    *out = tr;
    return SU2_OK;
}

su2_status su2_trainer_destroy(su2_trainer *tr)
{
    if (!tr) return SU2_OK;
    DeviceGuard guard(tr->device);
    device_free(tr->losses, sizeof(float) * (size_t)tr->losses_cap, tr->device, tr->stream);
    device_free(tr->block, tr->block_bytes, tr->device, tr->stream);
    const cudaError_t e = cudaStreamSynchronize(tr->stream);
    delete tr;
    return e == cudaSuccess ? SU2_OK : cuda_fail(e, "su2_trainer_destroy");
}

su2_status su2_trainer_set_input_scaling(su2_trainer *tr, const float *dev_pairs, size_t n)
{
    if (!tr || !dev_pairs || n < 2) return SU2_E_INVAL;
    DeviceGuard guard(tr->device);
    train::input_scaling_kernel<<<1, 256, 0, tr->stream>>>((const float2 *)dev_pairs, (long long)n, tr->w);
    SU2_CUDA(cudaGetLastError());
    SU2_CUDA(cudaStreamSynchronize(tr->stream));
    return SU2_OK;
}

su2_status su2_trainer_gradient(su2_trainer *tr, const float *dev_pairs, size_t n, double *loss, float *grad)
{
    if (!tr || !dev_pairs || n == 0 || n % train::kRows != 0 || n > (size_t)kMaxBatch) {
        set_last_error("su2_trainer_gradient: n must be a positive multiple of 128, at most 65536");
        return SU2_E_INVAL;
    }
    DeviceGuard guard(tr->device);
    SU2_CUDA(cudaMemsetAsync(tr->err, 0, sizeof(unsigned int), tr->stream));
    su2_status st = trainer_launch(tr, dev_pairs, (long long)n, (int)n, 1, 0.0f, tr->loss);
    if (st != SU2_OK) return st;
    float l = 0.0f;
    if (grad)
        SU2_CUDA(cudaMemcpyAsync(grad, tr->grad, sizeof(float) * learned::kTrainable, cudaMemcpyDeviceToHost,
                                 tr->stream));
    SU2_CUDA(cudaMemcpyAsync(&l, tr->loss, sizeof l, cudaMemcpyDeviceToHost, tr->stream));
    st = trainer_check(tr);
    if (loss) *loss = l;
    return st;
}

su2_status su2_trainer_fit(su2_trainer *tr, const float *dev_pairs, size_t n, int steps, int batch, double lr,
                           float *loss_per_step)
{
    if (!tr || !dev_pairs || n == 0 || steps < 0 || batch < train::kRows || batch % train::kRows != 0 ||
        batch > kMaxBatch || !(lr > 0.0)) {
        set_last_error("su2_trainer_fit: batch must be a multiple of 128 in [128, 65536], lr > 0");
        return SU2_E_INVAL;
    }
    DeviceGuard guard(tr->device);
    if (steps > tr->losses_cap) {
        device_free(tr->losses, sizeof(float) * (size_t)tr->losses_cap, tr->device, tr->stream);
        tr->losses = (float *)device_alloc(sizeof(float) * (size_t)steps, tr->device, tr->stream);
        tr->losses_cap = tr->losses ? steps : 0;
        if (!tr->losses) return SU2_E_NOMEM;
    }
    SU2_CUDA(cudaMemsetAsync(tr->err, 0, sizeof(unsigned int), tr->stream));
    for (int s = 0; s < steps; ++s) {
        su2_status st = trainer_launch(tr, dev_pairs, (long long)n, batch, 0, (float)lr, tr->losses + s);
        if (st != SU2_OK) return st;
    }
    if (loss_per_step && steps > 0)
        SU2_CUDA(cudaMemcpyAsync(loss_per_step, tr->losses, sizeof(float) * steps, cudaMemcpyDeviceToHost,
                                 tr->stream));
    return trainer_check(tr);
}

su2_status su2_trainer_get_weights(su2_trainer *tr, float *host)
{
    if (!tr || !host) return SU2_E_INVAL;
    DeviceGuard guard(tr->device);
    SU2_CUDA(cudaMemcpyAsync(host, tr->w, sizeof(float) * learned::kWeights, cudaMemcpyDeviceToHost, tr->stream));
    SU2_CUDA(cudaStreamSynchronize(tr->stream));
    return SU2_OK;
}

}  // extern "C"
