// perc_mlp.cu -- the learned bisection bracket: a small network 8 -> 64 -> 64 -> 3 (ReLU) from a
// sample's zone-mask bits and ln L to three quantiles (taus 0.01, 0.5, 0.99) of ln(n* / L^5),
// trained with the pinball loss and Adam by the kernels below, FP32 throughout.  Not part of the
// paper: it only proposes the bracket that perc_nstar verifies before using it.
//
// Flat parameter layout: W1[64][8], b1[64], W2[64][64], b2[64], W3[3][64], b3[3] (h = W x + b).
// Pinball loss of a row: sum_k max(tau_k u_k, (tau_k - 1) u_k), u_k = y - q_k; the batch loss is
// the mean over rows.  d/dq_k = (1 - tau_k) if u_k < 0 else -tau_k (u_k = 0 takes -tau_k).
#include <cmath>

#include "perc_common.cuh"

namespace perc {

constexpr int kIn = 8, kH = 64, kOut = 3;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kOut * kH, kNParam = oB3 + kOut;
static_assert(kNParam == PERC_MLP_NPARAM, "parameter count");

__constant__ float c_taus[kOut] = {0.01f, 0.5f, 0.99f};

constexpr int kRows = 128;          // rows per block in the gradient kernel (one per thread)
constexpr int kPad = kRows + 1;     // column stride of the [feature][row] shared arrays

__device__ __forceinline__ void load_params(float *w, const float *params)
{
    for (int i = threadIdx.x; i < kNParam; i += blockDim.x) w[i] = params[i];
}

// Forward of one row; writes q[3].
__device__ __forceinline__ void row_forward(const float *w, const float x[kIn], float q[kOut])
{
    float h1[kH];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
        float a = w[oB1 + j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) a = fmaf(w[oW1 + j * kIn + k], x[k], a);
        h1[j] = fmaxf(a, 0.0f);
    }
#pragma unroll
    for (int m = 0; m < kOut; ++m) q[m] = w[oB3 + m];
    for (int j = 0; j < kH; ++j) {
        float a = w[oB2 + j];
#pragma unroll
        for (int k = 0; k < kH; ++k) a = fmaf(w[oW2 + j * kH + k], h1[k], a);
        a = fmaxf(a, 0.0f);
#pragma unroll
        for (int m = 0; m < kOut; ++m) q[m] = fmaf(w[oW3 + m * kH + j], a, q[m]);
    }
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ params,
                                                     const float *__restrict__ X, uint32_t B,
                                                     float *__restrict__ Q)
{
    __shared__ float w[kNParam];
    load_params(w, params);
    __syncthreads();
    const uint32_t row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= B) return;
    float x[kIn], q[kOut];
#pragma unroll
    for (int k = 0; k < kIn; ++k) x[k] = X[size_t(row) * kIn + k];
    row_forward(w, x, q);
#pragma unroll
    for (int m = 0; m < kOut; ++m) Q[size_t(row) * kOut + m] = q[m];
}

// Gradient of the mean pinball loss.  Each block takes kRows rows: per row (one thread) the forward
// activations and the back-propagated signals go to shared memory as [feature][row] columns, then
// the block sums the outer products over its rows and adds them to grad with atomics.
__global__ void __launch_bounds__(kRows) k_mlp_grad(const float *__restrict__ params,
                                                    const float *__restrict__ X,
                                                    const float *__restrict__ y, uint32_t B,
                                                    float *__restrict__ grad, float *__restrict__ loss)
{
    extern __shared__ __align__(16) float sm[];
    float *w = sm;                      // kNParam
    float *sx = w + kNParam;            // [kIn][kPad]
    float *sa1 = sx + kIn * kPad;       // [kH][kPad]
    float *sa2 = sa1 + kH * kPad;       // [kH][kPad]
    float *sg1 = sa2 + kH * kPad;       // [kH][kPad] dL/dz1
    float *sg2 = sg1 + kH * kPad;       // [kH][kPad] dL/dz2
    float *sgq = sg2 + kH * kPad;       // [kOut][kPad] dL/dq
    __shared__ float red[kRows / 32];

    load_params(w, params);
    __syncthreads();
    const int t = threadIdx.x;
    const uint32_t row = blockIdx.x * kRows + t;
    const bool valid = row < B;
    const float invB = 1.0f / static_cast<float>(B);
    float row_loss = 0.0f;
    {
        float x[kIn];
#pragma unroll
        for (int k = 0; k < kIn; ++k) {
            x[k] = valid ? X[size_t(row) * kIn + k] : 0.0f;
            sx[k * kPad + t] = x[k];
        }
        for (int j = 0; j < kH; ++j) {
            float a = w[oB1 + j];
#pragma unroll
            for (int k = 0; k < kIn; ++k) a = fmaf(w[oW1 + j * kIn + k], x[k], a);
            sa1[j * kPad + t] = valid ? fmaxf(a, 0.0f) : 0.0f;
        }
        float q[kOut];
#pragma unroll
        for (int m = 0; m < kOut; ++m) q[m] = w[oB3 + m];
        for (int j = 0; j < kH; ++j) {
            float a = w[oB2 + j];
            for (int k = 0; k < kH; ++k) a = fmaf(w[oW2 + j * kH + k], sa1[k * kPad + t], a);
            a = valid ? fmaxf(a, 0.0f) : 0.0f;
            sa2[j * kPad + t] = a;
#pragma unroll
            for (int m = 0; m < kOut; ++m) q[m] = fmaf(w[oW3 + m * kH + j], a, q[m]);
        }
        const float yt = valid ? y[row] : 0.0f;
        float gq[kOut];
#pragma unroll
        for (int m = 0; m < kOut; ++m) {
            const float u = yt - q[m];
            const float tau = c_taus[m];
            row_loss += valid ? fmaxf(tau * u, (tau - 1.0f) * u) : 0.0f;
            gq[m] = valid ? ((u < 0.0f ? 1.0f - tau : -tau) * invB) : 0.0f;
            sgq[m * kPad + t] = gq[m];
        }
        for (int j = 0; j < kH; ++j) {
            float g = 0.0f;
#pragma unroll
            for (int m = 0; m < kOut; ++m) g = fmaf(gq[m], w[oW3 + m * kH + j], g);
            sg2[j * kPad + t] = sa2[j * kPad + t] > 0.0f ? g : 0.0f;
        }
        for (int k = 0; k < kH; ++k) {
            float g = 0.0f;
            for (int j = 0; j < kH; ++j) g = fmaf(sg2[j * kPad + t], w[oW2 + j * kH + k], g);
            sg1[k * kPad + t] = sa1[k * kPad + t] > 0.0f ? g : 0.0f;
        }
    }
    // loss of the block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) row_loss += __shfl_xor_sync(0xffffffffu, row_loss, o);
    if ((t & 31) == 0) red[t >> 5] = row_loss;
    __syncthreads();
    if (t == 0 && loss) {
        float s = 0.0f;
        for (int i = 0; i < kRows / 32; ++i) s += red[i];
        atomicAdd(loss, s * invB);
    }
    const int rows = kRows;  // rows past B were zero-filled above and add nothing
    for (int o = t; o < kNParam; o += kRows) {
        float s = 0.0f;
        if (o < oB1) {                      // W1[j][k]
            const int j = o / kIn, k = o % kIn;
            for (int r = 0; r < rows; ++r) s = fmaf(sg1[j * kPad + r], sx[k * kPad + r], s);
        } else if (o < oW2) {               // b1[j]
            const int j = o - oB1;
            for (int r = 0; r < rows; ++r) s += sg1[j * kPad + r];
        } else if (o < oB2) {               // W2[j][k]
            const int j = (o - oW2) / kH, k = (o - oW2) % kH;
            for (int r = 0; r < rows; ++r) s = fmaf(sg2[j * kPad + r], sa1[k * kPad + r], s);
        } else if (o < oW3) {               // b2[j]
            const int j = o - oB2;
            for (int r = 0; r < rows; ++r) s += sg2[j * kPad + r];
        } else if (o < oB3) {               // W3[m][j]
            const int m = (o - oW3) / kH, j = (o - oW3) % kH;
            for (int r = 0; r < rows; ++r) s = fmaf(sgq[m * kPad + r], sa2[j * kPad + r], s);
        } else {                            // b3[m]
            const int m = o - oB3;
            for (int r = 0; r < rows; ++r) s += sgq[m * kPad + r];
        }
        atomicAdd(grad + o, s);
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, uint32_t n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void __launch_bounds__(256) k_bracket(const float *__restrict__ params,
                                                 const perc_sample *__restrict__ samples, uint32_t num,
                                                 float margin, uint32_t *__restrict__ bracket)
{
    __shared__ float w[kNParam];
    load_params(w, params);
    __syncthreads();
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= num) return;
    const uint32_t L = samples[s].L, mask = samples[s].zone_mask;
    float x[kIn], q[kOut];
#pragma unroll
    for (int k = 0; k < 7; ++k) x[k] = static_cast<float>((mask >> k) & 1u);
    x[7] = logf(static_cast<float>(L));
    row_forward(w, x, q);
    const double N = static_cast<double>(num_sites(L));
    double lo = floor(N * static_cast<double>(expf(q[0] - margin)));
    double hi = ceil(N * static_cast<double>(expf(q[2] + margin)));
    lo = fmin(fmax(lo, 1.0), N);
    hi = fmin(fmax(hi, lo), N);
    bracket[2 * size_t(s)] = static_cast<uint32_t>(lo);
    bracket[2 * size_t(s) + 1] = static_cast<uint32_t>(hi);
}

static size_t grad_smem_bytes()
{
    return sizeof(float) * (kNParam + kIn * kPad + 4 * kH * kPad + kOut * kPad);
}

static int launch_grad(const float *params, const float *X, const float *y, uint32_t B, float *grad,
                       float *loss, cudaStream_t stream)
{
    const size_t smem = grad_smem_bytes();
    if (ensure_smem_attr(kAttrMlpGrad, reinterpret_cast<const void *>(k_mlp_grad), smem) != PERC_OK)
        return PERC_ECUDA;  // (set once per device)
    if (cudaMemsetAsync(grad, 0, sizeof(float) * kNParam, stream) != cudaSuccess) return PERC_ECUDA;
    if (loss && cudaMemsetAsync(loss, 0, sizeof(float), stream) != cudaSuccess) return PERC_ECUDA;
    k_mlp_grad<<<(B + kRows - 1) / kRows, kRows, smem, stream>>>(params, X, y, B, grad, loss);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

static int launch_adam(float *params, const float *grad, float *m, float *v, uint32_t n, uint32_t t,
                       float lr, float b1, float b2, float eps, cudaStream_t stream)
{
    const float bc1 = static_cast<float>(1.0 - std::pow(static_cast<double>(b1), double(t)));
    const float bc2 = static_cast<float>(1.0 - std::pow(static_cast<double>(b2), double(t)));
    k_adam<<<(n + 255) / 256, 256, 0, stream>>>(params, grad, m, v, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

}  // namespace perc

using namespace perc;

extern "C" int perc_mlp_forward(const float *params, const float *X, uint32_t B, float *Q, void *stream)
{
    if (!params || !X || !Q || B == 0) return PERC_EINVAL;
    k_mlp_forward<<<(B + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, X, B, Q);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

extern "C" int perc_mlp_grad(const float *params, const float *X, const float *y, uint32_t B, float *grad,
                             float *loss, void *stream)
{
    if (!params || !X || !y || !grad || B == 0) return PERC_EINVAL;
    return launch_grad(params, X, y, B, grad, loss, static_cast<cudaStream_t>(stream));
}

extern "C" int perc_adam(float *params, const float *grad, float *m, float *v, uint32_t n, uint32_t t,
                         float lr, float beta1, float beta2, float eps, void *stream)
{
    if (!params || !grad || !m || !v || n == 0 || t == 0) return PERC_EINVAL;
    return launch_adam(params, grad, m, v, n, t, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream));
}

extern "C" int perc_mlp_train(float *params, float *m, float *v, float *grad, const float *X, const float *y,
                              uint32_t B, uint32_t t0, uint32_t steps, float lr, float *losses, void *stream)
{
    if (!params || !m || !v || !grad || !X || !y || B == 0) return PERC_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (uint32_t k = 0; k < steps; ++k) {
        int rc = launch_grad(params, X, y, B, grad, losses ? losses + k : nullptr, st);
        if (rc != PERC_OK) return rc;
        rc = launch_adam(params, grad, m, v, kNParam, t0 + k + 1, lr, 0.9f, 0.999f, 1e-8f, st);
        if (rc != PERC_OK) return rc;
    }
    return PERC_OK;
}

extern "C" int perc_bracket(const float *params, const perc_sample *samples, uint32_t num_samples, float margin,
                            uint32_t *bracket, void *stream)
{
    if (!params || !samples || !bracket || num_samples == 0) return PERC_EINVAL;
    k_bracket<<<(num_samples + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, samples,
                                                                                      num_samples, margin, bracket);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}
