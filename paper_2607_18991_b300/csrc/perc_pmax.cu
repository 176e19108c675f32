// perc_pmax.cu -- from S_max(n) to P_max(p) (eq. Pmax; Methods, "Computational methods": the
// Newman--Ziff results in the domain of the occupied-site count n are convolved with the binomial
// distribution of n to reach the domain of the occupation probability p):
//   S_max(p) = sum_n B(N, n, p) S_max(n),  B(N, n, p) = C(N, n) p^n (1 - p)^(N - n),
//   P_max(p) = S_max(p) / N,  N = L^5.
//
// The weights are evaluated one by one in FP64 from Loader's saddle-point form of the binomial
// probability (C. Loader, "Fast and accurate computation of binomial probabilities", 2000):
//   log B = delta(N) - delta(n) - delta(N - n) - D(n, Np) - D(N - n, Nq) - 1/2 log(2 pi n (N - n) / N),
// where delta(m) = log m! - [(m + 1/2) log m - m + 1/2 log 2 pi] is the remainder of Stirling's
// formula and D(x, M) = x log(x / M) + M - x.  D is summed as a series in v = (x - M) / (x + M)
// when x is close to M, where the direct form would cancel:
//   x log(x/M) = x log((1 + v)/(1 - v)) = 2x (v + v^3/3 + v^5/5 + ...),  M - x = -(x - M),
//   so D = (x - M) v + sum_{j >= 1} 2x v^(2j+1) / (2j + 1).
// delta(m) for m >= 16 is the Stirling series 1/(12m) - 1/(360m^3) + 1/(1260m^5) - 1/(1680m^7)
// + 1/(1188m^9) (Bernoulli numbers B_2k / (2k (2k - 1) m^(2k-1))), whose next term is below 1e-16;
// for m <= 15 it is taken from log m! with m! exact in FP64.
//
// The convolution is a plain FP64 weighted sum per (sample, p).
#include <cmath>

#include "perc_common.cuh"

namespace perc {

constexpr double kHalfLog2Pi = 0.91893853320467274178;  // log(2 pi) / 2
constexpr double kLog2Pi = 1.8378770664093454836;

__constant__ double c_fact[16] = {1.0,         1.0,          2.0,           6.0,
                                  24.0,        120.0,        720.0,         5040.0,
                                  40320.0,     362880.0,     3628800.0,     39916800.0,
                                  479001600.0, 6227020800.0, 87178291200.0, 1307674368000.0};

// delta(m) for integer m >= 1.
__device__ __forceinline__ double stirling_rem(double m)
{
    if (m <= 15.0) return log(c_fact[static_cast<int>(m)]) - (m + 0.5) * log(m) + m - kHalfLog2Pi;
    const double r = 1.0 / m, r2 = r * r;
    return r * (1.0 / 12.0 - r2 * (1.0 / 360.0 - r2 * (1.0 / 1260.0 - r2 * (1.0 / 1680.0 - r2 / 1188.0))));
}

// D(x, M) = x log(x / M) + M - x for x >= 0, M > 0.
__device__ __forceinline__ double deviance(double x, double M)
{
    const double d = x - M;
    if (fabs(d) < 0.1 * (x + M)) {
        const double v = d / (x + M), v2 = v * v;
        double s = d * v, term = 2.0 * x * v;
        for (int j = 1; j < 64; ++j) {  // |v| < 0.1: each term is below 1% of the one before
            term *= v2;
            const double s1 = s + term / (2 * j + 1);
            if (s1 == s) break;
            s = s1;
        }
        return s;
    }
    return x * log(x / M) + M - x;
}

// B(N, n, p) for 0 <= n <= N, N >= 1, p in [0, 1]; NaN for p outside [0, 1].
__device__ double binomial_pmf(double N, double n, double p)
{
    if (!(p >= 0.0 && p <= 1.0)) return __longlong_as_double(0x7ff8000000000000ll);
    if (p == 0.0) return n == 0.0 ? 1.0 : 0.0;
    if (p == 1.0) return n == N ? 1.0 : 0.0;
    const double q = 1.0 - p;
    if (n == 0.0) return exp(N * log1p(-p));
    if (n == N) return exp(N * log(p));
    const double m = N - n;
    const double lc = stirling_rem(N) - stirling_rem(n) - stirling_rem(m) - deviance(n, N * p) - deviance(m, N * q);
    const double lf = kLog2Pi + log(n) + log1p(-n / N);  // log(2 pi n (N - n) / N)
    return exp(lc - 0.5 * lf);
}

__global__ void k_binomial_weights(const uint64_t *__restrict__ Ng, const uint64_t *__restrict__ n_lo,
                                   const uint32_t *__restrict__ count, uint32_t groups, uint32_t window,
                                   const double *__restrict__ p, uint32_t np, double *__restrict__ w)
{
    const uint64_t total = uint64_t(groups) * np * window;
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < total;
         i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t row = i / window;  // g * np + j
        const uint32_t k = static_cast<uint32_t>(i - row * window);
        const uint32_t g = static_cast<uint32_t>(row / np);
        const uint64_t N = Ng[g], n = n_lo[g] + k;
        const bool skip = N == 0 || n > N || (count && k >= count[g]);
        w[i] = skip ? 0.0 : binomial_pmf(double(N), double(n), p[row]);
    }
}

constexpr int kPmaxThreads = 256;
constexpr int kPmaxTile = 8;  // probabilities summed together per pass over a sample's window

// One block per sample: pmax[s][j] = sum_k w[g][j][k] smax[s][k] / N[g].
__global__ void __launch_bounds__(kPmaxThreads)
k_pmax(const uint32_t *__restrict__ smax, const uint32_t *__restrict__ group, uint32_t num, uint32_t window,
       const double *__restrict__ w, const uint64_t *__restrict__ Ng, const uint32_t *__restrict__ count,
       uint32_t groups, uint32_t np, double *__restrict__ pmax)
{
    __shared__ double red[kPmaxTile][kPmaxThreads / 32];
    for (uint32_t s = blockIdx.x; s < num; s += gridDim.x) {
        const uint32_t g = group[s];
        const uint32_t *row = smax + size_t(s) * window;
        if (g >= groups) {
            for (uint32_t j = threadIdx.x; j < np; j += blockDim.x)
                pmax[size_t(s) * np + j] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        const double invN = 1.0 / double(Ng[g]);
        const uint32_t len = count ? min(count[g], window) : window;
        for (uint32_t j0 = 0; j0 < np; j0 += kPmaxTile) {
            double acc[kPmaxTile];
#pragma unroll
            for (int t = 0; t < kPmaxTile; ++t) acc[t] = 0.0;
            const double *wg = w + (size_t(g) * np + j0) * window;
            for (uint32_t k = threadIdx.x; k < len; k += blockDim.x) {
                const double v = double(__ldg(row + k));
#pragma unroll
                for (int t = 0; t < kPmaxTile; ++t)
                    if (j0 + t < np) acc[t] = fma(__ldg(wg + size_t(t) * window + k), v, acc[t]);
            }
#pragma unroll
            for (int t = 0; t < kPmaxTile; ++t) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
                if ((threadIdx.x & 31u) == 0u) red[t][threadIdx.x >> 5] = acc[t];
            }
            __syncthreads();
            if (threadIdx.x < kPmaxTile && j0 + threadIdx.x < np) {
                double sum = 0.0;
                for (int q = 0; q < kPmaxThreads / 32; ++q) sum += red[threadIdx.x][q];
                pmax[size_t(s) * np + j0 + threadIdx.x] = sum * invN;
            }
            __syncthreads();
        }
    }
}

}  // namespace perc

using namespace perc;

extern "C" int perc_binomial_weights(const uint64_t *N, const uint64_t *n_lo, const uint32_t *count, uint32_t groups,
                                     uint32_t window, const double *p, uint32_t np, double *w, void *stream_)
{
    if (!N || !n_lo || !p || !w || groups == 0 || window == 0 || np == 0) return PERC_EINVAL;
    const uint64_t total = uint64_t(groups) * np * window;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PERC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERC_ECUDA;
    uint64_t blocks = (total + 255) / 256;
    const uint64_t cap = uint64_t(sms) * 8;
    if (blocks > cap) blocks = cap;
    k_binomial_weights<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream_)>>>(
        N, n_lo, count, groups, window, p, np, w);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

extern "C" int perc_pmax(const uint32_t *smax, const uint32_t *group, uint32_t num_samples, uint32_t window,
                         const double *w, const uint64_t *N, const uint32_t *count, uint32_t groups, uint32_t np,
                         double *pmax, void *stream_)
{
    if (!smax || !group || !w || !N || !pmax || num_samples == 0 || window == 0 || groups == 0 || np == 0)
        return PERC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PERC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERC_ECUDA;
    uint32_t blocks = num_samples;
    const uint32_t cap = static_cast<uint32_t>(sms) * 8u;
    if (blocks > cap) blocks = cap;
    k_pmax<<<blocks, kPmaxThreads, 0, static_cast<cudaStream_t>(stream_)>>>(smax, group, num_samples, window, w, N,
                                                                            count, groups, np, pmax);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}
