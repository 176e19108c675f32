// perc_peaks.cu -- on-chip throughput probes: the peaks the n* kernels are measured against.
//
// The connected-component kernels keep their data on chip (the bitmap, the chunk arrays and the
// first union-find nodes in shared memory, the rest of the forest and the site orders in L2), so
// their bound is not HBM bandwidth but L2 bandwidth, shared-memory bandwidth and the rate of
// shared-memory and L2 atomics.  Each probe is one launch over every SM; the caller times it and
// divides the units it reports (bytes or operations) by the time.
#include <cstdint>

#include "perc_common.cuh"

namespace perc {

constexpr int kMbThreads = 512;
constexpr uint32_t kMbSmemWords = 8192;  // 32 KiB of shared memory per CTA

// 16-byte loads streaming over buf (L2 only: ld.global.cg), `iters` passes.
__global__ void __launch_bounds__(kMbThreads) k_mb_l2_read(const uint4 *__restrict__ buf, size_t n16, uint32_t iters,
                                                          uint32_t *sink)
{
    uint32_t acc = 0;
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    for (uint32_t it = 0; it < iters; ++it)
        for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n16; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads
}

// 16-byte shared-memory loads, conflict-free (consecutive lanes, consecutive 16 bytes).
__global__ void __launch_bounds__(kMbThreads) k_mb_smem_read(uint32_t iters, uint32_t *sink)
{
    __shared__ uint4 s[kMbSmemWords / 4];
    for (uint32_t i = threadIdx.x; i < kMbSmemWords / 4; i += blockDim.x) s[i] = make_uint4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    uint32_t acc = 0;
    for (uint32_t it = 0; it < iters; ++it)
#pragma unroll 8
        for (uint32_t k = 0; k < kMbSmemWords / 4 / kMbThreads; ++k) {
            const uint4 v = s[(k * blockDim.x + threadIdx.x + it) & (kMbSmemWords / 4 - 1)];
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9E3779B9u) sink[0] = acc;
}

// Shared-memory atomics, one word per lane (no two lanes of a warp on one bank): add, or
// compare-and-swap as the union-find hooks use it.
template <bool kCas>
__global__ void __launch_bounds__(kMbThreads) k_mb_smem_atomic(uint32_t iters, uint32_t *sink)
{
    __shared__ uint32_t s[kMbThreads];
    s[threadIdx.x] = 0u;
    __syncthreads();
    uint32_t v = 0;
    for (uint32_t it = 0; it < iters; ++it) {
        if (kCas)
            v = atomicCAS(s + threadIdx.x, v, v + 1u) + 1u;
        else
            atomicAdd(s + threadIdx.x, 1u);
    }
    __syncthreads();
    if (s[threadIdx.x] == 0xFFFFFFFFu) sink[0] = v;
}

// L2 atomics: atomicAdd on distinct words spread over buf, every thread `iters` times.
__global__ void __launch_bounds__(kMbThreads) k_mb_l2_atomic(uint32_t *buf, size_t nwords, uint32_t iters)
{
    const size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    for (uint32_t it = 0; it < iters; ++it) atomicAdd(buf + ((t * 97u + size_t(it) * 1021u) % nwords), 1u);
}

}  // namespace perc

using namespace perc;

extern "C" int perc_microbench(int which, void *buf, size_t bytes, uint32_t iters, double *units, void *stream_)
{
    if (!buf || !units || iters == 0 || bytes < 4096 || which < PERC_MB_L2_READ || which > PERC_MB_L2_ATOMIC)
        return PERC_EINVAL;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    uint32_t ctas = 0;
    if (resident_ctas(kAttrMicrobench, reinterpret_cast<const void *>(k_mb_l2_read), kMbThreads, 0, ctas) != PERC_OK)
        return PERC_ECUDA;
    uint32_t *sink = static_cast<uint32_t *>(buf);
    switch (which) {
    case PERC_MB_L2_READ: {
        const size_t n16 = bytes / 16;
        k_mb_l2_read<<<ctas, kMbThreads, 0, stream>>>(static_cast<const uint4 *>(buf), n16, iters, sink);
        *units = double(n16) * 16.0 * iters;
        break;
    }
    case PERC_MB_SMEM_READ:
        k_mb_smem_read<<<ctas, kMbThreads, 0, stream>>>(iters, sink);
        *units = double(ctas) * kMbSmemWords * 4.0 * iters;
        break;
    case PERC_MB_SMEM_ATOMIC:
        k_mb_smem_atomic<false><<<ctas, kMbThreads, 0, stream>>>(iters, sink);
        *units = double(ctas) * kMbThreads * iters;
        break;
    case PERC_MB_SMEM_CAS:
        k_mb_smem_atomic<true><<<ctas, kMbThreads, 0, stream>>>(iters, sink);
        *units = double(ctas) * kMbThreads * iters;
        break;
    case PERC_MB_L2_ATOMIC:
        k_mb_l2_atomic<<<ctas, kMbThreads, 0, stream>>>(static_cast<uint32_t *>(buf), bytes / 4, iters);
        *units = double(ctas) * kMbThreads * iters;
        break;
    default:
        return PERC_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}
