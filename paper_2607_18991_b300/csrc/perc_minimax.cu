// perc_minimax.cu -- n* as a min-max path value: a second, independent formulation of the first
// spanning n (Introduction: the spanning cluster appears at the threshold; Methods: clusters of
// the first n sites of the Newman--Ziff order).
//
// The first n sites hold a cluster that touches both borders x_{a+1} = 0 and x_{a+1} = L-1 exactly
// when some path of neighboring sites joins the two borders with every site of rank below n.  So
// n* = min over such paths of max over the path's sites of (rank + 1): a bottleneck (min-max) path
// value.  The kernel finds it by relaxation instead of union-find: every site carries a label, the
// smallest bottleneck of a path from the x_{a+1} = 0 border to it, which starts at rank + 1 on
// that border and at "none" elsewhere and is lowered by
//     label(i) = max(rank(i) + 1, min over neighbors j of label(j))
// until no label changes; n* is the smallest label on the x_{a+1} = L-1 border.  Labels only ever
// decrease and every value read is the bottleneck of some real path, so reading a neighbor's label
// while another thread lowers it changes the sweep count, not the fixed point (the minimal
// solution, which is the min-max path value).  Every sweep costs z neighbor reads a site, so this is
// a check for small lattices, not a fast path: the union-find kernels compute the same n* in one
// pass.
#include <cstddef>

#include "perc_common.cuh"

namespace perc {
namespace {

__constant__ ZoneTable c_mzones = kZones;

constexpr uint32_t kMiniThreads = 1024;
constexpr uint32_t kMiniMaxL = PERC_MINIMAX_MAX_L;
constexpr uint32_t kNoLabel = 0xFFFFFFFFu;

struct MiniHeader {
    int status;      // first device-side error (perc_check reads it)
    uint32_t queue;  // next sample
    uint32_t pad[62];
};
static_assert(sizeof(MiniHeader) == 256, "header is 256 bytes");

__host__ __device__ inline size_t mini_slot_bytes(uint64_t N) { return (size_t(N) * 4 + 255) & ~size_t(255); }

struct MiniShared {
    uint32_t sample;
    uint32_t z;
    uint32_t changed;
    uint32_t best;
    NbrEntry tab[kMaxOffsets];  // the neighborhood's offsets for this side
};

__device__ __forceinline__ uint32_t coord_along(const uint32_t x[5], uint32_t axis)
{
    return axis == 0u ? x[0] : axis == 1u ? x[1] : axis == 2u ? x[2] : axis == 3u ? x[3] : x[4];
}

// Per sample (persistent queue, one CTA a sample, labels in the CTA's global slot).
__global__ void __launch_bounds__(kMiniThreads, 1) k_minimax(const perc_sample *__restrict__ samples, uint32_t num,
                                                             uint32_t max_L, uint32_t *__restrict__ nstar_out,
                                                             char *ws, size_t slot_bytes)
{
    __shared__ MiniShared sh;
    MiniHeader *hdr = reinterpret_cast<MiniHeader *>(ws);
    uint32_t *lab = reinterpret_cast<uint32_t *>(ws + sizeof(MiniHeader) + size_t(blockIdx.x) * slot_bytes);
    for (;;) {
        if (threadIdx.x == 0) sh.sample = atomicAdd(&hdr->queue, 1u);
        __syncthreads();
        const uint32_t s = sh.sample;
        if (s >= num) break;
        const perc_sample smp = samples[s];
        const uint32_t L = smp.L, word = smp.zone_mask, mask = word & 0x7Fu, axis = word >> 8;
        const bool ok = L >= 1u && L <= max_L && mask != 0u && (word & ~0x77Fu) == 0u && axis < 5u && smp.rank;
        if (!ok) {
            if (threadIdx.x == 0) {
                nstar_out[s] = PERC_NEVER;
                set_status(&hdr->status, PERC_EDEVICE);
            }
            __syncthreads();
            continue;
        }
        const uint32_t N = static_cast<uint32_t>(num_sites(L));
        const FastDiv fd = make_fastdiv(L);
        // the neighborhood's offsets (linear delta and one-hot of the five components), one thread
        // per entry of the zone table
        uint32_t z = 0;
        for (int zone = 0; zone < kZoneCount; ++zone)
            if (mask & (1u << zone)) z += c_mzones.start[zone + 1] - c_mzones.start[zone];
        for (uint32_t t = threadIdx.x; t < uint32_t(kMaxOffsets); t += blockDim.x) {
            int zone = 0;
            while (t >= c_mzones.start[zone + 1]) ++zone;
            if (!(mask & (1u << zone))) continue;
            uint32_t pos = t;
            for (int q = 0; q < zone; ++q)
                if (!(mask & (1u << q))) pos -= c_mzones.start[q + 1] - c_mzones.start[q];
            sh.tab[pos] = make_nbr_entry(c_mzones.vec[t], L);
        }
        if (threadIdx.x == 0) {
            sh.z = z;
            sh.best = kNoLabel;
        }
        // labels: rank + 1 on the x_{a+1} = 0 border, none elsewhere
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
            uint32_t x[5];
            site_coords(i, fd, x);
            __stcg(lab + i, coord_along(x, axis) == 0u ? __ldg(smp.rank + i) + 1u : kNoLabel);
        }
        __syncthreads();
        // sweeps until no label changes; N + 1 sweeps always suffice (a label only takes values of
        // real path bottlenecks and the lowest ones settle first), more means a broken relaxation
        bool timed_out = true;
        for (uint32_t sweep = 0; sweep <= N + 1u; ++sweep) {
            if (threadIdx.x == 0) sh.changed = 0u;
            __syncthreads();
            uint32_t changed = 0u;
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
                uint32_t x[5];
                site_coords(i, fd, x);
                if (coord_along(x, axis) == 0u) continue;  // border labels are final
                uint32_t allowed = 0;
#pragma unroll
                for (int k = 0; k < 5; ++k) allowed |= allowed_bits(x[k], L) << (5 * k);
                uint32_t m = kNoLabel;
                for (uint32_t v = 0; v < sh.z; ++v) {
                    const NbrEntry e = sh.tab[v];
                    if (e.onehot & ~allowed) continue;
                    m = min(m, __ldcg(lab + static_cast<uint32_t>(static_cast<int32_t>(i) + e.delta)));
                }
                if (m == kNoLabel) continue;
                const uint32_t val = max(__ldg(smp.rank + i) + 1u, m);
                if (val < __ldcg(lab + i)) {
                    __stcg(lab + i, val);
                    changed = 1u;
                }
            }
            if (changed) sh.changed = 1u;
            __syncthreads();
            if (!sh.changed) {
                timed_out = false;
                break;
            }
        }
        // n* = the smallest label on the x_{a+1} = L-1 border
        uint32_t best = kNoLabel;
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
            uint32_t x[5];
            site_coords(i, fd, x);
            if (coord_along(x, axis) == L - 1u) best = min(best, __ldcg(lab + i));
        }
        best = __reduce_min_sync(0xffffffffu, best);
        if ((threadIdx.x & 31u) == 0u) atomicMin(&sh.best, best);
        __syncthreads();
        if (threadIdx.x == 0) {
            nstar_out[s] = timed_out ? PERC_NEVER : sh.best;  // kNoLabel == PERC_NEVER: nothing spans
            if (timed_out) set_status(&hdr->status, PERC_ETIMEOUT);
        }
        __syncthreads();
    }
}

int minimax_cfg(uint32_t max_L, uint32_t num, uint32_t &grid, size_t &slot)
{
    if (max_L < 1 || max_L > kMiniMaxL || num == 0) return PERC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PERC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERC_ECUDA;
    slot = mini_slot_bytes(num_sites(max_L));
    grid = static_cast<uint32_t>(num < uint32_t(sms) ? num : uint32_t(sms));
    return PERC_OK;
}

}  // namespace

size_t minimax_workspace_bytes(uint32_t max_L, uint32_t num)
{
    uint32_t grid = 0;
    size_t slot = 0;
    if (minimax_cfg(max_L, num, grid, slot) != PERC_OK) return 0;
    return sizeof(MiniHeader) + size_t(grid) * slot;
}

}  // namespace perc

using namespace perc;

extern "C" int perc_nstar_minimax(const perc_sample *samples, uint32_t num_samples, uint32_t max_L, uint32_t *nstar,
                                  void *workspace, size_t ws_bytes, void *stream_)
{
    if (!samples || !nstar || !workspace || num_samples == 0) return PERC_EINVAL;
    uint32_t grid = 0;
    size_t slot = 0;
    const int rc = minimax_cfg(max_L, num_samples, grid, slot);
    if (rc != PERC_OK) return rc;
    if (ws_bytes < sizeof(MiniHeader) + size_t(grid) * slot) return PERC_EWORKSPACE;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    // the queue starts again; the status word keeps the first error since the last perc_check
    if (cudaMemsetAsync(static_cast<char *>(workspace) + offsetof(MiniHeader, queue), 0, sizeof(uint32_t), stream) !=
        cudaSuccess)
        return PERC_ECUDA;
    k_minimax<<<grid, kMiniThreads, 0, stream>>>(samples, num_samples, max_L, nstar, static_cast<char *>(workspace),
                                                 slot);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}
