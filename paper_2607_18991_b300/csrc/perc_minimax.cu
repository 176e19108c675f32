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
// while another thread lowers it changes the number of sweeps, not the fixed point (the least
// solution, which is the min-max path value).
//
// Labels live in the CTA's slot as a 5D array [x1][x2][x3][x4][x5 padded to a multiple of 4], stored
// inverted (~label: 0 is "none"), and a sweep visits the lattice in tiles of 4^5 sites, one site a
// thread: the tile's labels and a radius-2 halo (x1..x4: 8 wide; x5: 12 wide, from the 16-byte
// boundary four sites before the tile) are brought into shared memory by one TMA tensor copy
// (cp.async.bulk.tensor.5d), relaxed there a few times (the halo fixed), and the changed labels
// written back.  Halo cells outside the lattice arrive as zeros ("none"); a neighbor outside the
// sample's lattice is skipped by its in-lattice test anyway (along x1 the box reaches into the
// neighboring slots).  Every neighbor read is from shared memory; the union-find kernels compute the
// same n* in one pass over the sites, so this is a check, not a fast path.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstddef>
#include <mutex>

#include "perc_common.cuh"

namespace perc {
namespace {

__constant__ ZoneTable c_mzones = kZones;

constexpr uint32_t kMiniThreads = 1024;  // one thread a site of a 4^5 tile
constexpr uint32_t kMiniMaxL = PERC_MINIMAX_MAX_L;
constexpr uint32_t kTileEdge = 4;
constexpr uint32_t kBoxE = 8;    // x1..x4: the tile and two sites each side
constexpr uint32_t kBoxX5 = 12;  // x5: from 4 sites before the tile (a 16-byte boundary) to 4 after
constexpr uint32_t kBoxWords = kBoxX5 * kBoxE * kBoxE * kBoxE * kBoxE;
constexpr uint32_t kBoxBytes = kBoxWords * 4u;  // 196,608
constexpr uint32_t kInTile = 8;  // relaxation rounds of a tile per visit (the halo fixed)
static_assert(kTileEdge * kTileEdge * kTileEdge * kTileEdge * kTileEdge == kMiniThreads, "one thread a site");

struct MiniHeader {
    int status;      // first device-side error (perc_check reads it)
    uint32_t queue;  // next sample
    uint32_t pad[62];
};
static_assert(sizeof(MiniHeader) == 256, "header is 256 bytes");

// Per offset: the linear offset inside the shared box and the one-hot of its five components.
struct BoxEntry {
    int32_t delta;
    uint32_t onehot;
};

struct MiniShared {
    unsigned long long bar;  // mbarrier of the tile copy
    uint32_t sample;
    uint32_t z;
    uint32_t best;
    BoxEntry tab[kMaxOffsets];
};

__host__ __device__ inline uint32_t pad4(uint32_t L) { return (L + 3u) & ~3u; }
__host__ __device__ inline size_t mini_slot_words(uint32_t L) { return size_t(pad4(L)) * L * L * L * L; }

__device__ __forceinline__ uint32_t smem_addr32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint32_t coord_along(const uint32_t x[5], uint32_t axis)
{
    return axis == 0u ? x[0] : axis == 1u ? x[1] : axis == 2u ? x[2] : axis == 3u ? x[3] : x[4];
}

// Polls of the tile copy's mbarrier phase, at most `limit` (try_wait for the default limit, which
// may suspend the thread; test_wait below it, which never does).
__device__ __forceinline__ bool bar_wait(unsigned long long *bar, uint32_t parity, uint32_t limit)
{
    const bool suspend = limit >= kSpinLimit;
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        if (suspend)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_addr32(bar)), "r"(parity)
                : "memory");
        else
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_addr32(bar)), "r"(parity)
                : "memory");
        if (done) return true;
    }
    return false;
}

// One thread: the tile's box into shared memory (coordinates innermost first; x5 a multiple of 4).
__device__ __forceinline__ void box_load(uint32_t *box, const CUtensorMap *tmap, int c5, int c4, int c3, int c2, int c1,
                                         unsigned long long *bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier writes to the box come first
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr32(bar)), "r"(kBoxBytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_addr32(box)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c5), "r"(c4), "r"(c3), "r"(c2), "r"(c1), "r"(smem_addr32(bar))
        : "memory");
}

// Per sample (persistent queue, one CTA a sample, its labels in the CTA's slot of the tensor).
__global__ void __launch_bounds__(kMiniThreads, 1) k_minimax(const perc_sample *__restrict__ samples, uint32_t num,
                                                             uint32_t max_L, uint32_t *__restrict__ nstar_out,
                                                             char *ws, const __grid_constant__ CUtensorMap tmap,
                                                             uint32_t spin)
{
    extern __shared__ __align__(128) uint32_t box[];
    __shared__ MiniShared sh;
    MiniHeader *hdr = reinterpret_cast<MiniHeader *>(ws);
    const uint32_t Lm = max_L, P5 = pad4(max_L);
    const size_t slot_words = mini_slot_words(max_L);
    uint32_t *lab = reinterpret_cast<uint32_t *>(ws + sizeof(MiniHeader)) + size_t(blockIdx.x) * slot_words;
    // this thread's site of a tile, and its cell in the box
    const uint32_t t = threadIdx.x;
    const uint32_t k[5] = {t >> 8, (t >> 6) & 3u, (t >> 4) & 3u, (t >> 2) & 3u, t & 3u};
    const uint32_t cell = ((((k[0] + 2u) * kBoxE + k[1] + 2u) * kBoxE + k[2] + 2u) * kBoxE + k[3] + 2u) * kBoxX5 + k[4] + 4u;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr32(&sh.bar)), "r"(1u) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (t == 0) sh.sample = atomicAdd(&hdr->queue, 1u);
        __syncthreads();
        const uint32_t s = sh.sample;
        if (s >= num) break;
        const perc_sample smp = samples[s];
        const uint32_t L = smp.L, word = smp.zone_mask, mask = word & 0x7Fu, axis = word >> 8;
        const bool ok = L >= 1u && L <= max_L && mask != 0u && (word & ~0x77Fu) == 0u && axis < 5u && smp.rank;
        if (!ok) {
            if (t == 0) {
                nstar_out[s] = PERC_NEVER;
                set_status(&hdr->status, PERC_EDEVICE);
            }
            __syncthreads();
            continue;
        }
        const uint32_t N = static_cast<uint32_t>(num_sites(L));
        // the neighborhood's offsets as box offsets (one thread per entry of the zone table)
        uint32_t z = 0;
        for (int zone = 0; zone < kZoneCount; ++zone)
            if (mask & (1u << zone)) z += c_mzones.start[zone + 1] - c_mzones.start[zone];
        for (uint32_t q = t; q < uint32_t(kMaxOffsets); q += blockDim.x) {
            int zone = 0;
            while (q >= c_mzones.start[zone + 1]) ++zone;
            if (!(mask & (1u << zone))) continue;
            uint32_t pos = q;
            for (int w = 0; w < zone; ++w)
                if (!(mask & (1u << w))) pos -= c_mzones.start[w + 1] - c_mzones.start[w];
            const uint32_t packed = c_mzones.vec[q];
            int32_t delta = 0;
            uint32_t onehot = 0;
#pragma unroll
            for (int w = 0; w < 5; ++w) {
                const int d = zone_component(packed, w);
                delta = delta * static_cast<int32_t>(w == 4 ? kBoxX5 : kBoxE) + d;
                onehot |= 1u << (5 * w + d + 2);
            }
            sh.tab[pos] = BoxEntry{delta, onehot};
        }
        if (t == 0) {
            sh.z = z;
            sh.best = 0u;
        }
        // labels (inverted): ~(rank + 1) on the x_{a+1} = 0 border, 0 (none) elsewhere and in the padding
        const FastDiv fm = make_fastdiv(Lm), f5 = make_fastdiv(P5);
        for (size_t e = t; e < slot_words; e += blockDim.x) {
            uint32_t r = static_cast<uint32_t>(e), x[5];
            x[4] = r - fdiv(r, f5) * P5;
            r = fdiv(r, f5);
#pragma unroll
            for (int w = 3; w >= 0; --w) {
                const uint32_t qd = fdiv(r, fm);
                x[w] = r - qd * Lm;
                r = qd;
            }
            uint32_t v = 0u;
            if (x[0] < L && x[1] < L && x[2] < L && x[3] < L && x[4] < L && coord_along(x, axis) == 0u) {
                const uint32_t i = (((x[0] * L + x[1]) * L + x[2]) * L + x[3]) * L + x[4];
                v = ~(__ldg(smp.rank + i) + 1u);
            }
            __stcg(lab + e, v);
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");  // the tile copies read these labels
        __syncthreads();
        const uint32_t T = (L + kTileEdge - 1u) / kTileEdge, tiles = T * T * T * T * T;
        bool timed_out = false, converged = false;
        for (uint32_t sweep = 0; sweep <= N + 1u && !converged && !timed_out; ++sweep) {
            uint32_t any = 0u;
            for (uint32_t tile = 0; tile < tiles; ++tile) {
                uint32_t tc[5], rem = tile;
#pragma unroll
                for (int w = 4; w >= 0; --w) {
                    tc[w] = rem % T;
                    rem /= T;
                }
                if (t == 0)
                    box_load(box, &tmap, static_cast<int>(4u * tc[4]) - 4, static_cast<int>(4u * tc[3]) - 2,
                             static_cast<int>(4u * tc[2]) - 2, static_cast<int>(4u * tc[1]) - 2,
                             static_cast<int>(blockIdx.x * Lm + 4u * tc[0]) - 2, &sh.bar);
                const bool landed = bar_wait(&sh.bar, phase, spin);
                phase ^= 1u;
                if (__syncthreads_or(!landed)) {  // the copy did not land in time
                    if (t == 0) {
                        set_status(&hdr->status, PERC_ETIMEOUT);
                        bar_wait(&sh.bar, phase ^ 1u, kSpinLimit);  // let it land before leaving
                    }
                    timed_out = true;
                    break;
                }
                uint32_t x[5];
#pragma unroll
                for (int w = 0; w < 5; ++w) x[w] = kTileEdge * tc[w] + k[w];
                const bool inside = x[0] < L && x[1] < L && x[2] < L && x[3] < L && x[4] < L;
                const bool fixed = !inside || coord_along(x, axis) == 0u;
                uint32_t allowed = 0, cap = 0, i = 0;
                if (inside) {
#pragma unroll
                    for (int w = 0; w < 5; ++w) allowed |= allowed_bits(x[w], L) << (5 * w);
                    i = (((x[0] * L + x[1]) * L + x[2]) * L + x[3]) * L + x[4];
                    cap = ~(__ldg(smp.rank + i) + 1u);  // a label is never below rank + 1
                }
                const uint32_t start = box[cell];
                for (uint32_t round = 0; round < kInTile; ++round) {
                    uint32_t changed = 0u;
                    if (!fixed) {
                        uint32_t m = 0u;
                        for (uint32_t v = 0; v < sh.z; ++v) {
                            const BoxEntry en = sh.tab[v];
                            if (en.onehot & ~allowed) continue;
                            m = max(m, box[static_cast<uint32_t>(static_cast<int32_t>(cell) + en.delta)]);
                        }
                        const uint32_t val = min(cap, m);
                        if (val > box[cell]) {
                            box[cell] = val;
                            changed = 1u;
                        }
                    }
                    if (!__syncthreads_or(changed)) break;
                }
                if (inside && box[cell] != start) {
                    __stcg(lab + ((((size_t(x[0]) * Lm + x[1]) * Lm + x[2]) * Lm + x[3]) * P5 + x[4]), box[cell]);
                    any = 1u;
                }
                // this thread's label and box writes are ordered before the next tile copy, which
                // reads the labels and overwrites the box
                asm volatile("fence.proxy.async.global;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
            }
            if (timed_out) break;
            converged = !__syncthreads_or(any);
        }
        if (timed_out) {
            if (t == 0) nstar_out[s] = PERC_NEVER;
            return;  // the CTA's barrier phase is no longer known; its remaining samples stay undone
        }
        if (!converged && t == 0) set_status(&hdr->status, PERC_ETIMEOUT);
        // n* = the smallest label on the x_{a+1} = L-1 border (the largest inverted one)
        uint32_t best = 0u;
        for (uint32_t e = t; e < N; e += blockDim.x) {
            uint32_t r = e, x[5];
#pragma unroll
            for (int w = 4; w >= 1; --w) {
                x[w] = r % L;
                r /= L;
            }
            x[0] = r;
            if (coord_along(x, axis) == L - 1u)
                best = max(best, __ldcg(lab + ((((size_t(x[0]) * Lm + x[1]) * Lm + x[2]) * Lm + x[3]) * P5 + x[4])));
        }
        best = __reduce_max_sync(0xffffffffu, best);
        if ((t & 31u) == 0u) atomicMax(&sh.best, best);
        __syncthreads();
        if (t == 0) nstar_out[s] = converged ? ~sh.best : PERC_NEVER;  // ~0 == PERC_NEVER: nothing spans
        __syncthreads();
    }
}

int minimax_cfg(uint32_t max_L, uint32_t num, uint32_t &grid, size_t &slot_bytes)
{
    if (max_L < 1 || max_L > kMiniMaxL || num == 0) return PERC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PERC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERC_ECUDA;
    slot_bytes = mini_slot_words(max_L) * 4u;
    grid = static_cast<uint32_t>(num < uint32_t(sms) ? num : uint32_t(sms));
    return PERC_OK;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
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
    char *labels = static_cast<char *>(workspace) + sizeof(MiniHeader);
    if (reinterpret_cast<uintptr_t>(labels) & 15u) return PERC_EINVAL;  // a tensor copy's base is 16-byte aligned
    PFN_cuTensorMapEncodeTiled_v12000 encode = encode_fn();
    if (!encode) return PERC_ECUDA;
    // the slots' labels as one 5D tensor: x5 (padded to P5), x4, x3, x2, and x1 of every slot in turn
    const cuuint64_t Lm = max_L, P5 = pad4(max_L);
    const cuuint64_t dims[5] = {P5, Lm, Lm, Lm, Lm * grid};
    const cuuint64_t strides[4] = {P5 * 4u, P5 * Lm * 4u, P5 * Lm * Lm * 4u, P5 * Lm * Lm * Lm * 4u};
    const cuuint32_t box[5] = {kBoxX5, kBoxE, kBoxE, kBoxE, kBoxE};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUtensorMap tmap;
    if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 5, labels, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return PERC_ECUDA;
    if (ensure_smem_attr(kAttrMinimax, reinterpret_cast<const void *>(k_minimax), kBoxBytes) != PERC_OK)
        return PERC_ECUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    // the queue starts again; the status word keeps the first error since the last perc_check
    if (cudaMemsetAsync(static_cast<char *>(workspace) + offsetof(MiniHeader, queue), 0, sizeof(uint32_t), stream) !=
        cudaSuccess)
        return PERC_ECUDA;
    k_minimax<<<grid, kMiniThreads, kBoxBytes, stream>>>(samples, num_samples, max_L, nstar,
                                                         static_cast<char *>(workspace), tmap, spin_limit());
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}
