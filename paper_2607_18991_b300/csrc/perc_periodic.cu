// perc_periodic.cu -- the periodic-boundary variants of the path: offsets wrap modulo L in every
// coordinate (the lattice is a 5-torus), a variant of the boundary conditions, which the paper does
// not state (Methods, "Computational methods").
//
//   perc_mass_periodic  S_max with the first n sites of the Newman--Ziff order occupied (eq. Pmax);
//   perc_nstar_wrap     the first n at which a cluster wraps around the torus along the sample's
//                       axis: it holds a closed path whose steps' x_{a+1} components do not sum to
//                       zero (the torus's counterpart of the spanning cluster, Introduction).
//
// One CTA per sample (persistent queue).  The forest of the first n sites: the bitmap of those
// sites, one union-find node per site in rank space, and every edge taken once, from its later site
// in rank order.  Each node word holds its parent and the displacement along the axis to it, so every
// cluster carries an unwrapped coordinate; an edge inside one cluster whose ends disagree with
// its step closes a winding path.  S_max counts the roots; n* is found by bisection over n
// (wrapping is monotone in n, and it holds at n = L^5: every zone has a step with a non-zero
// component along every axis, and repeating it L times winds around the torus), each probe
// extending the forest of the largest n known not to wrap.
#include <algorithm>

#include <cstddef>

#include "perc_common.cuh"

namespace perc {
namespace {

__constant__ ZoneTable c_tzones = kZones;

constexpr uint32_t kPerThreads = 1024;
constexpr uint32_t kTorusSmemMaxL = 16;  // up to L = 16 the bitmap (128 KiB) lives in shared memory
constexpr uint32_t kPeriodicMaxL = PERC_PERIODIC_MAX_L;  // displacements stay below 2 L^5 < 2^31
constexpr size_t kPeriodicBudget = size_t(16) << 30;  // bytes of per-CTA slots in one launch

struct PerHeader {
    int status;       // first device-side error (perc_check reads it)
    uint32_t queue;   // next sample
    uint32_t pad[62];
};
static_assert(sizeof(PerHeader) == 256, "header is 256 bytes");

__host__ __device__ inline size_t per_align(size_t b) { return (b + 255) & ~size_t(255); }
__host__ __device__ inline size_t per_bm_words(uint64_t N) { return size_t(N / 32 + 1); }

// Per-CTA slot: bitmap (one bit per site), two forests of node words (parent << 32 | displacement:
// the committed one and the probe's) and cluster counts.
__host__ __device__ inline size_t per_slot_bytes(uint64_t N)
{
    return per_align(per_bm_words(N) * 4) + 2 * per_align(size_t(N) * 8) + per_align(size_t(N) * 4);
}

__device__ __forceinline__ unsigned long long node_word(uint32_t parent, int32_t disp)
{
    return (static_cast<unsigned long long>(parent) << 32) | static_cast<uint32_t>(disp);
}
__device__ __forceinline__ uint32_t word_parent(unsigned long long w) { return static_cast<uint32_t>(w >> 32); }
__device__ __forceinline__ int32_t word_disp(unsigned long long w) { return static_cast<int32_t>(static_cast<uint32_t>(w)); }

// Root of x and pos(x) - pos(root) along the axis, with path halving (a compare-and-swap that may
// fail: every word read stays a true relative position, since positions inside a cluster never
// change once joined).  More than `cap` steps would mean a cycle in the forest: *bad is set.
__device__ uint32_t tfind(unsigned long long *nd, uint32_t x, int32_t &d, uint32_t cap, bool &bad)
{
    int32_t acc = 0;
    for (uint32_t it = 0; it <= cap; ++it) {
        const unsigned long long w = __ldcg(nd + x);
        const uint32_t p = word_parent(w);
        if (p == x) {
            d = acc;
            return x;
        }
        const unsigned long long w2 = __ldcg(nd + p);
        const uint32_t g = word_parent(w2);
        if (g == p) {
            d = acc + word_disp(w);
            return p;
        }
        const int32_t dxg = word_disp(w) + word_disp(w2);
        atomicCAS(nd + x, w, node_word(g, dxg));
        acc += dxg;
        x = g;
    }
    bad = true;
    d = acc;
    return x;
}

// Joins the clusters of nodes a and b over a step with pos(b) = pos(a) + step (the larger root
// goes under the smaller).  Returns true when a and b already were one cluster and the step
// disagrees with their coordinates: the edge closes a winding path.
__device__ bool tunite(unsigned long long *nd, uint32_t a, uint32_t b, int32_t step, uint32_t cap, bool &bad)
{
    for (uint32_t it = 0; it <= cap; ++it) {
        int32_t da, db;
        const uint32_t ra = tfind(nd, a, da, cap, bad);
        const uint32_t rb = tfind(nd, b, db, cap, bad);
        if (bad) return false;
        if (ra == rb) return da + step != db;
        if (ra < rb) {  // pos(rb) - pos(ra) = da + step - db
            if (atomicCAS(nd + rb, node_word(rb, 0), node_word(ra, da + step - db)) == node_word(rb, 0)) return false;
        } else {  // pos(ra) - pos(rb) = db - da - step
            if (atomicCAS(nd + ra, node_word(ra, 0), node_word(rb, db - da - step)) == node_word(ra, 0)) return false;
        }
    }
    bad = true;
    return false;
}

struct PerShared {
    uint32_t sample;
    uint32_t z;
    uint32_t flag;   // a winding path was found in the running pass
    uint32_t bad;    // a union-find loop ran out
    uint32_t best;   // largest cluster
    uint32_t offs[kMaxOffsets];  // the neighborhood's packed offsets
};

// Bitmap bits and singleton nodes of the sites of rank r0 .. r1-1.
__device__ void torus_add(uint32_t *bm, unsigned long long *nd, const uint32_t *perm, uint32_t r0, uint32_t r1)
{
    for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        __stcg(nd + r, node_word(r, 0));
        const uint32_t i = __ldg(perm + r);
        atomicOr(bm + (i >> 5), 1u << (i & 31u));
    }
}

// The sites of rank r0 .. r1-1 join the forest `nd` of the first r0 sites (the bitmap holds the
// first r1 sites, their nodes are set).  Every edge is taken by its later site in rank order, so
// the new sites' edges to each other and to the earlier sites are all seen.  kWrap: stop as soon as
// a winding path along `axis` closes (sh.flag).  Ends with a barrier.
template <bool kWrap>
__device__ void torus_link(PerShared &sh, const uint32_t *bm, bool smem_bm, unsigned long long *nd,
                           const uint32_t *perm, const uint32_t *rank, uint32_t L, uint32_t r0, uint32_t r1,
                           uint32_t axis)
{
    const uint32_t z = sh.z;
    bool bad = false;
    for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        if (kWrap && *reinterpret_cast<volatile uint32_t *>(&sh.flag)) break;
        const uint32_t i = __ldg(perm + r);
        // per axis k, the wrapped coordinates (x_k + d) mod L for d = -2..2, six bits each
        uint32_t wk[5], rest = i;
#pragma unroll
        for (int k = 4; k >= 0; --k) {
            const uint32_t xk = rest % L;
            rest /= L;
            uint32_t w = 0;
#pragma unroll
            for (uint32_t f = 0; f < 5u; ++f) w |= ((xk + 2u * L + f - 2u) % L) << (6u * f);
            wk[k] = w;
        }
        for (uint32_t v = 0; v < z; ++v) {
            const uint32_t packed = sh.offs[v];
            uint32_t j = 0;
#pragma unroll
            for (int k = 0; k < 5; ++k) j = j * L + ((wk[k] >> (6u * ((packed >> (3 * k)) & 7u))) & 63u);
            const uint32_t word = smem_bm ? bm[j >> 5] : __ldcg(bm + (j >> 5));
            if (!((word >> (j & 31u)) & 1u)) continue;
            const uint32_t rj = j == i ? r : __ldg(rank + j);
            if (rj > r || (!kWrap && rj == r)) continue;  // the later site takes the edge; loops only wind
            const int32_t step = zone_component(packed, static_cast<int>(axis));
            if (tunite(nd, r, rj, step, r1, bad) && kWrap) {
                *reinterpret_cast<volatile uint32_t *>(&sh.flag) = 1u;
                break;
            }
            if (bad) break;
        }
        if (bad) break;
    }
    if (bad) atomicOr(&sh.bad, 1u);
    __syncthreads();
}

// smem_L: samples with L <= smem_L keep the bitmap in the dynamic shared memory (0: none do).
template <bool kWrap>
__global__ void __launch_bounds__(kPerThreads, 1) k_torus(const perc_sample *__restrict__ samples, uint32_t num,
                                                          uint32_t max_L, uint32_t smem_L,
                                                          const uint64_t *__restrict__ n_in,
                                                          int64_t *__restrict__ mass_out,
                                                          uint32_t *__restrict__ nstar_out, char *ws, size_t slot_bytes)
{
    __shared__ PerShared sh;
    extern __shared__ uint32_t sbm[];
    PerHeader *hdr = reinterpret_cast<PerHeader *>(ws);
    char *slot = ws + sizeof(PerHeader) + size_t(blockIdx.x) * slot_bytes;
    for (;;) {
        if (threadIdx.x == 0) {
            sh.sample = atomicAdd(&hdr->queue, 1u);
            sh.bad = 0u;
        }
        __syncthreads();
        const uint32_t s = sh.sample;
        if (s >= num) break;
        const perc_sample smp = samples[s];
        const uint32_t L = smp.L, word = smp.zone_mask, mask = word & 0x7Fu, axis = word >> 8;
        const bool ok_word = mask != 0u && (word & ~0x77Fu) == 0u && axis < 5u;
        const bool ok = L >= 1u && L <= max_L && ok_word && smp.perm && smp.rank &&
                        (kWrap || n_in[s] <= num_sites(L));
        if (!ok) {
            if (threadIdx.x == 0) {
                if (kWrap)
                    nstar_out[s] = PERC_NEVER;
                else
                    mass_out[s] = -1;
                set_status(&hdr->status, PERC_EDEVICE);
            }
            __syncthreads();
            continue;
        }
        const uint32_t N = static_cast<uint32_t>(num_sites(L));
        const bool smem_bm = L <= smem_L;
        uint32_t *bm = smem_bm ? sbm : reinterpret_cast<uint32_t *>(slot);
        const size_t bm_bytes = per_align(per_bm_words(N) * 4), nd_bytes = per_align(size_t(N) * 8);
        unsigned long long *ndc = reinterpret_cast<unsigned long long *>(slot + bm_bytes);  // committed forest
        unsigned long long *ndw = reinterpret_cast<unsigned long long *>(slot + bm_bytes + nd_bytes);
        uint32_t *cnt = reinterpret_cast<uint32_t *>(slot + bm_bytes + 2 * nd_bytes);
        const uint32_t words = static_cast<uint32_t>(per_bm_words(N));
        for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) {
            if (smem_bm)
                bm[w] = 0u;
            else
                __stcg(bm + w, 0u);
        }
        if (threadIdx.x == 0) {  // the neighborhood's offsets, zone by zone
            uint32_t z = 0;
            for (int zone = 0; zone < kZoneCount; ++zone) {
                if (!(mask & (1u << zone))) continue;
                for (uint32_t k = c_tzones.start[zone]; k < c_tzones.start[zone + 1]; ++k) sh.offs[z++] = c_tzones.vec[k];
            }
            sh.z = z;
            sh.best = 0u;
        }
        __syncthreads();
        if (kWrap) {
            // bisection over n with the forest of the largest n known not to wrap (nc = lo - 1)
            // kept: a probe copies it and adds only the sites from nc up to the probe, and a probe
            // that wraps is dropped again (its bitmap bits cleared)
            uint32_t lo = 1, hi = N, nc = 0;  // wrap(N) holds (see the top of the file)
            while (lo < hi && !sh.bad) {
                const uint32_t mid = lo + (hi - lo) / 2u;  // > nc
                for (uint32_t r = threadIdx.x; r < nc; r += blockDim.x) __stcg(ndw + r, __ldcg(ndc + r));
                torus_add(bm, ndw, smp.perm, nc, mid);
                if (threadIdx.x == 0) sh.flag = 0u;
                __syncthreads();
                torus_link<true>(sh, bm, smem_bm, ndw, smp.perm, smp.rank, L, nc, mid, axis);
                const bool wrapped = sh.flag != 0u;
                __syncthreads();  // every thread has read the flag before the next probe clears it
                if (wrapped) {
                    hi = mid;
                    for (uint32_t r = nc + threadIdx.x; r < mid; r += blockDim.x) {
                        const uint32_t i = __ldg(smp.perm + r);
                        atomicAnd(bm + (i >> 5), ~(1u << (i & 31u)));
                    }
                    __syncthreads();  // cleared before the next probe sets bits again
                } else {
                    lo = mid + 1u;
                    unsigned long long *tmp = ndc;
                    ndc = ndw;
                    ndw = tmp;
                    nc = mid;
                }
            }
            if (threadIdx.x == 0) {
                nstar_out[s] = sh.bad ? PERC_NEVER : lo;
                if (sh.bad) set_status(&hdr->status, PERC_ETIMEOUT);
            }
        } else {
            const uint32_t n = static_cast<uint32_t>(n_in[s]);
            for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) __stcg(cnt + r, 0u);
            torus_add(bm, ndc, smp.perm, 0u, n);
            __syncthreads();
            torus_link<false>(sh, bm, smem_bm, ndc, smp.perm, smp.rank, L, 0u, n, axis);
            bool bad = sh.bad != 0u;
            for (uint32_t r = threadIdx.x; r < n && !bad; r += blockDim.x) {
                int32_t d;
                atomicAdd(cnt + tfind(ndc, r, d, n, bad), 1u);
            }
            if (bad) atomicOr(&sh.bad, 1u);
            __syncthreads();
            uint32_t best = 0;
            for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) best = max(best, __ldcg(cnt + r));
            best = __reduce_max_sync(0xffffffffu, best);
            if ((threadIdx.x & 31u) == 0u) atomicMax(&sh.best, best);
            __syncthreads();
            if (threadIdx.x == 0) {
                mass_out[s] = sh.bad ? -1 : static_cast<int64_t>(sh.best);
                if (sh.bad) set_status(&hdr->status, PERC_ETIMEOUT);
            }
        }
        __syncthreads();
    }
}

// Launch shape shared by the workspace query and the launch: one CTA per SM (1024 threads), at most
// one per sample and what the slot budget allows; the bitmap in shared memory when max_L <= 16.
int torus_cfg(uint32_t max_L, uint32_t num, uint32_t &grid, size_t &slot, size_t &smem)
{
    if (max_L < 1 || max_L > kPeriodicMaxL || num == 0) return PERC_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PERC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERC_ECUDA;
    slot = per_slot_bytes(num_sites(max_L));
    const size_t by_budget = std::max<size_t>(1, kPeriodicBudget / slot);
    grid = static_cast<uint32_t>(std::min<size_t>({size_t(num), size_t(sms), by_budget}));
    smem = max_L <= kTorusSmemMaxL ? per_bm_words(num_sites(max_L)) * 4 : 0;
    return PERC_OK;
}

template <bool kWrap>
int torus_launch(const perc_sample *samples, uint32_t num, uint32_t max_L, const uint64_t *n, int64_t *mass,
                 uint32_t *nstar, void *workspace, size_t ws_bytes, void *stream_)
{
    uint32_t grid = 0;
    size_t slot = 0, smem = 0;
    const int rc = torus_cfg(max_L, num, grid, slot, smem);
    if (rc != PERC_OK) return rc;
    if (ws_bytes < sizeof(PerHeader) + size_t(grid) * slot) return PERC_EWORKSPACE;
    // the dynamic shared-memory limit is per device: raised once per device to the largest asked for
    if (smem && ensure_smem_attr(kWrap ? kAttrTorusWrap : kAttrTorusMass, reinterpret_cast<const void *>(k_torus<kWrap>),
                                 smem) != PERC_OK)
        return PERC_ECUDA;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    // the queue starts again; the status word keeps the first error since the last perc_check
    if (cudaMemsetAsync(static_cast<char *>(workspace) + offsetof(PerHeader, queue), 0, sizeof(uint32_t), stream) !=
        cudaSuccess)
        return PERC_ECUDA;
    const uint32_t smem_L = smem ? max_L : 0u;
    k_torus<kWrap><<<grid, kPerThreads, smem, stream>>>(samples, num, max_L, smem_L, n, mass, nstar,
                                                        static_cast<char *>(workspace), slot);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

}  // namespace

size_t periodic_workspace_bytes(uint32_t max_L, uint32_t num)
{
    uint32_t grid = 0;
    size_t slot = 0, smem = 0;
    if (torus_cfg(max_L, num, grid, slot, smem) != PERC_OK) return 0;
    return sizeof(PerHeader) + size_t(grid) * slot;
}

}  // namespace perc

using namespace perc;

extern "C" int perc_mass_periodic(const perc_sample *samples, uint32_t num_samples, uint32_t max_L, const uint64_t *n,
                                  int64_t *mass, void *workspace, size_t ws_bytes, void *stream)
{
    if (!samples || !n || !mass || !workspace || num_samples == 0) return PERC_EINVAL;
    return torus_launch<false>(samples, num_samples, max_L, n, mass, nullptr, workspace, ws_bytes, stream);
}

extern "C" int perc_nstar_wrap(const perc_sample *samples, uint32_t num_samples, uint32_t max_L, uint32_t *nstar,
                               void *workspace, size_t ws_bytes, void *stream)
{
    if (!samples || !nstar || !workspace || num_samples == 0) return PERC_EINVAL;
    return torus_launch<true>(samples, num_samples, max_L, nullptr, nullptr, nstar, workspace, ws_bytes, stream);
}
