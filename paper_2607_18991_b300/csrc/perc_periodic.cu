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
// its step closes a winding path.  S_max counts the roots.  n* is found by a Newman--Ziff sweep in
// chunks of sites: the forest of the committed sites is kept, a chunk's hooks are tagged and logged,
// and a chunk that closes a winding path is undone and bisected, each probe extending the committed
// forest (wrapping is monotone in n, and it holds at n = L^5: every zone has a step with a non-zero
// component along every axis, and repeating it L times winds around the torus).
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
constexpr uint32_t kTorusRowCand = 625;  // (d1..d4) in {-2..2}^4
constexpr uint32_t kTorusRowMinL = 5, kTorusRowMaxL = 32;  // sides the row scan serves
constexpr uint32_t kWrapChunk = 512;  // sites one step of the wrap sweep adds (fastest of 256..2048 at L = 16)
constexpr unsigned long long kTag = 1ull << 63;  // node word bit: a hook of the running probe

struct PerHeader {
    int status;       // first device-side error (perc_check reads it)
    uint32_t queue;   // next sample
    uint32_t pad[62];
};
static_assert(sizeof(PerHeader) == 256, "header is 256 bytes");

__host__ __device__ inline size_t per_align(size_t b) { return (b + 255) & ~size_t(255); }
__host__ __device__ inline size_t per_bm_words(uint64_t N) { return size_t(N / 32 + 1); }

// Per-CTA slot: bitmap (one bit per site), the forest's node words (tag bit 63, parent at bits
// 32..62, displacement at bits 0..31) and one word per node: cluster counts (S_max) or the log of
// the running probe's hooks (n*).
__host__ __device__ inline size_t per_slot_bytes(uint64_t N)
{
    return per_align(per_bm_words(N) * 4) + per_align(size_t(N) * 8) + per_align(size_t(N) * 4);
}

__device__ __forceinline__ unsigned long long node_word(uint32_t parent, int32_t disp)
{
    return (static_cast<unsigned long long>(parent) << 32) | static_cast<uint32_t>(disp);
}
__device__ __forceinline__ uint32_t word_parent(unsigned long long w) { return static_cast<uint32_t>(w >> 32) & 0x7FFFFFFFu; }
__device__ __forceinline__ int32_t word_disp(unsigned long long w) { return static_cast<int32_t>(static_cast<uint32_t>(w)); }

// Root of x and pos(x) - pos(root) along the axis, with path halving by a compare-and-swap that
// may fail: every word read stays a true relative position, since positions inside a cluster never
// change once joined.  Halving shortcuts only untagged links, so a shortcut stays true when the
// running probe's tagged hooks are undone.  More than `cap` steps would mean a cycle in the forest:
// *bad is set.
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
        if (!((w | w2) & kTag)) atomicCAS(nd + x, w, node_word(g, dxg));
        acc += dxg;
        x = g;
    }
    bad = true;
    d = acc;
    return x;
}

// Joins the clusters of nodes a and b over a step with pos(b) = pos(a) + step (the larger root
// goes under the smaller).  With a log the hook is tagged and its node appended to the log.
// Returns true when a and b already were one cluster and the step disagrees with their
// coordinates: the edge closes a winding path.
__device__ bool tunite(unsigned long long *nd, uint32_t *log, uint32_t *logn, uint32_t a, uint32_t b, int32_t step,
                       uint32_t cap, bool &bad)
{
    const unsigned long long tag = log ? kTag : 0ull;
    for (uint32_t it = 0; it <= cap; ++it) {
        int32_t da, db;
        const uint32_t ra = tfind(nd, a, da, cap, bad);
        const uint32_t rb = tfind(nd, b, db, cap, bad);
        if (bad) return false;
        if (ra == rb) return da + step != db;
        const uint32_t lo = min(ra, rb), hi = max(ra, rb);
        const int32_t rel = ra < rb ? da + step - db : db - da - step;  // pos(hi) - pos(lo)
        if (atomicCAS(nd + hi, node_word(hi, 0), node_word(lo, rel) | tag) == node_word(hi, 0)) {
            if (log) __stcg(log + atomicAdd(logn, 1u), hi);
            return false;
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
    uint32_t logn;   // hooks in the running probe's log
    uint32_t nrows;  // row entries (row scan)
    uint32_t offs[kMaxOffsets];  // per offset: shifts 6 (d_k + 2) at bits 5k, d_axis + 2 at bits 28..30
    // per (d1..d4) with some d5 in the neighborhood: shifts 6 (d_k + 2) at bits 5k (k = 0..3), the
    // neighborhood's d5 values at bits 20..24 (bit d5 + 2), d_axis + 2 at bits 25..27 (axis < 4)
    uint32_t rows[kTorusRowCand];
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

// Clears the bitmap words of the sites of rank 0 .. r1-1 (every set bit belongs to one of them).
__device__ void torus_clear(uint32_t *bm, bool smem_bm, const uint32_t *perm, uint32_t r1)
{
    for (uint32_t r = threadIdx.x; r < r1; r += blockDim.x) {
        const uint32_t i = __ldg(perm + r);
        if (smem_bm)
            bm[i >> 5] = 0u;
        else
            __stcg(bm + (i >> 5), 0u);
    }
}

// The sites of rank a .. b-1 (bitmap bits and nodes set) join the forest `nd`: every edge is taken
// by its later site in rank order, so the sites' edges to each other and to the sites before a are
// all seen (the bitmap may hold later sites too; the rank test drops them).  With fewer sites than
// threads, 2..32 threads share a site's offsets.  With a log (the wrap sweep) the hooks are tagged
// and logged, and the pass stops once a winding path along the axis closes (sh.flag).  Ends with a
// barrier.
__device__ void torus_link(PerShared &sh, const uint32_t *bm, bool smem_bm, unsigned long long *nd, uint32_t *log,
                           const uint32_t *perm, const uint32_t *rank, const FastDiv &fd, uint32_t a, uint32_t b,
                           bool rows, bool axis4)
{
    const uint32_t L = fd.L, m = b - a, z = sh.z;
    const bool wrap = log != nullptr;
    uint32_t tps = 1;  // threads per site
    while (tps < 32u && 2u * tps * m <= blockDim.x) tps *= 2u;
    const uint32_t sub = threadIdx.x & (tps - 1u), stride = blockDim.x / tps;
    bool bad = false, stop = false;
    for (uint32_t k = threadIdx.x / tps; k < m && !stop; k += stride) {
        if (wrap && *reinterpret_cast<volatile uint32_t *>(&sh.flag)) break;
        const uint32_t r = a + k, i = __ldg(perm + r);
        // per axis q, the wrapped coordinates (x_q + d) mod L for d = -2..2, six bits each
        uint32_t x[5], wk[5];
        site_coords(i, fd, x);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            uint32_t w = 0;
#pragma unroll
            for (uint32_t f = 0; f < 5u; ++f) {
                uint32_t c;
                if (L >= 3u) {
                    const int32_t t = static_cast<int32_t>(x[q] + f) - 2;
                    c = static_cast<uint32_t>(t < 0 ? t + static_cast<int32_t>(L)
                                                    : (t >= static_cast<int32_t>(L) ? t - static_cast<int32_t>(L) : t));
                } else {
                    c = (x[q] + 2u * L + f - 2u) % L;
                }
                w |= c << (6u * f);
            }
            wk[q] = w;
        }
        // one neighbor j reached by a step along the axis: false ends this site's scan
        auto edge = [&](uint32_t j, int32_t step) -> bool {
            const uint32_t rj = j == i ? r : __ldg(rank + j);
            if (rj > r || (!wrap && rj == r)) return true;  // the later site takes the edge; loops only wind
            if (tunite(nd, log, &sh.logn, r, rj, step, b, bad) && wrap) {
                *reinterpret_cast<volatile uint32_t *>(&sh.flag) = 1u;
                return false;
            }
            return !bad;
        };
        if (rows) {
            // row scan: per (d1..d4) entry the x5 row of the wrapped (x1..x4) (L bits at bit row * L,
            // two words funnel-shifted), doubled so that the five bits (x5 - 2 .. x5 + 2) mod L are
            // contiguous, masked by the entry's d5 values
            const uint32_t x5s = x[4] + L - 2u >= L ? x[4] - 2u : x[4] + L - 2u;  // (x5 - 2) mod L
            const unsigned long long lmask = (1ull << L) - 1ull;
            for (uint32_t v = sub; v < sh.nrows && !stop; v += tps) {
                const uint32_t e = sh.rows[v];
                uint32_t row = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) row = row * L + ((wk[q] >> ((e >> (5 * q)) & 31u)) & 63u);
                const uint32_t bb = row * L, wi = bb >> 5;
                const uint32_t w0 = smem_bm ? bm[wi] : __ldcg(bm + wi), w1 = smem_bm ? bm[wi + 1u] : __ldcg(bm + wi + 1u);
                const unsigned long long bits = ((static_cast<unsigned long long>(w1) << 32 | w0) >> (bb & 31u)) & lmask;
                uint32_t win = static_cast<uint32_t>((bits | (bits << L)) >> x5s) & ((e >> 20) & 31u);
                while (win) {
                    const uint32_t t = __ffs(win) - 1u;
                    win &= win - 1u;
                    const uint32_t x5n = x5s + t >= L ? x5s + t - L : x5s + t;
                    const int32_t step = axis4 ? static_cast<int32_t>(t) - 2 : static_cast<int32_t>((e >> 25) & 7u) - 2;
                    if (!edge(bb + x5n, step)) {
                        stop = true;
                        break;
                    }
                }
            }
            continue;
        }
        for (uint32_t v = sub; v < z; v += tps) {
            const uint32_t o = sh.offs[v];
            uint32_t j = 0;
#pragma unroll
            for (int q = 0; q < 5; ++q) j = j * L + ((wk[q] >> ((o >> (5 * q)) & 31u)) & 63u);
            const uint32_t word = smem_bm ? bm[j >> 5] : __ldcg(bm + (j >> 5));
            if (!((word >> (j & 31u)) & 1u)) continue;
            if (!edge(j, static_cast<int32_t>((o >> 28) & 7u) - 2)) {
                stop = true;
                break;
            }
        }
    }
    if (bad) atomicOr(&sh.bad, 1u);
    __syncthreads();
}

// Ends the running probe of the wrap sweep: its logged hooks are undone (turned back into roots)
// or committed (their tags cleared).  Tagged words are never shortened by path halving, so each
// logged word is still the hook itself.  Ends with a barrier.
__device__ void torus_settle(const PerShared &sh, unsigned long long *nd, const uint32_t *log, bool undo)
{
    const uint32_t n = sh.logn;
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t x = __ldcg(log + k);
        __stcg(nd + x, undo ? node_word(x, 0) : (__ldcg(nd + x) & ~kTag));
    }
    __syncthreads();
}

// smem_L: samples with L <= smem_L keep the bitmap in the dynamic shared memory (0: none do).
// chunk: sites one step of the wrap sweep adds.
template <bool kWrap>
__global__ void __launch_bounds__(kPerThreads, 1) k_torus(const perc_sample *__restrict__ samples, uint32_t num,
                                                          uint32_t max_L, uint32_t smem_L,
                                                          const uint64_t *__restrict__ n_in,
                                                          int64_t *__restrict__ mass_out,
                                                          uint32_t *__restrict__ nstar_out, char *ws, size_t slot_bytes,
                                                          uint32_t chunk)
{
    __shared__ PerShared sh;
    extern __shared__ uint32_t sbm[];
    PerHeader *hdr = reinterpret_cast<PerHeader *>(ws);
    char *slot = ws + sizeof(PerHeader) + size_t(blockIdx.x) * slot_bytes;
    const uint32_t Nmax = static_cast<uint32_t>(num_sites(max_L));
    const size_t bm_bytes = per_align(per_bm_words(Nmax) * 4), nd_bytes = per_align(size_t(Nmax) * 8);
    unsigned long long *nd = reinterpret_cast<unsigned long long *>(slot + bm_bytes);
    uint32_t *aux = reinterpret_cast<uint32_t *>(slot + bm_bytes + nd_bytes);  // counts or hook log
    // the bitmaps start clear; each sample clears the words it set
    if (smem_L) {
        const uint32_t sw = static_cast<uint32_t>(per_bm_words(num_sites(smem_L)));
        for (uint32_t w = threadIdx.x; w < sw; w += blockDim.x) sbm[w] = 0u;
    } else {
        const uint32_t gw = static_cast<uint32_t>(per_bm_words(Nmax));
        uint32_t *gbm = reinterpret_cast<uint32_t *>(slot);
        for (uint32_t w = threadIdx.x; w < gw; w += blockDim.x) __stcg(gbm + w, 0u);
    }
    for (;;) {
        if (threadIdx.x == 0) {
            sh.sample = atomicAdd(&hdr->queue, 1u);
            sh.bad = 0u;
            sh.best = 0u;
            sh.nrows = 0u;
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
        const FastDiv fd = make_fastdiv(L);
        // the neighborhood's offsets, zone by zone, one thread per table entry
        uint32_t z = 0;
        for (int zone = 0; zone < kZoneCount; ++zone)
            if (mask & (1u << zone)) z += c_tzones.start[zone + 1] - c_tzones.start[zone];
        for (uint32_t t = threadIdx.x; t < uint32_t(kMaxOffsets); t += blockDim.x) {
            int zone = 0;
            while (t >= c_tzones.start[zone + 1]) ++zone;
            if (!(mask & (1u << zone))) continue;
            uint32_t pos = t;
            for (int q = 0; q < zone; ++q)
                if (!(mask & (1u << q))) pos -= c_tzones.start[q + 1] - c_tzones.start[q];
            const uint32_t packed = c_tzones.vec[t];
            uint32_t o = ((packed >> (3u * axis)) & 7u) << 28;
#pragma unroll
            for (int q = 0; q < 5; ++q) o |= (6u * ((packed >> (3 * q)) & 7u)) << (5 * q);
            sh.offs[pos] = o;
        }
        const bool rows = L >= kTorusRowMinL && L <= kTorusRowMaxL, axis4 = axis == 4u;
        if (rows) {  // the row entries: per (d1..d4) the d5 whose |v|^2 is one of the sample's zones
            for (uint32_t t = threadIdx.x; t < kTorusRowCand; t += blockDim.x) {
                uint32_t e = 0, s2 = 0, code = t;
#pragma unroll
                for (int q = 3; q >= 0; --q) {
                    const uint32_t f = code % 5u;  // d_q + 2
                    code /= 5u;
                    s2 += (f - 2u) * (f - 2u);
                    e |= (6u * f) << (5 * q);
                    if (static_cast<uint32_t>(q) == axis) e |= f << 25;
                }
                uint32_t d5m = 0;
#pragma unroll
                for (uint32_t f5 = 0; f5 < 5u; ++f5) {
                    const uint32_t r2 = s2 + (f5 - 2u) * (f5 - 2u);
                    if (r2 >= 1u && r2 <= 7u && ((mask >> (r2 - 1u)) & 1u)) d5m |= 1u << f5;
                }
                if (d5m) sh.rows[atomicAdd(&sh.nrows, 1u)] = e | (d5m << 20);
            }
        }
        if (threadIdx.x == 0) sh.z = z;
        __syncthreads();
        if (kWrap) {
            // the sweep: c sites committed, top sites in the bitmap with nodes set
            uint32_t c = 0, top = 0, res = 0;
            while (res == 0u) {
                uint32_t hi = min(N, c + chunk);
                if (hi <= c) {  // wrap(N) holds, so only a broken forest gets here
                    if (threadIdx.x == 0) sh.bad = 1u;
                    __syncthreads();
                    break;
                }
                torus_add(bm, nd, smp.perm, top, hi);
                top = hi;
                if (threadIdx.x == 0) {
                    sh.flag = 0u;
                    sh.logn = 0u;
                }
                __syncthreads();
                torus_link(sh, bm, smem_bm, nd, aux, smp.perm, smp.rank, fd, c, hi, rows, axis4);
                if (sh.bad) break;
                bool wrapped = sh.flag != 0u;
                torus_settle(sh, nd, aux, wrapped);
                if (!wrapped) {
                    c = hi;
                    continue;
                }
                // the first wrapping n lies in (c, hi]: bisection, each probe on the committed forest
                uint32_t lo = c + 1u;
                while (lo < hi) {
                    const uint32_t mid = lo + (hi - lo) / 2u;
                    if (threadIdx.x == 0) {
                        sh.flag = 0u;
                        sh.logn = 0u;
                    }
                    __syncthreads();
                    torus_link(sh, bm, smem_bm, nd, aux, smp.perm, smp.rank, fd, c, mid, rows, axis4);
                    if (sh.bad) break;
                    wrapped = sh.flag != 0u;
                    torus_settle(sh, nd, aux, wrapped);
                    if (wrapped) {
                        hi = mid;
                    } else {
                        c = mid;
                        lo = mid + 1u;
                    }
                }
                res = lo;
            }
            torus_clear(bm, smem_bm, smp.perm, top);
            if (threadIdx.x == 0) {
                nstar_out[s] = sh.bad ? PERC_NEVER : res;
                if (sh.bad) set_status(&hdr->status, PERC_ETIMEOUT);
            }
        } else {
            const uint32_t n = static_cast<uint32_t>(n_in[s]);
            for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) __stcg(aux + r, 0u);
            torus_add(bm, nd, smp.perm, 0u, n);
            __syncthreads();
            torus_link(sh, bm, smem_bm, nd, nullptr, smp.perm, smp.rank, fd, 0u, n, rows, axis4);
            bool bad = sh.bad != 0u;
            for (uint32_t r = threadIdx.x; r < n && !bad; r += blockDim.x) {
                int32_t d;
                atomicAdd(aux + tfind(nd, r, d, n, bad), 1u);
            }
            if (bad) atomicOr(&sh.bad, 1u);
            __syncthreads();
            uint32_t best = 0;
            for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) best = max(best, __ldcg(aux + r));
            best = __reduce_max_sync(0xffffffffu, best);
            if ((threadIdx.x & 31u) == 0u) atomicMax(&sh.best, best);
            torus_clear(bm, smem_bm, smp.perm, n);
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
                                                        static_cast<char *>(workspace), slot, kWrapChunk);
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
