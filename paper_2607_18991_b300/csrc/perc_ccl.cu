// perc_ccl.cu -- exact first-spanning n* (bisection over connected-component passes) and
// largest-cluster mass S_max(n) for 5D site percolation with complex neighborhoods.
//
// What is computed (paper: Introduction -- the spanning cluster appears for the first time at the
// threshold; Methods, "Computational methods" -- clusters of the first n sites of a random
// addition order; eq. Pmax -- S_max):
//   span(n) = some cluster of the sites with rank < n touches both x1 = 0 and x1 = L-1,
//   n*      = min { n : span(n) },  S_max(n) = size of the largest such cluster.
// span(n) is monotone in n (sites are only added), so n* is found by bisection; every probe is one
// connected-component pass.
//
// Design (one CTA per sample, persistent over a queue of samples):
//   * occupancy bitmap of the probe's n: 1 bit per site, in shared memory when L^5/8 bytes fit
//     (L <= 17: 177 KiB), otherwise in a per-CTA global slot; it is updated incrementally from the
//     rank prefix (set bits for ranks [n_old, n), clear them for [n, n_old));
//   * union-find in rank space: node r + 2 is the site of rank r, so a probe at n touches only n + 2
//     nodes; nodes 0 and 1 are the two borders (LO: x1 = 0, HI: x1 = L-1), and span(n) holds iff
//     node 1 has been hooked (it can only be hooked under node 0, the only smaller index);
//   * hooking: atomicCAS of the larger root onto the smaller root; pointer jumping: path halving
//     in every find;
//   * neighborhood offsets from the compile-time zone table in constant memory, expanded per
//     sample into (linear delta, 25-bit validity one-hot) pairs in shared memory;
//   * incremental probes: the union-find of the last non-spanning probe n_b is kept, and a probe
//     at n > n_b only merges the sites of rank [n_b, n) (each with its occupied neighbors of
//     smaller rank, the Newman--Ziff rule).  Hooks of roots that existed at n_b are tagged (bit
//     31) and logged; a spanning probe is undone by resetting the logged roots, a non-spanning
//     probe is committed by clearing their tags.  Path halving never shortcuts a tagged edge of
//     an old node, so the committed forest stays valid;
//   * a spanning probe stops as soon as node 1 is hooked (early exit), since span is decided.
#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "perc_common.cuh"

namespace perc {

constexpr uint32_t kTag = 0x80000000u;
constexpr uint32_t kSmemBitmapMaxL = 17;
constexpr uint32_t kSumMixL = 32;             // above this side a batch's region is that of side 16
constexpr size_t kSumReserve = size_t(16) << 10;  // shared memory kept for nodes and edges
constexpr size_t kSmemNodes = 16384;  // most union-find nodes a CTA keeps in shared memory
// Total per-CTA slot memory a launch aims at: a quarter of the device's memory (68 GiB on a B300).
constexpr uint32_t kSlotCapShare = 4;

__constant__ ZoneTable c_zones = kZones;

struct WsHeader {
    int status;
    uint32_t queue;
    uint32_t pad[62];
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

struct Ctl {
    uint32_t sample;
    uint32_t mid;     // probe n
    uint32_t nb;      // n of the committed (non-spanning) union-find
    uint32_t bm_n;    // n the bitmap currently holds
    uint32_t stop;    // early-exit flag of the running pass
    uint32_t logn;    // undo-log length
    uint32_t span;    // result of the last pass
    uint32_t bad;     // sample failed validation
    uint32_t z;       // offsets of the sample's neighborhood
    uint32_t R;       // row entries of the sample's neighborhood
    uint32_t NP;      // plane entries (L = 16 path)
    uint32_t Rhalf;   // row entries up to the centre row (d1..d4 = 0), which come first
    uint32_t NPhalf;  // plane entries up to the centre plane (d1..d3 = 0)
    uint32_t G;       // summary-group entries of the sample's neighborhood
    uint32_t Ghalf;   // summary-table entries up to the centre entry
    uint32_t axis;    // spanning axis of the sample: its borders are x_{axis+1} = 0 and = L-1
    uint32_t ecount[2];  // edge-list fill of the current and the next chunk
    unsigned long long hooks, new_sites, sites, unions, cyc_scan, cyc_link;
};

// ------------------------------------------------------------------------------------------------
// union-find on rank-space nodes.  The first `cap` nodes of a sample live in shared memory (the
// nodes of the earliest sites, which every later site reaches), the rest in the CTA's global slot
// (L2-coherent loads and stores).  Shared-memory accesses use explicit .shared instructions.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_cg(const uint32_t *p) { return __ldcg(p); }

__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v)
{
    asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t atoms_cas(uint32_t a, uint32_t cmp, uint32_t val)
{
    uint32_t old;
    asm volatile("atom.shared.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "r"(a), "r"(cmp), "r"(val) : "memory");
    return old;
}

struct Nodes {
    uint32_t *g;     // global nodes (node x at g[x], used for x >= cap)
    uint32_t sbase;  // shared-window address of node 0
    uint32_t cap;    // nodes held in shared memory
};

__device__ __forceinline__ uint32_t nd_ld(const Nodes &P, uint32_t x)
{
    return x < P.cap ? lds_u32(P.sbase + 4u * x) : __ldcg(P.g + x);
}

__device__ __forceinline__ void nd_st(const Nodes &P, uint32_t x, uint32_t v)
{
    if (x < P.cap)
        sts_u32(P.sbase + 4u * x, v);
    else
        __stcg(P.g + x, v);
}

__device__ __forceinline__ uint32_t nd_cas(const Nodes &P, uint32_t x, uint32_t cmp, uint32_t val)
{
    return x < P.cap ? atoms_cas(P.sbase + 4u * x, cmp, val) : atomicCAS(P.g + x, cmp, val);
}

// Root of x with path halving.  Nodes below nold existed at the committed state: their pointer is
// rewritten only when both skipped edges are untagged (committed edges).
__device__ __forceinline__ uint32_t uf_find(const Nodes &P, uint32_t x, uint32_t nold)
{
    for (;;) {
        const uint32_t p = nd_ld(P, x);
        const uint32_t pu = p & ~kTag;
        if (pu == x) return x;
        const uint32_t g = nd_ld(P, pu);
        const uint32_t gu = g & ~kTag;
        if (gu == pu) return pu;
        if (x >= nold || ((p | g) & kTag) == 0u) nd_st(P, x, gu);
        x = gu;
    }
}

// Merge the clusters of a and b; returns true if a hook was made.  Hooking node 1 (the x1 = L-1
// border, which only node 0 can take) decides the pass: it raises *stop.
__device__ __forceinline__ bool uf_unite(const Nodes &P, uint32_t a, uint32_t b, uint32_t nold,
                                         uint32_t *logb, uint32_t *logn, uint32_t *stop)
{
    a = uf_find(P, a, nold);
    b = uf_find(P, b, nold);
    while (a != b) {
        const uint32_t hi = a > b ? a : b;
        const uint32_t lo = a > b ? b : a;
        const bool old = hi < nold;
        const uint32_t seen = nd_cas(P, hi, hi, old ? (lo | kTag) : lo);
        if (seen == hi) {
            if (old) logb[atomicAdd(logn, 1u)] = hi;
            if (hi == 1u && stop) *reinterpret_cast<volatile uint32_t *>(stop) = 1u;
            return true;
        }
        a = uf_find(P, seen & ~kTag, nold);  // hi was hooked meanwhile: continue from its root
        b = uf_find(P, lo, nold);
    }
    return false;
}

// ------------------------------------------------------------------------------------------------
// per-sample setup: the neighborhood as "row offsets".  Offsets that share (d1..d4) differ only in
// d5, i.e. they hit one x5 row of the lattice; one row entry holds the linear offset of that row,
// the one-hot of d1..d4 (validity against the site's allowed mask) and the 5-bit set of d5 values
// of the neighborhood.  One funnel-shifted bitmap load then tests all d5 neighbors of a row.
// ------------------------------------------------------------------------------------------------
struct __align__(16) RowEntry {
    int32_t delta;    // ((d1*L + d2)*L + d3)*L + d4) * L
    uint32_t onehot;  // bit 5k + d_k + 2 for k = 0..3 (x1..x4)
    uint32_t d5mask;  // bit d5 + 2 for every d5 with (d1..d5) in the neighborhood
    uint32_t pad;
};
constexpr int kRowCand = 625;  // (d1..d4) in {-2..2}^4
// Rows are stored in ascending base-5 code of (d1+2, .., d4+2), i.e. in lexicographic order of
// (d1..d4).  The site index orders coordinates with x1 most significant, so an in-lattice neighbor
// has a smaller index than the site exactly when its offset's first non-zero component is
// negative: the rows before the centre row (code 312) hold only such neighbors, the centre row
// those with d5 < 0, and the rows after it none.
constexpr uint32_t kRowCentre = 312;

// Builds the row table of `mask` for side L (all threads; ends with a barrier); returns the count
// of rows and writes the number of offsets to *z.
__device__ uint32_t build_rows(uint32_t mask, uint32_t L, RowEntry *rows, uint32_t *scratch, Ctl &c)
{
    for (uint32_t t = threadIdx.x; t < kRowCand; t += blockDim.x) scratch[t] = 0u;
    __syncthreads();
    uint32_t z = 0;
    for (int zone = 0; zone < kZoneCount; ++zone)
        if (mask & (1u << zone)) z += c_zones.start[zone + 1] - c_zones.start[zone];
    for (uint32_t v = threadIdx.x; v < z; v += blockDim.x) {
        uint32_t k = v, packed = 0;
        for (int zone = 0; zone < kZoneCount; ++zone) {
            if (!(mask & (1u << zone))) continue;
            const uint32_t cnt = c_zones.start[zone + 1] - c_zones.start[zone];
            if (k < cnt) {
                packed = c_zones.vec[c_zones.start[zone] + k];
                break;
            }
            k -= cnt;
        }
        uint32_t key = 0;
        for (int d = 0; d < 4; ++d) key = key * 5u + static_cast<uint32_t>(zone_component(packed, d) + 2);
        atomicOr(scratch + key, 1u << (zone_component(packed, 4) + 2));
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        uint32_t count = 0, half = 0;
        for (uint32_t base = 0; base < static_cast<uint32_t>(kRowCand); base += 32) {
            const uint32_t key = base + lane;
            const uint32_t m = key < static_cast<uint32_t>(kRowCand) ? scratch[key] : 0u;
            const uint32_t bal = __ballot_sync(0xffffffffu, m != 0u);
            half += __popc(__ballot_sync(0xffffffffu, m != 0u && key <= kRowCentre));
            if (m) {
                RowEntry e;
                uint32_t kk = key, onehot = 0;
                int32_t delta = 0;
                int d[4];
                for (int q = 3; q >= 0; --q) {
                    d[q] = static_cast<int>(kk % 5u) - 2;
                    kk /= 5u;
                }
                for (int q = 0; q < 4; ++q) {
                    delta = delta * static_cast<int32_t>(L) + d[q];
                    onehot |= 1u << (5 * q + d[q] + 2);
                }
                e.delta = delta * static_cast<int32_t>(L);
                e.onehot = onehot;
                e.d5mask = m;
                e.pad = 0;
                rows[count + __popc(bal & ((1u << lane) - 1u))] = e;
            }
            count += __popc(bal);
        }
        if (lane == 0) {
            c.R = count;
            c.Rhalf = half;
            c.z = z;
        }
    }
    __syncthreads();
    return c.R;
}

__device__ __forceinline__ uint32_t site_allowed(const uint32_t x[5], uint32_t L)
{
    return allowed_bits(x[0], L) | (allowed_bits(x[1], L) << 5) | (allowed_bits(x[2], L) << 10) |
           (allowed_bits(x[3], L) << 15) | (allowed_bits(x[4], L) << 20);
}

// Bitmap layout: bit 64 + i is site i (two zero guard words before, two after), so the 5-bit window
// of a row starting at i - 2 never reaches below word 0.
constexpr uint32_t kBmGuard = 64;
__host__ __device__ inline uint32_t bm_words(uint64_t N) { return static_cast<uint32_t>((N + 2 * kBmGuard) / 32 + 1); }

template <bool kSmemBm>
__device__ __forceinline__ uint32_t bm_word(const uint32_t *bm, uint32_t k)
{
    return kSmemBm ? bm[k] : ld_cg(bm + k);
}

// Bitmap of the first n sites moves from bm_n to n.
__device__ void bitmap_update(uint32_t *bm, const uint32_t *perm, uint32_t bm_n, uint32_t n)
{
    if (n > bm_n) {
        for (uint32_t r = bm_n + threadIdx.x; r < n; r += blockDim.x) {
            const uint32_t i = __ldg(perm + r) + kBmGuard;
            atomicOr(bm + (i >> 5), 1u << (i & 31u));
        }
    } else {
        for (uint32_t r = n + threadIdx.x; r < bm_n; r += blockDim.x) {
            const uint32_t i = __ldg(perm + r) + kBmGuard;
            atomicAnd(bm + (i >> 5), ~(1u << (i & 31u)));
        }
    }
}

// ------------------------------------------------------------------------------------------------
// A connected-component pass over the new sites runs in chunks of up to blockDim sites, each in
// two phases:
//   scan  -- every thread tests the neighborhood of its site (or a share of it when a chunk has
//            few sites) against the bitmap and appends each hit as an edge (node, neighbor site) to
//            the CTA's edge list (shared memory, overflowing into the CTA's global slot);
//   unite -- every thread takes edges from the list, looks up the neighbor's rank, keeps the edge
//            if the neighbor came earlier (the Newman--Ziff rule: an edge is merged by its later
//            site) and merges the two clusters.
// Border edges (node 0 for x1 = 0, node 1 for x1 = L-1) carry kNodeFlag and skip the lookup.
// ------------------------------------------------------------------------------------------------
constexpr uint32_t kNodeFlag = 0x80000000u;

struct EdgeList {
    uint2 *s;       // shared part
    uint32_t scap;  // entries in the shared part
    uint2 *g;       // global overflow (entries scap..)
};

__device__ __forceinline__ void edge_put(const EdgeList &E, uint32_t k, uint2 v)
{
    if (k < E.scap)
        E.s[k] = v;
    else
        E.g[k - E.scap] = v;
}

__device__ __forceinline__ uint2 edge_get(const EdgeList &E, uint32_t k)
{
    return k < E.scap ? E.s[k] : E.g[k - E.scap];
}

// log2 of the threads that share one site in a chunk of `count` sites: one site per thread when
// there are enough sites, otherwise the neighborhood of a site is split over threads.
__device__ __forceinline__ uint32_t lanes_shift(uint32_t count, uint32_t R)
{
    uint32_t s = 0;
    while (s < 5u && (count << (s + 1)) <= blockDim.x && (1u << s) < R) ++s;
    return s;
}

// ------------------------------------------------------------------------------------------------
// L = 16 fast path: "planes".  With 16 sites per x5 row the five rows x4-2..x4+2 of a fixed
// (x1+d1, x2+d2, x3+d3) are 80 contiguous bits, and every plane offset is a multiple of 256 bits,
// so the bit shift of a site's 5x5 (d4, d5) block is the same for all planes.  Four word loads and
// three funnel shifts give the whole block; per-plane masks select the neighborhood's (d4, d5)
// and per-site masks the in-lattice ones.  Bit t of funnel F (F = 0..2) is site
// i + delta - 34 + 32F + t.
// ------------------------------------------------------------------------------------------------
constexpr uint32_t kPlaneL = 16;
constexpr int kPlaneCand = 125;  // (d1, d2, d3) in {-2..2}^3, stored in ascending base-5 code
constexpr uint32_t kPlaneCentre = 62;  // code of (0, 0, 0)

struct __align__(16) PlaneEntry {
    int32_t dword;   // plane offset / 32 (= ((d1*16 + d2)*16 + d3) * 8)
    uint32_t oh;     // bits 0..14: one-hot of d1..d3; bits 16..20: neighborhood mask of funnel 2
    uint32_t pm0;    // funnel 0: d4 = -2 in bits 0..4, d4 = -1 in bits 16..20 (bit d5 + 2)
    uint32_t pm1;    // funnel 1: d4 = 0 in bits 0..4, d4 = +1 in bits 16..20
};

// Plane table of `mask` from the row table (rows must be built; ends with a barrier).
__device__ uint32_t build_planes16(const RowEntry *rows, uint32_t R, PlaneEntry *planes, uint32_t *scratch, Ctl &c)
{
    // scratch[key * 5 + (d4 + 2)] = d5 mask, key = base-5 code of (d1, d2, d3)
    for (uint32_t t = threadIdx.x; t < kPlaneCand * 5; t += blockDim.x) scratch[t] = 0u;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < R; k += blockDim.x) {
        const RowEntry e = rows[k];
        int d[4];
        for (int q = 0; q < 4; ++q) {
            const uint32_t oh = (e.onehot >> (5 * q)) & 31u;
            d[q] = __ffs(oh) - 1 - 2;
        }
        const uint32_t key = static_cast<uint32_t>(((d[0] + 2) * 5 + (d[1] + 2)) * 5 + (d[2] + 2));
        scratch[key * 5 + static_cast<uint32_t>(d[3] + 2)] = e.d5mask;  // one row per (d1..d4)
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        uint32_t count = 0, half = 0;
        for (uint32_t base = 0; base < static_cast<uint32_t>(kPlaneCand); base += 32) {
            const uint32_t key = base + lane;
            uint32_t f[5] = {0u, 0u, 0u, 0u, 0u};
            if (key < static_cast<uint32_t>(kPlaneCand))
                for (int q = 0; q < 5; ++q) f[q] = scratch[key * 5 + q];
            const bool any = (f[0] | f[1] | f[2] | f[3] | f[4]) != 0u;
            const uint32_t bal = __ballot_sync(0xffffffffu, any);
            half += __popc(__ballot_sync(0xffffffffu, any && key <= kPlaneCentre));
            if (any) {
                const int d1 = static_cast<int>(key / 25u) - 2, d2 = static_cast<int>((key / 5u) % 5u) - 2,
                          d3 = static_cast<int>(key % 5u) - 2;
                PlaneEntry e;
                e.dword = ((d1 * 16 + d2) * 16 + d3) * 8;
                e.oh = (1u << (d1 + 2)) | (1u << (5 + d2 + 2)) | (1u << (10 + d3 + 2)) | (f[4] << 16);
                e.pm0 = f[0] | (f[1] << 16);
                e.pm1 = f[2] | (f[3] << 16);
                planes[count + __popc(bal & ((1u << lane) - 1u))] = e;
            }
            count += __popc(bal);
        }
        if (lane == 0) {
            c.NP = count;
            c.NPhalf = half;
        }
    }
    __syncthreads();
    return c.NP;
}

// ------------------------------------------------------------------------------------------------
// How a site's neighborhood is scanned (template parameter of the passes):
//   kScanRows    one funnel-shifted bitmap window per (d1..d4) row entry (any L);
//   kScanPlanes  L = 16: one 80-bit bitmap block per (d1, d2, d3) plane entry;
//   kScanGroups  with the occupancy summary in shared memory: per (d1, d2, d3) group entry one
//                5-bit summary window names the rows (d4) that may hold a neighbor, and only those
//                rows are read from the bitmap (any L);
//   kScanGroupsG the same with the summary in the CTA's global slot (lattices whose summary does
//                not fit in shared memory).
// The summary has one bit per lattice row (the L sites sharing x1..x4): bit kSumGuard + r is set
// once a site of row r = i / L is occupied.  It only ever gains bits, so the passes that use it are
// those whose occupancy only grows (the sweep, S_max windows, the mass pass).  It serves lattices
// whose bitmap lives in global memory (L above 17): near the threshold the occupancy is sparse
// (p_c z is of order one), so most summary windows are empty, and a site's scan reads 81 summary
// windows on chip instead of 297 bitmap rows through L2 (all seven zones).  While the whole bitmap
// sits in shared memory the row and plane tests are cheaper than the summary's data-dependent
// candidate loop, whose trip count differs from lane to lane.
// ------------------------------------------------------------------------------------------------
enum ScanMode : int { kScanRows = 0, kScanPlanes = 1, kScanGroups = 2, kScanGroupsG = 3 };
__host__ __device__ constexpr bool uses_sum(int m) { return m >= kScanGroups; }

constexpr uint32_t kSumGuard = 64;  // zero bits before the summary's row 0 (and 128 after the last row)
__host__ __device__ inline uint32_t sum_words(uint32_t L)
{
    const uint64_t rows = uint64_t(L) * L * L * L;
    return static_cast<uint32_t>((rows + kSumGuard + 128) / 32 + 1);
}
__host__ __device__ inline size_t sum_bytes(uint32_t L) { return (size_t(sum_words(L)) * 4 + 15) & ~size_t(15); }

// Group entry (kScanGroups): one (d1, d2, d3) triple of the neighborhood.
struct __align__(16) GroupEntry {
    int32_t rdelta;  // row offset of (d1, d2, d3, d4 = -2): ((d1*L + d2)*L + d3)*L - 2
    uint32_t oh;     // one-hot of d1, d2, d3: bit 5k + d_k + 2, k = 0..2
    uint32_t cm;     // bit d4 + 2 for every d4 whose row (d1..d4) is in the neighborhood
    uint32_t code;   // base-5 code of (d1, d2, d3, d4 = -2): index of its row in the d5 table
};

constexpr uint32_t kGroupCentre = 62;  // code of (0, 0, 0)
constexpr size_t kSumTabBytes = sizeof(GroupEntry) * 125;
constexpr size_t kD5Bytes = 640;                            // d5 masks of the 625 (d1..d4) rows

// Tables of the summary scan, pointers into shared memory (the summary may be global).
struct ScanTabs {
    const RowEntry *rows;
    const PlaneEntry *planes;
    const GroupEntry *tab;
    const uint8_t *d5m;    // d5 mask (bit d5 + 2) of every (d1..d4) row, by base-5 code
    uint32_t *sum;         // occupancy summary
};

// Builds the summary tables of `mask` for side L (all threads; ends with a barrier): the d5 mask of
// every (d1..d4) row, and the group entries in ascending code, those up to the centre entry first.
// scratch holds kRowCand words.
__device__ void build_sum_tabs(uint32_t mask, uint32_t L, GroupEntry *tab, uint8_t *d5m, uint32_t *scratch, Ctl &c)
{
    for (uint32_t t = threadIdx.x; t < kRowCand; t += blockDim.x) scratch[t] = 0u;
    __syncthreads();
    uint32_t z = 0;
    for (int zone = 0; zone < kZoneCount; ++zone)
        if (mask & (1u << zone)) z += c_zones.start[zone + 1] - c_zones.start[zone];
    for (uint32_t v = threadIdx.x; v < z; v += blockDim.x) {
        uint32_t k = v, packed = 0;
        for (int zone = 0; zone < kZoneCount; ++zone) {
            if (!(mask & (1u << zone))) continue;
            const uint32_t cnt = c_zones.start[zone + 1] - c_zones.start[zone];
            if (k < cnt) {
                packed = c_zones.vec[c_zones.start[zone] + k];
                break;
            }
            k -= cnt;
        }
        uint32_t key = 0;
        for (int d = 0; d < 4; ++d) key = key * 5u + static_cast<uint32_t>(zone_component(packed, d) + 2);
        atomicOr(scratch + key, 1u << (zone_component(packed, 4) + 2));
    }
    __syncthreads();
    uint8_t *d5w = d5m;
    for (uint32_t t = threadIdx.x; t < kRowCand; t += blockDim.x) d5w[t] = static_cast<uint8_t>(scratch[t]);
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x;
        uint32_t count = 0, half = 0;
        const int32_t Li = static_cast<int32_t>(L);
        {  // one lane per (d1, d2, d3) triple
            for (uint32_t base = 0; base < 125u; base += 32) {
                const uint32_t key = base + lane;
                uint32_t cm = 0;
                if (key < 125u)
                    for (uint32_t u = 0; u < 5; ++u) cm |= (scratch[key * 5u + u] ? 1u : 0u) << u;
                const uint32_t bal = __ballot_sync(0xffffffffu, cm != 0u);
                half += __popc(__ballot_sync(0xffffffffu, cm != 0u && key <= kGroupCentre));
                if (cm) {
                    const int32_t d1 = static_cast<int32_t>(key / 25u) - 2, d2 = static_cast<int32_t>((key / 5u) % 5u) - 2,
                                  d3 = static_cast<int32_t>(key % 5u) - 2;
                    GroupEntry e;
                    e.rdelta = ((d1 * Li + d2) * Li + d3) * Li - 2;
                    e.oh = (1u << (d1 + 2)) | (1u << (5 + d2 + 2)) | (1u << (10 + d3 + 2));
                    e.cm = cm;
                    e.code = key * 5u;
                    tab[count + __popc(bal & ((1u << lane) - 1u))] = e;
                }
                count += __popc(bal);
            }
        }
        if (lane == 0) {
            c.G = count;
            c.Ghalf = half;
            c.z = z;
        }
    }
    __syncthreads();
}

// Site geometry for the scan phase.
struct SiteGeo {
    uint32_t i;        // site index
    uint32_t allowed;  // rows / summary paths: 25-bit in-lattice mask of (d1..d5); plane path: (d1..d3) part
    uint32_t a5;       // in-lattice d5 values
    uint32_t a4;       // in-lattice d4 values (summary paths)
    uint32_t r0;       // row index i / L (summary group path)
    uint32_t sm0, sm1, sm2, sh, wbase;  // plane path only
    bool low, high;    // on the low / high border of the spanning axis (x_{axis+1} = 0 / L-1); false
                       // when the sample spans along any axis (axis kAnyAxis)
    uint32_t faces;    // bit 2k: x_{k+1} = 0, bit 2k + 1: x_{k+1} = L-1, k = 0..4
};

// Spanning along any axis (perc_nstar_any): the border flags of a cluster are the ten face bits of
// SiteGeo::faces, and a cluster spans once it holds both faces of some axis.
constexpr uint32_t kAnyAxis = 5u;
constexpr uint32_t kFaceLoBits = 0x155u;  // bit 2k of each axis k
__host__ __device__ inline bool spans_any(uint32_t f) { return (f & (f >> 1) & kFaceLoBits) != 0u; }

// A sample's zone_mask word: bits 0..6 the coordination zones, bits 8..10 the spanning axis 0..4,
// every other bit zero.
constexpr uint32_t kZoneBits = 0x7Fu, kAxisShift = 8u;
__device__ __forceinline__ bool valid_zone_word(uint32_t w)
{
    return (w & kZoneBits) != 0u && (w & ~(kZoneBits | (7u << kAxisShift))) == 0u && (w >> kAxisShift) < 5u;
}

template <int kMode>
__device__ __forceinline__ SiteGeo site_geo(uint32_t i, uint32_t L, const FastDiv &fd, uint32_t axis)
{
    SiteGeo s;
    s.i = i;
    s.a4 = s.r0 = 0u;
    if (kMode == kScanPlanes) {  // L = 16: coordinates are 4-bit fields of the index
        const uint32_t x1 = i >> 16, x2 = (i >> 12) & 15u, x3 = (i >> 8) & 15u, x4 = (i >> 4) & 15u, x5 = i & 15u;
        s.allowed = allowed_bits(x1, kPlaneL) | (allowed_bits(x2, kPlaneL) << 5) | (allowed_bits(x3, kPlaneL) << 10);
        const uint32_t a4 = allowed_bits(x4, kPlaneL);
        s.a5 = allowed_bits(x5, kPlaneL);
        s.sm0 = ((a4 & 1u) ? s.a5 : 0u) | ((a4 & 2u) ? (s.a5 << 16) : 0u);
        s.sm1 = ((a4 & 4u) ? s.a5 : 0u) | ((a4 & 8u) ? (s.a5 << 16) : 0u);
        s.sm2 = (a4 & 16u) ? s.a5 : 0u;
        s.sh = (i + 30u) & 31u;
        s.wbase = (i + 30u) >> 5;
        s.faces = 0u;
        const uint32_t xs[5] = {x1, x2, x3, x4, x5};
#pragma unroll
        for (int k = 0; k < 5; ++k)
            s.faces |= ((xs[k] == 0u) ? 1u : 0u) << (2 * k) | ((xs[k] == kPlaneL - 1u) ? 2u : 0u) << (2 * k);
        s.low = axis < kAnyAxis && ((s.faces >> (2u * axis)) & 1u);
        s.high = axis < kAnyAxis && ((s.faces >> (2u * axis + 1u)) & 1u);
    } else {
        uint32_t x[5];
        site_coords(i, fd, x);
        s.allowed = site_allowed(x, L);
        s.a5 = s.allowed >> 20;
        s.a4 = (s.allowed >> 15) & 31u;
        s.r0 = uses_sum(kMode) ? fdiv(i, fd) : 0u;
        s.sm0 = s.sm1 = s.sm2 = s.sh = s.wbase = 0u;
        s.faces = 0u;
#pragma unroll
        for (int k = 0; k < 5; ++k)
            s.faces |= ((x[k] == 0u) ? 1u : 0u) << (2 * k) | ((x[k] == L - 1u) ? 2u : 0u) << (2 * k);
        s.low = axis < kAnyAxis && ((s.faces >> (2u * axis)) & 1u);
        s.high = axis < kAnyAxis && ((s.faces >> (2u * axis + 1u)) & 1u);
    }
    return s;
}

// Hits of neighborhood entry k of a site: up to three 32-bit masks; bit t of mask f is the
// neighbor site base + 32 f + t.
template <bool kSmemBm, bool kPlanes>
__device__ __forceinline__ uint32_t entry_hits(const SiteGeo &g, const uint32_t *bm, const RowEntry *rows,
                                               const PlaneEntry *planes, uint32_t k, uint32_t h[3])
{
    h[0] = h[1] = h[2] = 0u;
    if (kPlanes) {
        // branch-free: a plane outside the lattice reads words 0..3 and is masked out, so that the
        // loads of successive entries need not wait on a divergent exit
        const PlaneEntry e = planes[k];
        const uint32_t ok = (e.oh & 0x7FFFu & ~g.allowed) == 0u ? 0xFFFFFFFFu : 0u;
        const uint32_t *w = bm + ((g.wbase + static_cast<uint32_t>(e.dword)) & ok);
        // the fourth word only matters when the 69-bit block starts past bit 27
        const uint32_t w0 = w[0], w1 = w[1], w2 = w[2], w3 = g.sh > 27u ? w[3] : 0u;
        h[0] = __funnelshift_r(w0, w1, g.sh) & e.pm0 & g.sm0 & ok;
        h[1] = __funnelshift_r(w1, w2, g.sh) & e.pm1 & g.sm1 & ok;
        h[2] = __funnelshift_r(w2, w3, g.sh) & (e.oh >> 16) & g.sm2 & ok;
        return g.i + static_cast<uint32_t>(e.dword) * 32u - 34u;
    } else {
        const RowEntry e = rows[k];
        if ((e.onehot & ~g.allowed) != 0u) return 0u;
        const uint32_t b = g.i + kBmGuard - 2u + static_cast<uint32_t>(e.delta);
        const uint32_t w = __funnelshift_r(bm_word<kSmemBm>(bm, b >> 5), bm_word<kSmemBm>(bm, (b >> 5) + 1u), b & 31u);
        h[0] = w & e.d5mask & g.a5;
        return g.i + static_cast<uint32_t>(e.delta) - 2u;
    }
}

template <int kMode>
__device__ __forceinline__ uint32_t sum_word(const uint32_t *sum, uint32_t k)
{
    return kMode == kScanGroupsG ? ld_cg(sum + k) : sum[k];
}

// Bits t of a 32-bit hit mask whose neighbor index base + t lies below the site: t < lim.
__device__ __forceinline__ uint32_t below_mask(int32_t lim)
{
    return lim <= 0 ? 0u : lim >= 32 ? 0xFFFFFFFFu : (1u << lim) - 1u;
}

// Summary scan of group k of a site: for every row of the group that the summary marks occupied,
// the row's 5-bit window of the bitmap (d5 = -2..2) masked by the neighborhood's d5 values and the
// lattice; emit(jb, h) for every non-empty one (bit t of h is the neighbor site jb + t).  kHalf keeps
// only neighbors below the site's index.
template <bool kSmemBm, int kMode, bool kHalf, class Emit>
__device__ __forceinline__ void sum_entry_hits(const SiteGeo &g, const uint32_t *bm, const ScanTabs &T, uint32_t L,
                                               uint32_t k, Emit &emit)
{
    {
        const GroupEntry e = T.tab[k];
        if ((e.oh & ~g.allowed & 0x7FFFu) != 0u) return;
        const uint32_t sb = g.r0 + kSumGuard + static_cast<uint32_t>(e.rdelta);
        uint32_t cand = __funnelshift_r(sum_word<kMode>(T.sum, sb >> 5), sum_word<kMode>(T.sum, (sb >> 5) + 1u), sb & 31u) &
                        e.cm & g.a4;
        while (cand) {
            const uint32_t u = __ffs(cand) - 1u;
            cand &= cand - 1u;
            const uint32_t m5 = T.d5m[e.code + u] & g.a5;
            const uint32_t jb = g.i + static_cast<uint32_t>(e.rdelta + static_cast<int32_t>(u)) * L - 2u;
            const uint32_t bb = jb + kBmGuard;
            uint32_t h =
                __funnelshift_r(bm_word<kSmemBm>(bm, bb >> 5), bm_word<kSmemBm>(bm, (bb >> 5) + 1u), bb & 31u) & m5;
            if (kHalf) h &= below_mask(static_cast<int32_t>(g.i - jb));
            if (h) emit(jb, h);
        }
    }
}

// The early-exit flag and the undo-log length live in shared memory for a one-CTA sample and in
// global memory (read L2-coherently) when a group of CTAs works on one sample; CTA `member` of a
// group of `members` takes every members-th chunk of the new sites.
template <bool kGroup>
__device__ __forceinline__ uint32_t read_flag(const uint32_t *f)
{
    return kGroup ? __ldcg(f) : *reinterpret_cast<const volatile uint32_t *>(f);
}

// kHalf: the pass covers every occupied site (r0 = 0 and the bitmap holds exactly the sites of rank
// below r1), so each edge is taken once, from its end with the larger site index: only the table
// entries up to the centre entry are scanned, their hits are cut to neighbors below the site, and
// every edge is merged (no rank-order rule).
template <bool kSmemBm, bool kFaces, int kMode, bool kGroup = false, bool kHalf = false>
__device__ __forceinline__ void union_pass(Ctl &c, const Nodes &P, uint32_t *logb, const uint32_t *bm,
                                           const ScanTabs &T, const EdgeList &E,
                                           const uint32_t *perm, const uint32_t *rank, uint32_t L,
                                           const FastDiv &fd, uint32_t r0, uint32_t r1, uint32_t nold,
                                           uint32_t *stop_flag = nullptr, uint32_t *logn = nullptr,
                                           uint32_t member = 0, uint32_t members = 1)
{
    constexpr bool kPlanes = kMode == kScanPlanes;
    const uint32_t R = uses_sum(kMode) ? (kHalf ? c.Ghalf : c.G)
                                       : kHalf ? (kPlanes ? c.NPhalf : c.Rhalf) : (kPlanes ? c.NP : c.R);
    const uint32_t gshift = lanes_shift(r1 - r0, R);
    const uint32_t gsize = 1u << gshift, gl = threadIdx.x & (gsize - 1u), grp = threadIdx.x >> gshift;
    const uint32_t chunk = blockDim.x >> gshift;
    if (!kGroup) {
        stop_flag = &c.stop;
        logn = &c.logn;
    }
    uint32_t *stopp = kFaces ? stop_flag : nullptr;
    uint32_t hooks = 0, sites = 0, unions = 0, parity = 0;
    for (uint32_t base = r0 + member * chunk; base < r1; base += members * chunk, parity ^= 1u) {
        uint32_t *ecount = &c.ecount[parity];
        const long long t_chunk = clock64();
        // ---- scan
        const uint32_t r = base + grp;
        if (r < r1) {
            const SiteGeo g = site_geo<kMode>(__ldg(perm + r), L, fd, c.axis);
            const uint32_t node = r + 2u;
            if (gl == 0u) {
                ++sites;
                if (kFaces && (g.low || g.high)) {
                    uint32_t k = atomicAdd(ecount, (g.low ? 1u : 0u) + (g.high ? 1u : 0u));
                    if (g.low) edge_put(E, k++, make_uint2(node, kNodeFlag | 0u));
                    if (g.high) edge_put(E, k, make_uint2(node, kNodeFlag | 1u));
                }
            }
            if constexpr (uses_sum(kMode)) {
                auto emit = [&](uint32_t jb, uint32_t h) {
                    uint32_t slot = atomicAdd(ecount, static_cast<uint32_t>(__popc(h)));
                    while (h) {
                        const uint32_t t = __ffs(h) - 1;
                        h &= h - 1u;
                        edge_put(E, slot++, make_uint2(node, jb + t));
                    }
                };
                for (uint32_t k = gl; k < R; k += gsize) sum_entry_hits<kSmemBm, kMode, kHalf>(g, bm, T, L, k, emit);
            } else for (uint32_t k = gl; k < R; k += gsize) {
                uint32_t h[3];
                const uint32_t jb = entry_hits<kSmemBm, kPlanes>(g, bm, T.rows, T.planes, k, h);
                if ((h[0] | h[1] | h[2]) == 0u) continue;
                if (kHalf) {  // only the centre entry reaches above the site (the same entry in every lane)
                    const int32_t lim = static_cast<int32_t>(g.i - jb);
                    if (lim < 96) {
                        h[0] &= below_mask(lim);
                        h[1] &= below_mask(lim - 32);
                        h[2] &= below_mask(lim - 64);
                    }
                }
                const uint32_t nh = __popc(h[0]) + __popc(h[1]) + __popc(h[2]);
                if (nh == 0u) continue;
                uint32_t slot = atomicAdd(ecount, nh);
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    uint32_t hf = h[f];
                    while (hf) {
                        const uint32_t t = __ffs(hf) - 1;
                        hf &= hf - 1u;
                        edge_put(E, slot++, make_uint2(node, jb + 32u * f + t));
                    }
                }
            }
        }
        __syncthreads();
        const long long t_scan = clock64();
        // ---- unite
        const uint32_t ne = *ecount;
        if (threadIdx.x == 0) c.ecount[parity ^ 1u] = 0u;  // the next chunk's counter
        // four edges a round: their rank lookups are issued together, then the unions follow
        for (uint32_t e0 = threadIdx.x; e0 < ne; e0 += 4u * blockDim.x) {
            if (kFaces && read_flag<kGroup>(stop_flag)) break;
            uint2 ed[4];
            uint32_t other[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t e = e0 + q * blockDim.x;
                ed[q] = e < ne ? edge_get(E, e) : make_uint2(0u, 0u);
                other[q] = (e < ne && !(ed[q].y & kNodeFlag)) ? __ldg(rank + ed[q].y) + 2u : (ed[q].y & ~kNodeFlag);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t e = e0 + q * blockDim.x;
                if (e >= ne) continue;
                if (!kHalf && !(ed[q].y & kNodeFlag) && other[q] >= ed[q].x) continue;  // the later site merges it
                ++unions;
                hooks += uf_unite(P, ed[q].x, other[q], nold, logb, logn, stopp) ? 1u : 0u;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long t_link = clock64();
            c.cyc_scan += static_cast<unsigned long long>(t_scan - t_chunk);
            c.cyc_link += static_cast<unsigned long long>(t_link - t_scan);
        }
        // span(n) is decided: stop.  In a group another CTA may raise the flag at any time, so the
        // CTA decides together (one barrier with an OR) and leaves the loop as a whole.
        if (kGroup) {
            if (kFaces && __syncthreads_or(read_flag<kGroup>(stop_flag) != 0u)) break;
        } else if (kFaces && read_flag<kGroup>(stop_flag)) {
            break;
        }
    }
    hooks = __reduce_add_sync(0xffffffffu, hooks);
    sites = __reduce_add_sync(0xffffffffu, sites);
    unions = __reduce_add_sync(0xffffffffu, unions);
    if ((threadIdx.x & 31u) == 0u) {
        if (hooks) atomicAdd(&c.hooks, static_cast<unsigned long long>(hooks));
        if (sites) atomicAdd(&c.sites, static_cast<unsigned long long>(sites));
        if (unions) atomicAdd(&c.unions, static_cast<unsigned long long>(unions));
    }
}

// Per-CTA global slot: union-find nodes, undo log, the bitmap when it does not fit in shared
// memory, and the overflow of the edge list (a chunk of blockDim sites with at most 892
// neighbors and 2 borders each).
__host__ __device__ inline size_t slot_edge_entries(uint32_t threads) { return size_t(threads) * (kMaxOffsets + 2); }

struct SlotPtrs {
    uint32_t *P, *logb, *gbm;
    uint2 *gedges;
    uint32_t *gsum;  // occupancy summary of lattices whose summary does not fit in shared memory
};

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// gsum_L: side whose occupancy summary the slot holds (0: none); log: the slot holds a second
// node-sized array (the bisection's undo log, the cluster counts of S_max and the mass pass; the
// sweep has none).
__host__ __device__ inline size_t slot_bytes_for(uint64_t Ncap, bool gbm, uint32_t threads, uint32_t gsum_L = 0,
                                                 bool log = true)
{
    return (log ? 2 : 1) * align256((Ncap + 2) * 4) + (gbm ? align256(size_t(bm_words(Ncap)) * 4) : 0) +
           align256(slot_edge_entries(threads) * sizeof(uint2)) + (gsum_L ? align256(sum_bytes(gsum_L)) : 0);
}

__device__ __forceinline__ SlotPtrs slot_ptrs(char *ws, size_t slot_bytes, uint64_t Ncap, bool gbm, bool gsum = false,
                                              bool log = true)
{
    char *base = ws + sizeof(WsHeader) + size_t(blockIdx.x) * slot_bytes;
    const size_t nodes = align256((Ncap + 2) * 4), arrays = (log ? 2 : 1) * nodes;
    const size_t bmb = gbm ? align256(size_t(bm_words(Ncap)) * 4) : 0;
    SlotPtrs s;
    s.P = reinterpret_cast<uint32_t *>(base);
    s.logb = log ? reinterpret_cast<uint32_t *>(base + nodes) : nullptr;
    s.gbm = gbm ? reinterpret_cast<uint32_t *>(base + arrays) : nullptr;
    s.gedges = reinterpret_cast<uint2 *>(base + arrays + bmb);
    s.gsum = gsum ? reinterpret_cast<uint32_t *>(base + arrays + bmb +
                                                 align256(slot_edge_entries(blockDim.x) * sizeof(uint2)))
                  : nullptr;
    return s;
}

// Shared-memory carve-up: [row table][plane table][bitmap of side smem_L][node_cap union-find
// nodes][edge list (the rest)]; the table-building scratch uses the start of the edge list.  The
// summary kernels use [summary tables][d5 masks][region][nodes][extra][edge list] instead
// (smem_ptrs_sum), with rows and planes null.
struct SmemPtrs {
    RowEntry *rows;
    PlaneEntry *planes;
    uint32_t *sbm;
    uint32_t *nodes;
    uint2 *edges;
    uint32_t *scratch;
    GroupEntry *tab;
    uint8_t *d5m;
};

__host__ __device__ inline size_t smem_tables_bytes() { return sizeof(RowEntry) * kRowCand + sizeof(PlaneEntry) * kPlaneCand; }

__host__ __device__ inline size_t smem_bitmap_bytes(uint32_t smem_L)
{
    return (size_t(bm_words(num_sites(smem_L))) * 4 + 15) & ~size_t(15);
}

__host__ __device__ inline size_t smem_nodes_bytes(uint32_t node_cap) { return (size_t(node_cap) * 4 + 15) & ~size_t(15); }

// `extra` bytes (a multiple of 16) between the nodes and the edge list belong to the caller (the
// window arrays of k_smax and k_nstar_sweep, which also lend them to the first pass as more nodes).
__device__ __forceinline__ SmemPtrs smem_ptrs(unsigned char *dyn, uint32_t smem_L, uint32_t node_cap, size_t extra = 0)
{
    SmemPtrs p;
    p.rows = reinterpret_cast<RowEntry *>(dyn);
    p.planes = reinterpret_cast<PlaneEntry *>(dyn + sizeof(RowEntry) * kRowCand);
    p.sbm = reinterpret_cast<uint32_t *>(dyn + smem_tables_bytes());
    const size_t nodes_at = smem_tables_bytes() + smem_bitmap_bytes(smem_L);
    p.nodes = reinterpret_cast<uint32_t *>(dyn + nodes_at);
    p.edges = reinterpret_cast<uint2 *>(dyn + nodes_at + smem_nodes_bytes(node_cap) + extra);
    p.scratch = reinterpret_cast<uint32_t *>(p.edges);
    p.tab = nullptr;
    p.d5m = nullptr;
    return p;
}

// Region of the summary kernels: a sample with L <= smem_L keeps its bitmap there, one with
// smem_L < L <= sum_L its occupancy summary (its bitmap is in the slot), a bigger one neither (both
// in the slot).
__host__ __device__ inline size_t region_bm_bytes(uint32_t L) { return L ? smem_bitmap_bytes(L) : 0; }

__host__ __device__ inline size_t smem_sum_tables_bytes() { return kSumTabBytes + kD5Bytes; }

// Shared memory of the summary kernels: [row table][plane table][group table][d5 masks][region]
// [node_cap nodes][extra][edge list].
__device__ __forceinline__ SmemPtrs smem_ptrs_sum(unsigned char *dyn, size_t region, uint32_t node_cap, size_t extra = 0)
{
    SmemPtrs p;
    p.rows = reinterpret_cast<RowEntry *>(dyn);
    p.planes = reinterpret_cast<PlaneEntry *>(dyn + sizeof(RowEntry) * kRowCand);
    p.tab = reinterpret_cast<GroupEntry *>(dyn + smem_tables_bytes());
    p.d5m = dyn + smem_tables_bytes() + kSumTabBytes;
    p.sbm = reinterpret_cast<uint32_t *>(dyn + smem_tables_bytes() + smem_sum_tables_bytes());
    const size_t nodes_at = smem_tables_bytes() + smem_sum_tables_bytes() + region;
    p.nodes = reinterpret_cast<uint32_t *>(dyn + nodes_at);
    p.edges = reinterpret_cast<uint2 *>(dyn + nodes_at + smem_nodes_bytes(node_cap) + extra);
    p.scratch = reinterpret_cast<uint32_t *>(p.edges);
    return p;
}

// This sample's bitmap and summary (see smem_ptrs_sum); sum is null while the bitmap is on chip.
__device__ __forceinline__ void sample_bm_sum(const SmemPtrs &sm, const SlotPtrs &sp, uint32_t L, uint32_t smem_L,
                                              uint32_t sum_L, uint32_t *&bm, uint32_t *&sum)
{
    if (L <= smem_L) {
        bm = sm.sbm;
        sum = nullptr;
    } else {
        bm = sp.gbm;
        sum = L <= sum_L ? sm.sbm : sp.gsum;
    }
}

// Per-sample setup of the summary kernels (all threads; ends with a barrier): bitmap (and summary)
// cleared, and the scan tables of the sample's path: rows (and planes at L = 16) while the bitmap is
// on chip, the summary groups otherwise.
__device__ __forceinline__ void sample_tables(Ctl &c, const SmemPtrs &sm, uint32_t *bm, uint32_t *sum, uint32_t L,
                                              uint32_t mask, bool smem_bm)
{
    const uint32_t words = bm_words(num_sites(L));
    for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
    if (smem_bm) {
        build_rows(mask, L, sm.rows, sm.scratch, c);
        if (L == kPlaneL) build_planes16(sm.rows, c.R, sm.planes, sm.scratch, c);
    } else {
        const uint32_t swords = sum_words(L);
        for (uint32_t w = threadIdx.x; w < swords; w += blockDim.x) sum[w] = 0u;
        build_sum_tabs(mask, L, sm.tab, sm.d5m, sm.scratch, c);
    }
}

// Bitmap and summary gain the sites of rank [n0, n1).
__device__ __forceinline__ void bitmap_add_sum(uint32_t *bm, uint32_t *sum, const uint32_t *perm, uint32_t n0,
                                               uint32_t n1, const FastDiv &fd)
{
    for (uint32_t r = n0 + threadIdx.x; r < n1; r += blockDim.x) {
        const uint32_t site = __ldg(perm + r), i = site + kBmGuard;
        atomicOr(bm + (i >> 5), 1u << (i & 31u));
        const uint32_t row = fdiv(site, fd) + kSumGuard;
        atomicOr(sum + (row >> 5), 1u << (row & 31u));
    }
}

struct PhaseClock {
    unsigned long long update = 0, unite = 0, commit = 0, setup = 0;
};

template <bool kSmemBm>
__device__ __forceinline__ uint32_t probe(Ctl &c, const Nodes &P, uint32_t *logb, uint32_t *bm,
                                          const SmemPtrs &sm, const EdgeList &E, const uint32_t *perm,
                                          const uint32_t *rank,
                                          uint32_t L, const FastDiv &fd, PhaseClock &clk, bool &stopped)
{
    const uint32_t mid = c.mid, nb = c.nb, bm_n = c.bm_n;
    if (kSmemBm) bm = sm.sbm;  // keep the shared-memory address space visible to the compiler
    const long long t0 = clock64();
    bitmap_update(bm, perm, bm_n, mid);
    for (uint32_t r = nb + threadIdx.x; r < mid; r += blockDim.x) nd_st(P, r + 2u, r + 2u);
    __syncthreads();
    const long long t1 = clock64();
    // (the chunk loop of the union pass ends with a block barrier, mid > nb gives at least one chunk)
    const ScanTabs T{sm.rows, sm.planes, nullptr, nullptr, nullptr};
    if (kSmemBm && L == kPlaneL)
        union_pass<true, true, kScanPlanes>(c, P, logb, sm.sbm, T, E, perm, rank, L, fd, nb, mid, nb + 2u);
    else
        union_pass<kSmemBm, true, kScanRows>(c, P, logb, bm, T, E, perm, rank, L, fd, nb, mid, nb + 2u);
    const long long t2 = clock64();
    clk.update += t1 - t0;
    clk.unite += t2 - t1;
    const uint32_t span = nd_ld(P, 1u) != 1u;
    const uint32_t logn = c.logn;
    stopped = c.stop != 0u;
    __syncthreads();  // every thread has read span before node 1 may be reset below
    for (uint32_t k = threadIdx.x; k < logn; k += blockDim.x) {
        const uint32_t b = logb[k];
        nd_st(P, b, span ? b : (nd_ld(P, b) & ~kTag));  // undo, or commit the hook
    }
    __syncthreads();
    clk.commit += clock64() - t2;
    return span;
}

__global__ void __launch_bounds__(1024, 1)
k_nstar(const perc_sample *__restrict__ samples, uint32_t num, uint32_t max_L, uint32_t smem_L, uint32_t node_cap,
        uint32_t edge_scap,
        const uint32_t *__restrict__ bracket, uint32_t *__restrict__ nstar_out,
        uint32_t *__restrict__ passes_out, perc_stats *stats, char *ws, size_t slot_bytes)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    const SmemPtrs sm = smem_ptrs(dyn, smem_L, node_cap);
    __shared__ Ctl c;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const uint64_t Ncap = num_sites(max_L);
    const SlotPtrs sp = slot_ptrs(ws, slot_bytes, Ncap, max_L > smem_L);
    const EdgeList E{sm.edges, edge_scap, sp.gedges};
    const Nodes P{sp.P, static_cast<uint32_t>(__cvta_generic_to_shared(sm.nodes)), node_cap};
    uint32_t *logb = sp.logb;
    unsigned long long tot_passes = 0, tot_probe = 0, tot_early = 0, tot_fb = 0, tot_ok = 0;
    PhaseClock clk;

    for (;;) {
        if (threadIdx.x == 0) {
            c.sample = atomicAdd(&hdr->queue, 1u);
            c.hooks = 0;
            c.new_sites = 0;
            c.sites = 0;
            c.unions = 0;
            c.cyc_scan = 0;
            c.cyc_link = 0;
        }
        __syncthreads();
        const long long t_setup = clock64();
        const uint32_t s = c.sample;
        if (s >= num) break;
        const perc_sample smp = samples[s];
        const uint32_t L = smp.L, mask = smp.zone_mask & kZoneBits, axis = smp.zone_mask >> kAxisShift;
        if (L < 1u || L > max_L || !valid_zone_word(smp.zone_mask) || !smp.perm || !smp.rank) {
            if (threadIdx.x == 0) {
                nstar_out[s] = PERC_NEVER;
                if (passes_out) passes_out[s] = 0;
                set_status(&hdr->status, PERC_EDEVICE);
            }
            __syncthreads();
            continue;
        }
        const uint32_t N = static_cast<uint32_t>(num_sites(L));
        const bool smem_bm = L <= smem_L;
        uint32_t *bm = smem_bm ? sm.sbm : sp.gbm;
        const uint32_t words = bm_words(N);
        for (uint32_t w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
        build_rows(mask, L, sm.rows, sm.scratch, c);
        if (smem_bm && L == kPlaneL) build_planes16(sm.rows, c.R, sm.planes, sm.scratch, c);
        if (threadIdx.x == 0) {
            nd_st(P, 0u, 0u);
            nd_st(P, 1u, 1u);
            c.axis = axis;
        }
        const FastDiv fd = make_fastdiv(L);
        __syncthreads();
        clk.setup += clock64() - t_setup;

        // bisection state (every thread keeps the same copy; all decisions are block-uniform).
        // A learned bracket [blo, bhi] is verified lazily: not span(blo - 1) is probed first (its
        // union-find is the base of every later probe); span(bhi) holds as soon as any bisection
        // probe spans, and is probed on its own only if none did.
        const uint32_t n_top = (L <= 2u) ? N + 1u : N;  // span(N) holds for every mask when L >= 3
        uint32_t lo = 1, hi = n_top, nb = 0, bm_n = 0, npass = 0;
        int stage = 2;  // 0: verify not span(blo - 1), 2: bisect
        bool hi_known = true;  // span(hi) is established (by a probe or, plain, by construction)
        uint32_t blo = 0, bhi = 0;
        if (bracket) {
            blo = bracket[2 * size_t(s)];
            bhi = bracket[2 * size_t(s) + 1];
            if (blo >= 1u && blo <= bhi && bhi <= N) {
                stage = blo > 1u ? 0 : 2;
                lo = blo;
                hi = bhi;
                hi_known = false;
            } else {
                ++tot_fb;
            }
        }
        for (;;) {
            uint32_t mid;
            if (stage == 0)
                mid = blo - 1u;
            else if (lo < hi)
                mid = lo + (hi - lo) / 2u;
            else if (!hi_known)
                mid = hi;  // every probe inside the bracket stayed below: check span(bhi) itself
            else
                break;
            if (threadIdx.x == 0) {
                c.mid = mid;
                c.nb = nb;
                c.bm_n = bm_n;
                c.stop = 0;
                c.logn = 0;
                c.ecount[0] = 0;
                c.new_sites += mid - nb;
            }
            __syncthreads();
            bool stopped = false;
            const uint32_t span = smem_bm ? probe<true>(c, P, logb, bm, sm, E, smp.perm, smp.rank, L, fd, clk, stopped)
                                          : probe<false>(c, P, logb, bm, sm, E, smp.perm, smp.rank, L, fd, clk, stopped);
            ++npass;
            tot_probe += mid;
            if (span && stopped) ++tot_early;
            bm_n = mid;
            if (!span) nb = mid;
            if (stage == 0) {
                if (span) {  // n* < blo: the bracket is wrong, bisect the full range
                    lo = 1; hi = n_top; nb = 0; hi_known = true; ++tot_fb;
                }
                stage = 2;
            } else if (lo == hi) {  // the lazy check of span(bhi)
                if (span) {
                    hi_known = true;
                } else {  // n* > bhi: the bracket is wrong, bisect the full range
                    lo = 1; hi = n_top; nb = 0; hi_known = true; ++tot_fb;
                }
            } else if (span) {
                hi = mid;
                hi_known = true;
            } else {
                lo = mid + 1u;
            }
            // no barrier here: after the probe's last barrier no thread reads the Ctl fields that
            // thread 0 rewrites for the next probe before that probe's first barrier
        }
        if (bracket && blo >= 1u && blo <= bhi && bhi <= N && lo >= blo && lo <= bhi && npass > 0) ++tot_ok;
        if (threadIdx.x == 0) {
            nstar_out[s] = (lo == N + 1u) ? PERC_NEVER : lo;
            if (passes_out) passes_out[s] = npass;
            tot_passes += npass;
            if (stats) {
                atomicAdd(&stats->hooks, c.hooks);
                atomicAdd(&stats->new_sites, c.new_sites);
                atomicAdd(&stats->sites_merged, c.sites);
                atomicAdd(&stats->unions, c.unions);
                atomicAdd(&stats->cyc_scan, c.cyc_scan);
                atomicAdd(&stats->cyc_link, c.cyc_link);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && stats) {
        atomicAdd(&stats->passes, tot_passes);
        atomicAdd(&stats->probe_sites, tot_probe);
        atomicAdd(&stats->early_exits, tot_early);
        atomicAdd(&stats->fallbacks, tot_fb);
        atomicAdd(&stats->verified, tot_ok);
        atomicAdd(&stats->cyc_setup, clk.setup);
        atomicAdd(&stats->cyc_update, clk.update);
        atomicAdd(&stats->cyc_union, clk.unite);
        atomicAdd(&stats->cyc_commit, clk.commit);
    }
}

// ------------------------------------------------------------------------------------------------
// k_nstar_group: `members` co-resident CTAs (a cooperative launch) share one sample, for lattices
// whose bitmap lives in global memory and batches too small to give every SM a sample of its own
// (e.g. L = 40).  The group's union-find, undo log and bitmap are in its global slot; the CTAs
// split the bitmap update, the chunks of new sites and the commit, and meet at group barriers.
// Every wait is bounded: a barrier that is not reached within `spin_limit` polls (kSpinLimit unless
// PERC_OPT_SPIN_LIMIT sets another) sets PERC_ETIMEOUT and an abort flag, and every CTA of the
// group returns.
// ------------------------------------------------------------------------------------------------

struct GroupState {  // at the start of a group's slot (256 bytes)
    uint32_t bar_count, bar_gen, abort, sample;
    uint32_t stop, logn, pad[58];
};
static_assert(sizeof(GroupState) == 256, "group state is 256 bytes");

// Returns false if the group aborted (a wait ran out); all threads of the CTA agree.
__device__ __forceinline__ bool group_sync(GroupState *gs, uint32_t members, int *status, uint32_t *ok_s,
                                           uint32_t spin_limit)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ok = 1u;
        const uint32_t gen = __ldcg(&gs->bar_gen);
        __threadfence();
        if (atomicAdd(&gs->bar_count, 1u) == members - 1u) {
            atomicExch(&gs->bar_count, 0u);
            __threadfence();
            atomicAdd(&gs->bar_gen, 1u);
        } else {
            uint32_t it = 0;
            while (__ldcg(&gs->bar_gen) == gen) {
                if (__ldcg(&gs->abort)) {
                    ok = 0u;
                    break;
                }
                if (++it >= spin_limit) {
                    set_status(status, PERC_ETIMEOUT);
                    atomicExch(&gs->abort, 1u);
                    ok = 0u;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *reinterpret_cast<volatile uint32_t *>(ok_s) = ok;
    }
    __syncthreads();
    return *reinterpret_cast<volatile uint32_t *>(ok_s) != 0u;
}

__host__ __device__ inline size_t group_slot_bytes(uint64_t Ncap, uint32_t threads, uint32_t members)
{
    return sizeof(GroupState) + 2 * align256((Ncap + 2) * 4) + align256(size_t(bm_words(Ncap)) * 4) +
           size_t(members) * align256(slot_edge_entries(threads) * sizeof(uint2));
}

__global__ void __launch_bounds__(1024, 1)
k_nstar_group(const perc_sample *__restrict__ samples, uint32_t num, uint32_t max_L, uint32_t members,
              uint32_t edge_scap, const uint32_t *__restrict__ bracket, uint32_t *__restrict__ nstar_out,
              uint32_t *__restrict__ passes_out, perc_stats *stats, char *ws, size_t slot_bytes,
              uint32_t spin_limit)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    // shared memory: [row table][plane table (unused)][edge list]
    RowEntry *rows = reinterpret_cast<RowEntry *>(dyn);
    uint2 *sedges = reinterpret_cast<uint2 *>(dyn + smem_tables_bytes());
    __shared__ Ctl c;
    __shared__ uint32_t ok_s;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const uint32_t group = blockIdx.x / members, member = blockIdx.x % members;
    const bool leader = member == 0u;
    const uint64_t Ncap = num_sites(max_L);
    char *base = ws + sizeof(WsHeader) + size_t(group) * slot_bytes;
    GroupState *gs = reinterpret_cast<GroupState *>(base);
    const size_t nodes_b = align256((Ncap + 2) * 4), bm_b = align256(size_t(bm_words(Ncap)) * 4);
    uint32_t *gP = reinterpret_cast<uint32_t *>(base + sizeof(GroupState));
    uint32_t *logb = reinterpret_cast<uint32_t *>(base + sizeof(GroupState) + nodes_b);
    uint32_t *bm = reinterpret_cast<uint32_t *>(base + sizeof(GroupState) + 2 * nodes_b);
    uint2 *gedges = reinterpret_cast<uint2 *>(base + sizeof(GroupState) + 2 * nodes_b + bm_b +
                                              size_t(member) * align256(slot_edge_entries(blockDim.x) * sizeof(uint2)));
    const EdgeList E{sedges, edge_scap, gedges};
    const Nodes P{gP, 0u, 0u};
    const uint32_t gthreads = members * blockDim.x, gtid = member * blockDim.x + threadIdx.x;
    unsigned long long tot_passes = 0, tot_probe = 0, tot_early = 0, tot_fb = 0, tot_ok = 0;
    PhaseClock clk;
    bool alive = true;

    while (alive) {
        if (threadIdx.x == 0) {
            c.hooks = 0;
            c.new_sites = 0;
            c.sites = 0;
            c.unions = 0;
            c.cyc_scan = 0;
            c.cyc_link = 0;
            if (leader) atomicExch(&gs->sample, atomicAdd(&hdr->queue, 1u));
        }
        if (!(alive = group_sync(gs, members, &hdr->status, &ok_s, spin_limit))) break;
        const long long t_setup = clock64();
        const uint32_t s = __ldcg(&gs->sample);
        if (!(alive = group_sync(gs, members, &hdr->status, &ok_s, spin_limit))) break;  // all have read it
        if (s >= num) break;
        const perc_sample smp = samples[s];
        const uint32_t L = smp.L, mask = smp.zone_mask & kZoneBits, axis = smp.zone_mask >> kAxisShift;
        if (L < 1u || L > max_L || !valid_zone_word(smp.zone_mask) || !smp.perm || !smp.rank) {
            if (leader && threadIdx.x == 0) {
                nstar_out[s] = PERC_NEVER;
                if (passes_out) passes_out[s] = 0;
                set_status(&hdr->status, PERC_EDEVICE);
            }
            continue;
        }
        const uint32_t N = static_cast<uint32_t>(num_sites(L));
        const uint32_t words = bm_words(N);
        for (uint32_t w = gtid; w < words; w += gthreads) __stcg(bm + w, 0u);
        build_rows(mask, L, rows, reinterpret_cast<uint32_t *>(sedges), c);
        if (leader && threadIdx.x == 0) {
            nd_st(P, 0u, 0u);
            nd_st(P, 1u, 1u);
        }
        if (threadIdx.x == 0) c.axis = axis;  // every member CTA's own copy
        const FastDiv fd = make_fastdiv(L);
        if (!(alive = group_sync(gs, members, &hdr->status, &ok_s, spin_limit))) break;
        clk.setup += clock64() - t_setup;

        const uint32_t n_top = (L <= 2u) ? N + 1u : N;
        uint32_t lo = 1, hi = n_top, nb = 0, bm_n = 0, npass = 0;
        int stage = 2;
        bool hi_known = true;
        uint32_t blo = 0, bhi = 0;
        if (bracket) {
            blo = bracket[2 * size_t(s)];
            bhi = bracket[2 * size_t(s) + 1];
            if (blo >= 1u && blo <= bhi && bhi <= N) {
                stage = blo > 1u ? 0 : 2;
                lo = blo;
                hi = bhi;
                hi_known = false;
            } else {
                ++tot_fb;
            }
        }
        for (;;) {
            uint32_t mid;
            if (stage == 0)
                mid = blo - 1u;
            else if (lo < hi)
                mid = lo + (hi - lo) / 2u;
            else if (!hi_known)
                mid = hi;
            else
                break;
            if (threadIdx.x == 0) {
                c.ecount[0] = 0;
                c.new_sites += mid - nb;
                if (leader) {
                    atomicExch(&gs->stop, 0u);
                    atomicExch(&gs->logn, 0u);
                }
            }
            if (!(alive = group_sync(gs, members, &hdr->status, &ok_s, spin_limit))) break;
            const long long t0 = clock64();
            // bitmap of the first mid sites and fresh nodes for the new ones, split over the group
            if (mid > bm_n) {
                for (uint32_t r = bm_n + gtid; r < mid; r += gthreads) {
                    const uint32_t i = __ldg(smp.perm + r) + kBmGuard;
                    atomicOr(bm + (i >> 5), 1u << (i & 31u));
                }
            } else {
                for (uint32_t r = mid + gtid; r < bm_n; r += gthreads) {
                    const uint32_t i = __ldg(smp.perm + r) + kBmGuard;
                    atomicAnd(bm + (i >> 5), ~(1u << (i & 31u)));
                }
            }
            for (uint32_t r = nb + gtid; r < mid; r += gthreads) nd_st(P, r + 2u, r + 2u);
            if (!(alive = group_sync(gs, members, &hdr->status, &ok_s, spin_limit))) break;
            const long long t1 = clock64();
            const ScanTabs T{rows, nullptr, nullptr, nullptr, nullptr};
            union_pass<false, true, kScanRows, true>(c, P, logb, bm, T, E, smp.perm, smp.rank, L, fd, nb, mid,
                                                 nb + 2u, &gs->stop, &gs->logn, member, members);
            if (!(alive = group_sync(gs, members, &hdr->status, &ok_s, spin_limit))) break;
            const long long t2 = clock64();
            const uint32_t span = nd_ld(P, 1u) != 1u;
            const uint32_t logn = __ldcg(&gs->logn);
            const bool stopped = __ldcg(&gs->stop) != 0u;
            if (!(alive = group_sync(gs, members, &hdr->status, &ok_s, spin_limit))) break;  // all have read span
            for (uint32_t k = gtid; k < logn; k += gthreads) {
                const uint32_t b = __ldcg(logb + k);
                nd_st(P, b, span ? b : (nd_ld(P, b) & ~kTag));
            }
            if (!(alive = group_sync(gs, members, &hdr->status, &ok_s, spin_limit))) break;
            clk.update += t1 - t0;
            clk.unite += t2 - t1;
            clk.commit += clock64() - t2;
            ++npass;
            tot_probe += mid;
            if (span && stopped) ++tot_early;
            bm_n = mid;
            if (!span) nb = mid;
            if (stage == 0) {
                if (span) {
                    lo = 1; hi = n_top; nb = 0; hi_known = true; ++tot_fb;
                }
                stage = 2;
            } else if (lo == hi) {
                if (span) {
                    hi_known = true;
                } else {
                    lo = 1; hi = n_top; nb = 0; hi_known = true; ++tot_fb;
                }
            } else if (span) {
                hi = mid;
                hi_known = true;
            } else {
                lo = mid + 1u;
            }
        }
        if (!alive) break;
        if (bracket && blo >= 1u && blo <= bhi && bhi <= N && lo >= blo && lo <= bhi && npass > 0) ++tot_ok;
        if (threadIdx.x == 0) {
            if (leader) {
                nstar_out[s] = (lo == N + 1u) ? PERC_NEVER : lo;
                if (passes_out) passes_out[s] = npass;
                tot_passes += npass;
            }
            if (stats) {
                atomicAdd(&stats->hooks, c.hooks);
                if (leader) atomicAdd(&stats->new_sites, c.new_sites);
                atomicAdd(&stats->sites_merged, c.sites);
                atomicAdd(&stats->unions, c.unions);
                atomicAdd(&stats->cyc_scan, c.cyc_scan);
                atomicAdd(&stats->cyc_link, c.cyc_link);
            }
        }
    }
    if (threadIdx.x == 0 && stats) {
        if (leader) {
            atomicAdd(&stats->passes, tot_passes);
            atomicAdd(&stats->probe_sites, tot_probe);
            atomicAdd(&stats->early_exits, tot_early);
            atomicAdd(&stats->fallbacks, tot_fb);
            atomicAdd(&stats->verified, tot_ok);
        }
        atomicAdd(&stats->cyc_setup, clk.setup);
        atomicAdd(&stats->cyc_update, clk.update);
        atomicAdd(&stats->cyc_union, clk.unite);
        atomicAdd(&stats->cyc_commit, clk.commit);
    }
}

// S_max(n) per sample: one full pass over the first n sites, then cluster sizes by root counting.
__global__ void __launch_bounds__(1024, 1)
k_mass(const perc_sample *__restrict__ samples, uint32_t num, uint32_t max_L, uint32_t smem_L, uint32_t sum_L,
       size_t region, uint32_t node_cap, uint32_t edge_scap,
       const uint64_t *__restrict__ n_in, int64_t *__restrict__ mass_out, char *ws, size_t slot_bytes)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    const SmemPtrs sm = smem_ptrs_sum(dyn, region, node_cap);
    __shared__ Ctl c;
    __shared__ uint32_t red[32];
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const uint64_t Ncap = num_sites(max_L);
    const SlotPtrs sp = slot_ptrs(ws, slot_bytes, Ncap, max_L > smem_L, max_L > sum_L);
    const EdgeList E{sm.edges, edge_scap, sp.gedges};
    const Nodes P{sp.P, static_cast<uint32_t>(__cvta_generic_to_shared(sm.nodes)), node_cap};
    uint32_t *cnt = sp.logb;

    for (;;) {
        if (threadIdx.x == 0) c.sample = atomicAdd(&hdr->queue, 1u);
        __syncthreads();
        const uint32_t s = c.sample;
        if (s >= num) break;
        const perc_sample smp = samples[s];
        const uint32_t L = smp.L, mask = smp.zone_mask & kZoneBits, axis = smp.zone_mask >> kAxisShift;
        const uint64_t n64 = n_in[s];
        if (L < 1u || L > max_L || !valid_zone_word(smp.zone_mask) || !smp.perm || !smp.rank ||
            n64 > num_sites(L)) {
            if (threadIdx.x == 0) {
                mass_out[s] = -1;
                set_status(&hdr->status, PERC_EDEVICE);
            }
            __syncthreads();
            continue;
        }
        const uint32_t N = static_cast<uint32_t>(num_sites(L));
        const uint32_t n = static_cast<uint32_t>(n64);
        const bool smem_bm = L <= smem_L;
        uint32_t *bm, *sum;
        sample_bm_sum(sm, sp, L, smem_L, sum_L, bm, sum);
        sample_tables(c, sm, bm, sum, L, mask, smem_bm);
        if (threadIdx.x == 0) {
            c.logn = 0;
            c.stop = 0;
            c.ecount[0] = 0;
            c.axis = axis;
        }
        const FastDiv fd = make_fastdiv(L);
        __syncthreads();
        if (smem_bm)
            bitmap_update(bm, smp.perm, 0u, n);
        else
            bitmap_add_sum(bm, sum, smp.perm, 0u, n, fd);
        for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) {
            nd_st(P, r + 2u, r + 2u);
            __stcg(cnt + r + 2u, 0u);
        }
        __syncthreads();
        const ScanTabs T{sm.rows, sm.planes, sm.tab, sm.d5m, sum};
        if (smem_bm && L == kPlaneL)
            union_pass<true, false, kScanPlanes, false, true>(c, P, nullptr, sm.sbm, T, E, smp.perm, smp.rank, L, fd, 0u, n, 0u);
        else if (smem_bm)
            union_pass<true, false, kScanRows, false, true>(c, P, nullptr, sm.sbm, T, E, smp.perm, smp.rank, L, fd, 0u, n, 0u);
        else if (L <= sum_L)
            union_pass<false, false, kScanGroups, false, true>(c, P, nullptr, bm, T, E, smp.perm, smp.rank, L, fd, 0u, n, 0u);
        else
            union_pass<false, false, kScanGroupsG, false, true>(c, P, nullptr, bm, T, E, smp.perm, smp.rank, L, fd, 0u, n, 0u);
        __syncthreads();
        for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) atomicAdd(cnt + uf_find(P, r + 2u, 0u), 1u);
        __syncthreads();
        uint32_t best = 0;
        for (uint32_t r = threadIdx.x; r < n; r += blockDim.x) best = max(best, ld_cg(cnt + r + 2u));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t b = 0;
            for (uint32_t w = 0; w < (blockDim.x >> 5); ++w) b = max(b, red[w]);
            mass_out[s] = static_cast<int64_t>(b);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------
// S_max(n) for every n of a window [n_lo, n_lo + W) (eq. Pmax; Methods, "Computational methods":
// the Newman--Ziff sweep adds one site at a time and reads the largest cluster after each), and the
// same sweep for n* (k_nstar_sweep, below).
//
// Per sample, one connected-component pass over the first n0 sites gives the forest (and, for
// S_max, every cluster's size by counting).  The next sites then follow in chunks of up to blockDim:
//   scan       -- each chunk site's occupied neighbors (bitmap through the chunk) as edges;
//   filter     -- an edge is kept when its neighbor came earlier (an edge belongs to its later site)
//                 and counted per site; a prefix sum places each site's records.  A chunk whose
//                 records would pass kRecCap is cut after the last site that fits;
//   resolve    -- a neighbor from before the chunk becomes the root of its cluster; every distinct
//                 root gets a local slot (shared-memory hash);
//   components -- the records join sites and slots into local components (shared-memory
//                 union-find); each component's total (size, or border flags) is summed and the
//                 chunk is written back to the forest at once;
//   replay     -- only a component that can change the result (S_max: its final size passes the
//                 running maximum; n*: it touches both borders) is replayed by one thread in rank
//                 order, union by size on the local slots, which gives the size (or flags) of the
//                 new site's cluster right after each of its sites.
// ------------------------------------------------------------------------------------------------
constexpr uint32_t kRecCap = 1536;    // kept edges of a window chunk (> 892: one site always fits)
constexpr uint32_t kRootHash = 2048;  // local slots of the distinct earlier roots one chunk touches
constexpr uint32_t kEmptySlot = 0xFFFFFFFFu;
constexpr uint32_t kRootBit = 0x80000000u;  // local union-find entry of a root: kRootBit | size
static_assert(kRecCap > kMaxOffsets && kRecCap < kRootHash && (kRootHash & (kRootHash - 1)) == 0,
              "record and hash capacities");

constexpr uint32_t kRecSlot = 0xFFFFu;  // a record is (chunk site << 16) | local slot
constexpr uint32_t kFlagLo = 1u, kFlagHi = 2u;  // a cluster touches x1 = 0 / x1 = L-1

// The window arrays, at fixed offsets from one base (computed where they are used, so that a kernel
// keeps one pointer live instead of twelve).
struct WinPtrs {
    uint32_t *u;  // start of the window arrays
    uint32_t C;   // chunk capacity (blockDim.x)
    __device__ __forceinline__ uint32_t *deg() const { return u; }           // [C] kept edges per chunk site
    __device__ __forceinline__ uint32_t *ev() const { return u + C; }        // [C] cluster size (or flags) per site
    __device__ __forceinline__ uint32_t *lp() const { return u + 2 * C; }    // [C + kRootHash] local union-find in time order: parent slot, or kRootBit | entry
    __device__ __forceinline__ uint32_t *hkey() const { return u + 3 * C + kRootHash; }  // [kRootHash] forest node of local slot C + h (kEmptySlot: free)
    __device__ __forceinline__ uint32_t *rec() const { return u + 3 * C + 2 * kRootHash; }  // [kRecCap] kept edges in site order: (chunk site << 16) | local slot
    __device__ __forceinline__ uint32_t *off() const { return u + 3 * C + 2 * kRootHash + kRecCap; }  // [C + 1] first record of each chunk site
    __device__ __forceinline__ uint32_t *cc() const { return u + 4 * C + 1 + 2 * kRootHash + kRecCap; }  // [C + kRootHash] components of the chunk's records
    __device__ __forceinline__ uint32_t *memb() const { return u + 5 * C + 1 + 3 * kRootHash + kRecCap; }  // [C] component of each chunk site
    __device__ __forceinline__ uint32_t *fl() const { return u + 6 * C + 1 + 3 * kRootHash + kRecCap; }  // [C] border flags of each chunk site (n* sweep)
    __device__ __forceinline__ uint32_t *gm() const { return u + 7 * C + 1 + 3 * kRootHash + kRecCap; }  // [C] smallest forest node of each component, then the replay list
    __device__ __forceinline__ uint32_t *cur() const { return u + 8 * C + 1 + 3 * kRootHash + kRecCap; }  // [C] placement cursor of each chunk site's records
    __device__ __forceinline__ uint32_t *tot() const { return u + 9 * C + 1 + 3 * kRootHash + kRecCap; }  // [C] per-component totals: border flags or cluster size
};

__host__ __device__ inline size_t smem_window_bytes(uint32_t threads)
{
    return ((size_t(threads) * 10 + 1 + kRecCap + 3 * kRootHash) * 4 + 15) & ~size_t(15);
}

__device__ __forceinline__ WinPtrs win_ptrs(unsigned char *at, uint32_t C)
{
    return WinPtrs{reinterpret_cast<uint32_t *>(at), C};
}

// The first pass of a sample keeps the nodes below PA.cap (its own nodes plus the window arrays'
// shared memory, which it does not use) on chip; afterwards the nodes in [P.cap, PA.cap) below
// n_nodes move to the global slot, where P finds them.  All threads; ends with a block barrier.
__device__ __forceinline__ void lend_back(const Nodes &P, const Nodes &PA, uint32_t n_nodes)
{
    const uint32_t hi = min(PA.cap, n_nodes);
    for (uint32_t x = P.cap + threadIdx.x; x < hi; x += blockDim.x) __stcg(P.g + x, lds_u32(PA.sbase + 4u * x));
    __syncthreads();
}

// Exclusive prefix sum of v over the block's threads (blockDim a multiple of 32); `total` gets the
// block's sum.  Uses wsum[32] and two block barriers.
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t v, uint32_t *wsum, uint32_t &total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    if (lane == 31u) wsum[warp] = x;
    __syncthreads();
    if (warp == 0u) {
        uint32_t t = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= static_cast<uint32_t>(o)) t += y;
        }
        if (lane < nw) wsum[lane] = t;
    }
    __syncthreads();
    total = wsum[nw - 1u];
    return (warp ? wsum[warp - 1u] : 0u) + x - v;
}

// Inclusive running maximum of v over the block's threads; uses wsum[32] and two block barriers.
__device__ __forceinline__ uint32_t block_inclusive_max(uint32_t v, uint32_t *wsum)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x = max(x, y);
    }
    if (lane == 31u) wsum[warp] = x;
    __syncthreads();
    if (warp == 0u) {
        uint32_t t = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= static_cast<uint32_t>(o)) t = max(t, y);
        }
        if (lane < nw) wsum[lane] = t;
    }
    __syncthreads();
    return warp ? max(wsum[warp - 1u], x) : x;
}


// Components of the chunk's records: lock-free union-find on shared memory, the larger root hooked
// under the smaller, so a component's root is its smallest slot (a chunk site, since earlier roots
// have slots above C).
__device__ __forceinline__ uint32_t cc_find(uint32_t *cc, uint32_t x)
{
    volatile uint32_t *v = cc;
    for (;;) {
        const uint32_t p = v[x];
        if (p == x) return x;
        const uint32_t g = v[p];
        if (g != p) v[x] = g;  // path halving: g is an ancestor of x
        x = g;
    }
}

__device__ __forceinline__ void cc_unite(uint32_t *cc, uint32_t a, uint32_t b)
{
    for (;;) {
        a = cc_find(cc, a);
        b = cc_find(cc, b);
        if (a == b) return;
        if (a > b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(cc + b, b, a) == b) return;
    }
}


// Local slot of forest root g: linear probing in the chunk's hash.  The thread that inserts g
// also stores the slot's entry: kRootBit | cluster size (S_max windows), or kRootBit | (1 << 2) |
// border flags of g's cluster (the n* sweep: root 0 is the x1 = 0 border, root 1 the x1 = L-1
// border).  Returns kEmptySlot only if the hash is full, which the capacities rule out (a chunk
// keeps at most kRecCap < kRootHash records).
template <bool kSpan>
__device__ __forceinline__ uint32_t root_slot(const WinPtrs &wp, const uint32_t *cnt, uint32_t g, uint32_t C)
{
    uint32_t h = (g * 2654435761u) >> (32 - 11);
    static_assert(kRootHash == 2048u, "hash width");
    for (uint32_t probe = 0; probe < kRootHash; ++probe) {
        const uint32_t prev = atomicCAS(wp.hkey() + h, kEmptySlot, g);
        if (prev == kEmptySlot) {
            wp.lp()[C + h] = kSpan ? (kRootBit | 4u | (g == 0u ? kFlagLo : g == 1u ? kFlagHi : 0u))
                                 : (kRootBit | __ldcg(cnt + g));
            return C + h;
        }
        if (prev == g) return C + h;
        h = (h + 1u) & (kRootHash - 1u);
    }
    return kEmptySlot;
}

// Scan of the window chunk [b, b + count): edges (local index of the site, occupied neighbor).  With
// one site per thread, `site` is the thread's site (loaded by the caller); with fl, each site's
// border flags go to fl and, for the n* sweep, its local union-find entry to lp.
template <bool kSmemBm, int kMode>
__device__ __forceinline__ void window_scan(const Ctl &c, const uint32_t *bm, const ScanTabs &T, const EdgeList &E,
                                            const uint32_t *perm, uint32_t L, const FastDiv &fd, uint32_t b,
                                            uint32_t count, uint32_t site, uint32_t *ecount, uint32_t *fl,
                                            uint32_t *lp)
{
    constexpr bool kPlanes = kMode == kScanPlanes;
    const uint32_t R = uses_sum(kMode) ? c.G : kPlanes ? c.NP : c.R;
    const uint32_t gshift = lanes_shift(count, R);
    const uint32_t gsize = 1u << gshift, gl = threadIdx.x & (gsize - 1u), t = threadIdx.x >> gshift;
    if (t >= count) return;
    const SiteGeo g = site_geo<kMode>(gshift ? __ldg(perm + b + t) : site, L, fd, c.axis);
    if (fl && gl == 0u) {
        const uint32_t f = c.axis == kAnyAxis ? g.faces : (g.low ? kFlagLo : 0u) | (g.high ? kFlagHi : 0u);
        fl[t] = f;
        lp[t] = kRootBit | 4u | f;
    }
    if constexpr (uses_sum(kMode)) {
        auto emit = [&](uint32_t jb, uint32_t h) {
            uint32_t slot = atomicAdd(ecount, static_cast<uint32_t>(__popc(h)));
            while (h) {
                const uint32_t bit = __ffs(h) - 1;
                h &= h - 1u;
                edge_put(E, slot++, make_uint2(t, jb + bit));
            }
        };
        for (uint32_t k = gl; k < R; k += gsize) sum_entry_hits<kSmemBm, kMode, false>(g, bm, T, L, k, emit);
    } else {
        for (uint32_t k = gl; k < R; k += gsize) {
            uint32_t h[3];
            const uint32_t jb = entry_hits<kSmemBm, kPlanes>(g, bm, T.rows, T.planes, k, h);
            if ((h[0] | h[1] | h[2]) == 0u) continue;
            const uint32_t nh = __popc(h[0]) + __popc(h[1]) + __popc(h[2]);
            uint32_t slot = atomicAdd(ecount, nh);
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                uint32_t hf = h[f];
                while (hf) {
                    const uint32_t bit = __ffs(hf) - 1;
                    hf &= hf - 1u;
                    edge_put(E, slot++, make_uint2(t, jb + 32u * f + bit));
                }
            }
        }
    }
}

struct SmaxShared {
    uint32_t run_max;  // S_max after the last site added
    uint32_t red[32];
};

// The front of a window chunk starting at rank b (all threads): the chunk's per-site arrays reset,
// bitmap through the chunk, scan, the kept records in site order (a chunk cut where they would pass
// kRecCap), earlier neighbors resolved to local slots, and the local components of the records.
// Returns the number of sites taken (>= 1); `comp` gets the component (its smallest site) of the
// thread's site (< tn).  The previous chunk must have ended with a block barrier after its last
// reader of the per-site arrays.
template <bool kSmemBm, int kMode, bool kSpan>
__device__ __forceinline__ uint32_t chunk_front(Ctl &c, SmaxShared &x, const Nodes &P, const uint32_t *cnt,
                                                uint32_t *bm, const ScanTabs &T, const WinPtrs &wp,
                                                const EdgeList &E, const perc_sample &smp, const FastDiv &fd,
                                                uint32_t b, uint32_t n_end, uint32_t &comp)
{
    const uint32_t C = blockDim.x;
    const uint32_t count = min(C, n_end - b);
    const long long t0 = clock64();
    wp.deg()[threadIdx.x] = 0u;
    wp.cur()[threadIdx.x] = 0u;
    wp.tot()[threadIdx.x] = 0u;
    wp.gm()[threadIdx.x] = kEmptySlot;
    wp.ev()[threadIdx.x] = 0u;
    if (!kSpan) wp.lp()[threadIdx.x] = kRootBit | 1u;
    for (uint32_t y = threadIdx.x; y < C + kRootHash; y += C) wp.cc()[y] = y;
    if (threadIdx.x == 0) c.ecount[0] = 0u;
    uint32_t site = 0u;
    if (threadIdx.x < count) {  // the chunk's sites join the bitmap (and the summary)
        site = __ldg(smp.perm + b + threadIdx.x);
        const uint32_t i = site + kBmGuard;
        atomicOr(bm + (i >> 5), 1u << (i & 31u));
        if (uses_sum(kMode)) {
            const uint32_t row = fdiv(site, fd) + kSumGuard;
            atomicOr(T.sum + (row >> 5), 1u << (row & 31u));
        }
    }
    __syncthreads();
    window_scan<kSmemBm, kMode>(c, bm, T, E, smp.perm, smp.L, fd, b, count, site, &c.ecount[0],
                                kSpan ? wp.fl() : nullptr, wp.lp());
    __syncthreads();
    const long long t1 = clock64();
    const uint32_t ne = c.ecount[0];
    // filter: keep the edges to earlier sites, count them per site (rank replaces the site)
    for (uint32_t e = threadIdx.x; e < ne; e += C) {
        const uint2 ed = edge_get(E, e);
        const uint32_t rj = __ldg(smp.rank + ed.y);
        const bool keep = rj < b + ed.x;
        if (keep) atomicAdd(wp.deg() + ed.x, 1u);
        edge_put(E, e, make_uint2(keep ? ed.x : kEmptySlot, rj));
    }
    __syncthreads();
    const uint32_t d = wp.deg()[threadIdx.x];
    uint32_t total;
    const uint32_t excl = block_exclusive_sum(d, x.red, total);
    wp.off()[threadIdx.x] = excl;
    if (threadIdx.x == C - 1u) wp.off()[C] = total;
    const uint32_t tn = __syncthreads_count(threadIdx.x < count && excl + d <= kRecCap);
    // resolve: earlier neighbors to local slots, records in site order
    for (uint32_t e = threadIdx.x; e < ne; e += C) {
        const uint2 ed = edge_get(E, e);
        if (ed.x >= tn) continue;  // dropped, or past the cut
        const uint32_t pos = wp.off()[ed.x] + atomicAdd(wp.cur() + ed.x, 1u);
        const uint32_t slot = ed.y >= b ? ed.y - b : root_slot<kSpan>(wp, cnt, uf_find(P, ed.y + 2u, 0u), C);
        wp.rec()[pos] = (ed.x << 16) | (slot & kRecSlot);
    }
    const uint32_t nrec = wp.off()[tn];
    __syncthreads();
    // the clusters a chunk builds only interact inside a component of its records
    for (uint32_t k = threadIdx.x; k < nrec; k += C) {
        const uint32_t r = wp.rec()[k], s2 = r & kRecSlot;
        if (s2 < C + kRootHash) cc_unite(wp.cc(), r >> 16, s2);
    }
    __syncthreads();
    comp = threadIdx.x < tn ? cc_find(wp.cc(), threadIdx.x) : 0u;
    if (threadIdx.x == 0) {
        c.cyc_scan += static_cast<unsigned long long>(t1 - t0);
        c.cyc_link += static_cast<unsigned long long>(clock64() - t1);
    }
    return tn;
}

__device__ __forceinline__ uint32_t smem_addr(const uint32_t *q)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(q));
}

// After chunk_front (all threads): each component's total -- border flags (n* sweep) or cluster
// size (S_max windows) -- and its smallest forest node, then (after one block barrier) the chunk
// written back to the forest, every component under one node: for the sweep along one axis node 0
// if the component touches x1 = 0, node 1 if it touches x1 = L-1, else its smallest node (so a
// cluster touching a border keeps that border's node as its root); for S_max windows its smallest
// node, which takes the component's size in cnt; for the sweep along any axis (cnt = the forest's
// face words, read here for the earlier clusters) its smallest node, whose face word store_faces
// writes later.  The caller's next block barrier orders the write-back.
template <bool kSpan>
__device__ __forceinline__ void chunk_components(const Nodes &P, uint32_t *cnt, const WinPtrs &wp, uint32_t b,
                                                 uint32_t tn, uint32_t comp)
{
    const uint32_t C = blockDim.x;
    if (threadIdx.x < tn) {
        wp.memb()[threadIdx.x] = comp;
        if (kSpan)
            atomicOr(wp.tot() + comp, wp.fl()[threadIdx.x]);
        else
            atomicAdd(wp.tot() + comp, 1u);
        atomicMin(wp.gm() + comp, b + threadIdx.x + 2u);
    }
    for (uint32_t h = threadIdx.x; h < kRootHash; h += C) {
        const uint32_t g = wp.hkey()[h];
        if (g == kEmptySlot) continue;
        const uint32_t ch = cc_find(wp.cc(), C + h);
        if (kSpan)  // the earlier cluster's border flags: its root's face word, or the border root it is
            atomicOr(wp.tot() + ch, cnt ? __ldcg(cnt + g) : g == 0u ? kFlagLo : g == 1u ? kFlagHi : 0u);
        else
            atomicAdd(wp.tot() + ch, wp.lp()[C + h] & ~kRootBit);
        atomicMin(wp.gm() + ch, g);
    }
    __syncthreads();
    auto root_of = [&](uint32_t cp) {
        if (kSpan && !cnt) {
            const uint32_t f = wp.tot()[cp];
            if (f & kFlagLo) return 0u;
            if (f & kFlagHi) return 1u;
        }
        return wp.gm()[cp];
    };
    if (threadIdx.x < tn) {
        const uint32_t node = b + threadIdx.x + 2u, r = root_of(comp);
        nd_st(P, node, r);
        if (!kSpan && r == node) __stcg(cnt + node, wp.tot()[comp]);
    }
    for (uint32_t h = threadIdx.x; h < kRootHash; h += C) {
        const uint32_t g = wp.hkey()[h];
        if (g == kEmptySlot) continue;
        const uint32_t ch = cc_find(wp.cc(), C + h), r = root_of(ch);
        if (r != g)
            nd_st(P, g, r);
        else if (!kSpan)
            __stcg(cnt + g, wp.tot()[ch]);
    }
}

// Sweep along any axis, after a chunk that does not span: each component's face word goes to its
// root (its smallest forest node).  Kept out of chunk_components because the first-spanning-site
// search of a spanning chunk reads the earlier clusters' face words as they were before the chunk.
__device__ __forceinline__ void store_faces(uint32_t *gflags, const WinPtrs &wp, uint32_t b, uint32_t tn,
                                            uint32_t comp)
{
    const uint32_t C = blockDim.x;
    if (threadIdx.x < tn && wp.gm()[comp] == b + threadIdx.x + 2u) __stcg(gflags + wp.gm()[comp], wp.tot()[comp]);
    for (uint32_t h = threadIdx.x; h < kRootHash; h += C) {
        const uint32_t g = wp.hkey()[h];
        if (g == kEmptySlot) continue;
        const uint32_t ch = cc_find(wp.cc(), C + h);
        if (wp.gm()[ch] == g) __stcg(gflags + g, wp.tot()[ch]);
    }
}

// The sites of the components to replay (need = this thread's site belongs to one), in rank order,
// compacted into wp.gm() (free after the write-back); returns their number.  All threads; contains
// block barriers.
__device__ __forceinline__ uint32_t replay_list(SmaxShared &x, const WinPtrs &wp, bool need)
{
    uint32_t tot;
    const uint32_t at = block_exclusive_sum(need ? 1u : 0u, x.red, tot);
    if (need) wp.gm()[at] = threadIdx.x;
    __syncthreads();
    return tot;
}

// Replay of the component rooted at chunk site t0 (one thread): its sites in rank order (found in
// the replay list), each merged with the clusters its records name (union by size on the local
// slots; entries kRootBit | size); ev[t] = the cluster size right after site t.
__device__ __forceinline__ void replay_component(const WinPtrs &wp, uint32_t t0, uint32_t nlist, uint32_t C,
                                                 int *status)
{
    const uint32_t s_lp = smem_addr(wp.lp());
    for (uint32_t i = 0; i < nlist; ++i) {
        const uint32_t t = wp.gm()[i];
        if (wp.memb()[t] != t0) continue;
        const uint32_t k0 = wp.off()[t], k1 = wp.off()[t + 1u];
        uint32_t ra = t, sa = lds_u32(s_lp + 4u * t) & ~kRootBit;  // no earlier record names site t: a root
        for (uint32_t k = k0; k < k1; ++k) {
            const uint32_t bs = wp.rec()[k] & kRecSlot;
            if (bs >= C + kRootHash) {  // full hash (ruled out by the capacities)
                set_status(status, PERC_EDEVICE);
                continue;
            }
            // root xr of bs (path halving) and its entry v
            uint32_t xr = bs, v = lds_u32(s_lp + 4u * bs);
            while (!(v & kRootBit)) {
                const uint32_t g = lds_u32(s_lp + 4u * v);
                if (g & kRootBit) {
                    xr = v;
                    v = g;
                    break;
                }
                sts_u32(s_lp + 4u * xr, g);
                xr = g;
                v = lds_u32(s_lp + 4u * g);
            }
            if (xr == ra) continue;
            const uint32_t sb = v & ~kRootBit;
            if (sa >= sb) {
                sts_u32(s_lp + 4u * xr, ra);
            } else {
                sts_u32(s_lp + 4u * ra, xr);
                ra = xr;
            }
            sa += sb;
            sts_u32(s_lp + 4u * ra, kRootBit | sa);
        }
        wp.ev()[t] = sa;
    }
}

// One sample of k_smax (all threads).  Writes row[k] = S_max(n_lo + k) for n_lo + k <= n_end.
template <bool kSmemBm, int kMode>
__device__ __forceinline__ void smax_sample(Ctl &c, SmaxShared &x, const Nodes &P, const Nodes &PA, uint32_t *cnt, uint32_t *bm,
                            const SmemPtrs &sm, const ScanTabs &T, const WinPtrs &wp, const EdgeList &E,
                            const perc_sample &smp, uint32_t n0, uint32_t n_end, uint64_t nlo, uint32_t window,
                            uint32_t *row, int *status)
{
    const uint32_t C = blockDim.x, L = smp.L;
    if (kSmemBm) bm = sm.sbm;
    const FastDiv fd = make_fastdiv(L);
    // ---- the forest of the first n0 sites (nodes PA), the cluster sizes and S_max(n0)
    if constexpr (uses_sum(kMode))
        bitmap_add_sum(bm, T.sum, smp.perm, 0u, n0, fd);
    else
        bitmap_update(bm, smp.perm, 0u, n0);
    for (uint32_t r = threadIdx.x; r < n0; r += C) {
        nd_st(PA, r + 2u, r + 2u);
        __stcg(cnt + r + 2u, 0u);
    }
    __syncthreads();
    if (n0 > 0u)
        union_pass<kSmemBm, false, kMode, false, true>(c, PA, nullptr, bm, T, E, smp.perm, smp.rank, L, fd, 0u, n0,
                                                       0u);
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < n0; r += C) atomicAdd(cnt + uf_find(PA, r + 2u, 0u), 1u);
    __syncthreads();
    uint32_t best = 0;
    for (uint32_t r = threadIdx.x; r < n0; r += C) best = max(best, ld_cg(cnt + r + 2u));
    best = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31u) == 0u) x.red[threadIdx.x >> 5] = best;
    lend_back(P, PA, n0 + 2u);
    for (uint32_t h = threadIdx.x; h < kRootHash; h += C) wp.hkey()[h] = kEmptySlot;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t bmax = 0;
        for (uint32_t w = 0; w < (C >> 5); ++w) bmax = max(bmax, x.red[w]);
        x.run_max = bmax;
        row[0] = bmax;  // n = n_lo = n0
    }
    // ---- the window's sites, a chunk at a time
    for (uint32_t b = n0; b < n_end;) {
        uint32_t comp;
        const uint32_t tn = chunk_front<kSmemBm, kMode, false>(c, x, P, cnt, bm, T, wp, E, smp, fd, b, n_end, comp);
        const uint32_t run0 = x.run_max;
        chunk_components<false>(P, cnt, wp, b, tn, comp);
        // a component can raise S_max only if its final size passes the running maximum: replay those
        const bool need = threadIdx.x < tn && wp.tot()[comp] > run0;
        if (__syncthreads_or(need)) {
            const uint32_t nlist = replay_list(x, wp, need);
            if (need && comp == threadIdx.x) replay_component(wp, threadIdx.x, nlist, C, status);
            __syncthreads();
        }
        const uint32_t v = threadIdx.x < tn ? wp.ev()[threadIdx.x] : 0u;
        const uint32_t run = max(block_inclusive_max(v, x.red), run0);
        if (threadIdx.x < tn) {
            const uint64_t k = uint64_t(b) + threadIdx.x + 1u - nlo;
            if (k < window) row[k] = run;
        }
        if (threadIdx.x == tn - 1u) x.run_max = run;
        for (uint32_t h = threadIdx.x; h < kRootHash; h += C) wp.hkey()[h] = kEmptySlot;
        b += tn;
        __syncthreads();  // the per-site arrays, the hash and run_max are read again by the next chunk
    }
}

// Union-find of the first-spanning-site search: entries that a probe hooks carry kProbeTag until the
// probe is committed, and path halving never shortcuts a tagged edge, so that undoing a probe (its
// hooked roots reset) leaves a valid committed forest.
constexpr uint32_t kProbeTag = 0x80000000u;

__device__ __forceinline__ uint32_t pcc_find(uint32_t *cc, uint32_t x)
{
    volatile uint32_t *v = cc;
    for (;;) {
        const uint32_t p = v[x], pu = p & ~kProbeTag;
        if (pu == x) return x;
        const uint32_t g = v[pu], gu = g & ~kProbeTag;
        if (gu == pu) return pu;
        if (((p | g) & kProbeTag) == 0u) v[x] = gu;  // both edges committed
        x = gu;
    }
}

__device__ __forceinline__ void pcc_unite(uint32_t *cc, uint32_t a, uint32_t b, uint32_t *log, uint32_t *logn)
{
    for (;;) {
        a = pcc_find(cc, a);
        b = pcc_find(cc, b);
        if (a == b) return;
        if (a > b) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(cc + b, b, a | kProbeTag) == b) {
            log[atomicAdd(logn, 1u)] = b;
            return;
        }
    }
}

// The first site of a spanning chunk whose cluster carries both border flags (all threads; the chunk
// spans once all its tn sites are added).  Bisection over m, the number of the chunk's sites added:
// the records of sites < m (stored in site order, the first off[m] of them) unite sites and earlier
// clusters' slots into local components (shared-memory union-find, smallest slot as root, so every
// component of a site has a site as root), each root ORs the border flags of its sites and of the
// earlier clusters it reaches (forest root 0: x1 = 0, root 1: x1 = L-1), and m spans when a root
// carries both.  span(0) is false (the earlier clusters do not span) and span(tn) true; the answer
// is the largest m that does not span.  The union-find of the largest non-spanning m found so far
// is kept: a probe only adds the records of the sites between it and the probe, and a probe that
// spans is undone from its log of hooked roots (in lp, which the sweep does not use), so the
// records are united about twice in all instead of once per round.  sh: four words of shared
// scratch.  With gflags (spanning along any axis) the flags are face words, the earlier clusters'
// flags come from the forest's face words, and m spans when a root holds both faces of an axis.
__device__ uint32_t first_span_site(const WinPtrs &wp, uint32_t tn, uint32_t *sh, const uint32_t *gflags)
{
    const uint32_t C = blockDim.x;
    uint32_t *cc = wp.cc(), *ev = wp.ev(), *log = wp.lp();
    for (uint32_t y = threadIdx.x; y < C + kRootHash; y += C) cc[y] = y;
    if (threadIdx.x < 4) sh[threadIdx.x] = threadIdx.x < 2 ? 0u : kEmptySlot;
    __syncthreads();
    for (uint32_t h = threadIdx.x; h < kRootHash; h += C) {
        const uint32_t g = wp.hkey()[h];
        if (gflags)  // any axis: the slot keeps its cluster's face word from here on (0: none)
            wp.hkey()[h] = g == kEmptySlot ? 0u : __ldcg(gflags + g);
        else if (g <= 1u)  // one axis: the local slots of the border roots
            sh[2 + g] = C + h;
    }
    if (gflags) __syncthreads();
    uint32_t lo = 0, hi = tn, round = 0;
    while (hi - lo > 1u) {
        const uint32_t m = (lo + hi) >> 1;
        uint32_t *logn = sh + (round & 1u);
        ev[threadIdx.x] = 0u;
        const uint32_t r1 = wp.off()[m];
        for (uint32_t k = wp.off()[lo] + threadIdx.x; k < r1; k += C) {
            const uint32_t r = wp.rec()[k], s2 = r & kRecSlot;
            if (s2 < C + kRootHash) pcc_unite(cc, r >> 16, s2, log, logn);
        }
        __syncthreads();
        if (threadIdx.x < m) atomicOr(ev + pcc_find(cc, threadIdx.x), wp.fl()[threadIdx.x]);
        if (gflags) {  // earlier clusters that touch faces, reached by a site below m
            for (uint32_t h = threadIdx.x; h < kRootHash; h += C) {
                const uint32_t f = wp.hkey()[h];
                if (!f) continue;
                const uint32_t rt = pcc_find(cc, C + h);
                if (rt < C) atomicOr(ev + rt, f);
            }
        } else if (threadIdx.x < 2u && sh[2 + threadIdx.x] != kEmptySlot) {
            const uint32_t rt = pcc_find(cc, sh[2 + threadIdx.x]);
            if (rt < C) atomicOr(ev + rt, threadIdx.x == 0u ? kFlagLo : kFlagHi);  // reached by a site below m
        }
        __syncthreads();
        const uint32_t fe = threadIdx.x < m ? ev[threadIdx.x] : 0u;
        const bool span = __syncthreads_or(gflags ? spans_any(fe) : fe == (kFlagLo | kFlagHi));
        const uint32_t nlog = *logn;
        for (uint32_t k = threadIdx.x; k < nlog; k += C) {
            const uint32_t b = log[k];
            cc[b] = span ? b : (cc[b] & ~kProbeTag);  // undo the probe, or commit its hooks
        }
        if (threadIdx.x == 0) sh[(round & 1u) ^ 1u] = 0u;  // the next round's log count
        __syncthreads();
        if (span)
            hi = m;
        else
            lo = m;
        ++round;
    }
    return hi - 1u;
}

// The n* sweep of one sample from n_s (all threads; the sites of rank < n_s are merged and do not
// span).  Returns n*, or PERC_NEVER if no n <= N spans; `chunks` counts the chunks taken.  Only a
// chunk whose components touch both borders at its end is searched for the first spanning site.
template <bool kSmemBm, int kMode>
__device__ __forceinline__ uint32_t span_sweep(Ctl &c, SmaxShared &x, const Nodes &P, uint32_t *bm, const SmemPtrs &sm,
                               const ScanTabs &T, const WinPtrs &wp, const EdgeList &E, const perc_sample &smp,
                               const FastDiv &fd, uint32_t N, uint32_t n_s, uint32_t &chunks,
                               unsigned long long &cyc_back, unsigned long long &cyc_span, int *status,
                               uint32_t *gflags)
{
    const uint32_t C = blockDim.x;
    if (kSmemBm) bm = sm.sbm;
    for (uint32_t h = threadIdx.x; h < kRootHash; h += C) wp.hkey()[h] = kEmptySlot;
    for (uint32_t b = n_s; b < N;) {
        ++chunks;
        uint32_t comp;
        const uint32_t tn = chunk_front<kSmemBm, kMode, true>(c, x, P, gflags, bm, T, wp, E, smp, fd, b, N, comp);
        const long long t0 = clock64();
        chunk_components<true>(P, gflags, wp, b, tn, comp);
        // only a component that spans at the end of the chunk can hold the first spanning site
        const uint32_t f = threadIdx.x < tn ? wp.tot()[comp] : 0u;
        const bool spans = gflags ? spans_any(f) : f == (kFlagLo | kFlagHi);
        uint32_t st = kEmptySlot;
        if (__syncthreads_or(spans)) {
            const long long t1 = clock64();
            st = first_span_site(wp, tn, x.red, gflags);
            if (threadIdx.x == 0) cyc_span += static_cast<unsigned long long>(clock64() - t1);
        } else if (gflags) {
            store_faces(gflags, wp, b, tn, comp);
        }
        if (threadIdx.x == 0) cyc_back += static_cast<unsigned long long>(clock64() - t0);
        for (uint32_t h = threadIdx.x; h < kRootHash; h += C) wp.hkey()[h] = kEmptySlot;
        if (st != kEmptySlot) return b + st + 1u;
        b += tn;
        __syncthreads();  // the per-site arrays and the hash are reset by the next chunk
    }
    return PERC_NEVER;
}

__global__ void __launch_bounds__(1024, 1)
k_smax(const perc_sample *__restrict__ samples, uint32_t num, uint32_t max_L, uint32_t smem_L, uint32_t sum_L,
       size_t region, uint32_t node_cap, uint32_t edge_scap, const uint64_t *__restrict__ n_lo,
       const uint32_t *__restrict__ count, uint32_t window, uint32_t *__restrict__ out, char *ws, size_t slot_bytes)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    const uint32_t C = blockDim.x;
    const SmemPtrs sm = smem_ptrs_sum(dyn, region, node_cap, smem_window_bytes(C));
    const WinPtrs wp = win_ptrs(reinterpret_cast<unsigned char *>(sm.nodes) + smem_nodes_bytes(node_cap), C);
    __shared__ Ctl c;
    __shared__ SmaxShared x;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const uint64_t Ncap = num_sites(max_L);
    const SlotPtrs sp = slot_ptrs(ws, slot_bytes, Ncap, max_L > smem_L, max_L > sum_L);
    const EdgeList E{sm.edges, edge_scap, sp.gedges};
    const Nodes P{sp.P, static_cast<uint32_t>(__cvta_generic_to_shared(sm.nodes)), node_cap};
    const Nodes PA{sp.P, P.sbase, node_cap + static_cast<uint32_t>(smem_window_bytes(C) / 4)};  // first pass

    for (;;) {
        if (threadIdx.x == 0) c.sample = atomicAdd(&hdr->queue, 1u);
        __syncthreads();
        const uint32_t s = c.sample;
        if (s >= num) break;
        const perc_sample smp = samples[s];
        const uint32_t L = smp.L, mask = smp.zone_mask & kZoneBits, axis = smp.zone_mask >> kAxisShift;
        uint32_t *row = out + size_t(s) * window;
        if (L < 1u || L > max_L || !valid_zone_word(smp.zone_mask) || !smp.perm || !smp.rank) {
            for (uint32_t k = threadIdx.x; k < window; k += C) row[k] = kEmptySlot;
            if (threadIdx.x == 0) set_status(&hdr->status, PERC_EDEVICE);
            __syncthreads();
            continue;
        }
        const uint32_t N = static_cast<uint32_t>(num_sites(L));
        const uint64_t nlo = n_lo[s];
        const uint32_t len = count ? min(count[s], window) : window;  // entries this sample computes
        for (uint32_t k = threadIdx.x; k < window; k += C)
            if (k >= len || nlo + k > N) row[k] = 0u;  // not asked for, or no such n
        if (nlo > N || len == 0u) {
            __syncthreads();
            continue;
        }
        const uint64_t last = nlo + len - 1u;  // the last n computed
        const uint32_t n0 = static_cast<uint32_t>(nlo), n_end = last < N ? static_cast<uint32_t>(last) : N;
        const bool smem_bm = L <= smem_L;
        uint32_t *bm, *sum;
        sample_bm_sum(sm, sp, L, smem_L, sum_L, bm, sum);
        sample_tables(c, sm, bm, sum, L, mask, smem_bm);
        if (threadIdx.x == 0) {
            c.logn = 0;
            c.stop = 0;
            c.ecount[0] = 0;
            c.axis = axis;  // S_max does not use borders; kept defined for the shared scan
        }
        __syncthreads();
        const ScanTabs T{sm.rows, sm.planes, sm.tab, sm.d5m, sum};
        if (smem_bm && L == kPlaneL)
            smax_sample<true, kScanPlanes>(c, x, P, PA, sp.logb, bm, sm, T, wp, E, smp, n0, n_end, nlo, window, row,
                                           &hdr->status);
        else if (smem_bm)
            smax_sample<true, kScanRows>(c, x, P, PA, sp.logb, bm, sm, T, wp, E, smp, n0, n_end, nlo, window, row,
                                         &hdr->status);
        else if (L <= sum_L)
            smax_sample<false, kScanGroups>(c, x, P, PA, sp.logb, bm, sm, T, wp, E, smp, n0, n_end, nlo, window, row,
                                            &hdr->status);
        else
            smax_sample<false, kScanGroupsG>(c, x, P, PA, sp.logb, bm, sm, T, wp, E, smp, n0, n_end, nlo, window, row,
                                             &hdr->status);
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------------
// k_nstar_sweep: n* by one sweep over the sites in rank order (the Newman--Ziff order), in chunks,
// instead of bisection.  A start n_s that does not span -- the learned bracket's lower end minus
// one, checked by one connected-component pass, else 0 -- is reached in one pass; the window
// chunks then follow with border flags in place of sizes, and only a component that touches both
// borders at the end of its chunk is replayed: its first site whose cluster carries both flags
// gives n*.  Between chunks the forest keeps the invariant of the passes: a cluster touching
// x1 = 0 has root node 0, one touching x1 = L-1 (and not x1 = 0) has root node 1.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024, 1)
k_nstar_sweep(const perc_sample *__restrict__ samples, uint32_t num, uint32_t max_L, uint32_t smem_L,
              uint32_t sum_L, size_t region, uint32_t node_cap, uint32_t edge_scap,
              const uint32_t *__restrict__ bracket, uint32_t *__restrict__ nstar_out,
              uint32_t *__restrict__ passes_out, perc_stats *stats, char *ws, size_t slot_bytes, uint32_t any,
              const uint32_t *__restrict__ share, uint32_t *__restrict__ unresolved)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    const uint32_t C = blockDim.x;
    const SmemPtrs sm = smem_ptrs_sum(dyn, region, node_cap, smem_window_bytes(C));
    const WinPtrs wp = win_ptrs(reinterpret_cast<unsigned char *>(sm.nodes) + smem_nodes_bytes(node_cap), C);
    __shared__ Ctl c;
    __shared__ SmaxShared x;
    WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
    const uint64_t Ncap = num_sites(max_L);
    // spanning along any axis: the slot's second node-sized array holds each root's face word
    const SlotPtrs sp = slot_ptrs(ws, slot_bytes, Ncap, max_L > smem_L, max_L > sum_L, any != 0u);
    uint32_t *const gflags = any ? sp.logb : nullptr;
    const EdgeList E{sm.edges, edge_scap, sp.gedges};
    const Nodes P{sp.P, static_cast<uint32_t>(__cvta_generic_to_shared(sm.nodes)), node_cap};
    const Nodes PA{sp.P, P.sbase, node_cap + static_cast<uint32_t>(smem_window_bytes(C) / 4)};  // first pass
    // per-CTA counters, kept in shared memory (thread 0 updates them) rather than in registers
    __shared__ unsigned long long tot_passes, tot_probe, tot_fb, tot_ok, tot_chunks;
    __shared__ unsigned long long cyc_setup, cyc_first, cyc_back, cyc_span;
    if (threadIdx.x == 0) tot_passes = tot_probe = tot_fb = tot_ok = tot_chunks = cyc_setup = cyc_first = cyc_back = cyc_span = 0;

    for (;;) {
        if (threadIdx.x == 0) {
            c.sample = atomicAdd(&hdr->queue, 1u);
            c.hooks = 0;
            c.new_sites = 0;
            c.sites = 0;
            c.unions = 0;
            c.cyc_scan = 0;
            c.cyc_link = 0;
        }
        __syncthreads();
        const long long t_setup = clock64();
        const uint32_t s = c.sample;
        if (s >= num) break;
        const perc_sample smp = samples[s];
        const uint32_t L = smp.L, mask = smp.zone_mask & kZoneBits, axis = smp.zone_mask >> kAxisShift;
        if (L < 1u || L > max_L || !valid_zone_word(smp.zone_mask) || !smp.perm || !smp.rank) {
            if (threadIdx.x == 0) {
                nstar_out[s] = PERC_NEVER;
                if (passes_out) passes_out[s] = 0;
                set_status(&hdr->status, PERC_EDEVICE);
            }
            __syncthreads();
            continue;
        }
        const uint32_t N = static_cast<uint32_t>(num_sites(L));
        // orders ranked only in part (perc_nstar_prefix): no site of rank >= lim is read; the share
        // is one word for the launch, or (share null, unresolved set) the sample's own bracket's
        uint32_t lim = N;
        if (share)
            lim = prefix_sites(N, *share);
        else if (unresolved && bracket)
            lim = prefix_sites(N, bracket_share(L, bracket[2 * size_t(s)], bracket[2 * size_t(s) + 1]));
        const bool smem_bm = L <= smem_L;
        uint32_t *bm, *sum;
        sample_bm_sum(sm, sp, L, smem_L, sum_L, bm, sum);
        sample_tables(c, sm, bm, sum, L, mask, smem_bm);
        // scan tables of the on-chip bitmap paths and of the summary paths
        const ScanTabs Tb{sm.rows, sm.planes, nullptr, nullptr, nullptr};
        const ScanTabs Ts{nullptr, nullptr, sm.tab, sm.d5m, sum};
        if (threadIdx.x == 0) {
            nd_st(PA, 0u, 0u);  // for the first pass
            nd_st(PA, 1u, 1u);
            nd_st(P, 0u, 0u);  // for the sweep (the same words when node_cap > 1)
            nd_st(P, 1u, 1u);
            c.axis = gflags ? kAnyAxis : axis;
            c.stop = 0;
            c.logn = 0;
            c.ecount[0] = 0;
        }
        const FastDiv fd = make_fastdiv(L);
        __syncthreads();
        const long long t_first = clock64();
        if (threadIdx.x == 0) cyc_setup += static_cast<unsigned long long>(t_first - t_setup);

        // the start: the bracket's lower end minus one, which must not span
        uint32_t n_s = 0, blo = 0, bhi = 0, npass = 0;
        bool have_br = false;
        if (bracket) {
            blo = bracket[2 * size_t(s)];
            bhi = bracket[2 * size_t(s) + 1];
            if (blo >= 1u && blo <= bhi && bhi <= N && blo <= lim) {
                n_s = blo - 1u;
                have_br = true;
            } else if (threadIdx.x == 0) {
                ++tot_fb;
            }
        }
        // A start that spans (n* below the bracket's lower end) retreats to three quarters of
        // itself, up to three times, then to 0: the half-neighborhood pass needs the bitmap to hold
        // exactly the sites below its end, so the bits of the sites given up are cleared (the
        // occupancy summary only ever over-reports, which costs a wasted row read, no error)
        if (n_s > 0u) {
            if (smem_bm)
                bitmap_update(bm, smp.perm, 0u, n_s);
            else
                bitmap_add_sum(bm, sum, smp.perm, 0u, n_s, fd);
        }
        for (uint32_t tries = 0; n_s > 0u; ++tries) {
            for (uint32_t r = threadIdx.x; r < n_s; r += C) {
                nd_st(PA, r + 2u, r + 2u);
                if (gflags) __stcg(gflags + r + 2u, 0u);
            }
            if (threadIdx.x == 0) {  // a pass starts with clear borders, no early exit, an empty edge list
                nd_st(PA, 0u, 0u);
                nd_st(PA, 1u, 1u);
                c.stop = 0u;
                c.ecount[0] = 0u;
                c.ecount[1] = 0u;
            }
            __syncthreads();
            if (smem_bm && L == kPlaneL)
                union_pass<true, true, kScanPlanes, false, true>(c, PA, nullptr, sm.sbm, Tb, E, smp.perm, smp.rank, L,
                                                                 fd, 0u, n_s, 0u);
            else if (smem_bm)
                union_pass<true, true, kScanRows, false, true>(c, PA, nullptr, sm.sbm, Tb, E, smp.perm, smp.rank, L, fd,
                                                               0u, n_s, 0u);
            else if (L <= sum_L)
                union_pass<false, true, kScanGroups, false, true>(c, PA, nullptr, bm, Ts, E, smp.perm, smp.rank, L, fd,
                                                                  0u, n_s, 0u);
            else
                union_pass<false, true, kScanGroupsG, false, true>(c, PA, nullptr, bm, Ts, E, smp.perm, smp.rank, L, fd,
                                                                   0u, n_s, 0u);
            __syncthreads();
            ++npass;
            if (threadIdx.x == 0) tot_probe += n_s;
            bool span;
            if (gflags) {  // the face words of the first pass's clusters, at their roots
                for (uint32_t r = threadIdx.x; r < n_s; r += C) {
                    const uint32_t f = site_geo<kScanRows>(__ldg(smp.perm + r), L, fd, kAnyAxis).faces;
                    if (f) atomicOr(gflags + uf_find(PA, r + 2u, 0u), f);
                }
                __syncthreads();
                bool any_span = false;
                for (uint32_t r = threadIdx.x; r < n_s && !any_span; r += C)
                    any_span = spans_any(__ldcg(gflags + uf_find(PA, r + 2u, 0u)));
                span = __syncthreads_or(any_span);
            } else {
                span = nd_ld(PA, 1u) != 1u;
            }
            lend_back(P, PA, n_s + 2u);  // (a barrier: every thread has read node 1)
            if (!span) break;
            if (threadIdx.x == 0) ++tot_fb;  // n* < n_s
            have_br = false;
            const uint32_t prev = n_s;
            n_s = (tries < 3u && prev >= 4096u) ? static_cast<uint32_t>(uint64_t(prev) * 3u / 4u) : 0u;
            bitmap_update(bm, smp.perm, prev, n_s);  // clears the bits of ranks n_s .. prev-1
            if (n_s == 0u && threadIdx.x == 0) {  // the sweep from the start
                nd_st(P, 0u, 0u);
                nd_st(P, 1u, 1u);
            }
            __syncthreads();
        }
        uint32_t chunks = 0, ns;
        if (threadIdx.x == 0) cyc_first += static_cast<unsigned long long>(clock64() - t_first);
        if (smem_bm && L == kPlaneL)
            ns = span_sweep<true, kScanPlanes>(c, x, P, bm, sm, Tb, wp, E, smp, fd, lim, n_s, chunks, cyc_back, cyc_span,
                                               &hdr->status, gflags);
        else if (smem_bm)
            ns = span_sweep<true, kScanRows>(c, x, P, bm, sm, Tb, wp, E, smp, fd, lim, n_s, chunks, cyc_back, cyc_span,
                                             &hdr->status, gflags);
        else if (L <= sum_L)
            ns = span_sweep<false, kScanGroups>(c, x, P, bm, sm, Ts, wp, E, smp, fd, lim, n_s, chunks, cyc_back, cyc_span,
                                                &hdr->status, gflags);
        else
            ns = span_sweep<false, kScanGroupsG>(c, x, P, bm, sm, Ts, wp, E, smp, fd, lim, n_s, chunks, cyc_back, cyc_span,
                                                 &hdr->status, gflags);
        npass += chunks;
        if (threadIdx.x == 0) {
            tot_chunks += chunks;
            if (have_br && ns >= blo && ns <= bhi) ++tot_ok;
        }
        if (threadIdx.x == 0) {
            nstar_out[s] = ns;
            if (ns == PERC_NEVER && lim < N && unresolved) atomicAdd(unresolved, 1u);  // past the prefix
            if (passes_out) passes_out[s] = npass;
            tot_passes += npass;
            if (stats) {
                atomicAdd(&stats->hooks, c.hooks);
                atomicAdd(&stats->sites_merged, c.sites);
                atomicAdd(&stats->unions, c.unions);
                atomicAdd(&stats->new_sites, static_cast<unsigned long long>(ns == PERC_NEVER ? N : ns));
                atomicAdd(&stats->cyc_scan, c.cyc_scan);
                atomicAdd(&stats->cyc_link, c.cyc_link);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && stats) {
        atomicAdd(&stats->passes, tot_passes);
        atomicAdd(&stats->probe_sites, tot_probe);
        atomicAdd(&stats->fallbacks, tot_fb);
        atomicAdd(&stats->verified, tot_ok);
        atomicAdd(&stats->chunks, tot_chunks);
        atomicAdd(&stats->cyc_setup, cyc_setup);
        atomicAdd(&stats->cyc_update, cyc_first);
        atomicAdd(&stats->cyc_commit, cyc_back);
        atomicAdd(&stats->cyc_union, cyc_span);
    }
}

// ------------------------------------------------------------------------------------------------
// host side: launch configuration and workspace layout
// ------------------------------------------------------------------------------------------------
struct LaunchCfg {
    int threads = 0;
    size_t smem = 0;
    uint32_t smem_L = 0;
    uint32_t sum_L = 0;   // summary kernels: largest side whose occupancy summary is in shared memory
    size_t region = 0;    // summary kernels: bytes of the shared bitmap / summary region
    uint32_t node_cap = 0;
    uint32_t edge_scap = 0;
    uint32_t grid = 0;
    uint32_t members = 1;  // CTAs per sample (> 1: the cooperative group kernel)
    size_t slot_bytes = 0;
};

static int env_int(const char *name, int dflt)
{
    const char *v = getenv(name);
    return v ? atoi(v) : dflt;
}

constexpr int kCfgDevices = 64;
static std::mutex g_attr_mutex;
static size_t g_attr_bytes[kAttrSlots][kCfgDevices];
static uint32_t g_attr_ctas[kAttrSlots][kCfgDevices];

int ensure_smem_attr(AttrSlot slot, const void *fn, size_t bytes)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCfgDevices) return PERC_ECUDA;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (g_attr_bytes[slot][dev] >= bytes) return PERC_OK;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes)) != cudaSuccess)
        return PERC_ECUDA;
    g_attr_bytes[slot][dev] = bytes;
    return PERC_OK;
}

static size_t g_dev_total[kCfgDevices];

// Slot memory a launch on the current device may take (a fixed share of its memory, cached per
// device so that the workspace query and the launch agree).
static int slot_cap_bytes(size_t &cap)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCfgDevices) return PERC_ECUDA;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    if (!g_dev_total[dev]) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || total_b == 0) return PERC_ECUDA;
        g_dev_total[dev] = total_b;
    }
    cap = g_dev_total[dev] / kSlotCapShare;
    return PERC_OK;
}

int resident_ctas(AttrSlot slot, const void *fn, int threads, size_t smem, uint32_t &ctas)
{
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCfgDevices) return PERC_ECUDA;
    {
        std::lock_guard<std::mutex> lock(g_attr_mutex);
        if (g_attr_ctas[slot][dev]) {
            ctas = g_attr_ctas[slot][dev];
            return PERC_OK;
        }
    }
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess)
        return PERC_ECUDA;
    ctas = static_cast<uint32_t>(sms * (occ > 0 ? occ : 1));
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    g_attr_ctas[slot][dev] = ctas;
    return PERC_OK;
}

struct CfgCache {
    int threads = 0, occ = 0;
    size_t smem = 0, attr_smem = 0;
    bool valid = false;
};
static CfgCache g_cfg_cache[4][kCfgDevices];
static std::mutex g_cfg_mutex;

// Launch options set through perc_set_launch_option (0 = automatic).
static int g_opt_threads = 0, g_opt_smem_nodes = -1, g_opt_max_ctas = 0, g_opt_group = 0, g_opt_method = 0;
static uint32_t g_opt_spin_limit = 0;  // polls of a bounded device wait; 0 = kSpinLimit

uint32_t spin_limit() { return g_opt_spin_limit ? g_opt_spin_limit : kSpinLimit; }
constexpr int kOpSweep = 100;     // launch configuration of k_nstar_sweep (perc_nstar, sweep method)
constexpr int kOpSweepAny = 101;  // k_nstar_sweep along any axis (perc_nstar_any): slots with face words
static CfgCache g_group_cache[kCfgDevices];

static int launch_cfg(int op, uint32_t max_L, uint32_t num, LaunchCfg &cfg, bool allow_group = true)
{
    if (max_L < 1 || max_L > PERC_MAX_L || num == 0) return PERC_EINVAL;
    const uint64_t Ncap = num_sites(max_L);
    cfg.smem_L = max_L < kSmemBitmapMaxL ? max_L : kSmemBitmapMaxL;
    int dflt_threads = max_L <= 8 ? 256 : (max_L <= 12 ? 512 : 1024);
    if (g_opt_threads > 0) dflt_threads = g_opt_threads;
    cfg.threads = env_int("PERC_THREADS", dflt_threads);
    if (cfg.threads < 32 || cfg.threads > 1024 || (cfg.threads & 31)) return PERC_EINVAL;
    int dev = 0, sms = 0, occ = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PERC_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERC_ECUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return PERC_ECUDA;
    // Shared memory per CTA: the register file holds 65536 / (threads * 64) CTAs per SM (64
    // registers a thread); each CTA takes an equal share.  What the tables and the bitmap leave
    // goes to union-find nodes (up to kSmemNodes, keeping room for 512 edges) and then to the
    // shared part of the edge list.
    const bool sweep_op = op == kOpSweep || op == kOpSweepAny;
    const size_t extra = (op == PERC_OP_SMAX || sweep_op) ? smem_window_bytes(cfg.threads) : 0;
    // The sweep, S_max windows and the mass pass keep one shared region for the bitmap of lattices
    // up to smem_L or the occupancy summary of lattices up to sum_L (whose bitmap is global).  A
    // batch whose largest side is above kSmemBitmapMaxL gives the region to summaries (and the rest
    // to union-find nodes), unless it also reaches past kSumMixL (mixed batches), where the region of
    // a side-16 bitmap also holds the summaries up to side 32.
    const bool sum_op = op == PERC_OP_MASS || op == PERC_OP_SMAX || sweep_op;
    if (sum_op) cfg.smem_L = max_L <= kSmemBitmapMaxL ? max_L : (max_L > kSumMixL ? kPlaneL : 0u);
    auto base_for = [&](uint32_t sL) {
        return sum_op ? smem_tables_bytes() + smem_sum_tables_bytes() + region_bm_bytes(sL) + extra
                      : smem_tables_bytes() + smem_bitmap_bytes(sL) + extra;
    };
    size_t base = base_for(cfg.smem_L);
    const size_t min_edges = size_t(kRowCand) * sizeof(uint32_t);  // table-building scratch
    int ctas = (65536 / (cfg.threads * 64)) > 0 ? 65536 / (cfg.threads * 64) : 1;
    while (ctas > 1 && size_t(optin) / ctas - 1024 < base + min_edges) --ctas;  // fewer, larger CTAs
    const size_t share = size_t(optin) / ctas - 1024;  // room for the static shared variables
    // a lattice whose bitmap does not fit beside the op's own arrays keeps it in global memory
    while (cfg.smem_L > (sum_op ? 0u : 1u) && base + min_edges > share) base = base_for(--cfg.smem_L);
    if (base + min_edges > share) return PERC_EINVAL;
    cfg.sum_L = max_L;
    if (sum_op) {
        // summaries of lattices above smem_L: as large as fits beside a reserve for nodes and edges
        cfg.region = region_bm_bytes(cfg.smem_L);
        const size_t fixed = smem_tables_bytes() + smem_sum_tables_bytes() + extra + min_edges + kSumReserve;
        const size_t room = std::max(cfg.region, share > fixed ? share - fixed : size_t(0));
        cfg.sum_L = cfg.smem_L;
        while (cfg.sum_L < max_L && sum_bytes(cfg.sum_L + 1) <= room) ++cfg.sum_L;
        cfg.region = std::max(cfg.region, sum_bytes(cfg.sum_L));
        base = smem_tables_bytes() + smem_sum_tables_bytes() + cfg.region + extra;
        if (base + min_edges > share) return PERC_EINVAL;
    }
    size_t room = share - base;
    size_t nodes = room > 512 * sizeof(uint2) ? (room - 512 * sizeof(uint2)) / 4 : 0;
    if (nodes > kSmemNodes) nodes = kSmemNodes;
    const int nodes_env = env_int("PERC_SMEM_NODES", g_opt_smem_nodes);
    if (nodes_env >= 0 && size_t(nodes_env) < nodes) nodes = nodes_env;
    nodes &= ~size_t(3);
    cfg.node_cap = static_cast<uint32_t>(nodes);
    room -= smem_nodes_bytes(cfg.node_cap);
    cfg.edge_scap = static_cast<uint32_t>(room / sizeof(uint2));
    cfg.smem = base + smem_nodes_bytes(cfg.node_cap) + size_t(cfg.edge_scap) * sizeof(uint2);
    // The attribute and the occupancy are queried once per (kernel, device, threads, shared memory)
    // and cached, so that a call made while a stream is being captured issues no such query.
    const int k = op == PERC_OP_MASS ? 1 : op == PERC_OP_SMAX ? 2 : sweep_op ? 3 : 0;
    const void *fn = k == 1   ? reinterpret_cast<const void *>(k_mass)
                     : k == 2 ? reinterpret_cast<const void *>(k_smax)
                     : k == 3 ? reinterpret_cast<const void *>(k_nstar_sweep)
                              : reinterpret_cast<const void *>(k_nstar);
    {
        std::lock_guard<std::mutex> lock(g_cfg_mutex);
        CfgCache &cc = g_cfg_cache[k][dev < kCfgDevices ? dev : 0];
        if (cc.threads == cfg.threads && cc.smem == cfg.smem && cc.valid) {
            occ = cc.occ;
        } else {
            if (cfg.smem > cc.attr_smem) {
                if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cfg.smem)) != cudaSuccess)
                    return PERC_ECUDA;
                cc.attr_smem = cfg.smem;
            }
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, cfg.threads, cfg.smem) != cudaSuccess)
                return PERC_ECUDA;
            cc.threads = cfg.threads;
            cc.smem = cfg.smem;
            cc.occ = occ;
            cc.valid = true;
        }
    }
    if (occ < 1) return PERC_EINVAL;
    cfg.slot_bytes = slot_bytes_for(Ncap, max_L > cfg.smem_L, cfg.threads, max_L > cfg.sum_L ? max_L : 0u, op != kOpSweep);
    // (the any-axis sweep keeps its face words in the second node-sized array)
    uint64_t grid = uint64_t(sms) * occ;
    const int cta_cap = env_int("PERC_MAX_CTAS", g_opt_max_ctas);
    if (cta_cap > 0 && uint64_t(cta_cap) < grid) grid = cta_cap;

    // CTAs per sample: a batch of big lattices (bitmap in global memory) with fewer samples than
    // SMs runs each sample on a cooperative group of CTAs; PERC_OPT_GROUP forces a size (1: never)
    if (op == PERC_OP_NSTAR && allow_group) {
        int members = env_int("PERC_GROUP", g_opt_group);
        if (members == 0) {
            members = 1;
            if (max_L > cfg.smem_L)
                while (members < 32 && uint64_t(members) * 2 * num <= grid) members *= 2;
        }
        if (members > 1) {
            // the group kernel keeps no bitmap or nodes in shared memory: tables and edges only
            const size_t gbase = smem_tables_bytes();
            const size_t gshare = size_t(optin) - 1024;
            cfg.members = static_cast<uint32_t>(members);
            cfg.node_cap = 0;
            cfg.edge_scap = static_cast<uint32_t>((gshare - gbase) / sizeof(uint2));
            cfg.smem = gbase + size_t(cfg.edge_scap) * sizeof(uint2);
            int gocc = 0;
            {
                std::lock_guard<std::mutex> lock(g_cfg_mutex);
                CfgCache &cc = g_group_cache[dev < kCfgDevices ? dev : 0];
                if (cc.valid && cc.threads == cfg.threads && cc.smem == cfg.smem) {
                    gocc = cc.occ;
                } else {
                    if (cfg.smem > cc.attr_smem) {
                        if (cudaFuncSetAttribute(k_nstar_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 int(cfg.smem)) != cudaSuccess)
                            return PERC_ECUDA;
                        cc.attr_smem = cfg.smem;
                    }
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gocc, k_nstar_group, cfg.threads, cfg.smem) !=
                        cudaSuccess)
                        return PERC_ECUDA;
                    cc.threads = cfg.threads;
                    cc.smem = cfg.smem;
                    cc.occ = gocc;
                    cc.valid = true;
                }
            }
            uint64_t resident = uint64_t(sms) * gocc;  // a cooperative launch must be co-resident
            if (cta_cap > 0 && uint64_t(cta_cap) < resident) resident = cta_cap;
            uint64_t groups = resident / members;
            if (groups < 1) return PERC_EINVAL;
            if (groups > num) groups = num;
            cfg.slot_bytes = group_slot_bytes(Ncap, cfg.threads, cfg.members);
            size_t cap_b = 0;
            if (slot_cap_bytes(cap_b) != PERC_OK) return PERC_ECUDA;
            const uint64_t mem_groups = cap_b / cfg.slot_bytes;
            if (groups > mem_groups) groups = mem_groups > 0 ? mem_groups : 1;
            cfg.grid = static_cast<uint32_t>(groups * members);
            return PERC_OK;
        }
    }
    if (grid > num) grid = num;
    size_t cap_b = 0;
    if (slot_cap_bytes(cap_b) != PERC_OK) return PERC_ECUDA;
    const uint64_t mem_cap = cap_b / cfg.slot_bytes;
    if (grid > mem_cap) grid = mem_cap > 0 ? mem_cap : 1;
    cfg.grid = static_cast<uint32_t>(grid);
    return PERC_OK;
}

}  // namespace perc

using namespace perc;

// A launch resets its work queue; the status word keeps the first device-side error since the last
// perc_check (the caller zeroes the header once when it allocates the workspace).
static cudaError_t reset_queue(void *workspace, cudaStream_t stream)
{
    return cudaMemsetAsync(static_cast<char *>(workspace) + offsetof(WsHeader, queue), 0, sizeof(uint32_t), stream);
}

// Workspace of a launch: the header and one slot per sample in flight -- per CTA, or per group of
// `members` CTAs for the cooperative group kernel (its CTAs share their group's slot).
static size_t cfg_ws_bytes(const LaunchCfg &cfg)
{
    return sizeof(WsHeader) + size_t(cfg.grid / cfg.members) * cfg.slot_bytes;
}

extern "C" size_t perc_workspace_bytes(int op, uint32_t max_L, uint32_t num)
{
    if (op == PERC_OP_RANK) {
        if (max_L < 1 || max_L > PERC_MAX_L || num == 0) return 0;
        return rank_workspace_bytes(max_L, num);
    }
    if (op == PERC_OP_PERIODIC) return periodic_workspace_bytes(max_L, num);
    if (op == PERC_OP_MINIMAX) return minimax_workspace_bytes(max_L, num);
    if (op == PERC_OP_NSTAR_ANY) {
        LaunchCfg any;
        return launch_cfg(kOpSweepAny, max_L, num, any) == PERC_OK ? cfg_ws_bytes(any) : 0;
    }
    if (op != PERC_OP_NSTAR && op != PERC_OP_MASS && op != PERC_OP_SMAX) return 0;
    LaunchCfg cfg;
    if (launch_cfg(op, max_L, num, cfg) != PERC_OK) return 0;
    size_t bytes = cfg_ws_bytes(cfg);
    LaunchCfg sw;  // perc_nstar may run either method: room for both
    if (op == PERC_OP_NSTAR && launch_cfg(kOpSweep, max_L, num, sw) == PERC_OK) bytes = std::max(bytes, cfg_ws_bytes(sw));
    return bytes;
}

// The method perc_nstar uses: bisection (1) or the sweep (2); a negative status if the sweep was
// asked for and cannot be configured.  Automatic (0): the sweep, unless the bisection would run
// cooperative groups (big lattices in small batches) or the sweep's shared-memory arrays do not fit.
static int nstar_method(uint32_t max_L, uint32_t num, const LaunchCfg &bis, LaunchCfg &sw)
{
    const int m = env_int("PERC_METHOD", g_opt_method);
    if (m == 1) return 1;
    const int rc = launch_cfg(kOpSweep, max_L, num, sw);
    if (m == 2) return rc == PERC_OK ? 2 : rc;
    return (rc == PERC_OK && bis.members == 1) ? 2 : 1;
}

extern "C" int perc_nstar(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                          const uint32_t *bracket, uint32_t *nstar, uint32_t *passes, perc_stats *stats,
                          void *workspace, size_t ws_bytes, void *stream_)
{
    if (!samples || !nstar || !workspace || num_samples == 0) return PERC_EINVAL;
    LaunchCfg cfg, sw;
    int rc = launch_cfg(PERC_OP_NSTAR, max_L, num_samples, cfg);
    if (rc != PERC_OK) return rc;
    const int method = nstar_method(max_L, num_samples, cfg, sw);
    if (method < 0) return method;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (method == 2) {
        if (ws_bytes < cfg_ws_bytes(sw)) return PERC_EWORKSPACE;
        if (reset_queue(workspace, stream) != cudaSuccess) return PERC_ECUDA;
        k_nstar_sweep<<<sw.grid, sw.threads, sw.smem, stream>>>(samples, num_samples, max_L, sw.smem_L, sw.sum_L,
                                                                sw.region, sw.node_cap, sw.edge_scap, bracket, nstar,
                                                                passes, stats, static_cast<char *>(workspace),
                                                                sw.slot_bytes, 0u, nullptr, nullptr);
        return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
    }
    if (ws_bytes < cfg_ws_bytes(cfg)) return PERC_EWORKSPACE;
    if (reset_queue(workspace, stream) != cudaSuccess) return PERC_ECUDA;
    if (cfg.members > 1) {
        // every group's barrier counters, abort flag and shared scalars start at zero
        if (cudaMemset2DAsync(static_cast<char *>(workspace) + sizeof(WsHeader), cfg.slot_bytes, 0, sizeof(GroupState),
                              cfg.grid / cfg.members, stream) != cudaSuccess)
            return PERC_ECUDA;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3(cfg.grid);
        lc.blockDim = dim3(cfg.threads);
        lc.dynamicSmemBytes = cfg.smem;
        lc.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&lc, k_nstar_group, samples, num_samples, max_L, cfg.members,
                                                 cfg.edge_scap, bracket, nstar, passes, stats,
                                                 static_cast<char *>(workspace), cfg.slot_bytes, spin_limit());
        return e == cudaSuccess ? PERC_OK : PERC_ECUDA;
    }
    k_nstar<<<cfg.grid, cfg.threads, cfg.smem, stream>>>(samples, num_samples, max_L, cfg.smem_L, cfg.node_cap, cfg.edge_scap, bracket,
                                                         nstar, passes, stats, static_cast<char *>(workspace),
                                                         cfg.slot_bytes);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

// n* under the any-axis spanning rule from the per-axis values: spanning along one axis is
// monotone in n, so the first n at which some axis spans is the smallest of the per-axis n*
// (PERC_NEVER, the largest uint32, drops out of the minimum unless every axis is PERC_NEVER).
namespace perc {
__global__ void __launch_bounds__(256) k_nstar_min_axes(const uint32_t *__restrict__ nstar, uint32_t num,
                                                        uint32_t axes, uint32_t *__restrict__ out)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= num) return;
    const uint32_t *row = nstar + size_t(k) * axes;
    uint32_t m = PERC_NEVER;
    for (uint32_t a = 0; a < axes; ++a) m = min(m, __ldg(row + a));
    out[k] = m;
}
}  // namespace perc

extern "C" int perc_nstar_min_axes(const uint32_t *nstar, uint32_t num, uint32_t axes, uint32_t *out,
                                   void *stream_)
{
    if (!nstar || !out || num == 0 || axes == 0 || axes > 5) return PERC_EINVAL;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    k_nstar_min_axes<<<(num + 255u) / 256u, 256, 0, stream>>>(nstar, num, axes, out);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

extern "C" int perc_nstar_any(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                              const uint32_t *bracket, uint32_t *nstar, uint32_t *passes, perc_stats *stats,
                              void *workspace, size_t ws_bytes, void *stream_)
{
    if (!samples || !nstar || !workspace || num_samples == 0) return PERC_EINVAL;
    LaunchCfg cfg;
    const int rc = launch_cfg(kOpSweepAny, max_L, num_samples, cfg);
    if (rc != PERC_OK) return rc;
    if (ws_bytes < cfg_ws_bytes(cfg)) return PERC_EWORKSPACE;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (reset_queue(workspace, stream) != cudaSuccess) return PERC_ECUDA;
    k_nstar_sweep<<<cfg.grid, cfg.threads, cfg.smem, stream>>>(samples, num_samples, max_L, cfg.smem_L, cfg.sum_L,
                                                               cfg.region, cfg.node_cap, cfg.edge_scap, bracket, nstar,
                                                               passes, stats, static_cast<char *>(workspace),
                                                               cfg.slot_bytes, 1u, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

// The sweep on orders ranked only up to prefix_sites(L^5, *share) (perc_nstar_prefix along the
// sample's axis, perc_nstar_any_prefix along any axis).
static int nstar_prefix(bool any, const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                        const uint32_t *bracket, const uint32_t *share, uint32_t *unresolved, uint32_t *nstar,
                        uint32_t *passes, perc_stats *stats, void *workspace, size_t ws_bytes, void *stream_)
{
    if (!samples || (!share && !bracket) || !unresolved || !nstar || !workspace || num_samples == 0)
        return PERC_EINVAL;
    LaunchCfg cfg;
    const int rc = launch_cfg(any ? kOpSweepAny : kOpSweep, max_L, num_samples, cfg);
    if (rc != PERC_OK) return rc;
    if (ws_bytes < cfg_ws_bytes(cfg)) return PERC_EWORKSPACE;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (reset_queue(workspace, stream) != cudaSuccess) return PERC_ECUDA;
    k_nstar_sweep<<<cfg.grid, cfg.threads, cfg.smem, stream>>>(samples, num_samples, max_L, cfg.smem_L, cfg.sum_L,
                                                               cfg.region, cfg.node_cap, cfg.edge_scap, bracket, nstar,
                                                               passes, stats, static_cast<char *>(workspace),
                                                               cfg.slot_bytes, any ? 1u : 0u, share, unresolved);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

extern "C" int perc_nstar_prefix(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                                 const uint32_t *bracket, const uint32_t *share, uint32_t *unresolved,
                                 uint32_t *nstar, uint32_t *passes, perc_stats *stats, void *workspace,
                                 size_t ws_bytes, void *stream)
{
    return nstar_prefix(false, samples, num_samples, max_L, bracket, share, unresolved, nstar, passes, stats,
                        workspace, ws_bytes, stream);
}

extern "C" int perc_nstar_any_prefix(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                                     const uint32_t *bracket, const uint32_t *share, uint32_t *unresolved,
                                     uint32_t *nstar, uint32_t *passes, perc_stats *stats, void *workspace,
                                     size_t ws_bytes, void *stream)
{
    return nstar_prefix(true, samples, num_samples, max_L, bracket, share, unresolved, nstar, passes, stats,
                        workspace, ws_bytes, stream);
}

extern "C" int perc_mass(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                         const uint64_t *n, int64_t *mass, void *workspace, size_t ws_bytes, void *stream_)
{
    if (!samples || !n || !mass || !workspace || num_samples == 0) return PERC_EINVAL;
    LaunchCfg cfg;
    int rc = launch_cfg(PERC_OP_MASS, max_L, num_samples, cfg);
    if (rc != PERC_OK) return rc;
    if (ws_bytes < cfg_ws_bytes(cfg)) return PERC_EWORKSPACE;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (reset_queue(workspace, stream) != cudaSuccess) return PERC_ECUDA;
    k_mass<<<cfg.grid, cfg.threads, cfg.smem, stream>>>(samples, num_samples, max_L, cfg.smem_L, cfg.sum_L, cfg.region,
                                                        cfg.node_cap, cfg.edge_scap, n, mass,
                                                        static_cast<char *>(workspace), cfg.slot_bytes);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

extern "C" int perc_smax_window(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                                const uint64_t *n_lo, const uint32_t *count, uint32_t window, uint32_t *smax,
                                void *workspace, size_t ws_bytes, void *stream_)
{
    if (!samples || !n_lo || !smax || !workspace || num_samples == 0 || window == 0) return PERC_EINVAL;
    if (uint64_t(num_samples) * window > (uint64_t(1) << 40)) return PERC_EINVAL;
    LaunchCfg cfg;
    int rc = launch_cfg(PERC_OP_SMAX, max_L, num_samples, cfg);
    if (rc != PERC_OK) return rc;
    if (ws_bytes < cfg_ws_bytes(cfg)) return PERC_EWORKSPACE;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (reset_queue(workspace, stream) != cudaSuccess) return PERC_ECUDA;
    k_smax<<<cfg.grid, cfg.threads, cfg.smem, stream>>>(samples, num_samples, max_L, cfg.smem_L, cfg.sum_L, cfg.region,
                                                        cfg.node_cap, cfg.edge_scap, n_lo, count, window, smax,
                                                        static_cast<char *>(workspace), cfg.slot_bytes);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

extern "C" int perc_set_launch_option(int option, int value)
{
    switch (option) {
    case PERC_OPT_THREADS:
        if (value != 0 && (value < 32 || value > 1024 || (value & 31))) return PERC_EINVAL;
        g_opt_threads = value;
        return PERC_OK;
    case PERC_OPT_SMEM_NODES:
        if (value < -1) return PERC_EINVAL;
        g_opt_smem_nodes = value;
        return PERC_OK;
    case PERC_OPT_MAX_CTAS:
        if (value < 0) return PERC_EINVAL;
        g_opt_max_ctas = value;
        return PERC_OK;
    case PERC_OPT_GROUP:
        if (value < 0 || value > 64) return PERC_EINVAL;
        g_opt_group = value;
        return PERC_OK;
    case PERC_OPT_METHOD:
        if (value < 0 || value > 2) return PERC_EINVAL;
        g_opt_method = value;
        return PERC_OK;
    case PERC_OPT_SPIN_LIMIT:
        if (value < 0) return PERC_EINVAL;
        g_opt_spin_limit = static_cast<uint32_t>(value);
        return PERC_OK;
    default:
        return PERC_EINVAL;
    }
}

extern "C" int perc_check(void *workspace, void *stream_)
{
    if (!workspace) return PERC_EINVAL;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (cudaStreamSynchronize(stream) != cudaSuccess) return PERC_ECUDA;
    int status = 0;
    if (cudaMemcpy(&status, workspace, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PERC_ECUDA;
    const int zero = 0;
    if (cudaMemcpy(workspace, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return PERC_ECUDA;
    return status;
}

extern "C" const char *perc_status_string(int status)
{
    switch (status) {
    case PERC_OK: return "ok";
    case PERC_EINVAL: return "invalid argument";
    case PERC_EWORKSPACE: return "workspace too small";
    case PERC_ECUDA: return "CUDA runtime error";
    case PERC_ETIMEOUT: return "bounded device wait ran out";
    case PERC_EDEVICE: return "device-side check failed (invalid sample)";
    default: return "unknown status";
    }
}

// ------------------------------------------------------------------------------------------------
// perc_nstar_noalloc: perc_nstar for callers that cannot allocate device memory themselves.
//
// Its scratch is one file-scope device array of kNoAllocBytes (64 MiB), which every GPU that
// loads this library keeps until the process exits.  The first call on a device, with that device
// current, looks the array's device address up with cudaGetSymbolAddress (in host code the
// array's name is only a host-side stand-in, not a device address) and caches it per device; make
// that first call before any stream capture.  The call itself allocates nothing.  All calls share
// the array, so calls that may overlap on the GPU (other streams, other host threads) race and
// must be serialised by the caller.  The persistent launch uses as many CTAs as there are slots of
// the launch's size in the array: lattices whose single slot does not fit are rejected with
// PERC_EWORKSPACE.
// ------------------------------------------------------------------------------------------------
#include <mutex>

namespace perc {
constexpr size_t kNoAllocBytes = size_t(64) << 20;
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static void *g_noalloc_ptr[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;
}  // namespace perc

extern "C" int perc_nstar_noalloc(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                                  const uint32_t *bracket, uint32_t *nstar, uint32_t *passes,
                                  perc_stats *stats, void *stream_)
{
    if (!samples || !nstar || num_samples == 0) return PERC_EINVAL;
    LaunchCfg cfg;
    int rc = launch_cfg(PERC_OP_NSTAR, max_L, num_samples, cfg, false);  // one CTA per sample here
    if (rc != PERC_OK) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return PERC_ECUDA;
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PERC_ECUDA;
            if (cudaMemset(p, 0, sizeof(WsHeader)) != cudaSuccess) return PERC_ECUDA;  // status and queue
            g_noalloc_ptr[dev] = p;
        }
        ws = g_noalloc_ptr[dev];
    }
    const size_t slots = (kNoAllocBytes - sizeof(WsHeader)) / cfg.slot_bytes;
    if (slots == 0) return PERC_EWORKSPACE;  // max_L too large for the static scratch
    const uint32_t grid = cfg.grid < slots ? cfg.grid : static_cast<uint32_t>(slots);
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (reset_queue(ws, stream) != cudaSuccess) return PERC_ECUDA;
    k_nstar<<<grid, cfg.threads, cfg.smem, stream>>>(samples, num_samples, max_L, cfg.smem_L, cfg.node_cap,
                                                     cfg.edge_scap, bracket, nstar, passes, stats,
                                                     static_cast<char *>(ws), cfg.slot_bytes);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}
