// perc_common.cuh -- device helpers shared by the kernels of libperc.so.
//
//  * the coordination-zone table of the 5D simple cubic lattice (eq. z; Table I): zone i holds the
//    lattice vectors v with |v|^2 = i, i = 1..7 (sizes 10, 40, 80, 90, 112, 240, 320), generated at
//    compile time into constant memory;
//  * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based generator that keys the
//    random site-addition order of the Newman--Ziff method;
//  * exact division by a runtime lattice side L through a 64-bit reciprocal.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/perc.h"

namespace perc {

// ------------------------------------------------------------------------------------------------
// Coordination zones.  Each vector is packed as five 3-bit fields (d_k + 2), k = 0 for x1 (the
// slowest lattice index) ... k = 4 for x5, field k at bits 3k..3k+2.
// ------------------------------------------------------------------------------------------------
constexpr int kZoneCount = 7;
constexpr int kMaxOffsets = 892;

struct ZoneTable {
    uint16_t vec[kMaxOffsets];
    uint16_t start[kZoneCount + 1];  // zone i occupies vec[start[i-1] .. start[i])
};

constexpr ZoneTable make_zone_table()
{
    ZoneTable t{};
    int cnt = 0;
    for (int zone = 1; zone <= kZoneCount; ++zone) {
        t.start[zone - 1] = static_cast<uint16_t>(cnt);
        for (int code = 0; code < 3125; ++code) {  // 5^5 vectors of {-2..2}^5
            int c = code, r2 = 0, packed = 0;
            for (int k = 4; k >= 0; --k) {
                const int d = c % 5 - 2;
                c /= 5;
                r2 += d * d;
                packed |= (d + 2) << (3 * k);
            }
            if (r2 == zone) t.vec[cnt++] = static_cast<uint16_t>(packed);
        }
    }
    t.start[kZoneCount] = static_cast<uint16_t>(cnt);
    return t;
}

constexpr ZoneTable kZones = make_zone_table();
static_assert(kZones.start[1] == 10 && kZones.start[2] == 50 && kZones.start[3] == 130 &&
                  kZones.start[4] == 220 && kZones.start[5] == 332 && kZones.start[6] == 572 &&
                  kZones.start[7] == 892,
              "zone sizes must be 10, 40, 80, 90, 112, 240, 320");

__host__ __device__ inline int zone_component(uint32_t packed, int k)
{
    return static_cast<int>((packed >> (3 * k)) & 7u) - 2;
}

// Neighbor entry for one (L, offset): linear index delta and a 25-bit one-hot of the five
// components (bit 5k + d_k + 2).  The site's "allowed" mask has bit 5k + d + 2 set when
// 0 <= x_k + d < L; the offset stays inside the lattice iff (onehot & ~allowed) == 0.
struct NbrEntry {
    int32_t delta;
    uint32_t onehot;
};

__host__ __device__ inline NbrEntry make_nbr_entry(uint32_t packed, uint32_t L)
{
    int32_t delta = 0;
    uint32_t onehot = 0;
    for (int k = 0; k < 5; ++k) {
        const int d = zone_component(packed, k);
        delta = delta * static_cast<int32_t>(L) + d;
        onehot |= 1u << (5 * k + d + 2);
    }
    return NbrEntry{delta, onehot};
}

// Allowed-offset bits of one coordinate x in [0, L): bit d+2 for d in {-2..2} with 0 <= x+d < L.
__device__ __forceinline__ uint32_t allowed_bits(uint32_t x, uint32_t L)
{
    uint32_t a = 4u;                 // d = 0
    a |= (x >= 1u) ? 2u : 0u;        // d = -1
    a |= (x >= 2u) ? 1u : 0u;        // d = -2
    a |= (x + 1u < L) ? 8u : 0u;     // d = +1
    a |= (x + 2u < L) ? 16u : 0u;    // d = +2
    return a;
}

// ------------------------------------------------------------------------------------------------
// Exact i / L for 32-bit i through M = ceil(2^64 / L): floor(i * M / 2^64) = floor(i / L) because
// the rounding term i * (M - 2^64/L) / 2^64 < 2^-32 never crosses an integer boundary.
// ------------------------------------------------------------------------------------------------
struct FastDiv {
    uint64_t M;
    uint32_t L;
};

__host__ __device__ inline FastDiv make_fastdiv(uint32_t L)
{
    FastDiv f;
    f.L = L;
    f.M = (L <= 1u) ? 0ull : (~0ull / L) + 1ull;
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t i, const FastDiv &f)
{
    return f.L == 1u ? i : static_cast<uint32_t>(__umul64hi(static_cast<uint64_t>(i), f.M));
}

// Coordinates (x1..x5) of site i; x[0] = x1 is the slowest index.
__device__ __forceinline__ void site_coords(uint32_t i, const FastDiv &f, uint32_t x[5])
{
#pragma unroll
    for (int k = 4; k >= 1; --k) {
        const uint32_t q = fdiv(i, f);
        x[k] = i - q * f.L;
        i = q;
    }
    x[0] = i;
}

// ------------------------------------------------------------------------------------------------
// Philox4x32-10: ten rounds; round: (hi0,lo0) = 0xD2511F53 * x0, (hi1,lo1) = 0xCD9E8D57 * x2,
// x' = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); the key gains (0x9E3779B9, 0xBB67AE85) between
// rounds.  Only word 0 of the output is needed for the site key.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t y0 = hi1 ^ c1 ^ k0;
        const uint32_t y2 = hi0 ^ c3 ^ k1;
        c0 = y0;
        c1 = lo1;
        c2 = y2;
        c3 = lo0;
    }
    return c0;
}

// Site key of index i for a 64-bit seed: counter (i,0,0,0), key (seed lo, seed hi).
__device__ __forceinline__ uint32_t site_key(uint64_t seed, uint32_t i)
{
    return philox_word0(i, 0u, 0u, 0u, static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// ------------------------------------------------------------------------------------------------
// Status word helpers.  The first error wins; later ones are dropped.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

__host__ __device__ inline uint64_t num_sites(uint32_t L)
{
    const uint64_t l = L;
    return l * l * l * l * l;
}

// Sites of each order that perc_rank_prefix ranks at least and perc_nstar_prefix may read, for a
// lattice of N sites (PERC_PREFIX_SITES: the share of the lattice, an eighth more and 64 sites).
__host__ __device__ inline uint32_t prefix_sites(uint64_t N, uint32_t share)
{
    return static_cast<uint32_t>(PERC_PREFIX_SITES(N, share));
}

// A sample's bracket (lo, hi) as a share of its lattice of side L: hi / L^5 in units of 2^-24,
// rounded up; a bracket that perc_nstar would not use (lo < 1, lo > hi, hi > L^5) or an invalid side
// counts as the whole lattice (2^24).
__host__ __device__ inline uint32_t bracket_share(uint32_t L, uint32_t lo, uint32_t hi)
{
    const uint64_t N = (L >= 1u && L <= PERC_MAX_L) ? num_sites(L) : 0u;
    if (N == 0u || lo < 1u || lo > hi || hi > N) return 1u << 24;
    return static_cast<uint32_t>(((uint64_t(hi) << 24) + N - 1u) / N);
}

// Polls a bounded device-side wait makes before it gives up with PERC_ETIMEOUT: kSpinLimit, or
// the value of PERC_OPT_SPIN_LIMIT (defined in perc_ccl.cu).  A wait that drains copies still in
// flight after a timeout always uses kSpinLimit.
constexpr uint32_t kSpinLimit = 1u << 26;
uint32_t spin_limit();

// Host-side per-device launch state (defined in perc_ccl.cu; thread-safe).  Kernel attributes such
// as the dynamic shared-memory limit are set per device, so each is set once on every device that
// launches the kernel.  Returns PERC_OK or PERC_ECUDA.
enum AttrSlot {
    kAttrMlpGrad,
    kAttrRankScatter,
    kAttrRankScatterTma,
    kAttrRankBCount,
    kAttrRankBPlace,
    kAttrRankBSortBig,
    kAttrTorusMass,
    kAttrTorusWrap,
    kAttrMicrobench,
    kAttrMinimax,
    kAttrSlots
};
int ensure_smem_attr(AttrSlot slot, const void *fn, size_t bytes);
// Resident CTAs of `fn` (threads, dynamic shared memory) times the SM count of the current device,
// cached per (slot, device).
int resident_ctas(AttrSlot slot, const void *fn, int threads, size_t smem, uint32_t &ctas);

// Workspace of perc_rank for num_seeds seeds of side L (defined in perc_rank.cu).
size_t rank_workspace_bytes(uint32_t L, uint32_t num_seeds);
// Workspace of the periodic-boundary calls (defined in perc_periodic.cu); 0 when not configurable.
size_t periodic_workspace_bytes(uint32_t max_L, uint32_t num);
// Workspace of perc_nstar_minimax (defined in perc_minimax.cu); 0 when not configurable.
size_t minimax_workspace_bytes(uint32_t max_L, uint32_t num);

}  // namespace perc
