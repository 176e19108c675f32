// perc_rank.cu -- the random site-addition order of the Newman--Ziff method (Methods,
// "Computational methods"), one per seed.
//
// The order of seed s sorts the sites ascending by (key_i, i), key_i = word 0 of
// Philox4x32-10(counter (i,0,0,0), key (s lo, s hi)).  It is built by a stable least-significant-
// digit radix sort of the 32-bit keys with the site index as payload: the input is in index order
// and every pass is stable, so equal keys stay in index order.  Four 8-bit passes, each
//   k_rank_hist    per-tile digit counts (pass 0 draws the keys itself, nothing is stored first),
//   k_rank_scan    exclusive scan per seed in digit-major order -> tile output offsets,
//   k_rank_scatter stable scatter: warp-level peer ranking (lanes with equal digits found with
//                  eight ballots), tile staged in shared memory in digit order, written in runs,
// and the last scatter also writes rank[perm[r]] = r.  Seeds are sorted in chunks that fit the
// workspace.
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "perc_common.cuh"

namespace perc {

constexpr int kRankThreads = 512;
constexpr int kRankWarps = kRankThreads / 32;
constexpr int kRankItems = 8;
constexpr int kRankTile = kRankThreads * kRankItems;  // 4096 keys per tile
constexpr int kRankMaxChunk = 64;                     // seeds per chunk (upper bound)
constexpr size_t kRankChunkBytes = size_t(4) << 30;   // workspace aimed at per chunk

static inline int env_int_rank(const char *name, int dflt)
{
    const char *v = getenv(name);
    return v ? atoi(v) : dflt;
}

static inline uint32_t rank_tiles(uint64_t N) { return static_cast<uint32_t>((N + kRankTile - 1) / kRankTile); }

static inline size_t rank_bytes_per_seed(uint64_t N)
{
    const size_t keys = size_t(N) * 8;                               // key + value, one ping-pong side
    const size_t hist = size_t(256) * rank_tiles(N) * sizeof(uint32_t);
    return ((keys + hist) + 255) & ~size_t(255);
}

static inline uint32_t rank_chunk(uint64_t N, uint32_t num_seeds)
{
    size_t per = rank_bytes_per_seed(N);
    size_t c = kRankChunkBytes / per;
    if (c < 1) c = 1;
    if (c > kRankMaxChunk) c = kRankMaxChunk;
    if (c > num_seeds) c = num_seeds;
    return static_cast<uint32_t>(c);
}

size_t rank_workspace_bytes(uint32_t L, uint32_t num_seeds)
{
    const uint64_t N = num_sites(L);
    return 256 + 16 + size_t(rank_chunk(N, num_seeds)) * rank_bytes_per_seed(N);  // (+16: hist alignment)
}

// Element e of a tile is read by warp (e / 256), round ((e / 32) % 8), lane (e % 32): warp-major,
// then round, then lane, i.e. in input order.
__device__ __forceinline__ uint32_t tile_elem(uint32_t tile, int warp, int k, int lane)
{
    return tile * kRankTile + warp * (32 * kRankItems) + k * 32 + lane;
}

__global__ void __launch_bounds__(kRankThreads, 2)
k_rank_hist(int pass, uint32_t N, uint32_t T, const uint64_t *__restrict__ seeds,
            const uint32_t *__restrict__ keys_in, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[256];
    const uint32_t s = blockIdx.y, tile = blockIdx.x;
    if (threadIdx.x < 256) h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t seed = pass == 0 ? seeds[s] : 0ull;
    const uint32_t *kin = keys_in + size_t(s) * N;
    const uint32_t shift = 8u * pass;
#pragma unroll
    for (int k = 0; k < kRankItems; ++k) {
        const uint32_t e = tile * kRankTile + k * kRankThreads + threadIdx.x;
        if (e < N) {
            const uint32_t key = pass == 0 ? site_key(seed, e) : __ldg(kin + e);
            atomicAdd(&h[(key >> shift) & 255u], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < 256) hist[(size_t(s) * 256 + threadIdx.x) * T + tile] = h[threadIdx.x];
}

// Exclusive scan of one seed's n counters (n a multiple of 4; the digit-major 256*T tile counts of
// the radix passes, or the bucket counts of the bucket path), one block per seed: rounds of
// 4 * blockDim consecutive counters, each thread reading four neighbours at once (coalesced 16-byte
// loads; rows start 16-byte aligned), a block scan of the threads' sums and a running carry.  With
// `copy`, the scanned row is also written there.
__global__ void __launch_bounds__(1024) k_rank_scan(uint32_t n, uint32_t *__restrict__ hist, uint32_t *__restrict__ copy)
{
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry_s;
    uint32_t *h = hist + size_t(blockIdx.x) * n;
    uint32_t *cp = copy ? copy + size_t(blockIdx.x) * n : nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < n; base += 4u * blockDim.x) {
        const uint32_t i = base + 4u * threadIdx.x;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (i < n) v = *reinterpret_cast<const uint4 *>(h + i);
        const uint32_t local = v.x + v.y + v.z + v.w;
        uint32_t x = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = lane < nw ? warp_sum[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) warp_sum[lane] = w;  // inclusive
            if (lane == nw - 1) carry_s = carry + w;
        }
        __syncthreads();
        if (i < n) {
            uint32_t run = carry + x - local + (warp > 0 ? warp_sum[warp - 1] : 0u);
            uint4 o;
            o.x = run;
            run += v.x;
            o.y = run;
            run += v.y;
            o.z = run;
            run += v.z;
            o.w = run;
            *reinterpret_cast<uint4 *>(h + i) = o;
            if (cp) *reinterpret_cast<uint4 *>(cp + i) = o;
        }
        carry = carry_s;
        __syncthreads();  // warp_sum and carry_s are rewritten by the next round
    }
}

// Stable scatter of one tile by digit `pass`.  Each key's place inside the tile comes from
// warp-level peer ranking (ballots over the digit bits) and per-warp digit counters; the tile is staged in
// shared memory in digit order and then written out in runs, so consecutive threads write
// consecutive addresses.  The last pass writes the order itself: perm[dst] = site and
// rank[site] = dst.
struct ScatterSmem {
    uint32_t wcnt[kRankWarps][256];  // per-warp digit counts, then per-warp exclusive offsets
    uint32_t tstart[256];            // exclusive start of each digit inside the tile
    uint32_t goff[256];              // global start of this tile's run of each digit
    uint32_t skey[kRankTile];
    uint32_t sval[kRankTile];
};

__global__ void __launch_bounds__(kRankThreads, 2)
k_rank_scatter(int pass, uint32_t N, uint32_t T, const uint64_t *__restrict__ seeds,
               const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
               uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
               uint32_t *__restrict__ rank_out, const uint32_t *__restrict__ hist)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem &S = *reinterpret_cast<ScatterSmem *>(smem_raw);
    const uint32_t s = blockIdx.y, tile = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kRankWarps * 256; d += kRankThreads) (&S.wcnt[0][0])[d] = 0u;
    if (threadIdx.x < 256) S.goff[threadIdx.x] = hist[(size_t(s) * 256 + threadIdx.x) * T + tile];
    __syncthreads();

    const uint64_t seed = pass == 0 ? seeds[s] : 0ull;
    const size_t row = size_t(s) * N;
    const uint32_t shift = 8u * pass;
    const uint32_t lanes_below = (1u << lane) - 1u;
    uint32_t key[kRankItems], val[kRankItems], pos[kRankItems], dig[kRankItems];
#pragma unroll
    for (int k = 0; k < kRankItems; ++k) {
        const uint32_t e = tile_elem(tile, warp, k, lane);
        const bool valid = e < N;
        uint32_t kk = 0u, vv = 0u;
        if (valid) {
            if (pass == 0) {
                kk = site_key(seed, e);
                vv = e;
            } else {
                kk = __ldg(kin + row + e);
                vv = __ldg(vin + row + e);
            }
        }
        const uint32_t d = valid ? ((kk >> shift) & 255u) : 256u;
        // lanes with the same digit: AND over the 8 digit bits of (ballot of the bit, or its complement)
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
        if (!valid) peers = ~peers;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
        const uint32_t leader = __ffs(peers) - 1;
        const uint32_t base = valid ? S.wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == static_cast<int>(leader)) S.wcnt[warp][d] = base + __popc(peers);
        __syncwarp();
        key[k] = kk;
        val[k] = vv;
        pos[k] = base + __popc(peers & lanes_below);
        dig[k] = d;
    }
    __syncthreads();
    if (threadIdx.x < 256) {  // per digit: exclusive offsets over warps, and the digit's tile total
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll 8
        for (int w = 0; w < kRankWarps; ++w) {
            const uint32_t c = S.wcnt[w][d];
            S.wcnt[w][d] = run;
            run += c;
        }
        S.tstart[d] = run;  // tile total for now
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the 256 tile totals (one warp, 8 per lane)
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            v[q] = S.tstart[lane * 8 + q];
            sum += v[q];
        }
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        uint32_t run = x - sum;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            S.tstart[lane * 8 + q] = run;
            run += v[q];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRankItems; ++k) {
        const uint32_t d = dig[k];
        if (d < 256u) {
            const uint32_t lp = S.tstart[d] + S.wcnt[warp][d] + pos[k];
            S.skey[lp] = key[k];
            S.sval[lp] = val[k];
        }
    }
    __syncthreads();
    const uint32_t tile_n = min(static_cast<uint32_t>(kRankTile), N - tile * kRankTile);
    const bool last = pass == 3;
    for (uint32_t lp = threadIdx.x; lp < tile_n; lp += kRankThreads) {
        const uint32_t kk = S.skey[lp];
        const uint32_t d = (kk >> shift) & 255u;
        const uint32_t dst = S.goff[d] + (lp - S.tstart[d]);
        const uint32_t vv = S.sval[lp];
        vout[row + dst] = vv;
        if (last)
            rank_out[row + vv] = dst;
        else
            kout[row + dst] = kk;
    }
}

// ------------------------------------------------------------------------------------------------
// Persistent scatter for passes 1..3 with bulk-async tile loads.  Each CTA walks the (seed, tile)
// work list; while it ranks and writes one tile, the copy engine (cp.async.bulk, completion on an
// mbarrier) already brings the next tile's keys and values into the other shared buffer.  The
// buffer just ranked also serves as the staging area of the digit-ordered tile.  Needs 16-byte
// aligned rows (L^5 a multiple of 4); otherwise k_rank_scatter is used.  Waits are bounded: a copy
// that does not land within `spin_limit` polls (kSpinLimit unless PERC_OPT_SPIN_LIMIT sets another)
// sets PERC_ETIMEOUT in the workspace status word and the CTA stops, after waiting (up to
// kSpinLimit polls each) for the copies it still has in flight, so that none of them lands in
// shared memory a later CTA owns.  The launch's outputs are then undefined.
// ------------------------------------------------------------------------------------------------

struct TmaScatterSmem {
    uint32_t key[2][kRankTile];
    uint32_t val[2][kRankTile];
    uint32_t wcnt[kRankWarps][256];
    uint32_t tstart[256];
    uint32_t goff[256];
    unsigned long long bar[2];
    uint32_t stop;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Waits for the phase `parity` of the mbarrier, at most `limit` polls.  With the default limit a
// poll is try_wait (the thread may be suspended until the phase completes or a hardware time limit
// passes); a smaller limit (PERC_OPT_SPIN_LIMIT) polls with test_wait, which never suspends, so that
// the wait can run out before a copy lands.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, uint32_t limit)
{
    const bool suspend = limit >= kSpinLimit;
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        if (suspend)
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_u32(bar)), "r"(parity)
                : "memory");
        else
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(smem_u32(bar)), "r"(parity)
                : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kRankThreads, 2)
k_rank_scatter_tma(int pass, uint32_t N, uint32_t T, uint32_t S, const uint32_t *__restrict__ kin,
                   const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                   uint32_t *__restrict__ rank_out, const uint32_t *__restrict__ hist, int *status,
                   uint32_t spin_limit)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TmaScatterSmem &S_ = *reinterpret_cast<TmaScatterSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t total = T * S;
    const uint32_t shift = 8u * pass;
    const bool last = pass == 3;
    const uint32_t lanes_below = (1u << lane) - 1u;

    auto issue = [&](uint32_t w, int b) {  // thread 0: bring work item w into buffer b
        const uint32_t s = w / T, tile = w % T;
        const uint32_t n = min(static_cast<uint32_t>(kRankTile), N - tile * kRankTile);
        const size_t off = size_t(s) * N + size_t(tile) * kRankTile;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&S_.bar[b], 2u * n * 4u);
        bulk_load(S_.key[b], kin + off, n * 4u, &S_.bar[b]);
        bulk_load(S_.val[b], vin + off, n * 4u, &S_.bar[b]);
    };

    if (threadIdx.x == 0) {
        mbar_init(&S_.bar[0], 1u);
        mbar_init(&S_.bar[1], 1u);
        S_.stop = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t w = blockIdx.x;
    if (threadIdx.x == 0 && w < total) issue(w, 0);
    uint32_t use[2] = {0u, 0u};
    for (int it = 0; w < total; w += gridDim.x, ++it) {
        const int b = it & 1;
        const uint32_t s = w / T, tile = w % T;
        const uint32_t tile_n = min(static_cast<uint32_t>(kRankTile), N - tile * kRankTile);
        const size_t row = size_t(s) * N;
        for (int d = threadIdx.x; d < kRankWarps * 256; d += kRankThreads) (&S_.wcnt[0][0])[d] = 0u;
        if (threadIdx.x < 256) S_.goff[threadIdx.x] = hist[(size_t(s) * 256 + threadIdx.x) * T + tile];
        // the other buffer was released by the barrier that ended the previous iteration
        const bool next = w + gridDim.x < total;
        if (threadIdx.x == 0 && next) issue(w + gridDim.x, b ^ 1);
        if (!mbar_wait(&S_.bar[b], use[b] & 1u, spin_limit)) {
            set_status(status, PERC_ETIMEOUT);
            S_.stop = 1u;
        }
        __syncthreads();
        if (S_.stop) {
            // drain: the copy into this buffer (whose wait gave up) and the one already issued into
            // the other must land before the CTA goes away.  If a drain wait runs out as well, the
            // status word keeps PERC_ETIMEOUT (the first error) and the launch's results are void.
            if (threadIdx.x == 0) {
                bool ok = mbar_wait(&S_.bar[b], use[b] & 1u, kSpinLimit);
                if (next) ok = mbar_wait(&S_.bar[b ^ 1], use[b ^ 1] & 1u, kSpinLimit) && ok;
                if (!ok) set_status(status, PERC_ETIMEOUT);
            }
            __syncthreads();
            break;
        }
        ++use[b];
        uint32_t key[kRankItems], val[kRankItems], pos[kRankItems], dig[kRankItems];
#pragma unroll
        for (int k = 0; k < kRankItems; ++k) {
            const uint32_t e = warp * (32 * kRankItems) + k * 32 + lane;  // element inside the tile
            const bool valid = e < tile_n;
            const uint32_t kk = valid ? S_.key[b][e] : 0u;
            const uint32_t vv = valid ? S_.val[b][e] : 0u;
            const uint32_t d = valid ? ((kk >> shift) & 255u) : 256u;
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
            if (!valid) peers = ~peers;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t bb = __ballot_sync(0xffffffffu, (d >> q) & 1u);
                peers &= ((d >> q) & 1u) ? bb : ~bb;
            }
            const uint32_t leader = __ffs(peers) - 1;
            const uint32_t base = valid ? S_.wcnt[warp][d] : 0u;
            __syncwarp();
            if (valid && lane == static_cast<int>(leader)) S_.wcnt[warp][d] = base + __popc(peers);
            __syncwarp();
            key[k] = kk;
            val[k] = vv;
            pos[k] = base + __popc(peers & lanes_below);
            dig[k] = d;
        }
        __syncthreads();
        if (threadIdx.x < 256) {
            const uint32_t d = threadIdx.x;
            uint32_t run = 0;
#pragma unroll 4
            for (int ww = 0; ww < kRankWarps; ++ww) {
                const uint32_t cnt = S_.wcnt[ww][d];
                S_.wcnt[ww][d] = run;
                run += cnt;
            }
            S_.tstart[d] = run;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t v[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                v[q] = S_.tstart[lane * 8 + q];
                sum += v[q];
            }
            uint32_t x = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            uint32_t run = x - sum;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                S_.tstart[lane * 8 + q] = run;
                run += v[q];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kRankItems; ++k) {  // stage in digit order, in the buffer just read
            const uint32_t d = dig[k];
            if (d < 256u) {
                const uint32_t lp = S_.tstart[d] + S_.wcnt[warp][d] + pos[k];
                S_.key[b][lp] = key[k];
                S_.val[b][lp] = val[k];
            }
        }
        __syncthreads();
        for (uint32_t lp = threadIdx.x; lp < tile_n; lp += kRankThreads) {
            const uint32_t kk = S_.key[b][lp];
            const uint32_t d = (kk >> shift) & 255u;
            const uint32_t dst = S_.goff[d] + (lp - S_.tstart[d]);
            const uint32_t vv = S_.val[b][lp];
            vout[row + dst] = vv;
            if (last)
                rank_out[row + vv] = dst;
            else
                kout[row + dst] = kk;
        }
        __syncthreads();  // buffer b is free for the copy issued in the next iteration
    }
    // every copy a CTA issues is for a work item it consumes, so none is in flight at exit
}

// ------------------------------------------------------------------------------------------------
// Bucket path (L^5 <= kBucketBigMaxN, which covers L <= 40).  The keys are uniform 32-bit values, so
// their top B bits split a seed's sites into 2^B buckets -- of about 512 sites up to L = 24, and of
// up to about 6,400 (B = 14) above, sorted by k_rank_bsort_big -- and every bucket is then sorted on
// its own, in shared memory:
//   k_rank_bcount  per tile of kBTile sites: keys drawn, a shared-memory histogram of their buckets,
//                  added into the seed's bucket counts (one global atomic per bucket and tile);
//   k_rank_scan    exclusive scan of each seed's counts -> bucket starts (copied into the cursors);
//   k_rank_bplace  per tile: keys drawn and kept in shared memory with their offsets among the
//                  tile's keys of the same bucket, each bucket's share of the tile reserved with one
//                  atomicAdd on its cursor, every (key, site) record written into its bucket;
//   k_rank_bsort   per bucket: its records into shared memory, a counting sort on the next
//                  kSubBits key bits (about one record per sub-bucket), an insertion sort by
//                  (key, site) inside each sub-bucket, then perm and rank written.
// Ranking only a prefix (perc_rank_prefix) places and sorts only the buckets up to the cut, the
// first bucket whose end reaches the K sites asked for.  While counting, k_rank_bcount also lists
// the sites of the buckets up to stage_last -- where about K + 8 sqrt(K) + 64 keys are expected to
// end -- at the end of the seed's record row, so that k_rank_bplace draws the keys of those sites
// only instead of every key of the order a second time.  The exact counts decide
// the cut; a cut past the staged buckets, or staged records that would not fit in half a row, sends
// k_rank_bplace back to drawing the keys (same result).
// Records reach a bucket in no fixed order; the bucket sort orders them completely by (key, site),
// so the result is the same order as the radix path's.  A bucket larger than kBCap (never seen:
// about 512 sites are expected, and a Poisson count that exceeds 1536 has probability far below
// 1e-100) is ordered by counting, for each record, the records before it: slow, exact at any size.
// ------------------------------------------------------------------------------------------------
constexpr uint32_t kBTileItems = 32;
constexpr uint32_t kBTile = kRankThreads * kBTileItems;  // 16384 sites per tile
constexpr uint32_t kBucketMaxBits = 14;
constexpr uint64_t kBucketMaxN = uint64_t(512) << kBucketMaxBits;  // 8,388,608 sites: small buckets
constexpr uint64_t kBucketBigMaxN = uint64_t(6400) << kBucketMaxBits;  // 104,857,600 sites (L <= 40)
constexpr uint32_t kBCap = 1536;
constexpr uint32_t kSubBits = 9;
constexpr uint32_t kSub = 1u << kSubBits;
constexpr uint32_t kBSortThreads = 256;

// Bucket bits B: the smallest with N / 2^B <= 512 (at most kBucketMaxBits).
__host__ __device__ inline uint32_t bucket_bits(uint64_t N)
{
    uint32_t b = 0;
    while (b < kBucketMaxBits && (N >> b) > 512u) ++b;
    return b;
}
// Counters per seed: 2^B rounded up to a multiple of 4 (the scan reads four at a time).
__host__ __device__ inline uint32_t bucket_row(uint32_t B) { return (1u << B) < 4u ? 4u : (1u << B); }

__device__ __forceinline__ uint32_t bucket_of(uint32_t key, uint32_t B) { return B ? key >> (32u - B) : 0u; }

// Staging of the prefix ranking: up to N / 2 site indices (32-bit) at the end of a seed's record
// row (the placed records of a staged seed, at most as many, end before them).
constexpr uint32_t kNoStage = 0xFFFFFFFFu;
static_assert(kBTileItems == 32, "k_rank_bcount keeps round k's ballot in lane k");
__host__ __device__ inline uint32_t stage_cap(uint32_t N) { return N / 2u; }

// Last bucket staged for a prefix of K sites: the one where K + 8 sqrt(K) + 64 keys are expected to
// end (a shorter count than K there has probability below 1e-15), or kNoStage when that many
// records would not fit the staging half of the row.
__device__ __forceinline__ uint32_t stage_last(uint32_t N, uint32_t B, uint32_t K)
{
    const uint64_t t = uint64_t(K) + 8u * static_cast<uint64_t>(sqrtf(static_cast<float>(K))) + 64u;
    if (t > stage_cap(N)) return kNoStage;
    const uint64_t b = (t << B) / N;
    return static_cast<uint32_t>(b < (1u << B) - 1u ? b : (1u << B) - 1u);
}

__device__ __forceinline__ uint32_t *stage_row(uint2 *recs, uint32_t N, uint32_t s)
{
    return reinterpret_cast<uint32_t *>(recs + size_t(s) * N) + (2u * N - stage_cap(N));
}

// Bucket counts of every key; with share (perc_rank_prefix) also the list of the sites whose keys
// fall in the buckets up to stage_last, at stage_row(recs, N, s), their number in stage_n[s].
__global__ void __launch_bounds__(kRankThreads)
k_rank_bcount(uint32_t N, uint32_t B, const uint64_t *__restrict__ seeds, uint32_t *__restrict__ counts,
              const uint32_t *__restrict__ share, uint32_t per_seed, uint2 *__restrict__ recs,
              uint32_t *__restrict__ stage_n)
{
    extern __shared__ uint32_t bh[];  // [2^B]
    __shared__ uint32_t wbase[kRankWarps];
    __shared__ uint32_t tile_base, tile_tot;
    const uint32_t s = blockIdx.y, nb = 1u << B;
    const uint32_t last = share ? stage_last(N, B, prefix_sites(N, per_seed ? share[s] : share[0])) : kNoStage;
    const bool stage = last != kNoStage;  // the same for the whole block
    for (uint32_t b = threadIdx.x; b < nb; b += kRankThreads) bh[b] = 0u;
    __syncthreads();
    const uint64_t seed = seeds[s];
    const uint32_t e0 = blockIdx.x * kBTile;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t mine = 0u;  // lane k: which lanes of the warp stage their key of round k
#pragma unroll 4
    for (uint32_t k = 0; k < kBTileItems; ++k) {
        const uint32_t e = e0 + k * kRankThreads + threadIdx.x;
        bool keep = false;
        if (e < N) {
            const uint32_t b = bucket_of(site_key(seed, e), B);
            atomicAdd(&bh[b], 1u);
            keep = b <= last;
        }
        if (stage) {
            const uint32_t m = __ballot_sync(0xffffffffu, keep);
            if (lane == k) mine = m;
        }
    }
    __syncthreads();
    uint32_t *row = counts + size_t(s) * bucket_row(B);
    for (uint32_t b = threadIdx.x; b < nb; b += kRankThreads)
        if (bh[b]) atomicAdd(row + b, bh[b]);
    if (!stage) return;
    // the tile's staged sites: warp-major, then round, then lane; one reservation a tile
    const uint32_t c = __popc(mine);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= static_cast<uint32_t>(o)) incl += y;
    }
    if (lane == 31u) wbase[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kRankWarps; ++w) {
            const uint32_t v = wbase[w];
            wbase[w] = t;
            t += v;
        }
        tile_tot = t;
        tile_base = t ? atomicAdd(stage_n + s, t) : 0u;
    }
    __syncthreads();
    const uint32_t cap = stage_cap(N);
    if (tile_tot == 0u || tile_base + tile_tot > cap) return;  // nothing, or past the staging area
    uint32_t *stg = stage_row(recs, N, s);
    const uint32_t wb = tile_base + wbase[warp], excl = incl - c;
#pragma unroll 4
    for (uint32_t k = 0; k < kBTileItems; ++k) {
        const uint32_t m = __shfl_sync(0xffffffffu, mine, k), off = __shfl_sync(0xffffffffu, excl, k);
        if ((m >> lane) & 1u) stg[wb + off + __popc(m & ((1u << lane) - 1u))] = e0 + k * kRankThreads + threadIdx.x;
    }
}

// cut (nullable): per seed the last bucket to place (perc_rank_prefix); later buckets are skipped.
// stage_n (nullable, with cut and share): a seed whose cut lies within its staged buckets, and
// whose staged sites all fit, draws the keys of its staged sites only; any other draws every key.
// Tiles are taken in steps of gridDim.x.
__global__ void __launch_bounds__(kRankThreads)
k_rank_bplace(uint32_t N, uint32_t B, const uint64_t *__restrict__ seeds, uint32_t *__restrict__ cursors,
              uint2 *__restrict__ recs, const uint32_t *__restrict__ cut, const uint32_t *__restrict__ share,
              uint32_t per_seed, const uint32_t *__restrict__ stage_n)
{
    // shared: [2^B] bucket counts of the tile, then the tile's first place in each bucket; the tile's
    // keys; each key's offset among the tile's keys of its bucket (one shared atomic a key)
    extern __shared__ uint32_t bh[];
    uint32_t *keys = bh + (1u << B);
    uint16_t *loc = reinterpret_cast<uint16_t *>(keys + kBTile);
    const uint32_t s = blockIdx.y, nb = 1u << B;
    const uint32_t last = cut ? cut[s] : nb - 1u;
    bool staged = false;
    uint32_t M = 0u;
    if (stage_n && cut && share) {
        const uint32_t sl = stage_last(N, B, prefix_sites(N, per_seed ? share[s] : share[0]));
        M = stage_n[s];
        staged = sl != kNoStage && last <= sl && M <= stage_cap(N);
    }
    const uint32_t tiles = ((staged ? M : N) + kBTile - 1u) / kBTile;
    const uint32_t *stg = stage_row(recs, N, s);
    uint2 *row = recs + size_t(s) * N;
    const uint64_t seed = seeds[s];
    uint32_t *cur = cursors + size_t(s) * bucket_row(B);
    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        for (uint32_t b = threadIdx.x; b < nb; b += kRankThreads) bh[b] = 0u;
        __syncthreads();
        const uint32_t e0 = tile * kBTile;
        if (staged) {
#pragma unroll 4
            for (uint32_t k = 0; k < kBTileItems; ++k) {
                const uint32_t j = k * kRankThreads + threadIdx.x, e = e0 + j;
                if (e < M) {
                    const uint32_t key = site_key(seed, __ldg(stg + e)), b = bucket_of(key, B);
                    keys[j] = key;
                    if (b <= last) loc[j] = static_cast<uint16_t>(atomicAdd(&bh[b], 1u));
                }
            }
        } else {
#pragma unroll 4
            for (uint32_t k = 0; k < kBTileItems; ++k) {
                const uint32_t j = k * kRankThreads + threadIdx.x, e = e0 + j;
                if (e < N) {
                    const uint32_t key = site_key(seed, e), b = bucket_of(key, B);
                    keys[j] = key;
                    if (b <= last) loc[j] = static_cast<uint16_t>(atomicAdd(&bh[b], 1u));
                }
            }
        }
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < nb; b += kRankThreads)
            if (bh[b]) bh[b] = atomicAdd(cur + b, bh[b]);  // this tile's first place in bucket b
        __syncthreads();
        if (staged) {
#pragma unroll 4
            for (uint32_t k = 0; k < kBTileItems; ++k) {
                const uint32_t j = k * kRankThreads + threadIdx.x, e = e0 + j;
                if (e < M) {
                    const uint32_t key = keys[j], b = bucket_of(key, B);
                    if (b <= last) row[bh[b] + loc[j]] = make_uint2(key, __ldg(stg + e));
                }
            }
        } else {
#pragma unroll 4
            for (uint32_t k = 0; k < kBTileItems; ++k) {
                const uint32_t j = k * kRankThreads + threadIdx.x, e = e0 + j;
                if (e < N) {
                    const uint32_t key = keys[j], b = bucket_of(key, B);
                    if (b <= last) row[bh[b] + loc[j]] = make_uint2(key, e);
                }
            }
        }
        __syncthreads();  // bh is reset for the next tile
    }
}

// Per seed of one order block (side L, num_seeds rows of L^5 sites from perm_base), the largest
// share of the samples whose order is a row of that block (shares zeroed by the caller).
__global__ void __launch_bounds__(256) k_prefix_shares(const perc_sample *__restrict__ samples, uint32_t num,
                                                       const uint32_t *__restrict__ bracket, const uint32_t *perm_base,
                                                       uint32_t L, uint32_t num_seeds, uint32_t *__restrict__ shares)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= num) return;
    const perc_sample smp = samples[k];
    if (smp.L != L || smp.perm < perm_base) return;
    const uint64_t N = num_sites(L), off = static_cast<uint64_t>(smp.perm - perm_base);  // in sites
    if (off % N != 0u || off / N >= num_seeds) return;
    atomicMax(shares + off / N, bracket_share(L, bracket[2 * size_t(k)], bracket[2 * size_t(k) + 1]));
}

// perc_rank_prefix: per seed the first bucket whose end reaches prefix_sites(N, *share) sites (the
// starts are the exclusive scan of the bucket counts), one thread a seed.
__global__ void __launch_bounds__(256) k_bucket_cut(uint32_t N, uint32_t B, uint32_t S,
                                                    const uint32_t *__restrict__ starts,
                                                    const uint32_t *__restrict__ share, uint32_t per_seed,
                                                    uint32_t *__restrict__ cut)
{
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const uint32_t nb = 1u << B, K = prefix_sites(N, per_seed ? share[s] : share[0]);
    const uint32_t *st = starts + size_t(s) * bucket_row(B);
    uint32_t lo = 0u, hi = nb - 1u;  // the last bucket ends at N >= K
    while (lo < hi) {
        const uint32_t m = lo + (hi - lo) / 2u;
        const uint32_t end = m + 1u < nb ? st[m + 1u] : N;
        if (end >= K)
            hi = m;
        else
            lo = m + 1u;
    }
    cut[s] = lo;
}

// The largest upper bracket end as a share of its sample's lattice, in units of 2^-24 rounded up
// (one block of 1024 threads).  A bracket that perc_nstar would not use (lo < 1, lo > hi, hi > N)
// or an invalid side counts as the whole lattice.
__global__ void __launch_bounds__(1024) k_prefix_share(const perc_sample *__restrict__ samples,
                                                       const uint32_t *__restrict__ bracket, uint32_t num,
                                                       uint32_t *__restrict__ share)
{
    __shared__ uint32_t wmax[32];
    uint32_t m = 0u;
    for (uint32_t k = threadIdx.x; k < num; k += blockDim.x)
        m = max(m, bracket_share(samples[k].L, bracket[2 * size_t(k)], bracket[2 * size_t(k) + 1]));
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31u) == 0u) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32u) {
        uint32_t v = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0u;
        v = __reduce_max_sync(0xffffffffu, v);
        if (threadIdx.x == 0u) *share = min(v, 1u << 24);
    }
}

// (key, site) order of two records
__device__ __forceinline__ bool rec_less(uint2 a, uint2 b) { return a.x < b.x || (a.x == b.x && a.y < b.y); }

struct BSortSmem {
    uint2 in[kBCap];
    uint2 out[kBCap];
    uint32_t start[kSub + 1];  // sub-bucket starts (exclusive scan of the counts), start[kSub] = size
    uint32_t cur[kSub];
    uint32_t wsum[kBSortThreads / 32];
};

__global__ void __launch_bounds__(kBSortThreads)
k_rank_bsort(uint32_t N, uint32_t B, const uint32_t *__restrict__ starts, const uint2 *__restrict__ recs,
             uint32_t *__restrict__ perm, uint32_t *__restrict__ rank_out, const uint32_t *__restrict__ cut)
{
    __shared__ BSortSmem S_;
    const uint32_t s = blockIdx.y, b = blockIdx.x, nb = 1u << B;
    if (cut && b > cut[s]) return;  // past the prefix (perc_rank_prefix)
    const uint32_t *st = starts + size_t(s) * bucket_row(B);
    const uint32_t lo = st[b], hi = b + 1u < nb ? st[b + 1u] : N, n = hi - lo;
    const uint2 *in = recs + size_t(s) * N + lo;
    uint32_t *po = perm + size_t(s) * N;
    uint32_t *ro = rank_out + size_t(s) * N;
    if (n > kBCap) {  // exact at any size: each record's place is the number of records before it
        for (uint32_t j = threadIdx.x; j < n; j += kBSortThreads) {
            const uint2 r = in[j];
            uint32_t before = 0;
            for (uint32_t i = 0; i < n; ++i) before += rec_less(in[i], r) ? 1u : 0u;
            po[lo + before] = r.y;
            ro[r.y] = lo + before;
        }
        return;
    }
    const uint32_t shift = 32u - B - kSubBits;
    for (uint32_t q = threadIdx.x; q < kSub; q += kBSortThreads) S_.cur[q] = 0u;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n; j += kBSortThreads) {
        const uint2 r = in[j];
        S_.in[j] = r;
        atomicAdd(&S_.cur[(r.x >> shift) & (kSub - 1u)], 1u);
    }
    __syncthreads();
    // exclusive scan of the kSub counts: four consecutive per thread, then a block scan of the sums
    constexpr uint32_t per = kSub / kBSortThreads;
    uint32_t v[per], sum = 0;
#pragma unroll
    for (uint32_t q = 0; q < per; ++q) {
        v[q] = S_.cur[threadIdx.x * per + q];
        sum += v[q];
    }
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    if (lane == 31u) S_.wsum[warp] = x;
    __syncthreads();
    uint32_t run = x - sum;
    for (uint32_t w = 0; w < warp; ++w) run += S_.wsum[w];
#pragma unroll
    for (uint32_t q = 0; q < per; ++q) {
        S_.start[threadIdx.x * per + q] = run;
        S_.cur[threadIdx.x * per + q] = run;
        run += v[q];
    }
    if (threadIdx.x == 0) S_.start[kSub] = n;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n; j += kBSortThreads) {
        const uint2 r = S_.in[j];
        S_.out[atomicAdd(&S_.cur[(r.x >> shift) & (kSub - 1u)], 1u)] = r;
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < kSub; q += kBSortThreads) {  // insertion sort of each sub-bucket
        const uint32_t a = S_.start[q], z = S_.start[q + 1u];
        for (uint32_t j = a + 1u; j < z; ++j) {
            const uint2 r = S_.out[j];
            uint32_t i = j;
            while (i > a && rec_less(r, S_.out[i - 1u])) {
                S_.out[i] = S_.out[i - 1u];
                --i;
            }
            S_.out[i] = r;
        }
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n; j += kBSortThreads) {
        const uint32_t site = S_.out[j].y;
        po[lo + j] = site;
        ro[site] = lo + j;
    }
}

// Large buckets (kBucketMaxN < L^5 <= kBucketBigMaxN: 2^14 buckets of up to about 6,400 sites):
// one CTA of 1024 threads a bucket, its records read twice from global memory (a counting pass on
// the next sub_bits key bits, then a placing pass into shared memory), an insertion sort inside each
// sub-bucket (about one record each), perm and rank written.  Shared memory (dynamic): cap records,
// then 2^sub_bits + 1 sub-bucket starts and 2^sub_bits cursors.  A bucket over cap records is
// ordered by counting the records before each (exact at any size).
constexpr uint32_t kBSortBigThreads = 1024;

__host__ __device__ inline void big_bucket_shape(uint64_t N, uint32_t B, uint32_t &sub_bits, uint32_t &cap)
{
    const uint64_t mean = (N + (uint64_t(1) << B) - 1) >> B;
    sub_bits = 9;
    while ((uint64_t(1) << sub_bits) < mean) ++sub_bits;  // about one record a sub-bucket
    cap = (sub_bits <= 11 ? 4u : 2u) << sub_bits;            // 2.5 to 8 times the mean
}

__host__ __device__ inline size_t big_bucket_smem(uint32_t sub_bits, uint32_t cap)
{
    return size_t(cap) * sizeof(uint2) + (size_t(2) * (1u << sub_bits) + 1) * sizeof(uint32_t);
}

__global__ void __launch_bounds__(kBSortBigThreads)
k_rank_bsort_big(uint32_t N, uint32_t B, uint32_t sub_bits, uint32_t cap, const uint32_t *__restrict__ starts,
                 const uint2 *__restrict__ recs, uint32_t *__restrict__ perm, uint32_t *__restrict__ rank_out,
                 const uint32_t *__restrict__ cut)
{
    if (cut && blockIdx.x > cut[blockIdx.y]) return;  // past the prefix (perc_rank_prefix)
    extern __shared__ __align__(16) unsigned char bs_raw[];
    uint2 *out = reinterpret_cast<uint2 *>(bs_raw);
    const uint32_t S = 1u << sub_bits;
    uint32_t *start = reinterpret_cast<uint32_t *>(out + cap);  // [S + 1]
    uint32_t *cur = start + S + 1;                              // [S]
    __shared__ uint32_t wsum[kBSortBigThreads / 32];
    const uint32_t s = blockIdx.y, b = blockIdx.x, nb = 1u << B;
    const uint32_t *st = starts + size_t(s) * bucket_row(B);
    const uint32_t lo = st[b], hi = b + 1u < nb ? st[b + 1u] : N, n = hi - lo;
    const uint2 *in = recs + size_t(s) * N + lo;
    uint32_t *po = perm + size_t(s) * N;
    uint32_t *ro = rank_out + size_t(s) * N;
    if (n > cap) {
        for (uint32_t j = threadIdx.x; j < n; j += kBSortBigThreads) {
            const uint2 r = in[j];
            uint32_t before = 0;
            for (uint32_t i = 0; i < n; ++i) before += rec_less(in[i], r) ? 1u : 0u;
            po[lo + before] = r.y;
            ro[r.y] = lo + before;
        }
        return;
    }
    const uint32_t shift = 32u - B - sub_bits;
    for (uint32_t q = threadIdx.x; q < S; q += kBSortBigThreads) cur[q] = 0u;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n; j += kBSortBigThreads) atomicAdd(&cur[(in[j].x >> shift) & (S - 1u)], 1u);
    __syncthreads();
    // exclusive scan of the S counts: a contiguous run per thread, then a block scan of the sums
    const uint32_t per = (S + kBSortBigThreads - 1) / kBSortBigThreads;
    const uint32_t q0 = min(S, threadIdx.x * per), q1 = min(S, q0 + per);
    uint32_t sum = 0;
    for (uint32_t q = q0; q < q1; ++q) sum += cur[q];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<uint32_t>(o)) x += y;
    }
    if (lane == 31u) wsum[warp] = x;
    __syncthreads();
    uint32_t run = x - sum;
    for (uint32_t w = 0; w < warp; ++w) run += wsum[w];
    for (uint32_t q = q0; q < q1; ++q) {
        const uint32_t c = cur[q];
        start[q] = run;
        cur[q] = run;
        run += c;
    }
    if (threadIdx.x == 0) start[S] = n;
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n; j += kBSortBigThreads) {
        const uint2 r = in[j];
        out[atomicAdd(&cur[(r.x >> shift) & (S - 1u)], 1u)] = r;
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < S; q += kBSortBigThreads) {  // insertion sort of each sub-bucket
        const uint32_t a = start[q], z = start[q + 1u];
        for (uint32_t j = a + 1u; j < z; ++j) {
            const uint2 r = out[j];
            uint32_t i = j;
            while (i > a && rec_less(r, out[i - 1u])) {
                out[i] = out[i - 1u];
                --i;
            }
            out[i] = r;
        }
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < n; j += kBSortBigThreads) {
        const uint32_t site = out[j].y;
        po[lo + j] = site;
        ro[site] = lo + j;
    }
}

}  // namespace perc

using namespace perc;

// share (nullable): rank only the first buckets of each order, up to prefix_sites(N, *share) sites
// (bucket path; the radix path ranks every site).
static int rank_impl(uint32_t L, const uint64_t *seeds, uint32_t num_seeds, const uint32_t *share, bool per_seed,
                     uint32_t *perm, uint32_t *rank, void *workspace, size_t ws_bytes, void *stream_)
{
    if (L < 1 || L > PERC_MAX_L || num_seeds == 0 || !seeds || !perm || !rank || !workspace)
        return PERC_EINVAL;
    if (ws_bytes < rank_workspace_bytes(L, num_seeds)) return PERC_EWORKSPACE;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    const uint64_t N = num_sites(L);
    const uint32_t T = rank_tiles(N);
    const uint32_t chunk = rank_chunk(N, num_seeds);
    char *ws = static_cast<char *>(workspace) + 256;
    uint32_t *a_keys = reinterpret_cast<uint32_t *>(ws);
    uint32_t *a_vals = a_keys + size_t(chunk) * N;
    // the histograms start 16-byte aligned: k_rank_scan reads and writes them four at a time
    uint32_t *hist = reinterpret_cast<uint32_t *>((reinterpret_cast<uintptr_t>(a_vals + size_t(chunk) * N) + 15) &
                                                  ~uintptr_t(15));

    // attributes and the resident CTA count are per device (set and cached once per device)
    uint32_t tma_ctas = 0;
    if (ensure_smem_attr(kAttrRankScatter, reinterpret_cast<const void *>(k_rank_scatter), sizeof(ScatterSmem)) !=
            PERC_OK ||
        ensure_smem_attr(kAttrRankScatterTma, reinterpret_cast<const void *>(k_rank_scatter_tma),
                         sizeof(TmaScatterSmem)) != PERC_OK ||
        resident_ctas(kAttrRankScatterTma, reinterpret_cast<const void *>(k_rank_scatter_tma), kRankThreads,
                      sizeof(TmaScatterSmem), tma_ctas) != PERC_OK)
        return PERC_ECUDA;
    // bulk-async tile loads need 16-byte aligned sources: rows of a multiple of 4 keys, and perm and
    // rank (which passes 2 and 3 read) starting on 16-byte boundaries; otherwise the plain scatter
    const bool aligned = ((reinterpret_cast<uintptr_t>(perm) | reinterpret_cast<uintptr_t>(rank) |
                           reinterpret_cast<uintptr_t>(workspace)) & 15u) == 0u;
    const bool use_tma = (N % 4u) == 0u && aligned && env_int_rank("PERC_RANK_TMA", 1) != 0;
    int *status = static_cast<int *>(workspace);  // keeps the first error since the last perc_check
    if (N <= kBucketBigMaxN && env_int_rank("PERC_RANK_BUCKET", 1) != 0) {
        // bucket path: the records (8 bytes a site) take the radix path's key and value buffers, the
        // bucket counts and cursors its histogram area
        const uint32_t Bb = bucket_bits(N), nb = 1u << Bb, row = bucket_row(Bb);
        const uint32_t Tb = static_cast<uint32_t>((N + kBTile - 1) / kBTile);
        const size_t smem_count = size_t(nb) * 4, smem_place = size_t(nb) * 4 + size_t(kBTile) * 6;
        const bool big = N > kBucketMaxN;
        uint32_t sub_bits = 0, cap = 0;
        if (big) big_bucket_shape(N, Bb, sub_bits, cap);
        const size_t smem_big = big ? big_bucket_smem(sub_bits, cap) : 0;
        if (ensure_smem_attr(kAttrRankBCount, reinterpret_cast<const void *>(k_rank_bcount), smem_count) != PERC_OK ||
            ensure_smem_attr(kAttrRankBPlace, reinterpret_cast<const void *>(k_rank_bplace), smem_place) != PERC_OK ||
            (big && ensure_smem_attr(kAttrRankBSortBig, reinterpret_cast<const void *>(k_rank_bsort_big), smem_big) !=
                        PERC_OK))
            return PERC_ECUDA;
        uint2 *recs = reinterpret_cast<uint2 *>(a_keys);  // a_keys then a_vals: chunk * N * 8 bytes
        // counts, staged record counts (prefix; padded to 16 bytes), cursors and (prefix) the per-seed
        // last bucket: within the radix histogram area
        const size_t pad = (size_t(chunk) + 3u) & ~size_t(3);
        if (size_t(2) * chunk * row + pad + chunk > size_t(256) * T * chunk) return PERC_EINVAL;
        // prefix: records staged while counting (PERC_RANK_STAGE=0 turns it off), and a grid of about
        // eight CTAs an SM over the chunk's seeds that takes the staged tiles in steps
        const bool stage = share && env_int_rank("PERC_RANK_STAGE", 1) != 0;
        int dev = 0, sms = 0;
        if (share && (cudaGetDevice(&dev) != cudaSuccess ||
                      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess))
            return PERC_ECUDA;
        for (uint32_t s0 = 0; s0 < num_seeds; s0 += chunk) {
            const uint32_t S = min(chunk, num_seeds - s0);
            const size_t padS = (size_t(S) + 3u) & ~size_t(3);
            uint32_t *counts = hist, *stage_n = hist + size_t(S) * row, *cursors = stage_n + padS;
            uint32_t *cut = share ? cursors + size_t(S) * row : nullptr;
            const uint32_t *sh = share ? (per_seed ? share + s0 : share) : nullptr;
            if (cudaMemsetAsync(counts, 0, (size_t(S) * row + padS) * 4, stream) != cudaSuccess) return PERC_ECUDA;
            k_rank_bcount<<<dim3(Tb, S), kRankThreads, smem_count, stream>>>(
                uint32_t(N), Bb, seeds + s0, counts, stage ? sh : nullptr, per_seed ? 1u : 0u, recs, stage_n);
            k_rank_scan<<<S, 1024, 0, stream>>>(row, counts, cursors);
            if (cut)
                k_bucket_cut<<<(S + 255) / 256, 256, 0, stream>>>(uint32_t(N), Bb, S, counts, sh, per_seed ? 1u : 0u,
                                                                 cut);
            const uint32_t gx = share ? min(Tb, max(1u, (8u * uint32_t(sms) + S - 1u) / S)) : Tb;
            k_rank_bplace<<<dim3(gx, S), kRankThreads, smem_place, stream>>>(
                uint32_t(N), Bb, seeds + s0, cursors, recs, cut, sh, per_seed ? 1u : 0u, stage ? stage_n : nullptr);
            if (big)
                k_rank_bsort_big<<<dim3(nb, S), kBSortBigThreads, smem_big, stream>>>(
                    uint32_t(N), Bb, sub_bits, cap, counts, recs, perm + size_t(s0) * N, rank + size_t(s0) * N, cut);
            else
                k_rank_bsort<<<dim3(nb, S), kBSortThreads, 0, stream>>>(uint32_t(N), Bb, counts, recs,
                                                                       perm + size_t(s0) * N, rank + size_t(s0) * N,
                                                                       cut);
        }
        return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
    }
    for (uint32_t s0 = 0; s0 < num_seeds; s0 += chunk) {
        const uint32_t S = min(chunk, num_seeds - s0);
        const uint64_t *sd = seeds + s0;
        uint32_t *b_keys = rank + size_t(s0) * N;  // keys of passes 1-2, then the inverse order
        uint32_t *b_vals = perm + size_t(s0) * N;
        const dim3 grid(T, S);
        for (int pass = 0; pass < 4; ++pass) {
            // ping-pong: gen -> A, A -> B, B -> A, A -> (perm, rank)
            const uint32_t *kin = (pass == 2) ? b_keys : a_keys;
            const uint32_t *vin = (pass == 2) ? b_vals : a_vals;
            uint32_t *kout = (pass == 0 || pass == 2) ? a_keys : b_keys;
            uint32_t *vout = (pass == 0 || pass == 2) ? a_vals : b_vals;
            k_rank_hist<<<grid, kRankThreads, 0, stream>>>(pass, uint32_t(N), T, sd, kin, hist);
            k_rank_scan<<<S, 1024, 0, stream>>>(256u * T, hist, nullptr);
            if (pass > 0 && use_tma) {
                const uint32_t work = T * S;
                const uint32_t g = work < tma_ctas ? work : tma_ctas;
                k_rank_scatter_tma<<<g, kRankThreads, sizeof(TmaScatterSmem), stream>>>(
                    pass, uint32_t(N), T, S, kin, vin, kout, vout, b_keys, hist, status, spin_limit());
            } else {
                k_rank_scatter<<<grid, kRankThreads, sizeof(ScatterSmem), stream>>>(pass, uint32_t(N), T, sd, kin, vin,
                                                                                    kout, vout, b_keys, hist);
            }
        }
    }
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

extern "C" int perc_rank(uint32_t L, const uint64_t *seeds, uint32_t num_seeds, uint32_t *perm, uint32_t *rank,
                         void *workspace, size_t ws_bytes, void *stream)
{
    return rank_impl(L, seeds, num_seeds, nullptr, false, perm, rank, workspace, ws_bytes, stream);
}

extern "C" int perc_rank_prefix(uint32_t L, const uint64_t *seeds, uint32_t num_seeds, const uint32_t *share,
                                uint32_t *perm, uint32_t *rank, void *workspace, size_t ws_bytes, void *stream)
{
    if (!share) return PERC_EINVAL;
    return rank_impl(L, seeds, num_seeds, share, false, perm, rank, workspace, ws_bytes, stream);
}

extern "C" int perc_rank_prefix_seeds(uint32_t L, const uint64_t *seeds, uint32_t num_seeds, const uint32_t *shares,
                                      uint32_t *perm, uint32_t *rank, void *workspace, size_t ws_bytes, void *stream)
{
    if (!shares) return PERC_EINVAL;
    return rank_impl(L, seeds, num_seeds, shares, true, perm, rank, workspace, ws_bytes, stream);
}

extern "C" int perc_prefix_shares(const perc_sample *samples, uint32_t num_samples, const uint32_t *bracket,
                                  const uint32_t *perm, uint32_t L, uint32_t num_seeds, uint32_t *shares, void *stream_)
{
    if (!samples || !bracket || !perm || !shares || num_samples == 0 || num_seeds == 0 || L < 1 || L > PERC_MAX_L)
        return PERC_EINVAL;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    if (cudaMemsetAsync(shares, 0, size_t(num_seeds) * sizeof(uint32_t), stream) != cudaSuccess) return PERC_ECUDA;
    k_prefix_shares<<<(num_samples + 255) / 256, 256, 0, stream>>>(samples, num_samples, bracket, perm, L, num_seeds,
                                                                   shares);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}

extern "C" int perc_prefix_share(const perc_sample *samples, uint32_t num_samples, const uint32_t *bracket,
                                 uint32_t *share, void *stream)
{
    if (!samples || !bracket || !share || num_samples == 0) return PERC_EINVAL;
    k_prefix_share<<<1, 1024, 0, static_cast<cudaStream_t>(stream)>>>(samples, bracket, num_samples, share);
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}
