// perc_rank.cu -- the random site-addition order of the Newman--Ziff method (Methods,
// "Computational methods"), one per seed.
//
// The order of seed s sorts the sites ascending by (key_i, i), key_i = word 0 of
// Philox4x32-10(counter (i,0,0,0), key (s lo, s hi)).  It is built by a stable least-significant-
// digit radix sort of the 32-bit keys with the site index as payload: the input is in index order
// and every pass is stable, so equal keys stay in index order.  Four 8-bit passes, each
//   k_rank_hist    per-tile digit counts (pass 0 draws the keys itself, nothing is stored first),
//   k_rank_scan    exclusive scan per seed in digit-major order -> tile output offsets,
//   k_rank_scatter stable scatter: warp-level peer ranking with __match_any_sync,
// then k_rank_invert writes rank[perm[r]] = r.  Seeds are sorted in chunks that fit the workspace.
#include <cstdio>

#include "perc_common.cuh"

namespace perc {

constexpr int kRankThreads = 256;
constexpr int kRankItems = 8;
constexpr int kRankTile = kRankThreads * kRankItems;  // 2048 keys per tile
constexpr int kRankMaxChunk = 64;                     // seeds per chunk (upper bound)
constexpr size_t kRankChunkBytes = size_t(4) << 30;   // workspace aimed at per chunk

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
    return 256 + size_t(rank_chunk(N, num_seeds)) * rank_bytes_per_seed(N);
}

__global__ void __launch_bounds__(kRankThreads)
k_rank_hist(int pass, uint32_t N, uint32_t T, const uint64_t *__restrict__ seeds,
            const uint32_t *__restrict__ keys_in, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t h[256];
    const uint32_t s = blockIdx.y, tile = blockIdx.x;
    h[threadIdx.x] = 0;
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
    hist[(size_t(s) * 256 + threadIdx.x) * T + tile] = h[threadIdx.x];
}

// Exclusive scan of one seed's 256*T counters (digit-major), one block per seed.
__global__ void __launch_bounds__(1024) k_rank_scan(uint32_t T, uint32_t *__restrict__ hist)
{
    __shared__ uint32_t warp_sum[32];
    uint32_t *h = hist + size_t(blockIdx.x) * 256 * T;
    const uint32_t n = 256u * T;
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per;
    const uint32_t e = min(n, b + per);
    uint32_t local = 0;
    for (uint32_t i = b; i < e; ++i) local += h[i];
    // block-wide exclusive scan of `local`
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? warp_sum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sum[lane] = w;  // inclusive
    }
    __syncthreads();
    uint32_t run = x - local + (warp > 0 ? warp_sum[warp - 1] : 0u);
    for (uint32_t i = b; i < e; ++i) {
        const uint32_t c = h[i];
        h[i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(kRankThreads)
k_rank_scatter(int pass, uint32_t N, uint32_t T, const uint64_t *__restrict__ seeds,
               const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
               uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
               const uint32_t *__restrict__ hist, int write_keys)
{
    __shared__ uint32_t wcnt[kRankThreads / 32][256];
    __shared__ uint32_t goff[256];
    const uint32_t s = blockIdx.y, tile = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < (kRankThreads / 32) * 256; d += kRankThreads) (&wcnt[0][0])[d] = 0u;
    goff[threadIdx.x] = hist[(size_t(s) * 256 + threadIdx.x) * T + tile];
    __syncthreads();

    const uint64_t seed = pass == 0 ? seeds[s] : 0ull;
    const size_t row = size_t(s) * N;
    const uint32_t shift = 8u * pass;
    const uint32_t lanes_below = (1u << lane) - 1u;
    uint32_t key[kRankItems], val[kRankItems], pos[kRankItems], dig[kRankItems];
#pragma unroll
    for (int k = 0; k < kRankItems; ++k) {
        // element order inside the tile: warp-major, then round, then lane (the input order)
        const uint32_t e = tile * kRankTile + warp * (32 * kRankItems) + k * 32 + lane;
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
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t leader = __ffs(peers) - 1;
        const uint32_t base = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == static_cast<int>(leader)) wcnt[warp][d] = base + __popc(peers);
        __syncwarp();
        key[k] = kk;
        val[k] = vv;
        pos[k] = base + __popc(peers & lanes_below);
        dig[k] = d;
    }
    __syncthreads();
    {
        const uint32_t d = threadIdx.x;  // 256 threads, one digit each
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kRankThreads / 32; ++w) {
            const uint32_t c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRankItems; ++k) {
        const uint32_t d = dig[k];
        if (d < 256u) {
            const uint32_t dst = goff[d] + wcnt[warp][d] + pos[k];
            vout[row + dst] = val[k];
            if (write_keys) kout[row + dst] = key[k];
        }
    }
}

__global__ void k_rank_invert(uint32_t N, uint32_t S, const uint32_t *__restrict__ perm,
                              uint32_t *__restrict__ rank)
{
    const size_t total = size_t(N) * S;
    for (size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x; t < total;
         t += size_t(gridDim.x) * blockDim.x) {
        const size_t s = t / N;
        const uint32_t r = static_cast<uint32_t>(t - s * N);
        rank[s * N + __ldg(perm + t)] = r;
    }
}

}  // namespace perc

using namespace perc;

extern "C" int perc_rank(uint32_t L, const uint64_t *seeds, uint32_t num_seeds, uint32_t *perm,
                         uint32_t *rank, void *workspace, size_t ws_bytes, void *stream_)
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
    uint32_t *hist = a_vals + size_t(chunk) * N;

    for (uint32_t s0 = 0; s0 < num_seeds; s0 += chunk) {
        const uint32_t S = min(chunk, num_seeds - s0);
        const uint64_t *sd = seeds + s0;
        uint32_t *b_keys = rank + size_t(s0) * N;  // scratch until the final inversion
        uint32_t *b_vals = perm + size_t(s0) * N;
        const dim3 grid(T, S);
        for (int pass = 0; pass < 4; ++pass) {
            // ping-pong: gen -> A, A -> B, B -> A, A -> B (values only on the last pass)
            const uint32_t *kin = (pass == 2) ? b_keys : a_keys;
            const uint32_t *vin = (pass == 2) ? b_vals : a_vals;
            uint32_t *kout = (pass == 0 || pass == 2) ? a_keys : b_keys;
            uint32_t *vout = (pass == 0 || pass == 2) ? a_vals : b_vals;
            k_rank_hist<<<grid, kRankThreads, 0, stream>>>(pass, uint32_t(N), T, sd, kin, hist);
            k_rank_scan<<<S, 1024, 0, stream>>>(T, hist);
            k_rank_scatter<<<grid, kRankThreads, 0, stream>>>(pass, uint32_t(N), T, sd, kin, vin, kout,
                                                              vout, hist, pass != 3);
        }
        const size_t total = size_t(N) * S;
        const size_t want = (total + 255) / 256;
        const uint32_t blocks = static_cast<uint32_t>(want < size_t(148 * 64) ? want : size_t(148 * 64));
        k_rank_invert<<<blocks, 256, 0, stream>>>(uint32_t(N), S, b_vals, b_keys);
    }
    return cudaGetLastError() == cudaSuccess ? PERC_OK : PERC_ECUDA;
}
