/*
 * perc_oracle.c -- the oracle for exact 5D site percolation with complex neighborhoods.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It is a plain, slow, sequential CPU
 * implementation of what the GPU path computes, written from the paper, and it shares no code,
 * header, table or constant generator with the CUDA library.
 *
 * What it computes (Methods, "Computational methods"; Introduction for spanning):
 *   - coordination zones of the 5D simple cubic lattice (eq. z, eq. zeta; Table I z column);
 *   - the random site-addition order of one sample (the Newman--Ziff order), here keyed by the
 *     Philox4x32-10 counter-based generator (Salmon et al., SC'11) and ordered by (key, index);
 *   - the Newman--Ziff sweep: add the sites one at a time in that order and merge clusters with
 *     union-find, which gives, for every n, the largest cluster S_max(n) (eq. Pmax) and the first
 *     n at which a cluster touches both borders x1 = 0 and x1 = L-1 (the spanning cluster), or,
 *     as a variant of the spanning rule, both borders x_a = 0 and x_a = L-1 of another axis a, or
 *     of any axis;
 *   - independent cross-checks used only to pin the sweep: a breadth-first flood fill at a fixed
 *     n, and the bottleneck (minimax) path identity for the first spanning n;
 *   - the periodic-boundary variant: S_max(n) on the 5-torus and the first n at which a cluster
 *     wraps around it along one axis, with its own flood-fill cross-check;
 *   - the binomial convolution that turns S_max(n) into S_max(p).
 *
 * Readings of what the paper leaves open (all are stated here so a reader can check them):
 *   open boundaries (offsets leaving [0,L)^5 are dropped); spanning means touching x1 = 0 and
 *   x1 = L-1; site index i = (((x1*L+x2)*L+x3)*L+x4)*L+x5; key_i = word 0 of
 *   Philox4x32-10(counter = (i,0,0,0), key = (seed mod 2^32, seed / 2^32)); ties of keys are
 *   broken by ascending index.  n* = ORC_NEVER when no n spans.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_NEVER 0xFFFFFFFFu

/* ------------------------------------------------------------------------------------------ */
/* Coordination zones (eq. z, eq. zeta; Table I).  Zone i holds the lattice vectors v of the    */
/* 5D simple cubic lattice with |v|^2 = i.  For i <= 7 every component lies in {-2..2}.          */
/* ------------------------------------------------------------------------------------------ */

/* Writes the offsets of zone `zone` (1..7) as 5 int8 each into out (may be NULL); returns count. */
int orc_zone_offsets(int zone, int8_t *out)
{
    int cnt = 0;
    for (int a = -2; a <= 2; ++a)
        for (int b = -2; b <= 2; ++b)
            for (int c = -2; c <= 2; ++c)
                for (int d = -2; d <= 2; ++d)
                    for (int e = -2; e <= 2; ++e) {
                        if (a * a + b * b + c * c + d * d + e * e != zone)
                            continue;
                        if (out) {
                            int8_t *o = out + 5 * cnt;
                            o[0] = (int8_t)a; o[1] = (int8_t)b; o[2] = (int8_t)c;
                            o[3] = (int8_t)d; o[4] = (int8_t)e;
                        }
                        ++cnt;
                    }
    return cnt;
}

/* A neighborhood is a non-empty union of zones; bit (i-1) of mask selects zone i. */
int orc_mask_offsets(int mask, int8_t *out)
{
    int cnt = 0;
    for (int zone = 1; zone <= 7; ++zone)
        if (mask & (1 << (zone - 1)))
            cnt += orc_zone_offsets(zone, out ? out + 5 * cnt : NULL);
    return cnt;
}

/* z = sum of zone sizes (eq. z); zeta = sum of z_i * r_i with r_i = sqrt(i) (eq. zeta). */
void orc_mask_z_zeta(int mask, int *z, double *zeta)
{
    int zz = 0;
    double zt = 0.0;
    for (int zone = 1; zone <= 7; ++zone)
        if (mask & (1 << (zone - 1))) {
            int zi = orc_zone_offsets(zone, NULL);
            zz += zi;
            zt += zi * sqrt((double)zone);
        }
    *z = zz;
    *zeta = zt;
}

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64 multiplies   */
/* with the multipliers 0xD2511F53 and 0xCD9E8D57; the key is bumped by the Weyl constants     */
/* 0x9E3779B9 and 0xBB67AE85 before every round after the first.                                */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The per-site key of a sample: word 0 of Philox4x32-10 with counter (i,0,0,0). */
uint32_t orc_site_key(uint64_t seed, uint32_t i)
{
    uint32_t ctr[4] = {i, 0u, 0u, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}

/* ------------------------------------------------------------------------------------------ */
/* Site order of one sample: perm = indices sorted ascending by (key, index); rank = perm^-1.  */
/* The Newman--Ziff method adds the sites in a uniformly random order; this fixes that order.  */
/* ------------------------------------------------------------------------------------------ */
typedef struct { uint32_t key, idx; } orc_kv;

static int orc_kv_cmp(const void *a, const void *b)
{
    const orc_kv *x = (const orc_kv *)a, *y = (const orc_kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

uint64_t orc_num_sites(uint32_t L)
{
    return (uint64_t)L * L * L * L * L;
}

/* Fills perm[N] and rank[N] (N = L^5) for one seed.  Returns 0, or -1 on bad input / no memory. */
int orc_rank(uint32_t L, uint64_t seed, uint32_t *perm, uint32_t *rank)
{
    uint64_t N = orc_num_sites(L);
    if (L == 0 || N >= 0xFFFFFFFFull) return -1;
    orc_kv *kv = (orc_kv *)malloc(sizeof(orc_kv) * (size_t)N);
    if (!kv) return -1;
    for (uint64_t i = 0; i < N; ++i) {
        kv[i].key = orc_site_key(seed, (uint32_t)i);
        kv[i].idx = (uint32_t)i;
    }
    qsort(kv, (size_t)N, sizeof(orc_kv), orc_kv_cmp);
    for (uint64_t r = 0; r < N; ++r) {
        perm[r] = kv[r].idx;
        rank[kv[r].idx] = (uint32_t)r;
    }
    free(kv);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Lattice helpers.                                                                              */
/* ------------------------------------------------------------------------------------------ */
static void orc_coords(uint32_t L, uint32_t i, int x[5])
{
    for (int k = 4; k >= 0; --k) {
        x[k] = (int)(i % L);
        i /= L;
    }
}

/* Neighbor of i along offset v, or -1 when it leaves [0,L)^5 (open boundaries). */
static int64_t orc_neighbor(uint32_t L, const int x[5], const int8_t *v)
{
    int64_t j = 0;
    for (int k = 0; k < 5; ++k) {
        int y = x[k] + v[k];
        if (y < 0 || y >= (int)L) return -1;
        j = j * L + y;
    }
    return j;
}

/* ------------------------------------------------------------------------------------------ */
/* Newman--Ziff sweep (Methods, "Computational methods").  Sites are added in rank order; each   */
/* new site is merged with every already occupied neighbor by union-find (union by size, path   */
/* compression).  A cluster carries ten border flags: bit 2a (has a site with x_{a+1} = 0) and  */
/* bit 2a+1 (has a site with x_{a+1} = L-1), a = 0..4.  The spanning rule `span` is an axis     */
/* 0..4 (x1..x5: the cluster carries both flags of that axis) or ORC_SPAN_ANY (both flags of     */
/* some axis).  Adding one site can only make its own cluster spanning, so the first n at which  */
/* the new site's cluster spans is n*.  S_max is tracked after every addition.                   */
/* ------------------------------------------------------------------------------------------ */
#define ORC_SPAN_ANY 5u

static uint16_t orc_site_flags(uint32_t L, const int x[5])
{
    uint16_t f = 0;
    for (int a = 0; a < 5; ++a) {
        if (x[a] == 0) f |= (uint16_t)(1u << (2 * a));
        if (x[a] == (int)L - 1) f |= (uint16_t)(1u << (2 * a + 1));
    }
    return f;
}

static int orc_spans(uint16_t f, uint32_t span)
{
    for (uint32_t a = 0; a < 5; ++a)
        if ((span == ORC_SPAN_ANY || span == a) && ((f >> (2 * a)) & 3u) == 3u) return 1;
    return 0;
}

static uint32_t orc_find(uint32_t *parent, uint32_t a)
{
    uint32_t root = a;
    while (parent[root] != root) root = parent[root];
    while (parent[a] != root) {
        uint32_t next = parent[a];
        parent[a] = root;
        a = next;
    }
    return root;
}

/*
 * Runs the sweep for one (L, mask) on a given order over the first n_limit sites (n_limit <= N).
 * Outputs:
 *   *nstar_out            first spanning n <= n_limit under the rule `span` (ORC_NEVER if none);
 *   smax_at[q]            S_max after nq[q] sites (nq[q] in [0, n_limit]); nq may be NULL when nnq = 0;
 *   smax_all (optional)   S_max(n) for n = 0..n_limit (n_limit+1 entries), NULL to skip.
 * Returns 0, or -1 on bad input / no memory.
 */
static int orc_sweep(uint32_t L, uint32_t mask, uint32_t span, const uint32_t *perm, const uint32_t *rank,
                     const uint64_t *nq, uint32_t nnq, int64_t *smax_at, uint32_t *nstar_out,
                     int64_t *smax_all, uint64_t n_limit)
{
    uint64_t N = orc_num_sites(L);
    if (L == 0 || N >= 0xFFFFFFFFull || mask < 1 || mask > 127 || span > ORC_SPAN_ANY || n_limit > N)
        return -1;
    for (uint32_t q = 0; q < nnq; ++q)
        if (nq[q] > n_limit) return -1;

    int8_t offs[892 * 5];
    int z = orc_mask_offsets((int)mask, offs);

    uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    uint32_t *size = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    uint16_t *flags = (uint16_t *)malloc(sizeof(uint16_t) * (size_t)N);
    if (!parent || !size || !flags) {
        free(parent); free(size); free(flags);
        return -1;
    }

    uint32_t nstar = ORC_NEVER;
    uint32_t smax = 0;
    uint64_t last_query = 0; /* the sweep may stop once n* and every queried n are known */
    for (uint32_t q = 0; q < nnq; ++q) {
        if (nq[q] == 0) smax_at[q] = 0;
        if (nq[q] > last_query) last_query = nq[q];
    }
    if (smax_all) smax_all[0] = 0;

    for (uint64_t r = 0; r < n_limit; ++r) {
        uint32_t i = perm[r];
        int x[5];
        orc_coords(L, i, x);
        parent[i] = i;
        size[i] = 1;
        flags[i] = orc_site_flags(L, x);
        for (int v = 0; v < z; ++v) {
            int64_t j = orc_neighbor(L, x, offs + 5 * v);
            if (j < 0 || rank[j] >= r) continue; /* empty neighbor */
            uint32_t a = orc_find(parent, i), b = orc_find(parent, (uint32_t)j);
            if (a == b) continue;
            if (size[a] < size[b]) { uint32_t t = a; a = b; b = t; }
            parent[b] = a;
            size[a] += size[b];
            flags[a] |= flags[b];
        }
        uint32_t root = orc_find(parent, i);
        if (size[root] > smax) smax = size[root];
        uint64_t n = r + 1;
        if (nstar == ORC_NEVER && orc_spans(flags[root], span)) nstar = (uint32_t)n;
        for (uint32_t q = 0; q < nnq; ++q)
            if (nq[q] == n) smax_at[q] = smax;
        if (smax_all) smax_all[n] = smax;
        else if (nstar != ORC_NEVER && n >= last_query) break;
    }
    *nstar_out = nstar;
    free(parent); free(size); free(flags);
    return 0;
}

/* The whole sweep (n = 0..N); arguments as orc_sweep with n_limit = N. */
int orc_nz(uint32_t L, uint32_t mask, const uint32_t *perm, const uint32_t *rank,
           const uint64_t *nq, uint32_t nnq, int64_t *smax_at, uint32_t *nstar_out,
           int64_t *smax_all)
{
    return orc_sweep(L, mask, 0, perm, rank, nq, nnq, smax_at, nstar_out, smax_all, orc_num_sites(L));
}

/* n* alone under the spanning rule `span` (0..4: axis x_{span+1}; ORC_SPAN_ANY: any axis). */
int orc_nstar_span(uint32_t L, uint32_t mask, uint32_t span, const uint32_t *perm, const uint32_t *rank,
                   uint32_t *nstar_out)
{
    return orc_sweep(L, mask, span, perm, rank, NULL, 0, NULL, nstar_out, NULL, orc_num_sites(L));
}

/* S_max(n) for n = 0..n_stop (n_stop + 1 entries): the sweep stopped after n_stop sites. */
int orc_smax_prefix(uint32_t L, uint32_t mask, const uint32_t *perm, const uint32_t *rank,
                    uint64_t n_stop, int64_t *smax_prefix)
{
    uint32_t nstar;
    if (!smax_prefix) return -1;
    return orc_sweep(L, mask, 0, perm, rank, NULL, 0, NULL, &nstar, smax_prefix, n_stop);
}

/* ------------------------------------------------------------------------------------------ */
/* Brute force at a fixed n: occupy the sites with rank < n and flood-fill every cluster.        */
/* Independent of the sweep (no union-find, no border flags); used only to pin it on tiny        */
/* lattices.  A cluster spans axis a when it holds a site with x_{a+1} = 0 and one with          */
/* x_{a+1} = L-1; `span` as for the sweep.                                                       */
/* ------------------------------------------------------------------------------------------ */
int orc_bfs_span(uint32_t L, uint32_t mask, uint32_t span, const uint32_t *rank, uint64_t n,
                 int *spans, int64_t *smax)
{
    uint64_t N = orc_num_sites(L);
    if (L == 0 || N >= 0xFFFFFFFFull || mask < 1 || mask > 127 || span > ORC_SPAN_ANY || n > N) return -1;
    int8_t offs[892 * 5];
    int z = orc_mask_offsets((int)mask, offs);
    uint8_t *seen = (uint8_t *)calloc((size_t)N, 1);
    uint32_t *stack = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(N ? N : 1));
    if (!seen || !stack) {
        free(seen); free(stack);
        return -1;
    }
    int sp_any = 0;
    int64_t best = 0;
    for (uint64_t s = 0; s < N; ++s) {
        if (rank[s] >= n || seen[s]) continue;
        int64_t count = 0;
        int lo[5] = {0, 0, 0, 0, 0}, hi[5] = {0, 0, 0, 0, 0};
        uint64_t top = 0;
        stack[top++] = (uint32_t)s;
        seen[s] = 1;
        while (top) {
            uint32_t u = stack[--top];
            int x[5];
            orc_coords(L, u, x);
            ++count;
            for (int a = 0; a < 5; ++a) {
                if (x[a] == 0) lo[a] = 1;
                if (x[a] == (int)L - 1) hi[a] = 1;
            }
            for (int v = 0; v < z; ++v) {
                int64_t j = orc_neighbor(L, x, offs + 5 * v);
                if (j < 0 || rank[j] >= n || seen[j]) continue;
                seen[j] = 1;
                stack[top++] = (uint32_t)j;
            }
        }
        for (uint32_t a = 0; a < 5; ++a)
            if ((span == ORC_SPAN_ANY || span == a) && lo[a] && hi[a]) sp_any = 1;
        if (count > best) best = count;
    }
    *spans = sp_any;
    *smax = best;
    free(seen); free(stack);
    return 0;
}

int orc_bfs(uint32_t L, uint32_t mask, const uint32_t *rank, uint64_t n, int *spans, int64_t *smax)
{
    return orc_bfs_span(L, mask, 0, rank, n, spans, smax);
}

/* ------------------------------------------------------------------------------------------ */
/* Bottleneck-path identity: n* = 1 + min over paths from the face x_a = 0 to the face          */
/* x_a = L-1 (a = axis + 1) of the largest rank on the path.  Computed by Dijkstra's algorithm with the path     */
/* cost "max" instead of "+", on a binary heap.  Independent of the sweep and of the flood fill. */
/* ------------------------------------------------------------------------------------------ */
typedef struct { uint32_t cost, site; } orc_he;

static void orc_heap_push(orc_he *h, uint64_t *len, orc_he e)
{
    uint64_t k = (*len)++;
    h[k] = e;
    while (k > 0) {
        uint64_t p = (k - 1) / 2;
        if (h[p].cost <= h[k].cost) break;
        orc_he t = h[p]; h[p] = h[k]; h[k] = t;
        k = p;
    }
}

static orc_he orc_heap_pop(orc_he *h, uint64_t *len)
{
    orc_he top = h[0];
    h[0] = h[--(*len)];
    uint64_t k = 0;
    for (;;) {
        uint64_t l = 2 * k + 1, r = l + 1, m = k;
        if (l < *len && h[l].cost < h[m].cost) m = l;
        if (r < *len && h[r].cost < h[m].cost) m = r;
        if (m == k) break;
        orc_he t = h[m]; h[m] = h[k]; h[k] = t;
        k = m;
    }
    return top;
}

uint32_t orc_minimax_nstar_axis(uint32_t L, uint32_t mask, uint32_t axis, const uint32_t *rank)
{
    uint64_t N = orc_num_sites(L);
    if (L == 0 || N >= 0xFFFFFFFFull || mask < 1 || mask > 127 || axis > 4) return ORC_NEVER;
    int8_t offs[892 * 5];
    int z = orc_mask_offsets((int)mask, offs);
    uint32_t *best = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    uint8_t *done = (uint8_t *)calloc((size_t)N, 1);
    /* every push improves best[] of its site, so at most N*(z+1) entries; bound by a growable heap */
    uint64_t cap = N * 4 + 16, len = 0;
    orc_he *heap = (orc_he *)malloc(sizeof(orc_he) * (size_t)cap);
    if (!best || !done || !heap) {
        free(best); free(done); free(heap);
        return ORC_NEVER;
    }
    for (uint64_t i = 0; i < N; ++i) best[i] = ORC_NEVER;
    for (uint64_t i = 0; i < N; ++i) {
        int x[5];
        orc_coords(L, (uint32_t)i, x);
        if (x[axis] != 0) continue; /* sources: the face x_a = 0 */
        best[i] = rank[i];
        orc_heap_push(heap, &len, (orc_he){rank[i], (uint32_t)i});
    }
    uint32_t answer = ORC_NEVER;
    while (len) {
        orc_he e = orc_heap_pop(heap, &len);
        if (done[e.site] || e.cost != best[e.site]) continue;
        done[e.site] = 1;
        int x[5];
        orc_coords(L, e.site, x);
        if (x[axis] == (int)L - 1) { /* first target settled carries the minimum bottleneck */
            answer = e.cost;
            break;
        }
        for (int v = 0; v < z; ++v) {
            int64_t j = orc_neighbor(L, x, offs + 5 * v);
            if (j < 0 || done[j]) continue;
            uint32_t c = e.cost > rank[j] ? e.cost : rank[j];
            if (c < best[j]) {
                best[j] = c;
                if (len == cap) {
                    cap *= 2;
                    orc_he *nh = (orc_he *)realloc(heap, sizeof(orc_he) * (size_t)cap);
                    if (!nh) { free(best); free(done); free(heap); return ORC_NEVER; }
                    heap = nh;
                }
                orc_heap_push(heap, &len, (orc_he){c, (uint32_t)j});
            }
        }
    }
    free(best); free(done); free(heap);
    return answer == ORC_NEVER ? ORC_NEVER : answer + 1;
}

uint32_t orc_minimax_nstar(uint32_t L, uint32_t mask, const uint32_t *rank)
{
    return orc_minimax_nstar_axis(L, mask, 0, rank);
}

/* ------------------------------------------------------------------------------------------ */
/* Periodic boundaries (a variant; the paper does not state its boundary conditions): offsets    */
/* wrap modulo L in every coordinate, so the lattice is a 5-torus and every site has all z       */
/* neighbors (at small L several offsets may reach the same site, or the site itself).  No       */
/* border exists; the spanning cluster becomes a wrapping one: a cluster wraps along axis a when */
/* it holds a closed path whose steps' x_{a+1} components do not sum to zero.  The sweep keeps,  */
/* beside each union-find parent, the displacement along axis a to it, so every cluster carries  */
/* an unwrapped coordinate; an edge inside one cluster whose two ends disagree with the step     */
/* closes such a path.                                                                           */
/* ------------------------------------------------------------------------------------------ */
static int64_t orc_neighbor_periodic(uint32_t L, const int x[5], const int8_t *v)
{
    int64_t j = 0;
    for (int k = 0; k < 5; ++k) {
        int y = ((x[k] + v[k]) % (int)L + (int)L) % (int)L;
        j = j * L + y;
    }
    return j;
}

/* Root of a and the displacement pos(a) - pos(root) along the axis; compresses the path. */
static uint32_t orc_find_disp(uint32_t *parent, int64_t *dpar, uint32_t a, int64_t *disp)
{
    uint32_t root = a;
    int64_t d = 0;
    while (parent[root] != root) {
        d += dpar[root];
        root = parent[root];
    }
    int64_t rem = d; /* displacement of x to the root */
    uint32_t x = a;
    while (x != root && parent[x] != root) {
        uint32_t next = parent[x];
        int64_t dx = dpar[x];
        parent[x] = root;
        dpar[x] = rem;
        rem -= dx;
        x = next;
    }
    *disp = d;
    return root;
}

/*
 * The sweep with periodic boundaries for one (L, mask) on a given order.  Outputs the first n at
 * which a cluster wraps along axis `axis` (0..4; ORC_NEVER if none up to N) and S_max after nq[q]
 * sites.  Returns 0, or -1 on bad input / no memory.
 */
int orc_nz_periodic(uint32_t L, uint32_t mask, uint32_t axis, const uint32_t *perm, const uint32_t *rank,
                    const uint64_t *nq, uint32_t nnq, int64_t *smax_at, uint32_t *nwrap_out)
{
    uint64_t N = orc_num_sites(L);
    if (L == 0 || N >= 0xFFFFFFFFull || mask < 1 || mask > 127 || axis > 4) return -1;
    uint64_t last_query = 0;
    for (uint32_t q = 0; q < nnq; ++q) {
        if (nq[q] > N) return -1;
        if (nq[q] == 0) smax_at[q] = 0;
        if (nq[q] > last_query) last_query = nq[q];
    }
    int8_t offs[892 * 5];
    int z = orc_mask_offsets((int)mask, offs);
    uint32_t *parent = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    uint32_t *size = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    int64_t *dpar = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!parent || !size || !dpar) {
        free(parent); free(size); free(dpar);
        return -1;
    }
    uint32_t nwrap = ORC_NEVER, smax = 0;
    int wrapped = 0;
    for (uint64_t r = 0; r < N; ++r) {
        uint32_t i = perm[r];
        int x[5];
        orc_coords(L, i, x);
        parent[i] = i;
        size[i] = 1;
        dpar[i] = 0;
        for (int v = 0; v < z; ++v) {
            const int8_t *off = offs + 5 * v;
            uint32_t j = (uint32_t)orc_neighbor_periodic(L, x, off);
            if (j != i && rank[j] >= r) continue; /* empty neighbor (j == i: a loop through i) */
            int64_t da, db;
            uint32_t ra = orc_find_disp(parent, dpar, i, &da), rb = orc_find_disp(parent, dpar, j, &db);
            int64_t step = off[axis]; /* pos(j) = pos(i) + step */
            if (ra == rb) {
                if (da + step != db) wrapped = 1;
                continue;
            }
            if (size[ra] >= size[rb]) {
                parent[rb] = ra;
                dpar[rb] = step + da - db; /* pos(rb) - pos(ra) */
                size[ra] += size[rb];
            } else {
                parent[ra] = rb;
                dpar[ra] = db - da - step; /* pos(ra) - pos(rb) */
                size[rb] += size[ra];
            }
        }
        int64_t d;
        uint32_t root = orc_find_disp(parent, dpar, i, &d);
        if (size[root] > smax) smax = size[root];
        uint64_t n = r + 1;
        if (wrapped && nwrap == ORC_NEVER) nwrap = (uint32_t)n;
        for (uint32_t q = 0; q < nnq; ++q)
            if (nq[q] == n) smax_at[q] = smax;
        if (nwrap != ORC_NEVER && n >= last_query) break;
    }
    *nwrap_out = nwrap;
    free(parent); free(size); free(dpar);
    return 0;
}

/* Brute force at a fixed n with periodic boundaries: flood fill that gives every site of a      */
/* cluster an unwrapped coordinate along the axis when first reached; a step to a reached site   */
/* that disagrees with its coordinate closes a winding path.  No union-find; pins the sweep.    */
int orc_bfs_periodic(uint32_t L, uint32_t mask, uint32_t axis, const uint32_t *rank, uint64_t n,
                     int *wraps, int64_t *smax)
{
    uint64_t N = orc_num_sites(L);
    if (L == 0 || N >= 0xFFFFFFFFull || mask < 1 || mask > 127 || axis > 4 || n > N) return -1;
    int8_t offs[892 * 5];
    int z = orc_mask_offsets((int)mask, offs);
    uint8_t *seen = (uint8_t *)calloc((size_t)N, 1);
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    uint32_t *stack = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    if (!seen || !pos || !stack) {
        free(seen); free(pos); free(stack);
        return -1;
    }
    int any = 0;
    int64_t best = 0;
    for (uint64_t s = 0; s < N; ++s) {
        if (rank[s] >= n || seen[s]) continue;
        int64_t count = 0;
        uint64_t top = 0;
        stack[top++] = (uint32_t)s;
        seen[s] = 1;
        pos[s] = 0;
        while (top) {
            uint32_t u = stack[--top];
            int x[5];
            orc_coords(L, u, x);
            ++count;
            for (int v = 0; v < z; ++v) {
                const int8_t *off = offs + 5 * v;
                uint32_t w = (uint32_t)orc_neighbor_periodic(L, x, off);
                if (rank[w] >= n) continue;
                if (!seen[w]) {
                    seen[w] = 1;
                    pos[w] = pos[u] + off[axis];
                    stack[top++] = w;
                } else if (pos[w] != pos[u] + off[axis]) {
                    any = 1;
                }
            }
        }
        if (count > best) best = count;
    }
    *wraps = any;
    *smax = best;
    free(seen); free(pos); free(stack);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Binomial convolution (Methods, "Computational methods", after Newman and Ziff): the           */
/* canonical S_max(n), n = 0..N, becomes S_max(p) = sum_n B(N,n,p) S_max(n), with               */
/* B(N,n,p) = C(N,n) p^n (1-p)^(N-n).  The weights are built outward from the mode n0 with the  */
/* ratio B(n+1)/B(n) = (N-n)/(n+1) * p/(1-p), then normalised, which never forms C(N,n) itself.  */
/* orc_binomial_weights writes the normalised B(N,n,p), n = 0..N; returns -1 for p outside [0,1]. */
/* ------------------------------------------------------------------------------------------ */
int orc_binomial_weights(uint64_t N, double p, double *w)
{
    if (!w || !(p >= 0.0 && p <= 1.0)) return -1;
    for (uint64_t n = 0; n <= N; ++n) w[n] = 0.0;
    if (p == 0.0) { w[0] = 1.0; return 0; }
    if (p == 1.0) { w[N] = 1.0; return 0; }
    uint64_t n0 = (uint64_t)floor(p * (double)N);
    if (n0 > N) n0 = N;
    double ratio = p / (1.0 - p);
    w[n0] = 1.0;
    for (uint64_t n = n0; n < N; ++n)
        w[n + 1] = w[n] * ((double)(N - n) / (double)(n + 1)) * ratio;
    for (uint64_t n = n0; n > 0; --n)
        w[n - 1] = w[n] * ((double)n / (double)(N - n + 1)) / ratio;
    double norm = 0.0;
    for (uint64_t n = 0; n <= N; ++n) norm += w[n];
    for (uint64_t n = 0; n <= N; ++n) w[n] /= norm;
    return 0;
}

double orc_binomial_convolve(uint64_t N, const double *q_of_n, double p)
{
    if (p <= 0.0) return q_of_n[0];
    if (p >= 1.0) return q_of_n[N];
    double *w = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    if (!w || orc_binomial_weights(N, p, w) != 0) { free(w); return NAN; }
    double acc = 0.0;
    for (uint64_t n = 0; n <= N; ++n) acc += w[n] * q_of_n[n];
    free(w);
    return acc;
}
