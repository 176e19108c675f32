/*
 * perc.h -- C ABI of libperc.so: exact, batched first-spanning search and largest-cluster mass
 * for random site percolation on the 5D simple cubic lattice with complex neighborhoods
 * (neighborhood = any non-empty union of coordination zones 1..7, eq. z / eq. zeta, Table I).
 *
 * The quantities are those of the paper's Newman--Ziff study (Methods, "Computational methods";
 * eq. Pmax; Introduction):
 *   - a sample is a lattice side L, a zone mask and a random site-addition order;
 *   - n* is the smallest number n of occupied sites (the first n in that order) for which one
 *     cluster touches both borders x1 = 0 and x1 = L-1 (open boundaries); a sample may name
 *     another spanning axis a instead (borders x_{a+1} = 0 and x_{a+1} = L-1), and
 *     perc_nstar_min_axes turns the five per-axis values into n* for spanning along any axis;
 *   - S_max(n) is the size of the largest cluster with the first n sites occupied.
 * The order of a sample with seed s sorts the sites ascending by (key_i, i), where key_i is word 0
 * of Philox4x32-10 with counter (i, 0, 0, 0) and key (s mod 2^32, s >> 32), and
 * i = (((x1*L + x2)*L + x3)*L + x4)*L + x5.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" are caller-owned device memory; "host" pointers are read during
 *     the call only.  The library never allocates device memory: the caller sizes the workspace
 *     with perc_workspace_bytes() and passes it in.  The first 256 bytes of a workspace are its
 *     header (the status word and a work queue): the caller zeroes them once after allocating it.
 *   - Every call that takes a stream only enqueues work on it and returns; it is capturable in a
 *     CUDA graph.  Arguments that the host can check are checked before any launch
 *     (PERC_EINVAL / PERC_EWORKSPACE).  Errors found on the device (a sample with an invalid L or
 *     mask, a bounded wait that ran out) are written to the status word in the workspace, which
 *     keeps the first such error of all the calls made since the last perc_check() (so a batch of
 *     calls can be checked once at its end); perc_check() synchronises the stream, returns the
 *     status and clears it.
 *   - Returns PERC_OK (0) or a negative perc_status.
 */
#ifndef PERC_H
#define PERC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PERC_OK = 0,
    PERC_EINVAL = -1,     /* bad argument (L, mask, n, sizes, null pointer) */
    PERC_EWORKSPACE = -2, /* workspace smaller than perc_workspace_bytes() */
    PERC_ECUDA = -3,      /* a CUDA runtime call failed */
    PERC_ETIMEOUT = -4,   /* a bounded device-side wait ran out */
    PERC_EDEVICE = -5     /* a device-side check failed (bad sample found on the device) */
} perc_status;

/* n* of a sample in which no n spans (e.g. L = 2 with zones 6 and 7 only). */
#define PERC_NEVER 0xFFFFFFFFu

/* Largest lattice side: L^5 + 2 must stay below 2^31 (union-find node indices keep bit 31 free). */
#define PERC_MAX_L 73u

/* Operation codes for perc_workspace_bytes(). */
#define PERC_OP_RANK 1
#define PERC_OP_NSTAR 2
#define PERC_OP_MASS 3
#define PERC_OP_SMAX 4
#define PERC_OP_PERIODIC 5 /* perc_mass_periodic and perc_nstar_wrap */
#define PERC_OP_NSTAR_ANY 6 /* perc_nstar_any */
#define PERC_OP_MINIMAX 7   /* perc_nstar_minimax */

/* zone_mask word of a sample: bits 0..6 select coordination zones 1..7 (at least one); bits 8..10
 * hold the spanning axis a = 0..4 that perc_nstar tests (borders x_{a+1} = 0 and x_{a+1} = L-1;
 * 0, the x1 axis, is the default); every other bit is zero.  The neighborhoods are invariant under
 * exchanging coordinates, so n* along every axis has the same distribution; perc_bracket reads the
 * zone bits only, and perc_mass / perc_smax_window ignore the axis. */
#define PERC_ZONE_BITS 0x7Fu
#define PERC_AXIS_SHIFT 8u
#define PERC_ZONE_WORD(zones, axis) ((uint32_t)(zones) | ((uint32_t)(axis) << PERC_AXIS_SHIFT))

/* One sample.  perm/rank are this sample's site order (as written by perc_rank); samples that
 * share a seed point at the same arrays.  Layout: 24 bytes, 8-byte aligned. */
typedef struct {
    uint32_t L;           /* lattice side, 1 <= L <= max_L given to the call */
    uint32_t zone_mask;   /* PERC_ZONE_WORD(zones 1..127, spanning axis 0..4) */
    const uint32_t *perm; /* device [L^5]: perm[r] = site added r-th */
    const uint32_t *rank; /* device [L^5]: rank[perm[r]] = r */
} perc_sample;

/* Optional counters a call can accumulate into (device, zero them before the call). */
typedef struct {
    unsigned long long passes;       /* connected-component passes (bisection probes) */
    unsigned long long new_sites;    /* sites a pass had to merge, summed over passes (upper bound) */
    unsigned long long probe_sites;  /* sum over passes of the probe's n */
    unsigned long long hooks;        /* successful union-find hooks */
    unsigned long long early_exits;  /* passes that stopped as soon as a spanning cluster formed */
    unsigned long long fallbacks;    /* learned brackets that failed verification */
    unsigned long long verified;     /* learned brackets that passed verification */
    unsigned long long sites_merged; /* sites actually merged (early exits stop short) */
    unsigned long long unions;       /* union operations issued (edges of the NZ rule, borders included) */
    /* SM cycles (thread 0 of each CTA), bisection / sweep: */
    unsigned long long cyc_setup;    /* per-sample setup (bitmap clear, neighborhood table) */
    unsigned long long cyc_update;   /* updating the bitmap, initialising new nodes / the first pass */
    unsigned long long cyc_union;    /* the union passes / - */
    unsigned long long cyc_commit;   /* reading span, undoing or committing hooks / per-component
                                        totals, write-back and replay of the chunks */
    unsigned long long cyc_scan;     /* part of cyc_union: scanning neighborhoods into edge lists /
                                        the chunks' bitmap update and scan */
    unsigned long long cyc_link;     /* part of cyc_union: rank lookups and unions of the edges /
                                        the chunks' filter, record placement, resolve, components */
    unsigned long long chunks;       /* sweep method: chunks of sites after the first pass */
} perc_stats;

/*
 * Workspace bytes that `op` needs for a batch of `num` items (seeds for PERC_OP_RANK, samples
 * otherwise) whose largest lattice side is max_L.  Returns 0 for invalid arguments.
 */
size_t perc_workspace_bytes(int op, uint32_t max_L, uint32_t num);

/*
 * perc_rank -- the random addition order of the Newman--Ziff method (Methods, "Computational
 * methods"), one per seed: perm[s][r] = the site with the r-th smallest (key, index) for seed
 * seeds[s], and rank[s][perm[s][r]] = r.  The order does not depend on the neighborhood, so one
 * ranking serves all 127 masks.
 *   L          lattice side, 1..PERC_MAX_L
 *   seeds      device uint64[num_seeds]
 *   perm, rank device uint32[num_seeds][L^5] (outputs, row s for seed s)
 * Up to L^5 = 104,857,600 (L <= 40) a bucket sort on the keys' top bits, above it an LSD radix
 * sort; both give the same order.  Environment variables (for comparisons; results unchanged):
 * PERC_RANK_BUCKET=0 takes the radix sort at any L, PERC_RANK_TMA=0 its plain scatter instead of
 * the one fed by bulk copies.
 * Errors: PERC_EINVAL (L out of range, num_seeds 0, null pointer), PERC_EWORKSPACE.
 */
int perc_rank(uint32_t L, const uint64_t *seeds, uint32_t num_seeds, uint32_t *perm,
              uint32_t *rank, void *workspace, size_t ws_bytes, void *stream);

/*
 * perc_nstar -- exact first spanning n per sample (Introduction: the spanning cluster appears
 * for the first time at the threshold; Methods: clusters of the first n sites added in the
 * Newman--Ziff order).  Two methods (PERC_OPT_METHOD), same results:
 *   bisection  every probe n is one connected-component pass (union-find with hooking and pointer
 *              jumping) over the first n sites; span(n) is monotone in n;
 *   sweep      one pass over the sites below a start that does not span, then the sites in rank
 *              order, in chunks, until the first site whose cluster touches both borders (the
 *              Newman--Ziff sweep, chunk-parallel).
 *   samples     device perc_sample[num_samples]
 *   max_L       host bound on every sample's L (sizes the launch and the workspace)
 *   bracket     device uint32[num_samples][2] = (lo, hi) proposed by a model, or NULL for the plain
 *               bracket [1, L^5].  A bracket is verified: bisection checks span(hi) and not
 *               span(lo-1); the sweep starts at lo-1 after checking not span(lo-1) and needs no hi.
 *               One that fails, or is malformed, falls back to the plain bracket, so n* stays exact.
 *   nstar       device uint32[num_samples] (output; PERC_NEVER when nothing spans)
 *   passes      device uint32[num_samples] (output, may be NULL): passes spent on each sample
 *               (bisection probes; for the sweep, the first pass plus the chunks)
 *   stats       device perc_stats (accumulated, may be NULL)
 * Errors: PERC_EINVAL, PERC_EWORKSPACE, PERC_ECUDA; samples that fail the device check get
 * n* = PERC_NEVER and set PERC_EDEVICE in the status word.
 */
int perc_nstar(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
               const uint32_t *bracket, uint32_t *nstar, uint32_t *passes, perc_stats *stats,
               void *workspace, size_t ws_bytes, void *stream);

/*
 * perc_nstar_min_axes -- n* for spanning along any axis (a cluster touching both borders of some
 * axis; the paper names no direction, Introduction) from per-axis n*: spanning along one axis is
 * monotone in n, so out[k] = min over a < axes of nstar[k * axes + a].  The caller runs perc_nstar
 * on `axes` samples per (order, neighborhood) that differ only in the spanning axis, stored
 * consecutively.
 *   nstar  device uint32[num][axes] (per-axis n*, PERC_NEVER where an axis never spans)
 *   axes   1..5
 *   out    device uint32[num] (output; PERC_NEVER when no axis spans)
 * Errors: PERC_EINVAL (null pointer, num 0, axes outside 1..5), PERC_ECUDA.
 */
int perc_nstar_min_axes(const uint32_t *nstar, uint32_t num, uint32_t axes, uint32_t *out, void *stream);

/*
 * perc_nstar_any -- n* for spanning along any axis (the paper names no direction, Introduction): the
 * smallest n at which one cluster touches both borders x_{a+1} = 0 and x_{a+1} = L-1 of some axis a,
 * found by ONE Newman--Ziff sweep per sample in which every cluster carries ten face flags (two per
 * axis) -- the clusters do not depend on the axis, only the border flags do -- instead of five
 * per-axis sweeps and perc_nstar_min_axes.  The sample's axis bits are ignored.  Arguments,
 * bracket verification (the sweep starts at lo - 1 after checking that no cluster of the first
 * lo - 1 sites spans along any axis; a bracket that fails falls back to the sweep from 0) and errors
 * are those of perc_nstar; the workspace is perc_workspace_bytes(PERC_OP_NSTAR_ANY, max_L, num).
 */
int perc_nstar_any(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                   const uint32_t *bracket, uint32_t *nstar, uint32_t *passes, perc_stats *stats,
                   void *workspace, size_t ws_bytes, void *stream);

/*
 * Periodic boundaries (a variant; the paper does not state its boundary conditions): offsets wrap
 * modulo L in every coordinate, so the lattice is a 5-torus with no border.  Lattice sides up to
 * PERC_PERIODIC_MAX_L.  Workspace: perc_workspace_bytes(PERC_OP_PERIODIC, max_L, num_samples).
 * Samples that fail the device check get mass -1 / n* PERC_NEVER and set PERC_EDEVICE; a
 * union-find walk longer than the sample's node count (which a correct forest never needs) sets
 * PERC_ETIMEOUT and gives the same outputs.
 *
 * perc_mass_periodic -- S_max(n) on the torus: the largest cluster of each sample with its first
 * n[k] sites occupied (eq. Pmax).
 *   n     device uint64[num_samples], 0 <= n[k] <= L^5 (larger n is a device-side error)
 *   mass  device int64[num_samples] (output)
 *
 * perc_nstar_wrap -- the first n at which a cluster wraps around the torus along the sample's
 * axis (zone word bits 8..10): it holds a closed path whose steps' x_{a+1} components do not sum
 * to zero.  Found by a Newman--Ziff sweep over the site order in chunks of 512 sites, with a
 * union-find forest that carries, for every node, the displacement along the axis to its parent;
 * the chunk that first closes a winding path is undone and bisected.  Every neighborhood wraps at
 * n = L^5.
 *   nstar device uint32[num_samples] (output)
 * Errors: PERC_EINVAL (null pointer, num_samples 0, max_L outside 1..PERC_PERIODIC_MAX_L),
 * PERC_EWORKSPACE, PERC_ECUDA.
 */
#define PERC_PERIODIC_MAX_L 40u
int perc_mass_periodic(const perc_sample *samples, uint32_t num_samples, uint32_t max_L, const uint64_t *n,
                       int64_t *mass, void *workspace, size_t ws_bytes, void *stream);
int perc_nstar_wrap(const perc_sample *samples, uint32_t num_samples, uint32_t max_L, uint32_t *nstar,
                    void *workspace, size_t ws_bytes, void *stream);

/*
 * perc_nstar_minimax -- n* by a second, independent formulation (a check, not a fast path): the
 * first n at which the first n sites hold a cluster touching both borders of the sample's axis is
 * the smallest, over paths of neighboring sites joining the two borders, of the path's largest
 * rank + 1 (a min-max path value).  Found by relaxing one label per site -- rank + 1 on the
 * x_{a+1} = 0 border, then label(i) = max(rank(i) + 1, min over neighbors of label(j)) -- until no
 * label changes (at most L^5 + 2 sweeps; PERC_ETIMEOUT past them, which a correct relaxation
 * never reaches), and reading the smallest label on the x_{a+1} = L-1 border.  A sweep visits the
 * lattice in tiles of 4^5 sites: each tile's labels and a radius-2 halo are brought into shared
 * memory by one TMA tensor copy and relaxed there.  A tile copy that does not land within the
 * polls of PERC_OPT_SPIN_LIMIT ends the CTA's work with PERC_ETIMEOUT (outputs then undefined).
 * Needs every site's rank (perc_rank, not perc_rank_prefix); perm is not read.  Lattice sides up to
 * PERC_MINIMAX_MAX_L; workspace perc_workspace_bytes(PERC_OP_MINIMAX, max_L, num_samples) (one
 * label per site of the largest lattice, per CTA).
 *   nstar  device uint32[num_samples] (output)
 * Errors: PERC_EINVAL, PERC_EWORKSPACE, PERC_ECUDA; samples that fail the device check get
 * PERC_NEVER and set PERC_EDEVICE.
 */
#define PERC_MINIMAX_MAX_L 24u
int perc_nstar_minimax(const perc_sample *samples, uint32_t num_samples, uint32_t max_L, uint32_t *nstar,
                       void *workspace, size_t ws_bytes, void *stream);

/*
 * perc_mass -- largest-cluster size S_max(n) of each sample with its first n[k] sites occupied
 * (eq. Pmax; eq. M_vs_L uses it at n = p_c L^5).
 *   n     device uint64[num_samples], 0 <= n[k] <= L^5 (larger n is a device-side error)
 *   mass  device int64[num_samples] (output)
 */
int perc_mass(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
              const uint64_t *n, int64_t *mass, void *workspace, size_t ws_bytes, void *stream);

/*
 * perc_smax_window -- S_max(n) for every n of a window: the largest cluster of each sample with its
 * first n sites occupied, n = n_lo[k] .. n_lo[k] + window - 1 (eq. Pmax; Methods, "Computational
 * methods": the Newman--Ziff sweep reads S_max after every added site, and the binomial
 * convolution of perc_pmax needs it at every n where the weights are not negligible).
 *   n_lo    device uint64[num_samples]: first n of each sample's window (any value; n > L^5 has no
 *           S_max and reads 0)
 *   count   device uint32[num_samples] or NULL: entries sample k computes (min(count[k], window));
 *           NULL computes all `window` entries of every sample
 *   window  row length of smax, >= 1; num_samples * window <= 2^40
 *   smax    device uint32[num_samples][window] (output): smax[k][j] = S_max(n_lo[k] + j) for
 *           j < count[k]; 0 where j >= count[k] or n_lo[k] + j > L^5; 0xFFFFFFFF in every entry
 *           of a sample that fails the device-side check (the status word then holds PERC_EDEVICE)
 *   workspace  perc_workspace_bytes(PERC_OP_SMAX, max_L, num_samples) bytes
 * Cost: one connected-component pass over the first n_lo sites, then work proportional to the
 * sites n_lo .. n_lo + count - 2 and their earlier neighbors.
 */
int perc_smax_window(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                     const uint64_t *n_lo, const uint32_t *count, uint32_t window, uint32_t *smax,
                     void *workspace, size_t ws_bytes, void *stream);

/*
 * perc_binomial_weights -- the binomial distribution of the occupied-site count n at occupation
 * probability p, B(N, n, p) = C(N, n) p^n (1-p)^(N-n), over a window of n (Methods, "Computational
 * methods": the convolution that takes S_max(n) to S_max(p)).  Evaluated in FP64 as
 * exp(log B) with log B from Loader's saddle-point form (C. Loader, "Fast and accurate computation
 * of binomial probabilities", 2000): Stirling-series remainders of N!, n!, (N-n)! and the
 * deviance terms n log(n/Np) + Np - n computed by their series near the mean, so no factorial or
 * large power is ever formed; relative error about 1e-13.
 *   For group g (0 <= g < groups) and probability j (0 <= j < np):
 *   N      device uint64[groups]: sites L^5 of the group (1 <= N < 2^32)
 *   n_lo   device uint64[groups]: first n of the group's window
 *   count  device uint32[groups] or NULL: entries of the group's window (NULL: all `window`)
 *   p      device double[groups][np], each in [0, 1] (otherwise the row is NaN)
 *   w      device double[groups][np][window] (output): w[g][j][k] = B(N[g], n_lo[g] + k, p[g][j])
 *          for k < count[g]; 0 where k >= count[g] or n_lo[g] + k > N[g]
 * Returns PERC_EINVAL for null pointers or a zero size.
 */
int perc_binomial_weights(const uint64_t *N, const uint64_t *n_lo, const uint32_t *count, uint32_t groups,
                          uint32_t window, const double *p, uint32_t np, double *w, void *stream);

/*
 * perc_pmax -- P_max(p) = S_max(p) / L^5 with S_max(p) = sum_n B(N, n, p) S_max(n) over the window
 * (eq. Pmax and the binomial convolution of Methods, "Computational methods"), for every sample
 * and probability.  The window must cover the n where the weights matter: the neglected part is
 * at most 1 - sum_k w[g][j][k] (S_max(n) / N <= 1).
 *   smax    device uint32[num_samples][window] from perc_smax_window
 *   group   device uint32[num_samples]: weight group of each sample (< groups, else the row is NaN)
 *   w       device double[groups][np][window] from perc_binomial_weights
 *   N       device uint64[groups]: L^5 of each group
 *   count   device uint32[groups] or NULL: entries summed per group (NULL: all `window`)
 *   pmax    device double[num_samples][np] (output), FP64 sums
 */
int perc_pmax(const uint32_t *smax, const uint32_t *group, uint32_t num_samples, uint32_t window,
              const double *w, const uint64_t *N, const uint32_t *count, uint32_t groups, uint32_t np,
              double *pmax, void *stream);

/*
 * perc_nstar_noalloc -- perc_nstar without a caller-provided workspace, for callers that cannot
 * allocate device memory (code that runs inside a framework which owns every device allocation,
 * or that must not allocate once a fixed memory budget is set).  The paper has no counterpart;
 * it is an entry point of this library only.
 *   Arguments and results are those of perc_nstar with the bisection method (PERC_OPT_METHOD
 *   does not apply: n* is the same, `passes` counts bisection probes).  The scratch is a 64 MiB array that the
 *   library keeps in device memory (every GPU that loads the library holds it until exit); the
 *   call allocates nothing.  The first call on a device looks the array's address up and should
 *   come before any stream capture.  Calls share the array: calls that may overlap on the GPU race
 *   and must be serialised by the caller.  The launch uses as many CTAs as slots of its size fit
 *   in the array (a slot is about 15 MiB at L = 16, 57 MiB at L = 23, one CTA from L = 21),
 *   so it is slower than perc_nstar; a max_L whose single slot does not fit (L above 23) returns
 *   PERC_EWORKSPACE.  Device-side sample
 *   errors give n* = PERC_NEVER; the status word is not exposed.
 */
int perc_nstar_noalloc(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                       const uint32_t *bracket, uint32_t *nstar, uint32_t *passes, perc_stats *stats,
                       void *stream);

/*
 * perc_set_launch_option -- process-wide launch parameters of perc_nstar / perc_mass /
 * perc_workspace_bytes (not in the paper; set by the autotuner).  Query the workspace size again
 * after changing one.  Environment variables PERC_THREADS, PERC_SMEM_NODES and PERC_MAX_CTAS
 * override these.
 *   PERC_OPT_THREADS     threads per CTA, a multiple of 32 in 32..1024; 0 = by lattice size
 *   PERC_OPT_SMEM_NODES  most union-find nodes kept in shared memory; -1 = as many as fit (<= 16384)
 *   PERC_OPT_MAX_CTAS    cap on the persistent grid; 0 = SMs x resident CTAs
 *   PERC_OPT_GROUP       CTAs that share one sample in perc_nstar (a cooperative launch whose
 *                        bitmap and union-find live in global memory); 0 = automatic (groups for
 *                        batches of lattices above L = 17 with fewer samples than CTAs), 1 = never,
 *                        2..64 = that many
 *   PERC_OPT_METHOD      perc_nstar's method: 0 = automatic (the sweep, unless the bisection would
 *                        run cooperative groups), 1 = bisection, 2 = sweep
 *   PERC_OPT_SPIN_LIMIT  polls a bounded device-side wait makes before it gives up with
 *                        PERC_ETIMEOUT (the cooperative groups' barriers in perc_nstar, the tile
 *                        copies of perc_rank and of perc_nstar_minimax); 0 = the default, 2^26.  A small value makes those
 *                        waits run out on purpose, so that the timeout path can be tested: the
 *                        kernels then return early, the call's outputs are undefined, and
 *                        perc_check reports PERC_ETIMEOUT.  After a timeout in perc_rank each CTA
 *                        still waits (default limit) for the tile copies it has in flight.
 * Returns PERC_EINVAL for an unknown option or value.  Environment variables PERC_GROUP and
 * PERC_METHOD override PERC_OPT_GROUP and PERC_OPT_METHOD.
 */
#define PERC_OPT_THREADS 1
#define PERC_OPT_SMEM_NODES 2
#define PERC_OPT_MAX_CTAS 3
#define PERC_OPT_GROUP 4
#define PERC_OPT_METHOD 5
#define PERC_OPT_SPIN_LIMIT 6
int perc_set_launch_option(int option, int value);

/*
 * perc_check -- synchronise `stream`, read and clear the device status word of `workspace`
 * (written by perc_nstar / perc_mass), and return it (PERC_OK if nothing went wrong).
 */
int perc_check(void *workspace, void *stream);

/* ---------------------------------------------------------------------------------------- */
/* Learned bisection bracket.  Not in the paper: a small network maps a sample's zone-mask bits */
/* and ln L to three quantiles of ln(n* / L^5) (taus 0.01, 0.5, 0.99). Parameters are FP32 in  */
/* the flat layout W1[64][8], b1[64], W2[64][64], b2[64], W3[3][64], b3[3] (4931 floats);      */
/* features are rows of 8 floats [bit0..bit6 of the mask, ln L].                               */
/* ---------------------------------------------------------------------------------------- */
#define PERC_MLP_NPARAM 4931

/* Q[B][3] = network(X[B][8]).  All pointers device. */
int perc_mlp_forward(const float *params, const float *X, uint32_t B, float *Q, void *stream);

/* grad[4931] = d/dparams of the mean pinball loss over the batch (overwritten, not accumulated);
 * loss (device float, may be NULL) = that loss.  y[B] are the targets ln(n* / L^5). */
int perc_mlp_grad(const float *params, const float *X, const float *y, uint32_t B, float *grad,
                  float *loss, void *stream);

/* One Adam step (Kingma and Ba) at step count t >= 1 on n parameters, in place. */
int perc_adam(float *params, const float *grad, float *m, float *v, uint32_t n, uint32_t t,
              float lr, float beta1, float beta2, float eps, void *stream);

/* `steps` full-batch Adam steps from step count t0 + 1; grad is a device scratch of 4931 floats;
 * losses (device float[steps], may be NULL) receives the loss before each step. */
int perc_mlp_train(float *params, float *m, float *v, float *grad, const float *X, const float *y,
                   uint32_t B, uint32_t t0, uint32_t steps, float lr, float *losses, void *stream);

/* bracket[k] = (lo, hi) for samples[k]: lo = floor(N e^(q0 - margin)), hi = ceil(N e^(q2 + margin)),
 * N = L^5, clamped to 1 <= lo <= hi <= N. */
int perc_bracket(const float *params, const perc_sample *samples, uint32_t num_samples,
                 float margin, uint32_t *bracket, void *stream);

/*
 * Ranking only the start of each order (not in the paper; the Newman--Ziff sweep reads the order
 * only up to n*, and a verified bracket bounds n* from above in all but rare samples).  Three
 * calls, in this order on one stream:
 *
 * perc_prefix_share -- *share = the largest upper bracket end hi[k] / L_k^5 over the samples, in
 *   units of 2^-24, rounded up (at most 2^24).  A bracket that perc_nstar would not use (lo < 1,
 *   lo > hi, hi > L^5) or an invalid side counts as the whole lattice.
 *     samples, bracket  device, as for perc_nstar (bracket as perc_bracket writes it)
 *     share             device uint32 (output)
 *
 * perc_rank_prefix -- perc_rank for the first K = PERC_PREFIX_SITES(L^5, *share) sites of every
 *   order (the share of the lattice plus an eighth and 64 sites, at most L^5): for each seed,
 *   perm[s][0..P) holds the P >= K sites of smallest (key, index) in order and rank[s][site] is set
 *   for those sites, P ending at a key-bucket boundary (the top bits of the key).  Every other entry
 *   of perm and rank is left as it was.  For L^5 above 104,857,600 (the radix path) every site is
 *   ranked.  The keys are drawn once for every site (bucket counts) and once more only for the
 *   sites whose keys fall in the buckets where about K + 8 sqrt(K) + 64 keys are expected to end,
 *   listed in the workspace while counting; a seed whose cut lies past them, or whose list would
 *   pass half its order, draws all its keys again (the same result; PERC_RANK_STAGE=0 in the
 *   environment always does).  Arguments and workspace as for perc_rank, plus
 *     share  device uint32, as perc_prefix_share writes it (read on the device)
 *
 * perc_nstar_prefix -- perc_nstar's sweep on such orders: no site of rank >= K (K from *share and
 *   the sample's L^5, as above) is read.  A sample whose sweep reaches K without spanning gets
 *   nstar = PERC_NEVER and adds one to *unresolved; it needs its order in full (perc_rank) and
 *   perc_nstar.  Arguments, workspace (PERC_OP_NSTAR) and errors as for perc_nstar (the sweep
 *   method always), plus
 *     share       device uint32, as for perc_rank_prefix (the same value); or NULL when the orders
 *                 were ranked per seed (perc_rank_prefix_seeds): each sample then reads up to the
 *                 K of its own bracket's share (bracket required)
 *     unresolved  device uint32, incremented (the caller zeroes it)
 *
 * Per seed, for batches whose seeds serve different neighborhoods or sides (one seed per sample):
 * perc_prefix_shares -- for one order block (side L, num_seeds orders of L^5 sites from perm, laid
 *   out as for perc_rank), shares[s] = the largest share (as perc_prefix_share) over the samples
 *   whose perm points at order s of the block; samples of other blocks or sides are skipped.
 *   shares: device uint32[num_seeds] (output, zeroed first; 0 for an order no sample reads).
 * perc_rank_prefix_seeds -- perc_rank_prefix with shares[s] for seed s (device uint32[num_seeds]).
 *   Every sample's own K is at most its seed's, so perc_nstar_prefix with share NULL reads only
 *   ranked sites.
 *
 * perc_nstar_any_prefix -- the same for perc_nstar_any (spanning along any axis; workspace
 *   PERC_OP_NSTAR_ANY); its unresolved samples need perc_nstar_any on full orders.
 */
#define PERC_PREFIX_BASE_(N, share) \
    (((uint64_t)(N) * ((share) < (1u << 24) ? (uint64_t)(share) : (uint64_t)(1u << 24))) >> 24)
#define PERC_PREFIX_SITES(N, share)                                            \
    (PERC_PREFIX_BASE_(N, share) * 9u / 8u + 64u < (uint64_t)(N)               \
         ? PERC_PREFIX_BASE_(N, share) * 9u / 8u + 64u                         \
         : (uint64_t)(N))
int perc_prefix_share(const perc_sample *samples, uint32_t num_samples, const uint32_t *bracket,
                      uint32_t *share, void *stream);
int perc_rank_prefix(uint32_t L, const uint64_t *seeds, uint32_t num_seeds, const uint32_t *share,
                     uint32_t *perm, uint32_t *rank, void *workspace, size_t ws_bytes, void *stream);
int perc_nstar_prefix(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                      const uint32_t *bracket, const uint32_t *share, uint32_t *unresolved,
                      uint32_t *nstar, uint32_t *passes, perc_stats *stats, void *workspace,
                      size_t ws_bytes, void *stream);
int perc_prefix_shares(const perc_sample *samples, uint32_t num_samples, const uint32_t *bracket,
                       const uint32_t *perm, uint32_t L, uint32_t num_seeds, uint32_t *shares, void *stream);
int perc_rank_prefix_seeds(uint32_t L, const uint64_t *seeds, uint32_t num_seeds, const uint32_t *shares,
                           uint32_t *perm, uint32_t *rank, void *workspace, size_t ws_bytes, void *stream);
int perc_nstar_any_prefix(const perc_sample *samples, uint32_t num_samples, uint32_t max_L,
                          const uint32_t *bracket, const uint32_t *share, uint32_t *unresolved,
                          uint32_t *nstar, uint32_t *passes, perc_stats *stats, void *workspace,
                          size_t ws_bytes, void *stream);

/*
 * perc_microbench -- on-chip throughput probes (not in the paper): the peaks that the n* kernels,
 * which keep their data in shared memory and L2 rather than HBM, are measured against.  One launch
 * of one probe over every SM on `stream`; the caller times it (CUDA events) and divides *units by
 * the time.
 *   which  PERC_MB_L2_READ      16-byte L2-only loads streaming `iters` times over buf (choose
 *                               `bytes` well below the L2 size, after one warm-up launch); units
 *                               = bytes read
 *          PERC_MB_SMEM_READ    conflict-free 16-byte shared-memory loads; units = bytes read
 *          PERC_MB_SMEM_ATOMIC  shared-memory atomicAdd, one word per lane; units = operations
 *          PERC_MB_SMEM_CAS     shared-memory atomicCAS, one word per lane; units = operations
 *          PERC_MB_L2_ATOMIC    atomicAdd on distinct words spread over buf; units = operations
 *   buf    device scratch of `bytes` bytes (>= 4096; its contents are overwritten)
 *   iters  passes / operations per thread (>= 1)
 *   units  host double (output)
 * Errors: PERC_EINVAL (unknown probe, null pointer, bytes < 4096, iters 0), PERC_ECUDA.
 */
#define PERC_MB_L2_READ 1
#define PERC_MB_SMEM_READ 2
#define PERC_MB_SMEM_ATOMIC 3
#define PERC_MB_SMEM_CAS 4
#define PERC_MB_L2_ATOMIC 5
int perc_microbench(int which, void *buf, size_t bytes, uint32_t iters, double *units, void *stream);

/* Human-readable name of a perc_status value. */
const char *perc_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* PERC_H */
