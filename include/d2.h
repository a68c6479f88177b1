/*
 * libd2 -- single-GPU (GB300, sm_103a) D2-clustering hot path.
 *
 * C ABI of the library.  Method: Ye, Wu, Wang & Li, "Fast Discrete
 * Distribution Clustering Using Wasserstein Barycenter with Sparse Support"
 * (arXiv 1510.00012).  Each entry point cites the passage that defines the
 * operation it computes.
 *
 * Conventions shared by every call
 * --------------------------------
 *  * All array pointers are DEVICE pointers owned by the caller unless a
 *    parameter says "host".  The library never frees caller memory.
 *  * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are asynchronous on it unless they write a host output
 *    or validation is requested (D2_VALIDATE), in which case they synchronise
 *    the stream before returning.
 *  * Return value: D2_OK (0) or a negative status.  No C++ exception crosses
 *    the ABI.  d2_last_error() returns a message for the last failure on the
 *    context.  A context is not re-entrant: one host thread at a time.
 *  * Distributions ("bags") are stored raggedly (Section 2, notation list):
 *    bag k owns support rows offsets[k] .. offsets[k+1]-1 of the stacked
 *    matrix X^T (n x d, row-major) and the same entries of the weight vector.
 *  * Per-entry matrices (costs C and plans Pi) are stored "j-major": one row
 *    of m contiguous floats per SUPPORT ROW of a bag, i.e. the paper's
 *    Pi^(k) in R^{m x m_k} transposed, at rows offsets[k] .. offsets[k+1]-1 of
 *    an n x m array indexed by the global support row.  Entry (i, j) of
 *    Pi^(k) is at [(offsets[k] + j) * m + i].
 */
#ifndef D2_H
#define D2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define D2_OK        0
#define D2_EINVAL   (-1)  /* bad shape / pointer / weights (see d2_check_bags) */
#define D2_ENOMEM   (-2)  /* device allocation failed                          */
#define D2_ECUDA    (-3)  /* a CUDA runtime call or kernel launch failed       */
#define D2_ETIMEOUT (-4)  /* a bounded device-side wait expired                */
#define D2_ENOTSUP  (-5)  /* valid request outside what this build implements  */
#define D2_ENOCONV  (-6)  /* an exact W^2 solve reached its phase cap: that
                             pair's value (and the label it decides) is wrong */
#define D2_ESCRATCH (-7)  /* problem larger than d2_assign_noalloc's fixed scratch */

/* ---- options flags ---------------------------------------------------- */
#define D2_RULE_R1   1    /* Eq. (badmmw):  w_i  prop. to (1/N) sum_k wtilde_i^(k)        */
#define D2_RULE_R2   2    /* Eq. (badmmw2): sqrt(w_i) prop. to (1/N) sum_k sqrt(wtilde_i^(k)) */

#define D2_FIX_X     0x1  /* never move the support (pre-fixed support track, Section 4)  */
#define D2_FIX_W     0x2  /* keep w fixed: each member then solves OT(w, w^(k)) by B-ADMM  */
#define D2_VALIDATE  0x4  /* validate the bags on the device first (synchronises)          */
#define D2_NO_GRAPH  0x8  /* launch kernels directly instead of replaying a CUDA graph    */
#define D2_NO_PIPE   0x10 /* use the register-prefetch plan sweep instead of the
                             shared-memory pipelined one (both compute the same)  */
#define D2_ELKAN     0x20 /* d2_cluster: skip assignment pairs by the triangle
                             inequality of W (Section 5), when no pruner is given */
#define D2_ASSIGN_BOUNDED 0x200 /* d2_cluster: each round's assignment by d2_assign_bounded */
#define D2_PRUNE_RECALIBRATE 0x800 /* d2_cluster with a pruner: before every round's
                             assignment, d2_prune_calibrate on 1,000 bags (evenly
                             spaced ids) against the current centroids, quantile
                             0.999 (this updates the pruner's delta); a round
                             whose sample says the pruner cannot pay (r + f K >=
                             0.8 K, f its fall-back fraction) skips it: exact
                             assignment (certified-bound with D2_ASSIGN_BOUNDED),
                             every bag counted as a fall-back                 */
#define D2_SPLIT_STREAMS 0x400 /* badmm_barycenter: run two halves of the clusters
                             (split at half the members) concurrently on two
                             internal streams, each in a child context that
                             shares this context's per-entry workspaces; the
                             caller's stream waits for both.  Clusters are
                             independent in the update, so the results are
                             those of the single call.  Reads the split point
                             from cluster_offsets (one small synchronous copy),
                             so such a call cannot be captured in a CUDA graph
                             (it then runs as one half).                      */
#define D2_AUTOTUNE  0x100 /* badmm_barycenter: choose the plan sweep's launch shape
                             for this plan width m by timing candidates (see
                             d2_sweep_tuning); kept in the context for later calls */
/* Precision of the cost build c(x_i, y_j) = ||x_i - y_j||^2 (Section 2).  Default
 * (neither flag): FP32 on CUDA cores.  With one of these flags, and when the
 * support dimension makes the build a dense contraction (d >= 32, d % 4 == 0,
 * m % 4 == 0, a 16-byte-aligned support or vocabulary table), the cross term
 * <x_i, y_j> runs on the tensor cores (tcgen05) with an FP32 accumulator, and
 * the norms ||x_i||^2, ||y_j||^2 stay FP32 (all on coordinates centred at the
 * mean of the cluster's barycenter points).  Outside those conditions the
 * FP32 build is used.                                                      */
#define D2_COST_BF16   0x40 /* BF16 operands: about 8 mantissa bits per factor   */
#define D2_COST_BF16X3 0x80 /* each factor split hi + lo (BF16), three products:
                               about 16 mantissa bits                           */
#define D2_COST_BF16X6 0xC0 /* each factor split hi + mid + lo (BF16, exact for
                               FP32 inputs), six products: FP32-level error     */
/* Bags stored as vocabulary indices (symbolic supports, Section 5) with a
 * tensor-core cost precision: by default each cluster's cost rows are built
 * once per distinct word of its members (a per-call table) and gathered into
 * the j-major rows; the result is bitwise that of building every row.  This
 * flag builds every support row directly instead. */
#define D2_COST_ROWS 0x1000
/* Support update (Eq. updatex) on the tensor cores: with a tensor-core cost
 * precision, d >= 32, d % 4 == 0, m % 4 == 0 and m <= 64, the partial sums
 * sum_j pi_ij^(k,2) (y_j - mu_c) run as tcgen05 MMAs with split-BF16 operands
 * (hi + lo, three products; hi + mid + lo with D2_COST_BF16X6) and an FP32
 * accumulator in tensor memory, on coordinates centred at the cluster centre
 * mu_c.  Off by default: measured slower than the FP32 CUDA-core partials
 * on the shapes tested (the operands must be transposed and split). */
#define D2_SUPPORT_TC 0x2000
/* Testing only (d2_cost): the tensor-core build issues no MMA for each CTA's
 * first tile, so that CTA's bounded wait expires (about 2 s); the CTA then
 * stops, the call's output is undefined and d2_device_errors reports
 * D2_ETIMEOUT.  Exercises the expiry path without a fault or a hang. */
#define D2_TEST_EXPIRE_WAIT 0x8000

typedef struct d2_ctx d2_ctx;

/* A set of N discrete distributions (Section 2).  Supports are either dense
 * (`supp`, n x d), or indices into a shared table of points (`vocab_idx`
 * into `vocab`, V x d: the grid storage of Section 5), or symbols of a
 * symbolic set with a given symbol-to-symbol dissimilarity (`vocab_idx`
 * holds symbol ids in [0, V), `symcost` the V x V dissimilarities; supp and
 * vocab NULL, d = 1): the symbolic data of Sections 2 and 5, used only by the
 * *_sym entry points (the others return D2_EINVAL for them). */
typedef struct {
    int64_t        N;          /* number of distributions                         */
    int64_t        n;          /* total support rows = offsets[N] (host copy)     */
    int32_t        d;          /* support dimension, >= 1                         */
    int32_t        max_mk;     /* host copy of max_k m_k (launch sizing), >= 1     */
    const int64_t* offsets;    /* device, N+1, offsets[0] = 0, non-decreasing     */
    const float*   supp;       /* device, n x d row-major, or NULL with vocab     */
    const int32_t* vocab_idx;  /* device, n, or NULL                              */
    const float*   vocab;      /* device, V x d row-major, or NULL                */
    int64_t        V;          /* vocabulary rows                                 */
    const float*   wt;         /* device, n; each bag's weights >= 0, sum 1       */
    const float*   symcost;    /* device, V x V row-major, or NULL (see above)    */
} d2_bags;

/* Options of Algorithm badmm (Section 3.3). */
typedef struct {
    double  rho0;      /* Eq. (rho) scale, default 2 (Section 4, Fig. 1 setting)        */
    double  rho;       /* > 0: use this rho for every cluster instead of Eq. (rho)     */
    double  eps;       /* added after the exponential scalings, default 1e-16           */
    int32_t iters;     /* T, B-ADMM iterations per call, default 100 (Section 3.3)      */
    int32_t tau;       /* support update every tau iterations, default 10               */
    int32_t rule;      /* D2_RULE_R1 (default) or D2_RULE_R2                            */
    int32_t flags;     /* D2_FIX_X | D2_FIX_W | D2_VALIDATE | D2_NO_GRAPH | D2_NO_PIPE |
                          D2_ELKAN | D2_AUTOTUNE | D2_SPLIT_STREAMS |
                          D2_ASSIGN_BOUNDED | D2_PRUNE_RECALIBRATE | D2_COST_ROWS | D2_SUPPORT_TC |
                          one of D2_COST_BF16, _BF16X3, _BF16X6                        */
} d2_badmm_opts;

/* Fill `o` with the defaults above. */
void d2_badmm_opts_default(d2_badmm_opts* o);

/* Create a context on CUDA device `device`.  It owns the device workspaces
 * (duals, cost matrices, per-member partials) that the calls below grow on
 * demand and reuse.  Returns NULL on failure. */
d2_ctx* d2_create(int device);

/* Free a context and every workspace it owns (NULL is a no-op). */
void d2_destroy(d2_ctx* ctx);

/* Message describing the last failure on `ctx` ("" if none).  The string is
 * owned by the context and valid until the next call on it. */
const char* d2_last_error(const d2_ctx* ctx);

/* Bytes of device workspace the context currently holds. */
size_t d2_workspace_bytes(const d2_ctx* ctx);

/* ---- instrumentation ----------------------------------------------------
 * When timing is on, the context brackets each launch of the kinds below with
 * CUDA events recorded on the launching stream; d2_timing_read() waits for
 * them and returns the summed milliseconds and launch counts per kind. */
#define D2_KT_SWEEP_FUSED 0  /* plan sweep carrying both halves of an iteration      */
#define D2_KT_SWEEP_HALF  1  /* plan sweep carrying one half (first/last/support it.) */
#define D2_KT_COST        2  /* cost-matrix build                                     */
#define D2_KT_SUPPORT     3  /* support update, Eq. (updatex)                         */
#define D2_KT_ASSIGN      4  /* exact assignment                                      */
#define D2_KT_PRUNE       5  /* pruning network                                       */
#define D2_KT_OTHER       6
#define D2_KT_BOUND       7  /* lower bounds of the bounded exact assignment         */
#define D2_KT_COUNT       8
/* Turn per-launch timing on (1) or off (0); either way the totals restart. */
int d2_timing_enable(d2_ctx* ctx, int on);
/* Summed device milliseconds and launch counts per kind since the last
 * d2_timing_enable (arrays of D2_KT_COUNT; either may be NULL). Synchronous. */
int d2_timing_read(d2_ctx* ctx, double* ms, int64_t* launches);
/* Number of kernels this context has launched since it was created. */
int64_t d2_launch_count(const d2_ctx* ctx);

/* Sticky device-side error bits raised by this context's kernels since the
 * last call (synchronous; the bits are cleared).  Kernels never trap: a
 * bounded wait on the device that expires (about 2 s; the tensor-core cost
 * build waits on its MMAs) sets bit 0x40 and the kernel returns early; an
 * exact W^2 solve (d2_assign, d2_assign_bounded, d2_w2_pairs, d2_cluster,
 * d2_prune_calibrate) that reaches its phase cap sets bit 0x10 and returns
 * the cost of its unfinished flow.  Returns D2_ETIMEOUT when bit 0x40 was
 * set, else D2_ENOCONV when bit 0x10 was set, else D2_OK; *bits (host,
 * optional) receives the raw bits. */
int d2_device_errors(d2_ctx* ctx, int32_t* bits);

/* Cap on the shortest-path phases of one exact W^2 solve on this context
 * (0 restores the default 8 (m + max_mk) + 64; every phase routes flow to at
 * least one deficit sink, so a solve needs far fewer).  For testing the
 * reporting path: a low cap makes solves stop early, without any fault, and
 * report D2_ENOCONV.  Returns D2_EINVAL for a negative cap. */
int d2_set_phase_limit(d2_ctx* ctx, int32_t max_phases);

/* Flow store of the exact W^2 solver on this context (no counterpart in the
 * paper; the LP of Eq. primal is the same either way).  store = 0 (default):
 * per size class of bags, the store that keeps more warps resident per SM;
 * 1: dense flow tableaus; 2: sparse (per-point bitmasks and a pool of nonzero
 * flows).  A pair whose sparse pool overflows is solved again with the dense
 * store in the same call (up to 65,536 pairs per call; beyond that a pair is
 * reported like a phase-cap hit, D2_ENOCONV).  pool_cap > 0 caps the pool's
 * entries below its default 2 (m + m_k), to exercise that path in tests.
 * Returns D2_EINVAL for a store outside 0..2 or a negative cap. */
int d2_set_flow_store(d2_ctx* ctx, int32_t store, int32_t pool_cap);

/* Entropic dual bound of d2_assign_bounded on this context (no counterpart in
 * the paper; the argmin and its value stay those of the exact LP of Eq.
 * primal).  For every pair that the cheap bounds leave, up to `iters` Sinkhorn
 * iterations of the problem regularised by eps = eps_rel x the pair's mean
 * cost give dual potentials, made feasible for the dual of Eq. (primal) by a
 * c-transform; the dual objective is then a lower bound on W^2 that replaces
 * the cheap one when larger, so fewer pairs need the exact solve (every 10
 * iterations the bound is checked and the pair stops once excluded).  Applies
 * for m <= 64.  iters = -1 (default): 40 iterations when m >= 32, none below;
 * 0: off.  eps_rel = 0: the default 0.05.  Returns D2_EINVAL for iters
 * outside -1..10000 or eps_rel outside [0, 100]. */
int d2_set_dual_bound(d2_ctx* ctx, int32_t iters, float eps_rel);

/* Cheap lower bounds of d2_assign_bounded on this context: path = 0 (default)
 * computes their cost entries as tensor-core contractions (tcgen05, split-
 * BF16 operands, FP32 accumulation; each bound lowered by a bound on the
 * products' error, so it stays below W^2) for bags of <= 64 points,
 * 64 <= d <= 320 and m dividing 128 (m >= 16), else on the CUDA cores;
 * path = 1 always on the CUDA cores.  The labels and distances are the exact
 * ones either way.  Returns D2_EINVAL for another path. */
int d2_set_bound_kernels(d2_ctx* ctx, int32_t path);

/* Pruning network kernels on this context: path = 0 (default) runs the
 * forward's layers 1 and 2 as tensor-core GEMMs (tcgen05, FP16 operands,
 * FP32 accumulation in tensor memory) where d <= 128 and H <= 128 with H a
 * multiple of 32, and the backward's weight-gradient contractions on the
 * tensor cores (split-BF16 operands) where both sides are <= 128 wide, else
 * on the CUDA cores; path = 1 always on the CUDA cores (the forward's
 * operands are the same FP16-rounded values; the results differ in the order
 * of FP32 additions and, for the gradients, by the split's 2^-16).  Returns
 * D2_EINVAL for another path. */
int d2_set_prune_forward(d2_ctx* ctx, int32_t path);

/* Validate a bag set on the device (synchronous): offsets non-decreasing with
 * offsets[N] == n and every m_k in [1, max_mk]; weights finite, >= 0 and each
 * bag's sum within 1e-5 of 1 (Section 2: w in the simplex); vocabulary indices
 * in [0, V).  Returns D2_OK or D2_EINVAL with the first problem described. */
int d2_check_bags(d2_ctx* ctx, const d2_bags* bags, void* stream);

/* Squared-Euclidean cost matrices C(x_c, x^(k)) = (||x_i - x_j^(k)||^2)_{i,j}
 * (Section 2 notation list; c(.,.) under Eq. (primal) with p = 2) between the
 * barycenter support of each cluster and each of its members.
 *
 *   cluster_offsets : device, K+1; members[cluster_offsets[c] ..
 *                     cluster_offsets[c+1]-1] are the bag ids of cluster c
 *   members         : device, P bag ids (a bag may appear at most once)
 *   x               : device, K x m x d, barycenter supports (row-major)
 *   C_out           : device, n x m; the j-major rows of every listed member
 *                     are written, other rows are left untouched
 *   flags           : 0 (FP32) or D2_COST_BF16 / _BF16X3 / _BF16X6 (tensor
 *                     cores, see those flags); with vocabulary bags and a
 *                     tensor-core precision the rows come from the
 *                     per-(cluster, word) table unless D2_COST_ROWS is set
 * Requires 1 <= m <= 256.  Arithmetic on coordinates centred at the mean of
 * each cluster's barycenter points; entries are clamped at 0. */
int d2_cost(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets,
            const int64_t* members, int64_t P, int32_t K, int32_t m,
            const float* x, float* C_out, int32_t flags, void* stream);

/* Centroid update with B-ADMM (Algorithm badmm, Section 3.3) for K clusters
 * at once, every cluster advancing through the same T iterations:
 *   Lambda := 0; Pi^(2),0 := warm plan or w_i w_j^(k) (Section 5);
 *   repeat T times: x by Eq. (updatex) every tau iterations (n > 0);
 *   Pi^(k,1) by Eqs. (badmmc0b, badmmc0); wtilde^(k) from Eq. (badmmc1b);
 *   w by Eq. (badmmw) or (badmmw2); Pi^(k,2) by Eq. (badmmc1);
 *   Lambda by Eq. (badmm2).   rho by Eq. (rho) per cluster (rho0 x mean C).
 *
 *   cluster_offsets, members, P : the clustering, as for d2_cost; P host
 *   x      : device, K x m x d, in: initial support, out: final support
 *   w      : device, K x m, in: initial weights (simplex), out: final w
 *   plan   : device, n x m (j-major, see above).  In: cached Pi^(k,2) rows of
 *            members whose warm_mask entry is non-zero.  Out: the final
 *            Pi^(k,2) of every listed member.  Rows of unlisted bags are left
 *            untouched.  Between calls it is the warm-start cache of Section 5.
 *   warm_mask : device, N bytes (indexed by bag id) or NULL = all cold
 *   obj    : device, K doubles, out: (1/N_c) sum_k <C_k, Pi^(k,1)> with the
 *            final support (0 for an empty cluster)
 * Clusters with no member keep x and w unchanged.  Requires 1 <= m <= 256,
 * iters >= 1, tau >= 1.  Plans, duals and exponentials are FP32; the
 * cross-member weight sums and the objective are FP64 and deterministic. */
int badmm_barycenter(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets,
                     const int64_t* members, int64_t P, int32_t K, int32_t m,
                     float* x, float* w, float* plan, const uint8_t* warm_mask,
                     const d2_badmm_opts* opts, double* obj, void* stream);

/* ---- member-parallel trunks (the parallel implementation of Section 5) ----
 * Every cross-member sum of Algorithm badmm (the weight consensus of every
 * iteration, the support partials of every support update, the cost sum of
 * Eq. rho, the objective, the member counts) is an exact sum of 64-bit
 * fixed-point integers, whose result does not depend on the order of its
 * terms.  A caller that splits the members of every cluster over several
 * processes (each calling badmm_barycenter with its own members, in whole
 * groups of 64 consecutive members of a cluster as one process would order
 * them, so that every per-group partial sum is the same) installs a reducer
 * that sums (or takes the maximum of) an int64 buffer element-wise across the
 * processes, in place, ordered on the given stream -- an NCCL all-reduce, or
 * host code.  The results (x, w, the plans of each process's members, the
 * objective) are then bitwise those of one process holding every member.
 * The library calls the reducer while it enqueues work (about one call per
 * iteration, two per support update); with a reducer installed it launches
 * kernels directly (no CUDA graph, no D2_SPLIT_STREAMS).  fn returns 0 on
 * success; anything else makes the call fail with D2_ECUDA.  fn = NULL
 * removes it.  No counterpart in the paper beyond the trunks themselves. */
#define D2_REDUCE_SUM 0
#define D2_REDUCE_MAX 1
typedef int (*d2_reducer_fn)(void* user, int32_t op, int64_t* buf, int64_t count, void* stream);
int d2_set_reducer(d2_ctx* ctx, d2_reducer_fn fn, void* user);

/* Plan-sweep autotuner (no counterpart in the paper; Algorithm badmm fixes
 * what is computed, not how it is laid out on a GPU).  The first
 * badmm_barycenter call on a context with D2_AUTOTUNE in opts->flags and plan
 * width m runs its fused passes (iterations that carry both halves of
 * Eqs. badmmc1/badmm2 and badmmc0b/badmmc0) with each candidate launch shape
 * in turn, `reps` passes per candidate, timing each with CUDA events; every
 * candidate computes the same iteration, so the call's results are valid (up
 * to FP32 rounding order).  The fastest shape is kept in the context and used
 * by later calls with that m (with or without the flag).  Candidates: the
 * shared-memory pipelined sweep with 2 or 1 float4s per lane (m/8 or m/4
 * lanes per plan row), the register-prefetch sweep, each with 1..max
 * persistent CTAs per SM (members per warp follow from the grid).
 *   ncand, chosen : host, out (chosen = -1 and ncand = 0 when m is untuned)
 *   ms            : host, D2_TUNE_MAX floats: mean fused-pass milliseconds
 *   shape         : host, D2_TUNE_MAX x 4 int32: kind (0 pipelined,
 *                   1 prefetch), lanes per row, float4s per lane, CTAs/SM */
#define D2_TUNE_MAX 16
int d2_sweep_tuning(const d2_ctx* ctx, int32_t m, int32_t* ncand, int32_t* chosen,
                    float* ms, int32_t* shape);

/* Exact W^2 solves (stats[0]) and pruner fall-backs (stats[1]) of the last
 * d2_cluster call on this context (host, 2 int64). */
int d2_cluster_stats(const d2_ctx* ctx, int64_t* stats);

/* ---- learned candidate pruning (no counterpart in the paper) --------------
 * An MLP embedding f of a distribution (per-point d -> H -> H with ReLU,
 * weight-pooled, then H -> E), used to rank centroids by
 *   What^2(P, Q) = ||mu_P - mu_Q||^2 + ||f(P) - f(Q)||^2
 * before the exact assignment; see d2_assign.  Parameters are FP32 masters,
 * the forward/backward GEMMs take FP16 inputs with FP32 accumulation. */
typedef struct d2_prune d2_prune;

/* Create a pruner for support dimension d with hidden width H and embedding
 * width E (H, E multiples of 16, <= 256).  `init` (host, optional) holds the
 * parameters W1 (H x d), b1 (H), W2 (H x H), b2 (H), W3 (E x H) packed in that
 * order; NULL draws them from SplitMix64(seed) (uniform +-sqrt(6/fan_in)). */
d2_prune* d2_prune_create(d2_ctx* ctx, int32_t d, int32_t H, int32_t E,
                          const float* init, uint64_t seed);
void d2_prune_destroy(d2_prune* p);
/* Number of packed parameters. */
int64_t d2_prune_param_count(const d2_prune* p);
/* Copy the packed parameters to / from host memory (synchronous). */
int d2_prune_get_params(d2_ctx* ctx, const d2_prune* p, float* host_out);
int d2_prune_set_params(d2_ctx* ctx, d2_prune* p, const float* host_in);
/* Candidate count r (1..16) and margin delta (>= 0) of the margin test;
 * d2_prune_train sets delta to the 99.9% quantile of |What^2 - W^2| on its
 * held-out pairs. */
int d2_prune_set_margin(d2_prune* p, int32_t r, float delta);
int d2_prune_get_margin(const d2_prune* p, int32_t* r, float* delta);

/* Recalibrate the margin delta against centroids (x, w): exact W^2 of every
 * (bag ids[t], centroid) pair (device ids, nids) by the solver of d2_assign,
 * and delta := the `quantile` (in (0, 1]) of |What^2 - W^2| over those pairs.
 * Centroids move between the rounds of Algorithm 1, so a delta measured on
 * the training centroids need not cover later ones.  Synchronous. */
int d2_prune_calibrate(d2_ctx* ctx, d2_prune* p, const d2_bags* bags, int32_t K, int32_t m,
                       const float* x, const float* w, const int64_t* ids, int64_t nids,
                       float quantile, void* stream);
/* Fraction of the last d2_prune_calibrate sample whose margin test fails
 * under the new delta (those bags would be solved against all K); -1 before
 * any calibration. */
int d2_prune_get_calibration(const d2_prune* p, float* fallback_frac);

/* Embeddings f(P) of the bags listed in `ids` (device, cnt) -> emb (device,
 * cnt x E) and their means mu (device, cnt x d). */
int d2_prune_embed(d2_ctx* ctx, const d2_prune* p, const d2_bags* bags,
                   const int64_t* ids, int64_t cnt, float* emb, float* mu, void* stream);

/* Loss L = (1/B) sum_b (||f(P_a) - f(Q_q)||^2 - (t_b - ||mu_a - mu_q||^2))^2
 * over B pairs (bag a_b of `bags`, centroid q_b of (x, w)) and its gradient
 * (device, packed like the parameters).  loss (device, 1 double). */
int d2_prune_loss_grad(d2_ctx* ctx, const d2_prune* p, const d2_bags* bags,
                       int32_t K, int32_t m, const float* x, const float* w,
                       const int64_t* pair_bag, const int32_t* pair_cent,
                       const float* target, int64_t B, double* loss, float* grad,
                       void* stream);

/* Train with Adam (lr, beta1 0.9, beta2 0.999) for `steps` minibatches of
 * `batch` pairs drawn by SplitMix64(seed) from the npairs training pairs;
 * loss_out (host, steps) receives each minibatch loss.  Synchronous. */
int d2_prune_train(d2_ctx* ctx, d2_prune* p, const d2_bags* bags,
                   int32_t K, int32_t m, const float* x, const float* w,
                   const int64_t* pair_bag, const int32_t* pair_cent,
                   const float* target, int64_t npairs, int32_t steps, int32_t batch,
                   float lr, uint64_t seed, float* loss_out);

/* Assignment step of Algorithm 1: labels[k] = argmin_i W^2(Q_i, P^(k)) with
 * W^2 the exact transportation LP of Eq. (primal) (ties -> lowest i), and
 * dist[k] that minimum.
 *   x, w   : device, K x m x d and K x m, the centroids Q_i
 *   prune  : NULL = solve all K pairs exactly.  Otherwise solve the r
 *            centroids of smallest What^2 exactly and accept the best b
 *            among them when every other centroid has
 *            max(||mu_P - mu_Qi||^2, What^2_i - delta) > b; else solve all K.
 *   labels : device, N int32;  dist : device, N floats
 *   stats  : optional host int64[3]: exact solves, fall-backs, solves that
 *            reached the phase cap (synchronises when given)
 * The exact solver is successive shortest paths with node potentials, one
 * warp per (bag, centroid) pair, flows and costs in FP32, the final cost
 * summed in FP64.  Requires 32 ceil(m / 32) + max_mk <= 256 and the two m x max_mk FP32
 * tableaus of a pair within 200 KiB (D2_ENOTSUP otherwise).  A solve that
 * reaches its phase cap (see d2_set_phase_limit) gives a wrong value: with
 * stats the call then returns D2_ENOCONV; without stats (asynchronous) it
 * sets the context's sticky bit 0x10, which d2_device_errors reports as
 * D2_ENOCONV. */
int d2_assign(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m,
              const float* x, const float* w, const d2_prune* prune,
              int32_t* labels, float* dist, int64_t* stats, void* stream);

/* Assignment step of Algorithm 1 with the same result as d2_assign without a
 * pruner (exact argmin of W^2, ties -> lowest i), solving far fewer LPs.  For
 * every (bag, centroid) pair it computes a certified lower bound on W^2:
 * the larger of the two one-sided relaxations of the LP of Eq. (primal)
 * (each bag point ships its mass to its nearest centroid point, and the
 * reverse) and ||mu_P - mu_Q||^2 (Jensen), and for m <= 64 where enabled
 * the entropic dual bound (d2_set_dual_bound).  It solves each bag's r
 * smallest-bound centroids exactly (r = 1, 2 where the dual bound runs, or
 * the pruner's r candidates when `prune` is given), then the centroid of
 * smallest remaining bound if that bound does not exceed the best value
 * found, then every other centroid whose bound does not exceed the best value
 * found times (1 + 1e-4) (covering FP32 rounding).  Requires
 * max_mk <= 128 and the conditions of d2_assign.  stats and D2_ENOCONV: as
 * for d2_assign (fall-backs stay 0). */
int d2_assign_bounded(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m,
                      const float* x, const float* w, const d2_prune* prune,
                      int32_t* labels, float* dist, int64_t* stats, void* stream);

/* Exact W^2 (Eq. primal, the same solver as d2_assign) for an explicit list
 * of npairs (bag pair_bag[p], centroid pair_cent[p]) -> out[p] (device
 * floats).  Used to produce training targets for the pruner.  Asynchronous: a
 * solve that reaches its phase cap sets the sticky bit that d2_device_errors
 * reports as D2_ENOCONV. */
int d2_w2_pairs(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m,
                const float* x, const float* w, const int64_t* pair_bag,
                const int32_t* pair_cent, int64_t npairs, float* out, void* stream);

/* Exact assignment without any device allocation.  The paper has no
 * counterpart: this is d2_assign with prune = NULL for callers that may not
 * allocate device memory themselves or have a library do it (a process
 * whose device memory is owned by another framework's fixed pool, or a
 * service that must not allocate after start-up).  It takes no context.
 * Scratch: one fixed file-scope device array holding up to
 * D2_NOALLOC_MAX_PAIRS (2^20) pair distances, so it needs N * K <= 2^20 and
 * returns D2_ESCRATCH beyond that.  Every GPU that loads the library keeps
 * the array (about 4 MiB) until the process exits.  The first call on a
 * device resolves the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.
 * The cached address is not refreshed after cudaDeviceReset: do not call
 * this entry point again in a process that has reset the device.
 * All calls share the array and it keeps the last call's contents (the
 * counters are cleared by each call): calls that overlap on the GPU, on any
 * streams, race.  Other arguments and results as for d2_assign.  The call is
 * synchronous: it reads back how many solves reached the phase cap.
 * Returns D2_OK, D2_EINVAL (bad pointers or sizes; supp and vocab both given
 * or both missing), D2_ESCRATCH (N * K > D2_NOALLOC_MAX_PAIRS), D2_ENOTSUP
 * (32 ceil(m / 32) + max_mk > 256, or the per-pair tableaus of d2_assign
 * exceed 200 KiB),
 * D2_ENOCONV (some solve reached the phase cap: its value and label are
 * wrong) or D2_ECUDA. */
#define D2_NOALLOC_MAX_PAIRS (1 << 20)
int d2_assign_noalloc(const d2_bags* bags, int32_t K, int32_t m, const float* x, const float* w,
                      int32_t* labels, float* dist, void* stream);

/* ---- symbolic supports (Sections 2 and 5) ---------------------------------
 * Distributions over a symbolic set with a given symbol-to-symbol
 * dissimilarity c(s, t) = symcost[s V + t] (any nonnegative values; squared
 * distances for D2-clustering).  The centroids' supports are symbols too and
 * never move ("the step of updating the support vectors can be skipped since
 * the set of symbols is fixed", Section 5): a centroid is m symbols
 * csym[c m .. c m + m - 1] and their weights. */

/* Cost matrices C_k[j, i] = c(csym_c,i, symbol of row j) of every listed
 * member, j-major like d2_cost (cluster_offsets, members, P, K, m as there;
 * csym: device, K x m symbol ids in [0, V)). */
int d2_sym_cost(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets, const int64_t* members,
                int64_t P, int32_t K, int32_t m, const int32_t* csym, float* C_out, void* stream);

/* Algorithm badmm (Section 3.3) with fixed symbolic supports: the plans and
 * the weights w (device, K x m, in/out) of every cluster, the costs taken
 * from the table, rho by Eq. (rho), Eq. (updatex) skipped.  Other arguments
 * and results as for badmm_barycenter (D2_FIX_X is implied; D2_SPLIT_STREAMS
 * and the cost precision flags are ignored). */
int badmm_barycenter_sym(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets,
                         const int64_t* members, int64_t P, int32_t K, int32_t m, const int32_t* csym,
                         float* w, float* plan, const uint8_t* warm_mask, const d2_badmm_opts* opts,
                         double* obj, void* stream);

/* Assignment step of Algorithm 1 with symbolic supports: labels[k] =
 * argmin_i W^2(Q_i, P^(k)) by the exact solver of d2_assign on the table's
 * costs (ties -> lowest i); stats and D2_ENOCONV as for d2_assign. */
int d2_assign_sym(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const int32_t* csym,
                  const float* w, int32_t* labels, float* dist, int64_t* stats, void* stream);

/* D2-clustering (Algorithm 1) of symbolic distributions, every centroid
 * supported on the same m symbols sym (device, m ids).  Initialisation: K
 * distinct bags drawn by a partial Fisher-Yates shuffle of all bag ids driven
 * by SplitMix64(seed); centroid c's weight on sym_i is the mass of the c-th
 * bag's symbols whose nearest centroid symbol (smallest c(sym_i, t), first
 * minimum) is sym_i.  Rounds as in d2_cluster: exact assignment, then
 * badmm_barycenter_sym over all K clusters with the plans of unchanged
 * members warm-started (Section 5).  w_out: device K x m; labels_out: device
 * N; obj_per_round: host, rounds doubles.  Synchronous; D2_ENOCONV as for
 * d2_cluster. */
int d2_cluster_sym(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const int32_t* sym, uint64_t seed,
                   int32_t rounds, const d2_badmm_opts* opts, float* w_out, int32_t* labels_out,
                   double* obj_per_round, void* stream);

/* Greedy merge of Eq. (merge) (Section 5): reduce bag ids[c] to m support
 * points for c = 0..cnt-1 -> x (device cnt x m x d), w (device cnt x m).
 * Ties: first minimum in lexicographic (i, j) order.  A bag with fewer than
 * m points is copied and padded with zero-weight copies of its last point. */
int d2_merge_init(d2_ctx* ctx, const d2_bags* bags, const int64_t* ids, int64_t cnt,
                  int32_t m, float* x, float* w, void* stream);

/* D2-clustering (Algorithm 1 with the Section 5 choices), all on the device:
 * K distinct bags with m_k >= m chosen by a partial Fisher-Yates shuffle
 * driven by SplitMix64(seed) and reduced by Eq. (merge) (when fewer than K
 * bags have m points, the threshold drops to the K-th largest m_k and the
 * picks are padded with zero-weight copies); then `rounds` rounds
 * of { d2_assign (with `prune` if non-NULL; else, with D2_ELKAN in
 * opts->flags, Elkan's triangle-inequality skipping of Section 5 with the
 * metric W = sqrt(W^2): lower bounds per (bag, centroid) carried across
 * rounds and lowered by the centroid shifts, centroid-centroid distances,
 * and an exact distance to each bag's current centroid every round; with
 * D2_ASSIGN_BOUNDED, d2_assign_bounded, which also takes `prune`);
 * badmm_barycenter over all K clusters, warm-starting Pi^(k,2) of every bag
 * whose label is unchanged }.
 *   x_out, w_out, labels_out : device, K x m x d, K x m, N
 *   obj_per_round : host, rounds doubles: (1/N) sum_k W^2(Q_{l_k}, P^(k)) at
 *                   each round's assignment
 * Synchronous.  Empty clusters keep their previous centroid.  Returns
 * D2_ENOCONV (after writing every output) when some exact W^2 solve of the
 * assignment steps reached its phase cap. */
int d2_cluster(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, uint64_t seed,
               int32_t rounds, const d2_badmm_opts* opts, const d2_prune* prune,
               float* x_out, float* w_out, int32_t* labels_out, double* obj_per_round,
               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* D2_H */
