// Internal definitions of libd2: the context, its device workspaces, error
// plumbing and small device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/d2.h"

#define D2_LOG2E 1.4426950408889634

// Workspace slots owned by a context; each grows on demand and is reused.
enum WsSlot {
    WS_LAM = 0,      // n x m floats: duals Lambda (j-major)
    WS_COST,         // n x m floats: cost matrices C (j-major)
    WS_POS_CLUSTER,  // P int32: cluster of each member position
    WS_POS_R,        // P x m floats: member row sums r_k of Pi-tilde^(k,1)
    WS_POS_PART,     // P x m doubles: per-member wtilde^(k) (or its sqrt)
    WS_POS_OBJ,      // P doubles: per-member <C_k, Pi^(k,1)>
    WS_CHUNKS,       // chunk table + per-cluster chunk ranges
    WS_CHUNK_SUM,    // per-chunk FP64 cost sum and row count
    WS_XPART,        // per-chunk partial support sums (m x d floats)
    WS_CLUSTER,      // per-cluster small arrays (rho, beta, mu, xt, norms, w buffers, counters)
    WS_SCAN,         // scratch for scans
    WS_ASSIGN,       // assignment scratch
    WS_CLUSTER_LOOP, // d2_cluster state (labels, plan cache, ...)
    WS_PRUNE,        // pruning scratch
    WS_ELKAN,        // triangle-inequality bounds carried across rounds
    WS_SPLIT,        // rebased cluster offsets of the second half of a split call
    WS_VOCAB,        // vocabulary cost table: word flags, slots, pseudo-members, chunks
    WS_VOCAB_T,      // vocabulary cost table rows (<= min(n, K V) x m floats)
    WS_ASSIGN_OVF,   // exact solver: pairs whose sparse flow pool overflowed
    WS_FIXED,        // exact fixed-point reductions: counts, consensus sums, scratch
    WS_MLP,          // pruning network forward on the tensor cores: point offsets, pooled partials
    WS_LBTC,         // bounded assignment: centroid points as tensor-core tiles, their largest norms
    WS_NSLOTS
};

// Launch shape of the plan sweep chosen by the autotuner for one plan width m
// (D2_TUNE_MAX candidates at most, see d2.h).
struct SweepTune {
    int m = 0;
    const void* fn = nullptr;       // kernel
    size_t smem = 0;                // dynamic shared memory
    int per_sm = 1;                 // persistent CTAs per SM
    int ncand = 0, chosen = -1;
    float ms[D2_TUNE_MAX] = {};     // mean fused-pass time per candidate
    int shape[D2_TUNE_MAX][4] = {}; // kind (0 pipelined, 1 prefetch), lanes/row, float4s/lane, CTAs/SM
};

struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
};

struct d2_ctx {
    int device = 0;
    std::string err;
    void* ws[WS_NSLOTS] = {};
    size_t ws_bytes[WS_NSLOTS] = {};
    int* dev_flags = nullptr;       // device-side error flags (see D2F_*)
    unsigned long long generation = 0;  // bumps whenever a workspace moves
    int64_t launches = 0;           // kernels launched so far
    bool timing = false;
    std::vector<TimedLaunch> timed;     // pending event pairs
    std::vector<cudaEvent_t> ev_pool;   // recycled events
    double t_ms[D2_KT_COUNT] = {};
    int64_t t_n[D2_KT_COUNT] = {};
    // last captured badmm_barycenter launch sequence and what it was built for
    std::vector<uint64_t> graph_key;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_launches = 0;
    // exact W^2 solves and pruner fall-backs of the last d2_cluster call
    int64_t cluster_solves = 0, cluster_fallbacks = 0;
    // sweep launch shapes chosen by the autotuner, one per plan width m
    std::vector<SweepTune> tuned;
    // testing: the next tensor-core cost build lets its first wait expire
    int expire_test = 0;
    // cap on the exact solver's shortest-path phases per pair (0: default)
    int phase_limit = 0;
    // member-parallel trunks: sum / max of int64 buffers across processes
    d2_reducer_fn reducer = nullptr;
    void* reducer_user = nullptr;
    // exact solver's flow store: 0 automatic, 1 dense, 2 sparse; and a cap on
    // the sparse pool's entries (0: none) -- testing and tuning
    int flow_store = 0;
    int pool_cap = 0;
    // entropic dual bound of d2_assign_bounded: Sinkhorn iterations (-1:
    // automatic) and eps as a fraction of the pair's mean cost (0: default)
    int dual_iters = -1;
    float dual_eps = 0.f;
    // pruning network forward on the CUDA cores even where the tensor-core
    // kernel applies (testing: the two forwards side by side)
    int mlp_cuda_cores = 0;
    // cheap bounds of the bounded assignment on the CUDA cores even where the
    // tensor-core kernel applies (testing: the two side by side)
    int bound_cuda_cores = 0;
    // split calls (D2_SPLIT_STREAMS): two child contexts, each on its own
    // stream, with the per-entry workspaces lent by this context
    d2_ctx* child[2] = {nullptr, nullptr};
    cudaStream_t cstream[2] = {nullptr, nullptr};
    cudaEvent_t cev[3] = {nullptr, nullptr, nullptr};
    unsigned borrowed = 0;          // bit s: ws[s] belongs to the parent
};

// Event bracket around one launch when timing is on (no-ops otherwise).
void d2_time_begin(d2_ctx* ctx, int kind, cudaStream_t st);
void d2_time_end(d2_ctx* ctx, cudaStream_t st);

// Device error flags (atomicOr'ed by kernels instead of faulting).
#define D2F_BAD_OFFSETS   0x01
#define D2F_BAD_WEIGHTS   0x02
#define D2F_BAD_VOCAB     0x04
#define D2F_BAD_MEMBER    0x08
#define D2F_PIVOT_LIMIT   0x10   // an exact W^2 solve reached its phase cap (sticky word)
#define D2F_BAD_SIZE      0x20
#define D2F_DEV_TIMEOUT   0x40   // a bounded device-side wait expired
// Word of dev_flags that accumulates sticky device errors (read and cleared
// by d2_device_errors); word 0 is per-call validation scratch.
#define D2_DEV_ERR_WORD   1

int d2_fail(d2_ctx* ctx, int code, const char* fmt, ...);
int d2_cuda_fail(d2_ctx* ctx, cudaError_t e, const char* what);
// Pointer to workspace `slot` with at least `bytes` bytes (grows on demand).
int d2_ws(d2_ctx* ctx, int slot, size_t bytes, void** out);

#define D2_CK(ctx, call)                                          \
    do {                                                          \
        cudaError_t e__ = (call);                                 \
        if (e__ != cudaSuccess) return d2_cuda_fail(ctx, e__, #call); \
    } while (0)

#define D2_LAUNCH_CK(ctx, what)                                   \
    do {                                                          \
        (ctx)->launches++;                                        \
        cudaError_t e__ = cudaGetLastError();                     \
        if (e__ != cudaSuccess) return d2_cuda_fail(ctx, e__, what); \
    } while (0)

static inline cudaStream_t d2_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

static inline int64_t d2_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Host-side validation of a bag descriptor (pointers and sizes only):
// coordinate bags (dense or through a point table), or symbolic bags.
int d2_check_bags_host(d2_ctx* ctx, const d2_bags* b);
int d2_check_sym_bags_host(d2_ctx* ctx, const d2_bags* b);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Support row `row` of a bag set, dense or through the vocabulary.
__device__ __forceinline__ const float* d2_row_ptr(const float* supp, const int32_t* vidx,
                                                   const float* vocab, int d, int64_t row) {
    return supp ? supp + row * (int64_t)d : vocab + (int64_t)vidx[row] * d;
}

template <int W>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int W>
__device__ __forceinline__ float group_max(float v) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int W>
__device__ __forceinline__ float group_min(float v) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int W>
__device__ __forceinline__ double group_sum_d(double v) {
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Chunk of consecutive member positions [p0, p1) that all belong to cluster c.
struct Chunk {
    int64_t p0, p1;
    int32_t c, pad;
};

// Members per chunk for the per-chunk kernels (cost build, support update).
#define D2_CHUNK 64

// Per-cluster layout inside WS_CLUSTER (offsets in bytes computed on host).
struct ClusterWs {
    float* rho;       // K
    float* beta;      // K   log2(e) / rho
    float* mu;        // K x d      centre used for the cost (mean of x_c)
    float* xt;        // K x m x d  x_c - mu_c
    float* xn;        // K x m      ||x_c,i - mu_c||^2
    float* wb[2];     // K x m      double-buffered barycenter weights (FP32)
    double* w64;      // K x m      FP64 weights of the last consensus
    int* counters;    // K          arrivals per cluster in the current sweep
    double* csum;     // K          FP64 cost sum (rho)
    int64_t* nrows;   // K          support rows per cluster
    int64_t* chunk_first;  // K+1   chunk range of each cluster
    int64_t* nchunks;      // 1     total chunks
    Chunk* chunks;         // chunk table (bound: ceil(P/CH) + K)
};

int d2_cluster_ws(d2_ctx* ctx, int64_t K, int m, int d, int64_t P, ClusterWs* cw);

// Builds the member-position -> cluster map and the chunk table.
int d2_setup_clusters(d2_ctx* ctx, const int64_t* cofs, int64_t P, int K, int32_t** pos_cluster,
                      ClusterWs* cw, cudaStream_t st);

// Centre and norms of each barycenter (mu_c, x_c - mu_c, ||x_c,i - mu_c||^2).
int d2_prep_x(d2_ctx* ctx, const float* x, int K, int m, int d, const ClusterWs& cw, cudaStream_t st);

// Cost precision requested by a flags word: 0 (FP32 CUDA cores),
// D2_COST_BF16, D2_COST_BF16X3 or D2_COST_BF16X6 (tensor cores, where they apply).
static inline int d2_cost_prec(int flags) {
    if ((flags & D2_COST_BF16X6) == D2_COST_BF16X6) return D2_COST_BF16X6;
    return (flags & D2_COST_BF16X3) ? D2_COST_BF16X3 : (flags & D2_COST_BF16) ? D2_COST_BF16 : 0;
}

// Sets the launch attributes d2_cost_rows will need (done before a capture).
int d2_cost_prepare(d2_ctx* ctx, const d2_bags* b, int m, int prec);

// Tensor-core build (cost_tc.cu); *used = false when (d, m, prec) is outside
// what it covers, and then nothing is launched.
int d2_cost_tc_prepare(d2_ctx* ctx, const d2_bags* b, int m, int prec, bool* used);
int d2_cost_tc_rows(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t maxch, int m, int prec,
                    const ClusterWs& cw, float* C, double* chunk_sum, int64_t* chunk_rows, cudaStream_t st,
                    bool* used);

// Tensor-core support partials (support_tc.cu): applies with a tensor-core
// cost precision, d >= 32 and m <= 128; partial sums of the centred support
// per chunk into xpart (chunk x m x d).
bool d2_support_tc_applies(const d2_bags* b, int m, int prec);
int d2_support_tc_prepare(d2_ctx* ctx, const d2_bags* b, int m, int prec);
int d2_support_tc(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t maxch, int m, int prec,
                  const float* plan, const ClusterWs& cw, float* xpart, cudaStream_t st);

// Symbolic supports (symbolic.cu): cost rows gathered from the bags' symbol
// table for the centroid symbols csym (K x m), with the FP64 chunk sums of
// Eq. rho when chunk_sum is given; the exact assignment on those costs
// (counters: solves, fall-backs, phase-cap hits; cleared here).
int d2_sym_cost_rows(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t P, int K, int m,
                     const int32_t* csym, const ClusterWs& cw, float* C, double* chunk_sum, int64_t* chunk_rows,
                     cudaStream_t st);
int d2_assign_sym_impl(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const int32_t* csym,
                       const float* w, int32_t* labels, float* dist, int64_t* counters, cudaStream_t st);

// Exact fixed-point cross-member reductions (reduce.cu), reduced across
// processes by the installed reducer.  gcount: K + 1 int64 (member counts
// per cluster over every process, then their total).
int d2_reduce(d2_ctx* ctx, int op, int64_t* buf, int64_t count, cudaStream_t st);
int d2_fx_counts(d2_ctx* ctx, int K, const int64_t* cofs, int64_t* gcount, cudaStream_t st);
int d2_fx_consensus(d2_ctx* ctx, int K, int m, const Chunk* chunks, const int64_t* nchunks, int64_t maxch,
                    const float* pos_part, bool r2, const int64_t* gcount, long long* S, float* w_next,
                    double* w_next64, cudaStream_t st);
int d2_fx_rho(d2_ctx* ctx, int K, int m, const int64_t* chunk_first, const double* chunk_sum,
              const int64_t* chunk_rows, const int64_t* gcount, double rho0, double rho_fixed, float* rho,
              float* beta, int64_t* nrows, long long* fx, cudaStream_t st);
int d2_fx_support(d2_ctx* ctx, int K, int m, int d, const int64_t* chunk_first, int64_t nseg, const float* xpart,
                  const int64_t* gcount, const float* w, const float* mu, float* x, long long* fx, cudaStream_t st);
int d2_fx_finish(d2_ctx* ctx, int K, int m, const int64_t* cofs, const double* pos_obj, const int64_t* gcount,
                 const float* wfin, float* w_out, double* obj, long long* fx, cudaStream_t st);

// Builds the chunk table of a cluster-offsets array (no position map).
int d2_build_chunks(d2_ctx* ctx, const int64_t* cofs, int K, const ClusterWs& cw, cudaStream_t st);

// Whether the tensor-core build covers (d, m, prec) for these bags.
bool d2_cost_tc_applies(const d2_bags* b, int m, int prec);

// Vocabulary cost table (cost_vocab.cu): used for bags stored as vocabulary
// indices when the tensor-core build applies, unless flags has D2_COST_ROWS.
enum { D2_VT_OFF = 0, D2_VT_SETUP = 1, D2_VT_REUSE = 2 };
bool d2_vocab_table_applies(const d2_bags* b, int K, int m, int prec, int flags);
// Sizes its workspaces (before a graph capture, so the capture allocates nothing).
int d2_vocab_reserve(d2_ctx* ctx, const d2_bags* b, int K, int m, const ClusterWs& cw);
int d2_vocab_cost_rows(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t P, int K, int m,
                       const ClusterWs& cw, float* C, double* chunk_sum, int64_t* chunk_rows, bool setup,
                       int prec, cudaStream_t st);

// Cost rows of every member position; FP64 sums per chunk for Eq. (rho) when
// want_sums.  vt: D2_VT_OFF builds every row directly; D2_VT_SETUP builds the
// vocabulary table's word lists for this membership first; D2_VT_REUSE reuses
// the lists of the previous D2_VT_SETUP call with the same membership.
int d2_cost_rows(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t P, int K, int m,
                 const ClusterWs& cw, float* C, bool want_sums, int prec, int vt, cudaStream_t st);
int d2_cost_rows_direct(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t P, int K, int m,
                        const ClusterWs& cw, float* C, double* chunk_sum, int64_t* chunk_rows, int prec,
                        cudaStream_t st);
