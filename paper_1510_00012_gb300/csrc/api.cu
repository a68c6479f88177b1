// Context, errors, workspaces, bag validation and the per-call cluster set-up
// shared by the cost build and the B-ADMM barycenter update.
#include <cstdarg>
#include <cstring>
#include <vector>

#include "d2_internal.cuh"

// ---------------------------------------------------------------------------
// errors and context
// ---------------------------------------------------------------------------

int d2_fail(d2_ctx* ctx, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return code;
}

int d2_cuda_fail(d2_ctx* ctx, cudaError_t e, const char* what) {
    int code = (e == cudaErrorMemoryAllocation) ? D2_ENOMEM : D2_ECUDA;
    return d2_fail(ctx, code, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

extern "C" void d2_badmm_opts_default(d2_badmm_opts* o) {
    if (!o) return;
    o->rho0 = 2.0;
    o->rho = 0.0;
    o->eps = 1e-16;
    o->iters = 100;
    o->tau = 10;
    o->rule = D2_RULE_R1;
    o->flags = 0;
}

extern "C" d2_ctx* d2_create(int device) {
    if (cudaSetDevice(device) != cudaSuccess) return nullptr;
    d2_ctx* ctx = new d2_ctx();
    ctx->device = device;
    if (cudaMalloc(&ctx->dev_flags, 64) != cudaSuccess) {
        delete ctx;
        return nullptr;
    }
    cudaMemset(ctx->dev_flags, 0, 64);
    return ctx;
}

extern "C" void d2_destroy(d2_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& t : ctx->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    for (int h = 0; h < 2; ++h) {
        if (ctx->child[h]) d2_destroy(ctx->child[h]);
        if (ctx->cstream[h]) cudaStreamDestroy(ctx->cstream[h]);
    }
    for (int e = 0; e < 3; ++e)
        if (ctx->cev[e]) cudaEventDestroy(ctx->cev[e]);
    for (int s = 0; s < WS_NSLOTS; ++s)
        if (ctx->ws[s] && !((ctx->borrowed >> s) & 1u)) cudaFree(ctx->ws[s]);
    if (ctx->dev_flags) cudaFree(ctx->dev_flags);
    delete ctx;
}

extern "C" const char* d2_last_error(const d2_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

extern "C" size_t d2_workspace_bytes(const d2_ctx* ctx) {
    if (!ctx) return 0;
    size_t t = 0;
    for (int s = 0; s < WS_NSLOTS; ++s) t += ctx->ws_bytes[s];
    return t;
}

// ---------------------------------------------------------------------------
// instrumentation
// ---------------------------------------------------------------------------

static cudaEvent_t take_event(d2_ctx* ctx) {
    cudaEvent_t e = nullptr;
    if (!ctx->ev_pool.empty()) {
        e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
    } else {
        cudaEventCreate(&e);
    }
    return e;
}

void d2_time_begin(d2_ctx* ctx, int kind, cudaStream_t st) {
    if (!ctx->timing) return;
    TimedLaunch t;
    t.kind = kind;
    t.a = take_event(ctx);
    t.b = take_event(ctx);
    cudaEventRecord(t.a, st);
    ctx->timed.push_back(t);
}

void d2_time_end(d2_ctx* ctx, cudaStream_t st) {
    if (!ctx->timing || ctx->timed.empty()) return;
    cudaEventRecord(ctx->timed.back().b, st);
}

static void drain_timing(d2_ctx* ctx) {
    for (auto& t : ctx->timed) {
        float ms = 0.f;
        cudaEventSynchronize(t.b);
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            ctx->t_ms[t.kind] += ms;
            ctx->t_n[t.kind] += 1;
        }
        cudaGetLastError();
        ctx->ev_pool.push_back(t.a);
        ctx->ev_pool.push_back(t.b);
    }
    ctx->timed.clear();
}

extern "C" int d2_timing_enable(d2_ctx* ctx, int on) {
    if (!ctx) return D2_EINVAL;
    for (int h = 0; h < 2; ++h)
        if (ctx->child[h]) d2_timing_enable(ctx->child[h], on);
    drain_timing(ctx);
    for (int k = 0; k < D2_KT_COUNT; ++k) {
        ctx->t_ms[k] = 0.0;
        ctx->t_n[k] = 0;
    }
    ctx->timing = on != 0;
    return D2_OK;
}

extern "C" int d2_timing_read(d2_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx) return D2_EINVAL;
    drain_timing(ctx);
    for (int k = 0; k < D2_KT_COUNT; ++k) {
        if (ms) ms[k] = ctx->t_ms[k];
        if (launches) launches[k] = ctx->t_n[k];
    }
    // launches of split calls run in the child contexts (concurrently: their
    // times add up to more than the wall time)
    for (int h = 0; h < 2; ++h) {
        if (!ctx->child[h]) continue;
        double cm[D2_KT_COUNT];
        int64_t cn[D2_KT_COUNT];
        d2_timing_read(ctx->child[h], cm, cn);
        for (int k = 0; k < D2_KT_COUNT; ++k) {
            if (ms) ms[k] += cm[k];
            if (launches) launches[k] += cn[k];
        }
    }
    return D2_OK;
}

extern "C" int64_t d2_launch_count(const d2_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" int d2_device_errors(d2_ctx* ctx, int32_t* bits) {
    if (!ctx) return D2_EINVAL;
    D2_CK(ctx, cudaSetDevice(ctx->device));
    int v = 0;
    int* word = ctx->dev_flags + D2_DEV_ERR_WORD;
    D2_CK(ctx, cudaDeviceSynchronize());
    D2_CK(ctx, cudaMemcpy(&v, word, sizeof(int), cudaMemcpyDeviceToHost));
    D2_CK(ctx, cudaMemset(word, 0, sizeof(int)));
    if (bits) *bits = v;
    if (v & D2F_DEV_TIMEOUT) return d2_fail(ctx, D2_ETIMEOUT, "a bounded device-side wait expired");
    if (v & D2F_PIVOT_LIMIT)
        return d2_fail(ctx, D2_ENOCONV, "an exact W^2 solve reached its phase cap (its value and label are wrong)");
    return D2_OK;
}

extern "C" int d2_set_reducer(d2_ctx* ctx, d2_reducer_fn fn, void* user) {
    if (!ctx) return D2_EINVAL;
    ctx->reducer = fn;
    ctx->reducer_user = fn ? user : nullptr;
    return D2_OK;
}

extern "C" int d2_set_flow_store(d2_ctx* ctx, int32_t store, int32_t pool_cap) {
    if (!ctx || store < 0 || store > 2 || pool_cap < 0) return D2_EINVAL;
    ctx->flow_store = store;
    ctx->pool_cap = pool_cap;
    return D2_OK;
}

extern "C" int d2_set_bound_kernels(d2_ctx* ctx, int32_t path) {
    if (!ctx || path < 0 || path > 1) return D2_EINVAL;
    ctx->bound_cuda_cores = path;
    return D2_OK;
}

extern "C" int d2_set_prune_forward(d2_ctx* ctx, int32_t path) {
    if (!ctx || path < 0 || path > 1) return D2_EINVAL;
    ctx->mlp_cuda_cores = path;
    return D2_OK;
}

extern "C" int d2_set_dual_bound(d2_ctx* ctx, int32_t iters, float eps_rel) {
    if (!ctx || iters < -1 || iters > 10000 || !(eps_rel >= 0.f) || eps_rel > 100.f) return D2_EINVAL;
    ctx->dual_iters = iters;
    ctx->dual_eps = eps_rel;
    return D2_OK;
}

extern "C" int d2_set_phase_limit(d2_ctx* ctx, int32_t max_phases) {
    if (!ctx || max_phases < 0) return D2_EINVAL;
    ctx->phase_limit = max_phases;
    return D2_OK;
}

int d2_ws(d2_ctx* ctx, int slot, size_t bytes, void** out) {
    if (bytes == 0) bytes = 256;
    if (((ctx->borrowed >> slot) & 1u) && ctx->ws_bytes[slot] < bytes)
        return d2_fail(ctx, D2_EINVAL, "workspace slot %d lent by the parent is too small", slot);
    if (ctx->ws_bytes[slot] < bytes) {
        if (ctx->ws[slot]) {
            cudaDeviceSynchronize();  // a pending kernel may still use it
            cudaFree(ctx->ws[slot]);
            ctx->ws[slot] = nullptr;
            ctx->ws_bytes[slot] = 0;
        }
        size_t want = bytes + bytes / 8;  // headroom for slightly larger calls
        want = (want + 4095) & ~(size_t)4095;
        cudaError_t e = cudaMalloc(&ctx->ws[slot], want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            e = cudaMalloc(&ctx->ws[slot], bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ctx->ws[slot] = nullptr;
                return d2_fail(ctx, D2_ENOMEM, "workspace slot %d: cannot allocate %zu bytes", slot, bytes);
            }
            want = bytes;
        }
        ctx->ws_bytes[slot] = want;
        ctx->generation++;
    }
    *out = ctx->ws[slot];
    return D2_OK;
}

int d2_check_bags_host(d2_ctx* ctx, const d2_bags* b) {
    if (!b) return d2_fail(ctx, D2_EINVAL, "bags is NULL");
    if (b->symcost) return d2_fail(ctx, D2_EINVAL, "bags: symbolic bags need the *_sym entry points");
    if (b->N < 1 || b->n < 1 || b->d < 1 || b->max_mk < 1)
        return d2_fail(ctx, D2_EINVAL, "bags: need N, n, d, max_mk >= 1 (got %lld, %lld, %d, %d)",
                       (long long)b->N, (long long)b->n, b->d, b->max_mk);
    if (!b->offsets || !b->wt) return d2_fail(ctx, D2_EINVAL, "bags: offsets and wt are required");
    bool dense = b->supp != nullptr;
    bool voc = b->vocab_idx != nullptr && b->vocab != nullptr && b->V >= 1;
    if (dense == voc) return d2_fail(ctx, D2_EINVAL, "bags: give exactly one of supp or (vocab_idx, vocab, V)");
    if (dense && (reinterpret_cast<uintptr_t>(b->supp) & 15))
        return d2_fail(ctx, D2_EINVAL, "bags: supp must be 16-byte aligned");
    return D2_OK;
}

int d2_check_sym_bags_host(d2_ctx* ctx, const d2_bags* b) {
    if (!b) return d2_fail(ctx, D2_EINVAL, "bags is NULL");
    if (b->N < 1 || b->n < 1 || b->max_mk < 1 || b->V < 1)
        return d2_fail(ctx, D2_EINVAL, "symbolic bags: need N, n, max_mk, V >= 1");
    if (!b->offsets || !b->wt || !b->vocab_idx || !b->symcost)
        return d2_fail(ctx, D2_EINVAL, "symbolic bags: offsets, wt, vocab_idx (symbols) and symcost are required");
    if (b->supp || b->vocab) return d2_fail(ctx, D2_EINVAL, "symbolic bags: supp and vocab must be NULL");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// bag validation on the device
// ---------------------------------------------------------------------------

__global__ void k_check_bags(d2_bags b, int* flags) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k == 0) {
        if (b.offsets[0] != 0 || b.offsets[b.N] != b.n) atomicOr(flags, D2F_BAD_OFFSETS);
    }
    if (k >= b.N) return;
    int64_t a = b.offsets[k], e = b.offsets[k + 1];
    int64_t mk = e - a;
    if (mk < 1 || mk > b.max_mk || a < 0 || e > b.n) {
        atomicOr(flags, D2F_BAD_OFFSETS);
        return;
    }
    double s = 0.0;
    bool bad = false;
    for (int64_t r = a; r < e; ++r) {
        float v = b.wt[r];
        if (!(v >= 0.0f) || !isfinite(v)) bad = true;
        s += v;
        if (b.vocab_idx) {
            int32_t id = b.vocab_idx[r];
            if (id < 0 || id >= b.V) atomicOr(flags, D2F_BAD_VOCAB);
        }
    }
    if (bad || fabs(s - 1.0) > 1e-5) atomicOr(flags, D2F_BAD_WEIGHTS);
}

extern "C" int d2_check_bags(d2_ctx* ctx, const d2_bags* bags, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = (bags && bags->symcost) ? d2_check_sym_bags_host(ctx, bags) : d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    cudaStream_t st = d2_stream(stream);
    D2_CK(ctx, cudaMemsetAsync(ctx->dev_flags, 0, sizeof(int), st));
    int64_t nb = d2_ceil_div(bags->N, 256);
    k_check_bags<<<(unsigned)nb, 256, 0, st>>>(*bags, ctx->dev_flags);
    D2_LAUNCH_CK(ctx, "k_check_bags");
    int flags = 0;
    D2_CK(ctx, cudaMemcpyAsync(&flags, ctx->dev_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    D2_CK(ctx, cudaStreamSynchronize(st));
    if (flags & D2F_BAD_OFFSETS)
        return d2_fail(ctx, D2_EINVAL, "bags: offsets must start at 0, end at n, and give 1 <= m_k <= max_mk");
    if (flags & D2F_BAD_WEIGHTS)
        return d2_fail(ctx, D2_EINVAL, "bags: weights must be finite, >= 0 and sum to 1 (+-1e-5) per bag");
    if (flags & D2F_BAD_VOCAB) return d2_fail(ctx, D2_EINVAL, "bags: vocabulary index out of [0, V)");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// per-call cluster set-up
// ---------------------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int d2_cluster_ws(d2_ctx* ctx, int64_t K, int m, int d, int64_t P, ClusterWs* cw) {
    int64_t maxch = d2_ceil_div(P, D2_CHUNK) + K + 1;
    size_t off = 0;
    size_t o_rho = off;   off += align256(K * 4);
    size_t o_beta = off;  off += align256(K * 4);
    size_t o_mu = off;    off += align256((size_t)K * d * 4);
    size_t o_xt = off;    off += align256((size_t)K * m * d * 4);
    size_t o_xn = off;    off += align256((size_t)K * m * 4);
    size_t o_wb0 = off;   off += align256((size_t)K * m * 4);
    size_t o_wb1 = off;   off += align256((size_t)K * m * 4);
    size_t o_w64 = off;   off += align256((size_t)K * m * 8);
    size_t o_cnt = off;   off += align256(K * 4);
    size_t o_csum = off;  off += align256(K * 8);
    size_t o_nrows = off; off += align256(K * 8);
    size_t o_cf = off;    off += align256((K + 1) * 8);
    size_t o_nch = off;   off += align256(8);
    size_t o_ch = off;    off += align256(maxch * sizeof(Chunk));
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_CLUSTER, off, &base);
    if (rc) return rc;
    char* b = static_cast<char*>(base);
    cw->rho = reinterpret_cast<float*>(b + o_rho);
    cw->beta = reinterpret_cast<float*>(b + o_beta);
    cw->mu = reinterpret_cast<float*>(b + o_mu);
    cw->xt = reinterpret_cast<float*>(b + o_xt);
    cw->xn = reinterpret_cast<float*>(b + o_xn);
    cw->wb[0] = reinterpret_cast<float*>(b + o_wb0);
    cw->wb[1] = reinterpret_cast<float*>(b + o_wb1);
    cw->w64 = reinterpret_cast<double*>(b + o_w64);
    cw->counters = reinterpret_cast<int*>(b + o_cnt);
    cw->csum = reinterpret_cast<double*>(b + o_csum);
    cw->nrows = reinterpret_cast<int64_t*>(b + o_nrows);
    cw->chunk_first = reinterpret_cast<int64_t*>(b + o_cf);
    cw->nchunks = reinterpret_cast<int64_t*>(b + o_nch);
    cw->chunks = reinterpret_cast<Chunk*>(b + o_ch);
    return D2_OK;
}

// position -> cluster by binary search: the last c in [0, K) with cofs[c] <= p
__global__ void k_pos_cluster(const int64_t* cofs, int K, int64_t P, int32_t* pos_cluster) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    int lo = 0, hi = K - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cofs[mid] <= p) lo = mid; else hi = mid - 1;
    }
    pos_cluster[p] = lo;
}

// exclusive scan of ceil(N_c / CH) over clusters in one block; writes
// chunk_first[0..K] and the total.
__global__ void k_chunk_scan(const int64_t* cofs, int K, int64_t* chunk_first, int64_t* total) {
    __shared__ int64_t s[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < K; base += 1024) {
        int c = base + threadIdx.x;
        int64_t v = 0;
        if (c < K) v = (cofs[c + 1] - cofs[c] + D2_CHUNK - 1) / D2_CHUNK;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
            int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (c < K) chunk_first[c] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        chunk_first[K] = carry;
        *total = carry;
    }
}

__global__ void k_chunk_fill(const int64_t* cofs, int K, const int64_t* chunk_first, Chunk* chunks) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    int64_t q = chunk_first[c];
    for (int64_t p = cofs[c]; p < cofs[c + 1]; p += D2_CHUNK, ++q) {
        Chunk ch;
        ch.p0 = p;
        ch.p1 = min(p + (int64_t)D2_CHUNK, cofs[c + 1]);
        ch.c = c;
        ch.pad = 0;
        chunks[q] = ch;
    }
}

int d2_build_chunks(d2_ctx* ctx, const int64_t* cofs, int K, const ClusterWs& cw, cudaStream_t st) {
    k_chunk_scan<<<1, 1024, 0, st>>>(cofs, K, cw.chunk_first, cw.nchunks);
    D2_LAUNCH_CK(ctx, "k_chunk_scan");
    k_chunk_fill<<<(unsigned)d2_ceil_div(K, 256), 256, 0, st>>>(cofs, K, cw.chunk_first, cw.chunks);
    D2_LAUNCH_CK(ctx, "k_chunk_fill");
    return D2_OK;
}

int d2_setup_clusters(d2_ctx* ctx, const int64_t* cofs, int64_t P, int K, int32_t** pos_cluster,
                      ClusterWs* cw, cudaStream_t st) {
    void* pc = nullptr;
    int rc = d2_ws(ctx, WS_POS_CLUSTER, (size_t)P * 4, &pc);
    if (rc) return rc;
    *pos_cluster = static_cast<int32_t*>(pc);
    if (P > 0) {
        k_pos_cluster<<<(unsigned)d2_ceil_div(P, 256), 256, 0, st>>>(cofs, K, P, *pos_cluster);
        D2_LAUNCH_CK(ctx, "k_pos_cluster");
    }
    k_chunk_scan<<<1, 1024, 0, st>>>(cofs, K, cw->chunk_first, cw->nchunks);
    D2_LAUNCH_CK(ctx, "k_chunk_scan");
    k_chunk_fill<<<(unsigned)d2_ceil_div(K, 256), 256, 0, st>>>(cofs, K, cw->chunk_first, cw->chunks);
    D2_LAUNCH_CK(ctx, "k_chunk_fill");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// barycenter centring: mu_c = mean_i x_c,i ; xt = x - mu ; xn = ||xt||^2
// ---------------------------------------------------------------------------

__global__ void k_prep_x(const float* x, int m, int d, float* mu, float* xt, float* xn) {
    int c = blockIdx.x;
    const float* xc = x + (int64_t)c * m * d;
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
        float s = 0.f;
        for (int i = 0; i < m; ++i) s += xc[(int64_t)i * d + t];
        mu[(int64_t)c * d + t] = s / (float)m;
    }
    __syncthreads();
    for (int i = threadIdx.x >> 5; i < m; i += blockDim.x >> 5) {
        float s = 0.f;
        for (int t = threadIdx.x & 31; t < d; t += 32) {
            float v = xc[(int64_t)i * d + t] - mu[(int64_t)c * d + t];
            xt[((int64_t)c * m + i) * d + t] = v;
            s += v * v;
        }
        s = group_sum<32>(s);
        if ((threadIdx.x & 31) == 0) xn[(int64_t)c * m + i] = s;
    }
}

int d2_prep_x(d2_ctx* ctx, const float* x, int K, int m, int d, const ClusterWs& cw, cudaStream_t st) {
    if (K <= 0) return D2_OK;
    k_prep_x<<<K, 256, 0, st>>>(x, m, d, cw.mu, cw.xt, cw.xn);
    D2_LAUNCH_CK(ctx, "k_prep_x");
    return D2_OK;
}
