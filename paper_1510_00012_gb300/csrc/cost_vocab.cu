// Cost build for bags stored as vocabulary indices (the symbolic supports of
// Section 5): the cost row C[j, :] = (||x_c,i - y_j||^2)_i of a support point
// depends only on its cluster c and its word w = vocab_idx[j], and the bags of
// one cluster reuse words heavily (a Zipf-like word law), so each cluster's
// costs are built once per distinct word it uses and then gathered into the
// j-major rows.
//
//   setup (once per call; membership is fixed within it):
//     mark    flag[c, w] = 1 for every word of every member of cluster c
//     scan    slot[c, w] = rank of w among the words of c; U_c = their count
//     layout  table rows of cluster c: tbase[c] .. tbase[c] + U_c, cut into
//             pseudo-members of VT_ROWS rows (so the row builder's chunks of
//             <= 64 members hold <= 4,096 rows)
//     fill    words[tbase[c] + slot[c, w]] = w
//   each build:
//     table   T[t, :] by the ordinary row builder on the pseudo-members (rows
//             gathered from the vocabulary by `words`), in cluster c's frame
//     gather  C[j, :] = T[tbase[c] + slot[c, vocab_idx[j]], :]
//
// Every table row is computed by the same kernel and arithmetic as the direct
// build of a support row with that word, and the gather sums each chunk's
// rows for Eq. (rho) in the direct tensor-core build's order, so C and the
// sums are bitwise those of the direct build.
#include <algorithm>

#include "d2_internal.cuh"

namespace {

constexpr int VT_ROWS = 64;        // table rows per pseudo-member
constexpr int VT_GATHER = 128;     // gather threads per chunk (one row each per pass)

__global__ void k_vt_mark(const Chunk* chunks, const int64_t* nchunks, const int64_t* members,
                          const int64_t* offsets, const int32_t* vidx, int64_t V, uint8_t* flag, int* err) {
    const int64_t q = blockIdx.x;
    if (q >= *nchunks) return;
    const Chunk ch = chunks[q];
    uint8_t* fc = flag + (int64_t)ch.c * V;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t p = ch.p0 + warp; p < ch.p1; p += blockDim.x / 32) {
        const int64_t k = members[p];
        for (int64_t j = offsets[k] + lane; j < offsets[k + 1]; j += 32) {
            const int32_t w = vidx[j];
            if (w < 0 || w >= V) {
                atomicOr(err, D2F_BAD_VOCAB);
                continue;
            }
            fc[w] = 1;
        }
    }
}

// Exclusive scan of cluster c's word flags (one CTA per cluster).
__global__ void __launch_bounds__(1024) k_vt_scan(const uint8_t* flag, int64_t V, int32_t* slot, int64_t* ucount) {
    __shared__ int32_t s[1024];
    __shared__ int32_t carry;
    const int c = blockIdx.x, t = threadIdx.x;
    const uint8_t* fc = flag + (int64_t)c * V;
    int32_t* sc = slot + (int64_t)c * V;
    if (t == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < V; base += 1024) {
        const int64_t w = base + t;
        const int32_t v = w < V ? fc[w] : 0;
        s[t] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
            const int32_t u = t >= o ? s[t - o] : 0;
            __syncthreads();
            s[t] += u;
            __syncthreads();
        }
        if (w < V) sc[w] = carry + s[t] - v;
        __syncthreads();
        if (t == 1023) carry += s[1023];
        __syncthreads();
    }
    if (t == 0) ucount[c] = carry;
}

// Table bases and pseudo-member ranges of every cluster (one CTA).
__global__ void __launch_bounds__(1024) k_vt_layout(const int64_t* ucount, int K, int64_t* tbase, int64_t* pcofs) {
    __shared__ int64_t s[2][1024];
    __shared__ int64_t carry[2];
    const int t = threadIdx.x;
    if (t == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    for (int base = 0; base < K; base += 1024) {
        const int c = base + t;
        const int64_t u = c < K ? ucount[c] : 0;
        const int64_t np = (u + VT_ROWS - 1) / VT_ROWS;
        s[0][t] = u;
        s[1][t] = np;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t a0 = t >= o ? s[0][t - o] : 0, a1 = t >= o ? s[1][t - o] : 0;
            __syncthreads();
            s[0][t] += a0;
            s[1][t] += a1;
            __syncthreads();
        }
        if (c < K) {
            tbase[c] = carry[0] + s[0][t] - u;
            pcofs[c] = carry[1] + s[1][t] - np;
        }
        __syncthreads();
        if (t == 1023) {
            carry[0] += s[0][1023];
            carry[1] += s[1][1023];
        }
        __syncthreads();
    }
    if (t == 0) {
        tbase[K] = carry[0];
        pcofs[K] = carry[1];
    }
}

// Pseudo-member row ranges and ids, and the word of every table row (one CTA
// per cluster).
__global__ void k_vt_fill(const uint8_t* flag, const int32_t* slot, int64_t V, int K, const int64_t* tbase,
                          const int64_t* pcofs, int64_t* poff, int64_t* pmem, int32_t* words) {
    const int c = blockIdx.x;
    for (int64_t q = pcofs[c] + threadIdx.x; q < pcofs[c + 1]; q += blockDim.x) {
        poff[q] = tbase[c] + (q - pcofs[c]) * VT_ROWS;
        pmem[q] = q;
    }
    if (c == K - 1 && threadIdx.x == 0) poff[pcofs[K]] = tbase[K];
    const uint8_t* fc = flag + (int64_t)c * V;
    const int32_t* sc = slot + (int64_t)c * V;
    for (int64_t w = threadIdx.x; w < V; w += blockDim.x)
        if (fc[w]) words[tbase[c] + sc[w]] = (int32_t)w;
}

// C rows of every member of a chunk from the table.  Thread t copies local
// rows t, t + 128, ... (the direct tensor-core build's row-to-thread map) and
// sums each row in column groups of 4, so the chunk sums match it bitwise.
__global__ void __launch_bounds__(VT_GATHER) k_vt_gather(const Chunk* chunks, const int64_t* nchunks,
                                                         const int64_t* members, const int64_t* offsets,
                                                         const int32_t* vidx, int64_t V, const int32_t* slot,
                                                         const int64_t* tbase, const float* T, int m, float* C,
                                                         double* chunk_sum, int64_t* chunk_rows) {
    __shared__ int64_t s_rs[D2_CHUNK];
    __shared__ int s_pre[D2_CHUNK + 1];
    __shared__ double s_red[VT_GATHER / 32];
    const int64_t q = blockIdx.x;
    if (q >= *nchunks) return;
    const Chunk ch = chunks[q];
    const int nm = (int)(ch.p1 - ch.p0);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < nm) {
        const int64_t k = members[ch.p0 + tid];
        s_rs[tid] = offsets[k];
        s_pre[tid + 1] = (int)(offsets[k + 1] - offsets[k]);
    }
    __syncthreads();
    if (tid == 0) {
        s_pre[0] = 0;
        for (int t = 0; t < nm; ++t) s_pre[t + 1] += s_pre[t];
    }
    __syncthreads();
    const int R = s_pre[nm];
    const int64_t tb = tbase[ch.c];
    const int32_t* sc = slot + (int64_t)ch.c * V;
    double acc = 0.0;
    for (int lr = tid; lr < R; lr += VT_GATHER) {
        int lo = 0, hi = nm - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= lr) lo = mid; else hi = mid - 1;
        }
        const int64_t g = s_rs[lo] + (lr - s_pre[lo]);
        const int32_t w = vidx[g];
        float rs = 0.f;
        if (w >= 0 && w < V) {  // (an index outside the vocabulary was reported by k_vt_mark)
            const float4* src = reinterpret_cast<const float4*>(T + (tb + sc[w]) * m);
            float4* dst = reinterpret_cast<float4*>(C + g * m);
            for (int i = 0; i < m / 4; ++i) {
                const float4 o = __ldg(src + i);
                __stcs(dst + i, o);
                rs += (o.x + o.y) + (o.z + o.w);
            }
        }
        acc += (double)rs;
    }
    if (chunk_sum) {
        const double sv = group_sum_d<32>(acc);
        if (lane == 0) s_red[warp] = sv;
        __syncthreads();
        if (tid == 0) {
            double sum = 0.0;
            for (int w = 0; w < VT_GATHER / 32; ++w) sum += s_red[w];
            chunk_sum[q] = sum;
            chunk_rows[q] = R;
        }
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct VocabWs {
    uint8_t* flag;
    int32_t* slot;
    int64_t *ucount, *tbase, *pcofs, *poff, *pmem;
    int32_t* words;
    ClusterWs pcw;  // chunk table over the pseudo-members (cluster arrays shared with the caller's)
    float* T;
    int64_t rows_bound, pmem_bound;
};

int vocab_ws(d2_ctx* ctx, const d2_bags* b, int K, int m, const ClusterWs& cw, VocabWs* v) {
    const int64_t V = b->V;
    v->rows_bound = std::min<int64_t>(b->n, (int64_t)K * V);
    v->pmem_bound = d2_ceil_div(v->rows_bound, VT_ROWS) + K;
    const int64_t maxch = d2_ceil_div(v->pmem_bound, D2_CHUNK) + K + 1;
    size_t off = 0;
    const size_t o_flag = off;  off += align256((size_t)K * V);
    const size_t o_slot = off;  off += align256((size_t)K * V * 4);
    const size_t o_uc = off;    off += align256((size_t)K * 8);
    const size_t o_tb = off;    off += align256((size_t)(K + 1) * 8);
    const size_t o_pc = off;    off += align256((size_t)(K + 1) * 8);
    const size_t o_po = off;    off += align256((size_t)(v->pmem_bound + 1) * 8);
    const size_t o_pm = off;    off += align256((size_t)v->pmem_bound * 8);
    const size_t o_wd = off;    off += align256((size_t)v->rows_bound * 4);
    const size_t o_cf = off;    off += align256((size_t)(K + 1) * 8);
    const size_t o_nc = off;    off += align256(8);
    const size_t o_ch = off;    off += align256((size_t)maxch * sizeof(Chunk));
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_VOCAB, off, &base);
    if (rc) return rc;
    void* tp = nullptr;
    if ((rc = d2_ws(ctx, WS_VOCAB_T, (size_t)v->rows_bound * m * 4, &tp))) return rc;
    char* p = static_cast<char*>(base);
    v->flag = reinterpret_cast<uint8_t*>(p + o_flag);
    v->slot = reinterpret_cast<int32_t*>(p + o_slot);
    v->ucount = reinterpret_cast<int64_t*>(p + o_uc);
    v->tbase = reinterpret_cast<int64_t*>(p + o_tb);
    v->pcofs = reinterpret_cast<int64_t*>(p + o_pc);
    v->poff = reinterpret_cast<int64_t*>(p + o_po);
    v->pmem = reinterpret_cast<int64_t*>(p + o_pm);
    v->words = reinterpret_cast<int32_t*>(p + o_wd);
    v->pcw = cw;
    v->pcw.chunk_first = reinterpret_cast<int64_t*>(p + o_cf);
    v->pcw.nchunks = reinterpret_cast<int64_t*>(p + o_nc);
    v->pcw.chunks = reinterpret_cast<Chunk*>(p + o_ch);
    v->T = static_cast<float*>(tp);
    return D2_OK;
}

}  // namespace

bool d2_vocab_table_applies(const d2_bags* b, int K, int m, int prec, int flags) {
    if (!b->vocab_idx || (flags & D2_COST_ROWS)) return false;
    if (!d2_cost_tc_applies(b, m, prec) || m % 4 != 0) return false;
    // the per-(cluster, word) scan is O(K V): keep it within a few times the rows
    return (int64_t)K * b->V <= 4 * b->n + (1 << 20) && (int64_t)K * b->V < (1ll << 31);
}

int d2_vocab_reserve(d2_ctx* ctx, const d2_bags* b, int K, int m, const ClusterWs& cw) {
    VocabWs v;
    return vocab_ws(ctx, b, K, m, cw, &v);
}

int d2_vocab_cost_rows(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t P, int K, int m,
                       const ClusterWs& cw, float* C, double* chunk_sum, int64_t* chunk_rows, bool setup,
                       int prec, cudaStream_t st) {
    VocabWs v;
    int rc = vocab_ws(ctx, b, K, m, cw, &v);
    if (rc) return rc;
    const int64_t maxch = d2_ceil_div(P, D2_CHUNK) + K + 1;
    if (setup) {
        D2_CK(ctx, cudaMemsetAsync(v.flag, 0, (size_t)K * b->V, st));
        k_vt_mark<<<(unsigned)maxch, 256, 0, st>>>(cw.chunks, cw.nchunks, members, b->offsets, b->vocab_idx, b->V,
                                                   v.flag, ctx->dev_flags + D2_DEV_ERR_WORD);
        D2_LAUNCH_CK(ctx, "k_vt_mark");
        k_vt_scan<<<(unsigned)K, 1024, 0, st>>>(v.flag, b->V, v.slot, v.ucount);
        D2_LAUNCH_CK(ctx, "k_vt_scan");
        k_vt_layout<<<1, 1024, 0, st>>>(v.ucount, K, v.tbase, v.pcofs);
        D2_LAUNCH_CK(ctx, "k_vt_layout");
        k_vt_fill<<<(unsigned)K, 256, 0, st>>>(v.flag, v.slot, b->V, K, v.tbase, v.pcofs, v.poff, v.pmem, v.words);
        D2_LAUNCH_CK(ctx, "k_vt_fill");
        if ((rc = d2_build_chunks(ctx, v.pcofs, K, v.pcw, st))) return rc;
    }
    // the table: the row builder on the pseudo-members, one row per used word
    d2_bags tb = *b;
    tb.N = v.pmem_bound;
    tb.n = v.rows_bound;
    tb.offsets = v.poff;
    tb.vocab_idx = v.words;
    if ((rc = d2_cost_rows_direct(ctx, &tb, v.pmem, v.pmem_bound, K, m, v.pcw, v.T, nullptr, nullptr, prec, st)))
        return rc;
    d2_time_begin(ctx, D2_KT_COST, st);
    k_vt_gather<<<(unsigned)maxch, VT_GATHER, 0, st>>>(cw.chunks, cw.nchunks, members, b->offsets, b->vocab_idx,
                                                       b->V, v.slot, v.tbase, v.T, m, C, chunk_sum, chunk_rows);
    d2_time_end(ctx, st);
    D2_LAUNCH_CK(ctx, "k_vt_gather");
    return D2_OK;
}
