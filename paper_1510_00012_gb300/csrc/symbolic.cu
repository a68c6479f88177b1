// Symbolic supports (Sections 2 and 5): distributions over a symbolic set
// with a given symbol-to-symbol dissimilarity c(s, t) = symcost[s V + t].
// The centroids' supports are fixed symbols, so the cost matrices of
// Algorithm badmm are gathered from the table once per call (no support
// update, no rebuild), and the assignment's exact solver reads its cost
// tableau from the table.
#include "d2_internal.cuh"

// Cost rows of one chunk (<= D2_CHUNK members of one cluster) per CTA:
// C[(row j) m + i] = c(csym_c,i, symbol of row j); with chunk_sum the FP64 sum
// of the chunk's entries and its row count (for Eq. rho).
__global__ void __launch_bounds__(256) k_sym_cost(const int64_t* members, const int64_t* offsets,
                                                  const int32_t* sym, const float* symcost, int64_t V,
                                                  const int32_t* csym, int m, const Chunk* chunks,
                                                  const int64_t* nchunks, float* C, double* chunk_sum,
                                                  int64_t* chunk_rows) {
    __shared__ int64_t s_rs[D2_CHUNK];
    __shared__ int s_pre[D2_CHUNK + 1];
    __shared__ int32_t s_cs[256];
    __shared__ double s_red[8];
    const int64_t q = blockIdx.x;
    if (q >= *nchunks) return;
    const Chunk ch = chunks[q];
    const int nm = (int)(ch.p1 - ch.p0);
    const int tid = threadIdx.x;
    if (tid < nm) {
        const int64_t k = members[ch.p0 + tid];
        s_rs[tid] = offsets[k];
        s_pre[tid + 1] = (int)(offsets[k + 1] - offsets[k]);
    }
    for (int i = tid; i < m; i += blockDim.x) s_cs[i] = csym[(int64_t)ch.c * m + i];
    __syncthreads();
    if (tid == 0) {
        s_pre[0] = 0;
        for (int t = 0; t < nm; ++t) s_pre[t + 1] += s_pre[t];
    }
    __syncthreads();
    const int R = s_pre[nm];
    double acc = 0.0;
    int mb = 0;  // member of local row lr (rows are visited in increasing order per thread)
    for (int e = tid; e < R * m; e += blockDim.x) {
        const int lr = e / m, i = e - lr * m;
        while (mb + 1 < nm && s_pre[mb + 1] <= lr) ++mb;
        const int64_t g = s_rs[mb] + (lr - s_pre[mb]);
        const float v = symcost[(int64_t)s_cs[i] * V + sym[g]];
        C[g * m + i] = v;
        acc += (double)v;
    }
    if (chunk_sum) {
        acc = group_sum_d<32>(acc);
        if ((tid & 31) == 0) s_red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
            chunk_sum[q] = t;
            chunk_rows[q] = R;
        }
    }
}

int d2_sym_cost_rows(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t P, int K, int m,
                     const int32_t* csym, const ClusterWs& cw, float* C, double* chunk_sum, int64_t* chunk_rows,
                     cudaStream_t st) {
    const int64_t maxch = d2_ceil_div(P, D2_CHUNK) + K + 1;
    d2_time_begin(ctx, D2_KT_COST, st);
    k_sym_cost<<<(unsigned)maxch, 256, 0, st>>>(members, b->offsets, b->vocab_idx, b->symcost, b->V, csym, m,
                                                cw.chunks, cw.nchunks, C, chunk_sum, chunk_rows);
    d2_time_end(ctx, st);
    D2_LAUNCH_CK(ctx, "k_sym_cost");
    return D2_OK;
}

extern "C" int d2_sym_cost(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets,
                           const int64_t* members, int64_t P, int32_t K, int32_t m, const int32_t* csym,
                           float* C_out, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_sym_bags_host(ctx, bags);
    if (rc) return rc;
    if (K < 1 || m < 1 || m > 256 || P < 0 || !cluster_offsets || (P > 0 && !members) || !csym || !C_out)
        return d2_fail(ctx, D2_EINVAL, "d2_sym_cost: need K >= 1, 1 <= m <= 256 and non-NULL arrays");
    if (P == 0) return D2_OK;
    cudaStream_t st = d2_stream(stream);
    ClusterWs cw;
    if ((rc = d2_cluster_ws(ctx, K, m, 1, P, &cw))) return rc;
    int32_t* pos_cluster = nullptr;
    if ((rc = d2_setup_clusters(ctx, cluster_offsets, P, K, &pos_cluster, &cw, st))) return rc;
    return d2_sym_cost_rows(ctx, bags, members, P, K, m, csym, cw, C_out, nullptr, nullptr, st);
}

int d2_assign_sym_exact(d2_ctx* ctx, const d2_bags* b, int K, int m, const int32_t* csym, const float* w,
                        int32_t* labels, float* dist, int64_t* counters, cudaStream_t st);

// counters: [0] exact solves, [1] fall-backs (0), [2] phase-cap hits
int d2_assign_sym_impl(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const int32_t* csym,
                       const float* w, int32_t* labels, float* dist, int64_t* counters, cudaStream_t st) {
    D2_CK(ctx, cudaMemsetAsync(counters, 0, 3 * sizeof(int64_t), st));
    return d2_assign_sym_exact(ctx, bags, K, m, csym, w, labels, dist, counters, st);
}

extern "C" int d2_assign_sym(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const int32_t* csym,
                             const float* w, int32_t* labels, float* dist, int64_t* stats, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_sym_bags_host(ctx, bags);
    if (rc) return rc;
    if (K < 1 || m < 1 || !csym || !w || !labels || !dist)
        return d2_fail(ctx, D2_EINVAL, "d2_assign_sym: need K >= 1, m >= 1 and non-NULL arrays");
    cudaStream_t st = d2_stream(stream);
    void* sc = nullptr;
    if ((rc = d2_ws(ctx, WS_SCAN, 64, &sc))) return rc;
    int64_t* counters = static_cast<int64_t*>(sc);
    if ((rc = d2_assign_sym_impl(ctx, bags, K, m, csym, w, labels, dist, counters, st))) return rc;
    if (stats) {
        D2_CK(ctx, cudaMemcpyAsync(stats, counters, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        D2_CK(ctx, cudaStreamSynchronize(st));
        if (stats[2] > 0)
            return d2_fail(ctx, D2_ENOCONV, "d2_assign_sym: %lld exact W^2 solves reached the phase cap",
                           (long long)stats[2]);
    }
    return D2_OK;
}
