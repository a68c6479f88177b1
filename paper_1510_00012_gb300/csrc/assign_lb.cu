// Exact assignment with certified lower bounds (assignment step of
// Algorithm 1; W^2 is the transportation LP of Eq. primal).
//
// For a bag P (points y_j, weights u_j) and a centroid Q (points x_i, weights
// v_i) with cost C_ij = ||x_i - y_j||^2, three quantities never exceed W^2:
//   * dropping the centroid-side marginal: each bag point ships all its mass
//     to its nearest centroid point,   LB1 = sum_j u_j min_i C_ij;
//   * dropping the bag-side marginal:  LB2 = sum_i v_i min_j C_ij;
//   * Jensen on the squared distance:  LB3 = ||mu_P - mu_Q||^2 (the means).
// (any plan feasible for the LP is feasible for each relaxation, and for LB3
// the plan's cost is at least the cost of moving the means).  The bounded
// assignment computes L = max(LB1, LB2, LB3) for every (bag, centroid) pair,
// solves each bag's r smallest-bound centroids exactly (or the pruner's r
// candidates), and then solves exactly every other centroid whose bound is
// not above the best value found, inflated by a slack that covers the FP32
// rounding of the bounds and of the solver.  A centroid left unsolved has
// W^2 >= L > best, so the argmin (ties -> lowest index) is the one the full
// N x K solve would return.
#include <algorithm>
#include <cstring>

#include "d2_internal.cuh"

// from assign.cu and prune.cu
int d2_solve_pair_list(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                       const int64_t* pair_bag, const int32_t* pair_cent, int64_t max_pairs,
                       const int64_t* npairs_dev, float* out, int64_t* fail_count, cudaStream_t st);
int d2_prune_candidates(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                        const d2_prune* p, int r, int32_t* cand, cudaStream_t st);

#define LB_WARPS 8
#define LB_JN 4          // bag points per lane: max_mk <= 128
#define LB_SLACK 1e-4f   // relative slack on the bound test

struct LbArgs {
    const int64_t* offsets;
    const float* supp;
    const int32_t* vidx;
    const float* vocab;
    const float* wt;
    int d, m, K, nmax, ystride;
    const float* x;    // K x m x d
    const float* w;    // K x m
    const float* xn;   // K x m   ||x_i||^2
    const float* mq;   // K x d   centroid means
    float* lb;         // N x K
    int64_t N;
};

// ||x_i||^2 and the weighted mean of every centroid
__global__ void k_centroid_stats(int K, int m, int d, const float* x, const float* w, float* xn, float* mq) {
    const int c = blockIdx.x;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const float* xi = x + ((int64_t)c * m + i) * d;
        float s = 0.f;
        for (int t = 0; t < d; ++t) s = fmaf(xi[t], xi[t], s);
        xn[(int64_t)c * m + i] = s;
    }
    for (int t = threadIdx.x; t < d; t += blockDim.x) {
        float s = 0.f;
        for (int i = 0; i < m; ++i) s = fmaf(w[(int64_t)c * m + i], x[((int64_t)c * m + i) * d + t], s);
        mq[(int64_t)c * d + t] = s;
    }
}

// One CTA per bag (grid-stride), the bag's rows in shared memory; warp w
// bounds centroids w, w + 8, ...; lanes own bag points j = lane + 32 t.
template <int JN>
__global__ void __launch_bounds__(LB_WARPS * 32) k_lb_pairs(LbArgs a) {
    extern __shared__ float lb_dyn[];
    const int rows = 32 * JN;                             // tile rows (>= max_mk)
    float* ys = lb_dyn;                                   // rows x ystride
    float* yn = ys + (size_t)rows * a.ystride;            // rows
    float* uy = yn + rows;                                // rows
    float* mp = uy + rows;                                // d
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d, m = a.m, K = a.K;
    for (int64_t bag = blockIdx.x; bag < a.N; bag += gridDim.x) {
        const int64_t r0 = a.offsets[bag];
        const int n = (int)(a.offsets[bag + 1] - r0);
        __syncthreads();
        for (int e = threadIdx.x; e < rows * d; e += blockDim.x) {
            const int j = e / d, t = e - j * d;
            ys[j * a.ystride + t] = j < n ? d2_row_ptr(a.supp, a.vidx, a.vocab, d, r0 + j)[t] : 0.f;
        }
        for (int j = threadIdx.x; j < n; j += blockDim.x) uy[j] = a.wt[r0 + j];
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            float s = 0.f;
            for (int t = 0; t < d; ++t) s = fmaf(ys[j * a.ystride + t], ys[j * a.ystride + t], s);
            yn[j] = s;
        }
        for (int t = threadIdx.x; t < d; t += blockDim.x) {
            float s = 0.f;
            for (int j = 0; j < n; ++j) s = fmaf(uy[j], ys[j * a.ystride + t], s);
            mp[t] = s;
        }
        __syncthreads();
        for (int c = warp; c < K; c += LB_WARPS) {
            const float* xc = a.x + (int64_t)c * m * d;
            float colmin[JN];
#pragma unroll
            for (int q = 0; q < JN; ++q) colmin[q] = 3.0e38f;
            float lb2 = 0.f;
            for (int i = 0; i < m; ++i) {
                const float* xi = xc + (int64_t)i * d;
                float dot[JN];
#pragma unroll
                for (int q = 0; q < JN; ++q) dot[q] = 0.f;
                for (int t = 0; t < d; ++t) {
                    const float xv = __ldg(xi + t);
#pragma unroll
                    for (int q = 0; q < JN; ++q) {
                        // rows past n read zero-initialised tail rows of the tile (harmless)
                        dot[q] = fmaf(xv, ys[(lane + 32 * q) * a.ystride + t], dot[q]);
                    }
                }
                const float xni = a.xn[(int64_t)c * m + i];
                float rmin = 3.0e38f;
#pragma unroll
                for (int q = 0; q < JN; ++q) {
                    const int j = lane + 32 * q;
                    if (j < n) {
                        const float cij = fmaxf(fmaf(-2.f, dot[q], xni + yn[j]), 0.f);
                        colmin[q] = fminf(colmin[q], cij);
                        rmin = fminf(rmin, cij);
                    }
                }
                rmin = group_min<32>(rmin);
                lb2 = fmaf(a.w[(int64_t)c * m + i], rmin, lb2);
            }
            float lb1 = 0.f;
#pragma unroll
            for (int q = 0; q < JN; ++q) {
                const int j = lane + 32 * q;
                if (j < n) lb1 = fmaf(uy[j], colmin[q], lb1);
            }
            lb1 = group_sum<32>(lb1);
            float lb3 = 0.f;
            for (int t = lane; t < d; t += 32) {
                const float df = mp[t] - a.mq[(int64_t)c * d + t];
                lb3 = fmaf(df, df, lb3);
            }
            lb3 = group_sum<32>(lb3);
            if (lane == 0) a.lb[bag * K + c] = fmaxf(fmaxf(lb1, lb2), lb3);
        }
    }
}

// Per bag: the r smallest bounds (ties: lower index) as first candidates,
// unless the pruner already wrote them.
__global__ void k_lb_first(int64_t N, int K, int r, const float* lb, int32_t* cand) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N) return;
    const float* row = lb + k * K;
    float bv[16];
    int bi[16];
    for (int t = 0; t < r; ++t) {
        bv[t] = 3.4e38f;
        bi[t] = 0x7fffffff;
    }
    for (int i = 0; i < K; ++i) {
        const float s = row[i];
        if (s < bv[r - 1]) {
            int pos = r - 1;
            while (pos > 0 && s < bv[pos - 1]) {
                bv[pos] = bv[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bv[pos] = s;
            bi[pos] = i;
        }
    }
    for (int t = 0; t < r; ++t) cand[k * r + t] = bi[t];
}

// First-pass values into D (N x K, +inf elsewhere) and the pair list of every
// other centroid whose bound does not exceed the best first-pass value.
__global__ void k_lb_second(int64_t N, int K, int r, const float* lb, const int32_t* cand, const float* w2c,
                            float* D, int64_t* pb, int32_t* pc, int64_t* npairs) {
    const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    float best = 3.4e38f;
    for (int t = 0; t < r; ++t) best = fminf(best, w2c[k * r + t]);
    const float thr = best * (1.f + LB_SLACK) + 1e-6f;
    for (int i = lane; i < K; i += 32) {
        bool is_c = false;
        float v = 3.4e38f;
        for (int t = 0; t < r; ++t)
            if (cand[k * r + t] == i) {
                is_c = true;
                v = w2c[k * r + t];
            }
        D[k * K + i] = v;
        if (!is_c && lb[k * K + i] <= thr) {
            const unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long*>(npairs), 1ull);
            pb[pos] = k;
            pc[pos] = i;
        }
    }
}

__global__ void k_scatter_list(const int64_t* npairs, const int64_t* pb, const int32_t* pc, const float* val, int K,
                               float* D) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= *npairs) return;
    D[pb[t] * K + pc[t]] = val[t];
}

__global__ void k_lb_count(int64_t* counters, const int64_t* npairs, int64_t first) {
    counters[0] += first + *npairs;
}

// from assign.cu
int d2_argmin_rows(d2_ctx* ctx, const float* D, int64_t N, int K, int32_t* labels, float* dist, cudaStream_t st);
int d2_prune_solve_pairs(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w, int mode,
                         int64_t npairs, const int64_t* npairs_dev, const int32_t* cand, int r,
                         const int64_t* bag_list, float* out, int64_t* fail_count, cudaStream_t st);

int d2_assign_bounded_impl(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                           const d2_prune* prune, int r_first, int32_t* labels, float* dist, int64_t* counters,
                           cudaStream_t st) {
    const int64_t N = b->N;
    const int d = b->d;
    if (b->max_mk > 32 * LB_JN)
        return d2_fail(ctx, D2_ENOTSUP, "bounded assignment: max_mk %d > %d", b->max_mk, 32 * LB_JN);
    const int r = std::max(1, std::min(r_first, std::min(K, 16)));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_lb = take((size_t)N * K * 4), o_D = take((size_t)N * K * 4), o_cand = take((size_t)N * r * 4),
                 o_w2c = take((size_t)N * r * 4), o_pb = take((size_t)N * K * 8), o_pc = take((size_t)N * K * 4),
                 o_val = take((size_t)N * K * 4), o_xn = take((size_t)K * m * 4), o_mq = take((size_t)K * d * 4),
                 o_cnt = take(64);
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_ASSIGN, off, &base);
    if (rc) return rc;
    char* bb = static_cast<char*>(base);
    float* lb = reinterpret_cast<float*>(bb + o_lb);
    float* D = reinterpret_cast<float*>(bb + o_D);
    int32_t* cand = reinterpret_cast<int32_t*>(bb + o_cand);
    float* w2c = reinterpret_cast<float*>(bb + o_w2c);
    int64_t* pb = reinterpret_cast<int64_t*>(bb + o_pb);
    int32_t* pc = reinterpret_cast<int32_t*>(bb + o_pc);
    float* val = reinterpret_cast<float*>(bb + o_val);
    float* xn = reinterpret_cast<float*>(bb + o_xn);
    float* mq = reinterpret_cast<float*>(bb + o_mq);
    int64_t* cnt = reinterpret_cast<int64_t*>(bb + o_cnt);

    // bounds for every pair
    d2_time_begin(ctx, D2_KT_ASSIGN, st);
    k_centroid_stats<<<K, 128, 0, st>>>(K, m, d, x, w, xn, mq);
    d2_time_end(ctx, st);
    D2_LAUNCH_CK(ctx, "k_centroid_stats");
    LbArgs a;
    a.offsets = b->offsets;
    a.supp = b->supp;
    a.vidx = b->vocab_idx;
    a.vocab = b->vocab;
    a.wt = b->wt;
    a.d = d;
    a.m = m;
    a.K = K;
    a.nmax = b->max_mk;
    a.ystride = d | 1;  // odd stride: lanes reading one column of consecutive rows hit distinct banks
    a.x = x;
    a.w = w;
    a.xn = xn;
    a.mq = mq;
    a.lb = lb;
    a.N = N;
    const int JN = b->max_mk <= 32 ? 1 : b->max_mk <= 64 ? 2 : 4;
    const size_t smem = ((size_t)32 * JN * a.ystride + 2 * (size_t)32 * JN + d) * 4;
    if (smem > 200 * 1024) return d2_fail(ctx, D2_ENOTSUP, "bounded assignment: bag tile of %zu bytes", smem);
    const void* fn = JN == 1 ? (const void*)k_lb_pairs<1> : JN == 2 ? (const void*)k_lb_pairs<2> : (const void*)k_lb_pairs<4>;
    if (smem > 48 * 1024) D2_CK(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 152, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    D2_CK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LB_WARPS * 32, smem));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(N, (int64_t)sms * std::max(per_sm, 1) * 4));
    d2_time_begin(ctx, D2_KT_ASSIGN, st);
    if (JN == 1) k_lb_pairs<1><<<grid, LB_WARPS * 32, smem, st>>>(a);
    else if (JN == 2) k_lb_pairs<2><<<grid, LB_WARPS * 32, smem, st>>>(a);
    else k_lb_pairs<4><<<grid, LB_WARPS * 32, smem, st>>>(a);
    d2_time_end(ctx, st);
    D2_LAUNCH_CK(ctx, "k_lb_pairs");
    // first candidates: the pruner's r, else the r smallest bounds
    if (prune) {
        if ((rc = d2_prune_candidates(ctx, b, K, m, x, w, prune, r, cand, st))) return rc;
    } else {
        k_lb_first<<<(unsigned)d2_ceil_div(N, 128), 128, 0, st>>>(N, K, r, lb, cand);
        D2_LAUNCH_CK(ctx, "k_lb_first");
    }
    if ((rc = d2_prune_solve_pairs(ctx, b, K, m, x, w, 3, N * r, nullptr, cand, r, nullptr, w2c, counters + 2, st)))
        return rc;
    // every other centroid whose bound is not above the best value found
    D2_CK(ctx, cudaMemsetAsync(cnt, 0, 8, st));
    k_lb_second<<<(unsigned)d2_ceil_div(N, 8), 256, 0, st>>>(N, K, r, lb, cand, w2c, D, pb, pc, cnt);
    D2_LAUNCH_CK(ctx, "k_lb_second");
    if ((rc = d2_solve_pair_list(ctx, b, K, m, x, w, pb, pc, N * K, cnt, val, counters + 2, st))) return rc;
    k_scatter_list<<<(unsigned)d2_ceil_div(N * K, 256), 256, 0, st>>>(cnt, pb, pc, val, K, D);
    D2_LAUNCH_CK(ctx, "k_scatter_list");
    k_lb_count<<<1, 1, 0, st>>>(counters, cnt, N * r);
    D2_LAUNCH_CK(ctx, "k_lb_count");
    return d2_argmin_rows(ctx, D, N, K, labels, dist, st);
}
