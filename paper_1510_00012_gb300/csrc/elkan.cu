// Assignment with triangle-inequality skipping (Section 5: "skip unnecessary
// distance calculation by exploiting the triangle inequality of a metric"),
// following Elkan's bounds with the metric W = sqrt(W^2):
//   * every round, u_k = W(P_k, Q_{l_k}) is computed exactly (it also gives
//     the round's objective);
//   * centroid i != l_k is solved exactly only if u_k > lb_ki and
//     u_k > W(Q_{l_k}, Q_i) / 2; otherwise W(P_k, Q_i) >= u_k is certain;
//   * between rounds the lower bounds drop by the centroid shifts
//     W(Q_i^old, Q_i^new) (triangle inequality).
// Bounds are compared with a relative slack of 1e-5 so that FP32 rounding of
// the exact values never prunes a centroid that is not provably worse.  The
// label is the lowest index among the smallest solved W^2, as in d2_assign;
// a non-solved centroid at exactly the same W as the chosen one (a tie)
// would be the only difference from the full assignment.
#include <algorithm>
#include <cstring>

#include "d2_internal.cuh"

int d2_solve_pair_list(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                       const int64_t* pair_bag, const int32_t* pair_cent, int64_t max_pairs,
                       const int64_t* npairs_dev, float* out, int64_t* fail_count, cudaStream_t st);
int d2_assign_exact(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                    int32_t* labels, float* dist, int64_t* counters, cudaStream_t st);

#define EL_SLACK 1e-5f

__global__ void k_centroid_offsets(int K, int m, int64_t* off) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= K) off[i] = (int64_t)i * m;
}

// pairs (k, l_k) for every bag, then (i, i') for i < i' over centroids
__global__ void k_tight_pairs(int64_t N, const int32_t* labels, int64_t* pb, int32_t* pc) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < N) {
        pb[k] = k;
        pc[k] = labels[k];
    }
}
__global__ void k_cc_pairs(int K, int64_t* pb, int32_t* pc, int64_t* npairs) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)K * K;
    if (t == 0) *npairs = total;
    if (t < total) {
        pb[t] = t / K;          // "bag" = centroid i (centroids viewed as bags)
        pc[t] = (int32_t)(t % K);
    }
}
__global__ void k_shift_pairs(int K, int64_t* pb, int32_t* pc, int64_t* npairs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *npairs = K;
    if (i < K) {
        pb[i] = i;
        pc[i] = i;
    }
}

// half distance to the nearest other centroid; metric distances from W^2
__global__ void k_cc_finish(int K, const float* ccw2, float* ccd, float* half_min) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    float mn = 3.0e38f;
    for (int j = 0; j < K; ++j) {
        const float v = sqrtf(fmaxf(0.5f * (ccw2[(int64_t)i * K + j] + ccw2[(int64_t)j * K + i]), 0.f));
        ccd[(int64_t)i * K + j] = (i == j) ? 0.f : v;
        if (j != i) mn = fminf(mn, v);
    }
    half_min[i] = 0.5f * mn;
}

// bounds after the centroids moved by delta_i = W(Q_i^old, Q_i^new)
__global__ void k_shift_bounds(int64_t N, int K, const float* shw2, float* lb) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= N * K) return;
    const float di = sqrtf(fmaxf(shw2[e % K], 0.f));
    lb[e] = fmaxf(lb[e] - di * (1.f + EL_SLACK), 0.f);
}

// with exact u_k: list the centroids the bounds cannot rule out
__global__ void k_candidates(int64_t N, int K, const int32_t* labels, const float* tight_w2, const float* lb,
                             const float* ccd, const float* half_min, int64_t* pb, int32_t* pc, int64_t* npairs,
                             float* u) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int l = labels[k];
    const float uk = sqrtf(fmaxf(tight_w2[k], 0.f));
    u[k] = uk;
    const float ukp = uk * (1.f + EL_SLACK);
    if (ukp <= half_min[l]) return;  // no other centroid can be closer
    for (int i = 0; i < K; ++i) {
        if (i == l) continue;
        if (ukp > lb[k * K + i] && ukp > 0.5f * ccd[(int64_t)l * K + i]) {
            unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long*>(npairs), 1ull);
            pb[pos] = k;
            pc[pos] = i;
        }
    }
}

// scatter solved candidate values into the dense N x K table
__global__ void k_scatter_pairs(const int64_t* npairs, const int64_t* pb, const int32_t* pc, const float* val, int K,
                                float* D) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= *npairs) return;
    D[pb[t] * K + pc[t]] = val[t];
}

// new labels: lowest index among the smallest solved W^2 (same rule as
// d2_assign); solved values tighten their lower bounds
__global__ void k_elkan_pick(int64_t N, int K, int32_t* labels, const float* tight_w2, float* lb, const float* ccd,
                             const float* half_min, const float* u, const float* D, float* dist) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int l = labels[k];
    float best = tight_w2[k];
    int bi = l;
    lb[k * K + l] = u[k];
    const float ukp = u[k] * (1.f + EL_SLACK);
    if (ukp > half_min[l]) {
        for (int i = 0; i < K; ++i) {
            if (i == l) continue;
            if (ukp > lb[k * K + i] && ukp > 0.5f * ccd[(int64_t)l * K + i]) {
                const float v = D[k * K + i];
                lb[k * K + i] = sqrtf(fmaxf(v, 0.f));
                if (v < best || (v == best && i < bi)) {
                    best = v;
                    bi = i;
                }
            }
        }
    }
    labels[k] = bi;
    dist[k] = best;
}

__global__ void k_first_round_bounds(int64_t N, int K, const float* D, float* lb) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < N * K) lb[e] = sqrtf(fmaxf(D[e], 0.f));
}

__global__ void k_add_counts(int64_t* counters, const int64_t* a, const int64_t* b, int64_t c) {
    counters[0] += *a + *b + c;
}

// One Elkan assignment round.  state: lb (N x K), D (N x K), u (N), tight (N),
// ccw2/ccd (K x K), half (K), shift (K), pair lists (N x K), counters.
struct ElkanState {
    float *lb, *D, *u, *tight, *ccw2, *ccd, *half, *shift, *val;
    int64_t *pb, *np, *np2, *coff, *coff_prev;
    int32_t* pc;
};

int d2_elkan_state(d2_ctx* ctx, int64_t N, int K, ElkanState* s) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t NK = (size_t)N * K;
    const size_t KK = (size_t)K * K;
    const size_t cap = std::max(NK, KK);
    const size_t o_lb = take(NK * 4), o_D = take(NK * 4), o_u = take(N * 4), o_t = take(N * 4),
                 o_ccw = take(KK * 4), o_ccd = take(KK * 4), o_h = take(K * 4), o_sh = take(K * 4),
                 o_val = take(cap * 4), o_pb = take(cap * 8), o_np = take(64), o_np2 = take(64),
                 o_co = take((K + 1) * 8), o_cp = take((K + 1) * 8), o_pc = take(cap * 4);
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_ELKAN, off, &base);
    if (rc) return rc;
    char* b = static_cast<char*>(base);
    s->lb = reinterpret_cast<float*>(b + o_lb);
    s->D = reinterpret_cast<float*>(b + o_D);
    s->u = reinterpret_cast<float*>(b + o_u);
    s->tight = reinterpret_cast<float*>(b + o_t);
    s->ccw2 = reinterpret_cast<float*>(b + o_ccw);
    s->ccd = reinterpret_cast<float*>(b + o_ccd);
    s->half = reinterpret_cast<float*>(b + o_h);
    s->shift = reinterpret_cast<float*>(b + o_sh);
    s->val = reinterpret_cast<float*>(b + o_val);
    s->pb = reinterpret_cast<int64_t*>(b + o_pb);
    s->np = reinterpret_cast<int64_t*>(b + o_np);
    s->np2 = reinterpret_cast<int64_t*>(b + o_np2);
    s->coff = reinterpret_cast<int64_t*>(b + o_co);
    s->coff_prev = reinterpret_cast<int64_t*>(b + o_cp);
    s->pc = reinterpret_cast<int32_t*>(b + o_pc);
    return D2_OK;
}

int d2_launch_pairs_all(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w, float* out,
                        int64_t* fail_count, cudaStream_t st);
int d2_argmin_rows(d2_ctx* ctx, const float* D, int64_t N, int K, int32_t* labels, float* dist, cudaStream_t st);

// x_prev/w_prev: the centroids the bounds refer to (NULL on the first round).
// counters[0] accumulates the exact W^2 solves.
int d2_assign_elkan(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                    const float* x_prev, const float* w_prev, int32_t* labels, float* dist, int64_t* counters,
                    cudaStream_t st) {
    const int64_t N = b->N;
    ElkanState s;
    int rc = d2_elkan_state(ctx, N, K, &s);
    if (rc) return rc;
    const unsigned gN = (unsigned)d2_ceil_div(N, 256);
    const unsigned gNK = (unsigned)d2_ceil_div(N * (int64_t)K, 256);
    if (!x_prev) {
        // first round: every pair is solved and every bound is exact
        if ((rc = d2_launch_pairs_all(ctx, b, K, m, x, w, s.D, counters + 2, st))) return rc;
        if ((rc = d2_argmin_rows(ctx, s.D, N, K, labels, dist, st))) return rc;
        k_first_round_bounds<<<gNK, 256, 0, st>>>(N, K, s.D, s.lb);
        D2_LAUNCH_CK(ctx, "k_first_round_bounds");
        D2_CK(ctx, cudaMemsetAsync(s.np, 0, 8, st));
        D2_CK(ctx, cudaMemsetAsync(s.np2, 0, 8, st));
        k_add_counts<<<1, 1, 0, st>>>(counters, s.np, s.np2, N * (int64_t)K);
        D2_LAUNCH_CK(ctx, "k_add_counts");
        return D2_OK;
    }
    // centroids viewed as bags (K distributions of m points each)
    k_centroid_offsets<<<(unsigned)d2_ceil_div(K + 1, 256), 256, 0, st>>>(K, m, s.coff);
    D2_LAUNCH_CK(ctx, "k_centroid_offsets");
    d2_bags cb;
    memset(&cb, 0, sizeof(cb));
    cb.N = K;
    cb.n = (int64_t)K * m;
    cb.d = b->d;
    cb.max_mk = m;
    cb.offsets = s.coff;
    cb.wt = w_prev;
    cb.supp = x_prev;
    // 1) shifts W^2(Q_i^old, Q_i^new): bags = old centroids, centroids = new
    k_shift_pairs<<<(unsigned)d2_ceil_div(K, 256), 256, 0, st>>>(K, s.pb, s.pc, s.np);
    D2_LAUNCH_CK(ctx, "k_shift_pairs");
    if ((rc = d2_solve_pair_list(ctx, &cb, K, m, x, w, s.pb, s.pc, K, s.np, s.shift, counters + 2, st))) return rc;
    k_shift_bounds<<<gNK, 256, 0, st>>>(N, K, s.shift, s.lb);
    D2_LAUNCH_CK(ctx, "k_shift_bounds");
    // 2) centroid-centroid distances among the new centroids
    cb.wt = w;
    cb.supp = x;
    k_cc_pairs<<<(unsigned)d2_ceil_div((int64_t)K * K, 256), 256, 0, st>>>(K, s.pb, s.pc, s.np);
    D2_LAUNCH_CK(ctx, "k_cc_pairs");
    if ((rc = d2_solve_pair_list(ctx, &cb, K, m, x, w, s.pb, s.pc, (int64_t)K * K, s.np, s.ccw2, counters + 2, st)))
        return rc;
    k_cc_finish<<<(unsigned)d2_ceil_div(K, 128), 128, 0, st>>>(K, s.ccw2, s.ccd, s.half);
    D2_LAUNCH_CK(ctx, "k_cc_finish");
    // 3) exact distance to the current label (tight upper bound, round objective)
    k_tight_pairs<<<gN, 256, 0, st>>>(N, labels, s.pb, s.pc);
    D2_LAUNCH_CK(ctx, "k_tight_pairs");
    if ((rc = d2_solve_pair_list(ctx, b, K, m, x, w, s.pb, s.pc, N, nullptr, s.tight, counters + 2, st))) return rc;
    // 4) the centroids the bounds cannot rule out
    D2_CK(ctx, cudaMemsetAsync(s.np2, 0, 8, st));
    k_candidates<<<gN, 256, 0, st>>>(N, K, labels, s.tight, s.lb, s.ccd, s.half, s.pb, s.pc, s.np2, s.u);
    D2_LAUNCH_CK(ctx, "k_candidates");
    if ((rc = d2_solve_pair_list(ctx, b, K, m, x, w, s.pb, s.pc, N * (int64_t)K, s.np2, s.val, counters + 2, st)))
        return rc;
    k_scatter_pairs<<<gNK, 256, 0, st>>>(s.np2, s.pb, s.pc, s.val, K, s.D);
    D2_LAUNCH_CK(ctx, "k_scatter_pairs");
    k_elkan_pick<<<gN, 256, 0, st>>>(N, K, labels, s.tight, s.lb, s.ccd, s.half, s.u, s.D, dist);
    D2_LAUNCH_CK(ctx, "k_elkan_pick");
    D2_CK(ctx, cudaMemsetAsync(s.np, 0, 8, st));
    k_add_counts<<<1, 1, 0, st>>>(counters, s.np, s.np2, N + (int64_t)K * K + K);
    D2_LAUNCH_CK(ctx, "k_add_counts");
    return D2_OK;
}
