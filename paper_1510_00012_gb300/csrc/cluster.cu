// Assignment step and D2-clustering outer loop (Algorithm 1 with the
// Section 5 choices), plus the greedy merge initialisation of Eq. (merge).
#include <algorithm>
#include <cstring>
#include <vector>

#include <functional>

#include "d2_internal.cuh"

struct AssignArgs;
size_t d2_assign_warp_bytes(int m, int nmax);
int d2_argmin_rows(d2_ctx* ctx, const float* D, int64_t N, int K, int32_t* labels, float* dist,
                   cudaStream_t st);
int d2_assign_exact(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                    int32_t* labels, float* dist, int64_t* fail_count, cudaStream_t st);
int d2_assign_pruned(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                     const d2_prune* prune, int32_t* labels, float* dist, int64_t* counters,
                     cudaStream_t st);
int d2_assign_elkan(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                    const float* x_prev, const float* w_prev, int32_t* labels, float* dist, int64_t* counters,
                    cudaStream_t st);

// ---------------------------------------------------------------------------
// Eq. (merge): one CTA per picked bag, FP64 like the definition
// ---------------------------------------------------------------------------
#define MG_MAX 256

__global__ void k_merge(const int64_t* offsets, const float* supp, const int32_t* vidx, const float* vocab,
                        const float* wt, int d, const int64_t* ids, int m, float* xout, float* wout) {
    extern __shared__ double mg[];
    const int c = blockIdx.x;
    const int64_t k = ids[c];
    const int64_t r0 = offsets[k];
    const int mk = (int)min((int64_t)MG_MAX, offsets[k + 1] - r0);
    double* X = mg;                        // mk x d
    double* W = X + (size_t)mk * d;        // mk
    int* alive = reinterpret_cast<int*>(W + mk);
    __shared__ double s_best[256];
    __shared__ int s_bi[256], s_bj[256];
    for (int e = threadIdx.x; e < mk * d; e += blockDim.x) {
        int j = e / d, t = e - j * d;
        X[e] = (double)d2_row_ptr(supp, vidx, vocab, d, r0 + j)[t];
    }
    for (int j = threadIdx.x; j < mk; j += blockDim.x) {
        W[j] = (double)wt[r0 + j];
        alive[j] = 1;
    }
    __syncthreads();
    int cnt = mk;
    while (cnt > m) {
        // lexicographic (i, j), i < j, first minimum of w_i w_j ||x_i - x_j||^2 / (w_i + w_j)
        double best = 1e300;
        int bi = 0x7fffffff, bj = 0x7fffffff;
        for (int e = threadIdx.x; e < mk * mk; e += blockDim.x) {
            int i = e / mk, j = e - i * mk;
            if (i >= j || !alive[i] || !alive[j]) continue;
            double den = W[i] + W[j], dd = 0.0;
            for (int t = 0; t < d; ++t) {
                double df = X[i * d + t] - X[j * d + t];
                dd += df * df;
            }
            double crit = den > 0.0 ? W[i] * W[j] * dd / den : 0.0;
            if (crit < best || (crit == best && (i < bi || (i == bi && j < bj)))) {
                best = crit;
                bi = i;
                bj = j;
            }
        }
        s_best[threadIdx.x] = best;
        s_bi[threadIdx.x] = bi;
        s_bj[threadIdx.x] = bj;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = 1; t < (int)blockDim.x; ++t) {
                double v = s_best[t];
                int ti = s_bi[t], tj = s_bj[t];
                if (v < s_best[0] || (v == s_best[0] && (ti < s_bi[0] || (ti == s_bi[0] && tj < s_bj[0])))) {
                    s_best[0] = v;
                    s_bi[0] = ti;
                    s_bj[0] = tj;
                }
            }
        }
        __syncthreads();
        const int i = s_bi[0], j = s_bj[0];
        const double wb = W[i] + W[j];
        for (int t = threadIdx.x; t < d; t += blockDim.x) {
            X[i * d + t] = wb > 0.0 ? (W[i] * X[i * d + t] + W[j] * X[j * d + t]) / wb
                                    : 0.5 * (X[i * d + t] + X[j * d + t]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            W[i] = wb;
            alive[j] = 0;
        }
        __syncthreads();
        --cnt;
    }
    // write the survivors in index order; pad short bags with zero-weight copies
    if (threadIdx.x == 0) {
        int o = 0, last = 0;
        for (int j = 0; j < mk; ++j) {
            if (!alive[j]) continue;
            for (int t = 0; t < d; ++t) xout[((int64_t)c * m + o) * d + t] = (float)X[j * d + t];
            wout[(int64_t)c * m + o] = (float)W[j];
            last = j;
            ++o;
        }
        for (; o < m; ++o) {
            for (int t = 0; t < d; ++t) xout[((int64_t)c * m + o) * d + t] = (float)X[last * d + t];
            wout[(int64_t)c * m + o] = 0.f;
        }
    }
}

extern "C" int d2_merge_init(d2_ctx* ctx, const d2_bags* bags, const int64_t* ids, int64_t cnt, int32_t m,
                             float* x, float* w, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (cnt < 0 || m < 1 || !ids || !x || !w) return d2_fail(ctx, D2_EINVAL, "d2_merge_init: bad arguments");
    if (bags->max_mk > MG_MAX) return d2_fail(ctx, D2_ENOTSUP, "d2_merge_init: m_k > %d", MG_MAX);
    if (cnt == 0) return D2_OK;
    size_t smem = (size_t)bags->max_mk * (bags->d + 1) * 8 + (size_t)bags->max_mk * 4 + 16;
    if (smem > 200 * 1024) return d2_fail(ctx, D2_ENOTSUP, "d2_merge_init: m_k x d too large");
    cudaStream_t st = d2_stream(stream);
    D2_CK(ctx, cudaFuncSetAttribute(k_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_merge<<<(unsigned)cnt, 256, smem, st>>>(bags->offsets, bags->supp, bags->vocab_idx, bags->vocab, bags->wt,
                                              bags->d, ids, m, x, w);
    D2_LAUNCH_CK(ctx, "k_merge");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// stable partition of bag ids by label: cluster_offsets (K+1), members (N)
// ---------------------------------------------------------------------------

__global__ void k_label_hist(const int32_t* labels, int64_t N, int K, int64_t* counts) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < N) {
        int l = labels[k];
        if (l >= 0 && l < K) atomicAdd(reinterpret_cast<unsigned long long*>(counts + l), 1ull);
    }
}

__global__ void k_excl_scan(const int64_t* counts, int K, int64_t* offs) {
    __shared__ int64_t s[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < K; base += 1024) {
        int c = base + threadIdx.x;
        int64_t v = c < K ? counts[c] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (c < K) offs[c] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) offs[K] = carry;
}

// one CTA walks the bags in tiles of 1024 in id order; inside a tile the warps
// take turns, each lane finding its rank among equal labels with match_any
__global__ void k_stable_scatter(const int32_t* labels, int64_t N, int K, const int64_t* offs, int64_t* cursor,
                                 int64_t* members) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = threadIdx.x; c < K; c += blockDim.x) cursor[c] = offs[c];
    __syncthreads();
    for (int64_t base = 0; base < N; base += blockDim.x) {
        const int64_t k = base + threadIdx.x;
        const int l = k < N ? labels[k] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, l);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int leader = __ffs(peers) - 1;
        const int cntw = __popc(peers);
        for (int w = 0; w < nw; ++w) {
            if (warp == w && l >= 0 && l < K) {
                int64_t basepos = cursor[l];  // read before the leader advances it
                __syncwarp(peers);
                members[basepos + rank] = k;
                __syncwarp(peers);
                if (lane == leader) cursor[l] = basepos + cntw;
            }
            __syncthreads();
        }
    }
}

__global__ void k_acc_counts(int64_t* total, const int64_t* call) {
    total[0] += call[0];
    total[1] += call[1];
    total[2] += call[2];
}

__global__ void k_warm_mask(const int32_t* labels, const int32_t* prev, int64_t N, uint8_t* mask) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < N) mask[k] = (prev[k] >= 0 && prev[k] == labels[k]) ? 1 : 0;
}

__global__ void k_mean_dist(const float* dist, int64_t N, double* out) {
    __shared__ double s[1024];
    double acc = 0.0;
    for (int64_t k = threadIdx.x; k < N; k += blockDim.x) acc += (double)dist[k];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0] / (double)N;
}

// ---------------------------------------------------------------------------
// d2_assign
// ---------------------------------------------------------------------------

int d2_assign_bounded_impl(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                           const d2_prune* prune, int r_first, int32_t* labels, float* dist, int64_t* counters,
                           cudaStream_t st);

static int assign_any(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const float* x, const float* w,
                      const d2_prune* prune, bool bounded, int32_t* labels, float* dist, int64_t* stats,
                      void* stream);

extern "C" int d2_assign(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const float* x, const float* w,
                         const d2_prune* prune, int32_t* labels, float* dist, int64_t* stats, void* stream) {
    return assign_any(ctx, bags, K, m, x, w, prune, false, labels, dist, stats, stream);
}

extern "C" int d2_assign_bounded(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const float* x,
                                 const float* w, const d2_prune* prune, int32_t* labels, float* dist,
                                 int64_t* stats, void* stream) {
    return assign_any(ctx, bags, K, m, x, w, prune, true, labels, dist, stats, stream);
}

static int assign_any(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const float* x, const float* w,
                      const d2_prune* prune, bool bounded, int32_t* labels, float* dist, int64_t* stats,
                      void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (K < 1 || m < 1 || !x || !w || !labels || !dist)
        return d2_fail(ctx, D2_EINVAL, "d2_assign: need K >= 1, m >= 1 and non-NULL arrays");
    if (m + bags->max_mk > 32000) return d2_fail(ctx, D2_ENOTSUP, "d2_assign: m + max_mk too large");
    cudaStream_t st = d2_stream(stream);
    void* sc = nullptr;
    if ((rc = d2_ws(ctx, WS_SCAN, 64, &sc))) return rc;
    int64_t* counters = static_cast<int64_t*>(sc);  // [0] exact solves, [1] fall-backs, [2] limit hits
    D2_CK(ctx, cudaMemsetAsync(counters, 0, 3 * sizeof(int64_t), st));
    if (bounded) {
        // first exact solves per bag: 1, then at most one more (the smallest
        // remaining bound) unless it is excluded; 2 up front where the
        // entropic dual bound runs between the two (its threshold then comes
        // from two values)
        const int dual_iters = ctx->dual_iters >= 0 ? ctx->dual_iters : (m >= 32 ? 1 : 0);
        int32_t r = dual_iters > 0 && m <= 64 ? 2 : 1;
        float delta = 0.f;
        if (prune) d2_prune_get_margin(prune, &r, &delta);
        rc = d2_assign_bounded_impl(ctx, bags, K, m, x, w, prune, r, labels, dist, counters, st);
    } else if (prune) {
        rc = d2_assign_pruned(ctx, bags, K, m, x, w, prune, labels, dist, counters, st);
    } else {
        rc = d2_assign_exact(ctx, bags, K, m, x, w, labels, dist, counters, st);
    }
    if (rc) return rc;
    if (stats) {
        D2_CK(ctx, cudaMemcpyAsync(stats, counters, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        D2_CK(ctx, cudaStreamSynchronize(st));
        if (stats[2] > 0)
            return d2_fail(ctx, D2_ENOCONV, "d2_assign: %lld exact W^2 solves reached the phase cap",
                           (long long)stats[2]);
    }
    return D2_OK;
}

// ---------------------------------------------------------------------------
// d2_cluster
// ---------------------------------------------------------------------------

static uint64_t splitmix64_next(uint64_t& state) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" int d2_cluster(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, uint64_t seed, int32_t rounds,
                          const d2_badmm_opts* opts, const d2_prune* prune, float* x_out, float* w_out,
                          int32_t* labels_out, double* obj_per_round, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (K < 1 || m < 1 || m > 256 || rounds < 1 || !x_out || !w_out || !labels_out)
        return d2_fail(ctx, D2_EINVAL, "d2_cluster: need K >= 1, 1 <= m <= 256, rounds >= 1, non-NULL outputs");
    cudaStream_t st = d2_stream(stream);
    const int64_t N = bags->N, n = bags->n;

    // seeded pick: partial Fisher-Yates over the ids with m_k >= min(m, the
    // K-th largest m_k) in ascending order (with fewer than K distributions of
    // m points, the largest ones seed the centroids and are padded by the merge)
    if (K > N) return d2_fail(ctx, D2_EINVAL, "d2_cluster: K = %d exceeds N = %lld", K, (long long)N);
    std::vector<int64_t> off(N + 1);
    D2_CK(ctx, cudaMemcpyAsync(off.data(), bags->offsets, (N + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    D2_CK(ctx, cudaStreamSynchronize(st));
    std::vector<int64_t> sz(N);
    for (int64_t k = 0; k < N; ++k) sz[k] = off[k + 1] - off[k];
    std::vector<int64_t> srt(sz);
    std::nth_element(srt.begin(), srt.begin() + (K - 1), srt.end(), std::greater<int64_t>());
    const int64_t thr = std::min<int64_t>(m, srt[K - 1]);
    std::vector<int64_t> elig;
    for (int64_t k = 0; k < N; ++k)
        if (sz[k] >= thr) elig.push_back(k);
    uint64_t state = seed;
    const uint64_t E = elig.size();
    for (int t = 0; t < K; ++t) {
        uint64_t z = splitmix64_next(state);
        uint64_t j = t + z % (E - t);
        std::swap(elig[t], elig[j]);
    }

    // state lives in one workspace slot
    const size_t o_lab = 0;
    const size_t o_prev = o_lab + ((N * 4 + 255) & ~255ull);
    const size_t o_dist = o_prev + ((N * 4 + 255) & ~255ull);
    const size_t o_mask = o_dist + ((N * 4 + 255) & ~255ull);
    const size_t o_mem = o_mask + ((N + 255) & ~255ull);
    const size_t o_co = o_mem + ((N * 8 + 255) & ~255ull);
    const size_t o_cnt = o_co + (((K + 1) * 8 + 255) & ~255ull);
    const size_t o_cur = o_cnt + ((K * 8 + 255) & ~255ull);
    const size_t o_ids = o_cur + ((K * 8 + 255) & ~255ull);
    const size_t o_obj = o_ids + ((K * 8 + 255) & ~255ull);
    const size_t o_bobj = o_obj + 256;
    const size_t o_xp = o_bobj + ((K * 8 + 255) & ~255ull);
    const size_t o_wp = o_xp + (((size_t)K * m * bags->d * 4 + 255) & ~255ull);
    const size_t o_cnt2 = o_wp + (((size_t)K * m * 4 + 255) & ~255ull);
    const size_t o_plan = o_cnt2 + 256;
    const size_t total = o_plan + (size_t)n * m * 4;
    void* base = nullptr;
    if ((rc = d2_ws(ctx, WS_CLUSTER_LOOP, total, &base))) return rc;
    char* b = static_cast<char*>(base);
    int32_t* lab = reinterpret_cast<int32_t*>(b + o_lab);
    int32_t* prev = reinterpret_cast<int32_t*>(b + o_prev);
    float* dist = reinterpret_cast<float*>(b + o_dist);
    uint8_t* mask = reinterpret_cast<uint8_t*>(b + o_mask);
    int64_t* members = reinterpret_cast<int64_t*>(b + o_mem);
    int64_t* co = reinterpret_cast<int64_t*>(b + o_co);
    int64_t* counts = reinterpret_cast<int64_t*>(b + o_cnt);
    int64_t* cursor = reinterpret_cast<int64_t*>(b + o_cur);
    int64_t* ids = reinterpret_cast<int64_t*>(b + o_ids);
    double* dobj = reinterpret_cast<double*>(b + o_obj);
    double* bobj = reinterpret_cast<double*>(b + o_bobj);
    float* plan = reinterpret_cast<float*>(b + o_plan);
    float* x_prev = reinterpret_cast<float*>(b + o_xp);
    float* w_prev = reinterpret_cast<float*>(b + o_wp);
    int64_t* solves = reinterpret_cast<int64_t*>(b + o_cnt2);  // [0] exact solves, [1] fall-backs, [2] limit

    D2_CK(ctx, cudaMemcpyAsync(ids, elig.data(), K * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if ((rc = d2_merge_init(ctx, bags, ids, K, m, x_out, w_out, stream))) return rc;
    D2_CK(ctx, cudaMemsetAsync(prev, 0xff, N * 4, st));

    d2_badmm_opts o;
    if (opts) o = *opts; else d2_badmm_opts_default(&o);
    o.flags &= ~D2_VALIDATE;
    const bool elkan = (o.flags & D2_ELKAN) && !prune && !(o.flags & D2_ASSIGN_BOUNDED);
    const unsigned gN = (unsigned)d2_ceil_div(N, 256);
    D2_CK(ctx, cudaMemsetAsync(solves, 0, 3 * sizeof(int64_t), st));
    void* scnt = nullptr;
    if ((rc = d2_ws(ctx, WS_SCAN, 64, &scnt))) return rc;
    int64_t* acounters = static_cast<int64_t*>(scnt);
    int64_t bypass_fallbacks = 0;  // bags of the rounds that skipped the pruner
    for (int r = 0; r < rounds; ++r) {
        bool use_prune = prune != nullptr;
        if (elkan) {
            if ((rc = d2_assign_elkan(ctx, bags, K, m, x_out, w_out, r == 0 ? nullptr : x_prev,
                                      r == 0 ? nullptr : w_prev, lab, dist, solves, st)))
                return rc;
            D2_CK(ctx, cudaMemcpyAsync(x_prev, x_out, (size_t)K * m * bags->d * 4, cudaMemcpyDeviceToDevice, st));
            D2_CK(ctx, cudaMemcpyAsync(w_prev, w_out, (size_t)K * m * 4, cudaMemcpyDeviceToDevice, st));
        } else {
            if (prune && (o.flags & D2_PRUNE_RECALIBRATE)) {
                // the margin of the current centroids, from exact W^2 of evenly spaced bags
                const int64_t ns = std::min<int64_t>(N, 1000);
                std::vector<int64_t> hid(ns);
                for (int64_t t = 0; t < ns; ++t) hid[t] = t * N / ns;
                void* vid = nullptr;
                if ((rc = d2_ws(ctx, WS_SPLIT, (size_t)ns * 8, &vid))) return rc;
                D2_CK(ctx, cudaMemcpyAsync(vid, hid.data(), (size_t)ns * 8, cudaMemcpyHostToDevice, st));
                if ((rc = d2_prune_calibrate(ctx, const_cast<d2_prune*>(prune), bags, K, m, x_out, w_out,
                                             static_cast<int64_t*>(vid), ns, 0.999f, stream)))
                    return rc;
                // a round where most bags would fall back to all K anyway skips the pruner
                int32_t pr_r = 0;
                float pr_delta = 0.f, fb = 0.f;
                d2_prune_get_margin(prune, &pr_r, &pr_delta);
                d2_prune_get_calibration(prune, &fb);
                use_prune = !((double)pr_r + (double)fb * K >= 0.8 * K);
                if (!use_prune) bypass_fallbacks += N;
            }
            if ((rc = assign_any(ctx, bags, K, m, x_out, w_out, use_prune ? prune : nullptr,
                                 (o.flags & D2_ASSIGN_BOUNDED) != 0, lab, dist, nullptr, stream)))
                return rc;
            k_acc_counts<<<1, 1, 0, st>>>(solves, acounters);
            D2_LAUNCH_CK(ctx, "k_acc_counts");
        }
        k_mean_dist<<<1, 1024, 0, st>>>(dist, N, dobj);
        D2_LAUNCH_CK(ctx, "k_mean_dist");
        if (obj_per_round) {
            D2_CK(ctx, cudaMemcpyAsync(&obj_per_round[r], dobj, sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        k_warm_mask<<<gN, 256, 0, st>>>(lab, prev, N, mask);
        D2_LAUNCH_CK(ctx, "k_warm_mask");
        D2_CK(ctx, cudaMemsetAsync(counts, 0, K * 8, st));
        k_label_hist<<<gN, 256, 0, st>>>(lab, N, K, counts);
        D2_LAUNCH_CK(ctx, "k_label_hist");
        k_excl_scan<<<1, 1024, 0, st>>>(counts, K, co);
        D2_LAUNCH_CK(ctx, "k_excl_scan");
        k_stable_scatter<<<1, 1024, 0, st>>>(lab, N, K, co, cursor, members);
        D2_LAUNCH_CK(ctx, "k_stable_scatter");
        if ((rc = badmm_barycenter(ctx, bags, co, members, N, K, m, x_out, w_out, plan, mask, &o, bobj, stream)))
            return rc;
        D2_CK(ctx, cudaMemcpyAsync(prev, lab, N * 4, cudaMemcpyDeviceToDevice, st));
    }
    D2_CK(ctx, cudaMemcpyAsync(labels_out, lab, N * 4, cudaMemcpyDeviceToDevice, st));
    int64_t hs[3] = {0, 0, 0};
    D2_CK(ctx, cudaMemcpyAsync(hs, solves, sizeof(hs), cudaMemcpyDeviceToHost, st));
    D2_CK(ctx, cudaStreamSynchronize(st));
    ctx->cluster_solves = hs[0];
    ctx->cluster_fallbacks = hs[1] + bypass_fallbacks;
    if (hs[2] > 0)
        return d2_fail(ctx, D2_ENOCONV, "d2_cluster: %lld exact W^2 solves reached the phase cap",
                       (long long)hs[2]);
    return D2_OK;
}

// ---------------------------------------------------------------------------
// d2_cluster_sym: symbolic supports
// ---------------------------------------------------------------------------

// Initial centroid weights from the picked bags: the mass of each bag symbol
// goes to its nearest centroid symbol (smallest dissimilarity, first
// minimum); one thread per centroid, FP64 sums in row order.
__global__ void k_sym_project(const int64_t* ids, int K, const int64_t* offsets, const int32_t* bsym,
                              const float* bw, const float* symcost, int64_t V, const int32_t* sym, int m,
                              float* w_out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    const int64_t k = ids[c];
    float* wc = w_out + (int64_t)c * m;
    double acc[256];
    for (int i = 0; i < m; ++i) acc[i] = 0.0;
    double tot = 0.0;
    for (int64_t r = offsets[k]; r < offsets[k + 1]; ++r) {
        const float* col = symcost + bsym[r];  // c(s, t) for t = bsym[r] at col[s * V]
        int best = 0;
        float bv = col[(int64_t)sym[0] * V];
        for (int i = 1; i < m; ++i) {
            const float v = col[(int64_t)sym[i] * V];
            if (v < bv) {
                bv = v;
                best = i;
            }
        }
        acc[best] += (double)bw[r];
        tot += (double)bw[r];
    }
    for (int i = 0; i < m; ++i) wc[i] = tot > 0.0 ? (float)(acc[i] / tot) : 1.0f / (float)m;
}

__global__ void k_tile_sym(const int32_t* sym, int K, int m, int32_t* csym) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < (int64_t)K * m) csym[e] = sym[e % m];
}

extern "C" int d2_cluster_sym(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const int32_t* sym,
                              uint64_t seed, int32_t rounds, const d2_badmm_opts* opts, float* w_out,
                              int32_t* labels_out, double* obj_per_round, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_sym_bags_host(ctx, bags);
    if (rc) return rc;
    if (K < 1 || m < 1 || m > 256 || rounds < 1 || !sym || !w_out || !labels_out)
        return d2_fail(ctx, D2_EINVAL, "d2_cluster_sym: need K >= 1, 1 <= m <= 256, rounds >= 1, non-NULL arrays");
    const int64_t N = bags->N, n = bags->n;
    if (K > N) return d2_fail(ctx, D2_EINVAL, "d2_cluster_sym: K = %d exceeds N = %lld", K, (long long)N);
    cudaStream_t st = d2_stream(stream);
    // seeded pick: partial Fisher-Yates over all bag ids (no size condition:
    // a symbolic centroid is not merged from its seed)
    std::vector<int64_t> elig(N);
    for (int64_t k = 0; k < N; ++k) elig[k] = k;
    uint64_t state = seed;
    for (int t = 0; t < K; ++t) {
        const uint64_t z = splitmix64_next(state);
        const uint64_t j = t + z % (uint64_t)(N - t);
        std::swap(elig[t], elig[j]);
    }
    const size_t o_lab = 0;
    const size_t o_prev = o_lab + ((N * 4 + 255) & ~255ull);
    const size_t o_dist = o_prev + ((N * 4 + 255) & ~255ull);
    const size_t o_mask = o_dist + ((N * 4 + 255) & ~255ull);
    const size_t o_mem = o_mask + ((N + 255) & ~255ull);
    const size_t o_co = o_mem + ((N * 8 + 255) & ~255ull);
    const size_t o_cnt = o_co + (((K + 1) * 8 + 255) & ~255ull);
    const size_t o_cur = o_cnt + ((K * 8 + 255) & ~255ull);
    const size_t o_ids = o_cur + ((K * 8 + 255) & ~255ull);
    const size_t o_obj = o_ids + ((K * 8 + 255) & ~255ull);
    const size_t o_bobj = o_obj + 256;
    const size_t o_csym = o_bobj + ((K * 8 + 255) & ~255ull);
    const size_t o_cnt2 = o_csym + (((size_t)K * m * 4 + 255) & ~255ull);
    const size_t o_plan = o_cnt2 + 256;
    const size_t total = o_plan + (size_t)n * m * 4;
    void* base = nullptr;
    if ((rc = d2_ws(ctx, WS_CLUSTER_LOOP, total, &base))) return rc;
    char* b = static_cast<char*>(base);
    int32_t* lab = reinterpret_cast<int32_t*>(b + o_lab);
    int32_t* prev = reinterpret_cast<int32_t*>(b + o_prev);
    float* dist = reinterpret_cast<float*>(b + o_dist);
    uint8_t* mask = reinterpret_cast<uint8_t*>(b + o_mask);
    int64_t* members = reinterpret_cast<int64_t*>(b + o_mem);
    int64_t* co = reinterpret_cast<int64_t*>(b + o_co);
    int64_t* counts = reinterpret_cast<int64_t*>(b + o_cnt);
    int64_t* cursor = reinterpret_cast<int64_t*>(b + o_cur);
    int64_t* ids = reinterpret_cast<int64_t*>(b + o_ids);
    double* dobj = reinterpret_cast<double*>(b + o_obj);
    double* bobj = reinterpret_cast<double*>(b + o_bobj);
    int32_t* csym = reinterpret_cast<int32_t*>(b + o_csym);
    int64_t* solves = reinterpret_cast<int64_t*>(b + o_cnt2);  // [0] exact solves, [1] fall-backs, [2] limit
    float* plan = reinterpret_cast<float*>(b + o_plan);

    D2_CK(ctx, cudaMemcpyAsync(ids, elig.data(), K * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    k_tile_sym<<<(unsigned)d2_ceil_div((int64_t)K * m, 256), 256, 0, st>>>(sym, K, m, csym);
    D2_LAUNCH_CK(ctx, "k_tile_sym");
    k_sym_project<<<(unsigned)d2_ceil_div(K, 64), 64, 0, st>>>(ids, K, bags->offsets, bags->vocab_idx, bags->wt,
                                                               bags->symcost, bags->V, sym, m, w_out);
    D2_LAUNCH_CK(ctx, "k_sym_project");
    D2_CK(ctx, cudaMemsetAsync(prev, 0xff, N * 4, st));
    D2_CK(ctx, cudaMemsetAsync(solves, 0, 3 * sizeof(int64_t), st));
    void* scnt = nullptr;
    if ((rc = d2_ws(ctx, WS_SCAN, 64, &scnt))) return rc;
    int64_t* acounters = static_cast<int64_t*>(scnt);
    d2_badmm_opts o;
    if (opts) o = *opts; else d2_badmm_opts_default(&o);
    o.flags &= ~D2_VALIDATE;
    const unsigned gN = (unsigned)d2_ceil_div(N, 256);
    for (int r = 0; r < rounds; ++r) {
        if ((rc = d2_assign_sym_impl(ctx, bags, K, m, csym, w_out, lab, dist, acounters, st))) return rc;
        k_acc_counts<<<1, 1, 0, st>>>(solves, acounters);
        D2_LAUNCH_CK(ctx, "k_acc_counts");
        k_mean_dist<<<1, 1024, 0, st>>>(dist, N, dobj);
        D2_LAUNCH_CK(ctx, "k_mean_dist");
        if (obj_per_round)
            D2_CK(ctx, cudaMemcpyAsync(&obj_per_round[r], dobj, sizeof(double), cudaMemcpyDeviceToHost, st));
        k_warm_mask<<<gN, 256, 0, st>>>(lab, prev, N, mask);
        D2_LAUNCH_CK(ctx, "k_warm_mask");
        D2_CK(ctx, cudaMemsetAsync(counts, 0, K * 8, st));
        k_label_hist<<<gN, 256, 0, st>>>(lab, N, K, counts);
        D2_LAUNCH_CK(ctx, "k_label_hist");
        k_excl_scan<<<1, 1024, 0, st>>>(counts, K, co);
        D2_LAUNCH_CK(ctx, "k_excl_scan");
        k_stable_scatter<<<1, 1024, 0, st>>>(lab, N, K, co, cursor, members);
        D2_LAUNCH_CK(ctx, "k_stable_scatter");
        if ((rc = badmm_barycenter_sym(ctx, bags, co, members, N, K, m, csym, w_out, plan, mask, &o, bobj, stream)))
            return rc;
        D2_CK(ctx, cudaMemcpyAsync(prev, lab, N * 4, cudaMemcpyDeviceToDevice, st));
    }
    D2_CK(ctx, cudaMemcpyAsync(labels_out, lab, N * 4, cudaMemcpyDeviceToDevice, st));
    int64_t hs[3] = {0, 0, 0};
    D2_CK(ctx, cudaMemcpyAsync(hs, solves, sizeof(hs), cudaMemcpyDeviceToHost, st));
    D2_CK(ctx, cudaStreamSynchronize(st));
    ctx->cluster_solves = hs[0];
    ctx->cluster_fallbacks = 0;
    if (hs[2] > 0)
        return d2_fail(ctx, D2_ENOCONV, "d2_cluster_sym: %lld exact W^2 solves reached the phase cap",
                       (long long)hs[2]);
    return D2_OK;
}

extern "C" int d2_cluster_stats(const d2_ctx* ctx, int64_t* stats) {
    if (!ctx || !stats) return D2_EINVAL;
    stats[0] = ctx->cluster_solves;
    stats[1] = ctx->cluster_fallbacks;
    return D2_OK;
}
