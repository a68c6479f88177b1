// Exact, order-independent cross-member reductions of Algorithm badmm.
//
// Every sum over a cluster's members -- the weight consensus of Eq. (badmmw)
// or (badmmw2) each iteration, the support partials of Eq. (updatex), the cost
// sum of Eq. (rho) and the objective -- is taken in 64-bit fixed point: each
// term is rounded once to an integer q = round(v 2^F) at a scale 2^F that
// every participant derives from the same numbers, and the integers are
// added.  Integer addition is associative, so the result does not depend on
// the order of the terms nor on how the members are split between processes
// (the trunks of the paper's parallel implementation, Section 5): a caller
// that splits the members over several GPUs and sums these int64 buffers
// across them (the reducer installed with d2_set_reducer, e.g. an NCCL
// all-reduce) gets results bitwise equal to one GPU holding every member.
//   * consensus: terms in [0, 1] (wtilde or its square root), at most the
//     cluster's member count per sum: F = 62 - ceil(log2(P + 1)) with P the
//     total member count, known to every participant;
//   * cost sums, objective and support partials: F per cluster from the
//     largest magnitude among its terms (an exact max-reduce first) and a
//     bound on their count, so that no sum can reach 2^62.
// Quantisation: at most 2^-(F+1) per term, i.e. below 2^-62 of the largest
// possible sum -- far inside the FP32 rounding of the values themselves.
#include <algorithm>
#include <cmath>

#include "d2_internal.cuh"

// round(v 2^F) for v >= 0 finite with v 2^F < 2^62 (round half up), from the
// bits of v: exact and identical on every GPU
__device__ __forceinline__ int64_t fx_f32(float v, int F) {
    const uint32_t b = __float_as_uint(v);
    const int e = (int)(b >> 23);
    const uint64_t mant = (uint64_t)((b & 0x7fffffu) | (e ? 0x800000u : 0u));
    const int sh = (e ? e : 1) - 150 + F;
    if (sh >= 0) return (int64_t)(mant << sh);
    if (sh < -25) return 0;
    return (int64_t)((mant + (1ull << (-sh - 1))) >> (-sh));
}
// the same for signed values (symmetric rounding)
__device__ __forceinline__ int64_t fx_f32s(float v, int F) {
    const int64_t q = fx_f32(fabsf(v), F);
    return v < 0.f ? -q : q;
}
__device__ __forceinline__ int64_t fx_f64s(double v, int F) {
    return __double2ll_rn(ldexp(v, F));  // exact scaling, one rounding
}

// Scale for sums of at most `count` terms of magnitude at most `vmax`.
__device__ __forceinline__ int fx_scale(double vmax, int64_t count) {
    const double t = vmax * (double)(count + 1);
    if (!(t > 0.0) || !isfinite(t)) return 61;
    return 61 - (ilogb(t) + 1);
}
// consensus scale from the total member count (terms <= 1)
__device__ __forceinline__ int fx_cons_scale(int64_t total) {
    return 62 - (64 - __clzll((unsigned long long)total + 1ull));
}

// non-negative doubles order like their bit patterns (as int64)
__device__ __forceinline__ int64_t max_key(double v) { return __double_as_longlong(v); }
__device__ __forceinline__ double key_val(int64_t k) { return __longlong_as_double(k); }

int d2_reduce(d2_ctx* ctx, int op, int64_t* buf, int64_t count, cudaStream_t st) {
    if (!ctx->reducer || count <= 0) return D2_OK;
    const int rc = ctx->reducer(ctx->reducer_user, op, buf, count, st);
    if (rc != 0) return d2_fail(ctx, D2_ECUDA, "the installed reducer failed (%d)", rc);
    return D2_OK;
}

// ---------------------------------------------------------------------------
// member counts
// ---------------------------------------------------------------------------

__global__ void k_fx_counts(int K, const int64_t* cofs, int64_t* cnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < K) cnt[c] = cofs[c + 1] - cofs[c];
}
__global__ void k_fx_total(int K, int64_t* cnt) {  // cnt[K] = sum of cnt[0..K-1]
    __shared__ long long s[256];
    long long a = 0;
    for (int c = threadIdx.x; c < K; c += blockDim.x) a += cnt[c];
    s[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[K] = s[0];
}

int d2_fx_counts(d2_ctx* ctx, int K, const int64_t* cofs, int64_t* gcount, cudaStream_t st) {
    k_fx_counts<<<(unsigned)d2_ceil_div(K, 256), 256, 0, st>>>(K, cofs, gcount);
    D2_LAUNCH_CK(ctx, "k_fx_counts");
    int rc = d2_reduce(ctx, D2_REDUCE_SUM, gcount, K, st);
    if (rc) return rc;
    k_fx_total<<<1, 256, 0, st>>>(K, gcount);
    D2_LAUNCH_CK(ctx, "k_fx_total");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// weight consensus, Eq. (badmmw) / (badmmw2)
// ---------------------------------------------------------------------------

// S[c, i] += sum over one chunk's member positions (<= 64, all of cluster c)
// of round(part[p, i] 2^F): one CTA per chunk, thread (g, i) takes the
// positions p0 + g, p0 + g + G, ...; the chunk's total is added to S by an
// integer atomic (exact, so the order in which chunks land does not matter)
#define FX_CONS_THREADS 128
__global__ void __launch_bounds__(FX_CONS_THREADS) k_fx_cons(const Chunk* chunks, const int64_t* nchunks,
                                                             const float* pos_part, int m, const int64_t* gcount,
                                                             int K, long long* S) {
    __shared__ long long s_acc[FX_CONS_THREADS];
    const int64_t q = blockIdx.x;
    if (q >= *nchunks) return;
    const Chunk ch = chunks[q];
    const int F = fx_cons_scale(gcount[K]);
    const int t = threadIdx.x;
    for (int i0 = 0; i0 < m; i0 += FX_CONS_THREADS) {
        const int mm = min(m - i0, FX_CONS_THREADS);
        const int G = FX_CONS_THREADS / mm;
        const int i = t % mm, g = t / mm;
        long long acc = 0;
        if (g < G) {
            int64_t p = ch.p0 + g;
            for (; p + 3 * G < ch.p1; p += 4 * G) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = __ldcg(pos_part + (p + u * G) * m + i0 + i);
#pragma unroll
                for (int u = 0; u < 4; ++u) acc += fx_f32(v[u], F);
            }
            for (; p < ch.p1; p += G) acc += fx_f32(__ldcg(pos_part + p * m + i0 + i), F);
        }
        s_acc[t] = acc;
        __syncthreads();
        if (t < mm) {
            long long sum = 0;
            for (int h = 0; h < G; ++h) sum += s_acc[h * mm + t];
            if (sum != 0)
                atomicAdd(reinterpret_cast<unsigned long long*>(S + (int64_t)ch.c * m + i0 + t),
                          (unsigned long long)sum);
        }
        __syncthreads();
    }
}

// w_i = S_i / sum S (R1) or S_i^2 / sum S^2 (R2) of every cluster with members
// (on any participant); FP64, then FP32
__global__ void k_fx_cons_norm(int K, int m, long long* S, const int64_t* gcount, bool r2, float* w_next,
                               double* w_next64) {
    __shared__ double s_v[256];
    __shared__ double s_tot;
    const int c = blockIdx.x;
    if (gcount[c] == 0) return;  // no member anywhere: weights unchanged (its sums stay 0)
    const int F = fx_cons_scale(gcount[K]);
    const int t = threadIdx.x;
    if (t < m) {
        const double v = ldexp((double)S[(int64_t)c * m + t], -F);
        S[(int64_t)c * m + t] = 0;  // cleared for the next iteration's atomics
        s_v[t] = r2 ? v * v : v;
    }
    __syncthreads();
    if (t == 0) {
        double tot = 0.0;
        for (int h = 0; h < m; ++h) tot += s_v[h];
        s_tot = tot;
    }
    __syncthreads();
    if (t < m) {
        const double wv = s_v[t] / s_tot;
        w_next64[(int64_t)c * m + t] = wv;
        w_next[(int64_t)c * m + t] = (float)wv;
    }
}

int d2_fx_consensus(d2_ctx* ctx, int K, int m, const Chunk* chunks, const int64_t* nchunks, int64_t maxch,
                    const float* pos_part, bool r2, const int64_t* gcount, long long* S, float* w_next,
                    double* w_next64, cudaStream_t st) {
    // S is zero here: cleared at the start of the B-ADMM call and by each
    // normalisation after it has read the sums
    k_fx_cons<<<(unsigned)std::max<int64_t>(maxch, 1), FX_CONS_THREADS, 0, st>>>(chunks, nchunks, pos_part, m, gcount,
                                                                              K, S);
    D2_LAUNCH_CK(ctx, "k_fx_cons");
    int rc = d2_reduce(ctx, D2_REDUCE_SUM, reinterpret_cast<int64_t*>(S), (int64_t)K * m, st);
    if (rc) return rc;
    k_fx_cons_norm<<<K, 256, 0, st>>>(K, m, S, gcount, r2, w_next, w_next64);
    D2_LAUNCH_CK(ctx, "k_fx_cons_norm");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// segmented sums with a per-cluster scale: segment s of cluster c holds
// `width` values vals[s width .. s width + width - 1]; clusters own the
// segments seg_first[c] .. seg_first[c + 1] - 1 (chunks or member positions)
// ---------------------------------------------------------------------------

__device__ __forceinline__ float abs_max(float acc, float v) { return fmaxf(acc, fabsf(v)); }
__device__ __forceinline__ double abs_max(double acc, double v) { return fmax(acc, fabs(v)); }

// mkey[c] = max(mkey[c], key of the largest |value| of the cluster's
// segments); blocks (g, c), g < G, split the cluster's contiguous value range
// (the maximum is exact in the values' own type)
template <typename T>
__global__ void k_fx_segmax(int K, const int64_t* seg_first, const T* vals, int64_t width, int G, long long* mkey) {
    __shared__ long long s_m[256];
    const int c = blockIdx.y;
    const int64_t a = seg_first[c] * width, b = seg_first[c + 1] * width;
    T mx = 0;
    for (int64_t e = a + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < b; e += (int64_t)G * blockDim.x)
        mx = abs_max(mx, vals[e]);
    s_m[threadIdx.x] = max_key((double)mx);
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s_m[threadIdx.x] = max(s_m[threadIdx.x], s_m[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && s_m[0] > 0) atomicMax(&mkey[c], s_m[0]);
}

__device__ __forceinline__ int64_t fx_val(float v, int F) { return fx_f32s(v, F); }
__device__ __forceinline__ int64_t fx_val(double v, int F) { return fx_f64s(v, F); }

// out[c, e] = sum over the cluster's segments of round(vals 2^F_c), F_c from
// the cluster's (reduced) largest magnitude and the bound `cnt_bound[c]` on
// its number of segments; the FX_SY thread rows of a block take every
// FX_SY-th segment (integer sums: the split does not change the result)
#define FX_SX 128
#define FX_SY 8
template <typename T>
__global__ void __launch_bounds__(FX_SX * FX_SY) k_fx_segsum(int K, const int64_t* seg_first, const T* vals,
                                                            int64_t width, const long long* mkey,
                                                            const int64_t* cnt_bound, long long* out) {
    __shared__ long long s_acc[FX_SY][FX_SX];
    const int c = blockIdx.y;
    const int64_t e = blockIdx.x * (int64_t)FX_SX + threadIdx.x;
    const int F = fx_scale(key_val(mkey[c]), cnt_bound[c]);
    long long acc = 0;
    if (e < width)
        for (int64_t s = seg_first[c] + threadIdx.y; s < seg_first[c + 1]; s += FX_SY)
            acc += fx_val(vals[s * width + e], F);
    s_acc[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && e < width) {
        long long t = 0;
#pragma unroll
        for (int y = 0; y < FX_SY; ++y) t += s_acc[y][threadIdx.x];
        out[(int64_t)c * width + e] = t;
    }
}

// Exact per-cluster sums (K x width int64 in out, scale via fx_scale of the
// reduced max in mkey) of segmented values, reduced across participants.
template <typename T>
int d2_fx_segsum(d2_ctx* ctx, int K, const int64_t* seg_first, const T* vals, int64_t width, int64_t nseg,
                 const int64_t* cnt_bound, long long* mkey, long long* out, cudaStream_t st) {
    // blocks per cluster for the maximum: about 4,096 values per block on
    // average (the largest clusters hold far more than the average)
    const int G = (int)std::max<int64_t>(1, std::min<int64_t>(64, nseg * width / ((int64_t)K * 4096)));
    D2_CK(ctx, cudaMemsetAsync(mkey, 0, (size_t)K * sizeof(long long), st));
    k_fx_segmax<T><<<dim3((unsigned)G, (unsigned)K), 256, 0, st>>>(K, seg_first, vals, width, G, mkey);
    D2_LAUNCH_CK(ctx, "k_fx_segmax");
    int rc = d2_reduce(ctx, D2_REDUCE_MAX, reinterpret_cast<int64_t*>(mkey), K, st);
    if (rc) return rc;
    dim3 g((unsigned)d2_ceil_div(width, FX_SX), (unsigned)K);
    k_fx_segsum<T><<<g, dim3(FX_SX, FX_SY), 0, st>>>(K, seg_first, vals, width, mkey, cnt_bound, out);
    D2_LAUNCH_CK(ctx, "k_fx_segsum");
    return d2_reduce(ctx, D2_REDUCE_SUM, reinterpret_cast<int64_t*>(out), (int64_t)K * width, st);
}

// ---------------------------------------------------------------------------
// Eq. (rho): rho_c = rho0 x the mean cost entry of the cluster
// ---------------------------------------------------------------------------

__global__ void k_fx_rows(int K, const int64_t* chunk_first, const int64_t* chunk_rows, int64_t* rows) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    int64_t r = 0;
    for (int64_t q = chunk_first[c]; q < chunk_first[c + 1]; ++q) r += chunk_rows[q];
    rows[c] = r;
}

__global__ void k_fx_rho(int K, int m, const long long* mkey, const long long* ssum, const int64_t* gcount,
                         const int64_t* rows, double rho0, double rho_fixed, float* rho, float* beta,
                         int64_t* nrows) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    const int64_t r = rows[c];
    double v;
    if (rho_fixed > 0.0) {
        v = rho_fixed;
    } else if (r > 0) {
        const int F = fx_scale(key_val(mkey[c]), gcount[c]);
        v = rho0 * ldexp((double)ssum[c], -F) / ((double)m * (double)r);
    } else {
        v = 1.0;
    }
    if (!(v > 0.0) || !isfinite(v)) v = 1.0;  // all costs zero: any rho gives the same plans
    rho[c] = (float)v;
    beta[c] = (float)(D2_LOG2E / v);
    nrows[c] = r;
}

// chunk_sum / chunk_rows: the cost build's per-chunk FP64 cost sums and row
// counts; fx: 4 K int64 of scratch (max keys, sums, rows)
int d2_fx_rho(d2_ctx* ctx, int K, int m, const int64_t* chunk_first, const double* chunk_sum,
              const int64_t* chunk_rows, const int64_t* gcount, double rho0, double rho_fixed, float* rho,
              float* beta, int64_t* nrows, long long* fx, cudaStream_t st) {
    long long* mkey = fx;
    long long* ssum = fx + K;
    int64_t* rows = reinterpret_cast<int64_t*>(fx + 2 * K);
    int rc;
    if (chunk_sum) {
        if ((rc = d2_fx_segsum<double>(ctx, K, chunk_first, chunk_sum, 1, 0, gcount, mkey, ssum, st))) return rc;
        k_fx_rows<<<(unsigned)d2_ceil_div(K, 128), 128, 0, st>>>(K, chunk_first, chunk_rows, rows);
        D2_LAUNCH_CK(ctx, "k_fx_rows");
        if ((rc = d2_reduce(ctx, D2_REDUCE_SUM, rows, K, st))) return rc;
    } else {
        D2_CK(ctx, cudaMemsetAsync(fx, 0, (size_t)3 * K * sizeof(long long), st));
    }
    k_fx_rho<<<(unsigned)d2_ceil_div(K, 128), 128, 0, st>>>(K, m, mkey, ssum, gcount, rows, rho0, rho_fixed, rho,
                                                           beta, nrows);
    D2_LAUNCH_CK(ctx, "k_fx_rho");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// Eq. (updatex): x_i = (mu_c +) (sum of the chunk partials) / (N_c w_i)
// ---------------------------------------------------------------------------

__global__ void k_fx_xfinal(int K, int m, int d, const long long* mkey, const long long* sx, const int64_t* gcount,
                            const float* w, const float* mu, float* x) {
    const int c = blockIdx.y;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * d || gcount[c] == 0) return;
    const int i = (int)(e / d), dd = (int)(e - (int64_t)i * d);
    const int F = fx_scale(key_val(mkey[c]), gcount[c]);
    const double s = ldexp((double)sx[(int64_t)c * m * d + e], -F);
    const double mass = (double)gcount[c] * (double)w[(int64_t)c * m + i];
    if (mass > 0.0) {
        const double v = s / mass;
        x[(int64_t)c * m * d + e] = mu ? (float)((double)mu[(int64_t)c * d + dd] + v) : (float)v;
    }
}

// xpart: per chunk m x d FP32 partial sums; fx: K + K m d int64 of scratch
int d2_fx_support(d2_ctx* ctx, int K, int m, int d, const int64_t* chunk_first, int64_t nseg, const float* xpart,
                  const int64_t* gcount, const float* w, const float* mu, float* x, long long* fx, cudaStream_t st) {
    long long* mkey = fx;
    long long* sx = fx + K;
    const int64_t width = (int64_t)m * d;
    int rc = d2_fx_segsum<float>(ctx, K, chunk_first, xpart, width, nseg, gcount, mkey, sx, st);
    if (rc) return rc;
    dim3 g((unsigned)d2_ceil_div(width, 256), (unsigned)K);
    k_fx_xfinal<<<g, 256, 0, st>>>(K, m, d, mkey, sx, gcount, w, mu, x);
    D2_LAUNCH_CK(ctx, "k_fx_xfinal");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// objective (1/N_c) sum_k <C_k, Pi^(k,1)> and the final weights
// ---------------------------------------------------------------------------

__global__ void k_fx_finish(int K, int m, const long long* mkey, const long long* sobj, const int64_t* gcount,
                            const float* wfin, float* w_out, double* obj) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    if (gcount[c] == 0) {
        if (obj) obj[c] = 0.0;
        return;
    }
    if (obj) {
        const int F = fx_scale(key_val(mkey[c]), gcount[c]);
        obj[c] = ldexp((double)sobj[c], -F) / (double)gcount[c];
    }
    if (wfin != w_out)
        for (int i = 0; i < m; ++i) w_out[(int64_t)c * m + i] = wfin[(int64_t)c * m + i];
}

// pos_obj: per member position FP64 <C_k, Pi^(k,1)>; fx: 2 K int64 of scratch
int d2_fx_finish(d2_ctx* ctx, int K, int m, const int64_t* cofs, const double* pos_obj, const int64_t* gcount,
                 const float* wfin, float* w_out, double* obj, long long* fx, cudaStream_t st) {
    long long* mkey = fx;
    long long* sobj = fx + K;
    int rc = d2_fx_segsum<double>(ctx, K, cofs, pos_obj, 1, 0, gcount, mkey, sobj, st);
    if (rc) return rc;
    k_fx_finish<<<(unsigned)d2_ceil_div(K, 128), 128, 0, st>>>(K, m, mkey, sobj, gcount, wfin, w_out, obj);
    D2_LAUNCH_CK(ctx, "k_fx_finish");
    return D2_OK;
}
