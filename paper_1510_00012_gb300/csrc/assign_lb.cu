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
    bool vec;          // 16-byte loads of support rows (d % 4 == 0, aligned rows)
    int64_t ring_off;  // floats from the start of shared memory to the warps' rings
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

// Cost entries C_ij = max(||x_i||^2 + ||y_j||^2 - 2 <x_i, y_j>, 0) of the
// centroid points i0 .. i0 + 7 (rows past m repeat row m - 1) against the
// lane's bag points j = lane + 32 q, each dot product summed in dimension
// order.  With vec (d % 4 == 0, 16-byte aligned rows, ystride % 4 == 0) four
// dimensions per step from 16-byte loads: eight centroid rows and JN bag rows
// feed 32 JN multiply-adds.
template <int JN>
__device__ __forceinline__ void lb_cost8(const float* xc, const float* xn_c, int d, int m, int i0, const float* ys,
                                         int ystride, const float* yn, int lane, bool vec, float (&cij)[8][JN]) {
    float acc[8][JN];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int q = 0; q < JN; ++q) acc[u][q] = 0.f;
    if (vec) {
        for (int t = 0; t < d; t += 4) {
            float4 yv[JN];
#pragma unroll
            for (int q = 0; q < JN; ++q) yv[q] = *reinterpret_cast<const float4*>(&ys[(lane + 32 * q) * ystride + t]);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = min(i0 + u, m - 1);
                const float4 xv = __ldg(reinterpret_cast<const float4*>(xc + (int64_t)i * d + t));
#pragma unroll
                for (int q = 0; q < JN; ++q) {
                    acc[u][q] = fmaf(xv.x, yv[q].x, acc[u][q]);
                    acc[u][q] = fmaf(xv.y, yv[q].y, acc[u][q]);
                    acc[u][q] = fmaf(xv.z, yv[q].z, acc[u][q]);
                    acc[u][q] = fmaf(xv.w, yv[q].w, acc[u][q]);
                }
            }
        }
    } else {
        for (int t = 0; t < d; ++t) {
            float yv[JN];
#pragma unroll
            for (int q = 0; q < JN; ++q) yv[q] = ys[(lane + 32 * q) * ystride + t];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float xv = __ldg(xc + (int64_t)min(i0 + u, m - 1) * d + t);
#pragma unroll
                for (int q = 0; q < JN; ++q) acc[u][q] = fmaf(xv, yv[q], acc[u][q]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const float xni = xn_c[min(i0 + u, m - 1)];
#pragma unroll
        for (int q = 0; q < JN; ++q) cij[u][q] = fmaxf(fmaf(-2.f, acc[u][q], xni + yn[lane + 32 * q]), 0.f);
    }
}

// The same entries for every centroid point of a centroid, block by block
// of 8 points, with the centroid's rows streamed through the warp's private
// ring of LB_XS stages (8 rows x 32 dimensions each) by 16-byte asynchronous
// copies, LB_XS - 1 stages ahead (vec layouts only).  on_block(i0, cij)
// receives each block.  Each dot product is taken as two partial sums, of
// the even and of the odd dimensions (each in dimension order, by paired
// FP32 fused multiply-adds on adjacent dimensions), added at the end.
#define LB_XS 4
#define LB_XSTAGE 256   // floats per ring stage

__device__ __forceinline__ void lb_cp16(float* sdst, const float* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc));
}

__device__ __forceinline__ void lb_fma2(unsigned long long& acc, unsigned long long a, unsigned long long b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ float lb_hsum2(unsigned long long v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo + hi;
}

template <int JN, typename OnBlock>
__device__ __forceinline__ void lb_cost_stream(const float* xc, const float* xn_c, int d, int m, const float* ys,
                                               int ystride, const float* yn, int lane, float* ring,
                                               OnBlock&& on_block) {
    const int nch = (d + 31) >> 5, steps = ((m + 7) >> 3) * nch;
    auto issue = [&](int s) {
        if (s < steps) {
            const int ib = s / nch, ch = s - ib * nch;
            float* st = ring + (s % LB_XS) * LB_XSTAGE;
#pragma unroll
            for (int k = 0; k < 2; ++k) {  // 8 rows x 8 segments of 16 bytes
                const int e = lane + 32 * k, r = e >> 3, t = ch * 32 + (e & 7) * 4;
                if (t < d) lb_cp16(st + r * 32 + (e & 7) * 4, xc + (int64_t)min(ib * 8 + r, m - 1) * d + t);
            }
        }
        asm volatile("cp.async.commit_group;");
    };
#pragma unroll
    for (int s = 0; s < LB_XS - 1; ++s) issue(s);
    unsigned long long acc[8][JN];  // (even, odd) dimension partial sums
    for (int s = 0; s < steps; ++s) {
        issue(s + LB_XS - 1);  // into the stage read in step s - 1
        asm volatile("cp.async.wait_group %0;" ::"n"(LB_XS - 1));
        __syncwarp();
        const int ib = s / nch, ch = s - ib * nch;
        if (ch == 0) {
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int q = 0; q < JN; ++q) acc[u][q] = 0ull;
        }
        const float* st = ring + (s % LB_XS) * LB_XSTAGE;
        const int tn = min(32, d - ch * 32);
        for (int t = 0; t < tn; t += 4) {
            ulonglong2 yv[JN];  // dimensions (t, t + 1), (t + 2, t + 3)
#pragma unroll
            for (int q = 0; q < JN; ++q)
                yv[q] = *reinterpret_cast<const ulonglong2*>(&ys[(lane + 32 * q) * ystride + ch * 32 + t]);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const ulonglong2 xv = *reinterpret_cast<const ulonglong2*>(st + u * 32 + t);
#pragma unroll
                for (int q = 0; q < JN; ++q) {
                    lb_fma2(acc[u][q], xv.x, yv[q].x);
                    lb_fma2(acc[u][q], xv.y, yv[q].y);
                }
            }
        }
        __syncwarp();  // every lane has read the stage before it is refilled
        if (ch == nch - 1) {
            float cij[8][JN];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float xni = xn_c[min(ib * 8 + u, m - 1)];
#pragma unroll
                for (int q = 0; q < JN; ++q)
                    cij[u][q] = fmaxf(fmaf(-2.f, lb_hsum2(acc[u][q]), xni + yn[lane + 32 * q]), 0.f);
            }
            on_block(ib * 8, cij);
        }
    }
    asm volatile("cp.async.wait_group 0;");
    __syncwarp();
}

// One CTA per bag (grid-stride), the bag's rows in shared memory; warp w
// bounds centroids w, w + 8, ...; lanes own bag points j = lane + 32 t.
// The one-sided relaxations of centroid c against the bag in the tile, with
// JE bag-point slots per lane (JE = the smallest of 1, 2, 4 covering the bag:
// a tile sized for the largest bag costs no lanes on a smaller one).
template <int JE>
__device__ __forceinline__ void lb_cheap_pair(const LbArgs& a, int c, int n, const float* ys, const float* yn,
                                              const float* uy, int lane, float* ring, float& lb1, float& lb2) {
    const int d = a.d, m = a.m;
    const float* xc = a.x + (int64_t)c * m * d;
    float colmin[JE];
#pragma unroll
    for (int q = 0; q < JE; ++q) colmin[q] = 3.0e38f;
    lb2 = 0.f;
    // (rows past n read zero-initialised tail rows of the tile: harmless)
    auto on_block = [&](int i0, const float (&cij)[8][JE]) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (i0 + u >= m) break;
            float rmin = 3.0e38f;
#pragma unroll
            for (int q = 0; q < JE; ++q) {
                const int j = lane + 32 * q;
                if (j < n) {
                    colmin[q] = fminf(colmin[q], cij[u][q]);
                    rmin = fminf(rmin, cij[u][q]);
                }
            }
            rmin = group_min<32>(rmin);
            lb2 = fmaf(a.w[(int64_t)c * m + i0 + u], rmin, lb2);
        }
    };
    if (a.vec) {
        lb_cost_stream<JE>(xc, a.xn + (int64_t)c * m, d, m, ys, a.ystride, yn, lane, ring, on_block);
    } else {
        for (int i0 = 0; i0 < m; i0 += 8) {
            float cij[8][JE];
            lb_cost8<JE>(xc, a.xn + (int64_t)c * m, d, m, i0, ys, a.ystride, yn, lane, false, cij);
            on_block(i0, cij);
        }
    }
    lb1 = 0.f;
#pragma unroll
    for (int q = 0; q < JE; ++q) {
        const int j = lane + 32 * q;
        if (j < n) lb1 = fmaf(uy[j], colmin[q], lb1);
    }
    lb1 = group_sum<32>(lb1);
}

// The cheap bounds LB1, LB2 (the LP's one-sided relaxations) and LB3 (the
// means) of every (bag, centroid) pair on the CUDA cores: one CTA per bag
// (grid-stride) with the bag's rows in shared memory, warp w taking the
// centroids w, w + LB_WARPS, ...; writes max(LB1, LB2, LB3) to lb.
template <int JN>
__global__ void __launch_bounds__(LB_WARPS * 32) k_lb_pairs(LbArgs a) {
    extern __shared__ __align__(16) float lb_dyn[];
    const int rows = 32 * JN;                             // tile rows (>= max_mk)
    float* ys = lb_dyn;                                   // rows x ystride
    float* yn = ys + (size_t)rows * a.ystride;            // rows
    float* uy = yn + rows;                                // rows
    float* mp = uy + rows;                                // d
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d, K = a.K;
    // the warp's ring for streamed centroid rows (16-byte aligned: the host
    // pads the tile to a multiple of 4 floats)
    float* ring = lb_dyn + a.ring_off + (size_t)warp * LB_XS * LB_XSTAGE;
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
            float lb1, lb2;
            if constexpr (JN == 1) {
                lb_cheap_pair<1>(a, c, n, ys, yn, uy, lane, ring, lb1, lb2);
            } else {
                if (n <= 32) lb_cheap_pair<1>(a, c, n, ys, yn, uy, lane, ring, lb1, lb2);
                else if (JN == 2 || n <= 64) lb_cheap_pair<2>(a, c, n, ys, yn, uy, lane, ring, lb1, lb2);
                else lb_cheap_pair<JN>(a, c, n, ys, yn, uy, lane, ring, lb1, lb2);
            }
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

// Entropic dual bound.  The LP of Eq. (primal) has the dual
//     max sum_i v_i f_i + sum_j u_j g_j   s.t.  f_i + g_j <= C_ij,
// so every feasible (f, g) bounds W^2 from below.  Sinkhorn iterations of
// the entropy-regularised problem (regularisation eps) give potentials close
// to an optimal pair; the c-transform g'_j = min_i (C_ij - f_i) (or
// f'_i = min_j (C_ij - g_j)) makes them feasible.  Only the final transform
// and the two sums decide the bound's validity, so the iterations may use the
// hardware's approximate 2^x and log2 x.  For the pairs that the bounds above
// did not exclude, the larger of the two transformed duals replaces the
// bound when it is larger.  One warp per (bag, centroid) pair: the pair's
// m x m_k cost matrix in the warp's shared memory (m <= 64), potentials in
// log2 units (F = f / (eps ln 2), G = g / (eps ln 2)), lanes owning centroid
// points in the F update and bag points in the G update.
#define LB_DUAL_MMAX 64
#define LB_DUAL_KCAP 1024  // centroids listed per round of a bag
#define LB_DUAL_ITERS 40    // Sinkhorn iterations by default (m >= 32)
#define LB_DUAL_EPS 0.05f   // eps as a fraction of the pair's mean cost
#define LB_DUAL_CHECK 10    // iterations between checks of the bound against the threshold

struct DualArgs {
    const int32_t* cand;  // N x r first candidates (solved exactly)
    const float* w2c;     // N x r their values
    int r, iters, nw;
    float eps_rel;
};

__device__ __forceinline__ float lb_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lb_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The pair's cost matrix into the warp's Cw (rows cs floats apart) with JE
// bag-point slots per lane; returns the sum of its entries (every lane).
template <int JE>
__device__ __forceinline__ float lb_dual_cost(const LbArgs& a, int c, int n, const float* ys, const float* yn,
                                              int lane, float* ring, float* Cw, int cs) {
    const int d = a.d, m = a.m;
    const float* xc = a.x + (int64_t)c * m * d;
    float csum = 0.f;
    auto on_block = [&](int i0, const float (&cij)[8][JE]) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (i0 + u >= m) break;
#pragma unroll
            for (int q = 0; q < JE; ++q) {
                const int j = lane + 32 * q;
                if (j < n) {
                    Cw[(i0 + u) * cs + j] = cij[u][q];
                    csum += cij[u][q];
                }
            }
        }
    };
    if (a.vec) {
        lb_cost_stream<JE>(xc, a.xn + (int64_t)c * m, d, m, ys, a.ystride, yn, lane, ring, on_block);
    } else {
        for (int i0 = 0; i0 < m; i0 += 8) {
            float cij[8][JE];
            lb_cost8<JE>(xc, a.xn + (int64_t)c * m, d, m, i0, ys, a.ystride, yn, lane, false, cij);
            on_block(i0, cij);
        }
    }
    return group_sum<32>(csum);
}

// The entropic dual bound for the pairs that the cheap bounds leave above
// each bag's threshold (the best exact value of its first candidates, with
// the slack).  One CTA per bag (grid-stride), the bag's rows in shared
// memory; the bag's listed pairs are dealt to the da.nw warps in turn.  Per
// pair a warp builds the m x m_k cost matrix in its own shared memory, runs
// the Sinkhorn iterations in log2 units (checking the bound every
// LB_DUAL_CHECK iterations), and takes the larger of the two c-transformed
// dual objectives of Eq. (primal)'s dual, which never exceeds W^2; it
// replaces the pair's bound in lb when larger.
template <int JN>
__global__ void __launch_bounds__(LB_WARPS * 32, 1) k_lb_dual(LbArgs a, DualArgs da) {
    extern __shared__ __align__(16) float lb_dyn[];
    const int rows = 32 * JN;
    float* ys = lb_dyn;                                   // rows x ystride
    float* yn = ys + (size_t)rows * a.ystride;            // rows: ||y_j||^2
    float* uy = yn + rows;                                // rows: u_j
    float* ly = uy + rows;                                // rows: log2 u_j
    float* wbase = ly + rows;                             // per warp below
    __shared__ float s_thr;
    __shared__ int s_cnt;
    __shared__ int s_list[LB_DUAL_KCAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = a.d, m = a.m, K = a.K;
    constexpr int cs = 32 * JN + 1;  // cost row stride (odd: rows fall in distinct banks)
    float* Cw = wbase + (size_t)warp * (LB_DUAL_MMAX * cs + 2 * LB_DUAL_MMAX + rows);
    float* ring = lb_dyn + a.ring_off + (size_t)warp * LB_XS * LB_XSTAGE;
    float* Fa = Cw + LB_DUAL_MMAX * cs;   // F_i + log2 v_i (v_i > 0), else -inf
    float* Fs = Fa + LB_DUAL_MMAX;        // F_i
    float* Gb = Fs + LB_DUAL_MMAX;        // G_j + log2 u_j
    for (int64_t bag = blockIdx.x; bag < a.N; bag += gridDim.x) {
        const int64_t r0 = a.offsets[bag];
        const int n = (int)(a.offsets[bag + 1] - r0);
        __syncthreads();
        if (threadIdx.x == 0) {
            float best = 3.4e38f;
            for (int t = 0; t < da.r; ++t) best = fminf(best, da.w2c[bag * da.r + t]);
            s_thr = best * (1.f + LB_SLACK) + 1e-6f;
        }
        __syncthreads();
        // skip the bag when none of its other centroids is left to exclude
        int need = 0;
        for (int c = threadIdx.x; c < K; c += blockDim.x) {
            bool first = false;
            for (int t = 0; t < da.r; ++t) first |= da.cand[bag * da.r + t] == c;
            need |= !first && a.lb[bag * K + c] <= s_thr;
        }
        if (!__syncthreads_or(need)) continue;
        for (int e = threadIdx.x; e < rows * d; e += blockDim.x) {
            const int j = e / d, t = e - j * d;
            ys[j * a.ystride + t] = j < n ? d2_row_ptr(a.supp, a.vidx, a.vocab, d, r0 + j)[t] : 0.f;
        }
        for (int j = threadIdx.x; j < rows; j += blockDim.x) {
            const float u = j < n ? a.wt[r0 + j] : 0.f;
            uy[j] = u;
            ly[j] = u > 0.f ? lb_lg2(u) : -3.0e38f;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            float s = 0.f;
            for (int t = 0; t < d; ++t) s = fmaf(ys[j * a.ystride + t], ys[j * a.ystride + t], s);
            yn[j] = s;
        }
        __syncthreads();
        const float thr = s_thr;
        // the bag's pairs to bound, LB_DUAL_KCAP centroids at a time, dealt
        // to the warps in turn (each pair's result is its own: the order in
        // which they are listed does not matter)
        for (int c0 = 0; c0 < K; c0 += LB_DUAL_KCAP) {
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (int c = c0 + threadIdx.x; c < min(K, c0 + LB_DUAL_KCAP); c += blockDim.x) {
            bool first = false;
            for (int t = 0; t < da.r; ++t) first |= da.cand[bag * da.r + t] == c;
            if (!first && a.lb[bag * K + c] <= thr) s_list[atomicAdd(&s_cnt, 1)] = c;
        }
        __syncthreads();
        const int cnt = s_cnt;
        for (int li = warp; li < cnt; li += da.nw) {
            const int c = s_list[li];
            const float lb0 = a.lb[bag * K + c];
            // the cost matrix, C_ij = max(||x_i||^2 + ||y_j||^2 - 2 <x_i, y_j>, 0)
            float csum;
            if constexpr (JN == 1) {
                csum = lb_dual_cost<1>(a, c, n, ys, yn, lane, ring, Cw, cs);
            } else {
                csum = n <= 32                ? lb_dual_cost<1>(a, c, n, ys, yn, lane, ring, Cw, cs)
                       : (JN == 2 || n <= 64) ? lb_dual_cost<2>(a, c, n, ys, yn, lane, ring, Cw, cs)
                                              : lb_dual_cost<JN>(a, c, n, ys, yn, lane, ring, Cw, cs);
            }
            const float eps = da.eps_rel * csum / (float)(m * n);
            const float sc = eps > 0.f ? 1.4426950408889634f / eps : 0.f;  // 1 / (eps ln 2)
            const float* wc = a.w + (int64_t)c * m;
            // lanes own centroid points i = lane, lane + 32 in the F update
            float lw[2];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int i = lane + 32 * p;
                lw[p] = i < m && wc[i] > 0.f ? lb_lg2(wc[i]) : -3.0e38f;
                if (i < m) {
                    Fs[i] = 0.f;
                    Fa[i] = lw[p];
                }
            }
            for (int j = lane; j < rows; j += 32) Gb[j] = j < n ? ly[j] : -3.0e38f;
            __syncwarp();
            // both c-transforms, in cost units (f = F / sc, g = G / sc): the
            // larger dual objective (the same value on every lane)
            auto dual_obj = [&]() -> float {
                const float isc = sc > 0.f ? 1.f / sc : 0.f;
                float part_a = 0.f, part_b = 0.f;  // lane shares of the two dual objectives
#pragma unroll
                for (int q = 0; q < JN; ++q) {
                    const int j = lane + 32 * q;
                    if (j < n) {
                        float g2 = 3.0e38f;
                        for (int i = 0; i < m; ++i) g2 = fminf(g2, Cw[i * cs + j] - Fs[i] * isc);
                        part_a = fmaf(uy[j], g2, part_a);
                        part_b = fmaf(uy[j], (Gb[j] - ly[j]) * isc, part_b);
                    }
                }
                for (int i = lane; i < m; i += 32) {
                    const float* ci = Cw + i * cs;
                    float f2 = 3.0e38f;
                    for (int j = 0; j < n; ++j) f2 = fminf(f2, ci[j] - (Gb[j] - ly[j]) * isc);
                    part_a = fmaf(wc[i], Fs[i] * isc, part_a);
                    part_b = fmaf(wc[i], f2, part_b);
                }
                part_a = group_sum<32>(part_a);
                part_b = group_sum<32>(part_b);
                return fmaxf(part_a, part_b);
            };
            // Each log-sum-exp is shifted by the previous iteration's value of
            // the same potential (its sum of powers is then near 1); a sum
            // outside [2^-100, 2^100] is taken again with the exact maximum.
            // F_i from its row's sum (sh: the shift the sum was taken with)
            auto f_finish = [&](int i, float sh, float sum, float lwi) {
                if (!(sum >= 0x1p-100f && sum <= 0x1p100f)) {
                    const float* ci = Cw + i * cs;
                    sh = -3.0e38f;
                    for (int j = 0; j < n; ++j) sh = fmaxf(sh, fmaf(-sc, ci[j], Gb[j]));
                    sum = 0.f;
                    for (int j = 0; j < n; ++j) sum += lb_ex2(fmaf(-sc, ci[j], Gb[j]) - sh);
                }
                const float F = -(sh + lb_lg2(sum));
                Fs[i] = F;
                Fa[i] = lwi + F;
            };
            float dual = 0.f;
            bool early = false;
            for (int it = 0; sc > 0.f && it < da.iters; ++it) {
                // F_i = -log2 sum_j 2^(G_j + log2 u_j - sc C_ij): lanes own
                // rows i = lane (and lane + 32); several partial sums per row
                // keep the chains of dependent additions short
                if (m > 32) {
                    const int i1 = lane + 32;
                    const bool h1 = i1 < m;
                    const float* c0 = Cw + lane * cs;
                    const float* c1 = Cw + (h1 ? i1 : lane) * cs;
                    const float sh0 = -Fs[lane], sh1 = -Fs[h1 ? i1 : lane];
                    float s0a = 0.f, s0b = 0.f, s1a = 0.f, s1b = 0.f;
                    int j = 0;
                    for (; j + 1 < n; j += 2) {
                        const float g0 = Gb[j], g1 = Gb[j + 1];
                        s0a += lb_ex2(fmaf(-sc, c0[j], g0) - sh0);
                        s1a += lb_ex2(fmaf(-sc, c1[j], g0) - sh1);
                        s0b += lb_ex2(fmaf(-sc, c0[j + 1], g1) - sh0);
                        s1b += lb_ex2(fmaf(-sc, c1[j + 1], g1) - sh1);
                    }
                    if (j < n) {
                        const float g0 = Gb[j];
                        s0a += lb_ex2(fmaf(-sc, c0[j], g0) - sh0);
                        s1a += lb_ex2(fmaf(-sc, c1[j], g0) - sh1);
                    }
                    f_finish(lane, sh0, s0a + s0b, lw[0]);
                    if (h1) f_finish(i1, sh1, s1a + s1b, lw[1]);
                } else {
                    const int i0 = lane < m ? lane : 0;  // lanes past m: row 0, result unused
                    const float* c0 = Cw + i0 * cs;
                    const float sh0 = lane < m ? -Fs[lane] : 0.f;
                    float s[4] = {0.f, 0.f, 0.f, 0.f};
                    int j = 0;
                    for (; j + 3 < n; j += 4) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) s[t] += lb_ex2(fmaf(-sc, c0[j + t], Gb[j + t]) - sh0);
                    }
                    for (; j < n; ++j) s[0] += lb_ex2(fmaf(-sc, c0[j], Gb[j]) - sh0);
                    if (lane < m) f_finish(lane, sh0, (s[0] + s[1]) + (s[2] + s[3]), lw[0]);
                }
                __syncwarp();
                // G_j = -log2 sum_i 2^(F_i + log2 v_i - sc C_ij) for u_j > 0.
                // A lane per column for the first 32 floor(n / 32) columns
                // (four partial sums over i, no shuffles) ...
                const int nfull = n & ~31;
                for (int jb = 0; jb < nfull; jb += 32) {
                    const int j = jb + lane;
                    const float* cj = Cw + j;
                    const float sh = ly[j] - Gb[j];  // minus the previous G_j
                    float s[4] = {0.f, 0.f, 0.f, 0.f};
                    int i = 0;
                    for (; i + 3 < m; i += 4) {
#pragma unroll
                        for (int t = 0; t < 4; ++t) s[t] += lb_ex2(fmaf(-sc, cj[(i + t) * cs], Fa[i + t]) - sh);
                    }
                    for (; i < m; ++i) s[0] += lb_ex2(fmaf(-sc, cj[i * cs], Fa[i]) - sh);
                    float sum = (s[0] + s[1]) + (s[2] + s[3]), s2 = sh;
                    if (uy[j] > 0.f) {
                        if (!(sum >= 0x1p-100f && sum <= 0x1p100f)) {
                            s2 = -3.0e38f;
                            for (int i2 = 0; i2 < m; ++i2) s2 = fmaxf(s2, fmaf(-sc, cj[i2 * cs], Fa[i2]));
                            sum = 0.f;
                            for (int i2 = 0; i2 < m; ++i2) sum += lb_ex2(fmaf(-sc, cj[i2 * cs], Fa[i2]) - s2);
                        }
                        Gb[j] = -(s2 + lb_lg2(sum)) + ly[j];
                    }
                }
                // ... and gs lanes per column for the rest (rem gs <= 32): each
                // lane sums a contiguous block of rows, then a butterfly sum
                // within its group of gs lanes (the same value on all of them)
                const int rem = n - nfull;
                if (rem > 0) {
                    int lg = 5;
                    while ((rem << lg) > 32) --lg;
                    const int gs = 1 << lg;
                    const int g = lane >> lg, il = lane & (gs - 1);
                    const bool act = g < rem;
                    const int j = nfull + (act ? g : 0);  // idle groups read a real column
                    const int rpl = (m + gs - 1) >> lg;
                    const int ib = min(m, il * rpl), ie = min(m, ib + rpl);
                    const float* cj = Cw + j;
                    const float sh = ly[j] - Gb[j];
                    float s0 = 0.f, s1 = 0.f;
                    int i = ib;
                    for (; i + 1 < ie; i += 2) {
                        s0 += lb_ex2(fmaf(-sc, cj[i * cs], Fa[i]) - sh);
                        s1 += lb_ex2(fmaf(-sc, cj[(i + 1) * cs], Fa[i + 1]) - sh);
                    }
                    if (i < ie) s0 += lb_ex2(fmaf(-sc, cj[i * cs], Fa[i]) - sh);
                    float sum = s0 + s1, s2 = sh;
                    for (int o = gs >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                    const bool live = act && uy[j] > 0.f;
                    if (__any_sync(0xffffffffu, live && !(sum >= 0x1p-100f && sum <= 0x1p100f))) {
                        float mx = -3.0e38f;
                        for (int i2 = ib; i2 < ie; ++i2) mx = fmaxf(mx, fmaf(-sc, cj[i2 * cs], Fa[i2]));
                        for (int o = gs >> 1; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                        float v = 0.f;
                        for (int i2 = ib; i2 < ie; ++i2) v += lb_ex2(fmaf(-sc, cj[i2 * cs], Fa[i2]) - mx);
                        for (int o = gs >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (!(sum >= 0x1p-100f && sum <= 0x1p100f)) {
                            s2 = mx;
                            sum = v;
                        }
                    }
                    if (live && il == 0) Gb[j] = -(s2 + lb_lg2(sum)) + ly[j];
                }
                __syncwarp();
                // every LB_DUAL_CHECK iterations: stop once the pair is excluded
                if ((it + 1) % LB_DUAL_CHECK == 0 && it + 1 < da.iters) {
                    dual = dual_obj();
                    if (dual > thr) {
                        early = true;
                        break;
                    }
                }
            }
            if (!early) dual = dual_obj();
            if (lane == 0 && dual > lb0 && dual < 3.0e38f) a.lb[bag * K + c] = dual;
            __syncwarp();
        }
        __syncthreads();  // s_list is rebuilt for the next centroid range
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

// After the dual bound: per bag, the centroid of smallest bound among those
// not solved yet and not excluded (ties: lower index), as one extra exact
// solve (the bound being within about 1 % of W^2 there, it is usually the
// argmin, and its value tightens the exclusion test of every other one).
__global__ void k_lb_next(int64_t N, int K, int r, const float* lb, const int32_t* cand, const float* w2c,
                          int32_t* cand2, float* w2c2, int64_t* pb2, int32_t* pc2, int64_t* npairs2) {
    const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    float best = 3.4e38f;
    for (int t = 0; t < r; ++t) best = fminf(best, w2c[k * r + t]);
    const float thr = best * (1.f + LB_SLACK) + 1e-6f;
    float bv = 3.4e38f;
    int bi = 0x7fffffff;
    for (int i = lane; i < K; i += 32) {
        bool is_c = false;
        for (int t = 0; t < r; ++t) is_c |= cand[k * r + t] == i;
        const float v = lb[k * K + i];
        if (!is_c && v <= thr && v < bv) {  // lanes scan ascending i: the first minimum
            bv = v;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov < bv || (ov == bv && oi < bi)) {
            bv = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        w2c2[k] = 3.4e38f;
        cand2[k] = -1;
        if (bi != 0x7fffffff) {
            cand2[k] = bi;
            const unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long*>(npairs2), 1ull);
            pb2[pos] = k;
            pc2[pos] = bi;
        }
    }
}

__global__ void k_lb_next_scatter(const int64_t* npairs2, const int64_t* pb2, const float* val2, float* w2c2) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= *npairs2) return;
    w2c2[pb2[t]] = val2[t];
}

// First-pass values into D (N x K, +inf elsewhere) and the pair list of every
// other centroid whose bound does not exceed the best value found (the r
// first candidates and, when given, the extra one of k_lb_next)
__global__ void k_lb_second(int64_t N, int K, int r, const float* lb, const int32_t* cand, const float* w2c,
                            const int32_t* cand2, const float* w2c2, float* D, int64_t* pb, int32_t* pc,
                            int64_t* npairs) {
    const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    float best = 3.4e38f;
    for (int t = 0; t < r; ++t) best = fminf(best, w2c[k * r + t]);
    const int c2 = cand2 ? cand2[k] : -1;
    if (c2 >= 0) best = fminf(best, w2c2[k]);
    const float thr = best * (1.f + LB_SLACK) + 1e-6f;
    for (int i = lane; i < K; i += 32) {
        bool is_c = false;
        float v = 3.4e38f;
        for (int t = 0; t < r; ++t)
            if (cand[k * r + t] == i) {
                is_c = true;
                v = w2c[k * r + t];
            }
        if (i == c2) {
            is_c = true;
            v = w2c2[k];
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

__global__ void k_lb_count(int64_t* counters, const int64_t* npairs, const int64_t* npairs2, int64_t first) {
    counters[0] += first + *npairs + (npairs2 ? *npairs2 : 0);
}

// from assign_lb_tc.cu
int d2_lb_pairs_tc(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w, const float* xn,
                   const float* mq, float* lb, cudaStream_t st, bool* used);

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
                 o_cnt = take(64), o_c2 = take((size_t)N * 4), o_w2 = take((size_t)N * 4),
                 o_pb2 = take((size_t)N * 8), o_pc2 = take((size_t)N * 4), o_v2 = take((size_t)N * 4);
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
    int64_t* cnt = reinterpret_cast<int64_t*>(bb + o_cnt);  // [0]: list, [1]: extra candidates
    int32_t* cand2 = reinterpret_cast<int32_t*>(bb + o_c2);
    float* w2c2 = reinterpret_cast<float*>(bb + o_w2);
    int64_t* pb2 = reinterpret_cast<int64_t*>(bb + o_pb2);
    int32_t* pc2 = reinterpret_cast<int32_t*>(bb + o_pc2);
    float* val2 = reinterpret_cast<float*>(bb + o_v2);
    bool extra = false;

    // bounds for every pair
    d2_time_begin(ctx, D2_KT_BOUND, st);
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
    // 16-byte loads when every row starts on a 16-byte boundary; the tile's row
    // stride then a multiple of 4 floats with an odd quotient (8 consecutive
    // lanes' 16-byte reads of one column hit distinct bank groups), else odd
    // (lanes reading one column of consecutive rows hit distinct banks)
    a.vec = d % 4 == 0 && ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(b->supp ? b->supp : b->vocab)) & 15) == 0;
    a.ystride = a.vec ? ((d / 4) % 2 ? d : d + 4) : (d | 1);
    a.x = x;
    a.w = w;
    a.xn = xn;
    a.mq = mq;
    a.lb = lb;
    a.N = N;
    const int JN = b->max_mk <= 32 ? 1 : b->max_mk <= 64 ? 2 : 4;
    a.ring_off = ((int64_t)32 * JN * a.ystride + 2 * 32 * JN + d + 3) & ~(int64_t)3;
    const size_t smem = ((size_t)a.ring_off + (a.vec ? (size_t)LB_WARPS * LB_XS * LB_XSTAGE : 0)) * 4;
    if (smem > 200 * 1024) return d2_fail(ctx, D2_ENOTSUP, "bounded assignment: bag tile of %zu bytes", smem);
    const void* fn = JN == 1 ? (const void*)k_lb_pairs<1> : JN == 2 ? (const void*)k_lb_pairs<2> : (const void*)k_lb_pairs<4>;
    if (smem > 48 * 1024) D2_CK(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 152, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    // the cost entries on the tensor cores where that kernel applies
    bool tc_bounds = false;
    if ((rc = d2_lb_pairs_tc(ctx, b, K, m, x, w, xn, mq, lb, st, &tc_bounds))) return rc;
    if (!tc_bounds) {
        D2_CK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LB_WARPS * 32, smem));
        const unsigned grid =
            (unsigned)std::max<int64_t>(1, std::min<int64_t>(N, (int64_t)sms * std::max(per_sm, 1) * 4));
        d2_time_begin(ctx, D2_KT_BOUND, st);
        if (JN == 1) k_lb_pairs<1><<<grid, LB_WARPS * 32, smem, st>>>(a);
        else if (JN == 2) k_lb_pairs<2><<<grid, LB_WARPS * 32, smem, st>>>(a);
        else k_lb_pairs<4><<<grid, LB_WARPS * 32, smem, st>>>(a);
        d2_time_end(ctx, st);
        D2_LAUNCH_CK(ctx, "k_lb_pairs");
    }
    // first candidates: the pruner's r, else the r smallest bounds
    if (prune) {
        if ((rc = d2_prune_candidates(ctx, b, K, m, x, w, prune, r, cand, st))) return rc;
    } else {
        k_lb_first<<<(unsigned)d2_ceil_div(N, 128), 128, 0, st>>>(N, K, r, lb, cand);
        D2_LAUNCH_CK(ctx, "k_lb_first");
    }
    if ((rc = d2_prune_solve_pairs(ctx, b, K, m, x, w, 3, N * r, nullptr, cand, r, nullptr, w2c, counters + 2, st)))
        return rc;
    // the entropic dual bound for the pairs the cheap bounds left
    const int iters = ctx->dual_iters >= 0 ? ctx->dual_iters : (m >= 32 ? LB_DUAL_ITERS : 0);
    if (iters > 0 && m <= LB_DUAL_MMAX) {
        DualArgs da;
        da.cand = cand;
        da.w2c = w2c;
        da.r = r;
        da.iters = iters;
        da.eps_rel = ctx->dual_eps > 0.f ? ctx->dual_eps : LB_DUAL_EPS;
        const int cstride = 32 * JN + 1;  // the kernel's cost row stride (floats)
        const size_t tile = ((size_t)32 * JN * a.ystride + 3 * (size_t)32 * JN) * 4;
        const size_t per_warp = ((size_t)LB_DUAL_MMAX * cstride + 2 * LB_DUAL_MMAX + 32 * JN +
                                 (a.vec ? (size_t)LB_XS * LB_XSTAGE : 0)) * 4;
        int optin = 0;
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
        // (less the static shared memory of the kernel and the per-CTA reserve)
        const size_t avail = (size_t)std::max(0, optin - 1024 - (int)(LB_DUAL_KCAP * 4 + 64));
        da.nw = avail > tile ? (int)std::min<size_t>(LB_WARPS, (avail - tile) / per_warp) : 0;
        if (da.nw >= 1) {
            const size_t dsm = tile + (size_t)da.nw * per_warp;
            LbArgs ad = a;  // rings after the per-warp blocks (all sizes are multiples of 4 floats)
            ad.ring_off = (int64_t)(tile / 4) +
                          (int64_t)da.nw * (LB_DUAL_MMAX * cstride + 2 * LB_DUAL_MMAX + 32 * JN);
            const void* dfn = JN == 1 ? (const void*)k_lb_dual<1> : JN == 2 ? (const void*)k_lb_dual<2>
                                                                            : (const void*)k_lb_dual<4>;
            D2_CK(ctx, cudaFuncSetAttribute(dfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
            int dper = 1;
            D2_CK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dper, dfn, da.nw * 32, dsm));
            const unsigned dgrid =
                (unsigned)std::max<int64_t>(1, std::min<int64_t>(N, (int64_t)sms * std::max(dper, 1) * 4));
            d2_time_begin(ctx, D2_KT_BOUND, st);
            if (JN == 1) k_lb_dual<1><<<dgrid, da.nw * 32, dsm, st>>>(ad, da);
            else if (JN == 2) k_lb_dual<2><<<dgrid, da.nw * 32, dsm, st>>>(ad, da);
            else k_lb_dual<4><<<dgrid, da.nw * 32, dsm, st>>>(ad, da);
            d2_time_end(ctx, st);
            D2_LAUNCH_CK(ctx, "k_lb_dual");
        }
    }
    // one more exact solve per bag: its smallest remaining bound, if that
    // bound is not above the best value found so far
    D2_CK(ctx, cudaMemsetAsync(cnt + 1, 0, 8, st));
    k_lb_next<<<(unsigned)d2_ceil_div(N, 8), 256, 0, st>>>(N, K, r, lb, cand, w2c, cand2, w2c2, pb2, pc2, cnt + 1);
    D2_LAUNCH_CK(ctx, "k_lb_next");
    if ((rc = d2_solve_pair_list(ctx, b, K, m, x, w, pb2, pc2, N, cnt + 1, val2, counters + 2, st))) return rc;
    k_lb_next_scatter<<<(unsigned)d2_ceil_div(N, 256), 256, 0, st>>>(cnt + 1, pb2, val2, w2c2);
    D2_LAUNCH_CK(ctx, "k_lb_next_scatter");
    extra = true;
    // every other centroid whose bound is not above the best value found
    D2_CK(ctx, cudaMemsetAsync(cnt, 0, 8, st));
    k_lb_second<<<(unsigned)d2_ceil_div(N, 8), 256, 0, st>>>(N, K, r, lb, cand, w2c, extra ? cand2 : nullptr,
                                                               extra ? w2c2 : nullptr, D, pb, pc, cnt);
    D2_LAUNCH_CK(ctx, "k_lb_second");
    if ((rc = d2_solve_pair_list(ctx, b, K, m, x, w, pb, pc, N * K, cnt, val, counters + 2, st))) return rc;
    k_scatter_list<<<(unsigned)d2_ceil_div(N * K, 256), 256, 0, st>>>(cnt, pb, pc, val, K, D);
    D2_LAUNCH_CK(ctx, "k_scatter_list");
    k_lb_count<<<1, 1, 0, st>>>(counters, cnt, extra ? cnt + 1 : nullptr, N * r);
    D2_LAUNCH_CK(ctx, "k_lb_count");
    return d2_argmin_rows(ctx, D, N, K, labels, dist, st);
}
