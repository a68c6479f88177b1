// Ragged squared-Euclidean cost matrices C(x_c, x^(k)) (Section 2 notation
// list, c(.,.) under Eq. primal with p = 2) for every member of every cluster.
//
// One CTA per chunk of <= D2_CHUNK consecutive member positions of one
// cluster.  The cluster's centred barycenter support xt = x_c - mu_c is staged
// transposed in shared memory once per column tile; member rows are streamed
// through a transposed, padded shared tile, centred by the same mu_c, and each
// thread produces one full j-major row of C:
//     C[j, i] = ||xt_i||^2 + ||y_j - mu_c||^2 - 2 <xt_i, y_j - mu_c>.
// Centring removes the catastrophic cancellation of the plain norm expansion
// when the data sit far from the origin.
//
// d2_cost_rows dispatches: with a BF16 precision flag and d >= 32 the
// tensor-core build (cost_tc.cu) runs instead, and for bags stored as
// vocabulary indices the per-(cluster, word) table (cost_vocab.cu) on top
// of it; otherwise these FP32 kernels.
#include "d2_internal.cuh"

#define COST_THREADS 256
#define COST_DT 32
#define COST_YPAD (COST_THREADS + 1)

struct CostArgs {
    const int64_t* members;
    const int64_t* offsets;
    const float* supp;
    const int32_t* vidx;
    const float* vocab;
    int d, m;
    const float* xt;   // K x m x d
    const float* xn;   // K x m
    const float* mu;   // K x d
    const Chunk* chunks;
    const int64_t* nchunks;
    float* C;          // n x m
    double* chunk_sum; // per chunk (or null)
    int64_t* chunk_rows;
};

template <int MT>
__global__ void __launch_bounds__(COST_THREADS) k_cost(CostArgs a) {
    extern __shared__ float4 dyn4[];
    float* xs = reinterpret_cast<float*>(dyn4);          // d x MT (transposed tile of xt)
    float* ys = xs + (size_t)a.d * MT;                    // COST_DT x COST_YPAD
    __shared__ int64_t s_rs[D2_CHUNK];
    __shared__ int s_pre[D2_CHUNK + 1];
    __shared__ int64_t s_row[COST_THREADS];
    __shared__ double s_red[COST_THREADS / 32];

    const int64_t q = blockIdx.x;
    if (q >= *a.nchunks) return;
    const Chunk ch = a.chunks[q];
    const int c = ch.c;
    const int nm = (int)(ch.p1 - ch.p0);
    const int d = a.d, m = a.m;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (tid < nm) {
        int64_t k = a.members[ch.p0 + tid];
        s_rs[tid] = a.offsets[k];
        s_pre[tid + 1] = (int)(a.offsets[k + 1] - a.offsets[k]);
    }
    __syncthreads();
    if (tid == 0) {
        s_pre[0] = 0;
        for (int t = 0; t < nm; ++t) s_pre[t + 1] += s_pre[t];
    }
    __syncthreads();
    const int R = s_pre[nm];
    const float* mu = a.mu + (int64_t)c * d;
    double rowsum_acc = 0.0;

    for (int ct = 0; ct < m; ct += MT) {
        __syncthreads();
        for (int idx = tid; idx < d * MT; idx += COST_THREADS) {
            int dd = idx / MT, i = idx - dd * MT;
            xs[idx] = (ct + i < m) ? a.xt[((int64_t)c * m + ct + i) * d + dd] : 0.f;
        }

        for (int rbase = 0; rbase < R; rbase += COST_THREADS) {
            __syncthreads();
            {
                int lr = rbase + tid;
                int64_t grow = -1;
                if (lr < R) {
                    int lo = 0, hi = nm - 1;
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (s_pre[mid] <= lr) lo = mid; else hi = mid - 1;
                    }
                    grow = s_rs[lo] + (lr - s_pre[lo]);
                }
                s_row[tid] = grow;
            }
            const bool valid = rbase + tid < R;
            float acc[MT];
#pragma unroll
            for (int i = 0; i < MT; ++i) acc[i] = 0.f;
            float yn = 0.f;
            for (int d0 = 0; d0 < d; d0 += COST_DT) {
                const int dt = min(COST_DT, d - d0);
                __syncthreads();
                for (int r = warp; r < COST_THREADS; r += COST_THREADS / 32) {
                    int64_t g = s_row[r];
                    if (g < 0) break;  // rows beyond R are at the end
                    const float* yp = d2_row_ptr(a.supp, a.vidx, a.vocab, d, g);
                    if (lane < dt) ys[lane * COST_YPAD + r] = yp[d0 + lane] - mu[d0 + lane];
                }
                __syncthreads();
                if (valid) {
                    for (int dd = 0; dd < dt; ++dd) {
                        const float yv = ys[dd * COST_YPAD + tid];
                        yn = fmaf(yv, yv, yn);
                        const float* xr = xs + (size_t)(d0 + dd) * MT;
                        if constexpr (MT % 4 == 0) {
#pragma unroll
                            for (int i = 0; i < MT; i += 4) {
                                float4 xv = *reinterpret_cast<const float4*>(xr + i);
                                acc[i] = fmaf(xv.x, yv, acc[i]);
                                acc[i + 1] = fmaf(xv.y, yv, acc[i + 1]);
                                acc[i + 2] = fmaf(xv.z, yv, acc[i + 2]);
                                acc[i + 3] = fmaf(xv.w, yv, acc[i + 3]);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < MT; ++i) acc[i] = fmaf(xr[i], yv, acc[i]);
                        }
                    }
                }
            }
            if (valid) {
                const int64_t g = s_row[tid];
                float* out = a.C + g * m + ct;
                const float* xnr = a.xn + (int64_t)c * m + ct;
                const int nv = min(MT, m - ct);
                float rs = 0.f;
                if ((m & 3) == 0 && (MT % 4) == 0) {
#pragma unroll
                    for (int i = 0; i < MT; i += 4) {
                        if (i < nv) {
                            float4 v;
                            v.x = fmaxf(fmaf(-2.f, acc[i], xnr[i] + yn), 0.f);
                            v.y = fmaxf(fmaf(-2.f, acc[i + 1], xnr[i + 1] + yn), 0.f);
                            v.z = fmaxf(fmaf(-2.f, acc[i + 2], xnr[i + 2] + yn), 0.f);
                            v.w = fmaxf(fmaf(-2.f, acc[i + 3], xnr[i + 3] + yn), 0.f);
                            *reinterpret_cast<float4*>(out + i) = v;
                            rs += (v.x + v.y) + (v.z + v.w);
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < MT; ++i) {
                        if (i < nv) {
                            float v = fmaxf(fmaf(-2.f, acc[i], xnr[i] + yn), 0.f);
                            out[i] = v;
                            rs += v;
                        }
                    }
                }
                rowsum_acc += (double)rs;
            }
        }
    }
    if (a.chunk_sum) {
        double v = group_sum_d<32>(rowsum_acc);
        __syncthreads();
        if (lane == 0) s_red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < COST_THREADS / 32; ++w) s += s_red[w];
            a.chunk_sum[q] = s;
            a.chunk_rows[q] = R;
        }
    }
}


// ---------------------------------------------------------------------------
// Pipelined variant for d % 4 == 0: member rows are staged in d-tiles of 32
// floats with cp.async (a warp copies 4 rows of 128 B per instruction) into
// a double-buffered tile [256 rows][36 floats] (row stride 144 B keeps 16-B
// alignment and makes each thread's float4 reads of its own row
// bank-conflict free); the copy of tile t+1 overlaps the FMAs of tile t.
// ---------------------------------------------------------------------------
#define CP_DT 32
#define CP_STRIDE 36

__device__ __forceinline__ void cost_cp16(void* sdst, const void* gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cost_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cost_wait1() { asm volatile("cp.async.wait_group 1;"); }
__device__ __forceinline__ void cost_wait0() { asm volatile("cp.async.wait_group 0;"); }

// Two rows per thread (rows t and t + CP_THREADS of each 256-row pass): every
// broadcast load of the barycenter tile feeds 2 x 4 FMAs.
#define CP_THREADS 128
#define CP_ROWS 256

template <int MT>
__global__ void __launch_bounds__(CP_THREADS) k_cost_pipe(CostArgs a) {
    extern __shared__ float4 dyn4[];
    float* ys = reinterpret_cast<float*>(dyn4);                         // 2 x CP_ROWS x CP_STRIDE
    float* xs = ys + 2 * CP_ROWS * CP_STRIDE;                            // d x MT
    float* smu = xs + (size_t)a.d * MT;                                  // d
    __shared__ int64_t s_rs[D2_CHUNK];
    __shared__ int s_pre[D2_CHUNK + 1];
    __shared__ int64_t s_row[2][CP_ROWS];
    __shared__ double s_red[CP_THREADS / 32];

    const int64_t q = blockIdx.x;
    if (q >= *a.nchunks) return;
    const Chunk ch = a.chunks[q];
    const int c = ch.c;
    const int nm = (int)(ch.p1 - ch.p0);
    const int d = a.d, m = a.m;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < nm) {
        int64_t k = a.members[ch.p0 + tid];
        s_rs[tid] = a.offsets[k];
        s_pre[tid + 1] = (int)(a.offsets[k + 1] - a.offsets[k]);
    }
    for (int t = tid; t < d; t += CP_THREADS) smu[t] = a.mu[(int64_t)c * d + t];
    __syncthreads();
    if (tid == 0) {
        s_pre[0] = 0;
        for (int t = 0; t < nm; ++t) s_pre[t + 1] += s_pre[t];
    }
    __syncthreads();
    const int R = s_pre[nm];
    const int ntile = (d + CP_DT - 1) / CP_DT;
    const int npass = (R + CP_ROWS - 1) / CP_ROWS;
    const int nsteps = npass * ntile;   // (pass, d-tile) steps of one column tile
    double rowsum_acc = 0.0;

    // global rows of pass `ps` into s_row[ps & 1]
    auto rows_of = [&](int ps) {
        for (int rr = tid; rr < CP_ROWS; rr += CP_THREADS) {
            const int lr = ps * CP_ROWS + rr;
            int64_t grow = -1;
            if (lr < R) {
                int lo = 0, hi = nm - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (s_pre[mid] <= lr) lo = mid; else hi = mid - 1;
                }
                grow = s_rs[lo] + (lr - s_pre[lo]);
            }
            s_row[ps & 1][rr] = grow;
        }
    };
    // copy step `st` (pass st / ntile, d-tile st % ntile) into buffer st & 1
    auto issue = [&](int st) {
        const int ps = st / ntile, t = st - ps * ntile, b = st & 1;
        const int d0 = t * CP_DT;
        const int sub = lane >> 3, seg = lane & 7;
        for (int r0 = warp * 4; r0 < CP_ROWS; r0 += 4 * (CP_THREADS / 32)) {
            const int r = r0 + sub;
            const int64_t g = s_row[ps & 1][r];
            const int col = d0 + seg * 4;
            if (g >= 0 && col < d) {
                const float* src = d2_row_ptr(a.supp, a.vidx, a.vocab, d, g) + col;
                cost_cp16(ys + ((size_t)b * CP_ROWS + r) * CP_STRIDE + seg * 4, src);
            }
        }
        cost_commit();
    };

    for (int ct = 0; ct < m; ct += MT) {
        __syncthreads();
        for (int idx = tid; idx < d * MT; idx += CP_THREADS) {
            int dd = idx / MT, i = idx - dd * MT;
            xs[idx] = (ct + i < m) ? a.xt[((int64_t)c * m + ct + i) * d + dd] : 0.f;
        }
        rows_of(0);
        __syncthreads();
        issue(0);
        float acc_a[MT], acc_b[MT];
        float yna = 0.f, ynb = 0.f;
#pragma unroll
        for (int i = 0; i < MT; ++i) {
            acc_a[i] = 0.f;
            acc_b[i] = 0.f;
        }
        for (int stp = 0; stp < nsteps; ++stp) {
            const int ps = stp / ntile, t = stp - ps * ntile;
            if (stp + 1 < nsteps) {
                if (t == ntile - 1) {  // next step starts a new pass: its rows first
                    rows_of(ps + 1);
                    __syncthreads();
                }
                issue(stp + 1);
                cost_wait1();
            } else {
                cost_wait0();
            }
            __syncthreads();
            const int rbase = ps * CP_ROWS;
            const bool va = rbase + tid < R, vb = rbase + tid + CP_THREADS < R;
            if (va) {
                const float* yra = ys + ((size_t)(stp & 1) * CP_ROWS + tid) * CP_STRIDE;
                const float* yrb = yra + (size_t)CP_THREADS * CP_STRIDE;
                const int d0 = t * CP_DT;
                const int dt = min(CP_DT, d - d0);
                for (int dd = 0; dd < dt; dd += 4) {
                    const float4 a4 = *reinterpret_cast<const float4*>(yra + dd);
                    const float4 b4 = *reinterpret_cast<const float4*>(yrb + dd);
                    const float4 m4 = *reinterpret_cast<const float4*>(smu + d0 + dd);
                    const float ya[4] = {a4.x - m4.x, a4.y - m4.y, a4.z - m4.z, a4.w - m4.w};
                    const float yb[4] = {b4.x - m4.x, b4.y - m4.y, b4.z - m4.z, b4.w - m4.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        yna = fmaf(ya[u], ya[u], yna);
                        ynb = fmaf(yb[u], yb[u], ynb);
                        const float* xr = xs + (size_t)(d0 + dd + u) * MT;
#pragma unroll
                        for (int i = 0; i < MT; i += 4) {
                            const float4 xv = *reinterpret_cast<const float4*>(xr + i);
                            acc_a[i] = fmaf(xv.x, ya[u], acc_a[i]);
                            acc_a[i + 1] = fmaf(xv.y, ya[u], acc_a[i + 1]);
                            acc_a[i + 2] = fmaf(xv.z, ya[u], acc_a[i + 2]);
                            acc_a[i + 3] = fmaf(xv.w, ya[u], acc_a[i + 3]);
                            acc_b[i] = fmaf(xv.x, yb[u], acc_b[i]);
                            acc_b[i + 1] = fmaf(xv.y, yb[u], acc_b[i + 1]);
                            acc_b[i + 2] = fmaf(xv.z, yb[u], acc_b[i + 2]);
                            acc_b[i + 3] = fmaf(xv.w, yb[u], acc_b[i + 3]);
                        }
                    }
                }
            }
            if (t == ntile - 1) {  // the pass is complete: emit its rows
                const float* xnr = a.xn + (int64_t)c * m + ct;
                const int nv = min(MT, m - ct);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const bool v = h == 0 ? va : vb;
                    if (v) {
                        const float* acc = h == 0 ? acc_a : acc_b;
                        const float yn = h == 0 ? yna : ynb;
                        const int64_t g = s_row[ps & 1][tid + h * CP_THREADS];
                        float* out = a.C + g * m + ct;
                        float rs = 0.f;
#pragma unroll
                        for (int i = 0; i < MT; i += 4) {
                            if (i < nv) {
                                float4 o;
                                o.x = fmaxf(fmaf(-2.f, acc[i], xnr[i] + yn), 0.f);
                                o.y = fmaxf(fmaf(-2.f, acc[i + 1], xnr[i + 1] + yn), 0.f);
                                o.z = fmaxf(fmaf(-2.f, acc[i + 2], xnr[i + 2] + yn), 0.f);
                                o.w = fmaxf(fmaf(-2.f, acc[i + 3], xnr[i + 3] + yn), 0.f);
                                __stcs(reinterpret_cast<float4*>(out + i), o);
                                rs += (o.x + o.y) + (o.z + o.w);
                            }
                        }
                        rowsum_acc += (double)rs;
                    }
                }
#pragma unroll
                for (int i = 0; i < MT; ++i) {
                    acc_a[i] = 0.f;
                    acc_b[i] = 0.f;
                }
                yna = 0.f;
                ynb = 0.f;
            }
            __syncthreads();  // buffer stp & 1 is refilled two steps later
        }
    }
    if (a.chunk_sum) {
        double v = group_sum_d<32>(rowsum_acc);
        __syncthreads();
        if (lane == 0) s_red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double sum = 0.0;
            for (int w = 0; w < CP_THREADS / 32; ++w) sum += s_red[w];
            a.chunk_sum[q] = sum;
            a.chunk_rows[q] = R;
        }
    }
}

template <int MT>
static int launch_cost_pipe(d2_ctx* ctx, const CostArgs& a, int64_t maxch, cudaStream_t st) {
    size_t smem = ((size_t)2 * CP_ROWS * CP_STRIDE + (size_t)a.d * MT + a.d) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_cost_pipe<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return d2_cuda_fail(ctx, e, "k_cost_pipe smem attribute");
    d2_time_begin(ctx, D2_KT_COST, st);
    k_cost_pipe<MT><<<(unsigned)maxch, CP_THREADS, smem, st>>>(a);
    d2_time_end(ctx, st);
    D2_LAUNCH_CK(ctx, "k_cost_pipe");
    return D2_OK;
}

template <int MT>
static int launch_cost(d2_ctx* ctx, const CostArgs& a, int64_t maxch, cudaStream_t st) {
    size_t smem = ((size_t)a.d * MT + (size_t)COST_DT * COST_YPAD) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_cost<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return d2_cuda_fail(ctx, e, "k_cost smem attribute");
    }
    d2_time_begin(ctx, D2_KT_COST, st);
    k_cost<MT><<<(unsigned)maxch, COST_THREADS, smem, st>>>(a);
    d2_time_end(ctx, st);
    D2_LAUNCH_CK(ctx, "k_cost");
    return D2_OK;
}

int d2_cost_prepare(d2_ctx* ctx, const d2_bags* b, int m, int prec) {
    if (prec) {
        bool used = false;
        int rc = d2_cost_tc_prepare(ctx, b, m, prec, &used);
        if (rc || used) return rc;
    }
    const bool aligned16 = (b->d % 4 == 0) &&
        ((reinterpret_cast<uintptr_t>(b->supp ? b->supp : b->vocab) & 15) == 0) && (m % 4 == 0);
    const int MT = m <= 8 ? 8 : m <= 16 ? 16 : m <= 32 ? 32 : 64;
    size_t smem;
    const void* fn;
    if (aligned16 && ((size_t)2 * CP_ROWS * CP_STRIDE + (size_t)b->d * 64 + b->d) * 4 <= 200 * 1024) {
        smem = ((size_t)2 * CP_ROWS * CP_STRIDE + (size_t)b->d * MT + b->d) * sizeof(float);
        fn = MT == 8 ? (const void*)k_cost_pipe<8> : MT == 16 ? (const void*)k_cost_pipe<16>
           : MT == 32 ? (const void*)k_cost_pipe<32> : (const void*)k_cost_pipe<64>;
    } else {
        smem = ((size_t)b->d * MT + (size_t)COST_DT * COST_YPAD) * sizeof(float);
        fn = MT == 8 ? (const void*)k_cost<8> : MT == 16 ? (const void*)k_cost<16>
           : MT == 32 ? (const void*)k_cost<32> : (const void*)k_cost<64>;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return d2_cuda_fail(ctx, e, "cost kernel smem attribute");
    }
    return D2_OK;
}

int d2_cost_rows(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t P, int K, int m,
                 const ClusterWs& cw, float* C, bool want_sums, int prec, int vt, cudaStream_t st) {
    const int64_t maxch = d2_ceil_div(P, D2_CHUNK) + K + 1;
    double* chunk_sum = nullptr;
    int64_t* chunk_rows = nullptr;
    if (want_sums) {
        void* p = nullptr;
        int rc = d2_ws(ctx, WS_CHUNK_SUM, (size_t)maxch * 16, &p);
        if (rc) return rc;
        chunk_sum = static_cast<double*>(p);
        chunk_rows = reinterpret_cast<int64_t*>(static_cast<char*>(p) + (size_t)maxch * 8);
    }
    if (vt != D2_VT_OFF)
        return d2_vocab_cost_rows(ctx, b, members, P, K, m, cw, C, chunk_sum, chunk_rows, vt == D2_VT_SETUP, prec,
                                  st);
    return d2_cost_rows_direct(ctx, b, members, P, K, m, cw, C, chunk_sum, chunk_rows, prec, st);
}

int d2_cost_rows_direct(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t P, int K, int m,
                        const ClusterWs& cw, float* C, double* chunk_sum, int64_t* chunk_rows, int prec,
                        cudaStream_t st) {
    const int64_t maxch = d2_ceil_div(P, D2_CHUNK) + K + 1;
    CostArgs a;
    a.members = members;
    a.offsets = b->offsets;
    a.supp = b->supp;
    a.vidx = b->vocab_idx;
    a.vocab = b->vocab;
    a.d = b->d;
    a.m = m;
    a.xt = cw.xt;
    a.xn = cw.xn;
    a.mu = cw.mu;
    a.chunks = cw.chunks;
    a.nchunks = cw.nchunks;
    a.C = C;
    a.chunk_sum = chunk_sum;
    a.chunk_rows = chunk_rows;
    if (prec) {  // tensor cores where (d, m) make the build a dense contraction
        bool used = false;
        int rc = d2_cost_tc_rows(ctx, b, members, maxch, m, prec, cw, C, a.chunk_sum, a.chunk_rows, st, &used);
        if (rc || used) return rc;
    }
    if ((size_t)b->d * 64 * 4 + COST_DT * COST_YPAD * 4 > 200 * 1024)
        return d2_fail(ctx, D2_ENOTSUP, "d2_cost: support dimension %d too large for the cost tile", b->d);
    const bool aligned16 = (b->d % 4 == 0) &&
        ((reinterpret_cast<uintptr_t>(b->supp ? b->supp : b->vocab) & 15) == 0) && (m % 4 == 0);
    if (aligned16 && ((size_t)2 * CP_ROWS * CP_STRIDE + (size_t)b->d * 64 + b->d) * 4 <= 200 * 1024) {
        if (m <= 8) return launch_cost_pipe<8>(ctx, a, maxch, st);
        if (m <= 16) return launch_cost_pipe<16>(ctx, a, maxch, st);
        if (m <= 32) return launch_cost_pipe<32>(ctx, a, maxch, st);
        return launch_cost_pipe<64>(ctx, a, maxch, st);
    }
    if (m <= 8) return launch_cost<8>(ctx, a, maxch, st);
    if (m <= 16) return launch_cost<16>(ctx, a, maxch, st);
    if (m <= 32) return launch_cost<32>(ctx, a, maxch, st);
    return launch_cost<64>(ctx, a, maxch, st);
}

extern "C" int d2_cost(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets,
                       const int64_t* members, int64_t P, int32_t K, int32_t m, const float* x,
                       float* C_out, int32_t flags, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (K < 1 || m < 1 || m > 256 || P < 0 || !cluster_offsets || (P > 0 && !members) || !x || !C_out)
        return d2_fail(ctx, D2_EINVAL, "d2_cost: need K >= 1, 1 <= m <= 256 and non-NULL arrays");
    if (reinterpret_cast<uintptr_t>(C_out) & 15)
        return d2_fail(ctx, D2_EINVAL, "d2_cost: C_out must be 16-byte aligned");
    cudaStream_t st = d2_stream(stream);
    ClusterWs cw;
    rc = d2_cluster_ws(ctx, K, m, bags->d, P, &cw);
    if (rc) return rc;
    int32_t* pos_cluster = nullptr;
    rc = d2_setup_clusters(ctx, cluster_offsets, P, K, &pos_cluster, &cw, st);
    if (rc) return rc;
    rc = d2_prep_x(ctx, x, K, m, bags->d, cw, st);
    if (rc) return rc;
    const int prec = d2_cost_prec(flags);
    if ((rc = d2_cost_prepare(ctx, bags, m, prec))) return rc;
    const int vt = d2_vocab_table_applies(bags, K, m, prec, flags) ? D2_VT_SETUP : D2_VT_OFF;
    ctx->expire_test = (flags & D2_TEST_EXPIRE_WAIT) ? 1 : 0;
    rc = d2_cost_rows(ctx, bags, members, P, K, m, cw, C_out, false, prec, vt, st);
    ctx->expire_test = 0;
    return rc;
}
