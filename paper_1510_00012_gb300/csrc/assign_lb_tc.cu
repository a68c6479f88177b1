// Certified lower bounds of the bounded assignment (assignment step of
// Algorithm 1; W^2 is the transportation LP of Eq. primal) with the cost
// entries on the tensor cores (tcgen05 / TMEM, sm_103a).
//
// The bounds are those of k_lb_pairs: for a bag P (points y_j, weights u_j)
// and a centroid Q (points x_i, weights v_i), with C_ij = ||x_i - y_j||^2,
//   LB1 = sum_j u_j min_i C_ij,  LB2 = sum_i v_i min_j C_ij,
//   LB3 = ||mu_P - mu_Q||^2,
// each a lower bound of W^2.  Here, for one bag at a time, the dot products
// <x_i, y_j> against all K m centroid points are one contraction over the
// support dimensions: D = A B^T with
//   A (M = 128 centroid points x K = d padded to 64) = the centroid points,
//   B (N = 64 bag points x K)                        = the bag's points,
// both K-major as stored (a row is a point), issued as kind::f16 MMAs on BF16
// pieces (hi + lo: three products hi*hi + hi*lo + lo*hi) into FP32
// accumulators in tensor memory.  The centroid points are converted once per
// call into a buffer of 128-point tiles (L2-resident) and streamed through a
// ring of cp.async stages, one K block at a time; the bag's points are
// converted once per bag; two TMEM accumulators alternate so that the
// epilogue of one tile overlaps the MMAs of the next.
//
// The split pieces carry the dot products to within 3 * 2^-16 ||x_i|| ||y_j||
// and the FP32 accumulation adds at most d 2^-24 ||x_i|| ||y_j||, so each cost
// entry is known to within E = 2 (3 * 2^-16 + d 2^-24) max ||x_i|| max ||y_j||
// + 2^-22 (max ||x_i||^2 + max ||y_j||^2); LB1 and LB2 are lowered by E (the
// weights sum to 1), which keeps them below W^2.
// Every wait is bounded (about 2 s); on expiry the CTA records
// D2F_DEV_TIMEOUT, stops, frees its tensor memory and returns.
#include <algorithm>

#include "d2_internal.cuh"
#include "tc_util.cuh"

namespace {

constexpr int LT_M = 128;         // centroid points per tile (UMMA M, TMEM lanes)
constexpr int LT_N = 64;          // bag points (UMMA N); bags of <= 64 points
constexpr int LT_S = 3;           // A ring stages (one K block: hi + lo each)
constexpr uint32_t LT_ABLK = LT_M * 128;  // one piece of one K block of A (16 KB)
constexpr uint32_t LT_BBLK = LT_N * 128;  // one piece of one K block of B (8 KB)
constexpr int LT_CS = LT_N + 1;   // row stride of the cost tile in shared memory (floats)
constexpr int LT_KBMAX = 5;       // K blocks: d <= 320

struct LtArgs {
    const int64_t* offsets;
    const float* supp;
    const int32_t* vidx;
    const float* vocab;
    const float* wt;
    int d, m, K, nkb, ntile;
    const uint8_t* xp;    // ntile x nkb x 2 pieces x 16 KB, K-major swizzled
    const float* w;       // K x m
    const float* xn;      // K x m   ||x_i||^2
    const float* xmax;    // K       max_i ||x_i||
    const float* mq;      // K x d   centroid means
    float* lb;            // N x K
    int64_t N;
    int* err;
};

// The centroid points as A tiles: tile t holds points 128 t .. 128 t + 127
// of the K m points (zero past them), K block kb holds dimensions
// 64 kb .. 64 kb + 63 (zero past d), piece 0 the BF16 rounding, piece 1 the
// rounding of the remainder; blocks in (tile, K block) order.
__global__ void k_lt_xprep(const float* x, int K, int m, int d, int nkb, int ntile, uint8_t* xp) {
    const int64_t total = (int64_t)ntile * nkb * LT_M * 8;  // 16-byte chunks of one piece
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c8 = (int)(e & 7), r = (int)((e >> 3) % LT_M);
        const int64_t tk = e / (8 * LT_M);
        const int kb = (int)(tk % nkb), t = (int)(tk / nkb);
        const int64_t p = (int64_t)t * LT_M + r;
        float v[8], rem[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int col = kb * 64 + c8 * 8 + q;
            v[q] = (p < (int64_t)K * m && col < d) ? x[p * d + col] : 0.f;
            rem[q] = v[q] - bf16_round(v[q]);
        }
        uint8_t* blk = xp + (size_t)tk * 2 * LT_ABLK;
        const uint32_t off = sw128_off(r, c8 * 8);
        const uint2 h0 = pack_bf16x4(v[0], v[1], v[2], v[3]), h1 = pack_bf16x4(v[4], v[5], v[6], v[7]);
        const uint2 l0 = pack_bf16x4(rem[0], rem[1], rem[2], rem[3]), l1 = pack_bf16x4(rem[4], rem[5], rem[6], rem[7]);
        *reinterpret_cast<uint4*>(blk + off) = make_uint4(h0.x, h0.y, h1.x, h1.y);
        *reinterpret_cast<uint4*>(blk + LT_ABLK + off) = make_uint4(l0.x, l0.y, l1.x, l1.y);
    }
}

// max_i ||x_i|| of every centroid
__global__ void k_lt_xmax(int K, int m, const float* xn, float* xmax) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    float mx = 0.f;
    for (int i = 0; i < m; ++i) mx = fmaxf(mx, xn[(int64_t)c * m + i]);
    xmax[c] = sqrtf(mx);
}

__device__ __forceinline__ void lt_cp16(uint32_t sdst, const void* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sdst), "l"(gsrc));
}

// One CTA (4 warps) per bag at a time (grid-stride); thread r owns TMEM lane
// r, i.e. centroid point 128 t + r of tile t.
__global__ void __launch_bounds__(128) k_lb_pairs_tc(LtArgs a) {
    extern __shared__ uint8_t lt_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[LT_S + 2];  // A stage read by its MMAs; TMEM buffer complete
    __shared__ float s_yn[LT_N], s_u[LT_N], s_r2[LT_M], s_t1[8 * LT_N];
    __shared__ float s_ymax;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int d = a.d, m = a.m, K = a.K, nkb = a.nkb, ntile = a.ntile;
    const uint32_t raw = smem_u32(lt_raw);
    uint8_t* base = lt_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* Bs = base;                                    // nkb x 2 pieces x 8 KB
    uint8_t* As = Bs + (size_t)nkb * 2 * LT_BBLK;          // LT_S x 2 pieces x 16 KB
    float* Cs = reinterpret_cast<float*>(As + (size_t)LT_S * 2 * LT_ABLK);  // 128 x LT_CS
    float* mp = Cs + LT_M * LT_CS;                        // d: the bag's mean
    const uint32_t As_u = smem_u32(As);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(2u * LT_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < LT_S + 2; ++k) mbar_init(smem_u32(&s_bar[k]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t bar_st = smem_u32(&s_bar[0]), bar_tm = smem_u32(&s_bar[LT_S]);
    const uint32_t idesc = idesc_bf16_f32(LT_M, LT_N);
    const int steps = ntile * nkb, ncc = LT_M / m;
    uint32_t ph_st = 0u, ph_tm = 0u;  // per barrier: parity of the next phase to wait for
    bool dead = false;

    for (int64_t bag = blockIdx.x; bag < a.N && !dead; bag += gridDim.x) {
        const int64_t r0 = a.offsets[bag];
        const int n = (int)(a.offsets[bag + 1] - r0);
        // ---- the bag: B operand (split pieces), norms, weights, mean
        for (int e = tid; e < LT_N * nkb * 8; e += LT_M) {
            const int c8 = e & 7, j = (e >> 3) % LT_N, kb = (e >> 3) / LT_N;
            float v[8], rem[8];
            const float* yr = j < n ? d2_row_ptr(a.supp, a.vidx, a.vocab, d, r0 + j) : nullptr;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int col = kb * 64 + c8 * 8 + q;
                v[q] = (yr && col < d) ? yr[col] : 0.f;
                rem[q] = v[q] - bf16_round(v[q]);
            }
            uint8_t* blk = Bs + (size_t)kb * 2 * LT_BBLK;
            const uint32_t off = sw128_off(j, c8 * 8);
            const uint2 h0 = pack_bf16x4(v[0], v[1], v[2], v[3]), h1 = pack_bf16x4(v[4], v[5], v[6], v[7]);
            const uint2 l0 = pack_bf16x4(rem[0], rem[1], rem[2], rem[3]);
            const uint2 l1 = pack_bf16x4(rem[4], rem[5], rem[6], rem[7]);
            *reinterpret_cast<uint4*>(blk + off) = make_uint4(h0.x, h0.y, h1.x, h1.y);
            *reinterpret_cast<uint4*>(blk + LT_BBLK + off) = make_uint4(l0.x, l0.y, l1.x, l1.y);
        }
        if (tid < LT_N) {
            float s = 0.f;
            if (tid < n) {
                const float* yr = d2_row_ptr(a.supp, a.vidx, a.vocab, d, r0 + tid);
                for (int t = 0; t < d; ++t) s = fmaf(yr[t], yr[t], s);
            }
            s_yn[tid] = s;
            s_u[tid] = tid < n ? a.wt[r0 + tid] : 0.f;
        }
        for (int t = tid; t < d; t += LT_M) {
            float s = 0.f;
            for (int j = 0; j < n; ++j) s = fmaf(a.wt[r0 + j], d2_row_ptr(a.supp, a.vidx, a.vocab, d, r0 + j)[t], s);
            mp[t] = s;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            float mx = 0.f;
            for (int j = 0; j < n; ++j) mx = fmaxf(mx, s_yn[j]);
            s_ymax = sqrtf(mx);
        }

        // ---- A stages: step s = (tile s / nkb, K block s % nkb) into stage s % LT_S
        auto issue = [&](int s) {
            if (s < steps) {
                const int st = s % LT_S;
                if (s >= LT_S) {  // the MMAs of step s - LT_S read this stage
                    if (!mbar_wait_bounded(bar_st + 8 * st, (ph_st >> st) & 1u)) dead = true;
                    ph_st ^= 1u << st;
                }
                const uint8_t* src = a.xp + (size_t)s * 2 * LT_ABLK;  // blocks are stored in step order
                const uint32_t dst = As_u + (uint32_t)st * 2 * LT_ABLK;
                for (int e = tid; e < (int)(2 * LT_ABLK / 16); e += LT_M) lt_cp16(dst + e * 16, src + (size_t)e * 16);
            }
            asm volatile("cp.async.commit_group;");
        };
        // epilogue of tile t: minima per row and per column of each centroid's block
        auto epilogue = [&](int t) {
            const int tb = t & 1;
            if (!mbar_wait_bounded(bar_tm + 8 * tb, (ph_tm >> tb) & 1u)) dead = true;
            ph_tm ^= 1u << tb;
            tc_fence_after();
            const int64_t p = (int64_t)t * LT_M + tid;
            const bool valid = p < (int64_t)K * m;
            const float xn = valid ? a.xn[p] : 0.f;
            float rmin = 3.0e38f;
            for (int cb = 0; cb < LT_N; cb += 16) {
                float acc[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(tb * LT_N + cb), acc);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = cb + q;
                    if (j < n) {
                        const float cv = fmaxf(fmaf(-2.f, acc[q], xn + s_yn[j]), 0.f);
                        Cs[tid * LT_CS + j] = cv;
                        rmin = fminf(rmin, cv);
                    }
                }
            }
            s_r2[tid] = valid ? a.w[p] * rmin : 0.f;
            tc_fence_before();
            __syncthreads();
            for (int task = tid; task < ncc * LT_N; task += LT_M) {
                const int cc = task / LT_N, j = task - cc * LT_N;
                float cm = 3.0e38f;
                if (j < n)
                    for (int rr = 0; rr < m; ++rr) cm = fminf(cm, Cs[(cc * m + rr) * LT_CS + j]);
                s_t1[task] = j < n ? s_u[j] * cm : 0.f;
            }
            __syncthreads();
            if (tid < ncc) {
                const int c = t * ncc + tid;
                if (c < K) {
                    float lb1 = 0.f, lb2 = 0.f, lb3 = 0.f;
                    for (int j = 0; j < LT_N; ++j) lb1 += s_t1[tid * LT_N + j];
                    for (int rr = 0; rr < m; ++rr) lb2 += s_r2[tid * m + rr];
                    for (int k = 0; k < d; ++k) {
                        const float df = mp[k] - a.mq[(int64_t)c * d + k];
                        lb3 = fmaf(df, df, lb3);
                    }
                    const float xm = a.xmax[c], ym = s_ymax;
                    const float err = 2.f * (3.f * 0x1p-16f + (float)d * 0x1p-24f) * xm * ym +
                                      0x1p-22f * (xm * xm + ym * ym);
                    a.lb[bag * K + c] = fmaxf(fmaxf(lb1, lb2) - err, lb3);
                }
            }
            __syncthreads();
        };

        for (int s = 0; s < LT_S - 1; ++s) issue(s);
        for (int s = 0; s < steps; ++s) {
            issue(s + LT_S - 1);
            asm volatile("cp.async.wait_group %0;" ::"n"(LT_S - 1));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc_fence_before();
            if (__syncthreads_or(dead)) {
                dead = true;
                break;
            }
            tc_fence_after();
            const int t = s / nkb, kb = s - t * nkb, st = s % LT_S;
            if (tid == 0) {
                const uint32_t dtm = tmem + (uint32_t)((t & 1) * LT_N);
                const uint32_t a_hi = As_u + (uint32_t)st * 2 * LT_ABLK;
                const uint32_t b_hi = smem_u32(Bs + (size_t)kb * 2 * LT_BBLK);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint32_t ko = (uint32_t)ks * 32u;
                    umma_bf16(dtm, sdesc_sw128(a_hi + ko), sdesc_sw128(b_hi + ko), idesc, (kb | ks) ? 1u : 0u);
                    umma_bf16(dtm, sdesc_sw128(a_hi + ko), sdesc_sw128(b_hi + LT_BBLK + ko), idesc, 1u);
                    umma_bf16(dtm, sdesc_sw128(a_hi + LT_ABLK + ko), sdesc_sw128(b_hi + ko), idesc, 1u);
                }
                umma_commit(bar_st + 8 * st);
                if (kb == nkb - 1) umma_commit(bar_tm + 8 * (t & 1));
            }
            if (kb == nkb - 1 && t >= 1) epilogue(t - 1);
        }
        if (!dead && steps > 0) epilogue(ntile - 1);
        // drain: the last stages' completions (every commit is waited for once)
        asm volatile("cp.async.wait_group 0;");
        for (int s = steps > LT_S ? steps - LT_S : 0; s < steps && !dead; ++s) {
            const int st = s % LT_S;
            if (!mbar_wait_bounded(bar_st + 8 * st, (ph_st >> st) & 1u)) dead = true;
            ph_st ^= 1u << st;
        }
        dead = __syncthreads_or(dead);
    }
    if (dead && tid == 0) atomicOr(a.err, D2F_DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * LT_N) : "memory");
}

}  // namespace

// The cheap lower bounds of every (bag, centroid) pair into lb (N x K) on the
// tensor cores, for bags of <= 64 points, 64 <= d <= 320 and m dividing 128
// (16 <= m <= 128); *used = false (and nothing launched) otherwise, or when
// the context asks for the CUDA-core bounds.  xn and mq as from
// k_centroid_stats.
int d2_lb_pairs_tc(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w, const float* xn,
                   const float* mq, float* lb, cudaStream_t st, bool* used) {
    *used = false;
    const int d = b->d;
    // (below d = 64 the CUDA-core dot products cost less than the tile schedule)
    if (ctx->bound_cuda_cores || b->max_mk > LT_N || m < 16 || m > LT_M || LT_M % m != 0 || d < 64 ||
        d > 64 * LT_KBMAX || b->N < 1)
        return D2_OK;
    const int nkb = (d + 63) / 64;
    const int ntile = (int)d2_ceil_div((int64_t)K * m, LT_M);
    const size_t xp_bytes = (size_t)ntile * nkb * 2 * LT_ABLK;
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_LBTC, xp_bytes + (size_t)K * 4 + 256, &base);
    if (rc) return rc;
    uint8_t* xp = static_cast<uint8_t*>(base);
    float* xmax = reinterpret_cast<float*>(static_cast<char*>(base) + xp_bytes);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    d2_time_begin(ctx, D2_KT_BOUND, st);
    const int64_t chunks = (int64_t)ntile * nkb * LT_M * 8;
    k_lt_xprep<<<(unsigned)std::min<int64_t>(d2_ceil_div(chunks, 256), (int64_t)sms * 8), 256, 0, st>>>(
        x, K, m, d, nkb, ntile, xp);
    D2_LAUNCH_CK(ctx, "k_lt_xprep");
    k_lt_xmax<<<(unsigned)d2_ceil_div(K, 128), 128, 0, st>>>(K, m, xn, xmax);
    D2_LAUNCH_CK(ctx, "k_lt_xmax");
    LtArgs a;
    a.offsets = b->offsets;
    a.supp = b->supp;
    a.vidx = b->vocab_idx;
    a.vocab = b->vocab;
    a.wt = b->wt;
    a.d = d;
    a.m = m;
    a.K = K;
    a.nkb = nkb;
    a.ntile = ntile;
    a.xp = xp;
    a.w = w;
    a.xn = xn;
    a.xmax = xmax;
    a.mq = mq;
    a.lb = lb;
    a.N = b->N;
    a.err = ctx->dev_flags + D2_DEV_ERR_WORD;
    const size_t smem = 1024 + (size_t)nkb * 2 * LT_BBLK + (size_t)LT_S * 2 * LT_ABLK + (size_t)LT_M * LT_CS * 4 +
                        (size_t)d * 4;
    D2_CK(ctx, cudaFuncSetAttribute(k_lb_pairs_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)std::min<int64_t>(b->N, (int64_t)sms);  // one CTA per SM (shared memory)
    k_lb_pairs_tc<<<grid, LT_M, smem, st>>>(a);
    D2_LAUNCH_CK(ctx, "k_lb_pairs_tc");
    d2_time_end(ctx, st);
    *used = true;
    return D2_OK;
}
