// Learned candidate pruning for the assignment step (the paper has no
// learned part; its own accelerator is triangle-inequality skipping).
//
// Embedding of a distribution P = {(w_j, y_j)}: centred points u_j = y_j - mu_P,
//   h1_j = relu(W1 u_j + b1), h2_j = relu(W2 h1_j + b2), g = sum_j w_j h2_j, f = W3 g,
// and the predictor What^2(P, Q) = ||mu_P - mu_Q||^2 + ||f(P) - f(Q)||^2.
// The mean term is exact (translation identity of squared-Euclidean OT) and a
// certified lower bound of W^2.
//
// Forward: persistent CTAs of H threads, one distribution at a time; thread h
// owns hidden unit h; weights staged once per CTA in shared memory as FP16
// (transposed so that thread h reads consecutive addresses); points and
// hidden activations are FP16-rounded, every dot product accumulates in FP32.
// Backward: per-point gradients by the same layout, weight gradients as
// chunked sums of outer products over all points (fixed chunk order, so
// deterministic), Adam on the FP32 masters.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "d2_internal.cuh"
#include "tc_util.cuh"

struct AssignArgs;
size_t d2_assign_warp_bytes(int m, int nmax);

struct d2_prune {
    int d = 0, H = 0, E = 0;
    int r = 8;
    float delta = 0.f;
    float fb_frac = -1.f;      // fall-back fraction estimated by the last d2_prune_calibrate
    int64_t nparam = 0;
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0;
    float* params = nullptr;   // FP32 masters
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int64_t step = 0;
    int device = 0;
};

#define PT 32        // points per tile in the forward / backward kernels

// Slot: a distribution to embed.  kind 0 = bag `id` of the bag set,
// kind 1 = centroid `id` of (x, w) with m points.
struct MlpArgs {
    const int64_t* offsets;
    const float* supp;
    const int32_t* vidx;
    const float* vocab;
    const float* wt;
    const float* cx;   // centroids K x m x d
    const float* cw;   // K x m
    int m;
    int max_mk;        // largest bag (bounds the point count)
    int d, H, E;
    const float* params;
    int64_t oW1, ob1, oW2, ob2, oW3;
    // slots
    int64_t nslots;
    const int64_t* slot_id;   // nslots (bag id or centroid id), or null: slot s = id s
    int64_t nbag_slots;       // slots [0, nbag_slots) are bags, the rest centroids
    // outputs
    float* f;       // nslots x E
    float* mu;      // nslots x d
    float* g;       // nslots x H (optional)
    // per-point saves (training)
    const int64_t* pt_off;    // nslots + 1 (optional)
    float* pu;      // points x d
    float* ph1;     // points x H
    float* ph2;     // points x H
    float* pw;      // points
    // backward
    const float* df;   // nslots x E
    float* da1;     // points x H
    float* da2;     // points x H
};

__device__ __forceinline__ float hround(float v) { return __half2float(__float2half_rn(v)); }

__device__ __forceinline__ void slot_source(const MlpArgs& a, int64_t s, const float*& rows, const int32_t*& vrows,
                                            const float*& wts, int& cnt, bool& is_bag) {
    const int64_t id = a.slot_id ? a.slot_id[s] : (s < a.nbag_slots ? s : s - a.nbag_slots);
    is_bag = s < a.nbag_slots;
    if (is_bag) {
        const int64_t r0 = a.offsets[id];
        cnt = (int)(a.offsets[id + 1] - r0);
        rows = a.supp ? a.supp + r0 * a.d : nullptr;
        vrows = a.vidx ? a.vidx + r0 : nullptr;
        wts = a.wt + r0;
    } else {
        cnt = a.m;
        rows = a.cx + id * (int64_t)a.m * a.d;
        vrows = nullptr;
        wts = a.cw + id * (int64_t)a.m;
    }
}

__device__ __forceinline__ float point_coord(const MlpArgs& a, const float* rows, const int32_t* vrows, int j, int t) {
    return rows ? rows[(int64_t)j * a.d + t] : a.vocab[(int64_t)vrows[j] * a.d + t];
}

// shared layout: W1T (d x H) half, W2T (H x H) half, W3 (E x H) half,
// U (PT x d) half, H1 (PT x H) half, mu (d) float, g (H) float, w (PT) float
__global__ void k_mlp_fwd(MlpArgs a) {
    extern __shared__ float4 dyn4[];
    const int d = a.d, H = a.H, E = a.E;
    __half* W1T = reinterpret_cast<__half*>(dyn4);
    __half* W2T = W1T + (size_t)d * H;
    __half* W3h = W2T + (size_t)H * H;
    __half* U = W3h + (size_t)E * H;
    __half* H1 = U + (size_t)PT * d;
    float* smu = reinterpret_cast<float*>(H1 + (size_t)PT * H);
    float* sg = smu + d;
    float* sw = sg + H;
    const int h = threadIdx.x;
    const float* W1 = a.params + a.oW1;
    const float* W2 = a.params + a.oW2;
    const float* W3 = a.params + a.oW3;
    for (int e = threadIdx.x; e < d * H; e += blockDim.x) {
        int t = e / H, hh = e - t * H;
        W1T[e] = __float2half_rn(W1[(int64_t)hh * d + t]);
    }
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
        int t = e / H, hh = e - t * H;
        W2T[e] = __float2half_rn(W2[(int64_t)hh * H + t]);
    }
    for (int e = threadIdx.x; e < E * H; e += blockDim.x) W3h[e] = __float2half_rn(W3[e]);
    const float b1 = hround(a.params[a.ob1 + h]);
    const float b2 = hround(a.params[a.ob2 + h]);
    __syncthreads();

    for (int64_t s = blockIdx.x; s < a.nslots; s += gridDim.x) {
        const float* rows;
        const int32_t* vrows;
        const float* wts;
        int cnt;
        bool is_bag;
        slot_source(a, s, rows, vrows, wts, cnt, is_bag);
        // weighted mean (FP32)
        for (int t = h; t < d; t += blockDim.x) {
            float acc = 0.f;
            for (int j = 0; j < cnt; ++j) acc = fmaf(wts[j], point_coord(a, rows, vrows, j, t), acc);
            smu[t] = acc;
            a.mu[s * d + t] = acc;
        }
        __syncthreads();
        const int64_t pbase = a.pt_off ? a.pt_off[s] : 0;
        float gacc = 0.f;
        for (int j0 = 0; j0 < cnt; j0 += PT) {
            const int np = min(PT, cnt - j0);
            for (int e = threadIdx.x; e < np * d; e += blockDim.x) {
                int j = e / d, t = e - j * d;
                float u = hround(point_coord(a, rows, vrows, j0 + j, t) - smu[t]);
                U[j * d + t] = __float2half_rn(u);
                if (a.pu) a.pu[(pbase + j0 + j) * d + t] = u;
            }
            if (threadIdx.x < np) sw[threadIdx.x] = wts[j0 + threadIdx.x];
            __syncthreads();
            // layer 1: thread h, all points of the tile
            for (int j = 0; j < np; j += 4) {
                float acc[4] = {b1, b1, b1, b1};
                for (int t = 0; t < d; ++t) {
                    const float wv = __half2float(W1T[t * H + h]);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j + q < np) acc[q] = fmaf(wv, __half2float(U[(j + q) * d + t]), acc[q]);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (j + q < np) {
                        const float v = hround(fmaxf(acc[q], 0.f));
                        H1[(j + q) * H + h] = __float2half_rn(v);
                        if (a.ph1) a.ph1[(pbase + j0 + j + q) * H + h] = v;
                    }
            }
            __syncthreads();
            // layer 2 and pooling
            for (int j = 0; j < np; j += 4) {
                float acc[4] = {b2, b2, b2, b2};
                for (int t = 0; t < H; ++t) {
                    const float wv = __half2float(W2T[t * H + h]);
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (j + q < np) acc[q] = fmaf(wv, __half2float(H1[(j + q) * H + t]), acc[q]);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (j + q < np) {
                        const float v = fmaxf(acc[q], 0.f);
                        gacc = fmaf(sw[j + q], v, gacc);
                        if (a.ph2) a.ph2[(pbase + j0 + j + q) * H + h] = v;
                    }
            }
            if (a.pw && threadIdx.x < np) a.pw[pbase + j0 + threadIdx.x] = sw[threadIdx.x];
            __syncthreads();
        }
        sg[h] = hround(gacc);
        if (a.g) a.g[s * H + h] = gacc;
        __syncthreads();
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            float acc = 0.f;
            for (int t = 0; t < H; ++t) acc = fmaf(__half2float(W3h[e * H + t]), sg[t], acc);
            a.f[s * E + e] = acc;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Forward on the tensor cores (tcgen05 / TMEM) for d <= 128 and H <= 128.
// The points of all slots, numbered by the slots' point offsets, are cut into
// tiles of 128 (one per TMEM lane); a CTA (4 warps, thread = row) takes a tile
// at a time:
//   * the rows' centred, FP16-rounded points u_j form the A operand of layer 1
//     (K-major, 128-byte swizzle, K = d padded to 64);
//   * one thread issues kind::f16 MMAs (FP16 A and B, FP32 accumulator in
//     TMEM) against W1 (H x d, K-major as stored), waits on an mbarrier;
//   * each thread reads its row of the accumulator, adds b1, applies ReLU and
//     the FP16 rounding and writes the A operand of layer 2, which multiplies
//     W2 into the same TMEM columns;
//   * the layer-2 rows (b2 added, ReLU) go through shared memory to one
//     thread per column, which adds w_j h2_j row by row per slot: a partial sum
//     per (slot, tile), stored at index slot + tile (a slot that continues
//     into the next tile ends this one, so no two pairs share an index).
// k_mlp_pool then adds each slot's partials in tile order (a fixed order) and
// applies W3.  The products are those of the CUDA-core kernel (FP16 operands
// are exact in FP32); only the order of the FP32 additions differs.  Every
// mbarrier wait is bounded (about 2 s); on expiry the CTA records
// D2F_DEV_TIMEOUT, stops, frees its tensor memory and returns.
// ---------------------------------------------------------------------------
#define MT_ROWS 128
#define MT_HMAX 128

struct MlpTc {
    int nkb1, nkb2;     // K blocks of 64 halves for layer 1 (d) and layer 2 (H)
    int pc;             // columns per pooling pass (shared stage of 128 x (pc + 1) floats)
    uint32_t tcols;     // TMEM columns (power of 2 >= H)
    float* part;        // (nslots + tiles) x H pooled partials
    int* err;           // sticky device error word
};

// weighted mean of every slot, the centring of its points (FP32, point order)
__global__ void k_mlp_mu(MlpArgs a) {
    for (int64_t s = blockIdx.x; s < a.nslots; s += gridDim.x) {
        const float* rows;
        const int32_t* vrows;
        const float* wts;
        int cnt;
        bool is_bag;
        slot_source(a, s, rows, vrows, wts, cnt, is_bag);
        for (int t = threadIdx.x; t < a.d; t += blockDim.x) {
            float acc = 0.f;
            for (int j = 0; j < cnt; ++j) acc = fmaf(wts[j], point_coord(a, rows, vrows, j, t), acc);
            a.mu[s * a.d + t] = acc;
        }
    }
}

// exclusive prefix of the slots' point counts into pt_off (one block)
__global__ void k_mlp_pt_scan(MlpArgs a, int64_t* pt_off) {
    __shared__ int64_t sh[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < a.nslots; b0 += 1024) {
        const int64_t s = b0 + threadIdx.x;
        int64_t v = 0;
        if (s < a.nslots) {
            const float* rows;
            const int32_t* vrows;
            const float* wts;
            int cnt;
            bool is_bag;
            slot_source(a, s, rows, vrows, wts, cnt, is_bag);
            v = cnt;
        }
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t u = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += u;
            __syncthreads();
        }
        if (s < a.nslots) pt_off[s] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) pt_off[a.nslots] = carry;
}

__device__ __forceinline__ uint4 pack_half8(const float* v) {
    uint4 u;
    uint32_t* w = reinterpret_cast<uint32_t*>(&u);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __half2 h = __floats2half2_rn(v[2 * q], v[2 * q + 1]);
        w[q] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return u;
}

__global__ void __launch_bounds__(MT_ROWS) k_mlp_fwd_tc(MlpArgs a, MlpTc t) {
    extern __shared__ uint8_t mt_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int64_t s_slot[MT_ROWS];
    __shared__ float s_w[MT_ROWS];
    __shared__ float s_b1[MT_HMAX], s_b2[MT_HMAX];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int d = a.d, H = a.H;
    // shared layout (1024-byte aligned for the swizzle): W1, W2, A1, A2 (the
    // pooling stage reuses A2 once layer 2's MMAs have read it)
    const uint32_t raw = smem_u32(mt_raw);
    uint8_t* base = mt_raw + (((raw + 1023u) & ~1023u) - raw);
    uint8_t* W1s = base;                                   // nkb1 blocks of H rows x 128 B
    uint8_t* W2s = W1s + (size_t)t.nkb1 * H * 128;         // nkb2 blocks of H rows x 128 B
    uint8_t* A1 = W2s + (size_t)t.nkb2 * H * 128;          // nkb1 blocks of 128 rows x 128 B
    uint8_t* A2 = A1 + (size_t)t.nkb1 * MT_ROWS * 128;     // nkb2 blocks of 128 rows x 128 B
    float* P = reinterpret_cast<float*>(A2);
    const int PS = t.pc + 1;                               // odd row stride: conflict-free columns

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(t.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&s_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B operands: W1 (H x d) and W2 (H x H) as FP16, K padded with zeros
    const float* W1 = a.params + a.oW1;
    const float* W2 = a.params + a.oW2;
    for (int e = tid; e < H * t.nkb1 * 8; e += MT_ROWS) {
        const int h = e / (t.nkb1 * 8), rem = e - h * (t.nkb1 * 8), kb = rem >> 3, k0 = kb * 64 + (rem & 7) * 8;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = k0 + q < d ? W1[(int64_t)h * d + k0 + q] : 0.f;
        *reinterpret_cast<uint4*>(W1s + (size_t)kb * H * 128 + sw128_off(h, (rem & 7) * 8)) = pack_half8(v);
    }
    for (int e = tid; e < H * t.nkb2 * 8; e += MT_ROWS) {
        const int h = e / (t.nkb2 * 8), rem = e - h * (t.nkb2 * 8), kb = rem >> 3, k0 = kb * 64 + (rem & 7) * 8;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = k0 + q < H ? W2[(int64_t)h * H + k0 + q] : 0.f;
        *reinterpret_cast<uint4*>(W2s + (size_t)kb * H * 128 + sw128_off(h, (rem & 7) * 8)) = pack_half8(v);
    }
    for (int h = tid; h < H; h += MT_ROWS) {
        s_b1[h] = hround(a.params[a.ob1 + h]);
        s_b2[h] = hround(a.params[a.ob2 + h]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t bar = smem_u32(&s_bar);
    const uint32_t idesc = idesc_f16_f32(MT_ROWS, H);
    const int64_t npts = a.pt_off[a.nslots];
    const int64_t ntiles = (npts + MT_ROWS - 1) / MT_ROWS;
    uint32_t ph = 0;
    bool dead = false;

    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // this thread's row: point p of slot s (largest s with pt_off[s] <= p)
        const int64_t p = tile * MT_ROWS + tid;
        const bool valid = p < npts;
        int64_t s = -1;
        const float* rows = nullptr;
        const int32_t* vrows = nullptr;
        const float* wts = nullptr;
        int j = 0;
        if (valid) {
            int64_t lo = 0, hi = a.nslots - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (a.pt_off[mid] <= p) lo = mid; else hi = mid - 1;
            }
            s = lo;
            int cnt;
            bool is_bag;
            slot_source(a, s, rows, vrows, wts, cnt, is_bag);
            j = (int)(p - a.pt_off[s]);
        }
        s_slot[tid] = s;
        s_w[tid] = valid ? wts[j] : 0.f;
        // layer 1 operand: u = half(y - mu), zero past d and for rows past the points
        for (int kb = 0; kb < t.nkb1; ++kb)
            for (int c8 = 0; c8 < 8; ++c8) {
                float v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = kb * 64 + c8 * 8 + q;
                    v[q] = 0.f;
                    if (valid && k < d) {
                        v[q] = hround(point_coord(a, rows, vrows, j, k) - a.mu[s * d + k]);
                        if (a.pu) a.pu[p * d + k] = v[q];
                    }
                }
                *reinterpret_cast<uint4*>(A1 + (size_t)kb * MT_ROWS * 128 + sw128_off(tid, c8 * 8)) = pack_half8(v);
            }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            for (int kb = 0; kb < t.nkb1; ++kb)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    umma_bf16(tmem, sdesc_sw128(smem_u32(A1 + (size_t)kb * MT_ROWS * 128) + ks * 32),
                              sdesc_sw128(smem_u32(W1s + (size_t)kb * H * 128) + ks * 32), idesc,
                              (kb | ks) ? 1u : 0u);
            umma_commit(bar);
        }
        if (!mbar_wait_bounded(bar, ph)) dead = true;
        ph ^= 1u;
        if (__syncthreads_or(dead)) break;
        tc_fence_after();
        // layer 1 epilogue: h1 = half(relu(acc + b1)) into the layer 2 operand
        for (int cb = 0; cb < t.nkb2 * 64; cb += 16) {
            float acc[16];
            if (cb < H) tmem_ld16(trow + (uint32_t)cb, acc);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int col = cb + q;
                acc[q] = col < H ? hround(fmaxf(acc[q] + s_b1[col], 0.f)) : 0.f;
                if (valid && col < H && a.ph1) a.ph1[p * H + col] = acc[q];
            }
            uint8_t* blk = A2 + (size_t)(cb >> 6) * MT_ROWS * 128;
            *reinterpret_cast<uint4*>(blk + sw128_off(tid, cb & 63)) = pack_half8(acc);
            *reinterpret_cast<uint4*>(blk + sw128_off(tid, (cb & 63) + 8)) = pack_half8(acc + 8);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            for (int kb = 0; kb < t.nkb2; ++kb)
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    umma_bf16(tmem, sdesc_sw128(smem_u32(A2 + (size_t)kb * MT_ROWS * 128) + ks * 32),
                              sdesc_sw128(smem_u32(W2s + (size_t)kb * H * 128) + ks * 32), idesc,
                              (kb | ks) ? 1u : 0u);
            umma_commit(bar);
        }
        if (!mbar_wait_bounded(bar, ph)) dead = true;
        ph ^= 1u;
        if (__syncthreads_or(dead)) break;
        tc_fence_after();
        // layer 2 epilogue and pooling, pc columns at a time through shared memory
        for (int c0 = 0; c0 < H; c0 += t.pc) {
            const int nc = min(t.pc, H - c0);
            for (int cb = 0; cb < nc; cb += 16) {
                float acc[16];
                tmem_ld16(trow + (uint32_t)(c0 + cb), acc);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = c0 + cb + q;
                    if (cb + q < nc) {
                        const float v = fmaxf(acc[q] + s_b2[col], 0.f);
                        P[tid * PS + cb + q] = v;
                        if (valid && a.ph2) a.ph2[p * H + col] = v;
                    }
                }
            }
            __syncthreads();
            if (tid < nc) {
                float acc = 0.f;
                int64_t cur = -1;
                for (int r = 0; r < MT_ROWS; ++r) {
                    const int64_t sr = s_slot[r];
                    if (sr != cur) {
                        if (cur >= 0) t.part[(cur + tile) * H + c0 + tid] = acc;
                        acc = 0.f;
                        cur = sr;
                    }
                    if (sr >= 0) acc = fmaf(s_w[r], P[r * PS + tid], acc);
                }
                if (cur >= 0) t.part[(cur + tile) * H + c0 + tid] = acc;
            }
            __syncthreads();
        }
        if (valid && a.pw) a.pw[p] = s_w[tid];
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (dead && tid == 0) atomicOr(t.err, D2F_DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(t.tcols) : "memory");
}

// per slot: g = its partials added in tile order; f = W3 half(g)
__global__ void k_mlp_pool(MlpArgs a, const float* part) {
    __shared__ float sg[MT_HMAX];
    const int H = a.H, E = a.E;
    const float* W3 = a.params + a.oW3;
    for (int64_t s = blockIdx.x; s < a.nslots; s += gridDim.x) {
        const int64_t p0 = a.pt_off[s], p1 = a.pt_off[s + 1];
        for (int h = threadIdx.x; h < H; h += blockDim.x) {
            float g = 0.f;
            if (p1 > p0)
                for (int64_t tile = p0 / MT_ROWS; tile <= (p1 - 1) / MT_ROWS; ++tile) g += part[(s + tile) * H + h];
            if (a.g) a.g[s * H + h] = g;
            sg[h] = hround(g);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            float acc = 0.f;
            for (int q = 0; q < H; ++q) acc = fmaf(hround(W3[(int64_t)e * H + q]), sg[q], acc);
            a.f[s * E + e] = acc;
        }
        __syncthreads();
    }
}

// backward to per-point gradients da2 (of a2) and da1 (of a1):
//   dg = W3^T df; da2_j = w_j dg * [h2_j > 0]; da1_j = (W2^T da2_j) * [h1_j > 0]
__global__ void k_mlp_bwd(MlpArgs a) {
    extern __shared__ float4 dyn4[];
    const int H = a.H, E = a.E;
    __half* W2h = reinterpret_cast<__half*>(dyn4);      // H x H, row-major (W2[h][t])
    float* sdg = reinterpret_cast<float*>(W2h + (size_t)H * H);
    float* sda = sdg + H;                               // PT x H
    const int t = threadIdx.x;
    const float* W2 = a.params + a.oW2;
    const float* W3 = a.params + a.oW3;
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) W2h[e] = __float2half_rn(W2[e]);
    __syncthreads();
    for (int64_t s = blockIdx.x; s < a.nslots; s += gridDim.x) {
        const int64_t p0 = a.pt_off[s], p1 = a.pt_off[s + 1];
        const int cnt = (int)(p1 - p0);
        {
            float acc = 0.f;
            for (int e = 0; e < E; ++e) acc = fmaf(hround(W3[(int64_t)e * H + t]), a.df[s * E + e], acc);
            sdg[t] = acc;
        }
        __syncthreads();
        for (int j0 = 0; j0 < cnt; j0 += PT) {
            const int np = min(PT, cnt - j0);
            for (int j = 0; j < np; ++j) {
                const int64_t pj = p0 + j0 + j;
                const float v = a.ph2[pj * H + t] > 0.f ? a.pw[pj] * sdg[t] : 0.f;
                sda[j * H + t] = v;
                a.da2[pj * H + t] = v;
            }
            __syncthreads();
            for (int j = 0; j < np; ++j) {
                const int64_t pj = p0 + j0 + j;
                float acc = 0.f;
                for (int hh = 0; hh < H; ++hh) acc = fmaf(sda[j * H + hh], __half2float(W2h[hh * H + t]), acc);
                a.da1[pj * H + t] = a.ph1[pj * H + t] > 0.f ? acc : 0.f;
            }
            __syncthreads();
        }
    }
}

// partial[c][i][k] = sum_{r in chunk c} A[r][i] * B[r][k]  (A: R x NA, B: R x NB),
// and colsum partial[c][i] of A when want_sum.  Tiles of 32 x 32 outputs.
#define OS_ROWS 256
__global__ void k_outer_partial(const float* A, int NA, const float* B, int NB, int64_t R, float* part,
                                float* sum_part) {
    __shared__ float sa[32][33];
    __shared__ float sb[32][33];
    const int c = blockIdx.x;
    const int i0 = blockIdx.y * 32, k0 = blockIdx.z * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 warps
    const int64_t r0 = (int64_t)c * OS_ROWS, r1 = min(R, r0 + OS_ROWS);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float cs = 0.f;
    for (int64_t rb = r0; rb < r1; rb += 32) {
        for (int q = ty; q < 32; q += 8) {
            const int64_t r = rb + q;
            sa[q][tx] = (r < r1 && i0 + tx < NA) ? A[r * NA + i0 + tx] : 0.f;
            sb[q][tx] = (r < r1 && k0 + tx < NB) ? B[r * NB + k0 + tx] : 0.f;
        }
        __syncthreads();
        for (int q = 0; q < 32; ++q) {
            const float bv = sb[q][tx];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(sa[q][ty + 8 * u], bv, acc[u]);
            if (blockIdx.z == 0 && ty == 0) cs += sa[q][tx];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty + 8 * u, k = k0 + tx;
        if (i < NA && k < NB) part[((int64_t)c * NA + i) * NB + k] = acc[u];
    }
    if (sum_part && blockIdx.z == 0 && ty == 0 && i0 + tx < NA) sum_part[(int64_t)c * NA + i0 + tx] = cs;
}

__global__ void k_chunk_reduce(const float* part, int64_t nchunk, int64_t n, float* out) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    float s = 0.f;
    for (int64_t c = 0; c < nchunk; ++c) s += part[c * n + e];
    out[e] = s;
}

// Weight-gradient contractions on the tensor cores: part[c] = A_c^T B_c and
// sum_part[c] = the column sums of A_c over the OT_ROWS rows of chunk c
// (A: R x NA, B: R x NB, row-major; NA, NB <= 128).  In both operands the
// rows are the contraction index, so the row-major arrays are MN-major
// operands as they stand: each 64-row K chunk is split into BF16 pieces
// (hi + lo) element by element into the 128-byte-swizzled MN-major layout,
// and one thread issues kind::f16 MMAs (M = 128 rows of D = columns of A,
// zero past NA; N = NB rounded up to 64; the products hi*hi + hi*lo + lo*hi)
// into an FP32 accumulator in tensor memory, two operand buffers alternating
// so that the conversion of chunk k + 1 overlaps the MMAs of chunk k.  Every
// mbarrier wait is bounded (about 2 s); on expiry the CTA records
// D2F_DEV_TIMEOUT, stops, frees its tensor memory and returns.
#define OT_ROWS 512
#define OT_KC 64

__device__ __forceinline__ void split_bf16x8(const float* v, uint4& hi, uint4& lo) {
    float r[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = v[q] - bf16_round(v[q]);
    const uint2 h0 = pack_bf16x4(v[0], v[1], v[2], v[3]), h1 = pack_bf16x4(v[4], v[5], v[6], v[7]);
    const uint2 l0 = pack_bf16x4(r[0], r[1], r[2], r[3]), l1 = pack_bf16x4(r[4], r[5], r[6], r[7]);
    hi = make_uint4(h0.x, h0.y, h1.x, h1.y);
    lo = make_uint4(l0.x, l0.y, l1.x, l1.y);
}

__global__ void __launch_bounds__(128) k_outer_tc(const float* A, int NA, const float* B, int NB, int NBp,
                                                  int64_t R, float* part, float* sum_part, uint32_t tcols,
                                                  int* err) {
    extern __shared__ uint8_t ot_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ float s_cs[128][9];
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t raw = smem_u32(ot_raw);
    uint8_t* base = ot_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t sboA = 2048u, sboB = (uint32_t)(NBp >> 6) * 1024u;
    const uint32_t abytes = 8u * sboA, bbytes = 8u * sboB;  // 64 K rows = 8 groups
    const uint32_t bufbytes = 2u * (abytes + bbytes);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&s_bar[0]), 1);
        mbar_init(smem_u32(&s_bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t bar0 = smem_u32(&s_bar[0]);
    const uint32_t idesc = idesc_bf16_f32_mn(128, NBp);
    const int64_t r0 = blockIdx.x * (int64_t)OT_ROWS, r1 = min(R, r0 + OT_ROWS);
    const int nkc = (int)((r1 - r0 + OT_KC - 1) / OT_KC);
    float csum[8];  // column sums of A for columns 8 (tid % 16) .. + 7 over this thread's rows
#pragma unroll
    for (int q = 0; q < 8; ++q) csum[q] = 0.f;
    uint32_t ph = 0u, pend = 0u;
    bool dead = false;
    for (int kc = 0; kc < nkc; ++kc) {
        const int b = kc & 1;
        if ((pend >> b) & 1u) {  // the MMAs that last read this buffer
            if (!mbar_wait_bounded(bar0 + 8 * b, (ph >> b) & 1u)) dead = true;
            ph ^= 1u << b;
            pend &= ~(1u << b);
            if (__syncthreads_or(dead)) break;
        }
        uint8_t* Ahi = base + (size_t)b * bufbytes;
        uint8_t* Alo = Ahi + abytes;
        uint8_t* Bhi = Alo + abytes;
        uint8_t* Blo = Bhi + bbytes;
        const int64_t rk = r0 + (int64_t)kc * OT_KC;
        // A: 64 rows x 16 chunks of 8 columns (columns past NA are zero)
#pragma unroll
        for (int s8 = 0; s8 < 8; ++s8) {
            const int e = tid + 128 * s8, kk = e >> 4, c8 = e & 15;
            const int64_t r = rk + kk;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int col = c8 * 8 + q;
                v[q] = (r < r1 && col < NA) ? A[r * NA + col] : 0.f;
                csum[q] += v[q];
            }
            uint4 hi, lo;
            split_bf16x8(v, hi, lo);
            const uint32_t off = sw128_mn_off(kk, c8 * 8, sboA);
            *reinterpret_cast<uint4*>(Ahi + off) = hi;
            *reinterpret_cast<uint4*>(Alo + off) = lo;
        }
        // B: 64 rows x NBp / 8 chunks
        const int nbc = NBp >> 3;
        for (int e = tid; e < OT_KC * nbc; e += 128) {
            const int kk = e / nbc, c8 = e - kk * nbc;
            const int64_t r = rk + kk;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int col = c8 * 8 + q;
                v[q] = (r < r1 && col < NB) ? B[r * NB + col] : 0.f;
            }
            uint4 hi, lo;
            split_bf16x8(v, hi, lo);
            const uint32_t off = sw128_mn_off(kk, c8 * 8, sboB);
            *reinterpret_cast<uint4*>(Bhi + off) = hi;
            *reinterpret_cast<uint4*>(Blo + off) = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < OT_KC / 16; ++ks) {  // 16 K rows = two 8-row groups
                const uint32_t ao = (uint32_t)ks * 2u * sboA, bo = (uint32_t)ks * 2u * sboB;
                const uint64_t ah = sdesc_sw128_mn(smem_u32(Ahi) + ao, 1024u, sboA);
                const uint64_t al = sdesc_sw128_mn(smem_u32(Alo) + ao, 1024u, sboA);
                const uint64_t bh = sdesc_sw128_mn(smem_u32(Bhi) + bo, 1024u, sboB);
                const uint64_t bl = sdesc_sw128_mn(smem_u32(Blo) + bo, 1024u, sboB);
                umma_bf16(tmem, ah, bh, idesc, (kc | ks) ? 1u : 0u);
                umma_bf16(tmem, ah, bl, idesc, 1u);
                umma_bf16(tmem, al, bh, idesc, 1u);
            }
            umma_commit(bar0 + 8 * b);
        }
        pend |= 1u << b;
    }
    // drain: no MMA may still be in flight when the accumulator is read or freed
    for (int b = 0; b < 2; ++b) {
        if (((pend >> b) & 1u) && !dead) {
            if (!mbar_wait_bounded(bar0 + 8 * b, (ph >> b) & 1u)) dead = true;
            pend &= ~(1u << b);
        }
    }
    dead = __syncthreads_or(dead);
    tc_fence_after();
    if (!dead && nkc > 0) {
        const int i = tid;  // row i of D = TMEM lane i = column i of A
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int cb = 0; cb < NBp; cb += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)cb, v);
            if (i < NA)
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (cb + q < NB) part[((int64_t)blockIdx.x * NA + i) * NB + cb + q] = v[q];
        }
    }
    if (dead && tid == 0) atomicOr(err, D2F_DEV_TIMEOUT);
    // column sums: the 8 threads that took column chunk c8 = tid % 16, in thread order
#pragma unroll
    for (int q = 0; q < 8; ++q) s_cs[tid][q] = csum[q];
    __syncthreads();
    if (sum_part && tid < NA) {
        const int c8 = tid >> 3, q = tid & 7;
        float sv = 0.f;
        for (int t = c8; t < 128; t += 16) sv += s_cs[t][q];
        sum_part[(int64_t)blockIdx.x * NA + tid] = sv;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

// per pair b: residual of ||f_a - f_q||^2 against t - ||mu_a - mu_q||^2
__global__ void k_pair_loss(int64_t B, int E, int d, const float* f, const float* mu, int64_t nbag_slots,
                            const int32_t* pair_cent, const float* target, float* gd, double* lossb) {
    const int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    const int64_t sa = b, sq = nbag_slots + pair_cent[b];
    float mt = 0.f, pr = 0.f;
    for (int t = lane; t < d; t += 32) {
        float v = mu[sa * d + t] - mu[sq * d + t];
        mt = fmaf(v, v, mt);
    }
    for (int e = lane; e < E; e += 32) {
        float v = f[sa * E + e] - f[sq * E + e];
        pr = fmaf(v, v, pr);
    }
    mt = group_sum<32>(mt);
    pr = group_sum<32>(pr);
    const float res = pr - (target[b] - mt);
    const float coef = 4.f * res / (float)B;
    for (int e = lane; e < E; e += 32) gd[b * E + e] = coef * (f[sa * E + e] - f[sq * E + e]);
    if (lane == 0) lossb[b] = (double)res * (double)res / (double)B;
}

// df of the bag slots = gd; of centroid q = -sum of gd over its pairs (fixed order)
__global__ void k_df_gather(int64_t B, int K, int E, const int32_t* pair_cent, const float* gd, float* df) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx < B * E) {
        df[idx] = gd[idx];
        return;
    }
    const int64_t c = idx - B * E;
    if (c >= (int64_t)K * E) return;
    const int q = (int)(c / E), e = (int)(c - (int64_t)q * E);
    float s = 0.f;
    for (int64_t b = 0; b < B; ++b)
        if (pair_cent[b] == q) s += gd[b * E + e];
    df[B * E + c] = -s;
}

__global__ void k_sum_loss(const double* lossb, int64_t B, double* out) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += blockDim.x) acc += lossb[b];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}

__global__ void k_adam(float* p, float* mom, float* vel, const float* g, int64_t n, float lr, float b1, float b2,
                       float c1, float c2) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gv = g[e];
    const float mv = b1 * mom[e] + (1.f - b1) * gv;
    const float vv = b2 * vel[e] + (1.f - b2) * gv * gv;
    mom[e] = mv;
    vel[e] = vv;
    p[e] -= lr * (mv / c1) / (sqrtf(vv / c2) + 1e-8f);
}

__global__ void k_slot_counts(const int64_t* offsets, const int64_t* bag_ids, int64_t nb, int64_t ns, int m,
                              int64_t* pt_off) {
    // exclusive prefix of point counts over slots, one block
    __shared__ int64_t s[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < ns; base += 1024) {
        const int64_t i = base + threadIdx.x;
        int64_t v = 0;
        if (i < ns) v = i < nb ? offsets[bag_ids[i] + 1] - offsets[bag_ids[i]] : m;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < ns) pt_off[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) pt_off[ns] = carry;
}

__global__ void k_gather_pairs(const int64_t* idx, int64_t B, const int64_t* pb, const int32_t* pc, const float* pt,
                               int64_t* ob, int32_t* oc, float* ot) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int64_t s = idx[b];
    ob[b] = pb[s];
    oc[b] = pc[s];
    ot[b] = pt[s];
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

static size_t fwd_smem(const d2_prune* p) {
    size_t halves = (size_t)p->d * p->H + (size_t)p->H * p->H + (size_t)p->E * p->H + (size_t)PT * p->d +
                    (size_t)PT * p->H;
    size_t b = halves * 2;
    b = (b + 15) & ~(size_t)15;
    return b + (size_t)(p->d + p->H + PT) * 4;
}

static size_t bwd_smem(const d2_prune* p) {
    return (((size_t)p->H * p->H * 2 + 15) & ~(size_t)15) + (size_t)(p->H + PT * p->H) * 4;
}

static MlpArgs mlp_args(const d2_prune* p, const d2_bags* b, const float* cx, const float* cw, int m) {
    MlpArgs a;
    memset(&a, 0, sizeof(a));
    if (b) {
        a.offsets = b->offsets;
        a.supp = b->supp;
        a.vidx = b->vocab_idx;
        a.vocab = b->vocab;
        a.wt = b->wt;
        a.max_mk = b->max_mk;
    }
    a.cx = cx;
    a.cw = cw;
    a.m = m;
    a.d = p->d;
    a.H = p->H;
    a.E = p->E;
    a.params = p->params;
    a.oW1 = p->oW1;
    a.ob1 = p->ob1;
    a.oW2 = p->oW2;
    a.ob2 = p->ob2;
    a.oW3 = p->oW3;
    return a;
}

// The tensor-core forward covers d <= 128 and H <= 128 (H % 32 == 0): its
// weights and two operand tiles then fit in shared memory with room for two
// CTAs per SM; other shapes use the CUDA-core kernel.
static bool mlp_tc_applies(const d2_prune* p) { return p->d <= 128 && p->H <= MT_HMAX && p->H % 32 == 0; }

static int launch_fwd_tc(d2_ctx* ctx, const d2_prune* p, const MlpArgs& a0, cudaStream_t st) {
    MlpArgs a = a0;
    const int H = p->H;
    const int64_t maxpts = a.nbag_slots * (int64_t)a.max_mk + (a.nslots - a.nbag_slots) * (int64_t)a.m;
    const int64_t tiles = d2_ceil_div(std::max<int64_t>(maxpts, 1), MT_ROWS);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_pt = take((size_t)(a.nslots + 1) * 8), o_part = take((size_t)(a.nslots + tiles) * H * 4);
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_MLP, off, &base);
    if (rc) return rc;
    int64_t* ptoff = reinterpret_cast<int64_t*>(static_cast<char*>(base) + o_pt);
    float* part = reinterpret_cast<float*>(static_cast<char*>(base) + o_part);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    d2_time_begin(ctx, D2_KT_PRUNE, st);
    if (!a.pt_off) {
        k_mlp_pt_scan<<<1, 1024, 0, st>>>(a, ptoff);
        D2_LAUNCH_CK(ctx, "k_mlp_pt_scan");
        a.pt_off = ptoff;
    }
    const unsigned sgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(a.nslots, (int64_t)sms * 8));
    k_mlp_mu<<<sgrid, 128, 0, st>>>(a);
    D2_LAUNCH_CK(ctx, "k_mlp_mu");
    MlpTc t;
    t.nkb1 = (p->d + 63) / 64;
    t.nkb2 = (H + 63) / 64;
    t.pc = (t.nkb2 * 32 - 1) / 16 * 16;  // 128 rows of pc + 1 floats within the layer-2 operand
    uint32_t cols = 32;
    while ((int)cols < H) cols <<= 1;
    t.tcols = cols;
    t.part = part;
    t.err = ctx->dev_flags + D2_DEV_ERR_WORD;
    size_t smem = 1024 + (size_t)(t.nkb1 + t.nkb2) * H * 128 + (size_t)(t.nkb1 + t.nkb2) * MT_ROWS * 128;
    // at most 512 / cols resident CTAs per SM (tensor memory): size the request
    const int max_ctas = 512 / (int)cols;
    const size_t cap_req = (size_t)228 * 1024 / (size_t)(max_ctas + 1) + 1;
    if (max_ctas < 16 && smem < cap_req) smem = cap_req;
    D2_CK(ctx, cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    D2_CK(ctx, cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int per = 1;
    D2_CK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mlp_fwd_tc, MT_ROWS, smem));
    per = std::max(1, std::min(per, max_ctas));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * per));
    k_mlp_fwd_tc<<<grid, MT_ROWS, smem, st>>>(a, t);
    D2_LAUNCH_CK(ctx, "k_mlp_fwd_tc");
    k_mlp_pool<<<sgrid, 128, 0, st>>>(a, part);
    D2_LAUNCH_CK(ctx, "k_mlp_pool");
    d2_time_end(ctx, st);
    return D2_OK;
}

static int launch_fwd(d2_ctx* ctx, const d2_prune* p, const MlpArgs& a, cudaStream_t st) {
    if (a.nslots <= 0) return D2_OK;
    if (mlp_tc_applies(p) && !ctx->mlp_cuda_cores) return launch_fwd_tc(ctx, p, a, st);
    size_t smem = fwd_smem(p);
    if (smem > 220 * 1024) return d2_fail(ctx, D2_ENOTSUP, "pruner: d x H too large for shared memory");
    D2_CK(ctx, cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sms = 152, per = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mlp_fwd, p->H, smem);
    per = std::max(per, 1);
    unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(a.nslots, (int64_t)sms * per));
    d2_time_begin(ctx, D2_KT_PRUNE, st);
    k_mlp_fwd<<<grid, p->H, smem, st>>>(a);
    d2_time_end(ctx, st);
    D2_LAUNCH_CK(ctx, "k_mlp_fwd");
    return D2_OK;
}

static int outer_sum(d2_ctx* ctx, const float* A, int NA, const float* B, int NB, int64_t R, float* out,
                     float* colsum, float* scratch, cudaStream_t st) {
    if (R > 0 && NA <= 128 && NB <= 128 && !ctx->mlp_cuda_cores) {
        // tensor cores (k_outer_tc); chunks of OT_ROWS rows, no more than the
        // scratch's OS_ROWS chunks
        const int64_t nch = d2_ceil_div(R, OT_ROWS);
        float* part = scratch;
        float* spart = scratch + nch * (int64_t)NA * NB;
        const int NBp = (NB + 63) / 64 * 64;
        const uint32_t tcols = (uint32_t)NBp;  // 64 or 128
        const size_t smem = 1024 + (size_t)2 * 2 * (8 * 2048 + 8 * (NBp / 64) * 1024);
        D2_CK(ctx, cudaFuncSetAttribute(k_outer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_outer_tc<<<(unsigned)nch, 128, smem, st>>>(A, NA, B, NB, NBp, R, part, colsum ? spart : nullptr, tcols,
                                                     ctx->dev_flags + D2_DEV_ERR_WORD);
        D2_LAUNCH_CK(ctx, "k_outer_tc");
        const int64_t n = (int64_t)NA * NB;
        k_chunk_reduce<<<(unsigned)d2_ceil_div(n, 256), 256, 0, st>>>(part, nch, n, out);
        D2_LAUNCH_CK(ctx, "k_chunk_reduce");
        if (colsum) {
            k_chunk_reduce<<<(unsigned)d2_ceil_div(NA, 256), 256, 0, st>>>(spart, nch, NA, colsum);
            D2_LAUNCH_CK(ctx, "k_chunk_reduce");
        }
        return D2_OK;
    }
    const int64_t nch = std::max<int64_t>(1, d2_ceil_div(R, OS_ROWS));
    float* part = scratch;
    float* spart = scratch + nch * (int64_t)NA * NB;
    dim3 g((unsigned)nch, (unsigned)d2_ceil_div(NA, 32), (unsigned)d2_ceil_div(NB, 32));
    if (R == 0) {
        D2_CK(ctx, cudaMemsetAsync(out, 0, (size_t)NA * NB * 4, st));
        if (colsum) D2_CK(ctx, cudaMemsetAsync(colsum, 0, (size_t)NA * 4, st));
        return D2_OK;
    }
    k_outer_partial<<<g, 256, 0, st>>>(A, NA, B, NB, R, part, colsum ? spart : nullptr);
    D2_LAUNCH_CK(ctx, "k_outer_partial");
    const int64_t n = (int64_t)NA * NB;
    k_chunk_reduce<<<(unsigned)d2_ceil_div(n, 256), 256, 0, st>>>(part, nch, n, out);
    D2_LAUNCH_CK(ctx, "k_chunk_reduce");
    if (colsum) {
        k_chunk_reduce<<<(unsigned)d2_ceil_div(NA, 256), 256, 0, st>>>(spart, nch, NA, colsum);
        D2_LAUNCH_CK(ctx, "k_chunk_reduce");
    }
    return D2_OK;
}

static size_t outer_scratch_floats(int NA, int NB, int64_t R) {
    const int64_t nch = std::max<int64_t>(1, d2_ceil_div(R, OS_ROWS));
    return (size_t)nch * NA * NB + (size_t)nch * NA;
}

// Forward + loss + backward for B pairs; grad (device, packed), loss (device double).
static int loss_grad_impl(d2_ctx* ctx, const d2_prune* p, const d2_bags* bags, int K, int m, const float* x,
                          const float* w, const int64_t* pair_bag, const int32_t* pair_cent, const float* target,
                          int64_t B, double* loss, float* grad, cudaStream_t st) {
    const int d = p->d, H = p->H, E = p->E;
    const int64_t ns = B + K;
    const int64_t maxpts = B * (int64_t)bags->max_mk + (int64_t)K * m;
    // workspace layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_ids = take(ns * 8), o_ptoff = take((ns + 1) * 8), o_f = take(ns * E * 4), o_mu = take(ns * d * 4),
                 o_g = take(ns * H * 4), o_pu = take(maxpts * d * 4), o_ph1 = take(maxpts * H * 4),
                 o_ph2 = take(maxpts * H * 4), o_pw = take(maxpts * 4), o_da1 = take(maxpts * H * 4),
                 o_da2 = take(maxpts * H * 4), o_gd = take(B * E * 4), o_df = take(ns * E * 4),
                 o_lb = take(B * 8);
    const size_t nsc = std::max(std::max(outer_scratch_floats(H, H, maxpts), outer_scratch_floats(H, d, maxpts)),
                                outer_scratch_floats(E, H, ns));
    const size_t o_sc = take(nsc * 4);
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_PRUNE, off, &base);
    if (rc) return rc;
    char* bb = static_cast<char*>(base);
    int64_t* ids = reinterpret_cast<int64_t*>(bb + o_ids);
    int64_t* ptoff = reinterpret_cast<int64_t*>(bb + o_ptoff);
    float* f = reinterpret_cast<float*>(bb + o_f);
    float* mu = reinterpret_cast<float*>(bb + o_mu);
    float* g = reinterpret_cast<float*>(bb + o_g);
    float* pu = reinterpret_cast<float*>(bb + o_pu);
    float* ph1 = reinterpret_cast<float*>(bb + o_ph1);
    float* ph2 = reinterpret_cast<float*>(bb + o_ph2);
    float* pw = reinterpret_cast<float*>(bb + o_pw);
    float* da1 = reinterpret_cast<float*>(bb + o_da1);
    float* da2 = reinterpret_cast<float*>(bb + o_da2);
    float* gd = reinterpret_cast<float*>(bb + o_gd);
    float* df = reinterpret_cast<float*>(bb + o_df);
    double* lb = reinterpret_cast<double*>(bb + o_lb);
    float* sc = reinterpret_cast<float*>(bb + o_sc);

    // slot ids: B bags then centroids 0..K-1
    D2_CK(ctx, cudaMemcpyAsync(ids, pair_bag, B * 8, cudaMemcpyDeviceToDevice, st));
    {
        std::vector<int64_t> cids(K);
        for (int q = 0; q < K; ++q) cids[q] = q;
        D2_CK(ctx, cudaMemcpyAsync(ids + B, cids.data(), K * 8, cudaMemcpyHostToDevice, st));
        D2_CK(ctx, cudaStreamSynchronize(st));  // cids is a host temporary
    }
    k_slot_counts<<<1, 1024, 0, st>>>(bags->offsets, ids, B, ns, m, ptoff);
    D2_LAUNCH_CK(ctx, "k_slot_counts");
    MlpArgs a = mlp_args(p, bags, x, w, m);
    a.nslots = ns;
    a.nbag_slots = B;
    a.slot_id = ids;
    a.f = f;
    a.mu = mu;
    a.g = g;
    a.pt_off = ptoff;
    a.pu = pu;
    a.ph1 = ph1;
    a.ph2 = ph2;
    a.pw = pw;
    if ((rc = launch_fwd(ctx, p, a, st))) return rc;
    k_pair_loss<<<(unsigned)d2_ceil_div(B, 8), 256, 0, st>>>(B, E, d, f, mu, B, pair_cent, target, gd, lb);
    D2_LAUNCH_CK(ctx, "k_pair_loss");
    k_sum_loss<<<1, 256, 0, st>>>(lb, B, loss);
    D2_LAUNCH_CK(ctx, "k_sum_loss");
    k_df_gather<<<(unsigned)d2_ceil_div(ns * E, 256), 256, 0, st>>>(B, K, E, pair_cent, gd, df);
    D2_LAUNCH_CK(ctx, "k_df_gather");
    a.df = df;
    a.da1 = da1;
    a.da2 = da2;
    {
        size_t smem = bwd_smem(p);
        D2_CK(ctx, cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ns, (int64_t)sms * 2));
        k_mlp_bwd<<<grid, H, smem, st>>>(a);
        D2_LAUNCH_CK(ctx, "k_mlp_bwd");
    }
    // total points (device) -> use the bound; rows past the total are zero
    // because the per-point arrays are only written for real points: clear
    // the tail by computing the exact count on the host
    int64_t npts = 0;
    D2_CK(ctx, cudaMemcpyAsync(&npts, ptoff + ns, 8, cudaMemcpyDeviceToHost, st));
    D2_CK(ctx, cudaStreamSynchronize(st));
    float* gW1 = grad + p->oW1;
    float* gb1 = grad + p->ob1;
    float* gW2 = grad + p->oW2;
    float* gb2 = grad + p->ob2;
    float* gW3 = grad + p->oW3;
    if ((rc = outer_sum(ctx, da1, H, pu, d, npts, gW1, gb1, sc, st))) return rc;
    if ((rc = outer_sum(ctx, da2, H, ph1, H, npts, gW2, gb2, sc, st))) return rc;
    if ((rc = outer_sum(ctx, df, E, g, H, ns, gW3, nullptr, sc, st))) return rc;
    return D2_OK;
}

// ---------------------------------------------------------------------------
// pruned assignment
// ---------------------------------------------------------------------------

// per bag: What^2 to every centroid, r smallest (ties: lower index)
__global__ void k_topr(int64_t N, int K, int E, int d, int r, const float* fb, const float* mub, const float* fc,
                       const float* muc, int32_t* cand) {
    const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    // each lane keeps its own sorted top-r list of the centroids it scores
    float bv[16];
    int bi[16];
    for (int t = 0; t < r; ++t) {
        bv[t] = 3.0e38f;
        bi[t] = 0x7fffffff;
    }
    for (int i = lane; i < K; i += 32) {
        float s = 0.f;
        for (int t = 0; t < d; ++t) {
            float v = mub[k * d + t] - muc[(int64_t)i * d + t];
            s = fmaf(v, v, s);
        }
        for (int e = 0; e < E; ++e) {
            float v = fb[k * E + e] - fc[(int64_t)i * E + e];
            s = fmaf(v, v, s);
        }
        if (s < bv[r - 1] || (s == bv[r - 1] && i < bi[r - 1])) {
            int pos = r - 1;
            while (pos > 0 && (s < bv[pos - 1] || (s == bv[pos - 1] && i < bi[pos - 1]))) {
                bv[pos] = bv[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bv[pos] = s;
            bi[pos] = i;
        }
    }
    // merge the 32 lists: r rounds of warp argmin over the list heads
    int head = 0;
    for (int t = 0; t < r; ++t) {
        float v = head < r ? bv[head] : 3.0e38f;
        int ix = head < r ? bi[head] : 0x7fffffff;
        float mv = v;
        int mi = ix;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, mv, o);
            int oi = __shfl_xor_sync(0xffffffffu, mi, o);
            if (ov < mv || (ov == mv && oi < mi)) {
                mv = ov;
                mi = oi;
            }
        }
        if (ix == mi && head < r) ++head;
        if (lane == 0) cand[k * r + t] = mi;
    }
}

// margin test; passing bags get their label, the others are queued for all K
__global__ void k_margin(int64_t N, int K, int E, int d, int r, float delta, const float* fb, const float* mub,
                         const float* fc, const float* muc, const int32_t* cand, const float* w2c, int32_t* labels,
                         float* dist, int64_t* fb_list, int64_t* fb_count) {
    const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    float b = 3.0e38f;
    int best = 0x7fffffff;
    for (int t = 0; t < r; ++t) {
        const float v = w2c[k * r + t];
        const int i = cand[k * r + t];
        if (v < b || (v == b && i < best)) {
            b = v;
            best = i;
        }
    }
    bool fail = false;
    for (int i = lane; i < K; i += 32) {
        bool is_c = false;
        for (int t = 0; t < r; ++t) is_c |= (cand[k * r + t] == i);
        if (is_c) continue;
        float mt = 0.f, pr = 0.f;
        for (int t = 0; t < d; ++t) {
            float v = mub[k * d + t] - muc[(int64_t)i * d + t];
            mt = fmaf(v, v, mt);
        }
        for (int e = 0; e < E; ++e) {
            float v = fb[k * E + e] - fc[(int64_t)i * E + e];
            pr = fmaf(v, v, pr);
        }
        const float lb = fmaxf(mt, mt + pr - delta);
        if (!(lb > b)) fail = true;
    }
    fail = __any_sync(0xffffffffu, fail);
    if (lane == 0) {
        if (fail) {
            unsigned long long pos = atomicAdd(reinterpret_cast<unsigned long long*>(fb_count), 1ull);
            fb_list[pos] = k;
        } else {
            labels[k] = best;
            dist[k] = b;
        }
    }
}

__global__ void k_argmin_list(const int64_t* list, const int64_t* cnt, int K, const float* D, int32_t* labels,
                              float* dist) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= *cnt) return;
    const int64_t k = list[t];
    const float* row = D + k * K;
    float b = row[0];
    int bi = 0;
    for (int i = 1; i < K; ++i)
        if (row[i] < b) {
            b = row[i];
            bi = i;
        }
    labels[k] = bi;
    dist[k] = b;
}

__global__ void k_prune_count(int64_t* counters, const int64_t* fb_count, int64_t base, int K) {
    counters[0] += base + (*fb_count) * K;
    counters[1] += *fb_count;
}

// from assign.cu
int d2_prune_solve_pairs(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w, int mode,
                         int64_t npairs, const int64_t* npairs_dev, const int32_t* cand, int r,
                         const int64_t* bag_list, float* out, int64_t* fail_count, cudaStream_t st);

// The pruner's r candidates per bag (smallest What^2) into cand (N x r).
int d2_prune_candidates(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                        const d2_prune* p, int r, int32_t* cand, cudaStream_t st) {
    if (p->d != b->d) return d2_fail(ctx, D2_EINVAL, "d2_assign: pruner dimension %d != bag dimension %d", p->d, b->d);
    if (r > 16) return d2_fail(ctx, D2_ENOTSUP, "d2_assign: r > 16");
    const int64_t N = b->N;
    const int d = p->d, E = p->E;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_fb = take(N * E * 4), o_mub = take(N * d * 4), o_fc = take((size_t)K * E * 4),
                 o_muc = take((size_t)K * d * 4);
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_PRUNE, off, &base);
    if (rc) return rc;
    char* bb = static_cast<char*>(base);
    float* fb = reinterpret_cast<float*>(bb + o_fb);
    float* mub = reinterpret_cast<float*>(bb + o_mub);
    float* fc = reinterpret_cast<float*>(bb + o_fc);
    float* muc = reinterpret_cast<float*>(bb + o_muc);
    MlpArgs a = mlp_args(p, b, x, w, m);
    a.nslots = N;
    a.nbag_slots = N;
    a.f = fb;
    a.mu = mub;
    if ((rc = launch_fwd(ctx, p, a, st))) return rc;
    MlpArgs ac = mlp_args(p, b, x, w, m);
    ac.nslots = K;
    ac.nbag_slots = 0;
    ac.f = fc;
    ac.mu = muc;
    if ((rc = launch_fwd(ctx, p, ac, st))) return rc;
    k_topr<<<(unsigned)d2_ceil_div(N, 8), 256, 0, st>>>(N, K, E, d, r, fb, mub, fc, muc, cand);
    D2_LAUNCH_CK(ctx, "k_topr");
    return D2_OK;
}

int d2_assign_pruned(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                     const d2_prune* p, int32_t* labels, float* dist, int64_t* counters, cudaStream_t st) {
    if (p->d != b->d) return d2_fail(ctx, D2_EINVAL, "d2_assign: pruner dimension %d != bag dimension %d", p->d, b->d);
    const int64_t N = b->N;
    const int r = std::min(p->r, K);
    const int d = p->d, E = p->E;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_fb = take(N * E * 4), o_mub = take(N * d * 4), o_fc = take((size_t)K * E * 4),
                 o_muc = take((size_t)K * d * 4), o_cand = take(N * r * 4), o_w2c = take(N * r * 4),
                 o_list = take(N * 8), o_cnt = take(64), o_D = take(N * (size_t)K * 4);
    void* base = nullptr;
    int rc = d2_ws(ctx, WS_PRUNE, off, &base);
    if (rc) return rc;
    char* bb = static_cast<char*>(base);
    float* fb = reinterpret_cast<float*>(bb + o_fb);
    float* mub = reinterpret_cast<float*>(bb + o_mub);
    float* fc = reinterpret_cast<float*>(bb + o_fc);
    float* muc = reinterpret_cast<float*>(bb + o_muc);
    int32_t* cand = reinterpret_cast<int32_t*>(bb + o_cand);
    float* w2c = reinterpret_cast<float*>(bb + o_w2c);
    int64_t* list = reinterpret_cast<int64_t*>(bb + o_list);
    int64_t* cnt = reinterpret_cast<int64_t*>(bb + o_cnt);
    float* D = reinterpret_cast<float*>(bb + o_D);

    MlpArgs a = mlp_args(p, b, x, w, m);
    a.nslots = N;
    a.nbag_slots = N;
    a.f = fb;
    a.mu = mub;
    if ((rc = launch_fwd(ctx, p, a, st))) return rc;
    MlpArgs ac = mlp_args(p, b, x, w, m);
    ac.nslots = K;
    ac.nbag_slots = 0;
    ac.f = fc;
    ac.mu = muc;
    if ((rc = launch_fwd(ctx, p, ac, st))) return rc;
    if (r > 16) return d2_fail(ctx, D2_ENOTSUP, "d2_assign: r > 16");
    k_topr<<<(unsigned)d2_ceil_div(N, 8), 256, 0, st>>>(N, K, E, d, r, fb, mub, fc, muc, cand);
    D2_LAUNCH_CK(ctx, "k_topr");
    if ((rc = d2_prune_solve_pairs(ctx, b, K, m, x, w, 3, N * r, nullptr, cand, r, nullptr, w2c, counters + 2, st)))
        return rc;
    D2_CK(ctx, cudaMemsetAsync(cnt, 0, 8, st));
    k_margin<<<(unsigned)d2_ceil_div(N, 8), 256, 0, st>>>(N, K, E, d, r, p->delta, fb, mub, fc, muc, cand, w2c,
                                                          labels, dist, list, cnt);
    D2_LAUNCH_CK(ctx, "k_margin");
    if ((rc = d2_prune_solve_pairs(ctx, b, K, m, x, w, 2, N * (int64_t)K, cnt, nullptr, r, list, D, counters + 2, st)))
        return rc;
    k_argmin_list<<<(unsigned)d2_ceil_div(N, 256), 256, 0, st>>>(list, cnt, K, D, labels, dist);
    D2_LAUNCH_CK(ctx, "k_argmin_list");
    k_prune_count<<<1, 1, 0, st>>>(counters, cnt, N * r, K);
    D2_LAUNCH_CK(ctx, "k_prune_count");
    return D2_OK;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------

static uint64_t sm64(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" d2_prune* d2_prune_create(d2_ctx* ctx, int32_t d, int32_t H, int32_t E, const float* init, uint64_t seed) {
    if (!ctx || d < 1 || H < 32 || H > 256 || H % 32 || E < 1 || E > 256 || E % 16) {
        if (ctx) d2_fail(ctx, D2_EINVAL, "d2_prune_create: need d >= 1, H in {32..256} multiple of 32, E multiple of 16");
        return nullptr;
    }
    d2_prune* p = new d2_prune();
    p->d = d;
    p->H = H;
    p->E = E;
    p->device = ctx->device;
    p->oW1 = 0;
    p->ob1 = (int64_t)H * d;
    p->oW2 = p->ob1 + H;
    p->ob2 = p->oW2 + (int64_t)H * H;
    p->oW3 = p->ob2 + H;
    p->nparam = p->oW3 + (int64_t)E * H;
    std::vector<float> h(p->nparam);
    if (init) {
        memcpy(h.data(), init, p->nparam * 4);
    } else {
        uint64_t s = seed;
        auto fill = [&](int64_t o, int64_t n, int fan_in) {
            const double lim = std::sqrt(6.0 / fan_in);
            for (int64_t i = 0; i < n; ++i) {
                double u = (double)(sm64(s) >> 11) * (1.0 / 9007199254740992.0);
                h[o + i] = (float)((2.0 * u - 1.0) * lim);
            }
        };
        fill(p->oW1, (int64_t)H * d, d);
        for (int i = 0; i < H; ++i) h[p->ob1 + i] = 0.f;
        fill(p->oW2, (int64_t)H * H, H);
        for (int i = 0; i < H; ++i) h[p->ob2 + i] = 0.f;
        fill(p->oW3, (int64_t)E * H, H);
    }
    if (cudaMalloc(&p->params, p->nparam * 4) != cudaSuccess || cudaMalloc(&p->adam_m, p->nparam * 4) != cudaSuccess ||
        cudaMalloc(&p->adam_v, p->nparam * 4) != cudaSuccess) {
        d2_fail(ctx, D2_ENOMEM, "d2_prune_create: allocation failed");
        d2_prune_destroy(p);
        return nullptr;
    }
    cudaMemcpy(p->params, h.data(), p->nparam * 4, cudaMemcpyHostToDevice);
    cudaMemset(p->adam_m, 0, p->nparam * 4);
    cudaMemset(p->adam_v, 0, p->nparam * 4);
    return p;
}

extern "C" void d2_prune_destroy(d2_prune* p) {
    if (!p) return;
    if (p->params) cudaFree(p->params);
    if (p->adam_m) cudaFree(p->adam_m);
    if (p->adam_v) cudaFree(p->adam_v);
    delete p;
}

extern "C" int64_t d2_prune_param_count(const d2_prune* p) { return p ? p->nparam : 0; }

extern "C" int d2_prune_get_params(d2_ctx* ctx, const d2_prune* p, float* host_out) {
    if (!ctx || !p || !host_out) return D2_EINVAL;
    D2_CK(ctx, cudaDeviceSynchronize());
    D2_CK(ctx, cudaMemcpy(host_out, p->params, p->nparam * 4, cudaMemcpyDeviceToHost));
    return D2_OK;
}

extern "C" int d2_prune_set_params(d2_ctx* ctx, d2_prune* p, const float* host_in) {
    if (!ctx || !p || !host_in) return D2_EINVAL;
    D2_CK(ctx, cudaDeviceSynchronize());
    D2_CK(ctx, cudaMemcpy(p->params, host_in, p->nparam * 4, cudaMemcpyHostToDevice));
    return D2_OK;
}

__global__ void k_all_pairs(const int64_t* ids, int64_t nids, int K, int64_t* pb, int32_t* pc) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nids * K) return;
    pb[t] = ids[t / K];
    pc[t] = (int32_t)(t % K);
}

// from assign.cu
int d2_solve_pair_list(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                       const int64_t* pair_bag, const int32_t* pair_cent, int64_t max_pairs,
                       const int64_t* npairs_dev, float* out, int64_t* fail_count, cudaStream_t st);

extern "C" int d2_prune_calibrate(d2_ctx* ctx, d2_prune* p, const d2_bags* bags, int32_t K, int32_t m,
                                  const float* x, const float* w, const int64_t* ids, int64_t nids,
                                  float quantile, void* stream) {
    if (!ctx || !p) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (K < 1 || m < 1 || !x || !w || nids < 1 || !ids || !(quantile > 0.f && quantile <= 1.f))
        return d2_fail(ctx, D2_EINVAL, "d2_prune_calibrate: bad arguments");
    if (p->d != bags->d) return d2_fail(ctx, D2_EINVAL, "d2_prune_calibrate: pruner dimension %d != %d", p->d, bags->d);
    cudaStream_t st = d2_stream(stream);
    const int64_t np = nids * K;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_pb = take(np * 8), o_pc = take(np * 4), o_t = take(np * 4), o_f = take(nids * p->E * 4),
                 o_mu = take(nids * p->d * 4), o_fc = take((size_t)K * p->E * 4), o_muc = take((size_t)K * p->d * 4),
                 o_cnt = take(64);
    void* base = nullptr;
    if ((rc = d2_ws(ctx, WS_ASSIGN, off, &base))) return rc;
    char* b = static_cast<char*>(base);
    int64_t* pb = reinterpret_cast<int64_t*>(b + o_pb);
    int32_t* pc = reinterpret_cast<int32_t*>(b + o_pc);
    float* tg = reinterpret_cast<float*>(b + o_t);
    float* hf = reinterpret_cast<float*>(b + o_f);
    float* hmu = reinterpret_cast<float*>(b + o_mu);
    float* cf = reinterpret_cast<float*>(b + o_fc);
    float* cmu = reinterpret_cast<float*>(b + o_muc);
    int64_t* cnt = reinterpret_cast<int64_t*>(b + o_cnt);
    D2_CK(ctx, cudaMemsetAsync(cnt, 0, 16, st));
    k_all_pairs<<<(unsigned)d2_ceil_div(np, 256), 256, 0, st>>>(ids, nids, K, pb, pc);
    D2_LAUNCH_CK(ctx, "k_all_pairs");
    if ((rc = d2_solve_pair_list(ctx, bags, K, m, x, w, pb, pc, np, nullptr, tg, cnt + 1, st))) return rc;
    MlpArgs a = mlp_args(p, bags, x, w, m);
    a.nslots = nids;
    a.nbag_slots = nids;
    a.slot_id = ids;
    a.f = hf;
    a.mu = hmu;
    if ((rc = launch_fwd(ctx, p, a, st))) return rc;
    MlpArgs ac = mlp_args(p, bags, x, w, m);
    ac.nslots = K;
    ac.nbag_slots = 0;
    ac.f = cf;
    ac.mu = cmu;
    if ((rc = launch_fwd(ctx, p, ac, st))) return rc;
    D2_CK(ctx, cudaStreamSynchronize(st));
    std::vector<float> F(nids * p->E), MU(nids * p->d), FC((size_t)K * p->E), MUC((size_t)K * p->d), T(np);
    D2_CK(ctx, cudaMemcpy(F.data(), hf, F.size() * 4, cudaMemcpyDeviceToHost));
    D2_CK(ctx, cudaMemcpy(MU.data(), hmu, MU.size() * 4, cudaMemcpyDeviceToHost));
    D2_CK(ctx, cudaMemcpy(FC.data(), cf, FC.size() * 4, cudaMemcpyDeviceToHost));
    D2_CK(ctx, cudaMemcpy(MUC.data(), cmu, MUC.size() * 4, cudaMemcpyDeviceToHost));
    D2_CK(ctx, cudaMemcpy(T.data(), tg, T.size() * 4, cudaMemcpyDeviceToHost));
    std::vector<double> err(np), MT(np), PRED(np);
    for (int64_t i = 0; i < nids; ++i)
        for (int c = 0; c < K; ++c) {
            double mt = 0, pr = 0;
            for (int t = 0; t < p->d; ++t) {
                const double v = (double)MU[i * p->d + t] - MUC[(size_t)c * p->d + t];
                mt += v * v;
            }
            for (int e = 0; e < p->E; ++e) {
                const double v = (double)F[i * p->E + e] - FC[(size_t)c * p->E + e];
                pr += v * v;
            }
            MT[i * K + c] = mt;
            PRED[i * K + c] = mt + pr;
            err[i * K + c] = std::fabs(mt + pr - (double)T[i * K + c]);
        }
    const int64_t q = std::min<int64_t>(np - 1, std::max<int64_t>(0, (int64_t)std::ceil((double)quantile * np) - 1));
    std::nth_element(err.begin(), err.begin() + q, err.end());
    p->delta = (float)err[q];
    // the margin test of the pruned assignment replayed on the sample with the
    // new delta: candidates = the r smallest predictions (ties: lower index),
    // b = their best exact W^2; the bag falls back to all K when some other
    // centroid's bound max(mean term, prediction - delta) does not exceed b
    const int r = std::min(p->r, (int)K);
    int64_t fails = 0;
    std::vector<int> order(K);
    for (int64_t i = 0; i < nids; ++i) {
        const double* pi = PRED.data() + i * K;
        for (int c = 0; c < K; ++c) order[c] = c;
        std::partial_sort(order.begin(), order.begin() + r, order.end(),
                          [&](int a, int b) { return pi[a] < pi[b] || (pi[a] == pi[b] && a < b); });
        double b = 3.0e38;
        for (int t = 0; t < r; ++t) b = std::min(b, (double)T[i * K + order[t]]);
        bool fail = false;
        for (int t = r; t < K && !fail; ++t) {
            const int c = order[t];
            fail = !(std::max(MT[i * K + c], pi[c] - (double)p->delta) > b);
        }
        fails += fail;
    }
    p->fb_frac = (float)((double)fails / (double)nids);
    return D2_OK;
}

extern "C" int d2_prune_get_calibration(const d2_prune* p, float* fallback_frac) {
    if (!p || !fallback_frac) return D2_EINVAL;
    *fallback_frac = p->fb_frac;
    return D2_OK;
}

extern "C" int d2_prune_set_margin(d2_prune* p, int32_t r, float delta) {
    if (!p || r < 1 || r > 16 || !(delta >= 0.f)) return D2_EINVAL;
    p->r = r;
    p->delta = delta;
    return D2_OK;
}

extern "C" int d2_prune_get_margin(const d2_prune* p, int32_t* r, float* delta) {
    if (!p) return D2_EINVAL;
    if (r) *r = p->r;
    if (delta) *delta = p->delta;
    return D2_OK;
}

extern "C" int d2_prune_embed(d2_ctx* ctx, const d2_prune* p, const d2_bags* bags, const int64_t* ids, int64_t cnt,
                              float* emb, float* mu, void* stream) {
    if (!ctx || !p) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (bags->d != p->d || cnt < 0 || !emb || !mu) return d2_fail(ctx, D2_EINVAL, "d2_prune_embed: bad arguments");
    if (cnt == 0) return D2_OK;
    MlpArgs a = mlp_args(p, bags, nullptr, nullptr, 1);
    a.nslots = cnt;
    a.nbag_slots = cnt;
    a.slot_id = ids;
    a.f = emb;
    a.mu = mu;
    return launch_fwd(ctx, p, a, d2_stream(stream));
}

extern "C" int d2_prune_loss_grad(d2_ctx* ctx, const d2_prune* p, const d2_bags* bags, int32_t K, int32_t m,
                                  const float* x, const float* w, const int64_t* pair_bag, const int32_t* pair_cent,
                                  const float* target, int64_t B, double* loss, float* grad, void* stream) {
    if (!ctx || !p) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (bags->d != p->d || K < 1 || m < 1 || B < 1 || !x || !w || !pair_bag || !pair_cent || !target || !loss || !grad)
        return d2_fail(ctx, D2_EINVAL, "d2_prune_loss_grad: bad arguments");
    return loss_grad_impl(ctx, p, bags, K, m, x, w, pair_bag, pair_cent, target, B, loss, grad, d2_stream(stream));
}

extern "C" int d2_prune_train(d2_ctx* ctx, d2_prune* p, const d2_bags* bags, int32_t K, int32_t m, const float* x,
                              const float* w, const int64_t* pair_bag, const int32_t* pair_cent, const float* target,
                              int64_t npairs, int32_t steps, int32_t batch, float lr, uint64_t seed,
                              float* loss_out) {
    if (!ctx || !p) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (bags->d != p->d || K < 1 || m < 1 || npairs < 10 || steps < 1 || batch < 1 || !(lr > 0.f))
        return d2_fail(ctx, D2_EINVAL, "d2_prune_train: bad arguments");
    cudaStream_t st = 0;
    // the last tenth of the pairs is held out to calibrate delta
    const int64_t ntrain = npairs - npairs / 10;
    const int64_t nhold = npairs - ntrain;
    const int64_t B = std::min<int64_t>(batch, ntrain);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_idx = take(B * 8), o_pb = take(B * 8), o_pc = take(B * 4), o_pt = take(B * 4),
                 o_grad = take(p->nparam * 4), o_loss = take((size_t)steps * 8);
    void* base = nullptr;
    if ((rc = d2_ws(ctx, WS_CLUSTER_LOOP, off, &base))) return rc;
    char* bb = static_cast<char*>(base);
    int64_t* didx = reinterpret_cast<int64_t*>(bb + o_idx);
    int64_t* pb = reinterpret_cast<int64_t*>(bb + o_pb);
    int32_t* pc = reinterpret_cast<int32_t*>(bb + o_pc);
    float* pt = reinterpret_cast<float*>(bb + o_pt);
    float* grad = reinterpret_cast<float*>(bb + o_grad);
    double* losses = reinterpret_cast<double*>(bb + o_loss);
    std::vector<int64_t> hidx(B);
    uint64_t s = seed;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int it = 0; it < steps; ++it) {
        for (int64_t t = 0; t < B; ++t) hidx[t] = (int64_t)(sm64(s) % (uint64_t)ntrain);
        D2_CK(ctx, cudaMemcpyAsync(didx, hidx.data(), B * 8, cudaMemcpyHostToDevice, st));
        k_gather_pairs<<<(unsigned)d2_ceil_div(B, 256), 256, 0, st>>>(didx, B, pair_bag, pair_cent, target, pb, pc, pt);
        D2_LAUNCH_CK(ctx, "k_gather_pairs");
        if ((rc = loss_grad_impl(ctx, p, bags, K, m, x, w, pb, pc, pt, B, losses + it, grad, st))) return rc;
        p->step++;
        const float c1 = 1.f - std::pow(b1, (float)p->step), c2 = 1.f - std::pow(b2, (float)p->step);
        k_adam<<<(unsigned)d2_ceil_div(p->nparam, 256), 256, 0, st>>>(p->params, p->adam_m, p->adam_v, grad, p->nparam,
                                                                      lr, b1, b2, c1, c2);
        D2_LAUNCH_CK(ctx, "k_adam");
        D2_CK(ctx, cudaStreamSynchronize(st));  // hidx is reused
    }
    std::vector<double> hl(steps);
    D2_CK(ctx, cudaMemcpy(hl.data(), losses, steps * 8, cudaMemcpyDeviceToHost));
    if (loss_out)
        for (int it = 0; it < steps; ++it) loss_out[it] = (float)hl[it];
    // delta: the 99.9% quantile of |What^2 - W^2| on the held-out pairs
    if (nhold > 0) {
        const int64_t ns = 2 * nhold;
        size_t o2 = 0;
        auto take2 = [&](size_t bytes) {
            size_t o = o2;
            o2 += (bytes + 255) & ~(size_t)255;
            return o;
        };
        const size_t q_ids = take2(nhold * 8), q_f = take2(nhold * p->E * 4), q_mu = take2(nhold * p->d * 4),
                     q_fc = take2((size_t)K * p->E * 4), q_muc = take2((size_t)K * p->d * 4);
        void* b2p = nullptr;
        if ((rc = d2_ws(ctx, WS_ASSIGN, o2, &b2p))) return rc;
        (void)ns;
        char* c2b = static_cast<char*>(b2p);
        int64_t* hid = reinterpret_cast<int64_t*>(c2b + q_ids);
        float* hf = reinterpret_cast<float*>(c2b + q_f);
        float* hmu = reinterpret_cast<float*>(c2b + q_mu);
        float* cf = reinterpret_cast<float*>(c2b + q_fc);
        float* cmu = reinterpret_cast<float*>(c2b + q_muc);
        D2_CK(ctx, cudaMemcpy(hid, pair_bag + ntrain, nhold * 8, cudaMemcpyDeviceToDevice));
        MlpArgs a = mlp_args(p, bags, x, w, m);
        a.nslots = nhold;
        a.nbag_slots = nhold;
        a.slot_id = hid;
        a.f = hf;
        a.mu = hmu;
        if ((rc = launch_fwd(ctx, p, a, st))) return rc;
        MlpArgs ac = mlp_args(p, bags, x, w, m);
        ac.nslots = K;
        ac.nbag_slots = 0;
        ac.f = cf;
        ac.mu = cmu;
        if ((rc = launch_fwd(ctx, p, ac, st))) return rc;
        D2_CK(ctx, cudaStreamSynchronize(st));
        std::vector<float> F(nhold * p->E), MU(nhold * p->d), FC((size_t)K * p->E), MUC((size_t)K * p->d), T(nhold);
        std::vector<int32_t> C(nhold);
        D2_CK(ctx, cudaMemcpy(F.data(), hf, F.size() * 4, cudaMemcpyDeviceToHost));
        D2_CK(ctx, cudaMemcpy(MU.data(), hmu, MU.size() * 4, cudaMemcpyDeviceToHost));
        D2_CK(ctx, cudaMemcpy(FC.data(), cf, FC.size() * 4, cudaMemcpyDeviceToHost));
        D2_CK(ctx, cudaMemcpy(MUC.data(), cmu, MUC.size() * 4, cudaMemcpyDeviceToHost));
        D2_CK(ctx, cudaMemcpy(T.data(), target + ntrain, nhold * 4, cudaMemcpyDeviceToHost));
        D2_CK(ctx, cudaMemcpy(C.data(), pair_cent + ntrain, nhold * 4, cudaMemcpyDeviceToHost));
        std::vector<double> err(nhold);
        for (int64_t i = 0; i < nhold; ++i) {
            double mt = 0, pr = 0;
            for (int t = 0; t < p->d; ++t) {
                double v = (double)MU[i * p->d + t] - MUC[(size_t)C[i] * p->d + t];
                mt += v * v;
            }
            for (int e = 0; e < p->E; ++e) {
                double v = (double)F[i * p->E + e] - FC[(size_t)C[i] * p->E + e];
                pr += v * v;
            }
            err[i] = std::fabs(mt + pr - (double)T[i]);
        }
        std::sort(err.begin(), err.end());
        const int64_t q = std::min<int64_t>(nhold - 1, (int64_t)std::ceil(0.999 * nhold) - 1);
        p->delta = (float)err[std::max<int64_t>(q, 0)];
    }
    return D2_OK;
}
