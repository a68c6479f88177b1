// Tensor-core cost build (tcgen05 / TMEM, sm_103a) for support dimensions
// d >= 32: the squared-Euclidean cost c(x_i, y_j) = ||x_i - y_j||^2 of the
// Section 2 notation list, written in the expanded form
//     C[j, i] = ||xt_i||^2 + ||yt_j||^2 - 2 <xt_i, yt_j>,
// xt = x_c - mu_c, yt = y_j - mu_c (the cluster's centring), where the dot
// products of a tile of 128 support rows against the cluster's m barycenter
// points are one dense contraction D = A B^T (M = 128, N = m padded to 16,
// K = d padded to 64) issued on the 5th-generation tensor cores with BF16
// operands and an FP32 accumulator in tensor memory.  The two norms stay FP32,
// computed from the unrounded FP32 coordinates (the compensation of the
// BF16 cross term).  With split operands (x3 mode) every factor is written as
// hi + lo (both BF16) and the three products hi*hi + hi*lo + lo*hi restore
// about 16 mantissa bits; with three pieces (x6 mode) hi + mid + lo holds the
// FP32 value exactly and the six products down to 2^-16 of the leading one
// leave an error at the FP32 rounding level.
//
// Data flow per CTA (one chunk of <= 64 member positions of one cluster):
//   * the cluster's centred barycenter support is converted once to BF16 and
//     stored K-major in 128-byte-swizzled shared memory (the B operand);
//   * each step loads one 64-column block of 128 member rows from HBM into
//     registers (coalesced float4 loads, one step ahead of its use), centres
//     and converts it, and stores it as the swizzled K-major A operand;
//   * one thread issues the MMAs of the block and commits them to an
//     mbarrier; the next step's loads are in flight meanwhile;
//   * after the last block of a tile every warp reads its 32 TMEM lanes
//     (rows) with tcgen05.ld, adds the norms, clamps at 0 and streams the
//     j-major cost rows out; the FP64 row sums feed Eq. (rho).
// Every mbarrier wait is bounded (about 2 s of global time); on expiry the
// CTA records D2F_DEV_TIMEOUT in the context's device error word, skips the
// rest of its work, frees its tensor memory and returns.
#include "d2_internal.cuh"
#include "tc_util.cuh"

namespace {

constexpr int TC_ROWS = 128;     // UMMA M: support rows per tile (one per TMEM lane)

constexpr int TC_THREADS = 128;  // 4 warps: warp w owns TMEM lanes 32w..32w+31
constexpr int TC_TILE_BYTES = TC_ROWS * 128;  // one K block of A (16 KB)
constexpr int TC_MAX_SMEM = 200 * 1024;

struct TcArgs {
    const int64_t* members;
    const int64_t* offsets;
    const float* supp;
    const int32_t* vidx;
    const float* vocab;
    int d, m, NP, nkb;
    uint32_t tcols;       // TMEM columns allocated per CTA (power of 2 >= 32)
    const float* xt;      // K x m x d  centred barycenter support
    const float* xn;      // K x m      ||xt_i||^2
    const float* mu;      // K x d      centre
    const Chunk* chunks;
    const int64_t* nchunks;
    float* C;             // n x m, j-major
    double* chunk_sum;    // per chunk (or null)
    int64_t* chunk_rows;
    int* err;             // sticky device error word
    int expire_test;      // testing: no MMA for the first tile, so its wait expires
};

// NS = 1: BF16 operands; NS = 2: hi + lo pieces (three products); NS = 3:
// hi + mid + lo pieces (six products, FP32-equivalent operands).
template <int NS>
__global__ void __launch_bounds__(TC_THREADS) k_cost_tc(TcArgs a) {
    extern __shared__ uint8_t dyn_raw[];
    __shared__ int64_t s_rs[D2_CHUNK];
    __shared__ int s_pre[D2_CHUNK + 1];
    __shared__ int64_t s_row[2][TC_ROWS];
    __shared__ float s_yn[2][TC_ROWS];
    __shared__ __align__(16) float s_xn[256];
    __shared__ double s_red[TC_THREADS / 32];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_dead;

    const int64_t q = blockIdx.x;
    if (q >= *a.nchunks) return;
    const Chunk ch = a.chunks[q];
    const int c = ch.c;
    const int nm = (int)(ch.p1 - ch.p0);
    const int d = a.d, m = a.m, NP = a.NP, nkb = a.nkb;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // shared layout (1024-byte aligned for the swizzle): A buffers, B hi, B lo, mu
    const uint32_t raw = smem_u32(dyn_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* base = dyn_raw + pad;
    const int nbuf = nkb == 1 ? 1 : 2;
    uint8_t* A = base;                                           // nbuf x NS x 16 KB
    uint8_t* B = A + (size_t)nbuf * NS * TC_TILE_BYTES;           // NS x nkb x NP x 128 B
    const size_t bsz = (size_t)nkb * NP * 128;
    float* smu = reinterpret_cast<float*>(B + NS * bsz);          // nkb * 64 floats

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(a.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&s_bar[0]), 1);
        mbar_init(smem_u32(&s_bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_dead = 0;
    }
    if (tid < nm) {
        const int64_t k = a.members[ch.p0 + tid];
        s_rs[tid] = a.offsets[k];
        s_pre[tid + 1] = (int)(a.offsets[k + 1] - a.offsets[k]);
    }
    for (int t = tid; t < nkb * TC_KB; t += TC_THREADS) smu[t] = t < d ? a.mu[(int64_t)c * d + t] : 0.f;
    for (int i = tid; i < NP; i += TC_THREADS) s_xn[i] = i < m ? a.xn[(int64_t)c * m + i] : 0.f;
    // B operand: the centred barycenter points, rows i < NP, K padded with zeros
    for (int e = tid; e < NP * nkb * (TC_KB / 4); e += TC_THREADS) {
        const int i = e / (nkb * (TC_KB / 4));
        const int rem = e - i * (nkb * (TC_KB / 4));
        const int kb = rem / (TC_KB / 4), k4 = (rem - kb * (TC_KB / 4)) * 4;
        const int col = kb * TC_KB + k4;
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = (i < m && col + u < d) ? a.xt[((int64_t)c * m + i) * d + col + u] : 0.f;
        const uint32_t off = (uint32_t)(kb * NP * 128) + sw128_off(i, k4);
        store_pieces<NS>(B + off, bsz, v[0], v[1], v[2], v[3]);
    }
    __syncthreads();
    if (tid == 0) {
        s_pre[0] = 0;
        for (int t = 0; t < nm; ++t) s_pre[t + 1] += s_pre[t];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const int R = s_pre[nm];
    const int ntiles = (R + TC_ROWS - 1) / TC_ROWS;
    const int nsteps = ntiles * nkb;
    const uint32_t bar0 = smem_u32(&s_bar[0]);
    const uint32_t idesc = idesc_bf16_f32(TC_ROWS, NP);

    // global row of local row lr of the chunk (-1 past the end)
    auto row_of = [&](int lr) -> int64_t {
        if (lr >= R) return -1;
        int lo = 0, hi = nm - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= lr) lo = mid; else hi = mid - 1;
        }
        return s_rs[lo] + (lr - s_pre[lo]);
    };
    // loader mapping: 16 lanes per row (one float4 each), 8 rows per pass
    const int c4 = tid & 15, rsub = tid >> 4;
    float4 v[16];
    auto load_step = [&](int s) {
        const int t = s / nkb, kb = s - t * nkb;
        const int col = kb * TC_KB + c4 * 4;
#pragma unroll
        for (int qq = 0; qq < 16; ++qq) {
            const int64_t g = s_row[t & 1][rsub + 8 * qq];
            v[qq] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (g >= 0 && col < d)
                v[qq] = __ldg(reinterpret_cast<const float4*>(d2_row_ptr(a.supp, a.vidx, a.vocab, d, g) + col));
        }
    };

    s_row[0][tid] = row_of(tid);
    __syncthreads();
    if (nsteps > 0) load_step(0);

    float ynp[16];
    uint32_t pend = 0u, ph = 0u;  // per A buffer b: bit b = MMAs outstanding / phase parity
    bool dead = false;
    double rowsum_acc = 0.0;

    for (int s = 0; s < nsteps; ++s) {
        const int t = s / nkb, kb = s - t * nkb;
        const int buf = nbuf == 1 ? 0 : (s & 1);
        if (kb == 0) {
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) ynp[qq] = 0.f;
        }
        if ((pend >> buf) & 1u) {  // the MMAs that last read this A buffer
            if (!mbar_wait_bounded(bar0 + 8 * buf, (ph >> buf) & 1u)) dead = true;
            ph ^= 1u << buf;
            pend &= ~(1u << buf);
            if (__syncthreads_or(dead)) break;
        }
        // centre, accumulate norms, convert and store the A block(s)
        {
            uint8_t* Ahi = A + (size_t)buf * NS * TC_TILE_BYTES;
            const float4 mu4 = *reinterpret_cast<const float4*>(smu + kb * TC_KB + c4 * 4);
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) {
                const int r = rsub + 8 * qq;
                const float y0 = v[qq].x - mu4.x, y1 = v[qq].y - mu4.y;
                const float y2 = v[qq].z - mu4.z, y3 = v[qq].w - mu4.w;
                const bool ok = s_row[t & 1][r] >= 0 && kb * TC_KB + c4 * 4 < d;
                const float z0 = ok ? y0 : 0.f, z1 = ok ? y1 : 0.f, z2 = ok ? y2 : 0.f, z3 = ok ? y3 : 0.f;
                ynp[qq] = fmaf(z0, z0, fmaf(z1, z1, fmaf(z2, z2, fmaf(z3, z3, ynp[qq]))));
                store_pieces<NS>(Ahi + sw128_off(r, c4 * 4), TC_TILE_BYTES, z0, z1, z2, z3);
            }
        }
        const bool last_kb = kb == nkb - 1;
        if (last_kb) {
#pragma unroll
            for (int qq = 0; qq < 16; ++qq) {
                float sv = ynp[qq];
                sv += __shfl_xor_sync(0xffffffffu, sv, 8);
                sv += __shfl_xor_sync(0xffffffffu, sv, 4);
                sv += __shfl_xor_sync(0xffffffffu, sv, 2);
                sv += __shfl_xor_sync(0xffffffffu, sv, 1);
                if (c4 == 0) s_yn[t & 1][rsub + 8 * qq] = sv;
            }
        }
        const int64_t my_g = s_row[t & 1][tid];  // this thread's output row (epilogue)
        if (last_kb && t + 1 < ntiles) s_row[(t + 1) & 1][tid] = row_of((t + 1) * TC_ROWS + tid);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0 && !(a.expire_test && s == 0)) {
            const uint32_t a_hi = smem_u32(A + (size_t)buf * NS * TC_TILE_BYTES);
            const uint32_t b_hi = smem_u32(B + (size_t)kb * NP * 128);
            // products of the pieces: (a, b) with a + b <= NS - 1 (hi = 0),
            // i.e. every term down to 2^-8(NS-1) of the leading one
#pragma unroll
            for (int ks = 0; ks < TC_KB / 16; ++ks) {
                const uint32_t koff = (uint32_t)ks * 32u;
#pragma unroll
                for (int pa = 0; pa < NS; ++pa) {
#pragma unroll
                    for (int pb = 0; pa + pb < NS; ++pb) {
                        const bool first = kb == 0 && ks == 0 && pa == 0 && pb == 0;
                        umma_bf16(tmem, sdesc_sw128(a_hi + (uint32_t)(pa * TC_TILE_BYTES) + koff),
                                  sdesc_sw128(b_hi + (uint32_t)(pb * bsz) + koff), idesc, first ? 0u : 1u);
                    }
                }
            }
            umma_commit(bar0 + 8 * buf);
        }
        pend |= 1u << buf;
        if (s + 1 < nsteps) load_step(s + 1);  // in flight during the MMA and the epilogue
        if (last_kb) {
            if (!mbar_wait_bounded(bar0 + 8 * buf, (ph >> buf) & 1u)) dead = true;
            ph ^= 1u << buf;
            pend &= ~(1u << buf);
            if (__syncthreads_or(dead)) break;
            tc_fence_after();
            const float yn = s_yn[t & 1][tid];
            const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
            float rs = 0.f;
            for (int cb = 0; cb < NP; cb += 16) {
                float acc[16];
                tmem_ld16(trow + (uint32_t)cb, acc);
                if (my_g >= 0) {
                    float* out = a.C + my_g * m;
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        const int col = cb + i;
                        if (col < m) {
                            const float4 xv = *reinterpret_cast<const float4*>(s_xn + col);
                            float4 o;
                            o.x = fmaxf(fmaf(-2.f, acc[i], xv.x + yn), 0.f);
                            o.y = fmaxf(fmaf(-2.f, acc[i + 1], xv.y + yn), 0.f);
                            o.z = fmaxf(fmaf(-2.f, acc[i + 2], xv.z + yn), 0.f);
                            o.w = fmaxf(fmaf(-2.f, acc[i + 3], xv.w + yn), 0.f);
                            __stcs(reinterpret_cast<float4*>(out + col), o);
                            rs += (o.x + o.y) + (o.z + o.w);
                        }
                    }
                }
            }
            rowsum_acc += (double)rs;
            tc_fence_before();
        }
    }
    // drain: no MMA may still be in flight when tensor memory is released
    for (int b = 0; b < 2; ++b) {
        if (((pend >> b) & 1u) && !dead) {
            if (!mbar_wait_bounded(bar0 + 8 * b, (ph >> b) & 1u)) dead = true;
            pend &= ~(1u << b);
        }
    }
    if (dead && lane == 0) atomicOr(a.err, D2F_DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tcols) : "memory");
    if (a.chunk_sum) {
        const double sv = group_sum_d<32>(rowsum_acc);
        if (lane == 0) s_red[warp] = sv;
        __syncthreads();
        if (tid == 0) {
            double sum = 0.0;
            for (int w = 0; w < TC_THREADS / 32; ++w) sum += s_red[w];
            a.chunk_sum[q] = sum;
            a.chunk_rows[q] = R;
        }
    }
}

struct TcPlan {
    int NP, nkb, ns;
    uint32_t tcols;
    size_t smem;
    const void* fn;
};

// Launch shape of the tensor-core build for (d, m, precision); false when the
// problem is outside what it covers (then the FP32 build is used).
bool tc_plan(const d2_bags* b, int m, int prec, TcPlan* p) {
    if (prec != D2_COST_BF16 && prec != D2_COST_BF16X3 && prec != D2_COST_BF16X6) return false;
    const int d = b->d;
    const float* base = b->supp ? b->supp : b->vocab;
    if (d < 32 || d % 4 != 0 || m % 4 != 0 || m > 256 || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    p->NP = (m + 15) / 16 * 16;
    p->nkb = (d + TC_KB - 1) / TC_KB;
    p->ns = prec == D2_COST_BF16X6 ? 3 : prec == D2_COST_BF16X3 ? 2 : 1;
    uint32_t cols = 32;
    while ((int)cols < p->NP) cols <<= 1;
    p->tcols = cols;
    const int nbuf = p->nkb == 1 ? 1 : 2;
    size_t smem = 1024 + (size_t)nbuf * p->ns * TC_TILE_BYTES + (size_t)p->ns * p->nkb * p->NP * 128 +
                  (size_t)p->nkb * TC_KB * 4;
    if (smem > TC_MAX_SMEM) return false;
    // keep resident CTAs x TMEM columns within the SM's 512 columns: size the
    // shared-memory request so that at most 512 / cols CTAs fit on one SM
    const int max_ctas = 512 / (int)cols;
    // (static shared memory and the per-CTA reservation only add to it; 16
    // CTAs of 128 threads already fill the SM's 2048 threads)
    const size_t sm_bytes = 228 * 1024;
    const size_t cap_req = sm_bytes / (size_t)(max_ctas + 1) + 1;
    if (max_ctas < 16 && smem < cap_req) smem = cap_req;
    p->smem = smem;
    p->fn = p->ns == 3 ? (const void*)k_cost_tc<3> : p->ns == 2 ? (const void*)k_cost_tc<2>
                                                 : (const void*)k_cost_tc<1>;
    return true;
}

}  // namespace

bool d2_cost_tc_applies(const d2_bags* b, int m, int prec) {
    TcPlan p;
    return tc_plan(b, m, prec, &p);
}

int d2_cost_tc_prepare(d2_ctx* ctx, const d2_bags* b, int m, int prec, bool* used) {
    TcPlan p;
    *used = tc_plan(b, m, prec, &p);
    if (!*used) return D2_OK;
    cudaError_t e = cudaFuncSetAttribute(p.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return d2_cuda_fail(ctx, e, "k_cost_tc smem attribute");
    return D2_OK;
}

int d2_cost_tc_rows(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t maxch, int m, int prec,
                    const ClusterWs& cw, float* C, double* chunk_sum, int64_t* chunk_rows, cudaStream_t st,
                    bool* used) {
    TcPlan p;
    *used = tc_plan(b, m, prec, &p);
    if (!*used) return D2_OK;
    TcArgs a;
    a.members = members;
    a.offsets = b->offsets;
    a.supp = b->supp;
    a.vidx = b->vocab_idx;
    a.vocab = b->vocab;
    a.d = b->d;
    a.m = m;
    a.NP = p.NP;
    a.nkb = p.nkb;
    a.tcols = p.tcols;
    a.xt = cw.xt;
    a.xn = cw.xn;
    a.mu = cw.mu;
    a.chunks = cw.chunks;
    a.nchunks = cw.nchunks;
    a.C = C;
    a.chunk_sum = chunk_sum;
    a.chunk_rows = chunk_rows;
    a.err = ctx->dev_flags + D2_DEV_ERR_WORD;
    a.expire_test = ctx->expire_test;
    d2_time_begin(ctx, D2_KT_COST, st);
    if (p.ns == 3)
        k_cost_tc<3><<<(unsigned)maxch, TC_THREADS, p.smem, st>>>(a);
    else if (p.ns == 2)
        k_cost_tc<2><<<(unsigned)maxch, TC_THREADS, p.smem, st>>>(a);
    else
        k_cost_tc<1><<<(unsigned)maxch, TC_THREADS, p.smem, st>>>(a);
    d2_time_end(ctx, st);
    D2_LAUNCH_CK(ctx, "k_cost_tc");
    return D2_OK;
}
