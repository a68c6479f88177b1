// Tensor-core support partials (tcgen05 / TMEM, sm_103a) for the support
// update of Eq. (updatex):
//     x_i = (1 / (N w_i)) sum_k sum_j pi_ij^(k,2) y_j^(k)
// written on coordinates centred at the cluster's current centre mu_c,
//     x_i = mu_c + (1 / (N w_i)) sum_k sum_j pi_ij^(k,2) (y_j^(k) - mu_c),
// which is the same point because the plan's row sums add up to N w_i.  Per
// chunk of <= 64 member positions of one cluster, the sum over its support
// rows j is one dense contraction D = A B^T with
//     A (M = 128 support dimensions x K = rows) = (y - mu)^T,
//     B (N = m padded to 16 x K = rows)         = Pi^(2)^T,
// issued on the 5th-generation tensor cores with BF16 pieces of FP32 values
// (hi + lo: three products hi*hi + hi*lo + lo*hi, about 16 mantissa bits; or
// hi + mid + lo: six products, FP32-level) and an FP32 accumulator that stays
// in tensor memory across all row tiles of the chunk.
//
// Data flow per CTA (one chunk, one block of 64 support dimensions, which
// fill TMEM lanes 0..63 of the M = 128 accumulator; rows 64..127 of A are
// zero), warp-specialised:
//   * converter warps stage tiles of 64 rows in shared memory as FP32 by
//     asynchronous 16-byte copies, several tiles ahead of their use (as many
//     stages as fit), then centre each staged tile, split it into BF16
//     pieces and write it transposed into the 128-byte-swizzled K-major A and
//     B operands (one 16-byte store per piece and 8 rows), one or two
//     operand buffers;
//   * one lane of the MMA warp issues each tile's MMAs (4 K steps of 16 rows
//     x the piece products) once the converters have filled the buffer, and
//     commits them to the buffer's mbarrier;
//   * after the last tile two warps read the 64 TMEM lanes (support
//     dimensions) and write the chunk's m x d partial sums, which the exact
//     per-cluster sums of reduce.cu add up.
// Every wait is bounded (about 2 s of global time); on expiry the CTA records
// D2F_DEV_TIMEOUT in the context's device error word, skips the rest of its
// work, frees its tensor memory and returns.
#include <algorithm>

#include "d2_internal.cuh"
#include "tc_util.cuh"

namespace {

constexpr int XT_MAXT = 512;      // threads per CTA at most (256 + 4 m, m <= 64)
constexpr int XT_ROWS = 64;       // support rows per tile = one 64-element K block
constexpr int XT_M = 128;         // UMMA M (the support dimensions of a CTA fill lanes 0..63)
constexpr int XT_DW = 64;         // support dimensions per CTA
constexpr int XT_A_BYTES = XT_M * 128;  // one piece of A (16 KB; rows 64..127 stay zero)
constexpr int XT_YS = XT_DW + 4;  // staged y row stride (floats): 16-byte rows, conflict-free columns
constexpr int XT_MAX_SMEM = 227 * 1024 - 8 * 1024;  // dynamic part (static shared memory < 8 KB)
constexpr int XT_SMAX = 8;        // staging stages at most

struct XtArgs {
    const int64_t* members;
    const int64_t* offsets;
    const float* supp;
    const int32_t* vidx;
    const float* vocab;
    const float* plan;    // n x m, Pi^(2) rows (j-major)
    const float* mu;      // K x d, centre of each cluster
    int d, m, NP, PS, S;  // PS: staged plan row stride (floats); S: staging stages (<= XT_SMAX)
    int nbuf;             // operand buffers (1 or 2)
    int chunk_in_y;       // grid: (d blocks, chunks) when 1, else (chunks, d blocks)
    uint32_t tcols;
    const Chunk* chunks;
    const int64_t* nchunks;
    float* xpart;         // per chunk: m x d partial sums of the centred support
    int* err;             // sticky device error word
};

// v[0..7] (8 consecutive K elements) as NS BF16 pieces of 16 bytes, piece p
// at dst + p * stride: each piece is the round-to-nearest BF16 of what the
// previous pieces left over (hi, then lo; hi, mid, lo for NS = 3).
template <int NS>
__device__ __forceinline__ void split_store8(uint8_t* dst, size_t stride, float* v) {
#pragma unroll
    for (int p = 0; p < NS; ++p) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            w[q] = *reinterpret_cast<uint32_t*>(&b2);
        }
        *reinterpret_cast<uint4*>(dst + p * stride) = make_uint4(w[0], w[1], w[2], w[3]);
        if (p + 1 < NS) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[2 * q] -= __uint_as_float(w[q] << 16);
                v[2 * q + 1] -= __uint_as_float(w[q] & 0xffff0000u);
            }
        }
    }
}

// 16-byte asynchronous copy; nbytes = 0 fills the destination with zeros
__device__ __forceinline__ void cp16(uint32_t sdst, const void* gsrc, int nbytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sdst), "l"(gsrc), "r"(nbytes) : "memory");
}

// Barrier `id` over `count` threads that also ORs a flag across them.
__device__ __forceinline__ bool named_sync_or(int id, int count, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// One CTA per (chunk, block of 64 support dimensions), warp-specialised:
// warp 0 issues the MMAs; the 256 + 4 m converter threads behind it each own
// 2 conversion tasks (a support dimension or a point, and a group of 8 rows)
// and 4 of the 16-byte copies of every tile, the same every tile.  The
// converters synchronise among themselves (named barrier 1: a tile has
// landed, the stage converted before it may be refilled), hand a full
// operand buffer b to warp 0 by arriving on mbarrier full[b], and learn that
// buffer b is free again from mbarrier empty[b], where the MMAs' commit
// arrives.  Every wait is bounded; a wait that expires stops the role that
// waited (converters decide together, through the OR of named barrier 1), the
// other role's waits then expire too, and the chunk's result is discarded.
template <int NS>
__global__ void __launch_bounds__(XT_MAXT + 32, 1) k_xpartial_tc(XtArgs a) {
    extern __shared__ uint8_t dyn_raw[];
    __shared__ int64_t s_rs[D2_CHUNK];
    __shared__ int s_pre[D2_CHUNK + 1];
    __shared__ int64_t s_yoff[XT_SMAX][XT_ROWS];   // element offset of the y row (-1: past the chunk)
    __shared__ int32_t s_prow[XT_SMAX][XT_ROWS];   // support row (plan row) index, -1 past the chunk
    __shared__ __align__(16) float s_mu[XT_DW];
    __shared__ __align__(8) uint64_t s_bar[4];   // empty[0..1] (MMA commits), full[2..3] (converters)
    __shared__ uint32_t s_tmem;
    __shared__ int s_dead;

    const int64_t q = a.chunk_in_y ? blockIdx.y : blockIdx.x;
    const int db = a.chunk_in_y ? blockIdx.x : blockIdx.y;
    if (q >= *a.nchunks) return;
    const Chunk ch = a.chunks[q];
    const int c = ch.c;
    const int nm = (int)(ch.p1 - ch.p0);
    const int d = a.d, m = a.m, NP = a.NP, PS = a.PS, S = a.S, nbuf = a.nbuf;
    const int d0 = db * XT_DW;
    const int dv = min(XT_DW, d - d0);  // valid dimensions of this block
    const int nthr = blockDim.x, ncv = nthr - 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ct = tid - 32;  // converter index (warps 1..)

    // shared layout (1024-byte aligned for the swizzle): nbuf operand buffers
    // (NS pieces of A, then NS pieces of B of NP x 128 B), then S stages of
    // FP32 rows (64 x XT_YS of y, 64 x PS of the plan)
    const uint32_t raw = smem_u32(dyn_raw);
    const uint32_t pad = ((raw + 1023u) & ~1023u) - raw;
    uint8_t* base = dyn_raw + pad;
    const size_t bsz = (size_t)NP * 128;
    const size_t bufsz = (size_t)NS * XT_A_BYTES + NS * bsz;
    float* stage0 = reinterpret_cast<float*>(base + nbuf * bufsz);
    const int stage_floats = XT_ROWS * (XT_YS + PS);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(a.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_u32(&s_bar[0]), 1);
        mbar_init(smem_u32(&s_bar[1]), 1);
        mbar_init(smem_u32(&s_bar[2]), (uint32_t)ncv);
        mbar_init(smem_u32(&s_bar[3]), (uint32_t)ncv);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_dead = 0;
    }
    if (tid < nm) {
        const int64_t k = a.members[ch.p0 + tid];
        s_rs[tid] = a.offsets[k];
        s_pre[tid + 1] = (int)(a.offsets[k + 1] - a.offsets[k]);
    }
    if (tid < XT_DW) s_mu[tid] = tid < dv ? a.mu[(int64_t)c * d + d0 + tid] : 0.f;
    // rows 64..127 of A (no support dimension) and points >= m of B stay zero
    for (size_t e = (size_t)tid * 16; e < nbuf * bufsz; e += (size_t)nthr * 16)
        *reinterpret_cast<uint4*>(base + e) = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (warp == 0) {  // inclusive scan of the member sizes (2 per lane, nm <= 64)
        int v0 = 2 * lane < nm ? s_pre[2 * lane + 1] : 0;
        int v1 = 2 * lane + 1 < nm ? s_pre[2 * lane + 2] : 0;
        int sum = v0 + v1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, sum, o);
            if (lane >= o) sum += t;
        }
        if (2 * lane < nm) s_pre[2 * lane + 1] = sum - v1;
        if (2 * lane + 1 < nm) s_pre[2 * lane + 2] = sum;
        if (lane == 0) s_pre[0] = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const int R = s_pre[nm];
    const int ntiles = (R + XT_ROWS - 1) / XT_ROWS;
    const uint32_t tmem = s_tmem;
    const uint32_t bar0 = smem_u32(&s_bar[0]);   // empty[b] at bar0 + 8 b
    const uint32_t barf = smem_u32(&s_bar[2]);   // full[b] at barf + 8 b

    if (warp == 0) {
        // ---- MMA warp: one elected lane issues every tile's MMAs
        const uint32_t idesc = idesc_bf16_f32(XT_M, NP);
        uint32_t phf = 0u;  // per buffer: parity of its next fill
        for (int t = 0; t < ntiles; ++t) {
            const int buf = nbuf == 2 ? (t & 1) : 0;
            // the converters filled buffer buf with tile t
            int ok = 1;
            if (lane == 0) ok = mbar_wait_bounded(barf + 8 * buf, (phf >> buf) & 1u) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            phf ^= 1u << buf;
            if (!ok) {
                if (lane == 0) s_dead = 1;
                break;
            }
            tc_fence_after();
            if (lane == 0) {
                const uint32_t a_lo = smem_u32(base + (size_t)buf * bufsz);
                const uint64_t ad = sdesc_sw128(a_lo), bd = sdesc_sw128(a_lo + (uint32_t)(NS * XT_A_BYTES));
#pragma unroll
                for (int ks = 0; ks < XT_ROWS / 16; ++ks) {
#pragma unroll
                    for (int pa = 0; pa < NS; ++pa) {
#pragma unroll
                        for (int pb = 0; pa + pb < NS; ++pb) {
                            const bool first = t == 0 && ks == 0 && pa == 0 && pb == 0;
                            // start-address field in 16-byte units: pieces and the 32-byte K steps
                            umma_bf16(tmem, ad + (uint64_t)((pa * XT_A_BYTES + ks * 32) >> 4),
                                      bd + (uint64_t)((pb * bsz + ks * 32) >> 4), idesc, first ? 0u : 1u);
                        }
                    }
                }
                umma_commit(bar0 + 8 * buf);
            }
            __syncwarp();
        }
    } else {
        // ---- converters
        auto rows_of = [&](int t, int b) {  // offsets of the rows of tile t into slot b (converters 0..63)
            if (ct < XT_ROWS) {
                const int lr = t * XT_ROWS + ct;
                int64_t yo = -1;
                int32_t pr = -1;
                if (lr < R) {
                    int lo = 0, hi = nm - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_pre[mid] <= lr) lo = mid; else hi = mid - 1;
                    }
                    const int64_t g = s_rs[lo] + (lr - s_pre[lo]);
                    yo = a.supp ? g * d : (int64_t)a.vidx[g] * d;
                    pr = (int32_t)g;
                }
                s_yoff[b][ct] = yo;
                s_prow[b][ct] = pr;
            }
        };
        const float* ybase = a.supp ? a.supp : a.vocab;
        const int ysg = XT_DW / 4, psg = m / 4;
        const int ny = XT_ROWS * ysg, ncp = ny + XT_ROWS * psg;
        int cp_r[4], cp_col[4], cp_dst[4];  // row, source column (negative: plan column -1 - c), staging offset
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = ct + ncv * u;
            cp_r[u] = -1;
            cp_col[u] = 0;
            cp_dst[u] = 0;
            if (e < ny) {
                cp_r[u] = e / ysg;
                const int sg = e - cp_r[u] * ysg;
                cp_col[u] = 4 * sg;
                cp_dst[u] = cp_r[u] * XT_YS + 4 * sg;
            } else if (e < ncp) {
                const int f = e - ny;
                cp_r[u] = f / psg;
                const int sg = f - cp_r[u] * psg;
                cp_col[u] = -1 - 4 * sg;
                cp_dst[u] = XT_ROWS * XT_YS + cp_r[u] * PS + 4 * sg;
            }
        }
        auto issue = [&](int t, int b) {  // copies of tile t (row slot b) into stage b; one commit group
            if (t < ntiles) {
                const uint32_t sbase = smem_u32(stage0 + (size_t)b * stage_floats);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (cp_r[u] < 0) continue;
                    const uint32_t dst = sbase + 4u * (uint32_t)cp_dst[u];
                    if (cp_col[u] >= 0) {
                        const int64_t yo = s_yoff[b][cp_r[u]];
                        const bool ok = yo >= 0 && cp_col[u] < dv;
                        cp16(dst, ok ? ybase + yo + d0 + cp_col[u] : ybase, ok ? 16 : 0);
                    } else {
                        const int32_t pr = s_prow[b][cp_r[u]];
                        cp16(dst, pr >= 0 ? a.plan + (int64_t)pr * m + (-1 - cp_col[u]) : a.plan, pr >= 0 ? 16 : 0);
                    }
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        const int na = XT_DW * 8, ntask = na + m * 8;
        int tk_src[2], tk_dst[2], tk_dim[2], tk_rg[2];  // staging offset, operand offset, dd (A) / -1 (B) / -2, rg
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = ct + ncv * u;
            tk_dim[u] = -2;
            tk_rg[u] = 0;
            tk_src[u] = 0;
            tk_dst[u] = 0;
            if (e < na) {
                const int dd = e % XT_DW, rg = e / XT_DW;
                tk_dim[u] = dd;
                tk_rg[u] = rg;
                tk_src[u] = rg * 8 * XT_YS + dd;
                tk_dst[u] = (int)sw128_off(dd, rg * 8);
            } else if (e < ntask) {
                const int f = e - na;
                const int i = f % m, rg = f / m;
                tk_dim[u] = -1;
                tk_rg[u] = rg;
                tk_src[u] = XT_ROWS * XT_YS + rg * 8 * PS + i;
                tk_dst[u] = NS * XT_A_BYTES + (int)sw128_off(i, rg * 8);
            }
        }
        uint32_t ph = 0u;  // per operand buffer: parity of its next MMA completion
        bool dead = false;
        for (int t = 0; t < S - 1; ++t) rows_of(t, t);
        named_sync_or(1, ncv, false);
        for (int t = 0; t < S - 1; ++t) issue(t, t);
        if (S - 1 < ntiles) rows_of(S - 1, S - 1);
        for (int t = 0; t < ntiles; ++t) {
            const int buf = nbuf == 2 ? (t & 1) : 0, st = t % S;
            // tile t has landed when at most S - 2 later groups are outstanding
            switch (S) {
                case 2: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
                case 3: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
                case 4: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
                case 5: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
                case 6: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
                case 7: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
                default: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
            }
            // every converter's copies of tile t have landed; stage (t-1) % S is
            // free; stop together once any converter's wait has expired
            if (named_sync_or(1, ncv, dead)) break;
            issue(t + S - 1, (t + S - 1) % S);
            // buffer buf was last read by the MMAs of tile t - nbuf
            if (t >= nbuf) {
                if (!dead && !mbar_wait_bounded(bar0 + 8 * buf, (ph >> buf) & 1u)) dead = true;
                ph ^= 1u << buf;
            }
            if (!dead) {
                uint8_t* ob = base + (size_t)buf * bufsz;
                const float* sg = stage0 + (size_t)st * stage_floats;
                const int nvalid = min(XT_ROWS, R - t * XT_ROWS);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (tk_dim[u] == -2) continue;
                    float v[8];
                    if (tk_dim[u] >= 0) {  // A: centred support, zero past the chunk and past d
                        const float mu = s_mu[tk_dim[u]];
                        const bool okd = tk_dim[u] < dv;
#pragma unroll
                        for (int r = 0; r < 8; ++r)
                            v[r] = (okd && tk_rg[u] * 8 + r < nvalid) ? sg[tk_src[u] + r * XT_YS] - mu : 0.f;
                        split_store8<NS>(ob + tk_dst[u], XT_A_BYTES, v);
                    } else {               // B: plan (zero-filled past the chunk)
#pragma unroll
                        for (int r = 0; r < 8; ++r) v[r] = sg[tk_src[u] + r * PS];
                        split_store8<NS>(ob + tk_dst[u], bsz, v);
                    }
                }
                if (t + S < ntiles) rows_of(t + S, (t + S) % S);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tc_fence_before();
                mbar_arrive(barf + 8 * buf);  // buffer buf holds tile t
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (dead) s_dead = 1;
    }
    __syncthreads();
    // the accumulator is complete once the last commit has arrived (commits
    // complete in order, and the last covers every earlier MMA)
    if (tid == 0 && ntiles > 0 && !s_dead) {
        const int lb = nbuf == 2 ? ((ntiles - 1) & 1) : 0;
        // parity of that buffer's last completion: its uses so far minus one
        const int uses = nbuf == 2 ? (ntiles + 1 - lb) / 2 : ntiles;
        if (!mbar_wait_bounded(bar0 + 8 * lb, (uint32_t)((uses - 1) & 1))) s_dead = 1;
    }
    __syncthreads();
    tc_fence_after();
    const bool dead_all = s_dead != 0;
    if (!dead_all && ntiles > 0 && warp < 2) {
        const int dd = warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float* out = a.xpart + q * (int64_t)m * d + d0 + dd;
        for (int cb = 0; cb < NP; cb += 16) {
            float acc[16];
            tmem_ld16(trow + (uint32_t)cb, acc);
            if (dd < dv) {
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (cb + u < m) out[(int64_t)(cb + u) * d] = acc[u];
            }
        }
    }
    if (dead_all && tid == 0) atomicOr(a.err, D2F_DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tcols) : "memory");
}

struct XtPlan {
    int NP, ns, ndb, PS, S, nbuf;
    uint32_t tcols;
    size_t smem;
    const void* fn;
};

bool xt_plan(const d2_bags* b, int m, int prec, XtPlan* p) {
    if (prec != D2_COST_BF16 && prec != D2_COST_BF16X3 && prec != D2_COST_BF16X6) return false;
    const int d = b->d;
    const float* ybase = b->supp ? b->supp : b->vocab;
    if (d < 32 || d % 4 != 0 || m < 4 || m % 4 != 0 || m > 64 || (reinterpret_cast<uintptr_t>(ybase) & 15) ||
        b->n > INT32_MAX)
        return false;
    p->NP = (m + 15) / 16 * 16;
    p->PS = m + 4;
    p->ns = prec == D2_COST_BF16X6 ? 3 : 2;  // single-piece BF16 is too coarse for the support
    p->ndb = (d + XT_DW - 1) / XT_DW;
    uint32_t cols = 32;
    while ((int)cols < p->NP) cols <<= 1;
    p->tcols = cols;
    const size_t bufsz = (size_t)p->ns * XT_A_BYTES + (size_t)p->ns * p->NP * 128;
    const size_t stage = (size_t)XT_ROWS * (XT_YS + p->PS) * 4;
    // two CTAs per SM when one operand buffer and two stages fit in half the
    // SM's shared memory (CTA-wide barriers of one then overlap the other's
    // work); else one CTA with as many stages as fit and a second operand
    // buffer while 5 stages still fit
    const long half = (long)(228 * 1024) / 2 - 1024 - 8 * 1024;
    if (1024 + (long)bufsz + 2 * (long)stage <= half) {
        p->nbuf = 1;
        p->S = (int)std::min<long>(XT_SMAX, (half - 1024 - (long)bufsz) / (long)stage);
    } else {
        auto stages = [&](int nb) {
            const long room = (long)XT_MAX_SMEM - 1024 - (long)nb * (long)bufsz;
            return room < 0 ? 0 : std::min<long>(XT_SMAX, room / (long)stage);
        };
        p->nbuf = 2;
        p->S = (int)stages(2);
        if (p->S < 5) {
            p->nbuf = 1;
            p->S = (int)stages(1);
        }
    }
    if (p->S < 2) return false;
    p->smem = 1024 + (size_t)p->nbuf * bufsz + (size_t)p->S * stage;
    p->fn = p->ns == 3 ? (const void*)k_xpartial_tc<3> : (const void*)k_xpartial_tc<2>;
    return true;
}

}  // namespace

bool d2_support_tc_applies(const d2_bags* b, int m, int prec) {
    XtPlan p;
    return xt_plan(b, m, prec, &p);
}

int d2_support_tc_prepare(d2_ctx* ctx, const d2_bags* b, int m, int prec) {
    XtPlan p;
    if (!xt_plan(b, m, prec, &p)) return D2_OK;
    cudaError_t e = cudaFuncSetAttribute(p.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return d2_cuda_fail(ctx, e, "k_xpartial_tc smem attribute");
    return D2_OK;
}

// Partial sums of the centred support of every chunk (the caller adds them
// up, divides by N w_i and adds the centre back).
int d2_support_tc(d2_ctx* ctx, const d2_bags* b, const int64_t* members, int64_t maxch, int m, int prec,
                  const float* plan, const ClusterWs& cw, float* xpart, cudaStream_t st) {
    XtPlan p;
    if (!xt_plan(b, m, prec, &p)) return d2_fail(ctx, D2_ENOTSUP, "tensor-core support update does not apply");
    XtArgs a;
    a.members = members;
    a.offsets = b->offsets;
    a.supp = b->supp;
    a.vidx = b->vocab_idx;
    a.vocab = b->vocab;
    a.plan = plan;
    a.mu = cw.mu;
    a.d = b->d;
    a.m = m;
    a.NP = p.NP;
    a.PS = p.PS;
    a.S = p.S;
    a.nbuf = p.nbuf;
    a.tcols = p.tcols;
    a.chunks = cw.chunks;
    a.nchunks = cw.nchunks;
    a.xpart = xpart;
    a.err = ctx->dev_flags + D2_DEV_ERR_WORD;
    // the d blocks of one chunk run next to each other (their plan rows are
    // shared through L2) unless the chunk count exceeds the grid's y limit
    a.chunk_in_y = maxch <= 65535 ? 1 : 0;
    const dim3 grid = a.chunk_in_y ? dim3((unsigned)p.ndb, (unsigned)maxch) : dim3((unsigned)maxch, (unsigned)p.ndb);
    // an MMA warp and 256 + 4 m converters (2 conversion tasks, 4 copies each)
    const int nthr = 32 + (256 + 4 * m + 31) / 32 * 32;
    if (p.ns == 3)
        k_xpartial_tc<3><<<grid, nthr, p.smem, st>>>(a);
    else
        k_xpartial_tc<2><<<grid, nthr, p.smem, st>>>(a);
    D2_LAUNCH_CK(ctx, "k_xpartial_tc");
    return D2_OK;
}
