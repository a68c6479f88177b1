// Centroid update with B-ADMM (Algorithm badmm, Section 3.3) for all clusters
// at once.
//
// Plan sweep.  Between launches the only per-entry state is two n x m FP32
// arrays (the plan buffer and Lambda) plus the cost C; every launch streams
// them once.  One warp owns one member (one cluster position) and walks its
// m_k j-major rows; a row of m entries is split over LPR lanes holding NV
// vectors of VEC floats each, so the column normalisation of Eq. (badmmc0)
// (over the m barycenter points) is a shuffle reduction inside a lane group
// and the row sums r_{k,i} of Eq. (badmmc1b) (over the member's m_k points)
// are per-lane accumulators folded once per member.
//
// The iteration is re-associated so that the dual update of iteration n-1 and
// the plan update of iteration n share one pass (FUSED):
//   in : Pi1^n (plan buffer), Lambda^{n-1}, C, r^n_k, w^n
//   B  : Pt = Pi1 exp(Lambda/rho) + eps;  Pi2^n = Pt w_i / r_{k,i};
//        Lambda^n = Lambda^{n-1} + rho (Pi1^n - Pi2^n)                (Eqs. badmmc1, badmm2)
//   A  : T1 = Pi2^n exp(-(C + Lambda^n)/rho) + eps;
//        Pi1^{n+1} = T1 w_j^(k) / sum_i T1;                             (Eqs. badmmc0b, badmmc0)
//        r^{n+1}_{k,i} = sum_j (Pi1^{n+1} exp(Lambda^n/rho) + eps)     (Eq. badmmc1b)
//   out: Pi1^{n+1}, Lambda^n, r^{n+1}_k, wtilde^(k) = r_k / sum_i r_{k,i}
// so each iteration reads Pi, Lambda, C and writes Pi, Lambda: 20 bytes per
// entry.  The exponent of the A step is shifted by its row maximum s in the
// log2 domain and eps is scaled by 2^-s, which leaves Pi1 unchanged in exact
// arithmetic and keeps FP32 from underflowing on far-away points.
//
// Weight consensus (Eq. badmmw / badmmw2).  Each warp writes its member's
// wtilde^(k) (FP32, normalised by one reciprocal); a small kernel then sums
// every cluster's members in a fixed order in FP64 and publishes w^{n+1} for
// the next pass, so the result does not depend on scheduling and the sweep
// itself has no atomics, fences or barriers.  Warps are persistent and take
// member positions round-robin, so no warp idles waiting for a sibling that
// owns a longer member.
#include <algorithm>
#include <cstring>

#include "d2_internal.cuh"

#define SWEEP_WARPS 8
#define SWEEP_THREADS (SWEEP_WARPS * 32)
#ifndef D2_SWEEP_MINB
#define D2_SWEEP_MINB 3   // resident CTAs per SM the register budget must allow
#endif

enum SweepFlags {
    SW_B = 1,            // input plan buffer holds Pi1^n: do the B step
    SW_A = 2,            // do the A step
    SW_LAM_ZERO = 4,     // Lambda input is identically zero (not read)
    SW_LAM_OUT = 8,      // write Lambda^n
    SW_COLD = 16,        // (A only) Pi2^0 = w_i w_j^(k) unless warm_mask[k]
    SW_OBJ = 32,         // accumulate <C, Pi1^{n+1}> per member
    SW_R2 = 64,          // consensus rule R2 (store sqrt of wtilde)
};

struct SweepArgs {
    const int64_t* members;
    const int32_t* pos_cluster;
    int64_t P;
    const int64_t* offsets;
    const float* wt;
    float* plan;
    float* lam;
    const float* cost;
    float* pos_r;
    float* pos_part;
    double* pos_obj;
    const float* w_cur;
    float* w_next;       // null: weights fixed, no consensus
    double* w_next64;
    const float* beta;   // per cluster log2(e) / rho
    const float* rho;
    int* counters;
    const int64_t* cofs;
    const uint8_t* warm_mask;
    int m;
    float eps;
    float log2eps;
    int flags;
};

template <int VEC>
struct VecIO;
// plan, dual and cost rows are touched once per launch: stream them past L1
// and mark them evict-first in L2
template <>
struct VecIO<4> {
    static __device__ __forceinline__ void ld(const float* p, float* v) {
        float4 t = __ldcs(reinterpret_cast<const float4*>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float* p, const float* v) {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
    }
};
template <>
struct VecIO<1> {
    static __device__ __forceinline__ void ld(const float* p, float* v) { v[0] = __ldcs(p); }
    static __device__ __forceinline__ void st(float* p, const float* v) { __stcs(p, v[0]); }
};

// 2^x by the hardware approximation (relative error ~2^-22, flushes
// subnormal results to zero)
__device__ __forceinline__ float fast_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Double-float accumulation: a running sum held as an unevaluated pair
// hi + lo of FP32 numbers, updated by error-free transformations (Knuth's
// TwoSum; the product's rounding error by one FMA), so it carries about 48
// significant bits, like an FP64 running sum, with FP32 instructions only
// (FP64 throughput on this part is a small fraction of FP32).  The _rn
// intrinsics keep the compiler from contracting the steps into FMAs.
__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);  // a b = p + pe exactly
    df_add(hi, lo, p);
    lo = __fadd_rn(lo, pe);
}

template <int VEC, int LPR, int NV>
__global__ void __launch_bounds__(SWEEP_THREADS, D2_SWEEP_MINB) k_sweep(SweepArgs a) {
    constexpr int RPW = 32 / LPR;   // rows per warp step
    constexpr int NE = VEC * NV;    // floats per lane per row

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int sub = lane / LPR, cl = lane % LPR;
    const int m = a.m;
    const int fl = a.flags;
    const bool doA = fl & SW_A, doB = fl & SW_B;
    const int64_t nwarps = (int64_t)gridDim.x * SWEEP_WARPS;

    // persistent warps: member positions round-robin, no CTA-level barrier
    for (int64_t p = (int64_t)blockIdx.x * SWEEP_WARPS + wib; p < a.P; p += nwarps) {
        const int64_t k = a.members[p];
        const int c = a.pos_cluster[p];
        const int64_t row0 = a.offsets[k];
        const int mk = (int)(a.offsets[k + 1] - row0);
        const float beta = a.beta[c];
        const float rho = a.rho[c];
        const float eps = a.eps;
        const bool cold = (fl & SW_COLD) && !(a.warm_mask && a.warm_mask[k]);

        // per-lane column constants
        float coef[NE], wcol[NE];
        bool ok[NE];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int col = (cl + LPR * v) * VEC + e;
                const int x = v * VEC + e;
                ok[x] = col < m;
                float wc = ok[x] ? a.w_cur[(int64_t)c * m + col] : 0.f;
                wcol[x] = wc;
                coef[x] = (doB && ok[x]) ? wc / a.pos_r[p * m + col] : 0.f;
            }

        float racc[NE];
#pragma unroll
        for (int x = 0; x < NE; ++x) racc[x] = 0.f;
        float objhi = 0.f, objlo = 0.f;  // <C_k, Pi^(k,1)> of this lane's entries, double-float (objective pass)

        // one row group (RPW rows) per step; the next group's loads are issued
        // before the current group is computed
        const bool ldP = doB || !cold, ldL = !(fl & SW_LAM_ZERO);
        float pin[NE], lin[NE], cin[NE], wkj;
        auto load_step = [&](int base, float* P, float* L, float* Cc, float& wk) {
            const int j = base + sub;
#pragma unroll
            for (int x = 0; x < NE; ++x) { P[x] = 0.f; L[x] = 0.f; Cc[x] = 0.f; }
            wk = 0.f;
            if (j < mk) {
                const int64_t ro = (row0 + j) * (int64_t)m;
                wk = __ldg(a.wt + row0 + j);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int col0 = (cl + LPR * v) * VEC;
                    if (col0 < m) {
                        if (ldP) VecIO<VEC>::ld(a.plan + ro + col0, P + v * VEC);
                        if (ldL) VecIO<VEC>::ld(a.lam + ro + col0, L + v * VEC);
                        if (doA) VecIO<VEC>::ld(a.cost + ro + col0, Cc + v * VEC);
                    }
                }
            }
        };
        load_step(0, pin, lin, cin, wkj);
        for (int base = 0; base < mk; base += RPW) {
            float npin[NE], nlin[NE], ncin[NE], nwkj;
            if (base + RPW < mk) load_step(base + RPW, npin, nlin, ncin, nwkj);
            const int j = base + sub;
            const bool rv = j < mk;
            const int64_t rowoff = (row0 + (rv ? j : 0)) * (int64_t)m;
            // ---- B step: Pi2^n and Lambda^n from Pi1^n and Lambda^{n-1}
            float p2[NE], l2[NE];
#pragma unroll
            for (int x = 0; x < NE; ++x) {
                if (doB) {
                    const float pt = fmaf(pin[x], fast_exp2(lin[x] * beta), eps);
                    p2[x] = pt * coef[x];
                    l2[x] = fmaf(rho, pin[x] - p2[x], lin[x]);
                } else {
                    p2[x] = cold ? wcol[x] * wkj : pin[x];
                    l2[x] = lin[x];
                }
            }
            if (doA) {
                // ---- A step: Pi1^{n+1} with a row-max shift in the log2 domain
                float ex[NE];
                float s = -INFINITY;
#pragma unroll
                for (int x = 0; x < NE; ++x) {
                    ex[x] = -(cin[x] + l2[x]) * beta;
                    if (ok[x]) s = fmaxf(s, ex[x]);
                }
                s = group_max<LPR>(s);
                const float epss = fast_exp2(fminf(a.log2eps - s, 126.f));
                float t1[NE];
                float rs = 0.f;
#pragma unroll
                for (int x = 0; x < NE; ++x) {
                    t1[x] = ok[x] ? fmaf(p2[x], fast_exp2(ex[x] - s), epss) : 0.f;
                    rs += t1[x];
                }
                rs = group_sum<LPR>(rs);
                const float scale = rs > 0.f ? wkj / rs : 0.f;
                float p1n[NE];
#pragma unroll
                for (int x = 0; x < NE; ++x) {
                    p1n[x] = t1[x] * scale;
                    if (rv && ok[x]) racc[x] += fmaf(p1n[x], fast_exp2(l2[x] * beta), eps);
                }
                if (fl & SW_OBJ) {  // objective pass only
#pragma unroll
                    for (int x = 0; x < NE; ++x)
                        if (rv && ok[x]) df_add_prod(objhi, objlo, cin[x], p1n[x]);
                }
                if (rv) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const int col0 = (cl + LPR * v) * VEC;
                        if (col0 < m) {
                            VecIO<VEC>::st(a.plan + rowoff + col0, p1n + v * VEC);
                            if (fl & SW_LAM_OUT) VecIO<VEC>::st(a.lam + rowoff + col0, l2 + v * VEC);
                        }
                    }
                }
            } else if (rv) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    const int col0 = (cl + LPR * v) * VEC;
                    if (col0 < m) {
                        VecIO<VEC>::st(a.plan + rowoff + col0, p2 + v * VEC);
                        if (fl & SW_LAM_OUT) VecIO<VEC>::st(a.lam + rowoff + col0, l2 + v * VEC);
                    }
                }
            }
            if (base + RPW < mk) {
#pragma unroll
                for (int x = 0; x < NE; ++x) { pin[x] = npin[x]; lin[x] = nlin[x]; cin[x] = ncin[x]; }
                wkj = nwkj;
            }
        }

        if (doA) {
            // fold the row sums of the RPW row groups of the warp
#pragma unroll
            for (int x = 0; x < NE; ++x)
#pragma unroll
                for (int o = LPR; o < 32; o <<= 1) racc[x] += __shfl_xor_sync(0xffffffffu, racc[x], o);
            float tl = 0.f;
#pragma unroll
            for (int x = 0; x < NE; ++x)
                if (ok[x]) tl += racc[x];
            tl = group_sum<LPR>(tl);
            const float inv_tl = 1.0f / tl;
            if (sub == 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        const int col = (cl + LPR * v) * VEC + e;
                        const int x = v * VEC + e;
                        if (ok[x]) {
                            a.pos_r[p * m + col] = racc[x];
                            const float wtl = racc[x] * inv_tl;
                            a.pos_part[p * m + col] = (fl & SW_R2) ? sqrtf(wtl) : wtl;
                        }
                    }
            }
            if (fl & SW_OBJ) {
                double ov = group_sum_d<32>((double)objhi + (double)objlo);
                if (lane == 0) a.pos_obj[p] = ov;
            }
        }
    }
}


// ---------------------------------------------------------------------------
// Pipelined variant for m % 4 == 0 (NV float4s per lane per row: NV = 1 for
// m <= 128, NV = 2 for m % 8 == 0 up to 256).
// Each warp runs a PIPE_S-stage ring in shared memory: stage s holds one row
// group (RPW rows) of the plan buffer, Lambda and C, the rows' weights and,
// on the first row group of a member, that member's r_k and w slice.  Lanes
// copy exactly the bytes they will consume (cp.async, 16 B), so a stage is
// ready for a lane once its own copies have landed; PIPE_S - 1 row groups
// are in flight per warp while one is computed, without holding them in
// registers.  The issue side walks the same member sequence as the compute
// side and leaves each stage's member metadata next to its data.
// ---------------------------------------------------------------------------

struct PipeMeta {
    int64_t p;      // member position (-1: no more work)
    int64_t row0;   // first support row of the member
    int mk, base, c, flags;  // flags: 1 = first row group, 2 = plan was copied
};

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

template <int LPR, int NV, int S>
struct PipeWarp {
    float4 data[S][3][NV][32];    // plan, lambda, cost
    float4 hdr[S][2][NV][LPR];    // r_k and w columns of the member (first group)
    float wk[S][32 / LPR];        // row weights
    PipeMeta meta[S];
    PipeMeta cur;                 // issue cursor: member being issued, next row group
};

#ifndef D2_PIPE_MINB
#define D2_PIPE_MINB 2    // the ring's shared memory allows 2 CTAs/SM at NV = 2
#endif

template <int LPR, int NV, int S>
__global__ void __launch_bounds__(SWEEP_THREADS, D2_PIPE_MINB) k_sweep_pipe(SweepArgs a) {
    constexpr int RPW = 32 / LPR;
    constexpr int NE = 4 * NV;
    extern __shared__ float4 pipe_dyn[];
    PipeWarp<LPR, NV, S>* pw = reinterpret_cast<PipeWarp<LPR, NV, S>*>(pipe_dyn) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int sub = lane / LPR, cl = lane % LPR;
    const int m = a.m;
    const int fl = a.flags;
    const bool doA = fl & SW_A, doB = fl & SW_B;
    const bool ldL = !(fl & SW_LAM_ZERO);
    bool okv[NV];
    int colv[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        colv[v] = (cl + LPR * v) * 4;
        okv[v] = colv[v] < m;
    }
    const int64_t nw = (int64_t)gridDim.x * SWEEP_WARPS;

    // ---- issue cursor (lives in shared memory; lane 0 advances it)
    auto load_cursor = [&](int64_t ip) {
        __syncwarp();
        if (lane == 0) {
            PipeMeta cu;
            cu.p = ip < a.P ? ip : -1;
            cu.row0 = 0;
            cu.mk = 0;
            cu.base = 0;
            cu.c = 0;
            cu.flags = 0;
            if (ip < a.P) {
                const int64_t k = a.members[ip];
                cu.row0 = a.offsets[k];
                cu.mk = (int)(a.offsets[k + 1] - cu.row0);
                cu.c = a.pos_cluster[ip];
                const bool cold = (fl & SW_COLD) && !(a.warm_mask && a.warm_mask[k]);
                cu.flags = (doB || !cold) ? 2 : 0;
            }
            pw->cur = cu;
        }
        __syncwarp();
    };
    load_cursor((int64_t)blockIdx.x * SWEEP_WARPS + (threadIdx.x >> 5));
    auto issue = [&](int slot) {
        const PipeMeta cu = pw->cur;
        if (cu.p >= 0) {
            const int j = cu.base + sub;
            if (j < cu.mk) {
                const int64_t ro = (cu.row0 + j) * (int64_t)m;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (okv[v]) {
                        if (cu.flags & 2) cp_async16(&pw->data[slot][0][v][lane], a.plan + ro + colv[v]);
                        if (ldL) cp_async16(&pw->data[slot][1][v][lane], a.lam + ro + colv[v]);
                        if (doA) cp_async16(&pw->data[slot][2][v][lane], a.cost + ro + colv[v]);
                    }
                }
                if (cl == 0) cp_async4(&pw->wk[slot][sub], a.wt + cu.row0 + j);
            }
            if (cu.base == 0 && sub == 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (okv[v]) {
                        if (doB) cp_async16(&pw->hdr[slot][0][v][cl], a.pos_r + cu.p * m + colv[v]);
                        cp_async16(&pw->hdr[slot][1][v][cl], a.w_cur + (int64_t)cu.c * m + colv[v]);
                    }
                }
            }
            if (lane == 0) {
                PipeMeta mt = cu;
                mt.flags = cu.flags | (cu.base == 0 ? 1 : 0);
                pw->meta[slot] = mt;
            }
            if (cu.base + RPW >= cu.mk) {
                load_cursor(cu.p + nw);
            } else {
                __syncwarp();
                if (lane == 0) pw->cur.base = cu.base + RPW;
                __syncwarp();
            }
        } else if (lane == 0) {
            pw->meta[slot].p = -1;
        }
        cp_async_commit();
    };

#pragma unroll
    for (int s0 = 0; s0 < S - 1; ++s0) issue(s0);

    // ---- compute cursor state (per member)
    float coef[NE], wcol[NE], racc[NE];
    float beta = 0.f, rho = 0.f;
    float objhi = 0.f, objlo = 0.f;  // <C_k, Pi^(k,1)> of this lane's entries, double-float (objective pass)
    bool ldP = false;
    const float eps = a.eps;
    int slot = 0;
    for (;;) {
        cp_async_wait<S - 2>();
        __syncwarp();
        const PipeMeta mt = pw->meta[slot];
        if (mt.p < 0) break;
        const int64_t p = mt.p;
        const int c = mt.c;
        if (mt.flags & 1) {
            beta = a.beta[c];
            rho = a.rho[c];
            ldP = mt.flags & 2;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float4 wv = pw->hdr[slot][1][v][cl];
                const float4 rv4 = pw->hdr[slot][0][v][cl];
                const float wa[4] = {wv.x, wv.y, wv.z, wv.w};
                const float ra[4] = {rv4.x, rv4.y, rv4.z, rv4.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    wcol[v * 4 + e] = okv[v] ? wa[e] : 0.f;
                    coef[v * 4 + e] = (doB && okv[v]) ? wa[e] / ra[e] : 0.f;
                }
            }
#pragma unroll
            for (int x = 0; x < NE; ++x) racc[x] = 0.f;
            objhi = objlo = 0.f;
        }
        const int j = mt.base + sub;
        const bool rv = j < mt.mk;
        float pin[NE], lin[NE], cin[NE];
        float wkj = 0.f;
        if (rv) wkj = pw->wk[slot][sub];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            float4 tp = make_float4(0.f, 0.f, 0.f, 0.f), tl = tp, tc = tp;
            if (rv && okv[v]) {
                if (ldP) tp = pw->data[slot][0][v][lane];
                if (ldL) tl = pw->data[slot][1][v][lane];
                if (doA) tc = pw->data[slot][2][v][lane];
            }
            pin[v * 4] = tp.x; pin[v * 4 + 1] = tp.y; pin[v * 4 + 2] = tp.z; pin[v * 4 + 3] = tp.w;
            lin[v * 4] = tl.x; lin[v * 4 + 1] = tl.y; lin[v * 4 + 2] = tl.z; lin[v * 4 + 3] = tl.w;
            cin[v * 4] = tc.x; cin[v * 4 + 1] = tc.y; cin[v * 4 + 2] = tc.z; cin[v * 4 + 3] = tc.w;
        }
        const int64_t rowoff = (mt.row0 + (rv ? j : 0)) * (int64_t)m;
        float p2[NE], l2[NE];
#pragma unroll
        for (int x = 0; x < NE; ++x) {
            if (doB) {
                const float pt = fmaf(pin[x], fast_exp2(lin[x] * beta), eps);
                p2[x] = pt * coef[x];
                l2[x] = fmaf(rho, pin[x] - p2[x], lin[x]);
            } else {
                p2[x] = ldP ? pin[x] : wcol[x] * wkj;
                l2[x] = lin[x];
            }
        }
        if (doA) {
            float ex[NE];
            float smax = -INFINITY;
#pragma unroll
            for (int x = 0; x < NE; ++x) {
                ex[x] = -(cin[x] + l2[x]) * beta;
                if (okv[x / 4]) smax = fmaxf(smax, ex[x]);
            }
            smax = group_max<LPR>(smax);
            const float epss = fast_exp2(fminf(a.log2eps - smax, 126.f));
            float t1[NE];
            float rs = 0.f;
#pragma unroll
            for (int x = 0; x < NE; ++x) {
                t1[x] = okv[x / 4] ? fmaf(p2[x], fast_exp2(ex[x] - smax), epss) : 0.f;
                rs += t1[x];
            }
            rs = group_sum<LPR>(rs);
            const float scale = rs > 0.f ? wkj / rs : 0.f;
            float p1n[NE];
#pragma unroll
            for (int x = 0; x < NE; ++x) {
                p1n[x] = t1[x] * scale;
                if (rv && okv[x / 4]) racc[x] += fmaf(p1n[x], fast_exp2(l2[x] * beta), eps);
            }
            if (fl & SW_OBJ) {  // objective pass only
#pragma unroll
                for (int x = 0; x < NE; ++x)
                    if (rv && okv[x / 4]) df_add_prod(objhi, objlo, cin[x], p1n[x]);
            }
            if (rv) {
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    if (okv[v]) {
                        VecIO<4>::st(a.plan + rowoff + colv[v], p1n + v * 4);
                        if (fl & SW_LAM_OUT) VecIO<4>::st(a.lam + rowoff + colv[v], l2 + v * 4);
                    }
            }
        } else if (rv) {
#pragma unroll
            for (int v = 0; v < NV; ++v)
                if (okv[v]) {
                    VecIO<4>::st(a.plan + rowoff + colv[v], p2 + v * 4);
                    if (fl & SW_LAM_OUT) VecIO<4>::st(a.lam + rowoff + colv[v], l2 + v * 4);
                }
        }
        const bool last = mt.base + RPW >= mt.mk;
        __syncwarp();
        // refill the slot consumed one step earlier: stage n + S - 1 goes to
        // slot (n + S - 1) mod S
        issue(slot == 0 ? S - 1 : slot - 1);
        slot = (slot + 1 == S) ? 0 : slot + 1;

        if (last && doA) {
#pragma unroll
            for (int x = 0; x < NE; ++x)
#pragma unroll
                for (int o = LPR; o < 32; o <<= 1) racc[x] += __shfl_xor_sync(0xffffffffu, racc[x], o);
            float tl = 0.f;
#pragma unroll
            for (int x = 0; x < NE; ++x)
                if (okv[x / 4]) tl += racc[x];
            tl = group_sum<LPR>(tl);
            const float inv_tl = 1.0f / tl;
            if (sub == 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (!okv[v]) continue;
                    const float* rr = racc + v * 4;
                    *reinterpret_cast<float4*>(a.pos_r + p * m + colv[v]) = make_float4(rr[0], rr[1], rr[2], rr[3]);
                    float q[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float wtl = rr[e] * inv_tl;
                        q[e] = (fl & SW_R2) ? sqrtf(wtl) : wtl;
                    }
                    *reinterpret_cast<float4*>(a.pos_part + p * m + colv[v]) = make_float4(q[0], q[1], q[2], q[3]);
                }
            }
            if (fl & SW_OBJ) {
                double ov = group_sum_d<32>((double)objhi + (double)objlo);
                if (lane == 0) a.pos_obj[p] = ov;
            }
        }
    }
    cp_async_wait<0>();
}

typedef void (*SweepFn)(SweepArgs);

#ifndef D2_PIPE_NV
#define D2_PIPE_NV 2     // float4s per lane per row in the pipelined sweep (2: m % 8 == 0)
#endif
#ifndef D2_PIPE_S
#define D2_PIPE_S 4      // ring stages per warp
#endif

template <int LPR, int NV>
static SweepFn pipe_variant(size_t* smem, int* lpr) {
    *smem = SWEEP_WARPS * sizeof(PipeWarp<LPR, NV, D2_PIPE_S>);
    *lpr = LPR;
    return k_sweep_pipe<LPR, NV, D2_PIPE_S>;
}

// Pipelined sweep with NV float4s per lane (2 needs m % 8 == 0; 1 needs m <= 128).
static SweepFn pipe_with(int m, int nv, size_t* smem, int* lpr) {
    if (m % 4 != 0 || m > 256) return nullptr;
    if (nv == 2) {
        if (m < 8 || m % 8 != 0) return nullptr;
        if (m <= 8) return pipe_variant<1, 2>(smem, lpr);
        if (m <= 16) return pipe_variant<2, 2>(smem, lpr);
        if (m <= 32) return pipe_variant<4, 2>(smem, lpr);
        if (m <= 64) return pipe_variant<8, 2>(smem, lpr);
        if (m <= 128) return pipe_variant<16, 2>(smem, lpr);
        return pipe_variant<32, 2>(smem, lpr);
    }
    if (m > 128) return nullptr;
    if (m <= 4) return pipe_variant<1, 1>(smem, lpr);
    if (m <= 8) return pipe_variant<2, 1>(smem, lpr);
    if (m <= 16) return pipe_variant<4, 1>(smem, lpr);
    if (m <= 32) return pipe_variant<8, 1>(smem, lpr);
    if (m <= 64) return pipe_variant<16, 1>(smem, lpr);
    return pipe_variant<32, 1>(smem, lpr);
}

// Default shape without the autotuner: two float4s per lane unless that ring
// leaves room for only one CTA per SM and the one-float4 ring exists (at
// m = 64, 8 lanes x 2 float4 at 1 CTA/SM measured 18 % slower than 16 lanes x
// 1 float4 at 3 CTAs/SM).
static SweepFn pick_sweep_pipe(int m, size_t* smem) {
    int lpr = 0;
    size_t s2 = 0, s1 = 0;
    SweepFn f2 = D2_PIPE_NV == 2 ? pipe_with(m, 2, &s2, &lpr) : nullptr;
    SweepFn f1 = pipe_with(m, 1, &s1, &lpr);
    if (f2 && (s2 <= 110 * 1024 || !f1)) {
        *smem = s2;
        return f2;
    }
    if (f1) *smem = s1;
    return f1;
}

static SweepFn pick_sweep(int m, int* lpr = nullptr, int* nv = nullptr) {
    int l = 32, v = 1;
    SweepFn f;
    if (m % 4 == 0) {
        if (m <= 4) { f = k_sweep<4, 1, 1>; l = 1; }
        else if (m <= 8) { f = k_sweep<4, 2, 1>; l = 2; }
        else if (m <= 16) { f = k_sweep<4, 4, 1>; l = 4; }
        else if (m <= 32) { f = k_sweep<4, 8, 1>; l = 8; }
        else if (m <= 64) { f = k_sweep<4, 16, 1>; l = 16; }
        else if (m <= 128) { f = k_sweep<4, 32, 1>; l = 32; }
        else { f = k_sweep<4, 32, 2>; l = 32; v = 2; }
    } else {
        v = 0;  // scalar lanes
        if (m <= 1) { f = k_sweep<1, 1, 1>; l = 1; }
        else if (m <= 2) { f = k_sweep<1, 2, 1>; l = 2; }
        else if (m <= 4) { f = k_sweep<1, 4, 1>; l = 4; }
        else if (m <= 8) { f = k_sweep<1, 8, 1>; l = 8; }
        else if (m <= 16) { f = k_sweep<1, 16, 1>; l = 16; }
        else if (m <= 32) { f = k_sweep<1, 32, 1>; l = 32; }
        else if (m <= 64) f = k_sweep<1, 32, 2>;
        else if (m <= 128) f = k_sweep<1, 32, 4>;
        else f = k_sweep<1, 32, 8>;
    }
    if (lpr) *lpr = l;
    if (nv) *nv = v;
    return f;
}

// One candidate launch shape of the plan sweep for the autotuner.
struct SweepCand {
    SweepFn fn;
    size_t smem;
    int kind, lpr, nv, per_sm;
};

// Candidates for plan width m: pipelined with 2 or 1 float4s per lane and the
// register-prefetch sweep, each with 1 .. (max resident) persistent CTAs per SM.
static int sweep_candidates(d2_ctx* ctx, int m, std::vector<SweepCand>* out) {
    struct Base { SweepFn fn; size_t smem; int kind, lpr, nv; };
    std::vector<Base> bases;
    for (int nv = 2; nv >= 1; --nv) {
        size_t sm = 0;
        int lpr = 0;
        SweepFn f = pipe_with(m, nv, &sm, &lpr);
        if (f) bases.push_back({f, sm, 0, lpr, nv});
    }
    {
        int lpr = 0, nv = 0;
        SweepFn f = pick_sweep(m, &lpr, &nv);
        bases.push_back({f, 0, 1, lpr, nv});
    }
    for (const Base& b : bases) {
        if (b.smem > 48 * 1024)
            D2_CK(ctx, cudaFuncSetAttribute(b.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.smem));
        int occ = 1;
        D2_CK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, b.fn, SWEEP_THREADS, b.smem));
        occ = std::max(1, std::min(occ, 4));
        for (int k = 1; k <= occ && (int)out->size() < D2_TUNE_MAX; ++k)
            out->push_back({b.fn, b.smem, b.kind, b.lpr, b.nv, k});
    }
    return D2_OK;
}

static SweepTune* find_tune(d2_ctx* ctx, int m) {
    for (auto& t : ctx->tuned)
        if (t.m == m) return &t;
    return nullptr;
}

extern "C" int d2_sweep_tuning(const d2_ctx* ctx, int32_t m, int32_t* ncand, int32_t* chosen, float* ms,
                               int32_t* shape) {
    if (!ctx) return D2_EINVAL;
    if (ncand) *ncand = 0;
    if (chosen) *chosen = -1;
    for (const auto& t : ctx->tuned) {
        if (t.m != m) continue;
        if (ncand) *ncand = t.ncand;
        if (chosen) *chosen = t.chosen;
        for (int i = 0; i < t.ncand; ++i) {
            if (ms) ms[i] = t.ms[i];
            if (shape)
                for (int q = 0; q < 4; ++q) shape[i * 4 + q] = t.shape[i][q];
        }
    }
    return D2_OK;
}

// ---------------------------------------------------------------------------
// support update (Eq. updatex): per-chunk partial sums of Pi2^T Y (their
// exact sum per cluster and the division by N_c w_i are in reduce.cu)
// ---------------------------------------------------------------------------
#define XU_THREADS 256
#define XU_ROWS 32
#define XU_DT 64
#define XU_MT 32

__global__ void __launch_bounds__(XU_THREADS) k_xpartial(const int64_t* members, const int64_t* offsets,
                                                         const float* supp, const int32_t* vidx,
                                                         const float* vocab, int d, int m, const float* plan,
                                                         const Chunk* chunks, const int64_t* nchunks,
                                                         float* xpart) {
    __shared__ float ps[XU_ROWS][XU_MT + 1];
    __shared__ float ys[XU_ROWS][XU_DT + 1];
    __shared__ int64_t s_rs[D2_CHUNK];
    __shared__ int s_pre[D2_CHUNK + 1];
    __shared__ int64_t s_row[XU_ROWS];
    const int64_t q = blockIdx.x;
    if (q >= *nchunks) return;
    const int d0 = blockIdx.y * XU_DT, i0 = blockIdx.z * XU_MT;
    if (d0 >= d || i0 >= m) return;
    const Chunk ch = chunks[q];
    const int nm = (int)(ch.p1 - ch.p0);
    const int tid = threadIdx.x;
    if (tid < nm) {
        int64_t k = members[ch.p0 + tid];
        s_rs[tid] = offsets[k];
        s_pre[tid + 1] = (int)(offsets[k + 1] - offsets[k]);
    }
    __syncthreads();
    if (tid == 0) {
        s_pre[0] = 0;
        for (int t = 0; t < nm; ++t) s_pre[t + 1] += s_pre[t];
    }
    __syncthreads();
    const int R = s_pre[nm];
    const int dd = tid % XU_DT, ig = tid / XU_DT;  // 4 groups of i
    constexpr int NA = XU_MT / (XU_THREADS / XU_DT);
    float acc[NA];
#pragma unroll
    for (int t = 0; t < NA; ++t) acc[t] = 0.f;
    for (int rb = 0; rb < R; rb += XU_ROWS) {
        __syncthreads();
        if (tid < XU_ROWS) {
            int lr = rb + tid;
            int64_t g = -1;
            if (lr < R) {
                int lo = 0, hi = nm - 1;
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (s_pre[mid] <= lr) lo = mid; else hi = mid - 1;
                }
                g = s_rs[lo] + (lr - s_pre[lo]);
            }
            s_row[tid] = g;
        }
        __syncthreads();
        for (int idx = tid; idx < XU_ROWS * XU_MT; idx += XU_THREADS) {
            int r = idx / XU_MT, i = idx % XU_MT;
            int64_t g = s_row[r];
            ps[r][i] = (g >= 0 && i0 + i < m) ? plan[g * m + i0 + i] : 0.f;
        }
        for (int idx = tid; idx < XU_ROWS * XU_DT; idx += XU_THREADS) {
            int r = idx / XU_DT, t = idx % XU_DT;
            int64_t g = s_row[r];
            ys[r][t] = (g >= 0 && d0 + t < d) ? d2_row_ptr(supp, vidx, vocab, d, g)[d0 + t] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < XU_ROWS; ++r) {
            const float yv = ys[r][dd];
#pragma unroll
            for (int t = 0; t < NA; ++t) acc[t] = fmaf(ps[r][ig + 4 * t], yv, acc[t]);
        }
    }
    float* out = xpart + q * (int64_t)m * d;
    if (d0 + dd < d) {
#pragma unroll
        for (int t = 0; t < NA; ++t) {
            int i = i0 + ig + 4 * t;
            if (i < m) out[(int64_t)i * d + d0 + dd] = acc[t];
        }
    }
}


// Support partials on the CUDA cores for m % 4 == 0 and d % 4 == 0 (rows of
// 16-byte multiples).  A CTA owns one chunk and one 32 (i) x 64 (d) tile of
// the chunk's m x d partial sum; the CTAs of one chunk are adjacent in the
// grid, so the rows that several tiles read come from L2 after the first.
// Its XW_WARPS warps take the chunk's row tiles of XW_RW rows round-robin,
// each through a private ring of XW_S stages filled by 16-byte asynchronous
// copies (no CTA barrier until the end).  Each lane accumulates an 8 x 8
// block of the tile with paired FP32 fused multiply-adds (each product
// rounded once, as fmaf), reading 16 values per row from shared memory.  The
// warps' partial tiles are then added in warp order, so the result depends
// on the chunk alone, not on timing.
#define XW_WARPS 4
#define XW_RW 8
#define XW_S 4
#define XW_RED (64 + 4)   // row stride of the partial tiles in shared memory (floats)

struct XwStage {
    float p[XW_RW][32];   // Pi2 row slice i0 .. i0 + 31
    float y[XW_RW][64];   // support row slice d0 .. d0 + 63
};
static_assert(sizeof(XwStage) * XW_S >= 32 * XW_RED * 4, "a warp's ring holds its partial tile");
constexpr size_t XW_SMEM = sizeof(XwStage) * XW_S * XW_WARPS;

__device__ __forceinline__ void xp_cp16(void* sdst, const void* gsrc) {
    unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc));
}

__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__global__ void __launch_bounds__(XW_WARPS * 32, 4)
k_xpartial_warp(const int64_t* members, const int64_t* offsets, const float* supp, const int32_t* vidx,
                const float* vocab, int d, int m, const float* plan, const Chunk* chunks, const int64_t* nchunks,
                int ntd, int ntiles, float* xpart) {
    extern __shared__ __align__(16) unsigned char xw_raw[];
    __shared__ int64_t s_rs[D2_CHUNK];
    __shared__ int s_pre[D2_CHUNK + 1];
    const int64_t q = blockIdx.x / (unsigned)ntiles;
    const int tile = (int)(blockIdx.x - (unsigned)(q * ntiles));
    if (q >= *nchunks) return;
    const int i0 = (tile / ntd) * 32, d0 = (tile % ntd) * 64;
    const Chunk ch = chunks[q];
    const int nm = (int)(ch.p1 - ch.p0);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (w == 0) {
        // row starts of the members and the exclusive prefix sums of their
        // row counts (nm <= 64: two members per lane); entries past nm hold
        // the total
        const int t0 = 2 * lane, t1 = t0 + 1;
        int c0 = 0, c1 = 0;
        if (t0 < nm) {
            const int64_t k = members[ch.p0 + t0];
            s_rs[t0] = offsets[k];
            c0 = (int)(offsets[k + 1] - offsets[k]);
        }
        if (t1 < nm) {
            const int64_t k = members[ch.p0 + t1];
            s_rs[t1] = offsets[k];
            c1 = (int)(offsets[k + 1] - offsets[k]);
        }
        int incl = c0 + c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int excl = incl - c0 - c1;
        s_pre[t0] = excl;
        s_pre[t1] = excl + c0;
        if (lane == 31) s_pre[D2_CHUNK] = incl;
    }
    __syncthreads();
    const int R = s_pre[nm];
    const int NT = (R + XW_RW - 1) / XW_RW;
    XwStage* ring = reinterpret_cast<XwStage*>(xw_raw) + w * XW_S;
    const int np4 = min(32, m - i0) >> 2, ny4 = min(64, d - d0) >> 2;

    // stage j of this warp: its row tile w + j XW_WARPS (an empty group past
    // the end).  Lanes 0..7 find the row of plan row r = lane and lanes 8..15
    // the support row of row r = lane - 8 (member by a fixed six-step search of
    // the prefix sums, nm <= 64); each lane then copies two 16-byte Pi2
    // segments and four support segments.  Rows past the chunk read as zero.
    const int sr = lane & 7;
    auto issue = [&](int j) {
        const int t = w + j * XW_WARPS;
        if (t < NT) {
            XwStage& st = ring[j % XW_S];
            const int lr = t * XW_RW + sr;
            const float* rp = nullptr;
            if (lane < 16 && lr < R) {
                int lo = 0;
#pragma unroll
                for (int step = 32; step > 0; step >>= 1)
                    if (lo + step < nm && s_pre[lo + step] <= lr) lo += step;
                const int64_t g = s_rs[lo] + (lr - s_pre[lo]);
                rp = lane < 8 ? plan + g * m + i0 : d2_row_ptr(supp, vidx, vocab, d, g) + d0;
            }
#pragma unroll
            for (int it = 0; it < 2; ++it) {  // Pi2: 8 rows x 8 segments
                const int r = (lane >> 3) + 4 * it, sg = lane & 7;
                const float* src = reinterpret_cast<const float*>(__shfl_sync(0xffffffffu, (unsigned long long)rp, r));
                float* dst = &st.p[r][sg * 4];
                if (src && sg < np4) xp_cp16(dst, src + sg * 4);
                else if (!src) *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int it = 0; it < 4; ++it) {  // support: 8 rows x 16 segments
                const int r = (lane >> 4) + 2 * it, sg = lane & 15;
                const float* src =
                    reinterpret_cast<const float*>(__shfl_sync(0xffffffffu, (unsigned long long)rp, 8 + r));
                float* dst = &st.y[r][sg * 4];
                if (src && sg < ny4) xp_cp16(dst, src + sg * 4);
                else if (!src) *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
                // (a column past m or d of a real row keeps whatever the stage
                // held: it only meets accumulators that are never stored)
            }
        }
        asm volatile("cp.async.commit_group;");
    };

    // lane (ig, dg) owns i in {4 ig .. 4 ig + 3} + {0, 16} and d in {4 dg .. 4 dg + 3} + {0, 32}
    const int ig = lane & 3, dg = lane >> 2;
    unsigned long long acc[8][4];  // acc[a 4 + u][b 2 + h] = (i = 16 a + 4 ig + u; d = 32 b + 4 dg + 2 h, + 1)
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0ull;
#pragma unroll
    for (int j = 0; j < XW_S - 1; ++j) issue(j);
    const int nmine = NT > w ? (NT - w + XW_WARPS - 1) / XW_WARPS : 0;
    for (int j = 0; j < nmine; ++j) {
        issue(j + XW_S - 1);  // into the stage consumed in step j - 1
        asm volatile("cp.async.wait_group %0;" ::"n"(XW_S - 1));
        __syncwarp();
        const XwStage& st = ring[j % XW_S];
#pragma unroll 2
        for (int r = 0; r < XW_RW; ++r) {
            const float4 p0 = *reinterpret_cast<const float4*>(&st.p[r][4 * ig]);
            const float4 p1 = *reinterpret_cast<const float4*>(&st.p[r][16 + 4 * ig]);
            const float4 y0 = *reinterpret_cast<const float4*>(&st.y[r][4 * dg]);
            const float4 y1 = *reinterpret_cast<const float4*>(&st.y[r][32 + 4 * dg]);
            const unsigned long long yp[4] = {f2pack(y0.x, y0.y), f2pack(y0.z, y0.w), f2pack(y1.x, y1.y),
                                              f2pack(y1.z, y1.w)};
            const float pa[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const unsigned long long pu = f2pack(pa[u], pa[u]);
#pragma unroll
                for (int v = 0; v < 4; ++v) asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[u][v]) : "l"(pu), "l"(yp[v]));
            }
        }
        __syncwarp();  // every lane has read the stage before it is refilled
    }
    asm volatile("cp.async.wait_group 0;");
    __syncwarp();
    // this warp's partial tile into its own ring, then the sum over warps in warp order
    float* red = reinterpret_cast<float*>(ring);
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            float a0, a1, a2, a3;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(acc[u][2 * b]));
            asm("mov.b64 {%0, %1}, %2;" : "=f"(a2), "=f"(a3) : "l"(acc[u][2 * b + 1]));
            const int i = 16 * (u >> 2) + 4 * ig + (u & 3);
            *reinterpret_cast<float4*>(&red[i * XW_RED + 32 * b + 4 * dg]) = make_float4(a0, a1, a2, a3);
        }
    __syncthreads();
    float* out = xpart + q * (int64_t)m * d;
    const float* red0 = reinterpret_cast<const float*>(xw_raw);
    constexpr int WSTRIDE = (int)(sizeof(XwStage) * XW_S / 4);  // floats between two warps' rings
    for (int f = tid; f < 32 * 16; f += XW_WARPS * 32) {
        const int i = f >> 4, c = f & 15;
        if (i0 + i >= m || c >= ny4) continue;
        float4 s = *reinterpret_cast<const float4*>(&red0[i * XW_RED + c * 4]);
#pragma unroll
        for (int v = 1; v < XW_WARPS; ++v) {
            const float4 t = *reinterpret_cast<const float4*>(&red0[v * WSTRIDE + i * XW_RED + c * 4]);
            s.x += t.x;
            s.y += t.y;
            s.z += t.z;
            s.w += t.w;
        }
        *reinterpret_cast<float4*>(out + (int64_t)(i0 + i) * d + d0 + c * 4) = s;
    }
}



// Reads the autotuner's event pairs (synchronises the stream), averages them
// per candidate and keeps the fastest launch shape in the context.
static int d2_tune_finish(d2_ctx* ctx, int m, const std::vector<SweepCand>& cands,
                          const std::vector<cudaEvent_t>& tev, const std::vector<int>& tev_cand,
                          cudaStream_t st) {
    if (cands.empty() || tev_cand.empty()) return D2_OK;
    D2_CK(ctx, cudaStreamSynchronize(st));
    SweepTune t;
    t.m = m;
    t.ncand = (int)cands.size();
    std::vector<double> sum(cands.size(), 0.0);
    std::vector<int> cnt(cands.size(), 0);
    for (size_t i = 0; i < tev_cand.size(); ++i) {
        float ms = 0.f;
        D2_CK(ctx, cudaEventElapsedTime(&ms, tev[2 * i], tev[2 * i + 1]));
        sum[tev_cand[i]] += ms;
        cnt[tev_cand[i]]++;
    }
    double best = 1e300;
    for (int i = 0; i < t.ncand; ++i) {
        t.ms[i] = cnt[i] ? (float)(sum[i] / cnt[i]) : 0.f;
        t.shape[i][0] = cands[i].kind;
        t.shape[i][1] = cands[i].lpr;
        t.shape[i][2] = cands[i].nv;
        t.shape[i][3] = cands[i].per_sm;
        if (cnt[i] && sum[i] / cnt[i] < best) {
            best = sum[i] / cnt[i];
            t.chosen = i;
        }
    }
    if (t.chosen < 0) return D2_OK;
    t.fn = reinterpret_cast<const void*>(cands[t.chosen].fn);
    t.smem = cands[t.chosen].smem;
    t.per_sm = cands[t.chosen].per_sm;
    ctx->tuned.push_back(t);
    return D2_OK;
}

// ---------------------------------------------------------------------------
// split calls: two halves of the clusters on two streams (D2_SPLIT_STREAMS)
// ---------------------------------------------------------------------------

__global__ void k_rebase_offsets(const int64_t* src, int64_t cnt, int64_t* dst) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < cnt) dst[t] = src[t] - src[0];
}

// Runs clusters [0, K1) and [K1, K) (K1: half the members) as two calls in the
// child contexts on their own streams; *done = false when the call should run
// as one (fewer than two clusters, a capturing stream, offsets not from 0).
static int badmm_split(d2_ctx* ctx, const d2_bags* bags, const int64_t* cofs, const int64_t* members, int64_t P,
                       int32_t K, int32_t m, float* x, float* w, float* plan, const uint8_t* warm_mask,
                       const d2_badmm_opts& opts, double* obj, cudaStream_t st, bool* done) {
    *done = false;
    if (K < 2) return D2_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return D2_OK;
    }
    if (cap != cudaStreamCaptureStatusNone) return D2_OK;
    std::vector<int64_t> hc((size_t)K + 1);
    D2_CK(ctx, cudaMemcpyAsync(hc.data(), cofs, ((size_t)K + 1) * 8, cudaMemcpyDeviceToHost, st));
    D2_CK(ctx, cudaStreamSynchronize(st));
    if (hc[0] != 0 || hc[K] != P) return D2_OK;
    int K1 = (int)(std::lower_bound(hc.begin(), hc.end(), P / 2) - hc.begin());
    K1 = std::max(1, std::min(K - 1, K1));
    const int64_t P1 = hc[K1];
    if (P1 <= 0 || P1 >= P) return D2_OK;
    for (int h = 0; h < 2; ++h) {
        if (!ctx->child[h]) {
            ctx->child[h] = d2_create(ctx->device);
            if (!ctx->child[h]) return d2_fail(ctx, D2_ENOMEM, "badmm_barycenter: cannot create a child context");
            D2_CK(ctx, cudaStreamCreateWithFlags(&ctx->cstream[h], cudaStreamNonBlocking));
        }
    }
    for (int e = 0; e < 3; ++e)
        if (!ctx->cev[e]) D2_CK(ctx, cudaEventCreateWithFlags(&ctx->cev[e], cudaEventDisableTiming));
    // the per-entry arrays are indexed by global support row: the halves touch
    // disjoint rows, so both children use this context's arrays
    const size_t ent = (size_t)bags->n * m * 4;
    void* pv = nullptr;
    int rc;
    if ((rc = d2_ws(ctx, WS_LAM, ent, &pv))) return rc;
    if ((rc = d2_ws(ctx, WS_COST, ent, &pv))) return rc;
    for (int h = 0; h < 2; ++h) {
        d2_ctx* c = ctx->child[h];
        for (int slot : {(int)WS_LAM, (int)WS_COST}) {
            if (!((c->borrowed >> slot) & 1u) && c->ws[slot]) {
                cudaDeviceSynchronize();
                cudaFree(c->ws[slot]);
            }
            c->borrowed |= 1u << slot;
            if (c->ws[slot] != ctx->ws[slot] || c->ws_bytes[slot] != ctx->ws_bytes[slot]) {
                c->ws[slot] = ctx->ws[slot];
                c->ws_bytes[slot] = ctx->ws_bytes[slot];
                c->generation++;  // graphs captured with the old pointers are stale
            }
        }
        c->timing = ctx->timing;
        if (!find_tune(c, m)) {
            const SweepTune* t = find_tune(ctx, m);
            if (t) c->tuned.push_back(*t);
        }
    }
    void* vs = nullptr;
    if ((rc = d2_ws(ctx, WS_SPLIT, ((size_t)K - K1 + 1) * 8, &vs))) return rc;
    int64_t* cofs2 = static_cast<int64_t*>(vs);
    k_rebase_offsets<<<(unsigned)d2_ceil_div(K - K1 + 1, 256), 256, 0, st>>>(cofs + K1, K - K1 + 1, cofs2);
    D2_LAUNCH_CK(ctx, "k_rebase_offsets");
    D2_CK(ctx, cudaEventRecord(ctx->cev[0], st));
    for (int h = 0; h < 2; ++h) D2_CK(ctx, cudaStreamWaitEvent(ctx->cstream[h], ctx->cev[0], 0));
    d2_badmm_opts o = opts;
    o.flags &= ~(D2_SPLIT_STREAMS | D2_VALIDATE);
    const int64_t l0 = ctx->child[0]->launches + ctx->child[1]->launches;
    const int d = bags->d;
    rc = badmm_barycenter(ctx->child[0], bags, cofs, members, P1, K1, m, x, w, plan, warm_mask, &o, obj,
                          ctx->cstream[0]);
    if (rc == D2_OK)
        rc = badmm_barycenter(ctx->child[1], bags, cofs2, members + P1, P - P1, K - K1, m,
                              x + (size_t)K1 * m * d, w + (size_t)K1 * m, plan, warm_mask, &o, obj + K1,
                              ctx->cstream[1]);
    // join: the caller's stream waits for both halves
    cudaEventRecord(ctx->cev[1], ctx->cstream[0]);
    cudaEventRecord(ctx->cev[2], ctx->cstream[1]);
    cudaStreamWaitEvent(st, ctx->cev[1], 0);
    cudaStreamWaitEvent(st, ctx->cev[2], 0);
    ctx->launches += ctx->child[0]->launches + ctx->child[1]->launches - l0;
    if (!find_tune(ctx, m)) {
        const SweepTune* t = find_tune(ctx->child[0], m);
        if (t) ctx->tuned.push_back(*t);
    }
    if (rc != D2_OK) {
        const d2_ctx* bad = ctx->child[0]->err.empty() ? ctx->child[1] : ctx->child[0];
        return d2_fail(ctx, rc, "%s", bad->err.c_str());
    }
    *done = true;
    return D2_OK;
}

// ---------------------------------------------------------------------------
// entry point
// ---------------------------------------------------------------------------

// Algorithm badmm for coordinate supports (x, csym NULL) or fixed symbolic
// supports (csym, x NULL: costs from the bags' symbol table, no support
// update).
static int badmm_impl(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets, const int64_t* members,
                      int64_t P, int32_t K, int32_t m, float* x, const int32_t* csym, float* w, float* plan,
                      const uint8_t* warm_mask, const d2_badmm_opts* opts_in, double* obj, void* stream);

extern "C" int badmm_barycenter(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets,
                                const int64_t* members, int64_t P, int32_t K, int32_t m, float* x,
                                float* w, float* plan, const uint8_t* warm_mask, const d2_badmm_opts* opts_in,
                                double* obj, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (!x) return d2_fail(ctx, D2_EINVAL, "badmm_barycenter: x is NULL");
    return badmm_impl(ctx, bags, cluster_offsets, members, P, K, m, x, nullptr, w, plan, warm_mask, opts_in, obj,
                      stream);
}

extern "C" int badmm_barycenter_sym(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets,
                                    const int64_t* members, int64_t P, int32_t K, int32_t m, const int32_t* csym,
                                    float* w, float* plan, const uint8_t* warm_mask, const d2_badmm_opts* opts_in,
                                    double* obj, void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_sym_bags_host(ctx, bags);
    if (rc) return rc;
    if (!csym) return d2_fail(ctx, D2_EINVAL, "badmm_barycenter_sym: csym is NULL");
    d2_badmm_opts o;
    if (opts_in) o = *opts_in; else d2_badmm_opts_default(&o);
    o.flags |= D2_FIX_X;
    o.flags &= ~(D2_SPLIT_STREAMS | D2_COST_BF16X6 | D2_SUPPORT_TC | D2_COST_ROWS);
    return badmm_impl(ctx, bags, cluster_offsets, members, P, K, m, nullptr, csym, w, plan, warm_mask, &o, obj,
                      stream);
}

static int badmm_impl(d2_ctx* ctx, const d2_bags* bags, const int64_t* cluster_offsets, const int64_t* members,
                      int64_t P, int32_t K, int32_t m, float* x, const int32_t* csym, float* w, float* plan,
                      const uint8_t* warm_mask, const d2_badmm_opts* opts_in, double* obj, void* stream) {
    int rc = D2_OK;
    d2_badmm_opts opts;
    if (opts_in) opts = *opts_in; else d2_badmm_opts_default(&opts);
    if (K < 1 || m < 1 || m > 256 || P < 0 || !cluster_offsets || (P > 0 && !members) || !w || !plan)
        return d2_fail(ctx, D2_EINVAL, "badmm_barycenter: need K >= 1, 1 <= m <= 256 and non-NULL arrays");
    if (opts.iters < 1 || opts.tau < 1 || !(opts.eps >= 0.0) || !(opts.rho0 > 0.0) ||
        (opts.rule != D2_RULE_R1 && opts.rule != D2_RULE_R2))
        return d2_fail(ctx, D2_EINVAL, "badmm_barycenter: need iters >= 1, tau >= 1, eps >= 0, rho0 > 0, rule R1/R2");
    if ((reinterpret_cast<uintptr_t>(plan) & 15) || (reinterpret_cast<uintptr_t>(x) & 3))
        return d2_fail(ctx, D2_EINVAL, "badmm_barycenter: plan must be 16-byte aligned");
    cudaStream_t st = d2_stream(stream);
    if (opts.flags & D2_VALIDATE) {
        rc = d2_check_bags(ctx, bags, stream);
        if (rc) return rc;
    }
    if (P == 0) {
        if (ctx->reducer)  // the other processes would wait in the reductions
            return d2_fail(ctx, D2_EINVAL, "badmm_barycenter: with a reducer every process needs members");
        return D2_OK;
    }
    if (ctx->reducer) opts.flags &= ~D2_SPLIT_STREAMS;  // one call on one stream per process
    if (opts.flags & D2_SPLIT_STREAMS) {
        bool done = false;
        rc = badmm_split(ctx, bags, cluster_offsets, members, P, K, m, x, w, plan, warm_mask, opts, obj, st, &done);
        if (rc || done) return rc;
        opts.flags &= ~D2_SPLIT_STREAMS;
    }
    const int d = csym ? 1 : bags->d;
    const int64_t n = bags->n;

    // workspaces
    ClusterWs cw;
    rc = d2_cluster_ws(ctx, K, m, d, P, &cw);
    if (rc) return rc;
    void *vlam, *vcost, *vr, *vpart, *vobj, *vxp;
    if ((rc = d2_ws(ctx, WS_LAM, (size_t)n * m * 4, &vlam))) return rc;
    if ((rc = d2_ws(ctx, WS_COST, (size_t)n * m * 4, &vcost))) return rc;
    if ((rc = d2_ws(ctx, WS_POS_R, (size_t)P * m * 4, &vr))) return rc;
    if ((rc = d2_ws(ctx, WS_POS_PART, (size_t)P * m * 4, &vpart))) return rc;
    if ((rc = d2_ws(ctx, WS_POS_OBJ, (size_t)P * 8, &vobj))) return rc;
    const int64_t maxch = d2_ceil_div(P, D2_CHUNK) + K + 1;
    const bool fix_x = opts.flags & D2_FIX_X, fix_w = opts.flags & D2_FIX_W;
    if (!fix_x) {
        if ((rc = d2_ws(ctx, WS_XPART, (size_t)maxch * m * d * 4, &vxp))) return rc;
    }
    const bool need_sums = !(opts.rho > 0.0);
    // exact reductions: global member counts (K + 1), consensus sums (K m),
    // scratch for the rho / support / objective sums
    const size_t fx_scratch = std::max<size_t>((size_t)3 * K, fix_x ? 0 : (size_t)K + (size_t)K * m * d);
    void* vfx = nullptr;
    if ((rc = d2_ws(ctx, WS_FIXED, ((size_t)K + 1 + (size_t)K * m + fx_scratch) * 8, &vfx))) return rc;
    void *vpc = nullptr, *vcs = nullptr;
    if ((rc = d2_ws(ctx, WS_POS_CLUSTER, (size_t)std::max<int64_t>(P, 1) * 4, &vpc))) return rc;
    if (need_sums && (rc = d2_ws(ctx, WS_CHUNK_SUM, (size_t)maxch * 16, &vcs))) return rc;
    const int cost_prec = csym ? 0 : d2_cost_prec(opts.flags);
    const bool use_vt = !csym && d2_vocab_table_applies(bags, K, m, cost_prec, opts.flags);
    if (use_vt && (rc = d2_vocab_reserve(ctx, bags, K, m, cw))) return rc;
    // the cluster workspace may have moved while growing the others
    rc = d2_cluster_ws(ctx, K, m, d, P, &cw);
    if (rc) return rc;
    if (!csym && (rc = d2_cost_prepare(ctx, bags, m, cost_prec))) return rc;
    // the support update on the tensor cores only when asked for: measured
    // slower than the FP32 CUDA-core partials (its transposing BF16-piece
    // conversion issues more instructions per row than the FMAs it replaces)
    const bool xp_tc = !fix_x && (opts.flags & D2_SUPPORT_TC) && d2_support_tc_applies(bags, m, cost_prec);
    if (xp_tc && (rc = d2_support_tc_prepare(ctx, bags, m, cost_prec))) return rc;
    int32_t* pos_cluster = static_cast<int32_t*>(vpc);
    double* chunk_sum = need_sums ? static_cast<double*>(vcs) : nullptr;
    int64_t* chunk_rows = need_sums ? reinterpret_cast<int64_t*>(static_cast<char*>(vcs) + (size_t)maxch * 8) : nullptr;
    float* lam = static_cast<float*>(vlam);
    float* cost = static_cast<float*>(vcost);
    int64_t* gcount = static_cast<int64_t*>(vfx);
    long long* cons_sum = reinterpret_cast<long long*>(gcount + K + 1);
    long long* fx = cons_sum + (size_t)K * m;

    SweepArgs sa;
    sa.members = members;
    sa.pos_cluster = pos_cluster;
    sa.P = P;
    sa.offsets = bags->offsets;
    sa.wt = bags->wt;
    sa.plan = plan;
    sa.lam = lam;
    sa.cost = cost;
    sa.pos_r = static_cast<float*>(vr);
    sa.pos_part = static_cast<float*>(vpart);
    sa.pos_obj = static_cast<double*>(vobj);
    sa.beta = cw.beta;
    sa.rho = cw.rho;
    sa.counters = cw.counters;
    sa.cofs = cluster_offsets;
    sa.warm_mask = warm_mask;
    sa.m = m;
    sa.eps = (float)opts.eps;
    sa.log2eps = opts.eps > 0.0 ? (float)log2(opts.eps) : -INFINITY;
    sa.w_next64 = cw.w64;
    const int rflag = (opts.rule == D2_RULE_R2) ? SW_R2 : 0;
    size_t sweep_smem = 0;
    SweepFn sweep = nullptr;
    int dev_sms = 152, per_sm = 1;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const SweepTune* tuned = (opts.flags & D2_NO_PIPE) ? nullptr : find_tune(ctx, m);
    if (tuned) {  // launch shape chosen earlier by the autotuner
        sweep = reinterpret_cast<SweepFn>(const_cast<void*>(tuned->fn));
        sweep_smem = tuned->smem;
        per_sm = tuned->per_sm;
    } else {
        if (!(opts.flags & D2_NO_PIPE)) sweep = pick_sweep_pipe(m, &sweep_smem);
        if (!sweep) {
            sweep = pick_sweep(m);
            sweep_smem = 0;
        }
    }
    // (the shared-memory attribute must be set before the occupancy query)
    if (sweep_smem > 48 * 1024)
        D2_CK(ctx, cudaFuncSetAttribute(sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_smem));
    if (!tuned) {
        // persistent grid: as many CTAs as fit on the device at once
        D2_CK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep, SWEEP_THREADS, sweep_smem));
        if (per_sm < 1) per_sm = 1;
    }
    const unsigned grid = (unsigned)std::min<int64_t>(d2_ceil_div(P, SWEEP_WARPS), (int64_t)dev_sms * per_sm);
    // autotuning: the first fused passes cycle through the candidates
    const bool tuning = (opts.flags & D2_AUTOTUNE) && !(opts.flags & D2_NO_PIPE) && !tuned;
    std::vector<SweepCand> cands;
    std::vector<cudaEvent_t> tev;
    std::vector<int> tev_cand;
    int fused_seen = 0, tune_reps = 0;
    if (tuning) {
        if ((rc = sweep_candidates(ctx, m, &cands))) return rc;
        const int fused_total = std::max(0, opts.iters - 1 - (fix_x ? 0 : (opts.iters - 1) / opts.tau));
        tune_reps = cands.empty() ? 0 : std::min(3, fused_total / (int)cands.size());
    }
    const int T = opts.iters, tau = opts.tau;
    // the d % 4 == 0 and m % 4 == 0 path copies 16-byte slices of plan and y rows
    const int64_t xw_blocks = maxch * d2_ceil_div(d, 64) * d2_ceil_div(m, 32);
    const bool xp_pipe = (d % 4 == 0) && (m % 4 == 0) && xw_blocks < ((int64_t)1 << 31) &&
        ((reinterpret_cast<uintptr_t>(bags->supp ? bags->supp : bags->vocab) & 15) == 0) &&
        ((reinterpret_cast<uintptr_t>(plan) & 15) == 0);
    if (xp_pipe && !fix_x)
        D2_CK(ctx, cudaFuncSetAttribute(k_xpartial_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XW_SMEM));

  auto enqueue = [&]() -> int {
    int rc = D2_OK;
    if ((rc = d2_setup_clusters(ctx, cluster_offsets, P, K, &pos_cluster, &cw, st))) return rc;
    if ((rc = d2_fx_counts(ctx, K, cluster_offsets, gcount, st))) return rc;
    D2_CK(ctx, cudaMemsetAsync(cons_sum, 0, (size_t)K * m * sizeof(long long), st));
    D2_CK(ctx, cudaMemsetAsync(cw.counters, 0, (size_t)K * 4, st));
    D2_CK(ctx, cudaMemcpyAsync(cw.wb[0], w, (size_t)K * m * 4, cudaMemcpyDeviceToDevice, st));
    // initial cost and rho (Eq. rho)
    if (csym) {
        if ((rc = d2_sym_cost_rows(ctx, bags, members, P, K, m, csym, cw, cost, chunk_sum, chunk_rows, st))) return rc;
    } else {
        if ((rc = d2_prep_x(ctx, x, K, m, d, cw, st))) return rc;
        if ((rc = d2_cost_rows(ctx, bags, members, P, K, m, cw, cost, need_sums, cost_prec,
                               use_vt ? D2_VT_SETUP : D2_VT_OFF, st)))
            return rc;
    }
    if ((rc = d2_fx_rho(ctx, K, m, cw.chunk_first, chunk_sum, chunk_rows, gcount, opts.rho0, opts.rho, cw.rho,
                        cw.beta, cw.nrows, fx, st)))
        return rc;

    auto launch = [&](int flags, const float* wcur, float* wnext) -> int {
        SweepArgs s = sa;
        s.flags = flags | rflag;
        s.w_cur = wcur;
        s.w_next = fix_w ? nullptr : wnext;
        const bool fused = (flags & SW_A) && (flags & SW_B);
        d2_time_begin(ctx, fused ? D2_KT_SWEEP_FUSED : D2_KT_SWEEP_HALF, st);
        if (fused && fused_seen < (int)cands.size() * tune_reps) {
            const SweepCand& cd = cands[fused_seen % cands.size()];
            const unsigned g = (unsigned)std::min<int64_t>(d2_ceil_div(P, SWEEP_WARPS), (int64_t)dev_sms * cd.per_sm);
            cudaEvent_t e0, e1;
            D2_CK(ctx, cudaEventCreate(&e0));
            D2_CK(ctx, cudaEventCreate(&e1));
            tev.push_back(e0);
            tev.push_back(e1);
            tev_cand.push_back(fused_seen % (int)cands.size());
            D2_CK(ctx, cudaEventRecord(e0, st));
            cd.fn<<<g, SWEEP_THREADS, cd.smem, st>>>(s);
            D2_CK(ctx, cudaEventRecord(e1, st));
        } else {
            sweep<<<grid, SWEEP_THREADS, sweep_smem, st>>>(s);
        }
        if (fused) ++fused_seen;
        d2_time_end(ctx, st);
        D2_LAUNCH_CK(ctx, "k_sweep");
        if ((flags & SW_A) && s.w_next) {
            d2_time_begin(ctx, D2_KT_OTHER, st);
            const int crc = d2_fx_consensus(ctx, K, m, cw.chunks, cw.nchunks, maxch, sa.pos_part, rflag != 0, gcount,
                                            cons_sum, s.w_next, cw.w64, st);
            d2_time_end(ctx, st);
            if (crc) return crc;
        }
        return D2_OK;
    };
    auto wbuf = [&](int n) -> float* { return fix_w ? cw.wb[0] : cw.wb[n & 1]; };

    // n = 0: A step from Pi2^0 (cold w_i w_j^(k) or the cached plan), Lambda = 0
    if ((rc = launch(SW_A | SW_LAM_ZERO | SW_COLD | (T == 1 ? SW_OBJ : 0), wbuf(0), wbuf(1)))) return rc;
    bool lam_valid = false;
    for (int it = 1; it < T; ++it) {
        const int objf = (it == T - 1) ? SW_OBJ : 0;
        const int lamz = lam_valid ? 0 : SW_LAM_ZERO;
        if (!fix_x && it % tau == 0) {
            // B step alone: Pi2^n into the plan buffer, Lambda^n
            if ((rc = launch(SW_B | SW_LAM_OUT | lamz, wbuf(it), nullptr))) return rc;
            lam_valid = true;
            // Eq. (updatex) with Pi2^n and w^n, then the new cost
            dim3 g((unsigned)maxch, (unsigned)d2_ceil_div(d, XU_DT), (unsigned)d2_ceil_div(m, XU_MT));
            d2_time_begin(ctx, D2_KT_SUPPORT, st);
            if (xp_tc) {
                if ((rc = d2_support_tc(ctx, bags, members, maxch, m, cost_prec, plan, cw, static_cast<float*>(vxp),
                                        st)))
                    return rc;
            } else if (xp_pipe) {
                const int ntd = d2_ceil_div(d, 64), ntiles = ntd * d2_ceil_div(m, 32);
                k_xpartial_warp<<<(unsigned)(maxch * ntiles), XW_WARPS * 32, XW_SMEM, st>>>(
                    members, bags->offsets, bags->supp, bags->vocab_idx, bags->vocab, d, m, plan, cw.chunks,
                    cw.nchunks, ntd, ntiles, static_cast<float*>(vxp));
            } else {
                k_xpartial<<<g, XU_THREADS, 0, st>>>(members, bags->offsets, bags->supp, bags->vocab_idx,
                                                      bags->vocab, d, m, plan, cw.chunks, cw.nchunks,
                                                      static_cast<float*>(vxp));
            }
            D2_LAUNCH_CK(ctx, "k_xpartial");
            rc = d2_fx_support(ctx, K, m, d, cw.chunk_first, maxch, static_cast<float*>(vxp), gcount, wbuf(it),
                               xp_tc ? cw.mu : nullptr, x, fx, st);
            d2_time_end(ctx, st);
            if (rc) return rc;
            if ((rc = d2_prep_x(ctx, x, K, m, d, cw, st))) return rc;
            if ((rc = d2_cost_rows(ctx, bags, members, P, K, m, cw, cost, false, cost_prec,
                                   use_vt ? D2_VT_REUSE : D2_VT_OFF, st)))
                return rc;
            // A step from Pi2^n
            if ((rc = launch(SW_A | objf, wbuf(it), wbuf(it + 1)))) return rc;
        } else {
            if ((rc = launch(SW_B | SW_A | SW_LAM_OUT | lamz | objf, wbuf(it), wbuf(it + 1)))) return rc;
            lam_valid = true;
        }
    }
    // final B step: Pi2^T into the plan buffer (Lambda^T is not needed)
    if ((rc = launch(SW_B | (lam_valid ? 0 : SW_LAM_ZERO), wbuf(T), nullptr))) return rc;
    return d2_fx_finish(ctx, K, m, cluster_offsets, sa.pos_obj, gcount, wbuf(T), w, obj, fx, st);
  };

    // Replay the whole launch sequence as one CUDA graph when possible: on a
    // non-default stream that is not itself being captured, with per-launch
    // timing off.  The graph is rebuilt whenever anything it bakes in changes
    // (pointers, sizes, options, workspace placement).
    if (tuning) {  // direct launches; read the candidates' times and keep the fastest
        rc = enqueue();
        if (rc == D2_OK) rc = d2_tune_finish(ctx, m, cands, tev, tev_cand, st);
        for (auto e : tev) cudaEventDestroy(e);
        return rc;
    }
    const bool want_graph = !(opts.flags & D2_NO_GRAPH) && !ctx->timing && st != nullptr && !ctx->reducer;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (want_graph && cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return enqueue();
    }
    if (!want_graph || cap != cudaStreamCaptureStatusNone) return enqueue();
    auto u = [](const void* p) { return (uint64_t)reinterpret_cast<uintptr_t>(p); };
    uint64_t rho_bits, rho0_bits, eps_bits;
    memcpy(&rho_bits, &opts.rho, 8);
    memcpy(&rho0_bits, &opts.rho0, 8);
    memcpy(&eps_bits, &opts.eps, 8);
    const std::vector<uint64_t> key = {
        (uint64_t)ctx->generation, (uint64_t)bags->N, (uint64_t)bags->n, (uint64_t)bags->d, (uint64_t)bags->max_mk,
        u(bags->offsets), u(bags->supp), u(bags->vocab_idx), u(bags->vocab), (uint64_t)bags->V, u(bags->wt),
        u(cluster_offsets), u(members), (uint64_t)P, (uint64_t)K, (uint64_t)m, u(x), u(csym), u(bags->symcost),
        u(w), u(plan),
        u(warm_mask), u(obj), rho_bits, rho0_bits, eps_bits, (uint64_t)opts.iters, (uint64_t)opts.tau,
        (uint64_t)opts.rule, (uint64_t)opts.flags, u(reinterpret_cast<const void*>(sweep)), (uint64_t)per_sm};
    if (ctx->graph_exec && ctx->graph_key == key) {
        D2_CK(ctx, cudaGraphLaunch(ctx->graph_exec, st));
        ctx->launches += ctx->graph_launches;
        return D2_OK;
    }
    const int64_t l0 = ctx->launches;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return enqueue();
    }
    const int rc_cap = enqueue();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc_cap == D2_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    const int64_t nl = ctx->launches - l0;
    ctx->launches = l0;
    if (rc_cap != D2_OK || e != cudaSuccess || !exec) {  // capture refused: launch directly
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        return enqueue();
    }
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = exec;
    ctx->graph_key = key;
    ctx->graph_launches = nl;
    D2_CK(ctx, cudaGraphLaunch(exec, st));
    ctx->launches += nl;
    return D2_OK;
}
