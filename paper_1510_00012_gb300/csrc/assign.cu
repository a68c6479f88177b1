// Exact W^2 (the transportation LP of Eq. primal) for many (centroid, bag)
// pairs, and the assignment step of Algorithm 1 (argmin over centroids).
//
// One warp solves one pair with successive shortest paths on the residual
// bipartite graph (sources: the m centroid points with supplies w_i; sinks:
// the m_k bag points with demands w_j^(k)).  Node potentials keep every
// residual arc's reduced cost non-negative, so each phase is a dense Dijkstra
// (warp argmin over unvisited nodes, lanes relax one node's arcs in
// parallel) from all sources with remaining supply to the nearest sink with
// remaining demand (for problems of more than 64 nodes: until 4 such sinks
// are settled), followed by augmentations of the largest feasible amount
// along the shortest path to each (after the potential update every such
// path is tight).  Reduced-cost optimality holds throughout, so the final
// flow is optimal; unlike a simplex there are no degenerate pivots.  Start:
// pot_i = 0, pot_j = min_i C_ij and every sink sends what it can to its
// cheapest source (those arcs have zero reduced cost).  Costs, flows and
// potentials are FP32; the final cost sum_ij f_ij C_ij is accumulated in FP64.
//
// Flow storage.  Only the cost tableau needs dense random access: the
// shortest-path passes read whole cost rows and columns but ask of the flow
// only whether a backward arc exists.  The sparse store keeps, per bag point
// j, a bitmask of the centroid points with flow above tol into it, and the
// nonzero flows themselves in a small pool of entries linked per bag point
// (lane 0 alone edits it, during the greedy start and the augmentations).  A
// transportation flow built along shortest paths has about m + m_k - 1
// nonzeros; degenerate costs can add cycles, so a pair whose pool overflows
// is put on a list and solved again by the dense store afterwards.  Both
// stores do the same arithmetic in the same order, so a pair's flow does not
// depend on the store; only the order of the final FP64 sum differs.
#include <algorithm>
#include <cstring>

#include "d2_internal.cuh"

#define AS_DC 8        // support dimensions staged per step of the cost build
#define AS_INF 3.0e38f
// deficit sinks collected per shortest-path pass: one for problems of <= 64
// nodes (measured faster), else 4, or 8 with >= 64 centroid points
// (measured on one GPU: 8 is 5-7 % faster than 4 on 64 x 10..60 problems and
// 5 % slower on 32 x 16..64 ones; 4 halves the passes of one)
__device__ __forceinline__ int as_kt(int m, int V) { return V <= 64 ? 1 : m >= 64 ? 8 : 4; }

struct AssignArgs {
    const int64_t* offsets;
    const float* supp;
    const int32_t* vidx;
    const float* vocab;
    const float* wt;
    int d;
    const float* x;    // K x m x d (NULL for symbolic supports)
    const float* w;    // K x m
    // symbolic supports (Section 5): cost C_ij = symcost[csym[cent m + i] * V + vidx[row j]]
    const float* symcost;      // V x V, or NULL
    const int32_t* csym;       // K x m centroid symbols
    int64_t V;
    int m, K, nmax;
    int nlo;                   // this launch solves only bags with nlo < m_k <= nmax
    // pair enumeration
    int mode;                  // 0: all N*K pairs; 1: explicit list; 2: all K for listed bags;
                               // 3: r candidates per bag (bag p / r, centroid cand[p]);
                               // 4: explicit list with output slots (re-solves)
    int64_t npairs;            // mode 0/1 host count (mode 1: upper bound if npairs_dev)
    const int64_t* npairs_dev; // mode 1/2: device count (pairs, or bags for mode 2)
    const int64_t* pair_bag;   // mode 1
    const int32_t* pair_cent;  // mode 1
    const int64_t* bag_list;   // mode 2
    const int32_t* cand;       // mode 3
    int r;                     // mode 3
    float* out;                // mode 0/2: out[bag*K + cent]; mode 1: out[pair]; mode 4: out[pair_slot[p]]
    const int64_t* pair_slot;  // mode 4 (with pair_bag, pair_cent, npairs_dev)
    // pairs whose sparse flow pool overflowed, solved again by the dense store
    int64_t* ovf_bag;
    int32_t* ovf_cent;
    int64_t* ovf_slot;
    int64_t* ovf_cnt;
    int64_t ovf_cap;
    int pool_cap;              // > 0: fewer sparse pool entries than the layout's (testing)
    int* flags;
    int64_t* pivot_fail;       // count of pairs that hit the phase limit
    int max_phase;
    size_t warp_bytes;
};

// Per-warp shared memory (byte offsets from the warp's slice), for bags of
// at most ncap points: the cost tableau (m x ns floats, ns = ncap | 1); the
// flow store (dense: an m x ns tableau; sparse: E pool flows, the per-point
// bitmasks (ncap x MW words), the pool list heads and links); the initial
// potentials and excesses (moved to registers once the greedy start is done);
// the predecessor of every node; the cost-build staging (AS_DC x (m + ncap)
// floats), which shares the flow store's space when it fits there, since the
// flows are initialised only after the cost is built.
struct WarpLayout {
    size_t c, f, ef, mask, head, enext, esrc, pot, exc, pred, xs, ys, bytes;
    int E, MW;
};
__host__ __device__ inline size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }
// Node numbering: centroid point i is node i (i < m); bag point j is node
// B + j with B = 32 ceil(m / 32), so that a lane's register slots t < B / 32
// hold sources only and slots t >= B / 32 sinks only; nodes m .. B - 1 do not
// exist.  Valid nodes keep their relative order (ties resolve as with nodes
// numbered 0 .. m + n - 1).
__host__ __device__ inline int sink_base(int m) { return 32 * ((m + 31) / 32); }

__host__ __device__ inline WarpLayout warp_layout(int m, int ncap, bool sparse) {
    WarpLayout L;
    const int ns = ncap | 1, V = sink_base(m) + ncap;  // node span
    L.MW = (m + 31) / 32;
    L.E = sparse ? 2 * (m + ncap) : 0;
    L.c = 0;
    size_t o = al16((size_t)m * ns * 4);
    L.f = L.ef = L.mask = L.head = L.enext = L.esrc = o;
    size_t store;
    if (!sparse) {
        store = (size_t)m * ns * 4;
    } else {
        L.ef = o;
        L.mask = L.ef + (size_t)L.E * 4;
        L.head = L.mask + (size_t)ncap * L.MW * 4;
        L.enext = L.head + (size_t)ncap * 2;
        L.esrc = L.enext + (size_t)L.E * 2;
        store = L.esrc + (size_t)L.E * 2 - o;
    }
    const size_t stage = (size_t)AS_DC * (m + ncap) * 4;
    const bool stage_inside = stage <= store;
    o = al16(o + store);
    L.pot = o;
    L.exc = L.pot + (size_t)V * 4;
    L.pred = L.exc + (size_t)V * 4;
    o = al16(L.pred + (size_t)V * 2);
    if (stage_inside) {
        L.xs = L.f;
    } else {
        L.xs = o;
        o = al16(o + stage);
    }
    L.ys = L.xs + (size_t)AS_DC * m * 4;
    L.bytes = o;
    return L;
}

// Per-warp shared memory views (see WarpLayout).
struct WarpMem {
    float* C;        // m x ns
    float* F;        // dense store: m x ns
    float* ef;       // sparse store: E flows
    unsigned* mask;  // sparse store: ncap x MW words; bit i of word (j, i / 32): flow (i, j) > tol
    short* head;     // sparse store: ncap list heads (-1: no entry)
    short* enext;    // sparse store: E links (also the free list)
    short* esrc;     // sparse store: E centroid points
    int E, MW;
    float* pot;      // V
    float* exc;      // V
    short* pred;     // V
    float* xs;       // AS_DC x m
    float* ys;       // AS_DC x n
};

// ---- sparse flow store (lane 0 only) ------------------------------------
// pool entry holding flow (i, j), or -1; *prev receives its predecessor in
// the list of j (-1: the head).  Walks are bounded by the pool size.
__device__ __forceinline__ int pool_find(const WarpMem& s, int i, int j, int* prev) {
    int pv = -1, k = s.head[j];
    for (int g = 0; g < s.E && (unsigned)k < (unsigned)s.E; ++g) {
        if (s.esrc[k] == i) {
            *prev = pv;
            return k;
        }
        pv = k;
        k = s.enext[k];
    }
    *prev = -1;
    return -1;
}
__device__ __forceinline__ void pool_bit(const WarpMem& s, int i, int j, bool on) {
    unsigned* wd = s.mask + j * s.MW + (i >> 5);
    const unsigned b = 1u << (i & 31);
    *wd = on ? (*wd | b) : (*wd & ~b);
}
// new entry (i, j) with flow 0 at the head of j's list, or -1 when the pool is full
__device__ __forceinline__ int pool_new(const WarpMem& s, int i, int j, int& fbump, int& ffree) {
    int k = -1;
    if (ffree >= 0) {
        k = ffree;
        ffree = s.enext[k];
    } else if (fbump < s.E) {
        k = fbump++;
    }
    if (k < 0) return -1;
    s.esrc[k] = (short)i;
    s.ef[k] = 0.f;
    s.enext[k] = s.head[j];
    s.head[j] = (short)k;
    return k;
}
__device__ __forceinline__ void pool_free(const WarpMem& s, int j, int k, int prev, int& ffree) {
    if (prev < 0) s.head[j] = s.enext[k];
    else s.enext[prev] = s.enext[k];
    s.enext[k] = (short)ffree;
    ffree = k;
}

__device__ __forceinline__ void warp_argmin(float& v, int& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov < v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
}

// Value of node v's register (slot v / 32 of owner lane v mod 32), broadcast.
// (a predicated move per slot, so that the array stays in registers)
template <int TV>
__device__ __forceinline__ float node_bcast(const float (&r)[TV], int v) {
    const int tv = v >> 5;
    float x = r[0];
#pragma unroll
    for (int t = 1; t < TV; ++t) asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %2, %3;\n\t@p mov.f32 %0, %1;\n\t}"
                                     : "+f"(x) : "f"(r[t]), "r"(t), "r"(tv));
    return __shfl_sync(0xffffffffu, x, v & 31);
}

// Solve one pair; returns W^2 (all lanes).  TV >= (m + n) / 32 node slots per
// lane; SP selects the sparse flow store, whose pool overflow sets `overflow`
// (the result is then invalid and the pair must be solved again densely).
template <int TV, bool SP>
__device__ double solve_pair(const AssignArgs& a, WarpMem& s, int64_t bag, int cent, bool& hit_limit,
                             bool& overflow) {
    const int lane = threadIdx.x & 31;
    const int m = a.m, d = a.d;
    const int64_t r0 = a.offsets[bag];
    const int n = (int)(a.offsets[bag + 1] - r0);
    const int V = m + n;                 // nodes
    const int SS = (m + 31) >> 5, B = SS << 5;
    const int VS = B + n;                // node span (sinks start at B)
    const float* xc = a.x ? a.x + (int64_t)cent * m * d : nullptr;

    // ---- cost C[i][j] = sum_dd (x_i - y_j)^2 by direct differences, or the
    // given symbol-to-symbol dissimilarity; tableau rows are ns = n | 1 floats
    // apart (odd: a column walk across rows touches distinct banks)
    const int ns = n | 1;
    if (a.symcost) {
        const int32_t* cs = a.csym + (int64_t)cent * m;
        for (int e = lane; e < m * ns; e += 32) {
            const int i = e / ns, j = e - i * ns;
            s.C[e] = j < n ? a.symcost[(int64_t)cs[i] * a.V + a.vidx[r0 + j]] : 0.f;
        }
    } else {
    for (int e = lane; e < m * ns; e += 32) s.C[e] = 0.f;
    for (int d0 = 0; d0 < d; d0 += AS_DC) {
        const int dc = min(AS_DC, d - d0);
        __syncwarp();
        for (int e = lane; e < dc * m; e += 32) {
            int t = e / m, i = e - t * m;
            s.xs[t * m + i] = xc[(int64_t)i * d + d0 + t];
        }
        for (int e = lane; e < dc * n; e += 32) {
            int t = e / n, j = e - t * n;
            s.ys[t * n + j] = d2_row_ptr(a.supp, a.vidx, a.vocab, d, r0 + j)[d0 + t];
        }
        __syncwarp();
        for (int e = lane; e < m * n; e += 32) {
            int i = e / n, j = e - i * n;
            float acc = s.C[i * ns + j];
            for (int t = 0; t < dc; ++t) {
                float df = s.xs[t * m + i] - s.ys[t * n + j];
                acc = fmaf(df, df, acc);
            }
            s.C[i * ns + j] = acc;
        }
    }
    }
    // ---- initial state
    int fbump = 0, ffree = -1;  // sparse pool allocator (lane 0)
    overflow = false;
    __syncwarp();  // the cost build's staging may share the flow store's space
    if (SP) {
        for (int e = lane; e < n * s.MW; e += 32) s.mask[e] = 0u;
        for (int j = lane; j < n; j += 32) s.head[j] = -1;
    } else {
        for (int e = lane; e < m * ns; e += 32) s.F[e] = 0.f;
    }
    for (int v = lane; v < VS; v += 32) {
        s.exc[v] = (v < m) ? a.w[(int64_t)cent * m + v] : (v >= B ? a.wt[r0 + (v - B)] : 0.f);
        s.pot[v] = 0.f;
    }
    __syncwarp();
    // pot_j = min_i C_ij; column-minimum argmin per sink (first minimum)
    for (int j = lane; j < n; j += 32) {
        float mn = AS_INF;
        int am = 0;
        for (int i = 0; i < m; ++i) {
            float c = s.C[i * ns + j];
            if (c < mn) {
                mn = c;
                am = i;
            }
        }
        s.pot[B + j] = mn;
        s.pred[B + j] = (short)am;
    }
    __syncwarp();
    bool gov = false;  // sparse pool full during the greedy start (only under a test cap)
    if (lane == 0) {
        for (int j = 0; j < n; ++j) {
            int i = s.pred[B + j];
            float f = fminf(s.exc[B + j], s.exc[i]);
            if (f > 0.f) {
                if (SP) {
                    const int k = pool_new(s, i, j, fbump, ffree);
                    if (k < 0) {
                        gov = true;
                        break;
                    }
                    s.ef[k] += f;
                    if (s.ef[k] > 1e-9f) pool_bit(s, i, j, true);  // the tol below
                } else {
                    s.F[i * ns + j] += f;
                }
                s.exc[B + j] -= f;
                s.exc[i] -= f;
            }
        }
    }
    __syncwarp();
    const float tol = 1e-9f;
    hit_limit = false;
    if (SP && __shfl_sync(0xffffffffu, (int)gov, 0)) {
        overflow = true;
        return 0.0;
    }
    // node state in registers: node v is owned by lane v mod 32, slot v / 32
    float pot[TV], exc[TV], dist[TV];
#pragma unroll
    for (int t = 0; t < TV; ++t) {
        const int v = lane + 32 * t;
        pot[t] = v < VS ? s.pot[v] : 0.f;
        exc[t] = v < VS ? s.exc[v] : 0.f;
    }
    int phase = 0;
    for (;;) {
        // anything left to route?
        bool src = false, snk = false;
#pragma unroll
        for (int t = 0; t < TV; ++t) {
            const int v = lane + 32 * t;
            if (v < VS && exc[t] > tol) {
                if (v < m) src = true; else snk = true;
            }
        }
        src = __any_sync(0xffffffffu, src);
        snk = __any_sync(0xffffffffu, snk);
        if (!src || !snk) break;
        if (++phase > a.max_phase) {
            hit_limit = true;
            break;
        }
        // ---- Dijkstra from every source with remaining supply
        unsigned vis = 0;  // bit t: node lane + 32 t is settled
#pragma unroll
        for (int t = 0; t < TV; ++t) {
            const int v = lane + 32 * t;
            dist[t] = (v < m && exc[t] > tol) ? 0.f : AS_INF;
            if (v < VS) s.pred[v] = -1;
        }
        // up to kt_max deficit sinks per pass (settled in order of distance);
        // the shortest paths to all of them become tight arcs after the
        // potential update, so flow is pushed along each (primal-dual step)
        int kt = 0, tgl = -1;  // lane q < kt holds the q-th target
        const int kt_max = as_kt(m, V);
        for (int it = 0; it < V; ++it) {  // at most one settled node per step
            // warp argmin over unsettled nodes: smallest distance, then lowest index
            float bv = AS_INF;
            int bi = 0x7fffffff;
#pragma unroll
            for (int t = 0; t < TV; ++t) {
                const int v = lane + 32 * t;
                if (v < VS && !((vis >> t) & 1u) && dist[t] < bv) {
                    bv = dist[t];
                    bi = v;
                }
            }
            // non-negative floats order like their bit patterns
            const unsigned kmin = __reduce_min_sync(0xffffffffu, __float_as_uint(bv));
            if (__uint_as_float(kmin) >= AS_INF) break;
            const int u = (int)__reduce_min_sync(0xffffffffu, __float_as_uint(bv) == kmin ? (unsigned)bi : 0xffffffffu);
            const float du = __uint_as_float(kmin);
            if ((u & 31) == lane) vis |= 1u << (u >> 5);
            if (u >= B && node_bcast<TV>(exc, u) > tol) {
                if (lane == kt) tgl = u;
                if (++kt == kt_max) break;
            }
            const float pu = node_bcast<TV>(pot, u);
            if (u < m) {
                const float* crow = s.C + u * ns;
#pragma unroll
                for (int t = 0; t < TV; ++t) {
                    if (t < SS) continue;  // source slots (warp-uniform)
                    const int v = lane + 32 * t;
                    if (v < VS && !((vis >> t) & 1u)) {
                        const float rc = fmaxf(crow[v - B] + pu - pot[t], 0.f);
                        const float nd = du + rc;
                        if (nd < dist[t]) {
                            dist[t] = nd;
                            s.pred[v] = (short)u;
                        }
                    }
                }
            } else {
                const int j = u - B;
#pragma unroll
                for (int t = 0; t < TV; ++t) {
                    if (t >= SS) break;  // sink slots (warp-uniform)
                    const int i = lane + 32 * t;
                    const bool arc = SP ? (i < m && ((s.mask[j * s.MW + t] >> lane) & 1u))
                                        : (i < m && s.F[i * ns + j] > tol);
                    if (arc && !((vis >> t) & 1u)) {
                        const float rc = fmaxf(-s.C[i * ns + j] + pu - pot[t], 0.f);
                        const float nd = du + rc;
                        if (nd < dist[t]) {
                            dist[t] = nd;
                            s.pred[i] = (short)u;
                        }
                    }
                }
            }
        }
        if (kt == 0) {
            hit_limit = true;  // no augmenting path (cannot happen with balanced supplies)
            break;
        }
        // ---- potentials: pot += min(dist, dist of the last target)
        const int tlast = __shfl_sync(0xffffffffu, tgl, kt - 1);
        const float dt = node_bcast<TV>(dist, tlast);
#pragma unroll
        for (int t = 0; t < TV; ++t) pot[t] += ((vis >> t) & 1u) ? fminf(dist[t], dt) : dt;
        __syncwarp();
        // ---- augment along each target's path in turn: lane 0 walks it
        // (flows in shared memory); a path whose bottleneck an earlier push
        // used up carries nothing
        for (int q = 0; q < kt; ++q) {
            const int target = __shfl_sync(0xffffffffu, tgl, q);
            float dflow = AS_INF;
            int src_node = target;
            if (lane == 0) {
                int v = target;
                for (int guard = 0; guard <= V; ++guard) {
                    const int p = s.pred[v];
                    if (p < 0) {
                        src_node = v;
                        break;
                    }
                    if (v < m) {  // backward arc (v, p - B)
                        float fv;
                        if (SP) {
                            int pv;
                            const int k = pool_find(s, v, p - B, &pv);
                            fv = k >= 0 ? s.ef[k] : 0.f;
                        } else {
                            fv = s.F[v * ns + (p - B)];
                        }
                        dflow = fminf(dflow, fv);
                    }
                    v = p;
                }
            }
            src_node = __shfl_sync(0xffffffffu, src_node, 0);
            dflow = __shfl_sync(0xffffffffu, dflow, 0);
            const float delta = fminf(fminf(dflow, node_bcast<TV>(exc, target)), node_bcast<TV>(exc, src_node));
            if (!(delta > 0.f)) continue;
            bool ovf = false;
            if (lane == 0) {
                int v = target;
                for (int guard = 0; guard <= V; ++guard) {
                    const int p = s.pred[v];
                    if (p < 0) break;
                    if (SP) {
                        if (v >= m) {  // forward arc p -> v
                            int pv;
                            int k = pool_find(s, p, v - B, &pv);
                            if (k < 0) k = pool_new(s, p, v - B, fbump, ffree);
                            if (k < 0) {
                                ovf = true;
                                break;
                            }
                            s.ef[k] += delta;
                            pool_bit(s, p, v - B, s.ef[k] > tol);
                        } else {       // backward arc: flow on (v, p - B) decreases
                            int pv;
                            const int k = pool_find(s, v, p - B, &pv);
                            if (k >= 0) {
                                float f = s.ef[k] - delta;
                                f = f > 0.f ? f : 0.f;
                                if (f == 0.f) pool_free(s, p - B, k, pv, ffree);
                                else s.ef[k] = f;
                                pool_bit(s, v, p - B, f > tol);
                            }
                        }
                    } else {
                        if (v >= m) {  // forward arc p -> v
                            s.F[p * ns + (v - B)] += delta;
                        } else {       // backward arc: flow on (v, p - B) decreases
                            const float f = s.F[v * ns + (p - B)] - delta;
                            s.F[v * ns + (p - B)] = f > 0.f ? f : 0.f;
                        }
                    }
                    v = p;
                }
            }
            if (SP && __shfl_sync(0xffffffffu, (int)ovf, 0)) {
                overflow = true;
                break;
            }
#pragma unroll
            for (int t = 0; t < TV; ++t) {
                const int v = lane + 32 * t;
                if (v == target) exc[t] -= delta;
                if (v == src_node) exc[t] -= delta;
            }
            __syncwarp();
        }
        if (overflow) break;
    }
    // ---- cost of the flow, FP64
    double acc = 0.0;
    if (SP) {
        __syncwarp();
        for (int j = lane; j < n; j += 32) {
            int k = s.head[j];
            for (int g = 0; g < s.E && (unsigned)k < (unsigned)s.E; ++g) {
                acc += (double)s.ef[k] * (double)s.C[s.esrc[k] * ns + j];
                k = s.enext[k];
            }
        }
    } else {
        for (int e = lane; e < m * ns; e += 32) acc += (double)s.F[e] * (double)s.C[e];  // padding: F = 0, C = 0
    }
    acc = group_sum_d<32>(acc);
    return acc;
}

template <int TV, bool SP>
__global__ void k_w2_pairs(AssignArgs a) {
    extern __shared__ float4 dyn4[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    char* base = reinterpret_cast<char*>(dyn4) + (size_t)wib * a.warp_bytes;
    const int m = a.m, n = a.nmax;
    const WarpLayout L = warp_layout(m, n, SP);
    WarpMem s;
    s.C = reinterpret_cast<float*>(base + L.c);
    s.F = reinterpret_cast<float*>(base + L.f);
    s.ef = reinterpret_cast<float*>(base + L.ef);
    s.mask = reinterpret_cast<unsigned*>(base + L.mask);
    s.head = reinterpret_cast<short*>(base + L.head);
    s.enext = reinterpret_cast<short*>(base + L.enext);
    s.esrc = reinterpret_cast<short*>(base + L.esrc);
    s.E = (a.pool_cap > 0 && a.pool_cap < L.E) ? a.pool_cap : L.E;
    s.MW = L.MW;
    s.pot = reinterpret_cast<float*>(base + L.pot);
    s.exc = reinterpret_cast<float*>(base + L.exc);
    s.pred = reinterpret_cast<short*>(base + L.pred);
    s.xs = reinterpret_cast<float*>(base + L.xs);
    s.ys = reinterpret_cast<float*>(base + L.ys);

    int64_t total;
    if (a.mode == 0) total = a.npairs;
    else if (a.mode == 1 || a.mode == 4) total = a.npairs_dev ? min(*a.npairs_dev, a.npairs) : a.npairs;
    else if (a.mode == 2) total = (*a.npairs_dev) * a.K;
    else total = a.npairs;
    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    for (int64_t p = (int64_t)blockIdx.x * wpb + wib; p < total; p += nwarps) {
        int64_t bag;
        int cent;
        int64_t slot;
        if (a.mode == 0) {
            bag = p / a.K;
            cent = (int)(p - bag * a.K);
            slot = p;
        } else if (a.mode == 1) {
            bag = a.pair_bag[p];
            cent = a.pair_cent[p];
            slot = p;
        } else if (a.mode == 2) {
            int64_t b = p / a.K;
            cent = (int)(p - b * a.K);
            bag = a.bag_list[b];
            slot = bag * a.K + cent;
        } else if (a.mode == 3) {
            bag = p / a.r;
            cent = a.cand[p];
            slot = p;
        } else {
            bag = a.pair_bag[p];
            cent = a.pair_cent[p];
            slot = a.pair_slot[p];
        }
        // size class of this launch (the per-warp tableaus are sized for nmax)
        const int64_t mk = a.offsets[bag + 1] - a.offsets[bag];
        if (mk <= a.nlo || mk > a.nmax) continue;
        bool lim = false, ovf = false;
        double v = solve_pair<TV, SP>(a, s, bag, cent, lim, ovf);
        if (lane == 0) {
            if (SP && ovf) {
                // solved again by the dense store after this launch
                const int64_t q = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(a.ovf_cnt), 1ull);
                if (q < a.ovf_cap) {
                    a.ovf_bag[q] = bag;
                    a.ovf_cent[q] = cent;
                    a.ovf_slot[q] = slot;
                } else {  // the list is full: report the pair as unsolved
                    a.out[slot] = (float)v;
                    atomicOr(a.flags, D2F_PIVOT_LIMIT);
                    atomicAdd(reinterpret_cast<unsigned long long*>(a.pivot_fail), 1ull);
                }
            } else {
                a.out[slot] = (float)v;
                if (lim) {
                    atomicOr(a.flags, D2F_PIVOT_LIMIT);
                    atomicAdd(reinterpret_cast<unsigned long long*>(a.pivot_fail), 1ull);
                }
            }
        }
        __syncwarp();
    }
}

// labels[k] = argmin_i D[k][i] (ties -> lowest i), dist[k] = min
__global__ void k_argmin_rows(const float* D, int64_t N, int K, int32_t* labels, float* dist) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N) return;
    const float* r = D + k * K;
    float b = r[0];
    int bi = 0;
    for (int i = 1; i < K; ++i) {
        float v = r[i];
        if (v < b) {
            b = v;
            bi = i;
        }
    }
    labels[k] = bi;
    dist[k] = b;
}


size_t d2_assign_warp_bytes(int m, int nmax) { return warp_layout(m, nmax, false).bytes; }

// warps per block that maximise resident warps per SM for this footprint
static int pick_wpb(size_t warp_bytes) {
    const size_t per_sm = 227 * 1024;
    int best = 1, best_w = 0;
    for (int w = 1; w <= 8; ++w) {
        if (warp_bytes * w > 200 * 1024) break;
        const int res = (int)(per_sm / (warp_bytes * w)) * w;
        if (res >= best_w) {
            best_w = res;
            best = w;
        }
    }
    return best;
}

// Solver instance for m + nmax nodes (node slots per lane) and flow store,
// or null past 256 nodes.
typedef void (*W2Fn)(AssignArgs);
static W2Fn w2_kernel_for(int V, bool sparse) {
    if (V <= 64) return sparse ? k_w2_pairs<2, true> : k_w2_pairs<2, false>;
    if (V <= 128) return sparse ? k_w2_pairs<4, true> : k_w2_pairs<4, false>;
    if (V <= 256) return sparse ? k_w2_pairs<8, true> : k_w2_pairs<8, false>;
    return nullptr;
}

// Launch shape of the pair solver for 32 ceil(a.m / 32) + a.nmax node slots on `device` with
// the given flow store: kernel, warps per block, dynamic shared memory and a
// grid bound (the kernel is a persistent stride loop; `resident` = warps per
// SM).  Returns D2_OK, or D2_ENOTSUP when the per-warp memory exceeds 200 KiB
// or 32 ceil(m / 32) + max_mk exceeds 256 (then *why says which), or D2_ECUDA when a
// runtime call fails.
struct PairLaunch {
    W2Fn fn;
    int wpb;
    size_t smem;
    unsigned grid;
    int resident;
};
static int pair_launch_config(AssignArgs& a, int64_t max_units, int device, bool sparse, PairLaunch* L,
                              const char** why, cudaError_t* cerr) {
    a.warp_bytes = warp_layout(a.m, a.nmax, sparse).bytes;
    if (a.warp_bytes > 200 * 1024) {
        *why = "m * max_mk too large for the per-warp tableau";
        return D2_ENOTSUP;
    }
    L->fn = w2_kernel_for(sink_base(a.m) + a.nmax, sparse);
    if (!L->fn) {
        *why = "32 ceil(m / 32) + max_mk exceeds 256";
        return D2_ENOTSUP;
    }
    L->wpb = pick_wpb(a.warp_bytes);
    L->smem = a.warp_bytes * L->wpb;
    cudaError_t e = cudaFuncSetAttribute(L->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L->smem);
    if (e != cudaSuccess) {
        *why = "k_w2_pairs shared-memory attribute";
        *cerr = e;
        return D2_ECUDA;
    }
    int sms = 152, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, L->fn, L->wpb * 32, L->smem);
    per_sm = std::max(per_sm, 1);
    L->resident = per_sm * L->wpb;
    const int64_t want = d2_ceil_div(std::max<int64_t>(max_units, 1), L->wpb);
    L->grid = (unsigned)std::max<int64_t>(1, std::min(want, (int64_t)sms * per_sm * 8));
    return D2_OK;
}

// default cap on the shortest-path phases of one pair (each phase routes
// flow to at least one deficit sink, so a pair needs far fewer)
static inline int default_max_phase(int m, int nmax) { return 8 * (m + nmax) + 64; }

// Bags per size class of the solver's launches: one launch per class of
// AS_CLASS support points, each with per-warp tableaus sized for its largest
// bag, so that smaller bags fit more warps per SM.  A launch skips the pairs
// of other classes; a pair's arithmetic does not depend on its launch.
#define AS_CLASS 16

// Pairs of one call whose sparse flow pool may overflow and be solved again
// by the dense store (list capacity; beyond it a pair is reported as
// unsolved through the phase-cap flag and count).
#define AS_OVF_CAP 65536

// Launch the pair solver, one launch per size class of bags; grid is a bound
// (persistent stride loop).  Each class uses the flow store that keeps more
// warps resident per SM (the dense one on ties); when any class used the
// sparse store, a last launch re-solves its overflowed pairs densely.
int d2_launch_pairs(d2_ctx* ctx, AssignArgs a, int64_t max_units, cudaStream_t st) {
    PairLaunch L, Ls;
    const char* why = "";
    cudaError_t ce = cudaSuccess;
    const int nmax = a.nmax;
    int rc = pair_launch_config(a, max_units, ctx->device, false, &L, &why, &ce);
    if (rc == D2_ENOTSUP) return d2_fail(ctx, D2_ENOTSUP, "d2_assign: %s (m = %d, max_mk = %d)", why, a.m, a.nmax);
    if (rc) return d2_cuda_fail(ctx, ce, why);
    a.max_phase = ctx->phase_limit > 0 ? ctx->phase_limit : default_max_phase(a.m, nmax);
    bool any_sparse = false;
    for (int lo = 0; lo < nmax; lo += AS_CLASS) {
        AssignArgs b = a;
        b.nlo = lo;
        b.nmax = std::min(nmax, lo + AS_CLASS);
        AssignArgs bs = b;
        if ((rc = pair_launch_config(b, max_units, ctx->device, false, &L, &why, &ce)))
            return d2_cuda_fail(ctx, ce, why);
        const bool sparse_ok = ctx->flow_store != 1 &&
                               pair_launch_config(bs, max_units, ctx->device, true, &Ls, &why, &ce) == D2_OK;
        if (sparse_ok && (ctx->flow_store == 2 || Ls.resident > L.resident)) {
            bs.pool_cap = ctx->pool_cap;
            if (!any_sparse) {
                void* ov = nullptr;
                const size_t cap = AS_OVF_CAP;
                if ((rc = d2_ws(ctx, WS_ASSIGN_OVF, 64 + cap * (8 + 4 + 8), &ov))) return rc;
                char* ob = static_cast<char*>(ov);
                a.ovf_cnt = reinterpret_cast<int64_t*>(ob);
                a.ovf_bag = reinterpret_cast<int64_t*>(ob + 64);
                a.ovf_slot = reinterpret_cast<int64_t*>(ob + 64 + cap * 8);
                a.ovf_cent = reinterpret_cast<int32_t*>(ob + 64 + cap * 16);
                a.ovf_cap = (int64_t)cap;
                D2_CK(ctx, cudaMemsetAsync(a.ovf_cnt, 0, sizeof(int64_t), st));
                any_sparse = true;
            }
            bs.ovf_cnt = a.ovf_cnt;
            bs.ovf_bag = a.ovf_bag;
            bs.ovf_slot = a.ovf_slot;
            bs.ovf_cent = a.ovf_cent;
            bs.ovf_cap = a.ovf_cap;
            b = bs;
            L = Ls;
        }
        d2_time_begin(ctx, D2_KT_ASSIGN, st);
        L.fn<<<L.grid, L.wpb * 32, L.smem, st>>>(b);
        d2_time_end(ctx, st);
        D2_LAUNCH_CK(ctx, "k_w2_pairs");
    }
    if (any_sparse) {
        // the overflow list, densely, all size classes in one launch
        AssignArgs r = a;
        r.mode = 4;
        r.npairs = a.ovf_cap;
        r.npairs_dev = a.ovf_cnt;
        r.pair_bag = a.ovf_bag;
        r.pair_cent = a.ovf_cent;
        r.pair_slot = a.ovf_slot;
        r.nlo = 0;
        r.nmax = nmax;
        if ((rc = pair_launch_config(r, 1, ctx->device, false, &L, &why, &ce))) return d2_cuda_fail(ctx, ce, why);
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        L.grid = (unsigned)(sms * std::max(1, L.resident / L.wpb));
        d2_time_begin(ctx, D2_KT_ASSIGN, st);
        L.fn<<<L.grid, L.wpb * 32, L.smem, st>>>(r);
        d2_time_end(ctx, st);
        D2_LAUNCH_CK(ctx, "k_w2_pairs (overflow re-solve)");
    }
    return D2_OK;
}

AssignArgs d2_assign_args(const d2_bags* b, int K, int m, const float* x, const float* w, int* flags,
                          int64_t* pivot_fail) {
    AssignArgs a;
    memset(&a, 0, sizeof(a));
    a.offsets = b->offsets;
    a.supp = b->supp;
    a.vidx = b->vocab_idx;
    a.vocab = b->vocab;
    a.wt = b->wt;
    a.d = b->d;
    a.x = x;
    a.w = w;
    a.m = m;
    a.K = K;
    a.nmax = b->max_mk;
    a.flags = flags;
    a.pivot_fail = pivot_fail;
    return a;
}

int d2_argmin_rows(d2_ctx* ctx, const float* D, int64_t N, int K, int32_t* labels, float* dist,
                   cudaStream_t st) {
    k_argmin_rows<<<(unsigned)d2_ceil_div(N, 256), 256, 0, st>>>(D, N, K, labels, dist);
    D2_LAUNCH_CK(ctx, "k_argmin_rows");
    return D2_OK;
}

__global__ void k_add_i64(int64_t* p, int64_t v) { *p += v; }

// all N x K pairs, then argmin per bag
int d2_assign_exact(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                    int32_t* labels, float* dist, int64_t* counters, cudaStream_t st) {
    const int64_t N = b->N;
    void* pD = nullptr;
    int rc = d2_ws(ctx, WS_ASSIGN, (size_t)N * K * 4, &pD);
    if (rc) return rc;
    float* D = static_cast<float*>(pD);
    AssignArgs a = d2_assign_args(b, K, m, x, w, ctx->dev_flags + D2_DEV_ERR_WORD, counters + 2);
    a.mode = 0;
    a.npairs = N * K;
    a.out = D;
    if ((rc = d2_launch_pairs(ctx, a, N * K, st))) return rc;
    k_add_i64<<<1, 1, 0, st>>>(counters, N * K);
    D2_LAUNCH_CK(ctx, "k_add_i64");
    return d2_argmin_rows(ctx, D, N, K, labels, dist, st);
}

// all N x K pairs with symbolic supports (costs from the bags' symbol table),
// then argmin per bag
int d2_assign_sym_exact(d2_ctx* ctx, const d2_bags* b, int K, int m, const int32_t* csym, const float* w,
                        int32_t* labels, float* dist, int64_t* counters, cudaStream_t st) {
    const int64_t N = b->N;
    void* pD = nullptr;
    int rc = d2_ws(ctx, WS_ASSIGN, (size_t)N * K * 4, &pD);
    if (rc) return rc;
    float* D = static_cast<float*>(pD);
    AssignArgs a = d2_assign_args(b, K, m, nullptr, w, ctx->dev_flags + D2_DEV_ERR_WORD, counters + 2);
    a.d = 1;
    a.symcost = b->symcost;
    a.csym = csym;
    a.V = b->V;
    a.mode = 0;
    a.npairs = N * K;
    a.out = D;
    if ((rc = d2_launch_pairs(ctx, a, N * K, st))) return rc;
    k_add_i64<<<1, 1, 0, st>>>(counters, N * K);
    D2_LAUNCH_CK(ctx, "k_add_i64");
    return d2_argmin_rows(ctx, D, N, K, labels, dist, st);
}

// pair lists for the pruned assignment (mode 2: all K for a device-counted
// bag list; mode 3: r candidates per bag)
int d2_prune_solve_pairs(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w, int mode,
                         int64_t npairs, const int64_t* npairs_dev, const int32_t* cand, int r,
                         const int64_t* bag_list, float* out, int64_t* fail_count, cudaStream_t st) {
    AssignArgs a = d2_assign_args(b, K, m, x, w, ctx->dev_flags + D2_DEV_ERR_WORD, fail_count);
    a.mode = mode;
    a.npairs = npairs;
    a.npairs_dev = npairs_dev;
    a.cand = cand;
    a.r = r;
    a.bag_list = bag_list;
    a.out = out;
    return d2_launch_pairs(ctx, a, npairs, st);
}

extern "C" int d2_w2_pairs(d2_ctx* ctx, const d2_bags* bags, int32_t K, int32_t m, const float* x, const float* w,
                           const int64_t* pair_bag, const int32_t* pair_cent, int64_t npairs, float* out,
                           void* stream) {
    if (!ctx) return D2_EINVAL;
    int rc = d2_check_bags_host(ctx, bags);
    if (rc) return rc;
    if (K < 1 || m < 1 || npairs < 0 || !x || !w || (npairs > 0 && (!pair_bag || !pair_cent || !out)))
        return d2_fail(ctx, D2_EINVAL, "d2_w2_pairs: bad arguments");
    if (npairs == 0) return D2_OK;
    cudaStream_t st = d2_stream(stream);
    void* sc = nullptr;
    if ((rc = d2_ws(ctx, WS_SCAN, 64, &sc))) return rc;
    int64_t* counters = static_cast<int64_t*>(sc);
    D2_CK(ctx, cudaMemsetAsync(counters, 0, 3 * sizeof(int64_t), st));
    AssignArgs a = d2_assign_args(bags, K, m, x, w, ctx->dev_flags + D2_DEV_ERR_WORD, counters + 2);
    a.mode = 1;
    a.npairs = npairs;
    a.pair_bag = pair_bag;
    a.pair_cent = pair_cent;
    a.out = out;
    return d2_launch_pairs(ctx, a, npairs, st);
}

// All N x K pairs into D, then argmin per bag, with caller-provided scratch
// (D: N*K floats, flags: 1 int, fail_count: 1 int64, both already zeroed).
// No context, no allocation.  Returns D2_OK, D2_ENOTSUP (the shape limits of
// pair_launch_config) or D2_ECUDA (*cerr holds the runtime's error).
int d2_assign_exact_into(const d2_bags* b, int K, int m, const float* x, const float* w, int32_t* labels,
                         float* dist, float* D, int* flags, int64_t* fail_count, int device, cudaStream_t st,
                         cudaError_t* cerr) {
    AssignArgs a = d2_assign_args(b, K, m, x, w, flags, fail_count);
    a.mode = 0;
    a.npairs = b->N * (int64_t)K;
    a.out = D;
    PairLaunch L;
    const char* why = "";
    *cerr = cudaSuccess;
    const int nmax = a.nmax;
    int rc = pair_launch_config(a, a.npairs, device, false, &L, &why, cerr);
    if (rc) return rc;
    a.max_phase = default_max_phase(a.m, nmax);
    for (int lo = 0; lo < nmax; lo += AS_CLASS) {
        AssignArgs c = a;
        c.nlo = lo;
        c.nmax = std::min(nmax, lo + AS_CLASS);
        if ((rc = pair_launch_config(c, c.npairs, device, false, &L, &why, cerr))) return rc;
        L.fn<<<L.grid, L.wpb * 32, L.smem, st>>>(c);
        if ((*cerr = cudaGetLastError()) != cudaSuccess) return D2_ECUDA;
    }
    k_argmin_rows<<<(unsigned)d2_ceil_div(b->N, 256), 256, 0, st>>>(D, b->N, K, labels, dist);
    if ((*cerr = cudaGetLastError()) != cudaSuccess) return D2_ECUDA;
    return D2_OK;
}

// explicit pair list whose length is read on the device (<= max_pairs)
int d2_solve_pair_list(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w,
                       const int64_t* pair_bag, const int32_t* pair_cent, int64_t max_pairs,
                       const int64_t* npairs_dev, float* out, int64_t* fail_count, cudaStream_t st) {
    AssignArgs a = d2_assign_args(b, K, m, x, w, ctx->dev_flags + D2_DEV_ERR_WORD, fail_count);
    a.mode = 1;
    a.npairs = max_pairs;
    a.npairs_dev = npairs_dev;
    a.pair_bag = pair_bag;
    a.pair_cent = pair_cent;
    a.out = out;
    return d2_launch_pairs(ctx, a, max_pairs, st);
}

// all N x K pairs into out (N x K), no argmin
int d2_launch_pairs_all(d2_ctx* ctx, const d2_bags* b, int K, int m, const float* x, const float* w, float* out,
                        int64_t* fail_count, cudaStream_t st) {
    AssignArgs a = d2_assign_args(b, K, m, x, w, ctx->dev_flags + D2_DEV_ERR_WORD, fail_count);
    a.mode = 0;
    a.npairs = b->N * (int64_t)K;
    a.out = out;
    return d2_launch_pairs(ctx, a, a.npairs, st);
}
