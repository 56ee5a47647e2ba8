// cc_minlabel.cu -- the min-based finishes that need not be monotone
// (Section 3.3, "Liu-Tarjan's Algorithms", "Stergiou et al.'s Algorithm",
// "Shiloach-Vishkin and Label Propagation"; rules in the appendix's
// Liu-Tarjan list): the Liu-Tarjan framework's connect / update / shortcut
// / alter rules (all sixteen variants), Stergiou et al.'s two-array
// algorithm and label propagation.
//
// Composition with sampling (Section 3.3, "Sampling for Other Min-Based
// Algorithms"): the frequent cluster's label m0 is made the smallest id, so
// its vertices never change and their edges are never read.  Here the
// labels are held as keys during the finish: key(m0) = 0 and key(x) = x + 1
// for every other id (the identity without sampling), which ranks m0 first
// and keeps every other comparison.  At the end the keys go back to ids and
// each label is replaced by the smallest member of its class, giving the
// canonical min-id labels.
#include "cc_internal.h"

using namespace ccg;

namespace {

constexpr unsigned TPB = 256;

struct Keys {
    uint32_t m0;   // the frequent sampled label, NONE without sampling
    __device__ __forceinline__ uint32_t key(uint32_t x) const { return m0 == NONE ? x : (x == m0 ? 0u : x + 1); }
    __device__ __forceinline__ uint32_t id(uint32_t k) const { return m0 == NONE ? k : (k == 0 ? m0 : k - 1); }
};

__global__ void __launch_bounds__(256, 8) k_flag(uint32_t *err, uint32_t bits) { atomicOr(err, bits); }

__global__ void __launch_bounds__(256, 8) k_to_keys(uint32_t *P, uint32_t n, Keys ks) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        P[i] = ks.key(P[i]);
}

__global__ void __launch_bounds__(256, 8) k_from_keys(uint32_t *P, uint32_t n, Keys ks) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        P[i] = ks.id(P[i]);
}

// Canonical form: every label replaced by the smallest vertex that holds it.
__global__ void __launch_bounds__(256, 8) k_class_min(const uint32_t *P, uint32_t n, uint32_t *cmin) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = P[i];
        if (l < n && (uint32_t)i < ld_rel(cmin + l)) atomicMin(cmin + l, (uint32_t)i);
    }
}

__global__ void __launch_bounds__(256, 8) k_apply_class_min(uint32_t *P, uint32_t n, const uint32_t *cmin) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = P[i];
        if (l < n) P[i] = cmin[l];
    }
}

// ---------------------------------------------------------------- Liu-Tarjan
// Connect rules: CONNECT offers the endpoints as candidates for each other;
// PARENT_CONNECT offers the endpoints' parents to each other's parent;
// EXTENDED_CONNECT offers the parents to both the endpoints and their
// parents.  ROOTUP: a vertex takes a candidate only if it was a root at the
// round's start (prev holds the round's starting keys).  Every update is a
// writeMin, so a vertex ends a round with the smallest candidate it saw.
enum { LT_CONNECT = 0, LT_PARENT = 1, LT_EXTENDED = 2 };
template <int C, bool R>
struct RuleTag {
    static constexpr int c = C;
    static constexpr bool r = R;
};

// lower: every vertex is a candidate (no sampling), so each undirected
// edge is applied once, from its larger endpoint; the rules offer both
// ways, so the smaller endpoint's copy would repeat the same offers.
template <int CONN, bool ROOTUP>
struct LTRule {
    uint32_t *K;
    const uint32_t *prev;
    Keys ks;
    bool hit;
    bool lower;
    __device__ __forceinline__ void offer(uint32_t z, uint32_t cand) {
        if (cand < ld_rel(K + z) && (!ROOTUP || prev[z] == ks.key(z))) hit |= atomicMin(K + z, cand) > cand;
    }
    __device__ __forceinline__ void edge(uint32_t u, uint32_t w) {
        if (CONN == LT_CONNECT) {
            offer(u, ks.key(w));
            offer(w, ks.key(u));
        } else {
            const uint32_t ku = ld_rel(K + u), kw = ld_rel(K + w);
            const uint32_t x = ks.id(ku), y = ks.id(kw);
            if (CONN == LT_EXTENDED) {
                offer(u, kw);
                offer(w, ku);
            }
            offer(x, kw);
            offer(y, ku);
        }
    }
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j] && !(lower && v[j] > u)) edge(u, v[j]);
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j] && !(lower && v[j] > u[j])) edge(u[j], v[j]);
    }
};

// Candidate edges read from the CSR: light candidates one per thread, the
// heavier ones as warp chunks (the lists the binning pass built).
template <typename OffT, class F>
__global__ void __launch_bounds__(256, 8) k_lists(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                                                  const uint32_t *light, const uint32_t *nlight, const ChunkRef *chunks,
                                                  const uint32_t *nchunks, uint64_t cap, F f, uint32_t *changed,
                                                  Dev d) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t total = *nlight;
    for (uint64_t base = warp * 32; base < total; base += nw * 32) {
        const bool act = base + lane < total;
        const uint32_t u = act ? light[base + lane] : 0;
        uint64_t b = 0, e = 0;
        if (act) vertex_range(I, u, m, b, e, d);
        const uint64_t deg = e - b;   // <= LIGHT_MAX: the binning listed light vertices only
        warp_light_edges(u, b, deg > LIGHT_MAX ? LIGHT_MAX : (uint32_t)deg, A, n, f, d);
    }
    run_chunks(I, A, n, m, chunks, nchunks, cap, f, d);
    if (__any_sync(0xFFFFFFFFu, f.hit) && (threadIdx.x & 31) == 0) *changed = 1u;
}

// The same rules on an explicit edge list (the Alter variants rewrite it).
template <class F>
__global__ void __launch_bounds__(256, 8) k_pairs(const uint32_t *E, const uint32_t *count, F f, uint32_t *changed) {
    const uint32_t total = *count;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 e = reinterpret_cast<const uint2 *>(E)[i];
        f.edge(e.x, e.y);
    }
    if (__any_sync(0xFFFFFFFFu, f.hit) && (threadIdx.x & 31) == 0) *changed = 1u;
}

// Edge list of the candidates' edges (pairs (u, v) in no particular order).
struct PairOut {
    uint32_t *E;
    uint32_t *count;
    uint64_t cap;
    Dev d;
    bool hit;
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j] || v[j] == u) continue;
            const uint32_t k = append_one(count);
            if (k >= cap) { atomicOr(d.err, ERR_NONCONVERGED); continue; }
            reinterpret_cast<uint2 *>(E)[k] = make_uint2(u, v[j]);
        }
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j] || v[j] == u[j]) continue;
            const uint32_t k = append_one(count);
            if (k >= cap) { atomicOr(d.err, ERR_NONCONVERGED); continue; }
            reinterpret_cast<uint2 *>(E)[k] = make_uint2(u[j], v[j]);
        }
    }
};

// Alter: every edge (a, b) becomes (P[a], P[b]); edges inside one tree go.
// First in place (an edge that goes becomes (NONE, NONE)), so each edge's
// two parents are read once; then the survivors are compacted into the
// other buffer with one atomic per block.
__global__ void __launch_bounds__(256, 8) k_alter_in_place(uint32_t *E, const uint32_t *count, const uint32_t *K,
                                                           Keys ks) {
    const uint32_t total = *count;
    uint2 *e2 = reinterpret_cast<uint2 *>(E);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 e = e2[i];
        if (e.x == NONE) continue;
        const uint32_t a = ks.id(ld_rel(K + e.x)), b = ks.id(ld_rel(K + e.y));
        e2[i] = a == b ? make_uint2(NONE, NONE) : make_uint2(a, b);
    }
}

__global__ void __launch_bounds__(256, 8) k_alter_compact(const uint32_t *Ein, const uint32_t *cin, uint32_t *Eout,
                                                          uint32_t *cout) {
    const uint2 *ein = reinterpret_cast<const uint2 *>(Ein);
    block_compact(
        *cin, cout, [&](uint64_t i) { return ein[i].x != NONE; },
        [&](uint64_t i, uint32_t k) { reinterpret_cast<uint2 *>(Eout)[k] = ein[i]; });
}

// The edge list of every vertex's edges at their CSR positions, for the
// finish without sampling (every vertex is a candidate): no counter.  Each
// undirected edge is kept once, at its larger endpoint's copy (the connect
// rules offer both ways, and the symmetric CSR holds the other copy); the
// smaller endpoint's copy, a self-loop and a bad id become (NONE, NONE).
// The candidate lists drive it: light vertices walked by their warp
// together, heavier ones as CHUNK-edge pieces spread over the grid's warps
// (a hub's list is not left to one warp).
__device__ __forceinline__ uint2 pair_or_none(uint32_t u, uint32_t v, uint32_t n) {
    return (v >= u || v >= n) ? make_uint2(NONE, NONE) : make_uint2(u, v);
}

// Writes (u, v) or (NONE, NONE) at each light edge's own CSR position.
struct PositionPairs {
    uint2 *e2;
    uint32_t n;
    __device__ __forceinline__ void apply4p(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4],
                                            const uint64_t (&pos)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) e2[pos[j]] = pair_or_none(u[j], v[j], n);
    }
};

template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_pairs_at_positions(const OffT *I, const uint32_t *A, uint32_t n,
                                                               uint64_t m, const uint32_t *light,
                                                               const uint32_t *nlight, const ChunkRef *chunks,
                                                               const uint32_t *nchunks, uint64_t cap, uint32_t *E,
                                                               Dev d) {
    uint2 *e2 = reinterpret_cast<uint2 *>(E);
    const uint32_t nl = *nlight;
    const int lane = threadIdx.x & 31;
    {
        // light candidates: the warp walks its 32 vertices' edges together
        const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
        const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
        PositionPairs f{e2, n};
        for (uint64_t base = warp * 32; base < nl; base += nw * 32) {
            const bool act = base + lane < nl;
            const uint32_t u = act ? light[base + lane] : 0;
            uint64_t b = 0, e = 0;
            if (act) vertex_range(I, u, m, b, e, d);
            const uint64_t deg = e - b;
            warp_light_edges<PositionPairs, true>(u, b, deg > LIGHT_MAX ? LIGHT_MAX : (uint32_t)deg, A, n, f, d);
        }
    }
    const uint32_t total = (uint32_t)((uint64_t)*nchunks < cap ? (uint64_t)*nchunks : cap);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = warp; c < total; c += nwarps) {
        const ChunkRef cr = chunks[c];
        if (cr.u == NONE) continue;   // an empty slot of a warp's reservation
        uint64_t b, e;
        vertex_range(I, cr.u, m, b, e, d);
        const uint64_t cb = b + (uint64_t)cr.c * CHUNK, ce = cb + CHUNK < e ? cb + CHUNK : e;
        for (uint64_t x = cb + lane; x < ce; x += 128) {
            uint32_t v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = x + 32 * j < ce ? ld_stream(A + x + 32 * j) : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x + 32 * j < ce) e2[x + 32 * j] = pair_or_none(cr.u, v[j], n);
        }
    }
}

// Shortcut: one step of pointer jumping (P[v] <- P[P[v]]), or FullShortcut
// (repeated to a fixed point: every vertex points at its root).  Keys
// strictly decrease along parents, so the walk ends at a root.
template <bool FULL>
__global__ void __launch_bounds__(256, 8) k_key_shortcut(uint32_t *K, uint32_t n, Keys ks, uint32_t *changed, Dev d) {
    bool hit = false;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)i, k = ld_rel(K + v);
        uint32_t kr = k, r = ks.id(k);
        if (FULL) {
            Guard g;
            for (;;) {
                const uint32_t kp = ld_rel(K + r);
                if (kp == kr) break;   // r is a root
                kr = kp;
                r = ks.id(kp);
                if (!g.step(d)) break;
            }
        } else {
            kr = ld_rel(K + r);
        }
        if (kr < k) {
            K[v] = kr;
            hit = true;
        }
    }
    if (changed && __any_sync(0xFFFFFFFFu, hit) && (threadIdx.x & 31) == 0) *changed = 1u;
}

// ---------------------------------------------------------------- Stergiou
// Two arrays: each round copies cur into prev, runs ParentConnect with the
// candidates taken from prev and the updates written into cur (no root
// condition), then one Shortcut step on cur; rounds repeat until cur stops
// changing.
struct StergiouRule {
    uint32_t *cur;
    const uint32_t *prev;
    Keys ks;
    bool hit;
    bool lower;   // no sampling: each undirected edge from its larger endpoint (both offers are symmetric)
    __device__ __forceinline__ void offer(uint32_t z, uint32_t cand) {
        if (cand < ld_rel(cur + z)) hit |= atomicMin(cur + z, cand) > cand;
    }
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
        const uint32_t ku = prev[u];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j] || (lower && v[j] > u)) continue;
            const uint32_t kw = prev[v[j]];
            offer(ks.id(ku), kw);
            offer(ks.id(kw), ku);
        }
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
        uint32_t ku[4], kw[4];
        bool go[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            go[j] = ok[j] && !(lower && v[j] > u[j]);
            ku[j] = go[j] ? prev[u[j]] : 0;
            kw[j] = go[j] ? prev[v[j]] : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!go[j]) continue;
            offer(ks.id(ku[j]), kw[j]);
            offer(ks.id(kw[j]), ku[j]);
        }
    }
};

// ---------------------------------------------------------------- label propagation
// Each round, the vertices whose label changed in the previous round
// (first: every candidate) offer their label to their neighbours and take
// a smaller neighbour's label (writeMin both ways, so a label held by a
// vertex whose edges are skipped still spreads through its neighbours'
// edges); a vertex whose label dropped joins the next frontier once.
// in_front (bitmap of this round's frontier): an edge whose endpoints are
// both in the frontier is applied once, from its larger endpoint (the rule
// is symmetric in the endpoints).
struct LPRule {
    uint32_t *K;
    uint32_t *mark;      // bitmap: already in the next frontier
    uint32_t *next;
    uint32_t *nnext;
    const uint32_t *in_front;
    __device__ __forceinline__ bool twice(uint32_t u, uint32_t w) const {
        return w > u && ((in_front[w >> 5] >> (w & 31)) & 1u);
    }
    __device__ __forceinline__ void lowered(uint32_t z) {
        const uint32_t bit = 1u << (z & 31);
        if (ld_rel(mark + (z >> 5)) & bit) return;
        if (atomicOr(mark + (z >> 5), bit) & bit) return;
        next[append_one(nnext)] = z;
    }
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j] || twice(u, v[j])) continue;
            const uint32_t ku = ld_rel(K + u), kw = ld_rel(K + v[j]);
            if (ku < kw) {
                if (atomicMin(K + v[j], ku) > ku) lowered(v[j]);
            } else if (kw < ku) {
                if (atomicMin(K + u, kw) > kw) lowered(u);
            }
        }
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool one[4] = {ok[j], false, false, false};
            const uint32_t w[4] = {v[j], 0, 0, 0};
            apply4(u[j], w, one);
        }
    }
};

// Edges of a vertex list: light vertices one per thread, heavier ones by the
// whole warp.
template <typename OffT, class F>
__global__ void __launch_bounds__(256, 8) k_frontier(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                                                     const uint32_t *list, const uint32_t *count, F f, Dev d) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t total = *count;
    for (uint64_t base = warp * 32; base < total; base += nw * 32) {
        const bool act = base + lane < total;
        const uint32_t u = act ? list[base + lane] : 0;
        uint64_t b = 0, e = 0;
        if (act) vertex_range(I, u, m, b, e, d);
        const bool heavy = e - b > LIGHT_MAX;
        warp_light_edges(u, b, heavy ? 0u : (uint32_t)(e - b), A, n, f, d);
        uint32_t hm = __ballot_sync(0xFFFFFFFFu, heavy);
        while (hm) {
            const int l = __ffs(hm) - 1;
            hm &= hm - 1;
            const uint32_t hu = __shfl_sync(0xFFFFFFFFu, u, l);
            const uint64_t hb = __shfl_sync(0xFFFFFFFFu, b, l), he = __shfl_sync(0xFFFFFFFFu, e, l);
            warp_chunk_edges(hu, hb, he, A, n, f, d);
        }
    }
}

// Initial frontier: every vertex with edges outside the frequent cluster
// (whose key is 0 when there is one).
// The frontier's bitmap gets the same vertices (one OR per word per warp).
template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_lp_init(const OffT *I, uint32_t n, uint64_t m, const uint32_t *K, Keys ks,
                                                    uint32_t *list, uint32_t *count, uint32_t *in_front, Dev d) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = warp * 32; base < n; base += nw * 32) {
        const uint64_t i = base + lane;
        bool take = false;
        if (i < n) {
            uint64_t b, e;
            vertex_range(I, (uint32_t)i, m, b, e, d);
            take = e > b && !(ks.m0 != NONE && K[i] == 0);
        }
        const uint32_t bits = __ballot_sync(0xFFFFFFFFu, take);
        if (lane == 0 && bits) in_front[base >> 5] = bits;
        if (take) list[append_one(count)] = (uint32_t)i;
    }
}

struct Flags {
    uint32_t changed;
    uint32_t npairs[2];
    uint32_t nfront[2];
    uint32_t pad[3];
};

template <typename OffT>
cc_status run_minlabel(const MinLabelIn &in, const cc_finish_opt &fo, const DeviceInfo *di, const Dev &d,
                       cudaStream_t s, uint32_t *rounds_out) {
    const OffT *I = static_cast<const OffT *>(in.I);
    const uint32_t n = in.n;
    const unsigned gv = grid_for(di, n, TPB);
    auto ge_for = [&](uint64_t items) { return grid_for(di, items ? items : 1, TPB); };
    const bool alter = fo.kind == CC_FINISH_LIU_TARJAN && (fo.lt_rules & CC_LT_ALTER);
    const bool lp = fo.kind == CC_FINISH_LABEL_PROP;
    const bool rootup = fo.kind == CC_FINISH_LIU_TARJAN && (fo.lt_rules & CC_LT_ROOTUP);
    unsigned long long cand_edges = 0;
    uint32_t m0 = NONE;
    {
        cudaError_t e = cudaMemcpyAsync(&cand_edges, in.cand_edges, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && in.lmax_p) e = cudaMemcpyAsync(&m0, in.lmax_p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return from_cuda(e);
    }
    const Keys ks{m0};
    if (alter && cand_edges >= 0xFFFFFFFFull) return CC_ERR_UNSUPPORTED;   // edge-list counters are 32-bit
    const uint64_t words = (n + 31) / 32;
    Scratch sc;
    const size_t o_fl = sc.reserve(sizeof(Flags)), o_prev = sc.reserve((size_t)n * 4),
                 o_cmin = sc.reserve((size_t)n * 4);
    const size_t o_e0 = alter ? sc.reserve(cand_edges * 8) : 0, o_e1 = alter ? sc.reserve(cand_edges * 8) : 0;
    const size_t o_q0 = lp ? sc.reserve((size_t)n * 4) : 0, o_q1 = lp ? sc.reserve((size_t)n * 4) : 0,
                 o_mark = lp ? sc.reserve(2 * words * 4) : 0;   // next-frontier marks, this frontier's bitmap
    cc_status st = sc.alloc(s);
    if (st != CC_OK) return st;
    Flags *fl = sc.at<Flags>(o_fl);
    uint32_t *K = in.P, *prev = sc.at<uint32_t>(o_prev), *cmin = sc.at<uint32_t>(o_cmin);
    Flags hf;
    auto read_flags = [&]() -> cc_status {
        cudaError_t e = cudaMemcpyAsync(&hf, fl, sizeof(Flags), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return from_cuda(e);
    };
    cudaError_t ce = cudaMemsetAsync(fl, 0, sizeof(Flags), s);
    if (ce != cudaSuccess) return from_cuda(ce);
    {
        CC_PROF("k_to_keys", s);
        k_to_keys<<<gv, TPB, 0, s>>>(K, n, ks);
    }
    uint32_t *E[2] = {alter ? sc.at<uint32_t>(o_e0) : nullptr, alter ? sc.at<uint32_t>(o_e1) : nullptr};
    if (alter) {
        // The finish runs on the graph contracted by the sampling: its edges
        // are (P[u], P[v]).  So the list starts altered.  The edges are
        // taken as read, and then a round whose connect and shortcut change
        // nothing would end the loop before the first Alter.
        if (!in.lmax_p) {
            // no sampling: every edge at its CSR position, no counter
            const uint32_t m32 = (uint32_t)in.m;
            ce = cudaMemcpyAsync(&fl->npairs[1], &m32, 4, cudaMemcpyHostToDevice, s);
            if (ce != cudaSuccess) return from_cuda(ce);
            CC_PROF("k_pairs_build", s);
            k_pairs_at_positions<OffT><<<gv, TPB, 0, s>>>(I, in.A, n, in.m, in.light, in.nlight, in.chunks,
                                                          in.nchunks, in.chunk_cap, E[1], d);
        } else {
            PairOut po{E[1], &fl->npairs[1], cand_edges, d, false};
            CC_PROF("k_pairs_build", s);
            k_lists<OffT, PairOut><<<gv, TPB, 0, s>>>(I, in.A, n, in.m, in.light, in.nlight, in.chunks, in.nchunks,
                                                       in.chunk_cap, po, &fl->changed, d);
        }
        {
            CC_PROF("k_alter", s);
            k_alter_in_place<<<ge_for(cand_edges), TPB, 0, s>>>(E[1], &fl->npairs[1], K, ks);
        }
        CC_PROF("k_alter_compact", s);
        k_alter_compact<<<gv, TPB, 0, s>>>(E[1], &fl->npairs[1], E[0], &fl->npairs[0]);
    }
    if ((ce = cudaGetLastError()) != cudaSuccess) return from_cuda(ce);
    const uint64_t cap = lp ? (uint64_t)n + 2 : (uint64_t)round_cap();
    uint32_t rounds = 0;
    int cur = 0;
    if (lp) {
        uint32_t *q[2] = {sc.at<uint32_t>(o_q0), sc.at<uint32_t>(o_q1)};
        uint32_t *bm[2] = {sc.at<uint32_t>(o_mark), sc.at<uint32_t>(o_mark) + words};
        if ((ce = cudaMemsetAsync(bm[0], 0, words * 4, s)) != cudaSuccess) return from_cuda(ce);
        {
            CC_PROF("k_lp_init", s);
            k_lp_init<OffT><<<gv, TPB, 0, s>>>(I, n, in.m, K, ks, q[0], &fl->nfront[0], bm[0], d);
        }
        for (;;) {
            if ((st = read_flags()) != CC_OK) return st;
            if (hf.nfront[cur] == 0) break;
            if (rounds >= cap) {
                k_flag<<<1, 1, 0, s>>>(di->err, CC_DEVERR_NONCONVERGED);
                break;
            }
            const int nx = cur ^ 1;
            if ((ce = cudaMemsetAsync(&fl->nfront[nx], 0, 4, s)) != cudaSuccess) return from_cuda(ce);
            // bm[cur] marks this frontier; bm[nx] collects the next one
            if ((ce = cudaMemsetAsync(bm[nx], 0, words * 4, s)) != cudaSuccess) return from_cuda(ce);
            LPRule f{K, bm[nx], q[nx], &fl->nfront[nx], bm[cur]};
            {
                CC_PROF("k_lp_round", s);
                k_frontier<OffT, LPRule><<<gv, TPB, 0, s>>>(I, in.A, n, in.m, q[cur], &fl->nfront[cur], f, d);
            }
            if ((ce = cudaGetLastError()) != cudaSuccess) return from_cuda(ce);
            cur = nx;
            ++rounds;
        }
    } else {
        for (;;) {
            if (rounds >= cap) {
                k_flag<<<1, 1, 0, s>>>(di->err, CC_DEVERR_NONCONVERGED);
                break;
            }
            if ((ce = cudaMemsetAsync(&fl->changed, 0, 4, s)) != cudaSuccess) return from_cuda(ce);
            if (rootup || fo.kind == CC_FINISH_STERGIOU)
                if ((ce = cudaMemcpyAsync(prev, K, (size_t)n * 4, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                    return from_cuda(ce);
            if (fo.kind == CC_FINISH_STERGIOU) {
                CC_PROF("k_stergiou_connect", s);
                StergiouRule f{K, prev, ks, false, in.lmax_p == nullptr};
                k_lists<OffT, StergiouRule><<<gv, TPB, 0, s>>>(I, in.A, n, in.m, in.light, in.nlight, in.chunks,
                                                               in.nchunks, in.chunk_cap, f, &fl->changed, d);
            } else {
                const int conn = fo.lt_rules & 3;
                auto connect = [&](auto tag) {
                    constexpr int C = decltype(tag)::c;
                    constexpr bool R = decltype(tag)::r;
                    using Rule = LTRule<C, R>;
                    Rule f{K, prev, ks, false, in.lmax_p == nullptr};
                    if (alter) {
                        CC_PROF("k_lt_connect_pairs", s);
                        k_pairs<Rule><<<gv, TPB, 0, s>>>(E[cur], &fl->npairs[cur], f, &fl->changed);
                    } else {
                        CC_PROF("k_lt_connect", s);
                        k_lists<OffT, Rule><<<gv, TPB, 0, s>>>(I, in.A, n, in.m, in.light, in.nlight, in.chunks,
                                                               in.nchunks, in.chunk_cap, f, &fl->changed, d);
                    }
                };
                switch (conn * 2 + (rootup ? 1 : 0)) {
                    case 0: connect(RuleTag<LT_CONNECT, false>{}); break;
                    case 1: connect(RuleTag<LT_CONNECT, true>{}); break;
                    case 2: connect(RuleTag<LT_PARENT, false>{}); break;
                    case 3: connect(RuleTag<LT_PARENT, true>{}); break;
                    default: connect(RuleTag<LT_EXTENDED, false>{}); break;
                }
            }
            const bool full = fo.kind == CC_FINISH_LIU_TARJAN && (fo.lt_rules & CC_LT_FULL);
            if (full) {
                CC_PROF("k_key_shortcut_full", s);
                k_key_shortcut<true><<<gv, TPB, 0, s>>>(K, n, ks, &fl->changed, d);
            } else {
                CC_PROF("k_key_shortcut", s);
                k_key_shortcut<false><<<gv, TPB, 0, s>>>(K, n, ks, &fl->changed, d);
            }
            if (alter) {
                const int nx = cur ^ 1;
                if ((ce = cudaMemsetAsync(&fl->npairs[nx], 0, 4, s)) != cudaSuccess) return from_cuda(ce);
                {
                    CC_PROF("k_alter", s);
                    k_alter_in_place<<<ge_for(cand_edges), TPB, 0, s>>>(E[cur], &fl->npairs[cur], K, ks);
                }
                CC_PROF("k_alter_compact", s);
                k_alter_compact<<<gv, TPB, 0, s>>>(E[cur], &fl->npairs[cur], E[nx], &fl->npairs[nx]);
                cur = nx;
            }
            if ((ce = cudaGetLastError()) != cudaSuccess) return from_cuda(ce);
            ++rounds;
            if ((st = read_flags()) != CC_OK) return st;
            if (hf.changed == 0) break;
        }
    }
    {
        CC_PROF("k_from_keys", s);
        k_from_keys<<<gv, TPB, 0, s>>>(K, n, ks);
    }
    if ((ce = cudaMemsetAsync(cmin, 0xFF, (size_t)n * 4, s)) != cudaSuccess) return from_cuda(ce);
    {
        CC_PROF("k_class_min", s);
        k_class_min<<<gv, TPB, 0, s>>>(K, n, cmin);
    }
    {
        CC_PROF("k_apply_class_min", s);
        k_apply_class_min<<<gv, TPB, 0, s>>>(K, n, cmin);
    }
    if (rounds_out) *rounds_out = rounds;
    return from_cuda(cudaGetLastError());
}

}  // namespace

namespace ccg {

cc_status minlabel_finish(const MinLabelIn &in, const cc_finish_opt &fo, const DeviceInfo *di, const Dev &d,
                          cudaStream_t s, uint32_t *rounds_out) {
    return in.offsets_u64 ? run_minlabel<uint64_t>(in, fo, di, d, s, rounds_out)
                          : run_minlabel<uint32_t>(in, fo, di, d, s, rounds_out);
}

}  // namespace ccg
