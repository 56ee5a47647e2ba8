// cc_static.cu -- static connectivity, Algorithm 1: labels <- identity,
// SampleComponents (k-out / BFS / LDD, Section 3.2, Algorithms 4-6),
// IdentifyFrequent, FinishComponents (union-find, Algorithm 7 with the
// engines of Algorithms 8-10 and 14; Shiloach-Vishkin, Algorithm 15;
// Liu-Tarjan PRF, Appendix D) and a final shortcut to min-id labels.
//
// The parent array P is the caller's labels_out buffer throughout.  Every
// kernel grid-strides; edge work is degree-binned (cc_device.cuh) so that a
// hub's edges spread over many warps.
#include <algorithm>
#include <cmath>
#include <vector>

#include "cc_internal.h"
#include "cc_mlp.cuh"

using namespace ccg;

namespace {

constexpr unsigned TPB = 256;

// ================================================================ kernels
__global__ void __launch_bounds__(256, 8) k_iota(uint32_t *P, uint32_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        P[i] = (uint32_t)i;
}

__global__ void k_set_u32(uint32_t *p, uint32_t v) { *p = v; }
__global__ void k_or_u32(uint32_t *p, uint32_t v) { atomicOr(p, v); }

// Labels handed in by a caller must be a forest with P[v] <= v (sampled
// labels as cc_sample writes them satisfy it).  Out-of-range or increasing
// entries are flagged and reset to v so that every walk stays in bounds.
__global__ void __launch_bounds__(256, 8) k_check_forest(uint32_t *P, uint32_t n, Dev d) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t p = P[i];
        if (p > i) {
            atomicOr(d.err, ERR_BAD_EDGE);
            P[i] = (uint32_t)i;
        }
    }
}

// Point every vertex straight at its root: the full compression of
// Algorithm 4, the FullShortcut of Algorithm 15 / Appendix D, and the final
// shortcut to canonical labels (roots are component minima).  prev, when
// given, receives the new parents (the round-start snapshot of SV / LT).
// No link happens while it runs (only compression), so a root seen through
// L1 is a root and the walks use L1-cacheable loads; four vertices per
// thread step walk their chains in lock-step.  With COUNT, every non-root
// vertex also counts one for its root (IdentifyFrequent on flat labels, see
// identify_phase).
__device__ __forceinline__ void roots4(const uint32_t *P, uint32_t v0, uint32_t (&x)[4], uint32_t (&px)[4],
                                       const Dev &d, uint32_t *steps = nullptr) {
    bool act[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        x[j] = v0 + j;
        act[j] = px[j] != x[j];
    }
    Guard g;
    while (act[0] | act[1] | act[2] | act[3]) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (act[j]) {
                x[j] = px[j];
                px[j] = ld_ca(P + x[j]);
            }
#pragma unroll
        for (int j = 0; j < 4; ++j) act[j] = act[j] && px[j] != x[j];
        if (steps) *steps += (uint32_t)act[0] + act[1] + act[2] + act[3];
        if (!g.step(d)) break;
    }
}

// Full compression (FullShortcut).  COUNT: also count every non-root's
// root into cnt (the labels are then a flat forest) and leave the arg-max
// key (count << 32 | ~label, the largest count with ties to the smallest
// label) in *key, which must start at 0.
// The same walk over K vertices' chains at once.
template <int K>
__device__ __forceinline__ void rootsK(const uint32_t *P, uint32_t v0, uint32_t (&x)[K], uint32_t (&px)[K],
                                       const Dev &d) {
    bool act[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        x[j] = v0 + j;
        act[j] = px[j] != x[j];
    }
    Guard g;
    for (;;) {
        bool any = false;
#pragma unroll
        for (int j = 0; j < K; ++j) any |= act[j];
        if (!any) break;
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (act[j]) {
                x[j] = px[j];
                px[j] = ld_ca(P + x[j]);
            }
#pragma unroll
        for (int j = 0; j < K; ++j) act[j] = act[j] && px[j] != x[j];
        if (!g.step(d)) break;
    }
}

// Full compression alone (the union-find finish's final shortcut): eight
// consecutive vertices per thread step, two 16-byte loads and eight chains
// walked in lock-step, at six blocks per SM (40 registers, no spills).  The
// pass is bound by its dependent parent loads, so twice the vertices per
// step halves the steps a thread waits through: 0.080 -> 0.060 ms at R-MAT
// scale 26 after k-out, where most chains are one step.  (On the k-out
// mid-round compression, with longer chains, it measured 0.27 against
// 0.25 ms for k_shortcut.)  No link happens while it runs.  skip: as
// k_shortcut's.
__global__ void __launch_bounds__(256, 6) k_compress8(uint32_t *P, uint32_t n, Dev d,
                                                      const uint32_t *skip = nullptr) {
    if (skip && *skip) return;
    const uint64_t n8 = (reinterpret_cast<uintptr_t>(P) & 15) == 0 ? n / 8 : 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint64_t i = tid; i < n8; i += stride) {
        const uint4 a = __ldcg(reinterpret_cast<const uint4 *>(P) + 2 * i);
        const uint4 b = __ldcg(reinterpret_cast<const uint4 *>(P) + 2 * i + 1);
        uint32_t x[8], px[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        const uint32_t v0 = (uint32_t)(8 * i);
        rootsK<8>(P, v0, x, px, d);
        if (x[0] != a.x || x[1] != a.y || x[2] != a.z || x[3] != a.w)
            __stcg(reinterpret_cast<uint4 *>(P) + 2 * i, make_uint4(x[0], x[1], x[2], x[3]));
        if (x[4] != b.x || x[5] != b.y || x[6] != b.z || x[7] != b.w)
            __stcg(reinterpret_cast<uint4 *>(P) + 2 * i + 1, make_uint4(x[4], x[5], x[6], x[7]));
    }
    for (uint64_t v = 8 * n8 + tid; v < n; v += stride) {
        const uint32_t p = ld_rel(P + v);
        const uint32_t r = find_from<FIND_NAIVE>(P, (uint32_t)v, p, d);
        if (r != p) P[v] = r;
    }
}

// zero (may be null, 16-byte aligned): an n-word array this pass also
// clears (the count array of the next pass, cleared without a pass of its
// own while this one waits on its parent walks).  SPANS: the groups are
// taken in dynamic spans (counter pair `spans`), measured 28% faster for
// the k-out path's mid compression at R-MAT scale 26 but slower for the
// short rounds of SV / LT-PRF, which keep the static stride.
template <bool COUNT, bool SPANS = false>
__global__ void __launch_bounds__(256, 8) k_shortcut(uint32_t *P, uint32_t *prev, uint32_t n, uint32_t *cnt,
                                                     Dev d, unsigned long long *key = nullptr,
                                                     const uint32_t *skip = nullptr, uint32_t *zero = nullptr,
                                                     uint32_t *spans = nullptr) {
    if (skip && *skip) return;   // the selected path chose another finish
    // 16-byte vector accesses only when both arrays are 16-byte aligned (a
    // caller's label buffer may be any 4-byte-aligned slice)
    const bool vec = (reinterpret_cast<uintptr_t>(P) & 15) == 0 &&
                     (prev == nullptr || (reinterpret_cast<uintptr_t>(prev) & 15) == 0) &&
                     (zero == nullptr || (reinterpret_cast<uintptr_t>(zero) & 15) == 0);
    const uint64_t n4 = vec ? n / 4 : 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    LabelCounterArg lc;
    auto group = [&](uint64_t i) {
        uint4 p = __ldcg(reinterpret_cast<const uint4 *>(P) + i);
        uint32_t x[4], px[4] = {p.x, p.y, p.z, p.w};
        const uint32_t v0 = (uint32_t)(4 * i);
        roots4(P, v0, x, px, d);
        uint4 r = make_uint4(x[0], x[1], x[2], x[3]);
        if (r.x != p.x || r.y != p.y || r.z != p.z || r.w != p.w) __stcg(reinterpret_cast<uint4 *>(P) + i, r);
        if (prev) __stcg(reinterpret_cast<uint4 *>(prev) + i, r);
        if (zero) __stcg(reinterpret_cast<uint4 *>(zero) + i, make_uint4(0, 0, 0, 0));
        if (COUNT) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (x[j] != v0 + j) lc.add(cnt, x[j]);
        }
    };
    if constexpr (SPANS)
        warp_spans(spans, n4, 1024, [&](uint64_t i, bool act) {
            if (act) group(i);
        });
    else
        for (uint64_t i = tid; i < n4; i += stride) group(i);
    for (uint64_t v = 4 * n4 + tid; v < n; v += stride) {
        uint32_t p = ld_rel(P + v);
        uint32_t r = find_from<FIND_NAIVE>(P, (uint32_t)v, p, d);
        if (r != p) P[v] = r;
        if (prev) prev[v] = r;
        if (zero) zero[v] = 0;
        if (COUNT && r != v) lc.add(cnt, r);
    }
    if (COUNT) lc.flush(cnt, key);
}

// ---------------------------------------------------------------- degree statistics
// The degree statistics (FeatStats) of the selector's features, gathered
// by k_degree_stats on a second stream while the k-out sample runs.
struct DegStats {
    unsigned long long sd = 0, sd2 = 0, c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, e64 = 0, mk = 0;
    __device__ __forceinline__ void add(uint64_t deg, uint32_t v) {
        sd += deg;
        sd2 += deg * deg;
        c0 += deg == 0;
        c1 += deg == 1;
        c2 += deg == 2;
        c3 += deg >= 3 && deg <= 16;
        c4 += deg > 64;
        if (deg > 64) e64 += deg;
        const unsigned long long key = ((deg < 0xFFFFFFFFull ? deg : 0xFFFFFFFFull) << 32) | (uint32_t)~v;
        mk = key > mk ? key : mk;
    }
    // every thread of the block calls this once (it synchronises): warp
    // sums, then block sums in shared memory; thread 0 writes them to *out
    // with plain stores
    __device__ __forceinline__ void flush(FeatStats *out) {
        __shared__ unsigned long long bs[9];
        if (threadIdx.x < 9) bs[threadIdx.x] = 0;
        __syncthreads();
        unsigned long long c[5] = {c0, c1, c2, c3, c4};
        for (int o = 16; o > 0; o >>= 1) {
            sd += __shfl_xor_sync(0xFFFFFFFFu, sd, o);
            sd2 += __shfl_xor_sync(0xFFFFFFFFu, sd2, o);
            e64 += __shfl_xor_sync(0xFFFFFFFFu, e64, o);
            for (int j = 0; j < 5; ++j) c[j] += __shfl_xor_sync(0xFFFFFFFFu, c[j], o);
            const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, mk, o);
            mk = y > mk ? y : mk;
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&bs[0], sd);
            atomicAdd(&bs[1], sd2);
            atomicAdd(&bs[2], e64);
            for (int j = 0; j < 5; ++j) atomicAdd(&bs[3 + j], c[j]);
            atomicMax(&bs[8], mk);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            out->sum_deg = bs[0];
            out->sum_deg2 = bs[1];
            out->edges_gt64 = bs[2];
            for (int j = 0; j < 5; ++j) out->cnt[j] = bs[3 + j];
            out->maxkey = bs[8];
        }
    }
    // fold in another block's sums (the last block's total of the partials)
    __device__ __forceinline__ void merge(const FeatStats &f) {
        sd += f.sum_deg;
        sd2 += f.sum_deg2;
        e64 += f.edges_gt64;
        c0 += f.cnt[0];
        c1 += f.cnt[1];
        c2 += f.cnt[2];
        c3 += f.cnt[3];
        c4 += f.cnt[4];
        mk = f.maxkey > mk ? f.maxkey : mk;
    }
};

// One pass over the offsets: each block's partial sums go to its slot of
// part[] (plain stores); the last block to finish (a counter in done[0])
// adds the slots up, its threads taking slots in turn, into part[nparts],
// and resets the counter.  All sums are integers, so the total does not
// depend on the order.
template <typename OffT>
__global__ void __launch_bounds__(256, 4) k_degree_stats(const OffT *I, uint32_t n, uint64_t m, FeatStats *part,
                                                         uint32_t *done, Dev d) {
    DegStats ds;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t b, e;
        vertex_range(I, (uint32_t)v, m, b, e, d);
        ds.add(e - b, (uint32_t)v);
    }
    ds.flush(part + blockIdx.x);
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    DegStats tot;
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        FeatStats f;
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(part + b);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&f);
        for (int j = 0; j < (int)(sizeof(FeatStats) / 8); ++j) dst[j] = __ldcg(src + j);
        tot.merge(f);
    }
    tot.flush(part + gridDim.x);
    if (threadIdx.x == 0) *done = 0;
}

// ---------------------------------------------------------------- k-out
// Algorithm 4: each vertex of degree > 0 picks its first edge and k-1
// uniform random edges (with replacement; pick j of v draws
// out(seed ^ TAG_KOUT, v*k + j)), and each picked edge is a Union.  The
// picked edges are applied in two launches, picks [jb, je) each: the first
// edges, a full compression, then the random picks, whose unions then mostly
// find both endpoints already under one root (Afforest's schedule; the
// union-find result and the compressed labels are the same for any order).
// One vertex per thread step at full occupancy (launch bounds for eight
// 256-thread blocks per SM), with the next vertex's offsets prefetched.
constexpr int KOUT_MINB = 8;
// The first k-out pass keeps about 40 values live per thread (five offsets,
// four first edges, four picks and their positions): at eight blocks per
// SM it spilled 160-250 bytes per thread to local memory, so it runs at six
// (40 registers).
constexpr int HOOK_MINB = 6;
// The first k-out pass hands out its vertices in spans of up to
// KOUT_SPAN_MAX (eight warp steps of 128): a warp takes the next span from a
// counter when it has finished its last, so warps on faster SMs take more
// spans.  The span is the grid's share over four spans per warp, in whole
// warp steps, so a small graph still gives every warp work.  The first-edge
// queue has one region of `span` pairs per span, with the span's count
// beside it; the scratch is sized for the smallest span.
constexpr uint32_t KOUT_SPAN_MAX = 1024;
__host__ inline uint32_t kout_span_for(uint64_t n, uint64_t warps) {
    uint64_t s = n / (4 * warps) / 128 * 128;
    return (uint32_t)(s < 128 ? 128 : (s > KOUT_SPAN_MAX ? KOUT_SPAN_MAX : s));
}
__host__ inline uint64_t kout_spans_max(uint64_t n) { return (n + 127) / 128; }
__host__ inline uint64_t kout_defer_entries(uint64_t n) { return n + KOUT_SPAN_MAX; }

template <typename OffT, class E, int NB>
__global__ void __launch_bounds__(256, KOUT_MINB)
k_kout(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m, uint32_t k, uint32_t rule, uint64_t seed,
       uint32_t *P, Dev d, uint32_t jb, uint32_t je) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    // software pipeline: the next vertex's offsets are in flight while the
    // current vertex's edges and parents are read
    uint64_t o0 = 0, o1 = 0;
    if (v < n) { o0 = ld_off(I + v); o1 = ld_off(I + v + 1); }
    for (; v < n; v += stride) {
        const uint64_t vn = v + stride;
        uint64_t n0 = 0, n1 = 0;
        if (vn < n) { n0 = ld_off(I + vn); n1 = ld_off(I + vn + 1); }
        uint64_t b = 0, e = 0;
        clamp_range(o0, o1, m, b, e, d);
        const uint64_t deg = e - b;
        o0 = n0;
        o1 = n1;
        if (deg == 0) continue;
        for (uint32_t j0 = jb; j0 < je; j0 += NB) {
            uint32_t u[NB], w[NB];
            bool ok[NB];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const uint32_t pick = j0 + q;
                u[q] = (uint32_t)v;
                const uint64_t off = pick < je ? kout_offset(rule, seed, v, k, pick, deg) : NO_PICK;
                ok[q] = off != NO_PICK;
                w[q] = ok[q] ? ld_stream(A + b + off) : u[q];
                if (ok[q] && w[q] >= n) { atomicOr(d.err, ERR_BAD_EDGE); ok[q] = false; }
                if (ok[q] && w[q] == u[q]) ok[q] = false;
            }
            unite_pairs<E, NB>(P, u, w, ok, d);
        }
    }
}

// picks per thread step: one when a round has a single pick (k = 2), else four
template <typename OffT, class E>
void launch_kout(unsigned grid, cudaStream_t s, const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                 uint32_t k, uint32_t rule, uint64_t seed, uint32_t *P, Dev d, uint32_t jb, uint32_t je) {
    if (je - jb == 1) k_kout<OffT, E, 1><<<grid, 256, 0, s>>>(I, A, n, m, k, rule, seed, P, d, jb, je);
    else k_kout<OffT, E, 4><<<grid, 256, 0, s>>>(I, A, n, m, k, rule, seed, P, d, jb, je);
}

// First edges, part one (replaces the identity initialisation): each
// vertex v reads its first edge (v, w0).  If w0 < v, v is linked under w0
// with a plain store: in this pass only v's thread writes P[v], so v is
// still a root and the link keeps P[x] <= x.  Otherwise P[v] = v, and a
// vertex with w0 > v (all its neighbours larger) is queued for a real Union
// in part two as the pair (v, w0), so part two reads no offsets or edges.
// Warps take spans of `span` vertices (a multiple of 128): a warp's first
// span is its index in the grid, the rest come from *span_ctr (zero at
// launch; the next index asked for when a span starts, and only when the
// spans outnumber the warps); a span's queued pairs go to its own region of
// the queue (defer + its index * span, at most one per vertex) and their
// number to dcount[index], counted by the warp itself.
// (With static steps the busiest SM ran 16% above the mean; one global
// queue counter hit by every warp step serialised at the L2, about 2 ns per
// atomic, 0.5M of them at RMAT-26.)
template <typename OffT>
__global__ void __launch_bounds__(256, HOOK_MINB) k_kout_hook_first(const OffT *I, const uint32_t *A, uint32_t n,
                                                            uint64_t m, uint32_t *P, uint2 *defer,
                                                            uint32_t *dcount, uint32_t *span_ctr, uint32_t span_len,
                                                            uint32_t *pick1, uint32_t k, uint32_t rule, uint64_t seed,
                                                            uint32_t *nz, Dev d) {
    const int lane = threadIdx.x & 31;
    const uint32_t nspan = (uint32_t)(((uint64_t)n + span_len - 1) / span_len);
    // A warp step covers 128 consecutive vertices as four groups of 32;
    // lane L owns vertex base + 32j + L, so each load instruction touches a
    // contiguous stretch of offsets, first edges and labels.
    // o[j] = I[base + 32j + L] (j < 4), o[4] = I[base + 128 + L].
    uint64_t o[5];
    auto load = [&](uint64_t bs) {
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            const uint64_t idx = bs + 32 * j + lane;
            o[j] = idx <= n ? (uint64_t)ld_off(I + idx) : 0;
        }
    };
    // a warp's first span is its index in the grid; the counter hands out
    // the rest (none when the spans do not outnumber the warps)
    const uint32_t nwg = (gridDim.x * blockDim.x) >> 5;
    const bool dynamic = nspan > nwg;   // grid-uniform
    uint32_t span = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (span < nspan) load((uint64_t)span * span_len);
    while (span < nspan) {
        uint32_t next = nspan;
        if (dynamic && lane == 0) next = nwg + atomicAdd(span_ctr, 1u);
        uint2 *my_defer = defer + (uint64_t)span * span_len;
        uint32_t queued = 0;   // the span's queued pairs so far (warp-uniform)
        const uint64_t s0 = (uint64_t)span * span_len;
        const uint64_t s1 = s0 + span_len < n ? s0 + span_len : n;
        for (uint64_t base = s0; base < s1; base += 128) {
            uint64_t beg[4], end[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t nxt = __shfl_down_sync(0xFFFFFFFFu, o[j], 1);
                const uint64_t first = __shfl_sync(0xFFFFFFFFu, o[j + 1], 0);
                beg[j] = o[j];
                end[j] = lane < 31 ? nxt : first;
            }
            uint32_t w[4], r[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t v = base + 32 * j + lane;
                uint64_t b = 0, e = 0;
                if (v < n) clamp_range(beg[j], end[j], m, b, e, d);
                // nz (optional): bit v set iff v has an edge, one word per
                // 32 consecutive vertices (the later binning skips isolated
                // vertices without reading their offsets)
                const unsigned has = __ballot_sync(0xFFFFFFFFu, e > b);
                if (nz && lane == 0 && base + 32 * j < n) nz[(base >> 5) + j] = has;
                // pick 0 (the first edge, or a uniform pick under the pure rule)
                w[j] = e > b ? ld_stream(A + b + kout_offset(rule, seed, v, k, 0, e - b)) : NONE;
                // with k = 2 pick 1 is read here too and kept for the second
                // round, so that round reads no offsets or edges
                r[j] = NONE;
                if (pick1 && e > b) {
                    const uint64_t off = kout_offset(rule, seed, v, 2, 1, e - b);
                    if (off != NO_PICK) r[j] = ld_stream(A + b + off);
                }
            }
            // the next step's offsets load while this step's first edges are
            // read: the span's next step, or the first step of the next span
            if (base + 128 < s1) {
                load(base + 128);
            } else {
                const uint32_t nsp = __shfl_sync(0xFFFFFFFFu, next, 0);
                if (nsp < nspan) load((uint64_t)nsp * span_len);
            }
            uint32_t nd = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t v = base + 32 * j + lane;
                if (w[j] != NONE && w[j] >= n) { atomicOr(d.err, ERR_BAD_EDGE); w[j] = NONE; }
                if (v < n) P[v] = (w[j] != NONE && w[j] < v) ? w[j] : (uint32_t)v;
                if (d.forest && v < n && w[j] != NONE && w[j] < v) d.forest[v] = make_uint2((uint32_t)v, w[j]);
                nd += (w[j] != NONE && w[j] > v);
                if (pick1 && v < n) {
                    if (r[j] != NONE && r[j] >= n) { atomicOr(d.err, ERR_BAD_EDGE); r[j] = NONE; }
                    pick1[v] = r[j] == (uint32_t)v ? NONE : r[j];
                }
            }
            // the lane's slots in the span's region: an exclusive scan of the
            // lanes' counts after the pairs queued so far
            uint32_t incl = nd;
#pragma unroll
            for (int o2 = 1; o2 < 32; o2 <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o2);
                if (lane >= o2) incl += t;
            }
            uint32_t slot = queued + incl - nd;
            queued += __shfl_sync(0xFFFFFFFFu, incl, 31);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (w[j] != NONE && w[j] > base + 32 * j + lane) {
                    if (slot < span_len) my_defer[slot] = make_uint2((uint32_t)(base + 32 * j + lane), w[j]);
                    else atomicOr(d.err, ERR_NONCONVERGED);
                    ++slot;
                }
        }
        if (lane == 0) dcount[span] = queued < span_len ? queued : span_len;
        span = __shfl_sync(0xFFFFFFFFu, next, 0);
    }
}

// First edges, part two: Union(v, w0) for the queued (v, w0) pairs, one
// warp per span region (`regions` of them, `cap` pairs apart, dcount[r]
// used).  Block 0 then clears the first pass's span counter.
template <class E>
__global__ void __launch_bounds__(256, KOUT_MINB)
k_kout_defer(uint32_t n, uint32_t *P, const uint2 *defer, const uint32_t *dcount, uint32_t regions, uint32_t cap,
             uint32_t *span_ctr, Dev d) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && span_ctr) *span_ctr = 0;
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t r = warp; r < regions; r += nw) {
        const uint32_t total = dcount[r];
        const uint2 *q0 = defer + (uint64_t)r * cap;
        for (uint32_t i = lane; i < total; i += 32) {
            const uint2 q = q0[i];
            uint32_t u1[1] = {q.x}, w1[1] = {q.y};
            bool ok[1] = {q.y < n && q.y != q.x};
            unite_pairs<E, 1>(P, u1, w1, ok, d);
        }
    }
}

// Second round for k = 2: Union(v, pick1[v]) from the stash written in the
// first pass (coalesced reads of the stash and of P[v]).  (Zeroing the
// stash here, to reuse it as the count array, made this kernel 12x slower:
// 2.93 against 0.24 ms at R-MAT scale 26; the count array is cleared by the
// mid-round compression instead.)
template <class E>
__global__ void __launch_bounds__(256, 8) k_kout_apply_pick(const uint32_t *pick1, uint32_t n, uint32_t *P, Dev d) {
    // four consecutive vertices per thread step (one 16-byte stash load),
    // their eight parent loads in flight together
    const uint64_t n4 = (reinterpret_cast<uintptr_t>(pick1) & 15) == 0 ? n / 4 : 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint64_t i = tid; i < n4; i += stride) {
        const uint4 q = __ldcs(reinterpret_cast<const uint4 *>(pick1) + i);
        const uint32_t v0 = (uint32_t)(4 * i);
        uint32_t u4[4] = {v0, v0 + 1, v0 + 2, v0 + 3}, w4[4] = {q.x, q.y, q.z, q.w};
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) ok[j] = w4[j] != NONE;
        unite_pairs<E, 4>(P, u4, w4, ok, d);
    }
    for (uint64_t v = 4 * n4 + tid; v < n; v += stride) {
        const uint32_t w = pick1[v];
        uint32_t u1[1] = {(uint32_t)v}, w1[1] = {w};
        bool ok[1] = {w != NONE};
        unite_pairs<E, 1>(P, u1, w1, ok, d);
    }
}

// ---------------------------------------------------------------- IdentifyFrequent
// Exact: count every label into a count array (register heavy-hitter slots
// keep the frequent label's atomics off one address), then the arg-max with
// ties to the smallest label via a packed 64-bit max key
// (count << 32 | ~label).
// FLAT: the labels are a flat forest (label[v] = root of v, every root its
// own label, vertex 0 a root), as sampling leaves them.  Then a root's count
// is 1 + its non-root members and a non-root label counts 0, so the arg-max
// (ties to the smallest) is unchanged when only non-root vertices are
// counted; with none, every root ties at 1 and the answer is root 0.
template <bool FLAT>
__global__ void __launch_bounds__(256, 8) k_count_labels(const uint32_t *L, uint32_t n, uint32_t *cnt, Dev d,
                                                          const uint32_t *only_if = nullptr) {
    if (only_if && *only_if == 0) return;
    const uint64_t n4 = (reinterpret_cast<uintptr_t>(L) & 15) == 0 ? n / 4 : 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    LabelCounter lc;
    for (uint64_t i = tid; i < n4; i += stride) {
        uint4 q = __ldcs(reinterpret_cast<const uint4 *>(L) + i);
        uint32_t l[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (l[j] >= n) atomicOr(d.err, ERR_BAD_EDGE);
            else if (!FLAT || l[j] != 4 * i + j) lc.add(cnt, l[j]);
        }
    }
    for (uint64_t v = 4 * n4 + tid; v < n; v += stride) {
        uint32_t l = L[v];
        if (l >= n) atomicOr(d.err, ERR_BAD_EDGE);
        else if (!FLAT || l != v) lc.add(cnt, l);
    }
    lc.flush(cnt);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, x, o);
        x = y > x ? y : x;
    }
    return x;
}

__device__ __forceinline__ void keep_max(unsigned long long &best, uint32_t c, uint64_t i) {
    if (c) {
        unsigned long long k2 = ((unsigned long long)c << 32) | (uint32_t)~(uint32_t)i;
        best = k2 > best ? k2 : best;
    }
}

__global__ void __launch_bounds__(256, 8) k_argmax_counts(const uint32_t *cnt, uint32_t n, unsigned long long *key,
                                                           const uint32_t *only_if = nullptr) {
    if (only_if && *only_if == 0) return;
    __shared__ unsigned long long s[32];
    unsigned long long best = 0;
    const uint64_t n4 = (reinterpret_cast<uintptr_t>(cnt) & 15) == 0 ? n / 4 : 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint64_t i = tid; i < n4; i += stride) {
        uint4 c = __ldcs(reinterpret_cast<const uint4 *>(cnt) + i);
        keep_max(best, c.x, 4 * i);
        keep_max(best, c.y, 4 * i + 1);
        keep_max(best, c.z, 4 * i + 2);
        keep_max(best, c.w, 4 * i + 3);
    }
    for (uint64_t i = 4 * n4 + tid; i < n; i += stride) keep_max(best, cnt[i], i);
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0;
        best = warp_max_u64(best);
        if (threadIdx.x == 0 && best) atomicMax(key, best);
    }
}

// (an empty key only arises from flat counting with no non-root vertex,
// where every root ties and the smallest, vertex 0, wins)
__global__ void k_key_to_label(const unsigned long long *key, uint32_t *lmax) {
    unsigned long long k = *key;
    *lmax = k ? ~(uint32_t)(k & 0xFFFFFFFFull) : 0u;
}

// Estimate: the labels at S seeded positions out(seed ^ TAG_FREQ, i) mod n,
// counted in one block (S <= 4096 fits in shared memory).
__global__ void k_freq_sampled(const uint32_t *L, uint32_t n, uint32_t S, uint64_t seed, uint32_t *lmax) {
    __shared__ uint32_t lab[4096];
    __shared__ unsigned long long red[32];
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x)
        lab[i] = L[draw64(seed ^ TAG_FREQ, i) % n];
    __syncthreads();
    unsigned long long best = 0;
    for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) {
        uint32_t l = lab[i], c = 0;
        for (uint32_t j = 0; j < S; ++j) c += lab[j] == l;
        unsigned long long k2 = ((unsigned long long)c << 32) | (uint32_t)~l;
        best = k2 > best ? k2 : best;
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        best = warp_max_u64(best);
        if (threadIdx.x == 0) *lmax = best ? ~(uint32_t)(best & 0xFFFFFFFFull) : NONE;
    }
}

// ---------------------------------------------------------------- fused k-out binning
// A guess of L_max before the exact count: the most frequent root among 128
// seeded vertices that have an edge (ties to the smallest root), each root
// found by walking the not yet compressed forest (at most 64 steps; a walk
// that stops early just gives a worse guess).  One block of 128 threads.
// The guess only decides which vertices the fused binning treats as
// candidates; the exact L_max is checked against it afterwards.
constexpr uint64_t TAG_GUESS = 0x67756573ull;
__global__ void __launch_bounds__(128) k_guess_lmax(const uint32_t *P, const uint32_t *nz, uint32_t n, uint64_t seed,
                                                    Ctl *ctl) {
    // the fused pass appends and counts from zero
    if (threadIdx.x == 0) {
        ctl->nlight = 0;
        ctl->nchunks = 0;
        ctl->edges = 0;
        ctl->key = 0;
        ctl->rebin = 0;
        ctl->nonroots = 0;
        ctl->steps = 0;
        ctl->gcount = 0;
    }
    __shared__ uint32_t lab[128];
    __shared__ unsigned long long red[4];
    const uint32_t t = threadIdx.x;
    const uint32_t v = (uint32_t)(draw64(seed ^ TAG_GUESS, t) % n);
    uint32_t r = NONE;
    if ((nz[v >> 5] >> (v & 31)) & 1u) {
        r = v;
        for (int step = 0; step < 64; ++step) {
            const uint32_t p = ld_rel(P + r);
            if (p == r || p >= n) break;
            r = p;
        }
    }
    lab[t] = r;
    __syncthreads();
    unsigned long long best = 0;
    if (r != NONE) {
        uint32_t c = 0;
        for (int j = 0; j < 128; ++j) c += lab[j] == r;
        best = ((unsigned long long)c << 32) | (uint32_t)~r;
    }
    best = warp_max_u64(best);
    if ((t & 31) == 0) red[t >> 5] = best;
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < 4; ++w) best = red[w] > best ? red[w] : best;
        best = best > red[0] ? best : red[0];
        ctl->guess = best ? ~(uint32_t)(best & 0xFFFFFFFFull) : NONE;
    }
}

// The k-out sampling's last full compression, fused with IdentifyFrequent's
// count (non-roots counted into cnt, the arg-max key left in ctl->key) and
// with the finish's candidate binning (Algorithm 7's filter) against the
// guessed L_max: a vertex whose root differs from the guess and that has an
// edge (nz bit) is binned, light (degree <= LIGHT_MAX) to the light list,
// heavier as chunks.  Only candidates read offsets, so on a graph with a
// giant cluster this pass replaces the binning pass's read of every offset
// and label.  When the exact L_max differs from the guess (k_lmax_check)
// the lists are rebuilt by k_cand_bin.
template <typename OffT>
__global__ void __launch_bounds__(256, 6) k_compress_count_bin(uint32_t *P, uint32_t n, const OffT *I,
                                                               uint64_t m, const uint32_t *nz, Ctl *ctl,
                                                               uint32_t *light, ChunkRef *chunks, uint64_t cap,
                                                               Dev d) {
    const bool vec = (reinterpret_cast<uintptr_t>(P) & 15) == 0;
    const uint64_t n4 = vec ? n / 4 : 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint32_t guess = ctl->guess;
    const int lane = threadIdx.x & 31;
    WarpSlots ws;
    unsigned long long my_edges = 0, my_nonroots = 0, my_guess = 0;
    uint32_t my_steps = 0;
    // whole warps iterate together (the binning's appends are
    // warp-collective), taking groups of four vertices in dynamic spans
    warp_spans(ctl->spans[1], n4, 1024, [&](uint64_t i, bool act) {
        uint32_t x[4], px[4];
        const uint32_t v0 = (uint32_t)(4 * i);
        uint32_t nc[4] = {0, 0, 0, 0}, isl[4] = {0, 0, 0, 0};
        if (act) {
            uint4 p = __ldcg(reinterpret_cast<const uint4 *>(P) + i);
            px[0] = p.x; px[1] = p.y; px[2] = p.z; px[3] = p.w;
            roots4(P, v0, x, px, d, &my_steps);
            uint4 r = make_uint4(x[0], x[1], x[2], x[3]);
            if (r.x != p.x || r.y != p.y || r.z != p.z || r.w != p.w) __stcg(reinterpret_cast<uint4 *>(P) + i, r);
            const uint32_t bits = (nz[v0 >> 5] >> (v0 & 31)) & 15u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (x[j] != v0 + j) {
                    ++my_nonroots;
                    my_guess += x[j] == guess;
                }
                if (x[j] != guess && ((bits >> j) & 1u)) {
                    uint64_t b, e;
                    vertex_range(I, v0 + j, m, b, e, d);
                    const uint64_t deg = e - b;
                    my_edges += deg;
                    isl[j] = deg > 0 && deg <= LIGHT_MAX;
                    nc[j] = deg > LIGHT_MAX ? (uint32_t)((deg + CHUNK - 1) / CHUNK) : 0;
                }
            }
        }
        const uint32_t nls = isl[0] + isl[1] + isl[2] + isl[3], ncs = nc[0] + nc[1] + nc[2] + nc[3];
        // most warp steps of a graph with a giant cluster have no candidate
        if (!__any_sync(0xFFFFFFFFu, nls | ncs)) return;   // warp-uniform
        uint32_t sl = warp_append_full(&ctl->nlight, nls);
        uint32_t incl = ncs;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        uint64_t sc = tot ? ws.take(&ctl->nchunks, tot, chunks, cap) + incl - ncs : 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (isl[j]) light[sl++] = v0 + j;
            if (nc[j]) {
                if (sc + nc[j] > cap) atomicOr(d.err, ERR_NONCONVERGED);
                else
                    for (uint32_t c = 0; c < nc[j]; ++c) chunks[sc + c] = ChunkRef{v0 + j, c};
                sc += nc[j];
            }
        }
    });
    // the last n % 4 vertices (all of them when P is not 16-byte aligned),
    // one per thread: single appends
    for (uint64_t v = 4 * n4 + tid; v < n; v += stride) {
        uint32_t p = ld_rel(P + v);
        uint32_t r = find_from<FIND_NAIVE>(P, (uint32_t)v, p, d);
        if (r != p) P[v] = r;
        if (r != v) {
            ++my_nonroots;
            my_guess += r == guess;
        }
        if (r != guess && ((nz[v >> 5] >> (v & 31)) & 1u)) {
            uint64_t b, e;
            vertex_range(I, (uint32_t)v, m, b, e, d);
            const uint64_t deg = e - b;
            my_edges += deg;
            if (deg > 0 && deg <= LIGHT_MAX) {
                light[atomicAdd(&ctl->nlight, 1u)] = (uint32_t)v;
            } else if (deg > LIGHT_MAX) {
                const uint32_t ncv = (uint32_t)((deg + CHUNK - 1) / CHUNK);
                const uint64_t sc = atomicAdd(&ctl->nchunks, ncv);
                if (sc + ncv > cap) atomicOr(d.err, ERR_NONCONVERGED);
                else
                    for (uint32_t c = 0; c < ncv; ++c) chunks[sc + c] = ChunkRef{(uint32_t)v, c};
            }
        }
    }
    ws.close(chunks, cap);
    unsigned long long my_st = my_steps;
    for (int o = 16; o > 0; o >>= 1) {
        my_edges += __shfl_xor_sync(0xFFFFFFFFu, my_edges, o);
        my_nonroots += __shfl_xor_sync(0xFFFFFFFFu, my_nonroots, o);
        my_guess += __shfl_xor_sync(0xFFFFFFFFu, my_guess, o);
        my_st += __shfl_xor_sync(0xFFFFFFFFu, my_st, o);
    }
    if (lane == 0) {
        if (my_edges) atomicAdd(&ctl->edges, my_edges);
        if (my_nonroots) atomicAdd(&ctl->nonroots, my_nonroots);
        if (my_guess) atomicAdd(&ctl->gcount, my_guess);
        if (my_st) atomicAdd(&ctl->steps, my_st);
    }
}

// Exact L_max without counting every label, when possible: the fused pass
// counted the non-root vertices under the guess (gcount) and all non-root
// vertices.  If the guess holds more than half of them, every other root
// counts less, so the guess is the arg-max (no tie possible) and its key is
// written; otherwise `fallback` is set and the guarded count kernels
// (k_zero_if, k_count_labels, k_argmax_counts) find the key.
__global__ void k_lmax_majority(Ctl *ctl) {
    const unsigned long long gc = ctl->gcount, nr = ctl->nonroots;
    const bool maj = ctl->guess != NONE && 2 * gc > nr;
    ctl->fallback = !maj;
    ctl->key = maj ? ((gc << 32) | (uint32_t)~ctl->guess) : 0ull;
}

__global__ void __launch_bounds__(256, 8) k_zero_if(uint32_t *a, uint32_t n, const uint32_t *only_if) {
    if (*only_if == 0) return;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        a[i] = 0;
}

// L_max from the arg-max key; when it is not the guess the fused binning
// used, the lists are cleared and rebin is set (k_cand_bin then rebuilds
// them against the exact L_max).
__global__ void k_lmax_check(Ctl *ctl, uint32_t *lmax) {
    const unsigned long long k = ctl->key;
    const uint32_t l = k ? ~(uint32_t)(k & 0xFFFFFFFFull) : 0u;
    *lmax = l;
    const bool re = l != ctl->guess;
    ctl->rebin = re;
    if (re) {
        ctl->nlight = 0;
        ctl->nchunks = 0;
        ctl->edges = 0;
    }
}

// The selector's choice inside the default path (k-out + UF-Rem-CAS): the
// L_max check of k_lmax_check, then the 16 features from what the default
// path already computed, then the MLP's class, all in one block of 64
// threads.  The degree statistics come from k_degree_stats (a second
// stream, joined before this kernel).
// Features (floats): 0 log2(n+1), 1 log2(m+1), 2 m/n, 3 log2(max degree+1),
// 4 degree variance / mean^2, 5-7 fractions of vertices of degree 0, 1, 2,
// 8 fraction of degree 3..16, 9 fraction of degree > 64, 10 share of edges
// at vertices of degree > 64, 11 size of L_max's k-out cluster / n, 12
// vertices outside their own singleton after k-out / n, 13 edges left for
// the finish / m, 14 light candidate vertices of the finish / n, 15 parent
// steps per non-root in the last compression (how deep the k-out trees
// were, a cheap stand-in for the graph's depth).  params null: features
// only, class 0 (the default).  force >= 0 overrides the class.  The class
// goes to ctl->sel_class and, with rebin in bit 8, to *host_word (mapped
// host memory, may be null); ctl->skip = class != 0.
__global__ void __launch_bounds__(64) k_lmax_select(Ctl *ctl, uint32_t *lmax, const FeatStats *fs, uint32_t n,
                                                    uint64_t m, const float *params, int force, float *feat_out,
                                                    volatile int *host_word) {
    __shared__ float xin[MLP_IN], x[MLP_IN], h1[MLP_H], h2[MLP_H], z[MLP_OUT];
    __shared__ unsigned long long red[2][8];
    __shared__ double red2[2];
    __shared__ unsigned long long k_s, nonroots_s, edges_s, nlight_s, steps_s;
    __shared__ uint32_t re_s;
    const int t = threadIdx.x;
    // degree statistics, summed by k_degree_stats's last block
    if (t == 0) {
        const FeatStats f = *fs;
        red[0][0] = f.sum_deg;
        for (int j = 0; j < 5; ++j) red[0][1 + j] = f.cnt[j];
        red[0][6] = f.edges_gt64;
        red[0][7] = f.maxkey;
        red2[0] = (double)f.sum_deg2;
        for (int j = 0; j < 8; ++j) red[1][j] = 0;
        red2[1] = 0.0;
    }
    if (t == 0) {
        const unsigned long long k = ctl->key;
        const uint32_t l = k ? ~(uint32_t)(k & 0xFFFFFFFFull) : 0u;
        *lmax = l;
        k_s = k;
        nonroots_s = ctl->nonroots;
        edges_s = ctl->edges;
        nlight_s = ctl->nlight;
        steps_s = ctl->steps;
        const bool re = l != ctl->guess;
        ctl->rebin = re;
        re_s = re;
        if (re) {
            ctl->nlight = 0;
            ctl->nchunks = 0;
            ctl->edges = 0;
        }
    }
    __syncthreads();
    if (t < MLP_IN) {
        const float nn = (float)n, mm = m ? (float)m : 1.f;
        const unsigned long long sd = red[0][0] + red[1][0];
        const float mean = (float)sd / nn;
        float v = 0.f;
        switch (t) {
            case 0: v = log2f(nn + 1.f); break;
            case 1: v = log2f((float)m + 1.f); break;
            case 2: v = mean; break;
            case 3: {
                const unsigned long long mk = red[0][7] > red[1][7] ? red[0][7] : red[1][7];
                v = log2f((float)(mk >> 32) + 1.f);
                break;
            }
            case 4: {   // in double: the difference cancels on regular graphs
                const double md = (double)sd / (double)n, var = (red2[0] + red2[1]) / (double)n - md * md;
                v = md > 0.0 ? (float)(var / (md * md)) : 0.f;
                break;
            }
            case 5: case 6: case 7: case 8: case 9:
                v = (float)(red[0][t - 4] + red[1][t - 4]) / nn; break;
            case 10: v = (float)(red[0][6] + red[1][6]) / mm; break;
            case 11: v = ((float)(k_s >> 32) + 1.f) / nn; break;
            case 12: v = (float)nonroots_s / nn; break;
            case 13: v = (float)edges_s / mm; break;
            case 14: v = (float)nlight_s / nn; break;
            default: v = (float)steps_s / (nonroots_s > 1 ? (float)nonroots_s : 1.f); break;
        }
        xin[t] = v;
        if (feat_out) feat_out[t] = v;
    }
    __syncthreads();
    int cls = 0;
    if (params) {
        mlp_forward_one(params, xin, x, h1, h2, z);
        __syncthreads();
        cls = mlp_argmax(z);
    }
    if (force >= 0) cls = force;
    if (t == 0) {
        ctl->sel_class = (uint32_t)cls;
        ctl->skip = cls != 0;
        if (host_word) {
            *host_word = cls | ((int)re_s << 8);
            __threadfence_system();
        }
    }
}

// ---------------------------------------------------------------- edge passes
// The edge passes inline a union (or a frontier claim) per edge and keep a
// warp's chunk reservation live: at eight 256-thread blocks per SM (32
// registers) they spilled 70-280 bytes per thread to local memory, so they
// run at six (40 registers) on grids of one wave at that occupancy.  (The
// LDD passes and the light-vertex walks k_range_bin and k_light_list stay
// at eight: measured, on LDD and on graphs of light vertices (grids,
// G(n, M)) their latency hiding gains more from the warps than they lose to
// the spills.)
constexpr int EDGE_MINB = 6;
// Edge pass over a vertex range (union-find finish with nothing skipped, or
// a skip test on P[u] == L_max): light vertices run in the calling thread;
// heavier ones are cut into chunks for k_chunks.
template <typename OffT, class F>
__global__ void __launch_bounds__(256, 8) k_range_bin(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m, const uint32_t *P,
                            const uint32_t *lmax_p, F f, ChunkRef *chunks, uint32_t *nchunks,
                            uint64_t cap, unsigned long long *edges, Dev d) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t lmax = lmax_p ? *lmax_p : NONE;
    unsigned long long my_edges = 0;
    WarpSlots ws;
    for (uint64_t base = warp * 32; base < n; base += nw * 32) {
        uint32_t u = (uint32_t)(base + lane);
        bool act = base + lane < n;
        uint64_t b = 0, e = 0;
        if (act && lmax != NONE && ld_rel(P + u) == lmax) act = false;
        if (act) vertex_range(I, u, m, b, e, d);
        uint64_t deg = e - b;
        my_edges += deg;
        uint32_t nc = deg > LIGHT_MAX ? (uint32_t)((deg + CHUNK - 1) / CHUNK) : 0;
        warp_bin_chunks(ws, nchunks, chunks, cap, nc, u, d);
        warp_light_edges(u, b, nc ? 0u : (uint32_t)deg, A, n, f, d);
    }
    ws.close(chunks, cap);
    f.flush();
    for (int o = 16; o > 0; o >>= 1) my_edges += __shfl_xor_sync(0xFFFFFFFFu, my_edges, o);
    if (lane == 0 && edges && my_edges) atomicAdd(edges, my_edges);
}

template <typename OffT, class F>
__global__ void __launch_bounds__(256, EDGE_MINB) k_chunks(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m, const ChunkRef *chunks,
                         const uint32_t *nchunks, uint64_t cap, F f, Dev d, const uint32_t *skip = nullptr) {
    if (skip && *skip) return;
    run_chunks(I, A, n, m, chunks, nchunks, cap, f, d);
    f.flush();
}

// Vertex list (BFS / LDD frontiers): light vertices inline, heavier ones to
// the chunk list.
template <typename OffT, class F>
__global__ void __launch_bounds__(256, EDGE_MINB) k_list_bin(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m, const uint32_t *list,
                           const uint32_t *count, F f, ChunkRef *chunks, uint32_t *nchunks, uint64_t cap,
                           Dev d) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t total = *count;
    WarpSlots ws;
    for (uint64_t base = warp * 32; base < total; base += nw * 32) {
        bool act = base + lane < total;
        uint32_t u = act ? list[base + lane] : 0;
        uint64_t b = 0, e = 0;
        if (act) vertex_range(I, u, m, b, e, d);
        uint64_t deg = e - b;
        uint32_t nc = deg > LIGHT_MAX ? (uint32_t)((deg + CHUNK - 1) / CHUNK) : 0;
        warp_bin_chunks(ws, nchunks, chunks, cap, nc, u, d);
        warp_light_edges(u, b, nc ? 0u : (uint32_t)deg, A, n, f, d);
    }
    ws.close(chunks, cap);
    f.flush();
}

// Candidates of SV / LT (Algorithm 15's candidate set): vertices whose
// sampled label is not L_max and that have edges; light ones to a list,
// heavy ones to the chunk list.  Built once, reused every round.
template <typename OffT>
__global__ void __launch_bounds__(256, EDGE_MINB) k_cand_bin(const OffT *I, uint32_t n, uint64_t m, const uint32_t *P, const uint32_t *lmax_p,
                           uint32_t *light, uint32_t *nlight, ChunkRef *chunks, uint32_t *nchunks, uint64_t cap,
                           unsigned long long *edges, Dev d, const uint32_t *only_if = nullptr,
                           const uint32_t *skip = nullptr) {
    // only_if: the lists were built by the fused k-out pass; rebuild them
    // only when that pass's L_max guess was wrong.  skip: the selected path
    // chose another finish (which rebuilds them itself if needed)
    if ((only_if && *only_if == 0) || (skip && *skip)) return;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t lmax = lmax_p ? *lmax_p : NONE;
    unsigned long long my_edges = 0;
    WarpSlots ws;
    // a warp step covers 128 vertices, four per lane, read with vector loads
    for (uint64_t base = warp * 128; base < n; base += nw * 128) {
        const uint64_t v0 = base + 4 * lane;
        uint32_t pl[4];
        uint64_t o[5];
        load_labels4(P, v0, n, pl);
        load_offsets5(I, v0, n, o);
        uint32_t nl = 0, ncs = 0, nc[4];
        uint64_t bb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint64_t b = 0, e = 0;
            bool act = v0 + j < n && !(lmax != NONE && pl[j] == lmax);
            if (act) clamp_range(o[j], o[j + 1], m, b, e, d);
            uint64_t deg = e - b;
            my_edges += deg;
            bb[j] = deg;
            nl += (deg > 0 && deg <= LIGHT_MAX);
            nc[j] = deg > LIGHT_MAX ? (uint32_t)((deg + CHUNK - 1) / CHUNK) : 0;
            ncs += nc[j];
        }
        uint32_t sl = warp_append_full(nlight, nl);
        // the lane's chunks, in vertex order, from the warp's reservation
        uint32_t incl = ncs;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        uint64_t sc = tot ? ws.take(nchunks, tot, chunks, cap) + incl - ncs : 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (bb[j] > 0 && bb[j] <= LIGHT_MAX) light[sl++] = (uint32_t)(v0 + j);
            if (nc[j]) {
                if (sc + nc[j] > cap) atomicOr(d.err, ERR_NONCONVERGED);
                else
                    for (uint32_t c = 0; c < nc[j]; ++c) chunks[sc + c] = ChunkRef{(uint32_t)(v0 + j), c};
                sc += nc[j];
            }
        }
    }
    ws.close(chunks, cap);
    for (int o = 16; o > 0; o >>= 1) my_edges += __shfl_xor_sync(0xFFFFFFFFu, my_edges, o);
    if (lane == 0 && edges && my_edges) atomicAdd(edges, my_edges);
}

template <typename OffT, class F>
__global__ void __launch_bounds__(256, 8) k_light_list(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m, const uint32_t *list,
                             const uint32_t *count, F f, Dev d, const uint32_t *skip = nullptr) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t total = *count;
    for (uint64_t base = warp * 32; base < total; base += nw * 32) {
        const bool act = base + lane < total;
        const uint32_t u = act ? list[base + lane] : 0;
        uint64_t b = 0, e = 0;
        if (act) vertex_range(I, u, m, b, e, d);
        // the list holds light vertices only; a longer range (malformed
        // offsets) is cut to LIGHT_MAX edges rather than overrunning
        const uint64_t deg = e - b;
        warp_light_edges(u, b, deg > LIGHT_MAX ? LIGHT_MAX : (uint32_t)deg, A, n, f, d);
    }
    f.flush();
}

// ---------------------------------------------------------------- SV / LT edge rules
// Shiloach-Vishkin hook (Algorithm 15): l = min(P[u], P[v]), h = max; if
// l != h and h was a root at the round's start, writeMin(P[h], l).
struct SVEdge {
    uint32_t *P;
    const uint32_t *prev;
    uint32_t *changed;
    bool hit;
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
        uint32_t pu = ld_rel(P + u);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) continue;
            uint32_t pv = ld_rel(P + v[j]);
            uint32_t l = pu < pv ? pu : pv, h = pu < pv ? pv : pu;
            if (l != h && __ldg(prev + h) == h) {
                atomicMin(P + h, l);
                hit = true;
            }
        }
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
        uint32_t pu[4], pv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            pu[j] = ok[j] ? ld_rel(P + u[j]) : 0;
            pv[j] = ok[j] ? ld_rel(P + v[j]) : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t l = pu[j] < pv[j] ? pu[j] : pv[j], h = pu[j] < pv[j] ? pv[j] : pu[j];
            if (ok[j] && l != h && __ldg(prev + h) == h) {
                atomicMin(P + h, l);
                hit = true;
            }
        }
    }
    __device__ __forceinline__ void flush() {
        if (hit) *changed = 1u;
    }
};

// Liu-Tarjan ParentConnect with RootUpdate (Appendix D): the parents of an
// edge's endpoints are candidates for each other; x = P[u] takes y = P[v]
// (and symmetrically) when y is smaller and x was a root at the round's
// start.  A round changes something iff some writeMin lowered a parent.
struct LTEdge {
    uint32_t *P;
    const uint32_t *prev;
    uint32_t *changed;
    bool hit;
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) continue;
            uint32_t x = ld_rel(P + u), y = ld_rel(P + v[j]);
            if (y < x && __ldg(prev + x) == x) hit |= atomicMin(P + x, y) > y;
            if (x < y && __ldg(prev + y) == y) hit |= atomicMin(P + y, x) > x;
        }
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
        uint32_t x[4], y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            x[j] = ok[j] ? ld_rel(P + u[j]) : 0;
            y[j] = ok[j] ? ld_rel(P + v[j]) : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) continue;
            if (y[j] < x[j] && __ldg(prev + x[j]) == x[j]) hit |= atomicMin(P + x[j], y[j]) > y[j];
            if (x[j] < y[j] && __ldg(prev + y[j]) == y[j]) hit |= atomicMin(P + y[j], x[j]) > x[j];
        }
    }
    __device__ __forceinline__ void flush() {
        if (hit) *changed = 1u;
    }
};

// ---------------------------------------------------------------- BFS sampling
// Top-down step of the label-spreading BFS (Algorithm 5): claim unvisited
// neighbours in the visited bitmap, label them with the source, queue them.
struct BFSEdge {
    uint32_t *P;
    uint32_t *vis;
    uint32_t *next;
    uint32_t *nnext;
    uint32_t *minv;
    uint32_t src;
    uint32_t my_min;
    uint2 *forest;   // spanning forest: the tree edge (u, w) at the child w
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) continue;
            uint32_t w = v[j], bit = 1u << (w & 31);
            uint32_t *word = vis + (w >> 5);
            if (ld_rel(word) & bit) continue;
            if (atomicOr(word, bit) & bit) continue;
            P[w] = src;
            if (forest) forest[w] = make_uint2(u, w);
            next[append_one(nnext)] = w;
            my_min = w < my_min ? w : my_min;
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
    __device__ __forceinline__ void flush() {
        if (my_min != NONE && my_min < ld_rel(minv)) atomicMin(minv, my_min);
    }
};

// Bottom-up step: every unvisited vertex looks for a neighbour in the
// frontier bitmap and stops at the first one.
template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_bfs_pull(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m, uint32_t *P, uint32_t *vis,
                           const uint32_t *front_bm, uint32_t *next_bm, uint32_t src, uint32_t *nnext,
                           unsigned long long *next_edges, uint32_t *minv, Dev d) {
    uint32_t cnt = 0, mn = NONE;
    unsigned long long me = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t w = (uint32_t)i, bit = 1u << (w & 31);
        if (vis[w >> 5] & bit) continue;
        uint64_t b, e;
        vertex_range(I, w, m, b, e, d);
        for (uint64_t x = b; x < e; ++x) {
            uint32_t y = ld_stream(A + x);
            if (y >= n) { atomicOr(d.err, ERR_BAD_EDGE); continue; }
            if (front_bm[y >> 5] & (1u << (y & 31))) {
                P[w] = src;
                if (d.forest) d.forest[w] = make_uint2(y, w);
                atomicOr(next_bm + (w >> 5), bit);
                atomicOr(vis + (w >> 5), bit);
                ++cnt;
                me += e - b;
                mn = w < mn ? w : mn;
                break;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        me += __shfl_xor_sync(0xFFFFFFFFu, me, o);
        uint32_t t = __shfl_xor_sync(0xFFFFFFFFu, mn, o);
        mn = t < mn ? t : mn;
    }
    if ((threadIdx.x & 31) == 0) {
        if (cnt) atomicAdd(nnext, cnt);
        if (me) atomicAdd(next_edges, me);
        if (mn != NONE && mn < ld_rel(minv)) atomicMin(minv, mn);
    }
}

// Degree sum of a vertex list (frontier edges, for the direction switch).
template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_list_degrees(const OffT *I, uint64_t m, const uint32_t *list, const uint32_t *count,
                               unsigned long long *out, Dev d) {
    const uint32_t total = *count;
    unsigned long long s = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t b, e;
        vertex_range(I, list[i], m, b, e, d);
        s += e - b;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

__global__ void __launch_bounds__(256, 8) k_list_to_bitmap(const uint32_t *list, const uint32_t *count, uint32_t *bm) {
    const uint32_t total = *count;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t w = list[i];
        atomicOr(bm + (w >> 5), 1u << (w & 31));
    }
}

__global__ void __launch_bounds__(256, 8) k_bitmap_to_list(const uint32_t *bm, uint32_t n, uint32_t *list, uint32_t *count) {
    const uint32_t words = (n + 31) / 32;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t w = bm[i];
        if (!w) continue;
        uint32_t c = __popc(w);
        uint32_t base = atomicAdd(count, c);
        while (w) {
            int b = __ffs(w) - 1;
            w &= w - 1;
            list[base++] = (uint32_t)(i * 32 + b);
        }
    }
}

// Relabel the reached set to its smallest member (a min-rooted star).
__global__ void __launch_bounds__(256, 8) k_bfs_relabel(uint32_t *P, const uint32_t *vis, uint32_t n, const uint32_t *minv) {
    const uint32_t mn = *minv;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (vis[i >> 5] & (1u << (i & 31))) P[i] = mn;
}

// Top-down levels in one persistent launch.  A high-diameter graph (a road
// network, a grid) needs tens of thousands of levels whose frontiers are
// small; one launch sequence and one host round trip per level would
// dominate.  Here every block of a cooperative launch runs level after level
// with a grid barrier between them, and the launch returns to the host once
// the frontier is empty or holds more than BFS_LOOP_NF_MAX vertices, its
// edges exceed `mf_max`, or the direction rule asks for bottom-up (frontier
// edges > unexplored / 14).
// Frontier counts and edge sums rotate over three slots: level L reads slot
// L % 3, appends into slot (L + 1) % 3, and clears slot (L + 2) % 3, which no
// block reads after the barrier that ended level L - 1.  The edge sum a level
// leaves for the next is its own frontier's (read with the offsets it loads
// anyway), so the direction rule looks one level behind: that changes when
// the launch hands over to bottom-up, never which vertices are reached (the
// host takes the exact sum of the frontier it is handed).
// A frontier vertex of degree > BFS_HUB_DEG (a hub) is not left to one warp
// of this launch (a few warps per SM): its edges go to the chunk list as
// CHUNK-edge pieces, and after the level's barrier the launch ends with the
// level pending; the host runs the pieces as a full-occupancy chunk pass,
// which completes the level.  Every block reads the same piece count after
// the barrier, so all blocks leave together.
constexpr uint64_t BFS_HUB_DEG = 1024;

struct BfsLoop {
    GridBar bar;
    uint32_t cnt[3];
    uint32_t levels;
    uint32_t npiece[3];
    uint32_t pending;   // 1: level `levels` ran but its hubs' pieces (npiece[levels % 3]) did not
    unsigned long long mfc[3];
    unsigned long long reached;    // vertices claimed by the levels run
    unsigned long long explored;   // frontier edges of the levels run
};

struct BFSPushEdge {
    uint32_t *P;
    uint32_t *vis;
    uint32_t *next;
    uint32_t *nnext;
    uint32_t src;
    uint32_t my_min;
    unsigned long long my_edges;   // edges of the frontier vertices this thread expanded
    Dev d;
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) continue;
            const uint32_t w = v[j], bit = 1u << (w & 31);
            uint32_t *word = vis + (w >> 5);
            if (ld_rel(word) & bit) continue;
            if (atomicOr(word, bit) & bit) continue;
            P[w] = src;
            if (d.forest) d.forest[w] = make_uint2(u, w);
            next[append_one(nnext)] = w;
            my_min = w < my_min ? w : my_min;
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

constexpr unsigned BFS_LOOP_TPB = 512;
constexpr uint64_t BFS_LOOP_MF_MAX = 1ull << 24;   // frontier edges beyond which a level runs as its own launches
constexpr uint32_t BFS_LOOP_LEVELS = 1u << 16;      // levels per launch at most (a launch stays well under a second)
// frontier vertices beyond which a level runs as its own launches: the
// launch's edge estimate lags one level, and a frontier this large (an
// R-MAT level past the hubs) is where the lag would keep a level top-down
// that the exact count sends bottom-up; high-diameter frontiers stay far below
constexpr uint32_t BFS_LOOP_NF_MAX = 1u << 17;

template <typename OffT>
__global__ void __launch_bounds__(BFS_LOOP_TPB, 2) k_bfs_push_levels(const OffT *I, const uint32_t *A, uint32_t n,
                                                                  uint64_t m, uint32_t *P, uint32_t *vis,
                                                                  uint32_t *q0, uint32_t *q1, uint32_t src,
                                                                  BfsLoop *L, uint32_t *cnt_out0,
                                                                  uint32_t *cnt_out1, uint32_t *minv,
                                                                  uint64_t unexplored0, uint64_t mf_max,
                                                                  uint32_t max_levels, ChunkRef *chunks,
                                                                  uint64_t chunk_cap, Dev d) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t my_min = NONE;
    uint64_t explored = 0, reached = 0;
    uint32_t lv = 0, nf = 0;
    for (;; ++lv) {
        nf = ld_rel(&L->cnt[lv % 3]);
        const uint64_t mf = ld_rel64(&L->mfc[lv % 3]);
        if (lv > 0) reached += nf;
        const uint64_t unexplored = unexplored0 > explored ? unexplored0 - explored : 0;
        if (nf == 0 || lv == max_levels || nf > BFS_LOOP_NF_MAX || mf > mf_max || mf > unexplored / 14) break;
        uint32_t *cur = (lv & 1) ? q1 : q0;
        uint32_t *nx = (lv & 1) ? q0 : q1;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            L->cnt[(lv + 2) % 3] = 0;
            L->mfc[(lv + 2) % 3] = 0;
            L->npiece[(lv + 2) % 3] = 0;
        }
        BFSPushEdge f{P, vis, nx, &L->cnt[(lv + 1) % 3], src, NONE, 0ull, d};
        for (uint64_t base = warp * 32; base < nf; base += nwarps * 32) {
            const bool act = base + lane < nf;
            const uint32_t u = act ? cur[base + lane] : 0;
            uint64_t b = 0, e = 0;
            if (act) vertex_range(I, u, m, b, e, d);
            f.my_edges += e - b;
            const bool heavy = e - b > LIGHT_MAX;
            const uint32_t npc = e - b > BFS_HUB_DEG ? (uint32_t)((e - b + CHUNK - 1) / CHUNK) : 0;
            const uint32_t slot = warp_append_full(&L->npiece[lv % 3], npc);
            // the list has room for every heavy vertex's pieces; past it
            // (not reached) the warp walks the hub itself
            const bool hub = npc && (uint64_t)slot + npc <= chunk_cap;
            if (hub)
                for (uint32_t c = 0; c < npc; ++c) chunks[slot + c] = ChunkRef{u, c};
            warp_light_edges(u, b, heavy ? 0u : (uint32_t)(e - b), A, n, f, d);
            // heavier vertices short of a hub: the whole warp walks their edges
            uint32_t hm = __ballot_sync(0xFFFFFFFFu, heavy && !hub);
            while (hm) {
                const int l = __ffs(hm) - 1;
                hm &= hm - 1;
                const uint32_t hu = __shfl_sync(0xFFFFFFFFu, u, l);
                const uint64_t hb = __shfl_sync(0xFFFFFFFFu, b, l), he = __shfl_sync(0xFFFFFFFFu, e, l);
                warp_chunk_edges(hu, hb, he, A, n, f, d);
            }
        }
        unsigned long long me = f.my_edges;
        for (int o = 16; o > 0; o >>= 1) me += __shfl_xor_sync(0xFFFFFFFFu, me, o);
        if (lane == 0 && me) atomicAdd(&L->mfc[(lv + 1) % 3], me);
        explored += mf;
        if (!grid_sync(&L->bar, d)) break;
        my_min = f.my_min < my_min ? f.my_min : my_min;
        if (ld_rel(&L->npiece[lv % 3])) {
            if (blockIdx.x == 0 && threadIdx.x == 0) L->pending = 1;
            break;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const uint32_t t = __shfl_xor_sync(0xFFFFFFFFu, my_min, o);
        my_min = t < my_min ? t : my_min;
    }
    if (lane == 0 && my_min != NONE && my_min < ld_rel(minv)) atomicMin(minv, my_min);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        L->levels = lv;
        L->reached = reached;
        L->explored = explored;
        *((lv & 1) ? cnt_out1 : cnt_out0) = nf;
    }
}

// ---------------------------------------------------------------- LDD sampling
// Round r of the clustering (Algorithm 6): every uncovered id in [s0, s1)
// becomes a centre; then the frontier claims uncovered neighbours, the
// smallest claiming centre id winning (candidates first, commit after).
// stamp (spanning forest only, else null): the search step at which a
// vertex joined its cluster; a centre woken before step t has stamp t - 1,
// a vertex claimed in step t has stamp t.
__global__ void __launch_bounds__(256, 8) k_ldd_wake(uint32_t s0, uint32_t s1, uint32_t *P, uint32_t *vis, uint32_t *front,
                           uint32_t *nfront, uint32_t *last_round, uint32_t round, uint32_t *stamp,
                           uint32_t step, Ctl *ctl, int cur) {
    // the round's counters start at zero (the next round's frontier count
    // was cleared when the previous round ended)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->mf[cur] = 0;
        ctl->nchunks = 0;
        ctl->ldd_done = 0;
        ctl->ldd_minc[cur ^ 1] = NONE;   // the next frontier's, filled by this round's commit
    }
    // the uncovered ids of [s0, s1) join the frontier with one atomic per
    // block (block_compact; only this block touches its ids' bits, so the
    // two passes see the same ones)
    bool any = false;
    uint32_t vmin = NONE;
    block_compact(
        (uint64_t)(s1 - s0), nfront,
        [&](uint64_t i) {
            const uint32_t v = s0 + (uint32_t)i;
            return !((vis[v >> 5] >> (v & 31)) & 1u);
        },
        [&](uint64_t i, uint32_t k) {
            const uint32_t v = s0 + (uint32_t)i;
            atomicOr(vis + (v >> 5), 1u << (v & 31));
            P[v] = v;
            if (stamp) stamp[v] = step - 1;
            front[k] = v;
            any = true;
            vmin = v < vmin ? v : vmin;
        });
    if (any) atomicMax(last_round, round + 1);
    // the new centres' ids join the frontier's smallest centre
    vmin = __reduce_min_sync(0xFFFFFFFFu, vmin);
    if ((threadIdx.x & 31) == 0 && vmin != NONE) atomicMin(&ctl->ldd_minc[cur], vmin);
}

struct LDDEdge {
    const uint32_t *P;
    const uint32_t *vis;
    uint32_t *cand;
    uint32_t *next;
    uint32_t *nnext;
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
        uint32_t c = P[u];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) continue;
            uint32_t w = v[j];
            if (vis[w >> 5] & (1u << (w & 31))) continue;
            if (ld_rel(cand + w) <= c) continue;
            if (atomicMin(cand + w, c) == NONE) next[append_one(nnext)] = w;
        }
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
        uint32_t c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = ok[j] ? P[u[j]] : NONE;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) continue;
            const uint32_t w = v[j];
            if (vis[w >> 5] & (1u << (w & 31))) continue;
            if (ld_rel(cand + w) <= c[j]) continue;
            if (atomicMin(cand + w, c[j]) == NONE) next[append_one(nnext)] = w;
        }
    }
    __device__ __forceinline__ void flush() {}
};

// With fbm, the same launch also clears the frontier's bitmap words (the
// frontier list `front`, count *nfront), so the bitmap is empty for the
// next round.
__global__ void __launch_bounds__(256, 8) k_ldd_commit(uint32_t *P, uint32_t *vis, uint32_t *cand, const uint32_t *next,
                             const uint32_t *nnext, uint32_t *last_round, uint32_t round, uint32_t *stamp,
                             uint32_t step, uint32_t *fbm = nullptr, const uint32_t *front = nullptr,
                             const uint32_t *nfront = nullptr, uint32_t *minc_next = nullptr) {
    if (fbm) {
        const uint32_t nf = *nfront;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nf;
             i += (uint64_t)gridDim.x * blockDim.x)
            fbm[front[i] >> 5] = 0u;
    }
    const uint32_t total = *nnext;
    uint32_t cmin = NONE;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t w = next[i];
        const uint32_t c = cand[w];
        P[w] = c;
        cmin = c < cmin ? c : cmin;
        if (stamp) stamp[w] = step;
        cand[w] = NONE;
        atomicOr(vis + (w >> 5), 1u << (w & 31));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && total) atomicMax(last_round, round + 1);
    // the claimed vertices' centres: the next frontier's smallest centre
    if (minc_next) {
        cmin = __reduce_min_sync(0xFFFFFFFFu, cmin);
        if ((threadIdx.x & 31) == 0 && cmin != NONE) atomicMin(minc_next, cmin);
    }
}

// Bottom-up LDD rounds (direction optimisation, as for BFS): a top-down
// round reads the frontier's edges, a bottom-up one the uncovered
// vertices' edges (all of them: the smallest centre is wanted, so a scan
// cannot stop at the first frontier neighbour), and a round runs bottom-up
// when the uncovered vertices' edges are fewer than twice the frontier's (a
// bottom-up edge costs a bit test where a top-down one costs a candidate
// read and often a writeMin).  Beside its edge count, the frontier is
// marked in a bitmap every round, so any round can switch.  ldd_push_nf is
// the frontier size the top-down pass sees: 0 in a bottom-up round.  The
// frontier's smallest centre id (ldd_minc[cur], folded in by the commit
// that built the frontier and by the wake that added its new centres) lets
// a bottom-up scan stop when it meets it: no neighbour offers less.
template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_ldd_front(const OffT *I, uint32_t n, uint64_t m, const uint32_t *list,
                                                      const uint32_t *count, uint32_t *fbm, Ctl *ctl, int cur, Dev d) {
    const uint32_t total = *count;
    unsigned long long s = 0;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = warp * 32; base < total; base += nw * 32) {
        const bool act = base + lane < total;
        const uint32_t u = act ? list[base + lane] : 0;
        uint64_t b = 0, e = 0;
        if (act) vertex_range(I, u, m, b, e, d);
        s += e - b;
        // one OR per distinct bitmap word in the warp
        const uint32_t word = act ? (u >> 5) : NONE;
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, word);
        const uint32_t bits = __reduce_or_sync(grp, act ? 1u << (u & 31) : 0u);
        if (act && lane == __ffs(grp) - 1) atomicOr(fbm + word, bits);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0 && s) atomicAdd(&ctl->mf[cur], s);
    // the last block to finish takes the round's direction
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctl->ldd_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const unsigned long long mf = ld_rel64(&ctl->mf[cur]), ex = ctl->ldd_explored;
        const unsigned long long rest = m > ex + mf ? m - ex - mf : 0;   // edges of the uncovered vertices
        const uint32_t nf = total;
        const uint32_t pull = rest < 2 * mf;
        ctl->ldd_pull = pull;
        ctl->ldd_push_nf = pull ? 0u : nf;
        ctl->ldd_explored = ex + mf;
    }
}

// A bottom-up round scans the uncovered vertices' edges instead: an
// uncovered w with a frontier neighbour y takes P[y] as a candidate by the
// same writeMin as a top-down claim, so w ends the round with the smallest
// centre among its frontier neighbours either way, and the clustering does
// not depend on the direction.  The first candidate queues w for the commit.
// A scan keeps its smallest candidate in a register, makes one writeMin at
// its end, and ends early at the round's smallest frontier centre (the
// result cannot go lower, so it is exact).
struct LDDPullEdge {
    const uint32_t *P;
    const uint32_t *fbm;
    uint32_t *cand;
    uint32_t *next;
    uint32_t *nnext;
    // candidates of four edges: P[y] for frontier neighbours, else NONE
    // (the four bit loads issued together, then the parents)
    __device__ __forceinline__ uint32_t min4(const uint32_t (&y)[4], const bool (&ok)[4]) const {
        bool in[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) in[j] = ok[j] && ((fbm[y[j] >> 5] >> (y[j] & 31)) & 1u);
        uint32_t c[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) c[j] = in[j] ? P[y[j]] : NONE;
        const uint32_t c01 = c[0] < c[1] ? c[0] : c[1], c23 = c[2] < c[3] ? c[2] : c[3];
        return c01 < c23 ? c01 : c23;
    }
    __device__ __forceinline__ void offer(uint32_t w, uint32_t c) const {
        if (c != NONE && ld_rel(cand + w) > c && atomicMin(cand + w, c) == NONE) next[append_one(nnext)] = w;
    }
};

// PULL_PROBE: edges a lane scans of a heavier vertex before its chunks are
// listed (they are listed only if the probe did not meet the smallest
// centre).
constexpr uint32_t PULL_PROBE = 16;

// The candidate of w from edges [b, b + len), scanned by its lane four at a
// time until the smallest frontier centre turns up.
__device__ __forceinline__ uint32_t ldd_pull_scan(const LDDPullEdge &f, const uint32_t *A, uint64_t b,
                                                  uint32_t len, uint32_t n, uint32_t minc, const Dev &d) {
    uint32_t best = NONE;
    for (uint32_t x = 0; x < len && best != minc; x += 4) {
        uint32_t y[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ok[j] = x + j < len;
            y[j] = ok[j] ? ld_stream(A + b + x + j) : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j] && y[j] >= n) { atomicOr(d.err, ERR_BAD_EDGE); ok[j] = false; }
        const uint32_t c = f.min4(y, ok);
        best = c < best ? c : best;
    }
    return best;
}

// One LDD round's edge pass, either direction (the flag is the same for
// every thread): top-down, the frontier list's light vertices are walked
// by their warp and the heavier ones go to the chunk list; bottom-up, lane
// L of a warp step takes vertex base + L when its `vis` bit is clear, with
// the same split.
template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_ldd_bin(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                                                    const uint32_t *front, const uint32_t *vis, LDDEdge fpush,
                                                    LDDPullEdge fpull, ChunkRef *chunks, uint32_t *nchunks,
                                                    uint64_t cap, const Ctl *ctl, int cur, Dev d) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    WarpSlots ws;
    if (!ctl->ldd_pull) {
        const uint32_t total = ctl->ldd_push_nf;
        for (uint64_t base = warp * 32; base < total; base += nw * 32) {
            const bool act = base + lane < total;
            const uint32_t u = act ? front[base + lane] : 0;
            uint64_t b = 0, e = 0;
            if (act) vertex_range(I, u, m, b, e, d);
            const uint64_t deg = e - b;
            const uint32_t nc = deg > LIGHT_MAX ? (uint32_t)((deg + CHUNK - 1) / CHUNK) : 0;
            warp_bin_chunks(ws, nchunks, chunks, cap, nc, u, d);
            warp_light_edges(u, b, nc ? 0u : (uint32_t)deg, A, n, fpush, d);
        }
        ws.close(chunks, cap);
        return;
    }
    // bottom-up: lane L takes vertex base + L when its `vis` bit is clear
    // and scans its edges itself (a light vertex all of them, a heavier one
    // the first PULL_PROBE), stopping at the smallest frontier centre; a
    // heavier vertex whose probe did not meet it goes to the chunk list
    const uint32_t minc = ctl->ldd_minc[cur];
    for (uint64_t base = warp * 32; base < n; base += nw * 32) {
        const uint32_t vword = vis[base >> 5];
        if (vword == 0xFFFFFFFFu) continue;   // warp-uniform
        const uint64_t w = base + lane;
        uint64_t b = 0, e = 0;
        if (w < n && !((vword >> lane) & 1u)) vertex_range(I, (uint32_t)w, m, b, e, d);
        const uint64_t deg = e - b;
        const bool heavy = deg > LIGHT_MAX;
        const uint32_t best = ldd_pull_scan(fpull, A, b, heavy ? PULL_PROBE : (uint32_t)deg, n, minc, d);
        fpull.offer((uint32_t)w, best);
        const uint32_t nc = heavy && best != minc ? (uint32_t)((deg + CHUNK - 1) / CHUNK) : 0;
        warp_bin_chunks(ws, nchunks, chunks, cap, nc, (uint32_t)w, d);
    }
    ws.close(chunks, cap);
}

template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_ldd_chunks(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                                                       const ChunkRef *chunks, const uint32_t *nchunks, uint64_t cap,
                                                       LDDEdge fpush, LDDPullEdge fpull, const Ctl *ctl, int cur,
                                                       Dev d) {
    if (!ctl->ldd_pull) {
        run_chunks(I, A, n, m, chunks, nchunks, cap, fpush, d);
        return;
    }
    // bottom-up chunks: a warp per chunk, each lane its smallest candidate;
    // the warp stops once a lane meets the smallest frontier centre (or
    // skips the chunk if w already holds it), then offers the warp minimum
    const uint32_t minc = ctl->ldd_minc[cur];
    const int lane = threadIdx.x & 31;
    const uint32_t total = (uint32_t)((uint64_t)*nchunks < cap ? (uint64_t)*nchunks : cap);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = warp; i < total; i += nwarps) {
        const ChunkRef c = chunks[i];
        if (c.u == NONE || ld_rel(fpull.cand + c.u) == minc) continue;   // warp-uniform
        uint64_t b, e;
        vertex_range(I, c.u, m, b, e, d);
        const uint64_t cb = b + (uint64_t)c.c * CHUNK;
        const uint64_t ce = cb + CHUNK < e ? cb + CHUNK : e;
        uint32_t best = NONE;
        for (uint64_t x0 = cb; x0 < ce; x0 += 128) {
            uint32_t y[4];
            bool ok[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t x = x0 + 32 * j + lane;
                ok[j] = x < ce;
                y[j] = ok[j] ? ld_stream(A + x) : 0;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ok[j] && y[j] >= n) { atomicOr(d.err, ERR_BAD_EDGE); ok[j] = false; }
            const uint32_t cm = fpull.min4(y, ok);
            best = cm < best ? cm : best;
            if (__any_sync(0xFFFFFFFFu, best == minc)) break;
        }
        best = __reduce_min_sync(0xFFFFFFFFu, best);
        if (lane == 0) fpull.offer(c.u, best);
    }
}


// Spanning-forest edges of the LDD clusters (the searches' tree edges,
// assigned to the child): a non-centre w was claimed in step t by a
// frontier vertex of its own cluster that joined in step t - 1, so such a
// neighbour exists; any one of them is a valid parent, because following
// parents strictly lowers the step and ends at the cluster's only
// vertex without one, its centre.  Runs before the clusters are relabelled
// (P[w] is still w's centre; centres are the w with P[w] = w).
template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_ldd_tree_edges(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                                                           const uint32_t *P, const uint32_t *stamp, Dev d) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = (uint32_t)i, c = P[w];
        if (c == w) continue;
        const uint32_t want = stamp[w] - 1;
        uint64_t b, e;
        vertex_range(I, w, m, b, e, d);
        bool found = false;
        for (uint64_t x = b; x < e && !found; ++x) {
            const uint32_t u = ld_stream(A + x);
            if (u < n && P[u] == c && stamp[u] == want) {
                d.forest[w] = make_uint2(u, w);
                found = true;
            }
        }
        if (!found) atomicOr(d.err, ERR_NONCONVERGED);
    }
}

// Relabel clusters to their smallest members: cmin[c] = min{v : P[v] = c}
// (warp-grouped by cluster, one atomicMin per group, skipped when it cannot
// lower the current value), then P[v] = cmin[P[v]].
__global__ void __launch_bounds__(256, 8) k_cluster_min(const uint32_t *P, uint32_t n, uint32_t *cmin) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = warp * 32; base < n; base += nw * 32) {
        uint64_t v = base + lane;
        uint32_t c = v < n ? P[v] : NONE;
        unsigned grp = __match_any_sync(0xFFFFFFFFu, c);
        uint32_t mn = __reduce_min_sync(grp, (uint32_t)(v < n ? v : NONE));
        if (c != NONE && lane == __ffs(grp) - 1 && mn < ld_rel(cmin + c)) atomicMin(cmin + c, mn);
    }
}

__global__ void __launch_bounds__(256, 8) k_apply_cluster_min(uint32_t *P, uint32_t n, const uint32_t *cmin) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        P[i] = cmin[P[i]];
}

// ================================================================ host side
struct Graph {
    const void *I;
    bool u64;
    const uint32_t *A;
    uint32_t n;
    uint64_t m;
};

// Scratch layout of one call.
struct Work {
    Scratch sc;
    size_t o_defer = 0, o_dcount = 0, o_pick = 0;
    size_t o_ctl = 0, o_chunks = 0, o_counts = 0, o_prev = 0, o_light = 0, o_vis = 0, o_q0 = 0, o_q1 = 0,
           o_bm0 = 0, o_bm1 = 0, o_cand = 0, o_loop = 0, o_stamp = 0, o_sf = 0, o_ff = 0, o_fcount = 0,
           o_hooks = 0;
    bool has_hooks = false;
    bool has_counts = false, has_sv = false, has_bfs = false, has_ldd = false;
    // k-out with a finish: the nonzero-degree bitmap, and whether the fused
    // compression already built the finish's candidate lists
    bool has_nz = false, lists_built = false;
    size_t o_nz = 0;
    // the selected path: degree statistics gathered by the first k-out pass
    // and the choice made where L_max is checked (k_lmax_select)
    FeatStats *fs = nullptr;   // one partial per block of k_degree_stats, then their sum
    uint32_t fs_parts = 0;
    cudaEvent_t sel_join = nullptr;   // the degree statistics' stream, joined before the choice
    bool select = false;
    const float *sel_params = nullptr;
    int sel_force = -1;
    float *sel_feat = nullptr;
    volatile int *sel_host = nullptr;
    uint64_t sel_m = 0;
    uint64_t chunk_cap = 0;
    Ctl *ctl() const { return sc.at<Ctl>(o_ctl); }
};

// forest: also the spanning-forest arrays (sampling edges by child / hooked
// root, finish edges by hooked root, (NONE, NONE) where empty).
void plan(Work &w, const Graph &g, int sample_kind, uint32_t freq_samples, int finish_kind, bool finish_phase,
          bool forest = false) {
    const uint64_t n = g.n;
    if (finish_kind == CC_FINISH_UF_HOOKS) {
        w.has_hooks = true;
        w.o_hooks = w.sc.reserve(n * 4);
    }
    if (forest) {
        if (sample_kind == CC_SAMPLE_BFS || sample_kind == CC_SAMPLE_LDD) w.o_sf = w.sc.reserve(n * 8);
        w.o_ff = w.sc.reserve(n * 8);
        w.o_fcount = w.sc.reserve(8);
        if (sample_kind == CC_SAMPLE_LDD) w.o_stamp = w.sc.reserve(n * 4);
    }
    w.o_ctl = w.sc.reserve(sizeof(Ctl));
    w.chunk_cap = chunk_capacity(n, g.m) + CHUNK_SLACK;
    w.o_chunks = w.sc.reserve(w.chunk_cap * sizeof(ChunkRef));
    if (sample_kind == CC_SAMPLE_KOUT) {
        // the first-edge queue: one region of `span` pairs per span of
        // vertices, and the spans' counts
        w.o_defer = w.sc.reserve(kout_defer_entries(n) * 8);
        w.o_dcount = w.sc.reserve((size_t)kout_spans_max(n) * 4);
        w.o_pick = w.sc.reserve(n * 4);
    }
    if (sample_kind != CC_SAMPLE_NONE && freq_samples == 0) {
        w.has_counts = true;
        w.o_counts = w.sc.reserve(n * 4);
    }
    if (finish_phase) w.o_light = w.sc.reserve(n * 4);
    if (finish_phase && sample_kind == CC_SAMPLE_KOUT && freq_samples == 0) {
        w.has_nz = true;
        w.o_nz = w.sc.reserve(((n + 31) / 32 + 4) * 4);
    }
    if (finish_phase && (finish_kind == CC_FINISH_SV || finish_kind == CC_FINISH_LT_PRF)) {
        w.has_sv = true;
        w.o_prev = w.sc.reserve(n * 4);
    }
    const uint64_t words = (n + 31) / 32;
    if (sample_kind == CC_SAMPLE_BFS) {
        w.has_bfs = true;
        w.o_vis = w.sc.reserve(words * 4);
        w.o_q0 = w.sc.reserve(n * 4);
        w.o_q1 = w.sc.reserve(n * 4);
        w.o_bm0 = w.sc.reserve(words * 4);
        w.o_bm1 = w.sc.reserve(words * 4);
        w.o_loop = w.sc.reserve(sizeof(BfsLoop));
    }
    if (sample_kind == CC_SAMPLE_LDD) {
        w.has_ldd = true;
        w.o_vis = w.sc.reserve(words * 4);
        w.o_q0 = w.sc.reserve(n * 4);
        w.o_q1 = w.sc.reserve(n * 4);
        w.o_cand = w.sc.reserve(n * 4);
        w.o_bm0 = w.sc.reserve(words * 4);   // bottom-up rounds: the frontier's bitmap

    }
}

#define CC_TRY(x)                                   \
    do {                                            \
        cudaError_t e__ = (x);                      \
        if (e__ != cudaSuccess) return from_cuda(e__); \
    } while (0)
#define CC_LAUNCH() CC_TRY(cudaGetLastError())

// After the scratch is allocated: UF-Hooks' hooks array starts all free.
cc_status attach_hooks(Work &w, Dev &d, uint32_t n, cudaStream_t s) {
    if (!w.has_hooks) return CC_OK;
    d.hooks = w.sc.at<uint32_t>(w.o_hooks);
    CC_TRY(cudaMemsetAsync(d.hooks, 0xFF, (size_t)n * 4, s));
    return CC_OK;
}

template <class Fn>
cc_status with_engine(const cc_finish_opt &f, Fn &&fn) {
    return with_uf_engine(f.kind, f.find, f.splice, fn);
}

// ---------------------------------------------------------------- phases
template <typename OffT>
cc_status bfs_sample(const Graph &g, const cc_sample_opt &so, uint32_t *P, Work &w, const DeviceInfo *di,
                     const Dev &d, cudaStream_t s, int32_t *info) {
    const OffT *I = static_cast<const OffT *>(g.I);
    const uint32_t n = g.n;
    const uint64_t words = (n + 31) / 32;
    Ctl *ctl = w.ctl();
    uint32_t *vis = w.sc.at<uint32_t>(w.o_vis);
    uint32_t *q[2] = {w.sc.at<uint32_t>(w.o_q0), w.sc.at<uint32_t>(w.o_q1)};
    uint32_t *bm[2] = {w.sc.at<uint32_t>(w.o_bm0), w.sc.at<uint32_t>(w.o_bm1)};
    ChunkRef *chunks = w.sc.at<ChunkRef>(w.o_chunks);
    const unsigned gv = grid_for(di, n, TPB);
    const unsigned ge = grid_for(di, n, TPB, EDGE_MINB);
    // host-visible copies of the per-level counters
    struct Lv {
        uint32_t nnext;
        uint32_t pad;
        unsigned long long mf;
    };
    Lv *hl = nullptr;
    CC_TRY(cudaMallocHost(&hl, sizeof(Lv) + sizeof(BfsLoop)));
    struct Free {
        Lv *p;
        ~Free() { cudaFreeHost(p); }
    } fr{hl};
    BfsLoop *hloop = reinterpret_cast<BfsLoop *>(hl + 1);
    BfsLoop *loop = w.sc.at<BfsLoop>(w.o_loop);
    // persistent top-down levels: one cooperative launch of every co-resident block
    int per_sm = 0;
    CC_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_push_levels<OffT>, BFS_LOOP_TPB, 0));
    const unsigned loop_grid = (unsigned)(per_sm < 1 ? per_sm : 1) * di->sms;   // one block per SM: cheapest barrier
    *info = -1;
    for (uint32_t t = 0; t < so.bfs_tries; ++t) {
        const uint32_t src = (uint32_t)(draw64(so.seed ^ TAG_BFS, t) % n);
        {
            CC_PROF("k_iota", s);
            k_iota<<<gv, TPB, 0, s>>>(P, n);
        }
        // a failed try leaves no tree edges behind
        if (d.forest && t > 0) CC_TRY(cudaMemsetAsync(d.forest, 0xFF, (size_t)n * 8, s));
        CC_TRY(cudaMemsetAsync(vis, 0, words * 4, s));
        CC_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
        {
            CC_PROF("k_set_u32", s);
            k_set_u32<<<1, 1, 0, s>>>(&ctl->minv, src);
        }
        {
            CC_PROF("k_set_u32", s);
            k_set_u32<<<1, 1, 0, s>>>(q[0], src);
        }
        {
            CC_PROF("k_set_u32", s);
            k_set_u32<<<1, 1, 0, s>>>(&ctl->nfront[0], 1);
        }
        {
            CC_PROF("k_list_to_bitmap", s);
            k_list_to_bitmap<<<1, 32, 0, s>>>(q[0], &ctl->nfront[0], vis);
        }
        CC_LAUNCH();
        uint64_t reached = 1, nf = 1, explored_edges = 0;
        int cur = 0;
        bool pull = false;   // frontier kept as a bitmap (bm[cur]) when pulling
        // frontier edge count of the source
        CC_TRY(cudaMemsetAsync(&ctl->mf[0], 0, 8, s));
        {
            CC_PROF("k_list_degrees", s);
            k_list_degrees<OffT><<<1, 32, 0, s>>>(I, g.m, q[0], &ctl->nfront[0], &ctl->mf[0], d);
        }
        CC_TRY(cudaMemcpyAsync(&hl->mf, &ctl->mf[0], 8, cudaMemcpyDeviceToHost, s));
        CC_TRY(cudaStreamSynchronize(s));
        uint64_t mf = hl->mf;
        for (uint64_t level = 0; nf > 0 && level <= n; ++level) {
            // Direction choice (Beamer et al.'s heuristic, as in
            // direction-optimizing BFS): pull when the frontier's edges
            // exceed 1/14 of the unexplored edges, push when the frontier
            // is below n/24 vertices.
            const uint64_t unexplored = g.m > explored_edges ? g.m - explored_edges : 0;
            bool want_pull = pull ? (nf >= n / 24) : (mf > unexplored / 14);
            if (want_pull && !pull) {
                CC_TRY(cudaMemsetAsync(bm[cur], 0, words * 4, s));
                {
                    CC_PROF("k_list_to_bitmap", s);
                    k_list_to_bitmap<<<gv, TPB, 0, s>>>(q[cur], &ctl->nfront[cur], bm[cur]);
                }
                CC_LAUNCH();
            } else if (!want_pull && pull) {
                CC_TRY(cudaMemsetAsync(&ctl->nfront[cur], 0, 4, s));
                {
                    CC_PROF("k_bitmap_to_list", s);
                    k_bitmap_to_list<<<grid_for(di, words, TPB), TPB, 0, s>>>(bm[cur], n, q[cur], &ctl->nfront[cur]);
                }
                CC_LAUNCH();
            }
            pull = want_pull;
            const int nx = cur ^ 1;
            CC_TRY(cudaMemsetAsync(&ctl->nfront[nx], 0, 4, s));
            CC_TRY(cudaMemsetAsync(&ctl->mf[nx], 0, 8, s));
            if (pull) {
                CC_TRY(cudaMemsetAsync(bm[nx], 0, words * 4, s));
                {
                    CC_PROF("k_bfs_pull", s);
                    k_bfs_pull<OffT><<<gv, TPB, 0, s>>>(I, g.A, n, g.m, P, vis, bm[cur], bm[nx], src, &ctl->nfront[nx],
                                                        &ctl->mf[nx], &ctl->minv, d);
                }
                CC_LAUNCH();
            } else {
                if (loop_grid > 0 && mf <= BFS_LOOP_MF_MAX) {
                    memset(hloop, 0, sizeof(BfsLoop));
                    hloop->cnt[0] = (uint32_t)nf;
                    hloop->mfc[0] = mf;
                    CC_TRY(cudaMemcpyAsync(loop, hloop, sizeof(BfsLoop), cudaMemcpyHostToDevice, s));
                    uint32_t *qc = q[cur], *qn = q[nx], *c0 = &ctl->nfront[cur], *c1 = &ctl->nfront[nx];
                    uint32_t *mv = &ctl->minv;
                    const uint64_t unexplored0 = unexplored, mfmax = BFS_LOOP_MF_MAX;
                    uint32_t nn = n, srcv = src, maxl = BFS_LOOP_LEVELS;
                    uint64_t mm = g.m;
                    const OffT *Ip = I;
                    const uint32_t *Ap = g.A;
                    ChunkRef *ck = chunks;
                    uint64_t ccap = w.chunk_cap;
                    Dev dd = d;
                    void *args[] = {&Ip, &Ap, &nn, &mm, &P, &vis, &qc, &qn, &srcv, &loop, &c0, &c1, &mv,
                                    const_cast<uint64_t *>(&unexplored0), const_cast<uint64_t *>(&mfmax), &maxl,
                                    &ck, &ccap, &dd};
                    {
                        CC_PROF("k_bfs_push_levels", s);
                        CC_TRY(cudaLaunchCooperativeKernel((const void *)k_bfs_push_levels<OffT>, loop_grid,
                                                           BFS_LOOP_TPB, args, 0, s));
                    }
                    CC_TRY(cudaMemcpyAsync(hloop, loop, sizeof(BfsLoop), cudaMemcpyDeviceToHost, s));
                    CC_TRY(cudaStreamSynchronize(s));
                    if (hloop->bar.abort) return CC_ERR_NONCONVERGED;
                    const uint32_t L = hloop->levels;
                    if (hloop->pending) {
                        // level L ran but for its hubs' pieces: run them at
                        // full occupancy, then its next frontier is complete
                        const int qc = (L & 1) ? nx : cur, qn = qc ^ 1;
                        BFSEdge f{P, vis, q[qn], &loop->cnt[(L + 1) % 3], &ctl->minv, src, NONE, d.forest};
                        {
                            CC_PROF("k_chunks", s);
                            k_chunks<OffT, BFSEdge><<<grid_for(di, (uint64_t)1 << 40, TPB, EDGE_MINB), TPB, 0, s>>>(
                                I, g.A, n, g.m, chunks, &loop->npiece[L % 3], w.chunk_cap, f, d);
                        }
                        CC_LAUNCH();
                        CC_TRY(cudaMemcpyAsync(&ctl->nfront[qn], &loop->cnt[(L + 1) % 3], 4, cudaMemcpyDeviceToDevice,
                                               s));
                        CC_TRY(cudaMemsetAsync(&ctl->mf[qn], 0, 8, s));
                        {
                            CC_PROF("k_list_degrees", s);
                            k_list_degrees<OffT><<<gv, TPB, 0, s>>>(I, g.m, q[qn], &ctl->nfront[qn], &ctl->mf[qn], d);
                        }
                        CC_LAUNCH();
                        CC_TRY(cudaMemcpyAsync(&hl->nnext, &ctl->nfront[qn], 4, cudaMemcpyDeviceToHost, s));
                        CC_TRY(cudaMemcpyAsync(&hl->mf, &ctl->mf[qn], 8, cudaMemcpyDeviceToHost, s));
                        CC_TRY(cudaStreamSynchronize(s));
                        nf = hl->nnext;
                        mf = hl->mf;
                        reached += hloop->reached + nf;
                        explored_edges += hloop->explored;
                        level += L;
                        cur = qn;
                        continue;
                    }
                    if (L > 0) {
                        if (L & 1) cur = nx;
                        nf = hloop->cnt[L % 3];
                        reached += hloop->reached;
                        explored_edges += hloop->explored;
                        level += L - 1;
                        // the launch's edge sum for the frontier it hands
                        // over is one level behind: take the exact one
                        CC_TRY(cudaMemsetAsync(&ctl->mf[cur], 0, 8, s));
                        {
                            CC_PROF("k_list_degrees", s);
                            k_list_degrees<OffT><<<gv, TPB, 0, s>>>(I, g.m, q[cur], &ctl->nfront[cur], &ctl->mf[cur], d);
                        }
                        CC_LAUNCH();
                        CC_TRY(cudaMemcpyAsync(&hl->mf, &ctl->mf[cur], 8, cudaMemcpyDeviceToHost, s));
                        CC_TRY(cudaStreamSynchronize(s));
                        mf = hl->mf;
                        continue;
                    }
                }
                CC_TRY(cudaMemsetAsync(&ctl->nchunks, 0, 4, s));
                BFSEdge f{P, vis, q[nx], &ctl->nfront[nx], &ctl->minv, src, NONE, d.forest};
                {
                    CC_PROF("k_list_bin", s);
                    k_list_bin<OffT, BFSEdge><<<ge, TPB, 0, s>>>(I, g.A, n, g.m, q[cur], &ctl->nfront[cur], f, chunks,
                                                                 &ctl->nchunks, w.chunk_cap, d);
                }
                {
                    CC_PROF("k_chunks", s);
                    k_chunks<OffT, BFSEdge><<<grid_for(di, (uint64_t)1 << 40, TPB, EDGE_MINB), TPB, 0, s>>>(
                        I, g.A, n, g.m, chunks, &ctl->nchunks, w.chunk_cap, f, d);
                }
                {
                    CC_PROF("k_list_degrees", s);
                    k_list_degrees<OffT><<<gv, TPB, 0, s>>>(I, g.m, q[nx], &ctl->nfront[nx], &ctl->mf[nx], d);
                }
                CC_LAUNCH();
            }
            explored_edges += mf;
            CC_TRY(cudaMemcpyAsync(&hl->nnext, &ctl->nfront[nx], 4, cudaMemcpyDeviceToHost, s));
            CC_TRY(cudaMemcpyAsync(&hl->mf, &ctl->mf[nx], 8, cudaMemcpyDeviceToHost, s));
            CC_TRY(cudaStreamSynchronize(s));
            nf = hl->nnext;
            mf = hl->mf;
            reached += nf;
            cur = nx;
        }
        // the most frequent label is the source's (count = reached)
        if (10 * reached > (uint64_t)n) {
            {
                CC_PROF("k_bfs_relabel", s);
                k_bfs_relabel<<<gv, TPB, 0, s>>>(P, vis, n, &ctl->minv);
            }
            CC_LAUNCH();
            *info = (int32_t)t;
            return CC_OK;
        }
    }
    if (d.forest) CC_TRY(cudaMemsetAsync(d.forest, 0xFF, (size_t)n * 8, s));
    {
        CC_PROF("k_iota", s);
        k_iota<<<gv, TPB, 0, s>>>(P, n);
    }
    CC_LAUNCH();
    return CC_OK;
}

template <typename OffT>
cc_status ldd_sample(const Graph &g, const cc_sample_opt &so, uint32_t *P, Work &w, const DeviceInfo *di,
                     const Dev &d, cudaStream_t s, int32_t *info) {
    const OffT *I = static_cast<const OffT *>(g.I);
    const uint32_t n = g.n;
    const uint64_t words = (n + 31) / 32;
    Ctl *ctl = w.ctl();
    uint32_t *vis = w.sc.at<uint32_t>(w.o_vis);
    uint32_t *q[2] = {w.sc.at<uint32_t>(w.o_q0), w.sc.at<uint32_t>(w.o_q1)};
    uint32_t *cand = w.sc.at<uint32_t>(w.o_cand);
    uint32_t *stamp = d.forest ? w.sc.at<uint32_t>(w.o_stamp) : nullptr;
    uint32_t *fbm = w.sc.at<uint32_t>(w.o_bm0);
    ChunkRef *chunks = w.sc.at<ChunkRef>(w.o_chunks);
    const unsigned gv = grid_for(di, n, TPB);
    const unsigned gc = grid_for(di, (uint64_t)1 << 40, TPB);
    const unsigned ge = grid_for(di, n, TPB, EDGE_MINB);
    const unsigned gce = grid_for(di, (uint64_t)1 << 40, TPB, EDGE_MINB);
    CC_TRY(cudaMemsetAsync(vis, 0, words * 4, s));
    CC_TRY(cudaMemsetAsync(fbm, 0, words * 4, s));
    CC_TRY(cudaMemsetAsync(cand, 0xFF, (size_t)n * 4, s));
    CC_TRY(cudaMemsetAsync(ctl, 0, sizeof(Ctl), s));
    CC_TRY(cudaMemsetAsync(ctl->ldd_minc, 0xFF, sizeof(ctl->ldd_minc), s));
    uint64_t S = 0;
    int cur = 0;
    uint32_t r = 0;
    // Start schedule: round r starts the next floor(exp(beta r)) ids; the
    // rounds run until every id has been started, by which time every
    // vertex is covered.
    for (; S < n; ++r) {
        double x = std::floor(std::exp((double)so.ldd_beta * (double)r));
        if (x < 1.0) x = 1.0;
        if (x > 4294967295.0) x = 4294967295.0;
        uint64_t S1 = std::min<uint64_t>(n, S + (uint64_t)x);
        const int nx = cur ^ 1;
        {
            CC_PROF("k_ldd_wake", s);
            k_ldd_wake<<<grid_for(di, S1 - S, TPB), TPB, 0, s>>>((uint32_t)S, (uint32_t)S1, P, vis, q[cur],
                                                                  &ctl->nfront[cur], &ctl->last_round, r, stamp,
                                                                  r + 1, ctl, cur);
        }
        {
            CC_PROF("k_ldd_front", s);
            k_ldd_front<OffT><<<gv, TPB, 0, s>>>(I, n, g.m, q[cur], &ctl->nfront[cur], fbm, ctl, cur, d);
        }
        LDDEdge fpush{P, vis, cand, q[nx], &ctl->nfront[nx]};
        LDDPullEdge fpull{P, fbm, cand, q[nx], &ctl->nfront[nx]};
        {
            CC_PROF("k_ldd_bin", s);
            k_ldd_bin<OffT><<<gv, TPB, 0, s>>>(I, g.A, n, g.m, q[cur], vis, fpush, fpull, chunks, &ctl->nchunks,
                                               w.chunk_cap, ctl, cur, d);
        }
        {
            CC_PROF("k_ldd_chunks", s);
            k_ldd_chunks<OffT><<<gc, TPB, 0, s>>>(I, g.A, n, g.m, chunks, &ctl->nchunks, w.chunk_cap, fpush, fpull,
                                                  ctl, cur, d);
        }
        {
            CC_PROF("k_ldd_commit", s);
            k_ldd_commit<<<gv, TPB, 0, s>>>(P, vis, cand, q[nx], &ctl->nfront[nx], &ctl->last_round, r, stamp,
                                            r + 1, fbm, q[cur], &ctl->nfront[cur], &ctl->ldd_minc[nx]);
        }
        CC_TRY(cudaMemsetAsync(&ctl->nfront[cur], 0, 4, s));
        CC_LAUNCH();
        S = S1;
        cur = nx;
    }
    // the last frontier may still claim: run expansion rounds until it is empty
    for (uint32_t extra = 0; extra <= n; ++extra) {
        uint32_t nf = 0;
        CC_TRY(cudaMemcpyAsync(&nf, &ctl->nfront[cur], 4, cudaMemcpyDeviceToHost, s));
        CC_TRY(cudaStreamSynchronize(s));
        if (nf == 0) break;
        const int nx = cur ^ 1;
        CC_TRY(cudaMemsetAsync(&ctl->nfront[nx], 0, 4, s));
        CC_TRY(cudaMemsetAsync(&ctl->nchunks, 0, 4, s));
        LDDEdge f{P, vis, cand, q[nx], &ctl->nfront[nx]};
        {
            CC_PROF("k_list_bin", s);
            k_list_bin<OffT, LDDEdge><<<ge, TPB, 0, s>>>(I, g.A, n, g.m, q[cur], &ctl->nfront[cur], f, chunks,
                                                         &ctl->nchunks, w.chunk_cap, d);
        }
        {
            CC_PROF("k_chunks", s);
            k_chunks<OffT, LDDEdge><<<gce, TPB, 0, s>>>(I, g.A, n, g.m, chunks, &ctl->nchunks, w.chunk_cap, f, d);
        }
        {
            CC_PROF("k_ldd_commit", s);
            k_ldd_commit<<<gv, TPB, 0, s>>>(P, vis, cand, q[nx], &ctl->nfront[nx], &ctl->last_round, r, stamp,
                                            r + 1);
        }
        CC_TRY(cudaMemsetAsync(&ctl->nfront[cur], 0, 4, s));
        CC_LAUNCH();
        cur = nx;
        ++r;
    }
    if (stamp) {
        CC_PROF("k_ldd_tree_edges", s);
        k_ldd_tree_edges<OffT><<<gv, TPB, 0, s>>>(I, g.A, n, g.m, P, stamp, d);
    }
    // clusters -> min-id stars (cand is all NONE again and serves as cmin)
    {
        CC_PROF("k_cluster_min", s);
        k_cluster_min<<<gv, TPB, 0, s>>>(P, n, cand);
    }
    {
        CC_PROF("k_apply_cluster_min", s);
        k_apply_cluster_min<<<gv, TPB, 0, s>>>(P, n, cand);
    }
    CC_LAUNCH();
    uint32_t lr = 0;
    CC_TRY(cudaMemcpyAsync(&lr, &ctl->last_round, 4, cudaMemcpyDeviceToHost, s));
    CC_TRY(cudaStreamSynchronize(s));
    *info = (int32_t)lr;
    return CC_OK;
}

// count_into: when not null (k-out with exact IdentifyFrequent), the
// compression also counts the flat labels into this (zeroed here) array.
template <typename OffT>
cc_status sample_phase(const Graph &g, const cc_sample_opt &so, const cc_finish_opt &fo, uint32_t *P, Work &w,
                       const DeviceInfo *di, const Dev &d, cudaStream_t s, int32_t *info, uint32_t *count_into) {
    const unsigned gv = grid_for(di, g.n, TPB);
    *info = 0;
    if (so.kind == CC_SAMPLE_BFS) return bfs_sample<OffT>(g, so, P, w, di, d, s, info);
    if (so.kind == CC_SAMPLE_LDD) return ldd_sample<OffT>(g, so, P, w, di, d, s, info);
    if (so.kind == CC_SAMPLE_NONE) {
        {
            CC_PROF("k_iota", s);
            k_iota<<<gv, TPB, 0, s>>>(P, g.n);
        }
        CC_LAUNCH();
        return CC_OK;
    }
    // k-out: union-find over the picked edges, then full compression
    return with_engine(fo, [&](auto eng) -> cc_status {
        using E = decltype(eng);
        const OffT *I = static_cast<const OffT *>(g.I);
        uint2 *defer = w.sc.at<uint2>(w.o_defer);
        uint32_t *dcount = w.sc.at<uint32_t>(w.o_dcount);
        // the first pass's grid (one wave at its occupancy); its warps take
        // spans of vertices from a counter in the control block (zero: the
        // block is cleared before sampling, and the queue pass clears the
        // counter again after the spans are done)
        const unsigned gh = grid_for(di, g.n, TPB, HOOK_MINB);
        const uint32_t span_len = kout_span_for(g.n, (uint64_t)gh * (TPB / 32));
        const uint32_t nspan = (uint32_t)(((uint64_t)g.n + span_len - 1) / span_len);
        uint32_t *span_ctr = &w.ctl()->kout_span;
        uint32_t *pick1 = so.k == 2 ? w.sc.at<uint32_t>(w.o_pick) : nullptr;
        // the fused binning (k = 2, exact IdentifyFrequent, a finish to follow)
        const bool fuse = count_into && pick1 && w.has_nz;
        uint32_t *nz = fuse ? w.sc.at<uint32_t>(w.o_nz) : nullptr;
        {
            CC_PROF("k_kout_hook_first", s);
            k_kout_hook_first<OffT><<<gh, TPB, 0, s>>>(I, g.A, g.n, g.m, P, defer, dcount, span_ctr, span_len,
                                                       pick1, so.k, so.kout_rule, so.seed, nz, d);
        }
        {
            CC_PROF("k_kout_defer", s);
            k_kout_defer<E><<<gv, TPB, 0, s>>>(g.n, P, defer, dcount, nspan, span_len, span_ctr, d);
        }
        if (so.k > 1) {
            // full compression between the rounds: without it the second
            // round's unions walk the first round's uncompressed chains
            // through L2 (folding the compression into the second round's
            // pass measured 2.4 against 0.5 ms for the two at R-MAT scale
            // 26); it also clears the count array
            {
                CC_PROF("k_compress_mid", s);
                k_shortcut<false, true><<<gv, TPB, 0, s>>>(P, nullptr, g.n, nullptr, d, nullptr, nullptr, nullptr,
                                                           w.ctl()->spans[0]);
            }
            if (pick1) {
                CC_PROF("k_kout_apply_pick", s);
                k_kout_apply_pick<E><<<gv, TPB, 0, s>>>(pick1, g.n, P, d);
            } else {
                CC_PROF("k_kout_rest", s);
                launch_kout<OffT, E>(gv, s, I, g.A, g.n, g.m, so.k, so.kout_rule, so.seed, P, d, 1u, so.k);
            }
        }
        if (fuse) {
            // compression + count + arg-max key + the finish's candidate
            // lists against a sampled guess of L_max (checked in identify)
            Ctl *ctl = w.ctl();
            {
                CC_PROF("k_guess_lmax", s);
                k_guess_lmax<<<1, 128, 0, s>>>(P, nz, g.n, so.seed, ctl);
            }
            CC_PROF("k_compress_count", s);
            k_compress_count_bin<OffT><<<grid_for(di, g.n, TPB, 6), TPB, 0, s>>>(
                P, g.n, I, g.m, nz, ctl, w.sc.at<uint32_t>(w.o_light),
                                                          w.sc.at<ChunkRef>(w.o_chunks), w.chunk_cap, d);
            w.lists_built = true;
        } else if (count_into) {
            // the arg-max key is taken as the compression counts (identify
            // then only converts it)
            uint32_t *cnt = count_into;
            CC_TRY(cudaMemsetAsync(cnt, 0, (size_t)g.n * 4, s));
            CC_TRY(cudaMemsetAsync(&w.ctl()->key, 0, 8, s));
            CC_PROF("k_compress_count", s);
            k_shortcut<true><<<gv, TPB, 0, s>>>(P, nullptr, g.n, cnt, d, &w.ctl()->key);
        } else {
            CC_PROF("k_compress", s);
            k_shortcut<false><<<gv, TPB, 0, s>>>(P, nullptr, g.n, nullptr, d);
        }
        CC_LAUNCH();
        return CC_OK;
    });
}

// flat: labels form a flat forest (as sampling leaves them); counted: the
// count array was already filled (k-out's compression counts as it goes).
cc_status identify_phase(const uint32_t *L, uint32_t n, uint32_t samples, uint64_t seed, uint32_t *lmax_out,
                         Work &w, const DeviceInfo *di, const Dev &d, cudaStream_t s, bool flat, bool counted) {
    if (samples) {
        {
            CC_PROF("k_freq_sampled", s);
            k_freq_sampled<<<1, 1024, 0, s>>>(L, n, samples, seed, lmax_out);
        }
        CC_LAUNCH();
        return CC_OK;
    }
    uint32_t *cnt = w.sc.at<uint32_t>(w.o_counts);
    Ctl *ctl = w.ctl();
    const unsigned gv = grid_for(di, n, TPB);
    // counted: the compression that counted also left the arg-max key
    // (the fused k-out pass: counted below, from its guess)
    if (!counted && !w.lists_built) {
        CC_TRY(cudaMemsetAsync(cnt, 0, (size_t)n * 4, s));
        {
            CC_PROF("k_count_labels", s);
            if (flat) k_count_labels<true><<<gv, TPB, 0, s>>>(L, n, cnt, d);
            else k_count_labels<false><<<gv, TPB, 0, s>>>(L, n, cnt, d);
        }
        CC_TRY(cudaMemsetAsync(&ctl->key, 0, 8, s));
        CC_PROF("k_argmax_counts", s);
        k_argmax_counts<<<gv, TPB, 0, s>>>(cnt, n, &ctl->key);
    }
    if (w.lists_built) {
        // exact L_max: the guess when it holds a majority of the non-roots,
        // else a full count (guarded kernels, returning at once otherwise)
        {
            CC_PROF("k_lmax_majority", s);
            k_lmax_majority<<<1, 1, 0, s>>>(ctl);
        }
        {
            CC_PROF("k_count_fallback", s);
            k_zero_if<<<gv, TPB, 0, s>>>(cnt, n, &ctl->fallback);
            k_count_labels<true><<<gv, TPB, 0, s>>>(L, n, cnt, d, &ctl->fallback);
            k_argmax_counts<<<gv, TPB, 0, s>>>(cnt, n, &ctl->key, &ctl->fallback);
        }
        CC_LAUNCH();
    }
    if (w.lists_built && w.select) {
        // the check plus the selector's features and choice
        if (w.sel_join) CC_TRY(cudaStreamWaitEvent(s, w.sel_join, 0));
        CC_PROF("k_lmax_select", s);
        k_lmax_select<<<1, MLP_H, 0, s>>>(ctl, lmax_out, w.fs + w.fs_parts, n, w.sel_m, w.sel_params,
                                          w.sel_force, w.sel_feat, w.sel_host);
    } else if (w.lists_built) {
        // the fused k-out pass binned against a guess: check it
        CC_PROF("k_lmax_check", s);
        k_lmax_check<<<1, 1, 0, s>>>(ctl, lmax_out);
    } else {
        CC_PROF("k_key_to_label", s);
        k_key_to_label<<<1, 1, 0, s>>>(&ctl->key, lmax_out);
    }
    CC_LAUNCH();
    return CC_OK;
}

// lmax_p: device pointer to L_max, or nullptr for "skip nothing".
// skip (device word, may be null; union-find finishes only): when it reads
// 1 the finish's kernels return at once (the selected path chose another
// finish after these kernels were enqueued).
template <typename OffT>
cc_status finish_phase(const Graph &g, const cc_finish_opt &fo, const uint32_t *lmax_p, uint32_t *P, Work &w,
                       const DeviceInfo *di, const Dev &d, cudaStream_t s, uint32_t *rounds_out,
                       const uint32_t *skip = nullptr) {
    const OffT *I = static_cast<const OffT *>(g.I);
    const uint32_t n = g.n;
    Ctl *ctl = w.ctl();
    ChunkRef *chunks = w.sc.at<ChunkRef>(w.o_chunks);
    const unsigned gv = grid_for(di, n, TPB);
    const unsigned ge = grid_for(di, n, TPB, EDGE_MINB);
    const unsigned gce = grid_for(di, (uint64_t)1 << 40, TPB, EDGE_MINB);
    if (rounds_out) *rounds_out = 0;
    // lists built by the fused k-out pass (against the exact L_max, or
    // cleared by k_lmax_check and rebuilt by the guarded k_cand_bin below)
    const bool built = w.lists_built && lmax_p != nullptr;
    const uint32_t *only_if = built ? &ctl->rebin : nullptr;
    if (!built) {
        CC_TRY(cudaMemsetAsync(&ctl->nchunks, 0, 4, s));
        CC_TRY(cudaMemsetAsync(&ctl->edges, 0, 8, s));
    }
    uint32_t *light = w.sc.at<uint32_t>(w.o_light);
    if (fo.kind == CC_FINISH_UF_REM_CAS || fo.kind == CC_FINISH_UF_ASYNC || fo.kind == CC_FINISH_UF_HOOKS ||
        fo.kind == CC_FINISH_UF_EARLY) {
        // No vertex skipped: one pass, each undirected edge applied once
        // (from its larger endpoint).  With L_max: the candidate set
        // {u : label[u] != L_max} is fixed first (Algorithm 7's filter),
        // then its edges are applied.
        const bool lower_only = (lmax_p == nullptr);
        if (!lower_only) {
            if (!built) CC_TRY(cudaMemsetAsync(&ctl->nlight, 0, 4, s));
            {
                CC_PROF("k_cand_bin", s);
                k_cand_bin<OffT><<<ge, TPB, 0, s>>>(I, n, g.m, P, lmax_p, light, &ctl->nlight, chunks, &ctl->nchunks,
                                                    w.chunk_cap, &ctl->edges, d, only_if, skip);
            }
            CC_LAUNCH();
        }
        cc_status st = with_engine(fo, [&](auto eng) -> cc_status {
            using E = decltype(eng);
            UnionEdge<E> f{P, d, lower_only};
            if (lower_only)
                {
                    CC_PROF("k_range_bin", s);
                    k_range_bin<OffT, UnionEdge<E>><<<gv, TPB, 0, s>>>(I, g.A, n, g.m, P, nullptr, f, chunks,
                                                                       &ctl->nchunks, w.chunk_cap, &ctl->edges, d);
                }
            else
                {
                    CC_PROF("k_light_list", s);
                    k_light_list<OffT, UnionEdge<E>><<<gv, TPB, 0, s>>>(I, g.A, n, g.m, light, &ctl->nlight, f, d,
                                                                         skip);
                }
            {
                CC_PROF("k_chunks", s);
                k_chunks<OffT, UnionEdge<E>><<<gce, TPB, 0, s>>>(I, g.A, n, g.m, chunks, &ctl->nchunks, w.chunk_cap, f, d,
                                                                skip);
            }
            CC_LAUNCH();
            return CC_OK;
        });
        if (st != CC_OK) return st;
        {
            CC_PROF("k_final_shortcut", s);
            k_compress8<<<grid_for(di, n, TPB, 6), TPB, 0, s>>>(P, n, d, skip);
        }
        CC_LAUNCH();
        return CC_OK;
    }
    // SV / LT-PRF and the other min-label finishes: candidate lists once,
    // then rounds until nothing changes.
    if (!built) CC_TRY(cudaMemsetAsync(&ctl->nlight, 0, 4, s));
    {
        CC_PROF("k_cand_bin", s);
        k_cand_bin<OffT><<<ge, TPB, 0, s>>>(I, n, g.m, P, lmax_p, light, &ctl->nlight, chunks, &ctl->nchunks,
                                            w.chunk_cap, &ctl->edges, d, only_if);
    }
    CC_LAUNCH();
    if (fo.kind != CC_FINISH_SV && fo.kind != CC_FINISH_LT_PRF) {
        MinLabelIn in{g.I,     sizeof(OffT) == 8, g.A,           n,         g.m,          P,
                      lmax_p,  light,             &ctl->nlight, chunks,    &ctl->nchunks, w.chunk_cap,
                      &ctl->edges};
        return minlabel_finish(in, fo, di, d, s, rounds_out);
    }
    uint32_t *prev = w.sc.at<uint32_t>(w.o_prev);
    CC_TRY(cudaMemcpyAsync(prev, P, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    uint32_t *hchanged = nullptr;
    CC_TRY(cudaMallocHost(&hchanged, 4));
    struct Free {
        uint32_t *p;
        ~Free() { cudaFreeHost(p); }
    } fr{hchanged};
    const uint32_t cap = round_cap();
    uint32_t rounds = 0;
    for (;;) {
        if (rounds >= cap) {
            {
                CC_PROF("k_or_u32", s);
                k_or_u32<<<1, 1, 0, s>>>(di->err, CC_DEVERR_NONCONVERGED);
            }
            CC_LAUNCH();
            break;
        }
        CC_TRY(cudaMemsetAsync(&ctl->changed, 0, 4, s));
        if (fo.kind == CC_FINISH_SV) {
            SVEdge f{P, prev, &ctl->changed, false};
            {
                CC_PROF("k_light_list", s);
                k_light_list<OffT, SVEdge><<<gv, TPB, 0, s>>>(I, g.A, n, g.m, light, &ctl->nlight, f, d);
            }
            {
                CC_PROF("k_chunks", s);
                k_chunks<OffT, SVEdge><<<gce, TPB, 0, s>>>(I, g.A, n, g.m, chunks, &ctl->nchunks, w.chunk_cap, f, d);
            }
        } else {
            LTEdge f{P, prev, &ctl->changed, false};
            {
                CC_PROF("k_light_list", s);
                k_light_list<OffT, LTEdge><<<gv, TPB, 0, s>>>(I, g.A, n, g.m, light, &ctl->nlight, f, d);
            }
            {
                CC_PROF("k_chunks", s);
                k_chunks<OffT, LTEdge><<<gce, TPB, 0, s>>>(I, g.A, n, g.m, chunks, &ctl->nchunks, w.chunk_cap, f, d);
            }
        }
        {
            CC_PROF("k_shortcut", s);
            k_shortcut<false><<<gv, TPB, 0, s>>>(P, prev, n, nullptr, d);
        }
        CC_LAUNCH();
        ++rounds;
        CC_TRY(cudaMemcpyAsync(hchanged, &ctl->changed, 4, cudaMemcpyDeviceToHost, s));
        CC_TRY(cudaStreamSynchronize(s));
        if (*hchanged == 0) break;
    }
    if (rounds_out) *rounds_out = rounds;
    return CC_OK;
}

void resolve_opts(const cc_sample_opt *sp, const cc_finish_opt *fp, cc_sample_opt &so, cc_finish_opt &fo) {
    cc_default_opts(&so, &fo);
    if (sp) so = *sp;
    if (fp) fo = *fp;
}

template <typename OffT>
cc_status run_static(const Graph &g, const cc_sample_opt &so, const cc_finish_opt &fo, uint32_t *P,
                     cc_stats *stats, cudaStream_t s) {
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    Dev d = make_dev(di, g.n);
    Work w;
    plan(w, g, so.kind, so.freq_samples, fo.kind, true);
    cc_status st = w.sc.alloc(s);
    if (st != CC_OK) return st;
    if ((st = attach_hooks(w, d, g.n, s)) != CC_OK) return st;
    CC_TRY(cudaMemsetAsync(w.ctl(), 0, sizeof(Ctl), s));
    int32_t info = 0;
    const bool fused = so.kind == CC_SAMPLE_KOUT && so.freq_samples == 0;
    st = sample_phase<OffT>(g, so, fo, P, w, di, d, s, &info, fused ? w.sc.at<uint32_t>(w.o_counts) : nullptr);
    if (st != CC_OK) return st;
    const uint32_t *lmax_p = nullptr;
    if (so.kind != CC_SAMPLE_NONE) {
        st = identify_phase(P, g.n, so.freq_samples, so.seed, &w.ctl()->lmax, w, di, d, s, true, fused);
        if (st != CC_OK) return st;
        lmax_p = &w.ctl()->lmax;
    }
    uint32_t rounds = 0;
    st = finish_phase<OffT>(g, fo, lmax_p, P, w, di, d, s, &rounds);
    if (st != CC_OK) return st;
    if (stats) {
        Ctl h;
        CC_TRY(cudaMemcpyAsync(&h, w.ctl(), sizeof(Ctl), cudaMemcpyDeviceToHost, s));
        CC_TRY(cudaStreamSynchronize(s));
        stats->lmax = lmax_p ? h.lmax : NONE;
        stats->sample_info = info;
        stats->rounds = rounds;
        stats->reserved = 0;
        stats->edges_finish = h.edges;
    }
    return CC_OK;
}

// ---------------------------------------------------------------- spanning forest
// Filter step of the spanning-forest algorithm: the non-empty slots of the
// sampling and finish edge arrays, appended to out as (u, v) word pairs.
// A forest has at most n - 1 pairs; more would mean a broken invariant, so
// slots past n are flagged and not written (out holds n pairs).
// Two arrays (BFS / LDD sampling): items 0..n-1 are the sampling edges,
// n..2n-1 the finish edges.
__global__ void __launch_bounds__(256, 8) k_forest_compact(const uint2 *sf, const uint2 *ff, uint32_t n, uint32_t *out,
                                                           uint32_t *count, Dev d) {
    block_compact(
        2ull * n, count, [&](uint64_t i) { return (i < n ? sf[i] : ff[i - n]).x != NONE; },
        [&](uint64_t i, uint32_t k) {
            if (k >= n) { atomicOr(d.err, ERR_NONCONVERGED); return; }
            const uint2 e = i < n ? sf[i] : ff[i - n];
            out[2 * (uint64_t)k] = e.x;
            out[2 * (uint64_t)k + 1] = e.y;
        });
}

// One array (k-out / no sampling): every hooked root ends as a non-root and
// nothing else does, so slot v holds an edge exactly when label[v] != v.
__global__ void __launch_bounds__(256, 8) k_forest_compact_hooked(const uint2 *ff, const uint32_t *L, uint32_t n,
                                                                  uint32_t *out, uint32_t *count, Dev d) {
    block_compact(
        n, count, [&](uint64_t i) { return L[i] != (uint32_t)i; },
        [&](uint64_t i, uint32_t k) {
            if (k >= n) { atomicOr(d.err, ERR_NONCONVERGED); return; }
            const uint2 e = ff[i];
            out[2 * (uint64_t)k] = e.x;
            out[2 * (uint64_t)k + 1] = e.y;
        });
}

// The spanning-forest algorithm: labels and edge arrays initialised, the
// sampling emits its tree edges (k-out: the hooking edges; BFS: the tree
// edge at each child; LDD: the searches' tree edges), IdentifyFrequent, a
// root-based finish stores each hooking edge at the hooked root, and the
// non-empty slots are filtered out.  Sampling edges and finish edges live
// in separate arrays: the sampled clusters are relabelled to their minimum
// member, which may already hold its own tree edge from the sampling.
template <typename OffT>
cc_status run_forest(const Graph &g, const cc_sample_opt &so, const cc_finish_opt &fo, uint32_t *labels,
                     uint32_t *forest_out, uint64_t *count_out, cudaStream_t s) {
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    Dev d = make_dev(di, g.n);
    Work w;
    plan(w, g, so.kind, so.freq_samples, fo.kind, true, true);
    const size_t o_lab = labels ? 0 : w.sc.reserve((size_t)g.n * 4);
    cc_status st = w.sc.alloc(s);
    if (st != CC_OK) return st;
    if ((st = attach_hooks(w, d, g.n, s)) != CC_OK) return st;
    uint32_t *P = labels ? labels : w.sc.at<uint32_t>(o_lab);
    // k-out and no sampling hook roots in one union-find from start to end:
    // one edge array, and a slot is filled exactly when its vertex ends as a
    // non-root, so the array needs no clearing.  BFS / LDD tree edges sit at
    // children, which the relabelling to the smallest member can also make
    // hooked roots, so they take a second, cleared array.
    const bool one = so.kind == CC_SAMPLE_KOUT || so.kind == CC_SAMPLE_NONE;
    uint2 *ff = w.sc.at<uint2>(w.o_ff), *sf = one ? ff : w.sc.at<uint2>(w.o_sf);
    uint32_t *fcount = w.sc.at<uint32_t>(w.o_fcount);
    CC_TRY(cudaMemsetAsync(w.ctl(), 0, sizeof(Ctl), s));
    if (!one) {
        CC_TRY(cudaMemsetAsync(sf, 0xFF, (size_t)g.n * 8, s));
        CC_TRY(cudaMemsetAsync(ff, 0xFF, (size_t)g.n * 8, s));
    }
    CC_TRY(cudaMemsetAsync(fcount, 0, 8, s));
    Dev ds = d, df = d;
    ds.forest = sf;
    df.forest = ff;
    int32_t info = 0;
    const bool fused = so.kind == CC_SAMPLE_KOUT && so.freq_samples == 0;
    st = sample_phase<OffT>(g, so, fo, P, w, di, ds, s, &info, fused ? w.sc.at<uint32_t>(w.o_counts) : nullptr);
    if (st != CC_OK) return st;
    const uint32_t *lmax_p = nullptr;
    if (so.kind != CC_SAMPLE_NONE) {
        st = identify_phase(P, g.n, so.freq_samples, so.seed, &w.ctl()->lmax, w, di, d, s, true, fused);
        if (st != CC_OK) return st;
        lmax_p = &w.ctl()->lmax;
    }
    st = finish_phase<OffT>(g, fo, lmax_p, P, w, di, df, s, nullptr);
    if (st != CC_OK) return st;
    if (one) {
        CC_PROF("k_forest_compact", s);
        k_forest_compact_hooked<<<grid_for(di, g.n, TPB), TPB, 0, s>>>(ff, P, g.n, forest_out, fcount, d);
    } else {
        CC_PROF("k_forest_compact", s);
        k_forest_compact<<<grid_for(di, g.n, TPB), TPB, 0, s>>>(sf, ff, g.n, forest_out, fcount, d);
    }
    CC_LAUNCH();
    uint32_t hc = 0;
    CC_TRY(cudaMemcpyAsync(&hc, fcount, 4, cudaMemcpyDeviceToHost, s));
    CC_TRY(cudaStreamSynchronize(s));
    *count_out = hc < g.n ? hc : g.n;
    return CC_OK;
}

// Host-buffer entry, zero-copy form.  When the CSR lies in pinned host
// memory that the device can address (over NVLink-C2C on Grace-Blackwell),
// k-out sampling reads it in place: the offsets and about two 32-byte
// sectors per vertex, instead of a copy of the whole CSR.  If the frequent
// cluster then holds at least a quarter of the vertices, the finish reads in
// place too (it reads only the other vertices' edges); otherwise the CSR is
// copied to device memory first and the finish reads that copy.
template <typename OffT>
cc_status run_static_zero_copy(const Graph &gz, const void *h_off, const uint32_t *h_edg, const cc_sample_opt &so,
                               const cc_finish_opt &fo, uint32_t *labels_host, cudaStream_t s) {
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    Dev d = make_dev(di, gz.n);
    Work w;
    plan(w, gz, so.kind, so.freq_samples, fo.kind, true);
    const size_t o_lab = w.sc.reserve((size_t)gz.n * 4);
    cc_status st = w.sc.alloc(s);
    if (st != CC_OK) return st;
    if ((st = attach_hooks(w, d, gz.n, s)) != CC_OK) return st;
    uint32_t *P = w.sc.at<uint32_t>(o_lab);
    CC_TRY(cudaMemsetAsync(w.ctl(), 0, sizeof(Ctl), s));
    int32_t info = 0;
    const bool fused = so.freq_samples == 0;
    st = sample_phase<OffT>(gz, so, fo, P, w, di, d, s, &info, fused ? w.sc.at<uint32_t>(w.o_counts) : nullptr);
    if (st != CC_OK) return st;
    st = identify_phase(P, gz.n, so.freq_samples, so.seed, &w.ctl()->lmax, w, di, d, s, true, fused);
    if (st != CC_OK) return st;
    unsigned long long key = 0;
    CC_TRY(cudaMemcpyAsync(&key, &w.ctl()->key, 8, cudaMemcpyDeviceToHost, s));
    CC_TRY(cudaStreamSynchronize(s));
    // with exact counting the key holds the cluster's non-root count (size - 1)
    const uint64_t lsize = (key >> 32) + 1;
    Graph gf = gz;
    Scratch copy;
    if (so.freq_samples != 0 || 4 * lsize < gz.n) {
        const size_t ob = (size_t)(gz.n + 1ull) * sizeof(OffT);
        const size_t o_off = copy.reserve(ob), o_edg = copy.reserve((size_t)gz.m * 4);
        if ((st = copy.alloc(s)) != CC_OK) return st;
        CC_TRY(cudaMemcpyAsync(copy.at<void>(o_off), h_off, ob, cudaMemcpyHostToDevice, s));
        if (gz.m) CC_TRY(cudaMemcpyAsync(copy.at<void>(o_edg), h_edg, (size_t)gz.m * 4, cudaMemcpyHostToDevice, s));
        gf = Graph{copy.at<void>(o_off), gz.u64, gz.m ? copy.at<uint32_t>(o_edg) : nullptr, gz.n, gz.m};
    }
    uint32_t rounds = 0;
    st = finish_phase<OffT>(gf, fo, &w.ctl()->lmax, P, w, di, d, s, &rounds);
    if (st != CC_OK) return st;
    CC_TRY(cudaMemcpyAsync(labels_host, P, (size_t)gz.n * 4, cudaMemcpyDeviceToHost, s));
    CC_TRY(cudaStreamSynchronize(s));
    return CC_OK;
}

// Device address of `bytes` bytes of pinned host memory starting at p, or
// null.  Both the first and the last byte must lie in memory the device
// maps, at the same offset from the device view (one registered region), or
// the kernels could read past the mapping; the caller then takes the copying
// path, where a short buffer fails on the host instead.
const void *host_device_view(const void *p, size_t bytes) {
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a, z;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    const char *last = static_cast<const char *>(p) + (bytes - 1);
    if (cudaPointerGetAttributes(&z, last) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (z.type != cudaMemoryTypeHost || !z.devicePointer ||
        static_cast<const char *>(z.devicePointer) != static_cast<const char *>(a.devicePointer) + (bytes - 1))
        return nullptr;
    return a.devicePointer;
}

// ---------------------------------------------------------------- the selected path
// The learned selector's run (no counterpart in the paper, which picks by a
// hand-made decision tree, Section 4.7).  The default path (k-out k = 2 +
// UF-Rem-CAS) runs as usual; the first k-out pass also gathers the degree
// statistics, and the kernel that checks L_max also forms the 16 features
// and runs the MLP (k_lmax_select).  The default finish is enqueued right
// behind it, guarded by a device word; the host waits only for the choice
// (an event), while the GPU goes on.  If the choice is the default, the
// call returns with the finish in flight.  Otherwise the guarded kernels
// return at once and the host enqueues the chosen path: another finish on
// the same k-out sample and candidate lists, or (BFS / LDD sampling) the
// whole static path.  Every class computes the same labels.
//
// Classes: c = 4 * sampling + finish, sampling 0 k-out, 1 BFS, 2 LDD;
// finish 0 UF-Rem-CAS (FindNaive, SplitAtomicOne), 1 UF-Async (FindSplit),
// 2 SV, 3 Liu-Tarjan PRF.
void class_opts(int c, const cc_sample_opt &base, cc_sample_opt &so, cc_finish_opt &fo) {
    so = base;
    cc_default_opts(nullptr, &fo);
    const int sm = c / 4, fin = c % 4;
    so.kind = sm == 0 ? CC_SAMPLE_KOUT : sm == 1 ? CC_SAMPLE_BFS : CC_SAMPLE_LDD;
    fo.kind = fin == 0 ? CC_FINISH_UF_REM_CAS : fin == 1 ? CC_FINISH_UF_ASYNC : fin == 2 ? CC_FINISH_SV
                                                                                       : CC_FINISH_LT_PRF;
    fo.find = fin == 1 ? CC_FIND_SPLIT : CC_FIND_NAIVE;
}

// Per host thread and device: a word of mapped host memory the choosing
// kernel writes, and the event after that kernel.  (Kept until exit.)
struct SelHost {
    int device = -1;
    int *word = nullptr;
    int *dword = nullptr;
    cudaEvent_t ev = nullptr;
    cudaStream_t side = nullptr;          // the degree statistics run here
    cudaEvent_t fork = nullptr, join = nullptr;
};

cc_status sel_host(const DeviceInfo *di, SelHost **out) {
    thread_local SelHost h;
    if (h.device != di->device) {
        SelHost x;
        CC_TRY(cudaHostAlloc(reinterpret_cast<void **>(&x.word), 64, cudaHostAllocMapped | cudaHostAllocPortable));
        CC_TRY(cudaHostGetDevicePointer(reinterpret_cast<void **>(&x.dword), x.word, 0));
        CC_TRY(cudaEventCreateWithFlags(&x.ev, cudaEventDisableTiming));
        CC_TRY(cudaStreamCreateWithFlags(&x.side, cudaStreamNonBlocking));
        CC_TRY(cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming));
        CC_TRY(cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming));
        x.device = di->device;
        h = x;
    }
    *out = &h;
    return CC_OK;
}

// features_only: stop after the features (class 0, nothing else runs; P
// holds the k-out sample).  force >= 0: run that class whatever the MLP
// says (the selector's training times each class this way).
template <typename OffT>
cc_status run_select(const Graph &g, const float *params, int force, uint64_t seed, uint32_t *P, float *feat_out,
                     int32_t *class_out, bool features_only, cudaStream_t s) {
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    Dev d = make_dev(di, g.n);
    cc_sample_opt so;
    cc_finish_opt fo;
    cc_default_opts(&so, &fo);
    so.seed = seed;
    Work w;
    plan(w, g, CC_SAMPLE_KOUT, 0, CC_FINISH_UF_REM_CAS, true);
    // SV / LT-PRF on the same sample need the round-start copy
    w.has_sv = true;
    w.o_prev = w.sc.reserve((size_t)g.n * 4);
    // k_degree_stats runs grid_for(n) blocks, one partial each, plus the sum
    w.fs_parts = grid_for(di, g.n, TPB, 4);
    const size_t o_fs = w.sc.reserve((size_t)(w.fs_parts + 1) * sizeof(FeatStats));
    cc_status st = w.sc.alloc(s);
    if (st != CC_OK) return st;
    SelHost *h = nullptr;
    if ((st = sel_host(di, &h)) != CC_OK) return st;
    w.fs = w.sc.at<FeatStats>(o_fs);
    w.select = true;
    w.sel_params = features_only ? nullptr : params;
    w.sel_force = features_only ? -1 : force;
    w.sel_feat = feat_out;
    w.sel_host = features_only ? nullptr : h->dword;
    w.sel_m = g.m;
    CC_TRY(cudaMemsetAsync(w.ctl(), 0, sizeof(Ctl), s));
    // the degree statistics on the side stream, concurrent with the sample
    CC_TRY(cudaEventRecord(h->fork, s));
    CC_TRY(cudaStreamWaitEvent(h->side, h->fork, 0));
    {
        CC_PROF("k_degree_stats", h->side);
        k_degree_stats<OffT><<<w.fs_parts, TPB, 0, h->side>>>(static_cast<const OffT *>(g.I), g.n, g.m, w.fs,
                                                               &w.ctl()->stats_done, d);
    }
    CC_LAUNCH();
    CC_TRY(cudaEventRecord(h->join, h->side));
    w.sel_join = h->join;
    int32_t info = 0;
    if ((st = sample_phase<OffT>(g, so, fo, P, w, di, d, s, &info, w.sc.at<uint32_t>(w.o_counts))) != CC_OK)
        return st;
    if (!w.lists_built) return CC_ERR_INVALID;   // not reached: k = 2 with a finish always fuses
    if ((st = identify_phase(P, g.n, 0, seed, &w.ctl()->lmax, w, di, d, s, true, true)) != CC_OK) return st;
    if (features_only) {
        if (class_out) *class_out = 0;
        return CC_OK;
    }
    CC_TRY(cudaEventRecord(h->ev, s));
    const uint32_t *lmax_p = &w.ctl()->lmax;
    if ((st = finish_phase<OffT>(g, fo, lmax_p, P, w, di, d, s, nullptr, &w.ctl()->skip)) != CC_OK) return st;
    CC_TRY(cudaEventSynchronize(h->ev));
    const int cls = *h->word & 0xFF;
    if (class_out) *class_out = cls;
    if (cls == 0) return CC_OK;
    cc_sample_opt so2;
    cc_finish_opt fo2;
    class_opts(cls, so, so2, fo2);
    if (so2.kind == CC_SAMPLE_KOUT) {
        // another finish on the same sample (the lists are rebuilt first if
        // the L_max guess was wrong)
        uint32_t rounds = 0;
        return finish_phase<OffT>(g, fo2, lmax_p, P, w, di, d, s, &rounds);
    }
    w.sc.release();
    return run_static<OffT>(g, so2, fo2, P, nullptr, s);
}

}  // namespace

// ================================================================ C ABI
extern "C" {

cc_status cc_static_ex(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                       const cc_sample_opt *sample, const cc_finish_opt *finish, uint32_t *labels_out,
                       cc_stats *stats, void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK) return st;
    cc_sample_opt so;
    cc_finish_opt fo;
    resolve_opts(sample, finish, so, fo);
    if ((st = check_sample(so)) != CC_OK || (st = check_finish(fo)) != CC_OK) return st;
    if (n > 0 && (!labels_out || !aligned(labels_out, 4))) return CC_ERR_INVALID;
    if (n == 0) {
        if (stats) *stats = cc_stats{NONE, 0, 0, 0, 0};
        return CC_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Graph g{offsets, offsets_u64 != 0, edges, n, m};
    st = offsets_u64 ? run_static<uint64_t>(g, so, fo, labels_out, stats, s)
                     : run_static<uint32_t>(g, so, fo, labels_out, stats, s);
    if (st != CC_OK || !stats) return st;
    return cc_device_error(stream, nullptr);
}

cc_status cc_static(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                    const cc_sample_opt *sample, const cc_finish_opt *finish, uint32_t *labels_out, void *stream) {
    return cc_static_ex(offsets, offsets_u64, edges, n, m, sample, finish, labels_out, nullptr, stream);
}

cc_status cc_spanning_forest(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                             const cc_sample_opt *sample, const cc_finish_opt *finish, uint32_t *forest_out,
                             uint64_t *count_out, uint32_t *labels_out, void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK) return st;
    cc_sample_opt so;
    cc_finish_opt fo;
    resolve_opts(sample, finish, so, fo);
    if ((st = check_sample(so)) != CC_OK || (st = check_finish(fo)) != CC_OK) return st;
    // root-based union-find finishes only (not SV / Liu-Tarjan / Stergiou /
    // label propagation, not Rem with SpliceAtomic)
    if (fo.kind != CC_FINISH_UF_REM_CAS && fo.kind != CC_FINISH_UF_ASYNC && fo.kind != CC_FINISH_UF_HOOKS &&
        fo.kind != CC_FINISH_UF_EARLY)
        return CC_ERR_UNSUPPORTED;
    if (fo.kind == CC_FINISH_UF_REM_CAS && fo.splice == CC_SPLICE_ATOMIC) return CC_ERR_UNSUPPORTED;
    if (!count_out) return CC_ERR_INVALID;
    if (n > 0 && (!forest_out || !aligned(forest_out, 4))) return CC_ERR_INVALID;
    if (labels_out && !aligned(labels_out, 4)) return CC_ERR_INVALID;
    *count_out = 0;
    if (n == 0) return CC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Graph g{offsets, offsets_u64 != 0, edges, n, m};
    st = offsets_u64 ? run_forest<uint64_t>(g, so, fo, labels_out, forest_out, count_out, s)
                     : run_forest<uint32_t>(g, so, fo, labels_out, forest_out, count_out, s);
    if (st != CC_OK) return st;
    return cc_device_error(stream, nullptr);
}

cc_status cc_static_host(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                         const cc_sample_opt *sample, const cc_finish_opt *finish, uint32_t *labels_out,
                         void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK) return st;
    if (n == 0) return CC_OK;
    if (!labels_out) return CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t ob = (size_t)(n + 1ull) * (offsets_u64 ? 8 : 4);
    cc_sample_opt so;
    cc_finish_opt fo;
    resolve_opts(sample, finish, so, fo);
    if ((st = check_sample(so)) != CC_OK || (st = check_finish(fo)) != CC_OK) return st;
    const void *voff = host_device_view(offsets, ob), *vedg = m ? host_device_view(edges, (size_t)m * 4) : nullptr;
    if (so.kind == CC_SAMPLE_KOUT && voff && (vedg || !m) && aligned(voff, offsets_u64 ? 8 : 4) &&
        (!m || aligned(vedg, 4))) {
        Graph gz{voff, offsets_u64 != 0, static_cast<const uint32_t *>(vedg), n, m};
        st = offsets_u64 ? run_static_zero_copy<uint64_t>(gz, offsets, edges, so, fo, labels_out, s)
                         : run_static_zero_copy<uint32_t>(gz, offsets, edges, so, fo, labels_out, s);
        if (st != CC_OK) return st;
        return cc_device_error(stream, nullptr);
    }
    Scratch sc;
    const size_t o_off = sc.reserve(ob), o_edg = sc.reserve((size_t)m * 4), o_lab = sc.reserve((size_t)n * 4);
    if ((st = sc.alloc(s)) != CC_OK) return st;
    CC_TRY(cudaMemcpyAsync(sc.at<void>(o_off), offsets, ob, cudaMemcpyHostToDevice, s));
    if (m) CC_TRY(cudaMemcpyAsync(sc.at<void>(o_edg), edges, (size_t)m * 4, cudaMemcpyHostToDevice, s));
    st = cc_static(sc.at<void>(o_off), offsets_u64, m ? sc.at<uint32_t>(o_edg) : nullptr, n, m, sample, finish,
                   sc.at<uint32_t>(o_lab), stream);
    if (st != CC_OK) return st;
    CC_TRY(cudaMemcpyAsync(labels_out, sc.at<uint32_t>(o_lab), (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    sc.release();
    return cc_device_error(stream, nullptr);
}

cc_status cc_sample(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                    const cc_sample_opt *sample, uint32_t *labels_out, int32_t *sample_info_out, void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK) return st;
    cc_sample_opt so;
    cc_finish_opt fo;
    resolve_opts(sample, nullptr, so, fo);
    if ((st = check_sample(so)) != CC_OK) return st;
    if (n == 0) return CC_OK;
    if (!labels_out || !aligned(labels_out, 4)) return CC_ERR_INVALID;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Graph g{offsets, offsets_u64 != 0, edges, n, m};
    Work w;
    plan(w, g, so.kind, 1 /* no count array */, fo.kind, false);
    if ((st = w.sc.alloc(s)) != CC_OK) return st;
    CC_TRY(cudaMemsetAsync(w.ctl(), 0, sizeof(Ctl), s));
    int32_t info = 0;
    Dev d = make_dev(di, n);
    if ((st = attach_hooks(w, d, n, s)) != CC_OK) return st;
    st = offsets_u64 ? sample_phase<uint64_t>(g, so, fo, labels_out, w, di, d, s, &info, nullptr)
                     : sample_phase<uint32_t>(g, so, fo, labels_out, w, di, d, s, &info, nullptr);
    if (st != CC_OK) return st;
    if (sample_info_out) {
        CC_TRY(cudaStreamSynchronize(s));
        *sample_info_out = info;
    }
    return CC_OK;
}

cc_status cc_identify_frequent(const uint32_t *labels, uint32_t n, uint32_t freq_samples, uint64_t seed,
                               uint32_t *lmax_out, void *stream) {
    if (n == 0xFFFFFFFFu || freq_samples > 4096) return CC_ERR_INVALID;
    if (!lmax_out || (n > 0 && !labels) || !aligned(lmax_out, 4) || (labels && !aligned(labels, 4)))
        return CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        {
            CC_PROF("k_set_u32", s);
            k_set_u32<<<1, 1, 0, s>>>(lmax_out, NONE);
        }
        return from_cuda(cudaGetLastError());
    }
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    Work w;
    w.o_ctl = w.sc.reserve(sizeof(Ctl));
    if (freq_samples == 0) w.o_counts = w.sc.reserve((size_t)n * 4);
    cc_status st = w.sc.alloc(s);
    if (st != CC_OK) return st;
    return identify_phase(labels, n, freq_samples, seed, lmax_out, w, di, make_dev(di, n), s, false, false);
}

cc_status cc_finish(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                    const cc_finish_opt *finish, uint32_t lmax, uint32_t *labels_inout, uint32_t *rounds_out,
                    void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK) return st;
    cc_sample_opt so;
    cc_finish_opt fo;
    resolve_opts(nullptr, finish, so, fo);
    if ((st = check_finish(fo)) != CC_OK) return st;
    if (n == 0) return CC_OK;
    if (!labels_inout || !aligned(labels_inout, 4)) return CC_ERR_INVALID;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Graph g{offsets, offsets_u64 != 0, edges, n, m};
    Work w;
    plan(w, g, CC_SAMPLE_NONE, 1, fo.kind, true);
    if ((st = w.sc.alloc(s)) != CC_OK) return st;
    Dev d = make_dev(di, n);
    if ((st = attach_hooks(w, d, n, s)) != CC_OK) return st;
    CC_TRY(cudaMemsetAsync(w.ctl(), 0, sizeof(Ctl), s));
    {
        CC_PROF("k_check_forest", s);
        k_check_forest<<<grid_for(di, n, TPB), TPB, 0, s>>>(labels_inout, n, d);
    }
    {
        CC_PROF("k_set_u32", s);
        k_set_u32<<<1, 1, 0, s>>>(&w.ctl()->lmax, lmax);
    }
    CC_LAUNCH();
    const uint32_t *lmax_p = lmax == NONE ? nullptr : &w.ctl()->lmax;
    uint32_t rounds = 0;
    st = offsets_u64 ? finish_phase<uint64_t>(g, fo, lmax_p, labels_inout, w, di, d, s, &rounds)
                     : finish_phase<uint32_t>(g, fo, lmax_p, labels_inout, w, di, d, s, &rounds);
    if (rounds_out) *rounds_out = rounds;
    return st;
}

}  // extern "C"

extern "C" cc_status cc_features(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                                 uint64_t seed, float *feat_out, void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK) return st;
    if (n == 0 || !feat_out || !aligned(feat_out, 4)) return CC_ERR_INVALID;
    Graph g{offsets, offsets_u64 != 0, edges, n, m};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    const size_t op = sc.reserve((size_t)n * 4);
    if ((st = sc.alloc(s)) != CC_OK) return st;
    uint32_t *P = sc.at<uint32_t>(op);
    return offsets_u64 ? run_select<uint64_t>(g, nullptr, -1, seed, P, feat_out, nullptr, true, s)
                       : run_select<uint32_t>(g, nullptr, -1, seed, P, feat_out, nullptr, true, s);
}

extern "C" cc_status cc_select_static(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n,
                                      uint64_t m, const float *params, int force_class, uint64_t seed,
                                      uint32_t *labels_out, float *feat_out, int32_t *class_out, void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK) return st;
    if (!labels_out || !aligned(labels_out, 4) || (feat_out && !aligned(feat_out, 4))) return CC_ERR_INVALID;
    if (force_class >= CC_MLP_OUT || (force_class < 0 && !params)) return CC_ERR_INVALID;
    if (params && !aligned(params, 4)) return CC_ERR_INVALID;
    if (n == 0) {
        if (class_out) *class_out = force_class >= 0 ? force_class : 0;
        return CC_OK;
    }
    Graph g{offsets, offsets_u64 != 0, edges, n, m};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return offsets_u64 ? run_select<uint64_t>(g, params, force_class, seed, labels_out, feat_out, class_out, false, s)
                       : run_select<uint32_t>(g, params, force_class, seed, labels_out, feat_out, class_out, false, s);
}
