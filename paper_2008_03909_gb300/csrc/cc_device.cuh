// cc_device.cuh -- device primitives shared by the connectivity kernels:
// relaxed loads, bounded loops, counter-based draws, the union-find engines
// of Section 3.3.1 (Algorithms 8-10 and 14) and the degree-binned edge
// traversal every edge-processing kernel uses.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cooperative_groups.h>

namespace ccg {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t ERR_BAD_EDGE = 1u;
constexpr uint32_t ERR_BAD_OFFSETS = 2u;
constexpr uint32_t ERR_NONCONVERGED = 4u;
constexpr uint64_t OP_TIME_LIMIT_NS = 4000000000ull;  // one find/union may run 4 s at most

enum { FIND_NAIVE = 0, FIND_SPLIT = 1, FIND_HALVE = 2, FIND_COMPRESS = 3 };
enum { SPLICE_SPLIT_ONE = 0, SPLICE_HALVE_ONE = 1, SPLICE_ATOMIC = 2 };

// Degree binning: vertices of degree <= LIGHT_MAX are handled by one thread;
// the edges of heavier vertices are cut into chunks of <= CHUNK edges, each
// handled by one warp, so a hub with millions of edges spreads over the grid.
constexpr uint32_t LIGHT_MAX = 32;
constexpr uint32_t CHUNK = 2048;

// Per-launch context passed by value.
struct Dev {
    uint32_t *err;             // per-device sticky error word (CC_DEVERR_* bits)
    uint64_t cap;              // iteration cap of one device loop
    uint2 *forest = nullptr;   // spanning forest: edges[r] = the edge that hooked root r
    uint32_t *hooks = nullptr; // UF-Hooks: the hooks array H (NONE = free)
};

// ---------------------------------------------------------------- loads
// A relaxed, device-scope load of a parent slot: sees other SMs' writes
// (the starred reads of Algorithms 8, 9 and 14 are such loads).
__device__ __forceinline__ uint32_t ld_rel(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Streamed read-only input (CSR edges): evict-first in L1 and L2 so the
// parent array keeps the cache.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) { return __ldcs(p); }
template <typename T>
__device__ __forceinline__ T ld_off(const T *p) { return __ldg(p); }
// L1-cacheable read of a parent slot, for first reads whose staleness is
// harmless: parent values only ever decrease within one tree, so an older
// value is still an ancestor in the same set, two equal reads still prove
// "same set", and every CAS re-validates.  Hub slots read by millions of
// threads then hit in L1 instead of hammering one L2 slice.
__device__ __forceinline__ uint32_t ld_ca(const uint32_t *p) { return __ldca(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounds one device loop by an iteration cap and a wall-clock limit; when
// either is reached it records ERR_NONCONVERGED and tells the loop to stop.
struct Guard {
    uint64_t it = 0, t0 = 0;
    __device__ __forceinline__ bool step(const Dev &d) {
        if (++it > d.cap) { atomicOr(d.err, ERR_NONCONVERGED); return false; }
        if ((it & 1023) == 0) {
            uint64_t t = gtimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > OP_TIME_LIMIT_NS) { atomicOr(d.err, ERR_NONCONVERGED); return false; }
        }
        return true;
    }
};

// ---------------------------------------------------------------- grid barrier
__device__ __forceinline__ uint32_t ld_acq(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_rel64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over every block of a cooperative launch (all blocks are
// co-resident).  A block reads the generation, then arrives; the last
// arrival resets the count and publishes the next generation with a
// release store.  The wait is bounded by OP_TIME_LIMIT_NS: a block that
// gives up records ERR_NONCONVERGED and sets `abort`, and from then on
// every block's grid_sync returns false, so all blocks leave the kernel.
struct GridBar {
    uint32_t count;
    uint32_t gen;
    uint32_t abort;
    uint32_t pad;
};

__device__ __forceinline__ bool grid_sync(GridBar *b, const Dev &d, uint64_t limit_ns = OP_TIME_LIMIT_NS) {
    __shared__ uint32_t ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t g = ld_acq(&b->gen);
        __threadfence();
        bool ok = true;
        if (atomicAdd(&b->count, 1u) + 1 == gridDim.x) {
            atomicExch(&b->count, 0u);
            st_rel(&b->gen, g + 1);
        } else {
            const uint64_t t0 = gtimer();
            while (ld_acq(&b->gen) == g) {
                if (ld_rel(&b->abort)) { ok = false; break; }
                if (gtimer() - t0 > limit_ns) {
                    atomicOr(d.err, ERR_NONCONVERGED);
                    atomicExch(&b->abort, 1u);
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        ok_s = ok && ld_rel(&b->abort) == 0;
    }
    __syncthreads();
    return ok_s != 0;
}

// ---------------------------------------------------------------- draws
// Counter-based draws: the ctr-th output of a SplitMix64 sequence started at
// state s (Steele, Lea, Flood, OOPSLA 2014), mix64(s + (ctr+1) * gamma).
__host__ __device__ __forceinline__ uint64_t draw64(uint64_t s, uint64_t ctr) {
    uint64_t z = s + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
constexpr uint64_t TAG_KOUT = 0x6B6F7574ull;
constexpr uint64_t TAG_FREQ = 0x66726571ull;
constexpr uint64_t TAG_BFS = 0x62667373ull;

// k-out selection rules (Appendix C.4): hybrid takes the first edge and
// k - 1 uniform picks, afforest the first k edges, pure k uniform picks.
enum { KOUT_HYBRID = 0, KOUT_AFFOREST = 1, KOUT_PURE = 2 };
constexpr uint64_t NO_PICK = ~0ull;

// Position of pick j (0 <= j < k) of vertex v in its adjacency list of
// length deg > 0, or NO_PICK (afforest past the degree).  A uniform pick is
// floor(hi32(out(seed ^ TAG_KOUT, v*k + j)) * deg / 2^32), with replacement.
__device__ __forceinline__ uint64_t kout_offset(uint32_t rule, uint64_t seed, uint64_t v, uint32_t k, uint32_t j,
                                                uint64_t deg) {
    if (rule == KOUT_AFFOREST) return j < deg ? j : NO_PICK;
    if (rule == KOUT_HYBRID && j == 0) return 0;
    return ((draw64(seed ^ TAG_KOUT, v * k + j) >> 32) * deg) >> 32;
}

// ---------------------------------------------------------------- finds
// Root of x given px = P[x] (Algorithm 8): FindNaive follows parents;
// FindAtomicSplit points each visited node at its grandparent and moves to
// the parent; FindAtomicHalve does the same and moves to the grandparent;
// FindCompress finds the root r, then walks the path again pointing every
// node whose parent is above r straight at r (plain stores: the nodes are
// non-roots, which never become roots again, and r is an ancestor of each).
template <int FIND>
__device__ __forceinline__ uint32_t find_from(uint32_t *P, uint32_t x, uint32_t px, const Dev &d) {
    Guard g;
    if (FIND == FIND_NAIVE) {
        while (px != x) {
            x = px;
            px = ld_rel(P + x);
            if (!g.step(d)) break;
        }
        return x;
    } else if (FIND == FIND_SPLIT) {
        uint32_t v = px;
        if (v == x) return x;
        uint32_t w = ld_rel(P + v);
        while (v != w) {
            atomicCAS(P + x, v, w);
            x = v;
            v = w;
            w = ld_rel(P + v);
            if (!g.step(d)) break;
        }
        return v;
    } else if (FIND == FIND_HALVE) {
        uint32_t v = px;
        if (v == x) return x;
        uint32_t w = ld_rel(P + v);
        while (v != w) {
            atomicCAS(P + x, v, w);
            x = w;
            v = ld_rel(P + x);
            if (v == x) return x;
            w = ld_rel(P + v);
            if (!g.step(d)) break;
        }
        return v;
    } else {
        if (px == x) return x;
        uint32_t r = px, pr = ld_rel(P + r);
        while (pr != r) {
            r = pr;
            pr = ld_rel(P + r);
            if (!g.step(d)) return r;
        }
        uint32_t j = px;
        while (j > r) {
            P[x] = r;
            x = j;
            j = ld_rel(P + x);
            if (!g.step(d)) break;
        }
        return r;
    }
}

// ---------------------------------------------------------------- unions
// Every engine keeps P[x] <= x: a root is only ever linked under a smaller
// id, so every root is the minimum of its tree and the final roots are the
// canonical labels.  All but UF-Rem-CAS with SpliceAtomic are root-based in
// the sense of the spanning-forest appendix: a link hooks a root exactly
// once, so when d.forest is set the hooking edge (u, v) is stored at the
// hooked root's slot.  pu = P[u] and pv = P[v] are passed in already loaded
// (callers batch those loads); pu == pv means nothing to do.  unite returns
// the root it hooked, or NONE when the two were already in one tree.

// UF-Async (Algorithm 10; the CAS is on the larger root's own slot): find
// both roots, CAS the larger root under the smaller, retry from the current
// roots if another thread linked first.
template <int FIND>
struct UnionAsync {
    static constexpr int find_kind = FIND;
    __device__ static __forceinline__ uint32_t unite(uint32_t *P, uint32_t u, uint32_t v, uint32_t pu,
                                                 uint32_t pv, const Dev &d) {
        uint32_t ru = find_from<FIND>(P, u, pu, d);
        uint32_t rv = find_from<FIND>(P, v, pv, d);
        Guard g;
        while (ru != rv) {
            if (ru < rv) { uint32_t t = ru; ru = rv; rv = t; }
            uint32_t old = atomicCAS(P + ru, ru, rv);
            if (old == ru) {
                if (d.forest) d.forest[ru] = make_uint2(u, v);
                return ru;
            }
            ru = find_from<FIND>(P, ru, old, d);
            rv = find_from<FIND>(P, rv, ld_rel(P + rv), d);
            if (!g.step(d)) return NONE;
        }
        return NONE;
    }
};

// UF-Hooks (Algorithm 11; the CAS is read as on H[p_u]): as UF-Async, but
// the larger root is claimed by a CAS on the hooks array, and the winner
// then writes P[p_u] with a plain store (nobody else writes a claimed
// root's slot).  A thread that loses the claim continues from the parent
// the winner is writing (the hooks entry), instead of polling P[p_u].
template <int FIND>
struct UnionHooks {
    static constexpr int find_kind = FIND;
    __device__ static __forceinline__ uint32_t unite(uint32_t *P, uint32_t u, uint32_t v, uint32_t pu,
                                                 uint32_t pv, const Dev &d) {
        uint32_t ru = find_from<FIND>(P, u, pu, d);
        uint32_t rv = find_from<FIND>(P, v, pv, d);
        Guard g;
        while (ru != rv) {
            if (ru < rv) { uint32_t t = ru; ru = rv; rv = t; }
            uint32_t pr = ld_rel(P + ru);
            if (pr == ru) {
                const uint32_t h = atomicCAS(d.hooks + ru, NONE, rv);
                if (h == NONE) {
                    st_rel(P + ru, rv);
                    if (d.forest) d.forest[ru] = make_uint2(u, v);
                    return ru;
                }
                // claimed by another union whose store may not be visible
                // yet: continue from the parent it is about to write
                pr = h;
            }
            ru = find_from<FIND>(P, pr, ld_rel(P + pr), d);
            rv = find_from<FIND>(P, rv, ld_rel(P + rv), d);
            if (!g.step(d)) return NONE;
        }
        return NONE;
    }
};

// UF-Early (Algorithm 12; the CAS is read as on P[p_u]): walk both sides
// together; whenever the larger side is a root, try to hook it under the
// other side's current vertex (smaller, so in another tree); otherwise one
// path-halving step on the larger side.  Then the optional find from both
// endpoints compresses their paths.
template <int FIND>
struct UnionEarly {
    static constexpr int find_kind = FIND;
    __device__ static __forceinline__ uint32_t unite(uint32_t *P, uint32_t u, uint32_t v, uint32_t pu,
                                                 uint32_t pv, const Dev &d) {
        uint32_t ru = pu, rv = pv;
        uint32_t linked = NONE;
        Guard g;
        while (ru != rv) {
            if (!g.step(d)) return NONE;
            if (ru < rv) { uint32_t t = ru; ru = rv; rv = t; }
            const uint32_t z = ld_rel(P + ru);
            if (z == ru) {
                if (atomicCAS(P + ru, ru, rv) == ru) {
                    if (d.forest) d.forest[ru] = make_uint2(u, v);
                    linked = ru;
                    break;
                }
                continue;   // linked by another thread: no longer a root
            }
            const uint32_t w = ld_rel(P + z);
            if (w != z) atomicCAS(P + ru, z, w);
            ru = w;
        }
        if (FIND != FIND_NAIVE) {
            find_from<FIND>(P, u, ld_rel(P + u), d);
            find_from<FIND>(P, v, ld_rel(P + v), d);
        }
        return linked;
    }
};

// UF-Rem-CAS (Algorithm 14): walk r_u, r_v upward comparing parents; when
// the side with the larger parent is a root, CAS it under the other side's
// parent; otherwise take one splice step there (SplitAtomicOne: compact one
// link and move to the parent; HalveAtomicOne: compact and move to the
// grandparent; SpliceAtomic: swing r_u's parent to r_v's smaller parent and
// move to r_u's old parent, Algorithm 9).  After a successful link the
// optional Compress (FindAtomicSplit / FindAtomicHalve) runs from both
// endpoints.  SpliceAtomic moves non-roots between trees, so it is correct
// only phase-concurrently (unions and finds separated, as every caller
// here does) and is not root-based.
template <int SPLICE, int FIND>
struct UnionRem {
    static constexpr int find_kind = FIND;
    __device__ static __forceinline__ uint32_t unite(uint32_t *P, uint32_t u, uint32_t v, uint32_t pu,
                                                 uint32_t pv, const Dev &d) {
        uint32_t ru = u, rv = v, pru = pu, prv = pv;
        Guard g;
        while (pru != prv) {
            if (pru < prv) {
                uint32_t t = ru; ru = rv; rv = t;
                t = pru; pru = prv; prv = t;
            }
            if (ru == pru) {
                uint32_t old = atomicCAS(P + ru, ru, prv);
                if (old == ru) {
                    if (d.forest) d.forest[ru] = make_uint2(u, v);
                    if (FIND != FIND_NAIVE) {
                        find_from<FIND>(P, u, ld_rel(P + u), d);
                        find_from<FIND>(P, v, ld_rel(P + v), d);
                    }
                    return ru;
                }
                pru = old;
            } else if (SPLICE == SPLICE_SPLIT_ONE) {
                uint32_t w = ld_rel(P + pru);
                if (pru != w) atomicCAS(P + ru, pru, w);
                ru = pru;
                pru = w;
            } else if (SPLICE == SPLICE_ATOMIC) {
                atomicCAS(P + ru, pru, prv);
                ru = pru;
                pru = ld_rel(P + ru);
            } else {
                uint32_t w = ld_rel(P + pru);
                if (pru != w) {
                    atomicCAS(P + ru, pru, w);
                    ru = w;
                    pru = ld_rel(P + w);
                } else {
                    ru = pru;
                }
            }
            if (!g.step(d)) return NONE;
        }
        return NONE;
    }
};

// Calls fn(Engine{}) with the union-find engine the finish options name
// (kind, find, splice); the min-label finishes (SV, Liu-Tarjan, Stergiou,
// label propagation) use UF-Rem-CAS for their k-out sampling.  Options are
// validated before this is reached.
template <class Fn>
__host__ auto with_uf_engine(int kind, int find, int splice, Fn &&fn) {
    switch (kind) {
        case 1:   // UF-Async
            switch (find) {
                case FIND_NAIVE: return fn(UnionAsync<FIND_NAIVE>{});
                case FIND_SPLIT: return fn(UnionAsync<FIND_SPLIT>{});
                case FIND_HALVE: return fn(UnionAsync<FIND_HALVE>{});
                default: return fn(UnionAsync<FIND_COMPRESS>{});
            }
        case 4:   // UF-Hooks
            switch (find) {
                case FIND_NAIVE: return fn(UnionHooks<FIND_NAIVE>{});
                case FIND_SPLIT: return fn(UnionHooks<FIND_SPLIT>{});
                case FIND_HALVE: return fn(UnionHooks<FIND_HALVE>{});
                default: return fn(UnionHooks<FIND_COMPRESS>{});
            }
        case 5:   // UF-Early
            switch (find) {
                case FIND_NAIVE: return fn(UnionEarly<FIND_NAIVE>{});
                case FIND_SPLIT: return fn(UnionEarly<FIND_SPLIT>{});
                case FIND_HALVE: return fn(UnionEarly<FIND_HALVE>{});
                default: return fn(UnionEarly<FIND_COMPRESS>{});
            }
        default:
            break;
    }
    if (kind != 0) { find = FIND_NAIVE; splice = SPLICE_SPLIT_ONE; }   // k-out under the min-label finishes
    switch (splice * 3 + find) {
        case 0: return fn(UnionRem<SPLICE_SPLIT_ONE, FIND_NAIVE>{});
        case 1: return fn(UnionRem<SPLICE_SPLIT_ONE, FIND_SPLIT>{});
        case 2: return fn(UnionRem<SPLICE_SPLIT_ONE, FIND_HALVE>{});
        case 3: return fn(UnionRem<SPLICE_HALVE_ONE, FIND_NAIVE>{});
        case 4: return fn(UnionRem<SPLICE_HALVE_ONE, FIND_SPLIT>{});
        case 5: return fn(UnionRem<SPLICE_HALVE_ONE, FIND_HALVE>{});
        case 6: return fn(UnionRem<SPLICE_ATOMIC, FIND_NAIVE>{});
        case 7: return fn(UnionRem<SPLICE_ATOMIC, FIND_SPLIT>{});
        default: return fn(UnionRem<SPLICE_ATOMIC, FIND_HALVE>{});
    }
}

// ---------------------------------------------------------------- CSR ranges
__device__ __forceinline__ void clamp_range(uint64_t s, uint64_t t, uint64_t m, uint64_t &b, uint64_t &e,
                                            const Dev &d) {
    if (t > m || s > t) {
        atomicOr(d.err, ERR_BAD_OFFSETS);
        if (t > m) t = m;
        if (s > t) s = t;
    }
    b = s;
    e = t;
}

template <typename OffT>
__device__ __forceinline__ void vertex_range(const OffT *I, uint32_t u, uint64_t m, uint64_t &b,
                                             uint64_t &e, const Dev &d) {
    uint64_t s = (uint64_t)ld_off(I + u), t = (uint64_t)ld_off(I + u + 1);
    if (t > m || s > t) {
        atomicOr(d.err, ERR_BAD_OFFSETS);
        if (t > m) t = m;
        if (s > t) s = t;
    }
    b = s;
    e = t;
}

// Vertex-group loads: lane L of a warp owns vertices v0 = base + 4L ..
// v0 + 3 and reads their four labels and five offsets with 16-byte vector
// loads when the arrays are aligned (I[v0+4] comes from the next lane).
// Entries past n read as NONE / 0.  Every lane of the warp must call them.
__device__ __forceinline__ void load_labels4(const uint32_t *P, uint64_t v0, uint64_t n, uint32_t (&l)[4]) {
    if (v0 + 3 < n && ((reinterpret_cast<uintptr_t>(P) & 15) == 0)) {
        uint4 q = __ldcg(reinterpret_cast<const uint4 *>(P + v0));
        l[0] = q.x; l[1] = q.y; l[2] = q.z; l[3] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) l[j] = v0 + j < n ? P[v0 + j] : NONE;
    }
}

template <typename OffT>
__device__ __forceinline__ void load_offsets5(const OffT *I, uint64_t v0, uint64_t n, uint64_t (&o)[5]) {
    const int lane = threadIdx.x & 31;
    if (v0 + 3 < n && ((reinterpret_cast<uintptr_t>(I) & 15) == 0)) {
        if (sizeof(OffT) == 8) {
            const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(I + v0);
            ulonglong2 a = __ldg(q), b = __ldg(q + 1);
            o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
        } else {
            uint4 a = __ldg(reinterpret_cast<const uint4 *>(I + v0));
            o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = v0 + j <= n ? (uint64_t)ld_off(I + v0 + j) : 0;
    }
    uint64_t nxt = __shfl_down_sync(0xFFFFFFFFu, o[0], 1);
    if (lane == 31 || v0 + 4 >= n) nxt = v0 + 4 <= n ? (uint64_t)ld_off(I + v0 + 4) : 0;
    o[4] = nxt;
}

// Exclusive append for a whole warp: EVERY lane of the warp must call it
// (lanes with nothing to add pass 0).  Returns this lane's first slot.
__device__ __forceinline__ uint32_t warp_append_full(uint32_t *counter, uint32_t count) {
    const int lane = threadIdx.x & 31;
    uint32_t incl = count;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total) base = atomicAdd(counter, total);
    base = __shfl_sync(0xFFFFFFFFu, base, 31);
    return base + incl - count;
}

// Append one item from whichever lanes are active here (aggregated atomic).
__device__ __forceinline__ uint32_t append_one(uint32_t *counter) {
    cooperative_groups::coalesced_group g = cooperative_groups::coalesced_threads();
    uint32_t base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(counter, g.size());
    return g.shfl(base, 0) + g.thread_rank();
}

// ---------------------------------------------------------------- dynamic spans
// A streaming pass over items [0, total) in spans: a warp takes the next
// span from ctr[0] when it finishes its last (the next one asked for when a
// span starts), so warps on faster SMs take more spans where a static grid
// stride leaves the slowest SM setting the kernel's time.  A span is the
// grid's share of items over four spans per warp, in multiples of 32, at
// least 32 and at most `max_span` (small inputs keep every warp busy).
// A warp's first span is its own index in the grid; the counter hands out
// the spans after the grid's first (none when the spans do not outnumber
// the warps, so a small input pays no atomic latency).
// f(i, act) is called for item i = span start + 32 t + lane with
// every lane of the warp at each call (act false past the end), so f may
// use warp-collective operations.  The last warp of the grid to finish
// clears ctr[0] and ctr[1] (its done count): every other warp has had its
// last span number by then, and the next launch on the same counters starts
// from zero.  Every warp of the grid must call this exactly once.
template <class F>
__device__ __forceinline__ void warp_spans(uint32_t *ctr, uint64_t total, uint32_t max_span, F &&f) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps_grid = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t span = total / (4 * nwarps_grid) / 32 * 32;
    span = span < 32 ? 32 : (span > max_span ? max_span : span);
    const uint64_t nspan = (total + span - 1) / span;
    const bool dynamic = nspan > nwarps_grid;   // grid-uniform
    uint64_t s = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    while (s < nspan) {
        uint64_t nx = nspan;
        if (dynamic && lane == 0) nx = nwarps_grid + atomicAdd(ctr, 1u);
        const uint64_t b = s * span, e = b + span < total ? b + span : total;
        for (uint64_t i0 = b; i0 < e; i0 += 32) f(i0 + lane, i0 + lane < e);
        s = __shfl_sync(FULL, nx, 0);
    }
    if (dynamic && lane == 0) {
        const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
        if (atomicAdd(ctr + 1, 1u) == nwarps - 1) {
            ctr[0] = 0;
            ctr[1] = 0;
        }
    }
}

// ---------------------------------------------------------------- compaction
// Stream compaction of the index range [0, total) with one atomic per
// block: each block takes a contiguous slice, counts the items it keeps,
// reserves that many output slots with one atomicAdd on *count, then walks
// the slice again in 256-item tiles and writes its items in slice order
// (ballot prefix within a warp, warp totals through shared memory).  An
// append per warp on one counter, the simple form, serialises millions of
// atomics on one address.  Needs blockDim.x == 256.  keep(i) -> bool,
// emit(i, slot).
template <class Keep, class Emit>
__device__ __forceinline__ void block_compact(uint64_t total, uint32_t *count, Keep keep, Emit emit) {
    __shared__ uint32_t warp_sum[8];
    __shared__ uint32_t base_s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t per = (total + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = per * blockIdx.x, hi = lo + per < total ? lo + per : total;
    uint32_t c = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) c += keep(i) ? 1u : 0u;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) warp_sum[wid] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += warp_sum[w];
        base_s = t ? atomicAdd(count, t) : 0u;
    }
    __syncthreads();
    uint32_t run = base_s;
    for (uint64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
        const uint64_t i = t0 + threadIdx.x;
        const bool k = i < hi && keep(i);
        const uint32_t mask = __ballot_sync(0xFFFFFFFFu, k);
        __syncthreads();   // warp_sum free again
        if (lane == 0) warp_sum[wid] = __popc(mask);
        __syncthreads();
        uint32_t before = 0, tile = 0;
        for (int w = 0; w < 8; ++w) {
            before += w < wid ? warp_sum[w] : 0u;
            tile += warp_sum[w];
        }
        if (k) emit(i, run + before + __popc(mask & ((1u << lane) - 1)));
        run += tile;
    }
}

// ---------------------------------------------------------------- edge maps
// Edge functors provide
//   bool begin(u)                 -- false: skip u's edges (unused by callers here)
//   void apply4(u, v[4], ok[4])   -- apply up to four edges (u, v_j) of one vertex
// and are run over a vertex's edges in groups of four for memory-level
// parallelism.  Bad edge ids (>= n) are dropped and flagged here.

// Warp-cooperative light edges.  Every lane of the warp calls this (it is
// warp-synchronous) with its own vertex u and edge range [b, b + deg),
// deg <= LIGHT_MAX, or deg = 0 for none.  The warp walks the concatenation
// of the 32 ranges in steps of 128 positions: lane L takes positions
// step + 32j + L (j < 4), so the 32 lanes of one load instruction read 32
// consecutive positions, which are consecutive words of A inside a vertex's
// range, and no lane idles while another walks a longer list.  The owner of
// position t is the last lane whose exclusive degree prefix is <= t (a
// five-step shuffle search; a lane with deg = 0 is never that last lane for
// t below the total).  f.apply4u takes the four edges with their own sources
// (with POS, f.apply4p also takes their positions in A).
// When the lanes' lists are short and even (a grid, a sparse random graph),
// each lane walking its own list, four edges a step, takes no more steps
// and needs no search: the warp does that when ceil(max deg / 4) steps are
// at most one more than the concatenated walk's ceil(total / 128).
// (Aligned 16-byte group loads in the per-lane walk were tried and lost: a
// group straddles the range ends of low-degree vertices, doubling the
// functor calls on grids and sparse graphs.)
template <class F, bool POS = false>
__device__ __forceinline__ void warp_light_edges(uint32_t u, uint64_t b, uint32_t deg, const uint32_t *A, uint32_t n,
                                                 F &f, const Dev &d) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint32_t mx = __reduce_max_sync(FULL, deg);
    if ((mx + 3) / 4 <= (__reduce_add_sync(FULL, deg) + 127) / 128 + 1) {   // warp-uniform
        for (uint32_t x = 0; x < deg; x += 4) {
            uint32_t uu[4], v[4];
            uint64_t pos[4];
            bool ok[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uu[j] = u;
                pos[j] = b + x + j;
                ok[j] = x + j < deg;
                v[j] = ok[j] ? ld_stream(A + pos[j]) : u;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (ok[j] && v[j] >= n) {
                    atomicOr(d.err, ERR_BAD_EDGE);
                    if (!POS) ok[j] = false;
                }
            if constexpr (POS) f.apply4p(uu, v, ok, pos);
            else f.apply4(u, v, ok);
        }
        return;
    }
    uint32_t incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - deg;
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    // A index of position t within this lane's range: rel + t (mod 2^64)
    const uint64_t rel = b - excl;
    for (uint32_t s = 0; s < total; s += 128) {
        uint32_t uu[4], v[4];
        uint64_t pos[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uu[j] = 0;
            v[j] = 0;
            pos[j] = 0;
            ok[j] = false;
            if (s + 32 * j < total) {   // warp-uniform
                const uint32_t t = s + 32 * j + lane;
                int o = 0;
#pragma unroll
                for (int k = 16; k > 0; k >>= 1)
                    if (__shfl_sync(FULL, excl, o + k) <= t) o += k;
                uu[j] = __shfl_sync(FULL, u, o);
                pos[j] = __shfl_sync(FULL, rel, o) + t;
                ok[j] = t < total;
                v[j] = ok[j] ? ld_stream(A + pos[j]) : uu[j];
            }
        }
        // (with POS a bad edge stays in, flagged: the functor must write
        // something at its position and checks the id itself)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j] && v[j] >= n) {
                atomicOr(d.err, ERR_BAD_EDGE);
                if (!POS) ok[j] = false;
            }
        if constexpr (POS) f.apply4p(uu, v, ok, pos);
        else f.apply4u(uu, v, ok);
    }
}

// One warp applies f to edges [b, e) of vertex u, lane-strided, four loads
// in flight per lane.  (Aligned 16-byte group loads per lane were tried and
// lost: the no-sampling finish's chunk pass went from 4.4 to 17.8 ms at
// RMAT-26, the parent gathers of four neighbouring edges then sitting in one
// lane.)
template <class F>
__device__ __forceinline__ void warp_chunk_edges(uint32_t u, uint64_t b, uint64_t e, const uint32_t *A, uint32_t n,
                                                 F &f, const Dev &d) {
    const int lane = threadIdx.x & 31;
    for (uint64_t x = b + lane; x < e; x += 128) {
        uint32_t v[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ok[j] = x + 32 * j < e;
            v[j] = ok[j] ? ld_stream(A + x + 32 * j) : u;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j] && v[j] >= n) { atomicOr(d.err, ERR_BAD_EDGE); ok[j] = false; }
        f.apply4(u, v, ok);
    }
}

struct ChunkRef {
    uint32_t u;   // vertex
    uint32_t c;   // chunk index: edges [I[u] + c*CHUNK, min(I[u+1], I[u] + (c+1)*CHUNK))
};

// Chunk list capacity for a graph with m directed edges and n vertices:
// each vertex of degree > LIGHT_MAX gives ceil(deg / CHUNK) chunks.
__host__ __device__ inline uint64_t chunk_capacity(uint64_t n, uint64_t m) {
    uint64_t heavy = m / (LIGHT_MAX + 1);
    if (heavy > n) heavy = n;
    return heavy + m / CHUNK + 1;
}

// Record the nc chunks of vertex u at slots [slot, slot + nc).
__device__ __forceinline__ void write_chunks(ChunkRef *chunks, uint64_t cap, uint32_t slot, uint32_t nc,
                                             uint32_t u, const Dev &d) {
    if ((uint64_t)slot + nc > cap) { atomicOr(d.err, ERR_NONCONVERGED); return; }
    for (uint32_t c = 0; c < nc; ++c) chunks[slot + c] = ChunkRef{u, c};
}

// Chunk-list slots reserved by a warp in runs: one global atomic per run
// instead of one per warp step that has a heavy vertex (a single counter
// hit by every warp step serialised at the L2).  A warp's first run is
// exactly what it needs; each later run doubles, up to WARP_RES, so a warp
// that appends once leaves no gap and one that appends often takes few
// atomics.  Slots of a run that stay unused are filled with empty chunks
// (u = NONE) when the warp takes a new run or finishes (close()), and the
// chunk pass skips them.  A grid leaves at most WARP_RES - 1 empty slots
// per warp, which CHUNK_SLACK covers (64 warps per SM, up to 256 SMs).
constexpr uint32_t WARP_RES = 64;
constexpr uint64_t CHUNK_SLACK = 64ull * 256 * WARP_RES;

struct WarpSlots {
    uint64_t cur = 0, end = 0;   // warp-uniform
    uint32_t run = 0;            // size of the last run (warp-uniform)
    // every lane calls with the same total; returns the warp's first slot
    __device__ __forceinline__ uint64_t take(uint32_t *counter, uint32_t total, ChunkRef *chunks, uint64_t cap) {
        if (cur + total > end) {
            close(chunks, cap);
            uint32_t grow = run ? 2 * run : 0;
            grow = grow > WARP_RES ? WARP_RES : grow;
            const uint32_t want = total > grow ? total : grow;
            run = want;
            uint32_t b = 0;
            if ((threadIdx.x & 31) == 0) b = atomicAdd(counter, want);
            b = __shfl_sync(0xFFFFFFFFu, b, 0);
            cur = b;
            end = (uint64_t)b + want;
        }
        const uint64_t r = cur;
        cur += total;
        return r;
    }
    __device__ __forceinline__ void close(ChunkRef *chunks, uint64_t cap) {
        for (uint64_t x = cur + (threadIdx.x & 31); x < end && x < cap; x += 32) chunks[x] = ChunkRef{NONE, 0};
        cur = end;
    }
};

// Binning of one warp step's vertices: each lane's nc chunks go to slots
// from the warp's reservation.
__device__ __forceinline__ void warp_bin_chunks(WarpSlots &ws, uint32_t *counter, ChunkRef *chunks, uint64_t cap,
                                                uint32_t nc, uint32_t u, const Dev &d) {
    const int lane = threadIdx.x & 31;
    uint32_t incl = nc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total == 0) return;   // warp-uniform
    const uint64_t base = ws.take(counter, total, chunks, cap);
    const uint64_t slot = base + incl - nc;
    if (nc) {
        if (slot + nc > cap) { atomicOr(d.err, ERR_NONCONVERGED); return; }
        for (uint32_t c = 0; c < nc; ++c) chunks[slot + c] = ChunkRef{u, c};
    }
}

// Warps of the grid walk the chunk list [0, min(*count, cap)) (the count
// can pass the capacity only on malformed offsets, which is flagged).
// Empty slots (u = NONE, left by warp reservations) are skipped.
template <typename OffT, class F>
__device__ __forceinline__ void run_chunks(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                                           const ChunkRef *chunks, const uint32_t *count, uint64_t cap, F &f,
                                           const Dev &d) {
    const uint32_t total = (uint32_t)((uint64_t)*count < cap ? (uint64_t)*count : cap);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = warp; i < total; i += nwarps) {
        ChunkRef c = chunks[i];
        if (c.u == NONE) continue;
        uint64_t b, e;
        vertex_range(I, c.u, m, b, e, d);
        uint64_t cb = b + (uint64_t)c.c * CHUNK;
        uint64_t ce = cb + CHUNK < e ? cb + CHUNK : e;
        if (cb < ce) warp_chunk_edges(c.u, cb, ce, A, n, f, d);
    }
}

// ---------------------------------------------------------------- functors
// Union-find finish / sampling edge: apply Union(u, v) with the engine E.
// lower_only: apply only edges to smaller neighbours (each undirected edge is
// stored twice; used when no vertex is skipped, so the reverse copy exists).
// Union of NB independent pairs: all first parent reads are issued
// together (memory-level parallelism), then the pairs whose parents differ
// go through the engine.
template <class E, int NB>
__device__ __forceinline__ void unite_pairs(uint32_t *P, const uint32_t (&u)[NB], const uint32_t (&v)[NB],
                                            const bool (&ok)[NB], const Dev &d) {
    uint32_t pu[NB], pv[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        pu[q] = ok[q] ? ld_ca(P + u[q]) : 0;
        pv[q] = ok[q] ? ld_ca(P + v[q]) : 0;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q)
        if (ok[q] && pu[q] != pv[q]) E::unite(P, u[q], v[q], pu[q], pv[q], d);
}

template <class E>
struct UnionEdge {
    uint32_t *P;
    Dev d;
    bool lower_only;
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
        bool act[4];
        uint32_t pv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) act[j] = ok[j] && v[j] != u && (!lower_only || v[j] < u);
        if (!(act[0] | act[1] | act[2] | act[3])) return;
        uint32_t pu = ld_ca(P + u);
#pragma unroll
        for (int j = 0; j < 4; ++j) pv[j] = act[j] ? ld_ca(P + v[j]) : pu;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (act[j] && pv[j] != pu) {
                E::unite(P, u, v[j], pu, pv[j], d);
                pu = ld_rel(P + u);
            }
        }
    }
    // four edges with their own sources (warp_light_edges)
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
        bool act[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) act[j] = ok[j] && v[j] != u[j] && (!lower_only || v[j] < u[j]);
        unite_pairs<E, 4>(P, u, v, act, d);
    }
    __device__ __forceinline__ void flush() {}
};

// Label counting with little atomic contention: a thread keeps a sticky
// "hot" label and a candidate in registers (a two-slot heavy-hitter
// counter); other labels go straight to the count array.  flush() folds
// the warp's hot slots together, one atomic per distinct label.
struct LabelCounter {
    uint32_t hot = NONE, hot_c = 0, cand = NONE, cand_c = 0;
    __device__ __forceinline__ void add(uint32_t *cnt, uint32_t l) {
        if (l == hot) { ++hot_c; return; }
        if (l == cand) {
            if (++cand_c > hot_c) {
                uint32_t t = hot; hot = cand; cand = t;
                t = hot_c; hot_c = cand_c; cand_c = t;
            }
            return;
        }
        if (cand_c) atomicAdd(cnt + cand, cand_c);
        cand = l;
        cand_c = 1;
    }
    // every lane of the warp must call this
    __device__ __forceinline__ void flush(uint32_t *cnt) {
        if (cand_c) atomicAdd(cnt + cand, cand_c);
        const int lane = threadIdx.x & 31;
        unsigned grp = __match_any_sync(0xFFFFFFFFu, hot);
        uint32_t sum = __reduce_add_sync(grp, hot_c);
        if (hot != NONE && sum && lane == __ffs(grp) - 1) atomicAdd(cnt + hot, sum);
    }
};

// LabelCounter that also tracks the arg-max as it counts: every atomicAdd
// returns the count before it, so its issuer sees the count after it, and
// the last increment of each label sees that label's final count.  The
// largest (count << 32 | ~label) seen anywhere is therefore the arg-max with
// ties to the smallest label, with no pass over the count array.
struct LabelCounterArg {
    uint32_t hot = NONE, hot_c = 0, cand = NONE, cand_c = 0;
    unsigned long long best = 0;
    __device__ __forceinline__ void bump(uint32_t *cnt, uint32_t l, uint32_t c) {
        const uint32_t now = atomicAdd(cnt + l, c) + c;
        const unsigned long long k = ((unsigned long long)now << 32) | (uint32_t)~l;
        best = k > best ? k : best;
    }
    __device__ __forceinline__ void add(uint32_t *cnt, uint32_t l) {
        if (l == hot) { ++hot_c; return; }
        if (l == cand) {
            if (++cand_c > hot_c) {
                uint32_t t = hot; hot = cand; cand = t;
                t = hot_c; hot_c = cand_c; cand_c = t;
            }
            return;
        }
        if (cand_c) bump(cnt, cand, cand_c);
        cand = l;
        cand_c = 1;
    }
    // every lane of the warp must call this; then the warp's best goes to
    // *key (one atomicMax per warp; key may be null)
    __device__ __forceinline__ void flush(uint32_t *cnt, unsigned long long *key) {
        if (cand_c) bump(cnt, cand, cand_c);
        const int lane = threadIdx.x & 31;
        unsigned grp = __match_any_sync(0xFFFFFFFFu, hot);
        uint32_t sum = __reduce_add_sync(grp, hot_c);
        if (hot != NONE && sum && lane == __ffs(grp) - 1) bump(cnt, hot, sum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            best = y > best ? y : best;
        }
        if (lane == 0 && best && key) atomicMax(key, best);
    }
};

}  // namespace ccg
