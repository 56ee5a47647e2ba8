// cc_batched.cu -- static connectivity of many independent small graphs in
// one persistent launch (a packed form of Algorithm 1 with no sampling: the
// union-find finish of Algorithm 7 with Rem's CAS rule, Algorithm 14, then
// the final shortcut).  There is no counterpart in the paper, which labels
// one graph per call.
//
// A pre-pass orders the graphs largest first (four size classes per
// octave), so the biggest graphs start at once instead of setting the tail.
// Each CTA then takes whole graphs from a global queue in that order.  A
// graph of at most `smem_max_vertices` (<= 65536) vertices keeps its parent
// array in shared memory as 16-bit local ids (block-local atomics, one
// coalesced global write per vertex at the end); a graph of at most 65536
// vertices keeps ids below the threshold there and the rest in its slice of
// the output; a larger one uses its slice of the output as a 32-bit parent
// array in global memory (L2).
// Vertices are mapped one per thread (mode 0), one per warp (mode 1), or 32
// per warp with the warp walking the concatenation of their edge lists, 128
// consecutive edge words per step (mode 2, the static path's light-vertex
// walk; mode 3 the same at two 1024-thread CTAs per SM).  cc_batched_autotune times the candidate schedules on the caller's
// batch and returns the fastest.
#include <vector>

#include "cc_internal.h"

using namespace ccg;

namespace {

// A graph's parent array (local ids): 16-bit in shared memory (ParS), 32-bit
// in the graph's slice of the output (ParG), or split (ParH): ids below S in
// shared memory, the rest in the output slice, for graphs a little larger
// than the shared-memory threshold.  Reads are volatile (coherent for the
// block in shared memory, L2 in global memory).
struct ParS {
    uint16_t *s;
    __device__ __forceinline__ uint32_t ld(uint32_t i) const { return reinterpret_cast<volatile uint16_t *>(s)[i]; }
    __device__ __forceinline__ uint32_t cas(uint32_t i, uint32_t c, uint32_t v) const {
        return atomicCAS(reinterpret_cast<unsigned short *>(s + i), (unsigned short)c, (unsigned short)v);
    }
    __device__ __forceinline__ void set(uint32_t i, uint32_t v) const {
        reinterpret_cast<volatile uint16_t *>(s)[i] = (uint16_t)v;
    }
};
struct ParG {
    uint32_t *g;
    __device__ __forceinline__ uint32_t ld(uint32_t i) const { return reinterpret_cast<volatile uint32_t *>(g)[i]; }
    __device__ __forceinline__ uint32_t cas(uint32_t i, uint32_t c, uint32_t v) const { return atomicCAS(g + i, c, v); }
    __device__ __forceinline__ void set(uint32_t i, uint32_t v) const { reinterpret_cast<volatile uint32_t *>(g)[i] = v; }
};
struct ParH {
    uint16_t *s;
    uint32_t *g;
    uint32_t S;
    __device__ __forceinline__ uint32_t ld(uint32_t i) const {
        return i < S ? (uint32_t)reinterpret_cast<volatile uint16_t *>(s)[i] : reinterpret_cast<volatile uint32_t *>(g)[i];
    }
    __device__ __forceinline__ uint32_t cas(uint32_t i, uint32_t c, uint32_t v) const {
        return i < S ? (uint32_t)atomicCAS(reinterpret_cast<unsigned short *>(s + i), (unsigned short)c, (unsigned short)v)
                     : atomicCAS(g + i, c, v);
    }
    __device__ __forceinline__ void set(uint32_t i, uint32_t v) const {
        if (i < S) reinterpret_cast<volatile uint16_t *>(s)[i] = (uint16_t)v;
        else reinterpret_cast<volatile uint32_t *>(g)[i] = v;
    }
};

// Rem-CAS union (Algorithm 14) on a parent array, splitting the walked
// path as it goes (SplitOne).  The root link is a CAS; a split is a plain
// store: it writes into a non-root an ancestor of it, and a non-root only
// ever gains ancestors, so any interleaving of such stores leaves a valid
// forest over the same sets (the CAS of SplitAtomicOne is needed only
// where a root may be overwritten).  Plain stores keep the shared-memory
// atomics to the links alone.
template <class Par>
__device__ __forceinline__ void unite_any(const Par &P, uint32_t u, uint32_t v, const Dev &d) {
    uint32_t ru = u, rv = v, pru = P.ld(ru), prv = P.ld(rv);
    Guard g;
    while (pru != prv) {
        if (pru < prv) {
            uint32_t t = ru; ru = rv; rv = t;
            t = pru; pru = prv; prv = t;
        }
        if (ru == pru) {
            uint32_t old = P.cas(ru, ru, prv);
            if (old == ru) return;
            pru = old;
        } else {
            uint32_t w = P.ld(pru);
            if (pru != w) P.set(ru, w);
            ru = pru;
            pru = w;
        }
        if (!g.step(d)) return;
    }
}

template <class Par>
__device__ __forceinline__ uint32_t root_any(const Par &P, uint32_t x, const Dev &d) {
    uint32_t p = P.ld(x);
    Guard g;
    while (p != x) {
        x = p;
        p = P.ld(x);
        if (!g.step(d)) break;
    }
    return x;
}

// Edge functor of the warp walk: each undirected edge once, from its larger
// endpoint.
template <class Par>
struct BatchUnite {
    Par P;
    Dev d;
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j] && v[j] < u) unite_any(P, u, v[j], d);
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j] && v[j] < u[j]) unite_any(P, u[j], v[j], d);
    }
};

// Union-find over graph [vb, vb + ng) with parent array P (local ids).
template <typename OffT, int MODE, class Par>
__device__ __forceinline__ void batch_unions(const OffT *I, const uint32_t *A, uint64_t M, uint64_t vb, uint32_t ng,
                                             const Par &P, const Dev &d) {
    const int lane = threadIdx.x & 31;
    const uint32_t wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (MODE == 0) {
        for (uint32_t i = threadIdx.x; i < ng; i += blockDim.x) {
            uint64_t b, e;
            clamp_range((uint64_t)ld_off(I + vb + i), (uint64_t)ld_off(I + vb + i + 1), M, b, e, d);
            for (uint64_t x = b; x < e; ++x) {
                const uint32_t v = ld_stream(A + x);
                if (v >= ng) { atomicOr(d.err, ERR_BAD_EDGE); continue; }
                if (v < i) unite_any(P, i, v, d);
            }
        }
    } else if (MODE == 1) {
        for (uint32_t i = wid; i < ng; i += nwarp) {
            uint64_t b, e;
            clamp_range((uint64_t)ld_off(I + vb + i), (uint64_t)ld_off(I + vb + i + 1), M, b, e, d);
            for (uint64_t x = b + lane; x < e; x += 32) {
                const uint32_t v = ld_stream(A + x);
                if (v >= ng) { atomicOr(d.err, ERR_BAD_EDGE); continue; }
                if (v < i) unite_any(P, i, v, d);
            }
        }
    } else {
        BatchUnite<Par> f{P, d};
        // every lane of the warp takes part in each step (shuffles); the next
        // tile's offsets are loaded before this tile's edges are walked
        uint32_t base = wid * 32;
        uint64_t o0 = 0, o1 = 0;
        if (base + lane < ng) {
            o0 = (uint64_t)ld_off(I + vb + base + lane);
            o1 = (uint64_t)ld_off(I + vb + base + lane + 1);
        }
        for (; base < ng; base += nwarp * 32) {
            const uint32_t i = base + lane;
            const uint32_t nb = base + nwarp * 32;
            uint64_t n0 = 0, n1 = 0;
            if (nb + lane < ng) {
                n0 = (uint64_t)ld_off(I + vb + nb + lane);
                n1 = (uint64_t)ld_off(I + vb + nb + lane + 1);
            }
            uint64_t b = 0, e = 0;
            if (i < ng) clamp_range(o0, o1, M, b, e, d);
            const uint64_t dg = e - b;
            warp_light_edges(i < ng ? i : 0, b, dg > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)dg, A, ng, f, d);
            o0 = n0;
            o1 = n1;
        }
    }
}

// Graph order for the queue: largest vertex count first, by size class
// (four classes per octave; class 0 holds empty and malformed ranges).
// One block; the order inside a class is arbitrary (results do not depend
// on it).
constexpr int NCLS = 4 * 33 + 1;

__device__ __forceinline__ int size_class(uint64_t vb, uint64_t ve, uint64_t V) {
    if (ve <= vb || ve > V || ve - vb > 0xFFFFFFFEull) return 0;
    const uint32_t n = (uint32_t)(ve - vb);
    const int l = 31 - __clz(n);
    const int frac = l >= 2 ? (int)((n >> (l - 2)) & 3u) : 0;
    return 1 + 4 * l + frac;
}

__global__ void __launch_bounds__(1024) k_batch_order(const uint64_t *gv, uint32_t G, uint64_t V, uint32_t *order) {
    __shared__ uint32_t cnt[NCLS];
    for (int c = threadIdx.x; c < NCLS; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) atomicAdd(&cnt[size_class(gv[g], gv[g + 1], V)], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int c = NCLS - 1; c >= 0; --c) {   // descending classes
            const uint32_t x = cnt[c];
            cnt[c] = run;
            run += x;
        }
    }
    __syncthreads();
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x)
        order[atomicAdd(&cnt[size_class(gv[g], gv[g + 1], V)], 1u)] = g;
}

// MODE 3 is MODE 2 built for two 1024-thread CTAs per SM (64 warps, at most
// 32 registers a thread): more tiles in flight per SM.
template <typename OffT, int MODE>
__global__ void __launch_bounds__(1024, MODE == 3 ? 2 : 1) k_batched(const uint64_t *gv, const uint32_t *order, uint32_t G, uint64_t V,
                                                  const OffT *I, const uint32_t *A, uint64_t M, uint32_t *labels,
                                                  uint32_t *queue, uint32_t smem_max, Dev d) {
    extern __shared__ uint16_t Ps[];
    __shared__ uint32_t g_cur;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t q = atomicAdd(queue, 1u);
            g_cur = q < G ? order[q] : G;
        }
        __syncthreads();
        const uint32_t g = g_cur;
        __syncthreads();
        if (g >= G) break;
        const uint64_t vb = gv[g], ve = gv[g + 1];
        if (ve < vb || ve > V || ve - vb > 0xFFFFFFFEull) {
            if (threadIdx.x == 0) atomicOr(d.err, ERR_BAD_OFFSETS);
            continue;
        }
        const uint32_t ng = (uint32_t)(ve - vb);
        Dev dg = d;
        if (dg.cap == 0) dg.cap = 2ull * ng + 1024;
        constexpr int BM = MODE == 3 ? 2 : MODE;
        if (ng <= smem_max) {
            const ParS P{Ps};
            for (uint32_t i = threadIdx.x; i < ng; i += blockDim.x) P.set(i, i);
            __syncthreads();
            batch_unions<OffT, BM>(I, A, M, vb, ng, P, dg);
            __syncthreads();
            // final shortcut: the root of each tree is its smallest vertex
            for (uint32_t i = threadIdx.x; i < ng; i += blockDim.x) labels[vb + i] = root_any(P, i, dg);
        } else if (ng <= 65536u && smem_max > 0) {
            // ids below smem_max in shared memory, the rest in the output
            // slice; the final write of a vertex's root into its own slot
            // there is a valid compression for concurrent readers
            const ParH P{Ps, labels + vb, smem_max};
            for (uint32_t i = threadIdx.x; i < ng; i += blockDim.x) P.set(i, i);
            __syncthreads();
            batch_unions<OffT, BM>(I, A, M, vb, ng, P, dg);
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < ng; i += blockDim.x) labels[vb + i] = root_any(P, i, dg);
        } else {
            const ParG P{labels + vb};
            for (uint32_t i = threadIdx.x; i < ng; i += blockDim.x) P.set(i, i);
            __syncthreads();
            batch_unions<OffT, BM>(I, A, M, vb, ng, P, dg);
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < ng; i += blockDim.x) labels[vb + i] = root_any(P, i, dg);
        }
        __syncthreads();
    }
}

cc_status check_batch_opt(const cc_batch_opt &o) {
    if (o.threads != 128 && o.threads != 256 && o.threads != 512 && o.threads != 1024) return CC_ERR_INVALID;
    if (o.smem_max_vertices > 65536u) return CC_ERR_INVALID;
    if (o.vertex_mode > 3 || o.reserved != 0) return CC_ERR_INVALID;
    if (o.vertex_mode == 3 && o.threads != 1024) return CC_ERR_INVALID;
    return CC_OK;
}

template <typename OffT>
const void *batched_fn(uint32_t mode) {
    return mode == 3   ? (const void *)k_batched<OffT, 3>
           : mode == 2 ? (const void *)k_batched<OffT, 2>
           : mode == 1 ? (const void *)k_batched<OffT, 1>
                       : (const void *)k_batched<OffT, 0>;
}

template <typename OffT>
cc_status launch_batched(const uint64_t *gv, uint32_t G, uint64_t V, const void *offsets, const uint32_t *edges,
                         uint64_t M, const cc_batch_opt &o, uint32_t *labels, uint32_t *queue, uint32_t *order,
                         cudaStream_t s) {
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    const size_t smem = (size_t)o.smem_max_vertices * sizeof(uint16_t);
    const void *fn = batched_fn<OffT>(o.vertex_mode);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return from_cuda(e);
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, (int)o.threads, smem);
    if (e != cudaSuccess) return from_cuda(e);
    if (per_sm < 1) return CC_ERR_INVALID;
    uint64_t grid = (uint64_t)per_sm * di->sms;
    if (grid > G) grid = G;
    if (grid == 0) grid = 1;
    // cap 0: each graph gets 2 n_g + 1024 steps per loop (a test override wins)
    const uint64_t lc = loop_cap(0);
    const Dev d = Dev{di->err, lc == 1024 ? 0 : lc};
    e = cudaMemsetAsync(queue, 0, 4, s);
    if (e != cudaSuccess) return from_cuda(e);
    {
        CC_PROF("k_batch_order", s);
        k_batch_order<<<1, 1024, 0, s>>>(gv, G, V, order);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return from_cuda(e);
    const OffT *I = static_cast<const OffT *>(offsets);
    CC_PROF("k_batched", s);
    if (o.vertex_mode == 3)
        k_batched<OffT, 3><<<(unsigned)grid, o.threads, smem, s>>>(gv, order, G, V, I, edges, M, labels, queue,
                                                                    o.smem_max_vertices, d);
    else if (o.vertex_mode == 2)
        k_batched<OffT, 2><<<(unsigned)grid, o.threads, smem, s>>>(gv, order, G, V, I, edges, M, labels, queue,
                                                                    o.smem_max_vertices, d);
    else if (o.vertex_mode == 1)
        k_batched<OffT, 1><<<(unsigned)grid, o.threads, smem, s>>>(gv, order, G, V, I, edges, M, labels, queue,
                                                                    o.smem_max_vertices, d);
    else
        k_batched<OffT, 0><<<(unsigned)grid, o.threads, smem, s>>>(gv, order, G, V, I, edges, M, labels, queue,
                                                                    o.smem_max_vertices, d);
    return from_cuda(cudaGetLastError());
}

cc_status batched_args(const uint64_t *gv, uint32_t G, const void *offsets, int offsets_u64, const uint32_t *edges,
                       uint64_t V, uint64_t M, uint32_t *labels_out) {
    if (G == 0 || V == 0) return CC_OK;
    if (!gv || !offsets || !labels_out || (M > 0 && !edges)) return CC_ERR_INVALID;
    if (!aligned(gv, 8) || !aligned(offsets, offsets_u64 ? 8 : 4) || !aligned(labels_out, 4) ||
        (edges && !aligned(edges, 4)))
        return CC_ERR_INVALID;
    if (!offsets_u64 && M > 0xFFFFFFFFull) return CC_ERR_INVALID;
    return CC_OK;
}

}  // namespace

extern "C" {

void cc_batch_default_opt(cc_batch_opt *o) {
    if (!o) return;
    o->threads = 1024;
    o->smem_max_vertices = 65536;
    o->vertex_mode = 2;
    o->reserved = 0;
}

cc_status cc_batched(const uint64_t *gv, uint32_t G, const void *offsets, int offsets_u64, const uint32_t *edges,
                     uint64_t V, uint64_t M, const cc_batch_opt *opt, uint32_t *labels_out, void *stream) {
    cc_status st = batched_args(gv, G, offsets, offsets_u64, edges, V, M, labels_out);
    if (st != CC_OK || G == 0 || V == 0) return st;
    cc_batch_opt o;
    cc_batch_default_opt(&o);
    if (opt) o = *opt;
    if ((st = check_batch_opt(o)) != CC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    const size_t oq = sc.reserve(4), oo = sc.reserve((size_t)G * 4);
    if ((st = sc.alloc(s)) != CC_OK) return st;
    return offsets_u64 ? launch_batched<uint64_t>(gv, G, V, offsets, edges, M, o, labels_out, sc.at<uint32_t>(oq),
                                                  sc.at<uint32_t>(oo), s)
                       : launch_batched<uint32_t>(gv, G, V, offsets, edges, M, o, labels_out, sc.at<uint32_t>(oq),
                                                  sc.at<uint32_t>(oo), s);
}

cc_status cc_batched_autotune(const uint64_t *gv, uint32_t G, const void *offsets, int offsets_u64,
                              const uint32_t *edges, uint64_t V, uint64_t M, uint32_t *labels_out,
                              cc_batch_opt *best_out, float *best_ms_out, void *stream) {
    cc_status st = batched_args(gv, G, offsets, offsets_u64, edges, V, M, labels_out);
    if (st != CC_OK) return st;
    if (!best_out) return CC_ERR_INVALID;
    cc_batch_default_opt(best_out);
    if (best_ms_out) *best_ms_out = 0.f;
    if (G == 0 || V == 0) return CC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<cc_batch_opt> cands;
    // shared-memory thresholds 16384 / 28672 / 57344 / 65536 vertices take
    // 32 / 56 / 112 / 128 KB per CTA: 7, 4, 2 and 1 CTAs per SM
    for (uint32_t mode : {0u, 1u, 2u, 3u})
        for (uint32_t threads : {256u, 512u, 1024u})
            for (uint32_t smem : {0u, 16384u, 28672u, 57344u, 65536u})
                if (mode != 3 || threads == 1024) cands.push_back(cc_batch_opt{threads, smem, mode, 0});
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CC_ERR_CUDA;
    float best = -1.f;
    for (const cc_batch_opt &c : cands) {
        // one untimed run, then the better of two timed runs
        st = cc_batched(gv, G, offsets, offsets_u64, edges, V, M, &c, labels_out, stream);
        if (st == CC_ERR_INVALID) continue;
        if (st != CC_OK) break;
        float ms = 1e30f;
        for (int r = 0; r < 2; ++r) {
            cudaEventRecord(e0, s);
            st = cc_batched(gv, G, offsets, offsets_u64, edges, V, M, &c, labels_out, stream);
            cudaEventRecord(e1, s);
            if (st != CC_OK) break;
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = t < ms ? t : ms;
        }
        if (st != CC_OK) break;
        if (best < 0.f || ms < best) {
            best = ms;
            *best_out = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CC_OK && st != CC_ERR_INVALID) return st;
    if (best_ms_out) *best_ms_out = best;
    // leave labels_out computed with the winning schedule
    return cc_batched(gv, G, offsets, offsets_u64, edges, V, M, best_out, labels_out, stream);
}

}  // extern "C"
