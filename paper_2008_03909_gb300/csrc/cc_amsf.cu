// cc_amsf.cu -- approximate minimum spanning forest (Section 5.1).  The
// folklore algorithm: with Wmin the smallest weight, bucket i holds the
// edges of weight in [Wmin(1+eps)^i, Wmin(1+eps)^(i+1)); buckets are taken
// smallest first, and each adds a spanning forest of its edges over the
// connectivity of the buckets before it.  The union of those forests
// weighs at most (1 + eps) times a minimum spanning forest.
//
// Three forms, as the section names them:
//   AMSF-NF   every bucket reads the whole CSR and keeps its own edges;
//   AMSF-NF-S the same, skipping the vertices of the largest component of
//             the connectivity so far (their edges are applied from the
//             other endpoint);
//   AMSF-COO  the edges are first grouped by bucket (a counting sort into
//             an edge list), so every edge is read once.
// The unions are UF-Rem-CAS with SplitAtomicOne and FindNaive, as in the
// paper's evaluation; each link records its edge and weight at the hooked
// root, so the forest is the set of hooking edges (root-based, as in the
// spanning-forest appendix).
#include <cmath>
#include <vector>

#include "cc_internal.h"

using namespace ccg;

namespace {

constexpr unsigned TPB = 256;
using Engine = UnionRem<SPLICE_SPLIT_ONE, FIND_NAIVE>;

// Bit patterns of positive finite floats order like the floats.
__global__ void __launch_bounds__(256, 8) k_weight_range(const float *W, uint64_t m, uint32_t *lohi, Dev d) {
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    bool bad = false;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const float w = __ldcs(W + i);
        if (!(w > 0.0f) || !(w < INFINITY)) { bad = true; continue; }
        const uint32_t b = __float_as_uint(w);
        lo = b < lo ? b : lo;
        hi = b > hi ? b : hi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (lo != 0xFFFFFFFFu) atomicMin(lohi, lo);
        if (hi) atomicMax(lohi + 1, hi);
    }
    if (bad) atomicOr(d.err, ERR_BAD_EDGE);
}

// Bucket of w under the thresholds T[0..nb] (T[0] = Wmin, T[i] =
// Wmin(1+eps)^i rounded to float, T[nb] above every weight): a log2 guess,
// then corrected against T, so that every edge lands in exactly the bucket
// whose [T[i], T[i+1]) holds it.
__device__ __forceinline__ uint32_t bucket_of(float w, const float *T, uint32_t nb, float inv_log2_ratio, float wmin) {
    int b = (int)floorf(log2f(w / wmin) * inv_log2_ratio);
    b = b < 0 ? 0 : (b >= (int)nb ? (int)nb - 1 : b);
    while (b + 1 < (int)nb && w >= __ldg(T + b + 1)) ++b;
    while (b > 0 && w < __ldg(T + b)) --b;
    return (uint32_t)b;
}

struct BucketSpec {
    const float *T;
    uint32_t nb;
    float inv_log2_ratio;
    float wmin;
};

// Hook root r records the weight of the edge that hooked it.
__device__ __forceinline__ void unite_weighted(uint32_t *P, uint32_t u, uint32_t v, float w, float *fw,
                                               const Dev &d) {
    const uint32_t pu = ld_ca(P + u), pv = ld_ca(P + v);
    if (pu == pv) return;
    const uint32_t r = Engine::unite(P, u, v, pu, pv, d);
    if (r != NONE) fw[r] = w;
}

__global__ void __launch_bounds__(256, 8) k_amsf_coo(const uint32_t *cu, const uint32_t *cv, const float *cw,
                                                     uint64_t begin, uint64_t end, uint32_t *P, float *fw, Dev d) {
    for (uint64_t i = begin + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < end;
         i += (uint64_t)gridDim.x * blockDim.x)
        unite_weighted(P, __ldcs(cu + i), __ldcs(cv + i), __ldcs(cw + i), fw, d);
}

// Membership of the largest component at the start of a bucket, as a
// bitmap: the bucket's unions change P while it runs, and an edge must be
// skipped or applied by a rule that both endpoints see alike.
__global__ void __launch_bounds__(256, 8) k_mark_frequent(const uint32_t *P, uint32_t n, const uint32_t *lmax_p,
                                                          uint32_t *bm) {
    const uint32_t lmax = *lmax_p;
    const uint64_t words = (n + 31) / 32;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words;
         w += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t bits = 0;
        for (int j = 0; j < 32; ++j) {
            const uint64_t v = w * 32 + j;
            if (v < n && P[v] == lmax) bits |= 1u << j;
        }
        bm[w] = bits;
    }
}

__device__ __forceinline__ bool in_bm(const uint32_t *bm, uint32_t v) { return (bm[v >> 5] >> (v & 31)) & 1u; }

// ---------------------------------------------------------------- weighted edge walk
// Light vertices (degree <= LIGHT_MAX) are walked by their warp together,
// the 32 lanes' edge lists concatenated (the same walk as
// warp_light_edges), so one load instruction reads 32 consecutive weights;
// the heavier ones as CHUNK-edge pieces, one warp each, so a hub's edges
// spread over the whole grid.  Vertices whose bit is set in skip are not
// read.  F provides begin() / end() (per block), want(w) (is the edge read
// at all) and (u, v, w).  Weights are read first: an edge whose weight the
// pass does not want costs no edge read.
template <class F>
__device__ __forceinline__ void warp_light_wedges(uint32_t u, uint64_t b, uint32_t deg, const uint32_t *A,
                                                  const float *W, uint32_t n, F &f, const Dev &d) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    uint32_t incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    const uint32_t excl = incl - deg;
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    const uint64_t rel = b - excl;   // position t of this lane's list is edge rel + t (mod 2^64)
    for (uint32_t s = 0; s < total; s += 128) {
        uint32_t uu[4], v[4];
        uint64_t pos[4];
        float w[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uu[j] = 0;
            pos[j] = 0;
            w[j] = 0.0f;
            ok[j] = false;
            if (s + 32 * j < total) {   // warp-uniform
                const uint32_t t = s + 32 * j + lane;
                int o = 0;
#pragma unroll
                for (int k = 16; k > 0; k >>= 1)
                    if (__shfl_sync(FULL, excl, o + k) <= t) o += k;
                uu[j] = __shfl_sync(FULL, u, o);
                pos[j] = __shfl_sync(FULL, rel, o) + t;
                if (t < total) {
                    w[j] = __ldcs(W + pos[j]);
                    ok[j] = true;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) ok[j] = ok[j] && f.want(w[j]);
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = ok[j] ? ld_stream(A + pos[j]) : 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (ok[j] && v[j] >= n) { atomicOr(d.err, ERR_BAD_EDGE); ok[j] = false; }
            if (ok[j]) f(uu[j], v[j], w[j]);
        }
    }
}

template <typename OffT, class F>
__global__ void __launch_bounds__(256, 8) k_wedges(const OffT *I, const uint32_t *A, const float *W, uint32_t n,
                                                   uint64_t m, const ChunkRef *chunks, const uint32_t *nchunks,
                                                   uint64_t cap, const uint32_t *skip, F f, Dev d) {
    f.begin();
    const int lane = threadIdx.x & 31;
    {
        const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
        const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
        for (uint64_t base = warp * 32; base < n; base += nw * 32) {
            const uint64_t i = base + lane;
            uint64_t b = 0, e = 0;
            if (i < n && !(skip && in_bm(skip, (uint32_t)i))) vertex_range(I, (uint32_t)i, m, b, e, d);
            const uint64_t deg = e - b;
            warp_light_wedges((uint32_t)i, b, deg <= LIGHT_MAX ? (uint32_t)deg : 0u, A, W, n, f, d);
        }
    }
    const uint32_t total = (uint32_t)((uint64_t)*nchunks < cap ? (uint64_t)*nchunks : cap);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = warp; c < total; c += nwarps) {
        const ChunkRef cr = chunks[c];
        if (skip && in_bm(skip, cr.u)) continue;
        uint64_t b, e;
        vertex_range(I, cr.u, m, b, e, d);
        const uint64_t cb = b + (uint64_t)cr.c * CHUNK, ce = cb + CHUNK < e ? cb + CHUNK : e;
        for (uint64_t x0 = cb; x0 < ce; x0 += 128) {
            uint32_t v[4];
            float w[4];
            bool ok[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t x = x0 + 32 * j + lane;
                w[j] = x < ce ? __ldcs(W + x) : 0.0f;
                ok[j] = x < ce && f.want(w[j]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] = ok[j] ? ld_stream(A + x0 + 32 * j + lane) : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (ok[j] && v[j] >= n) { atomicOr(d.err, ERR_BAD_EDGE); ok[j] = false; }
                if (ok[j]) f(cr.u, v[j], w[j]);
            }
        }
    }
    f.end();
}

// Chunk list of the vertices of degree > LIGHT_MAX (built once).
template <typename OffT>
__global__ void __launch_bounds__(256, 8) k_heavy_chunks(const OffT *I, uint32_t n, uint64_t m, ChunkRef *chunks,
                                                         uint32_t *nchunks, uint64_t cap, Dev d) {
    for (uint64_t base = ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += (((uint64_t)gridDim.x * blockDim.x) >> 5) * 32) {
        const uint64_t v = base + (threadIdx.x & 31);
        uint64_t b = 0, e = 0;
        if (v < n) vertex_range(I, (uint32_t)v, m, b, e, d);
        const uint64_t deg = e - b;
        const uint32_t nc = deg > LIGHT_MAX ? (uint32_t)((deg + CHUNK - 1) / CHUNK) : 0;
        const uint32_t slot = warp_append_full(nchunks, nc);
        if (nc) write_chunks(chunks, cap, slot, nc, (uint32_t)v, d);
    }
}

// One bucket of AMSF-NF / NF-S: the edges with weight in [lo, hi), each
// applied once: from its larger endpoint, or (SKIP) from the endpoint
// outside the largest component.
template <bool SKIP>
struct BucketUnion {
    float lo, hi;
    uint32_t *P;
    const uint32_t *bm;
    float *fw;
    Dev d;
    __device__ __forceinline__ void begin() {}
    __device__ __forceinline__ void end() {}
    __device__ __forceinline__ bool want(float w) const { return w >= lo && w < hi; }
    __device__ __forceinline__ void operator()(uint32_t u, uint32_t v, float w) {
        if (v < u || (SKIP && in_bm(bm, v))) unite_weighted(P, u, v, w, fw, d);
    }
};

// AMSF-COO's counting sort of the edges (u, v), v < u, by bucket.  Pass 1
// counts per block in shared memory; the per-block counts give each block
// its own range in every bucket; pass 2 repeats the same walk and scatters
// (u, v, w) through shared-memory cursors.  Both passes launch the same
// grid, so each block sees the same edges.  With more buckets than fit in
// shared memory the counters are global instead (one row).
constexpr uint32_t SMEM_BUCKETS = 4096;

struct BucketCount {
    BucketSpec bs;
    uint32_t *rows;      // [blocks][nb] (or one global row)
    bool global;
    uint32_t *sh;
    __device__ __forceinline__ void begin() {
        extern __shared__ unsigned long long dyn_smem[];
        sh = global ? rows : reinterpret_cast<uint32_t *>(dyn_smem);
        if (!global) {
            for (uint32_t i = threadIdx.x; i < bs.nb; i += blockDim.x) sh[i] = 0;
            __syncthreads();
        }
    }
    __device__ __forceinline__ bool want(float w) const { return w > 0.0f && w < INFINITY; }
    __device__ __forceinline__ void operator()(uint32_t u, uint32_t v, float w) {
        if (v < u) atomicAdd(sh + bucket_of(w, bs.T, bs.nb, bs.inv_log2_ratio, bs.wmin), 1u);
    }
    __device__ __forceinline__ void end() {
        if (global) return;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < bs.nb; i += blockDim.x) rows[(uint64_t)blockIdx.x * bs.nb + i] = sh[i];
    }
};

struct BucketScatter {
    BucketSpec bs;
    unsigned long long *base;   // [blocks][nb] first slot of each block's range (or one global cursor row)
    bool global;
    uint32_t *cu, *cv;
    float *cw;
    unsigned long long *sh;
    __device__ __forceinline__ void begin() {
        extern __shared__ unsigned long long dyn_smem[];
        sh = global ? base : dyn_smem;
        if (!global) {
            for (uint32_t i = threadIdx.x; i < bs.nb; i += blockDim.x) sh[i] = base[(uint64_t)blockIdx.x * bs.nb + i];
            __syncthreads();
        }
    }
    __device__ __forceinline__ bool want(float w) const { return w > 0.0f && w < INFINITY; }
    __device__ __forceinline__ void operator()(uint32_t u, uint32_t v, float w) {
        if (!(v < u)) return;
        const unsigned long long pos = atomicAdd(sh + bucket_of(w, bs.T, bs.nb, bs.inv_log2_ratio, bs.wmin), 1ull);
        cu[pos] = u;
        cv[pos] = v;
        cw[pos] = w;
    }
    __device__ __forceinline__ void end() {}
};

// Per bucket: the blocks' ranges inside the bucket (an exclusive scan over
// blocks) and the bucket's total.
__global__ void k_bucket_scan(const uint32_t *rows, uint32_t blocks, uint32_t nb, unsigned long long *base,
                              unsigned long long *total) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        unsigned long long acc = 0;
        for (uint32_t k = 0; k < blocks; ++k) {
            base[(uint64_t)k * nb + b] = acc;
            acc += rows[(uint64_t)k * nb + b];
        }
        total[b] = acc;
    }
}

__global__ void k_bucket_offset(unsigned long long *base, uint32_t blocks, uint32_t nb,
                                const unsigned long long *start) {
    const uint64_t cnt = (uint64_t)blocks * nb;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cnt; i += (uint64_t)gridDim.x * blockDim.x)
        base[i] += start[i % nb];
}

__global__ void __launch_bounds__(256, 8) k_iota32(uint32_t *P, uint32_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        P[i] = (uint32_t)i;
}

// Every vertex points at its root (roots are component minima).
__global__ void __launch_bounds__(256, 8) k_compress(uint32_t *P, uint32_t n, Dev d) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)i, p = ld_rel(P + v);
        const uint32_t r = find_from<FIND_NAIVE>(P, v, p, d);
        if (r != p) P[v] = r;
    }
}

// IdentifyFrequent on a flat forest: count the non-roots under their root
// (a root's count is then its component size minus one, so the arg-max
// with ties to the smallest label is unchanged), then the arg-max as a
// packed (count << 32 | ~label) maximum.  Counts go through LabelCounter's
// register slots: once one component holds most vertices, one atomic per
// vertex on its root's counter would serialise on one address.
__global__ void __launch_bounds__(256, 8) k_count_flat(const uint32_t *P, uint32_t n, uint32_t *cnt) {
    LabelCounter lc;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = P[i];
        if (l != (uint32_t)i && l < n) lc.add(cnt, l);
    }
    lc.flush(cnt);
}

__global__ void __launch_bounds__(256, 8) k_argmax(const uint32_t *cnt, uint32_t n, unsigned long long *key) {
    unsigned long long best = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = ((unsigned long long)cnt[i] << 32) | (uint32_t)~(uint32_t)i;
        best = k > best ? k : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        best = t > best ? t : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(key, best);
}

__global__ void k_key_label(const unsigned long long *key, uint32_t *lmax) {
    *lmax = *key ? ~(uint32_t)(*key & 0xFFFFFFFFull) : 0u;
}

// Filter step: hooking edges and their weights into the output.
__global__ void __launch_bounds__(256, 8) k_amsf_compact(const uint2 *ff, const float *fw, uint32_t n, uint32_t *out,
                                                         uint32_t *count, double *wsum, Dev d) {
    double acc = 0.0;
    block_compact(
        n, count, [&](uint64_t i) { return ff[i].x != NONE; },
        [&](uint64_t i, uint32_t k) {
            acc += (double)fw[i];
            if (k >= n) { atomicOr(d.err, ERR_NONCONVERGED); return; }
            const uint2 e = ff[i];
            out[2 * (uint64_t)k] = e.x;
            out[2 * (uint64_t)k + 1] = e.y;
        });
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(wsum, acc);
}

struct AmsfCtl {
    uint32_t lohi[2];
    uint32_t count;
    uint32_t lmax;
    unsigned long long key;
    double wsum;
};

#define AM_TRY(x)                                     \
    do {                                              \
        cudaError_t e__ = (x);                        \
        if (e__ != cudaSuccess) return from_cuda(e__); \
    } while (0)

template <typename OffT>
cc_status run_amsf(const void *offsets, const uint32_t *A, const float *W, uint32_t n, uint64_t m, float eps,
                   int mode, uint32_t *forest_out, uint64_t *count_out, double *weight_out, uint32_t *labels,
                   cudaStream_t s) {
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    const Dev d0 = make_dev(di, n);
    const OffT *I = static_cast<const OffT *>(offsets);
    const unsigned gv = grid_for(di, n, TPB), ge = grid_for(di, m, TPB);
    // scratch part 1: control, forest arrays, labels if not the caller's
    Scratch sc;
    const size_t o_ctl = sc.reserve(sizeof(AmsfCtl)), o_ff = sc.reserve((size_t)n * 8), o_fw = sc.reserve((size_t)n * 4),
                 o_cnt = sc.reserve((size_t)n * 4), o_bm = sc.reserve(((size_t)n + 31) / 32 * 4),
                 o_lab = labels ? 0 : sc.reserve((size_t)n * 4);
    cc_status st = sc.alloc(s);
    if (st != CC_OK) return st;
    AmsfCtl *ctl = sc.at<AmsfCtl>(o_ctl);
    uint2 *ff = sc.at<uint2>(o_ff);
    float *fw = sc.at<float>(o_fw);
    uint32_t *cnt = sc.at<uint32_t>(o_cnt), *bm = sc.at<uint32_t>(o_bm);
    uint32_t *P = labels ? labels : sc.at<uint32_t>(o_lab);
    Dev d = d0;
    d.forest = ff;
    AmsfCtl h{};
    h.lohi[0] = 0xFFFFFFFFu;
    AM_TRY(cudaMemcpyAsync(ctl, &h, sizeof(AmsfCtl), cudaMemcpyHostToDevice, s));
    AM_TRY(cudaMemsetAsync(ff, 0xFF, (size_t)n * 8, s));
    {
        CC_PROF("k_iota", s);
        k_iota32<<<gv, TPB, 0, s>>>(P, n);
    }
    if (m) {
        CC_PROF("k_weight_range", s);
        k_weight_range<<<ge, TPB, 0, s>>>(W, m, ctl->lohi, d);
    }
    AM_TRY(cudaGetLastError());
    AM_TRY(cudaMemcpyAsync(&h, ctl, sizeof(AmsfCtl), cudaMemcpyDeviceToHost, s));
    AM_TRY(cudaStreamSynchronize(s));
    // thresholds T[i] = Wmin (1+eps)^i in double, rounded to float, until
    // one passes Wmax; T[nb] is above every weight
    std::vector<float> T;
    if (m && h.lohi[0] != 0xFFFFFFFFu) {
        float wmin, wmax;
        memcpy(&wmin, &h.lohi[0], 4);
        memcpy(&wmax, &h.lohi[1], 4);
        for (uint32_t i = 0;; ++i) {
            const double t = (double)wmin * std::pow(1.0 + (double)eps, (double)i);
            if (i > 0 && (float)t <= T.back()) return CC_ERR_INVALID;   // eps below float resolution here
            T.push_back((float)t);
            if ((float)t > wmax) break;
            if (T.size() > CC_AMSF_MAX_BUCKETS) return CC_ERR_INVALID;
        }
    }
    const uint32_t nb = T.empty() ? 0 : (uint32_t)T.size() - 1;
    // heavy vertices as CHUNK-edge pieces (one list for every pass)
    const uint64_t ccap = chunk_capacity(n, m);
    Scratch sc2;
    const size_t o_T = sc2.reserve((nb + 1) * 4), o_ch = sc2.reserve(ccap * sizeof(ChunkRef)), o_nch = sc2.reserve(4);
    if ((st = sc2.alloc(s)) != CC_OK) return st;
    float *dT = sc2.at<float>(o_T);
    ChunkRef *chunks = sc2.at<ChunkRef>(o_ch);
    uint32_t *nch = sc2.at<uint32_t>(o_nch);
    if (nb) AM_TRY(cudaMemcpyAsync(dT, T.data(), (nb + 1) * 4, cudaMemcpyHostToDevice, s));
    AM_TRY(cudaMemsetAsync(nch, 0, 4, s));
    {
        CC_PROF("k_heavy_chunks", s);
        k_heavy_chunks<OffT><<<gv, TPB, 0, s>>>(I, n, m, chunks, nch, ccap, d);
    }
    const BucketSpec bs{dT, nb, nb ? (float)(1.0 / std::log2(1.0 + (double)eps)) : 0.0f, nb ? T[0] : 1.0f};
    if (mode == CC_AMSF_COO && nb) {
        const bool global = nb > SMEM_BUCKETS;
        const uint64_t rows_n = global ? nb : (uint64_t)gv * nb;
        Scratch sc3;
        const size_t o_rows = sc3.reserve(rows_n * 4), o_base = sc3.reserve(rows_n * 8), o_tot = sc3.reserve(nb * 8ull),
                     o_start = sc3.reserve(nb * 8ull);
        if ((st = sc3.alloc(s)) != CC_OK) return st;
        uint32_t *rows = sc3.at<uint32_t>(o_rows);
        unsigned long long *base = sc3.at<unsigned long long>(o_base), *tot = sc3.at<unsigned long long>(o_tot),
                           *dstart = sc3.at<unsigned long long>(o_start);
        if (global) AM_TRY(cudaMemsetAsync(rows, 0, rows_n * 4, s));
        {
            CC_PROF("k_bucket_count", s);
            k_wedges<OffT, BucketCount><<<gv, TPB, global ? 0 : nb * 4, s>>>(
                I, A, W, n, m, chunks, nch, ccap, nullptr, BucketCount{bs, rows, global, nullptr}, d);
        }
        {
            CC_PROF("k_bucket_scan", s);
            k_bucket_scan<<<grid_for(di, nb, TPB), TPB, 0, s>>>(rows, global ? 1 : gv, nb, base, tot);
        }
        std::vector<unsigned long long> hh(nb), start(nb + 1, 0);
        AM_TRY(cudaMemcpyAsync(hh.data(), tot, (size_t)nb * 8, cudaMemcpyDeviceToHost, s));
        AM_TRY(cudaStreamSynchronize(s));
        for (uint32_t b = 0; b < nb; ++b) start[b + 1] = start[b] + hh[b];
        const uint64_t total = start[nb];
        AM_TRY(cudaMemcpyAsync(dstart, start.data(), (size_t)nb * 8, cudaMemcpyHostToDevice, s));
        {
            CC_PROF("k_bucket_offset", s);
            k_bucket_offset<<<grid_for(di, rows_n, TPB), TPB, 0, s>>>(base, global ? 1 : gv, nb, dstart);
        }
        Scratch sc4;
        const size_t o_u = sc4.reserve(total * 4), o_v = sc4.reserve(total * 4), o_w = sc4.reserve(total * 4);
        if ((st = sc4.alloc(s)) != CC_OK) return st;
        uint32_t *cu = sc4.at<uint32_t>(o_u), *cv = sc4.at<uint32_t>(o_v);
        float *cw = sc4.at<float>(o_w);
        {
            CC_PROF("k_bucket_scatter", s);
            k_wedges<OffT, BucketScatter><<<gv, TPB, global ? 0 : nb * 8, s>>>(
                I, A, W, n, m, chunks, nch, ccap, nullptr, BucketScatter{bs, base, global, cu, cv, cw, nullptr}, d);
        }
        for (uint32_t b = 0; b < nb; ++b) {
            if (!hh[b]) continue;
            CC_PROF("k_amsf_coo", s);
            k_amsf_coo<<<grid_for(di, hh[b], TPB), TPB, 0, s>>>(cu, cv, cw, start[b], start[b + 1], P, fw, d);
        }
        AM_TRY(cudaGetLastError());
        AM_TRY(cudaStreamSynchronize(s));   // the edge list is freed on return
    } else if (nb) {
        for (uint32_t b = 0; b < nb; ++b) {
            if (mode == CC_AMSF_NF_S) {
                {
                    CC_PROF("k_compress", s);
                    k_compress<<<gv, TPB, 0, s>>>(P, n, d);
                }
                AM_TRY(cudaMemsetAsync(cnt, 0, (size_t)n * 4, s));
                AM_TRY(cudaMemsetAsync(&ctl->key, 0, 8, s));
                {
                    CC_PROF("k_count_flat", s);
                    k_count_flat<<<gv, TPB, 0, s>>>(P, n, cnt);
                }
                {
                    CC_PROF("k_argmax", s);
                    k_argmax<<<gv, TPB, 0, s>>>(cnt, n, &ctl->key);
                }
                {
                    CC_PROF("k_key_label", s);
                    k_key_label<<<1, 1, 0, s>>>(&ctl->key, &ctl->lmax);
                }
                {
                    CC_PROF("k_mark_frequent", s);
                    k_mark_frequent<<<grid_for(di, ((uint64_t)n + 31) / 32, TPB), TPB, 0, s>>>(P, n, &ctl->lmax, bm);
                }
                CC_PROF("k_amsf_bucket", s);
                k_wedges<OffT, BucketUnion<true>><<<gv, TPB, 0, s>>>(
                    I, A, W, n, m, chunks, nch, ccap, bm, BucketUnion<true>{T[b], T[b + 1], P, bm, fw, d}, d);
            } else {
                CC_PROF("k_amsf_bucket", s);
                k_wedges<OffT, BucketUnion<false>><<<gv, TPB, 0, s>>>(
                    I, A, W, n, m, chunks, nch, ccap, nullptr, BucketUnion<false>{T[b], T[b + 1], P, nullptr, fw, d},
                    d);
            }
            AM_TRY(cudaGetLastError());
        }
    }
    {
        CC_PROF("k_final_shortcut", s);
        k_compress<<<gv, TPB, 0, s>>>(P, n, d);
    }
    {
        CC_PROF("k_amsf_compact", s);
        k_amsf_compact<<<gv, TPB, 0, s>>>(ff, fw, n, forest_out, &ctl->count, &ctl->wsum, d);
    }
    AM_TRY(cudaGetLastError());
    AM_TRY(cudaMemcpyAsync(&h, ctl, sizeof(AmsfCtl), cudaMemcpyDeviceToHost, s));
    AM_TRY(cudaStreamSynchronize(s));
    *count_out = h.count < n ? h.count : n;
    *weight_out = h.wsum;
    return CC_OK;
}

}  // namespace

extern "C" cc_status cc_amsf(const void *offsets, int offsets_u64, const uint32_t *edges, const float *weights,
                             uint32_t n, uint64_t m, float epsilon, int mode, uint32_t *forest_out,
                             uint64_t *count_out, double *weight_out, uint32_t *labels_out, void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK) return st;
    if (!count_out || !weight_out) return CC_ERR_INVALID;
    if (!(epsilon >= 1e-3f && epsilon <= 64.0f)) return CC_ERR_INVALID;
    if (mode != CC_AMSF_NF && mode != CC_AMSF_NF_S && mode != CC_AMSF_COO) return CC_ERR_INVALID;
    if (m && (!weights || !aligned(weights, 4))) return CC_ERR_INVALID;
    if (n > 0 && (!forest_out || !aligned(forest_out, 4))) return CC_ERR_INVALID;
    if (labels_out && !aligned(labels_out, 4)) return CC_ERR_INVALID;
    *count_out = 0;
    *weight_out = 0.0;
    if (n == 0) return CC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = offsets_u64 ? run_amsf<uint64_t>(offsets, edges, weights, n, m, epsilon, mode, forest_out, count_out,
                                          weight_out, labels_out, s)
                     : run_amsf<uint32_t>(offsets, edges, weights, n, m, epsilon, mode, forest_out, count_out,
                                          weight_out, labels_out, s);
    if (st != CC_OK) return st;
    return cc_device_error(stream, nullptr);
}
