// cc_incr.cu -- batch-incremental connectivity (Section 3.5, Algorithm 3,
// Appendix B.4).  A handle keeps the parent array P resident in device
// memory.  Initialize runs static connectivity on the base graph into P.
// With a union-find finish each batch's inserts are Unions (the handle's
// engine: Section 3.5's types 1 and 3); with SV or Liu-Tarjan PRF (type 2)
// the batch's pairs go through that finish's rounds (hooks, then a full
// shortcut) until a round changes nothing.  Queries compare the roots of
// both endpoints.  Inserts and queries are separate kernels on one stream,
// so a query sees every earlier insert.
#include "cc_internal.h"

using namespace ccg;

struct cc_incr {
    int device;
    uint32_t n;
    uint32_t *P;
    cc_finish_opt fo;
    uint32_t *hooks;   // UF-Hooks: the resident hooks array (all free after the base graph)
    uint32_t *prev;    // SV / LT-PRF: P at a round's start, plus one changed word at prev[n]
};

namespace {

constexpr unsigned TPB = 256;

__global__ void __launch_bounds__(256, 8) k_incr_iota(uint32_t *P, uint32_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        P[i] = (uint32_t)i;
}

// The four consecutive pairs [4g, 4g + 4) of a batch: two 16-byte loads
// when the pair array is 16-byte aligned and the group is whole (adjacent
// threads then read adjacent 32-byte sectors), else word loads.  ok[j] is
// false past the end and for ids >= n (flagged).
__device__ __forceinline__ void load_pairs4(const uint32_t *pairs, uint64_t g, uint64_t k, uint32_t n, bool vec,
                                            uint32_t (&u)[4], uint32_t (&v)[4], bool (&ok)[4], const Dev &d) {
    const uint64_t i0 = 4 * g;
    if (vec && i0 + 4 <= k) {
        const uint4 a = __ldcs(reinterpret_cast<const uint4 *>(pairs) + 2 * g);
        const uint4 b = __ldcs(reinterpret_cast<const uint4 *>(pairs) + 2 * g + 1);
        u[0] = a.x; v[0] = a.y; u[1] = a.z; v[1] = a.w;
        u[2] = b.x; v[2] = b.y; u[3] = b.z; v[3] = b.w;
#pragma unroll
        for (int j = 0; j < 4; ++j) ok[j] = true;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ok[j] = i0 + j < k;
            u[j] = ok[j] ? __ldcs(pairs + 2 * (i0 + j)) : 0;
            v[j] = ok[j] ? __ldcs(pairs + 2 * (i0 + j) + 1) : 0;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (ok[j] && (u[j] >= n || v[j] >= n)) { atomicOr(d.err, ERR_BAD_EDGE); ok[j] = false; }
}

// Insert(u, v) = Union(u, v) for every pair; four consecutive pairs per
// thread step, their eight parent loads issued before any union.  Four
// pairs, their parents and an inlined union loop do not fit 32 registers
// (eight blocks per SM spilled 120 bytes per thread), so the kernel runs at
// six blocks per SM (40 registers) on a grid of one wave at that occupancy.
constexpr int INSERT_MINB = 6;
template <class E>
__global__ void __launch_bounds__(256, INSERT_MINB) k_incr_insert(uint32_t *P, uint32_t n, const uint32_t *pairs, uint64_t k, Dev d) {
    const bool vec = (reinterpret_cast<uintptr_t>(pairs) & 15) == 0;
    const uint64_t groups = (k + 3) / 4;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < groups;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u[4], v[4], pu[4], pv[4];
        bool ok[4];
        load_pairs4(pairs, g, k, n, vec, u, v, ok, d);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            pu[j] = ok[j] ? ld_rel(P + u[j]) : 0;
            pv[j] = ok[j] ? ld_rel(P + v[j]) : 0;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j] && pu[j] != pv[j]) E::unite(P, u[j], v[j], pu[j], pv[j], d);
    }
}

// Type 2 (SV, Liu-Tarjan PRF): one round over a batch's pairs.  SV hooks
// the larger of the two parents under the smaller if it was a root at the
// round's start (writeMin); PRF offers each parent to the other parent
// under the same root condition.  P is flat (every vertex at its root)
// between rounds, so the parents are the roots.
template <bool SV>
__global__ void __launch_bounds__(256, 8) k_incr_round(uint32_t *P, const uint32_t *prev, uint32_t n,
                                                       const uint32_t *pairs, uint64_t k, uint32_t *changed,
                                                       Dev d) {
    bool hit = false;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < k; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = __ldcs(pairs + 2 * i), v = __ldcs(pairs + 2 * i + 1);
        if (u >= n || v >= n) { atomicOr(d.err, ERR_BAD_EDGE); continue; }
        const uint32_t x = ld_rel(P + u), y = ld_rel(P + v);
        if (SV) {
            const uint32_t l = x < y ? x : y, h = x < y ? y : x;
            if (l != h && prev[h] == h) hit |= atomicMin(P + h, l) > l;
        } else {
            if (y < x && prev[x] == x) hit |= atomicMin(P + x, y) > y;
            if (x < y && prev[y] == y) hit |= atomicMin(P + y, x) > x;
        }
    }
    if (hit) *changed = 1u;
}

__global__ void k_incr_flag(uint32_t *err, uint32_t bits) { atomicOr(err, bits); }

// FullShortcut: every vertex points at its root.
__global__ void __launch_bounds__(256, 8) k_incr_shortcut(uint32_t *P, uint32_t n, Dev d) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)i, p = ld_rel(P + v);
        const uint32_t r = find_from<FIND_NAIVE>(P, v, p, d);
        if (r != p) P[v] = r;
    }
}

// IsConnected(u, v): Find(u) == Find(v) with the handle's find option.
template <int FIND>
__global__ void __launch_bounds__(256, 8) k_incr_query(uint32_t *P, uint32_t n, const uint32_t *pairs, uint64_t q, uint8_t *ans, Dev d) {
    // four consecutive queries per thread step: pairs by two 16-byte loads,
    // all eight parent loads in flight, answers written as one word when
    // the answer array allows it
    const bool vec = (reinterpret_cast<uintptr_t>(pairs) & 15) == 0;
    const bool wvec = (reinterpret_cast<uintptr_t>(ans) & 3) == 0;
    const uint64_t groups = (q + 3) / 4;
    for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < groups;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u[4], v[4], pu[4], pv[4];
        bool ok[4];
        load_pairs4(pairs, g, q, n, vec, u, v, ok, d);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            pu[j] = ok[j] ? ld_rel(P + u[j]) : 0;
            pv[j] = ok[j] ? ld_rel(P + v[j]) : 0;
        }
        uint8_t a[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!ok[j]) { a[j] = 0; continue; }
            if (pu[j] == pv[j]) { a[j] = 1; continue; }
            const uint32_t ru = find_from<FIND>(P, u[j], pu[j], d);
            const uint32_t rv = find_from<FIND>(P, v[j], pv[j], d);
            a[j] = ru == rv;
        }
        const uint64_t i0 = 4 * g;
        if (wvec && i0 + 4 <= q) {
            *reinterpret_cast<uchar4 *>(ans + i0) = make_uchar4(a[0], a[1], a[2], a[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (i0 + j < q) ans[i0 + j] = a[j];
        }
    }
}

// Canonical labels of the current forest (roots are component minima).
__global__ void __launch_bounds__(256, 8) k_incr_labels(const uint32_t *P, uint32_t n, uint32_t *out, Dev d) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v = (uint32_t)i;
        out[i] = find_from<FIND_NAIVE>(const_cast<uint32_t *>(P), v, ld_rel(P + v), d);
    }
}


}  // namespace

extern "C" {

cc_status cc_incr_create(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                         const cc_sample_opt *sample, const cc_finish_opt *finish, void *stream, cc_incr **out) {
    if (!out) return CC_ERR_INVALID;
    *out = nullptr;
    if (n == 0xFFFFFFFFu) return CC_ERR_INVALID;
    if (m > 0) {
        cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
        if (st != CC_OK) return st;
    }
    cc_sample_opt so;
    cc_finish_opt fo;
    cc_default_opts(&so, &fo);
    if (sample) so = *sample;
    if (finish) fo = *finish;
    cc_status st = check_sample(so);
    if (st == CC_OK) st = check_finish(fo);
    if (st != CC_OK) return st;
    // union-find (types 1 and 3) and SV / Liu-Tarjan PRF (type 2); the
    // finishes that are not root-based have no batch-incremental form
    if (fo.kind == CC_FINISH_LIU_TARJAN || fo.kind == CC_FINISH_STERGIOU || fo.kind == CC_FINISH_LABEL_PROP)
        return CC_ERR_UNSUPPORTED;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cc_incr *h = new cc_incr{di->device, n, nullptr, fo, nullptr, nullptr};
    if (n > 0) {
        cudaError_t e = cudaMalloc(&h->P, (size_t)n * 4);
        if (e == cudaSuccess && fo.kind == CC_FINISH_UF_HOOKS) {
            e = cudaMalloc(&h->hooks, (size_t)n * 4);
            if (e == cudaSuccess) e = cudaMemsetAsync(h->hooks, 0xFF, (size_t)n * 4, s);
        }
        if (e == cudaSuccess && (fo.kind == CC_FINISH_SV || fo.kind == CC_FINISH_LT_PRF))
            e = cudaMalloc(&h->prev, ((size_t)n + 1) * 4);
        if (e != cudaSuccess) {
            if (h->P) cudaFree(h->P);
            if (h->hooks) cudaFree(h->hooks);
            if (h->prev) cudaFree(h->prev);
            delete h;
            return from_cuda(e);
        }
        if (m > 0 && offsets) {
            st = cc_static(offsets, offsets_u64, edges, n, m, &so, &fo, h->P, stream);
        } else {
            {
                CC_PROF("k_incr_iota", s);
                k_incr_iota<<<grid_for(di, n, TPB), TPB, 0, s>>>(h->P, n);
            }
            st = from_cuda(cudaGetLastError());
        }
        if (st != CC_OK) {
            cudaFree(h->P);
            if (h->hooks) cudaFree(h->hooks);
            if (h->prev) cudaFree(h->prev);
            delete h;
            return st;
        }
    }
    *out = h;
    return CC_OK;
}

cc_status cc_incr_insert_batch(cc_incr *h, const uint32_t *pairs, uint64_t k, void *stream) {
    if (!h) return CC_ERR_INVALID;
    if (k == 0) return CC_OK;
    if (!pairs || !aligned(pairs, 4)) return CC_ERR_INVALID;
    if (h->n == 0) return CC_ERR_INVALID;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Dev d = make_dev(di, h->n);
    d.hooks = h->hooks;
    if (h->prev) {
        // type 2: rounds until nothing changes; each round reads a flag on
        // the host, so this call synchronises the stream once per round
        const unsigned gk = grid_for(di, k, TPB), gn = grid_for(di, h->n, TPB);
        uint32_t *changed = h->prev + h->n;
        for (uint32_t r = 0;; ++r) {
            if (r >= round_cap()) {
                k_incr_flag<<<1, 1, 0, s>>>(di->err, CC_DEVERR_NONCONVERGED);
                return from_cuda(cudaGetLastError());
            }
            cudaError_t e = cudaMemsetAsync(changed, 0, 4, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->prev, h->P, (size_t)h->n * 4, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return from_cuda(e);
            {
                CC_PROF("k_incr_round", s);
                if (h->fo.kind == CC_FINISH_SV)
                    k_incr_round<true><<<gk, TPB, 0, s>>>(h->P, h->prev, h->n, pairs, k, changed, d);
                else
                    k_incr_round<false><<<gk, TPB, 0, s>>>(h->P, h->prev, h->n, pairs, k, changed, d);
            }
            {
                CC_PROF("k_incr_shortcut", s);
                k_incr_shortcut<<<gn, TPB, 0, s>>>(h->P, h->n, d);
            }
            uint32_t hc = 0;
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, changed, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return from_cuda(e);
            if (hc == 0) return CC_OK;
        }
    }
    const unsigned grid = grid_for(di, (k + 3) / 4, TPB, INSERT_MINB);
    return with_uf_engine(h->fo.kind, h->fo.find, h->fo.splice, [&](auto eng) -> cc_status {
        using E = decltype(eng);
        {
            CC_PROF("k_incr_insert", s);
            k_incr_insert<E><<<grid, TPB, 0, s>>>(h->P, h->n, pairs, k, d);
        }
        return from_cuda(cudaGetLastError());
    });
}

cc_status cc_incr_query_batch(cc_incr *h, const uint32_t *pairs, uint64_t q, uint8_t *answers_out, void *stream) {
    if (!h) return CC_ERR_INVALID;
    if (q == 0) return CC_OK;
    if (!pairs || !answers_out || h->n == 0 || !aligned(pairs, 4)) return CC_ERR_INVALID;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Dev d = make_dev(di, h->n);
    const unsigned grid = grid_for(di, (q + 3) / 4, TPB);
    switch (h->fo.find) {
        case CC_FIND_SPLIT: { CC_PROF("k_incr_query", s); k_incr_query<FIND_SPLIT><<<grid, TPB, 0, s>>>(h->P, h->n, pairs, q, answers_out, d); } break;
        case CC_FIND_HALVE: { CC_PROF("k_incr_query", s); k_incr_query<FIND_HALVE><<<grid, TPB, 0, s>>>(h->P, h->n, pairs, q, answers_out, d); } break;
        case CC_FIND_COMPRESS: { CC_PROF("k_incr_query", s); k_incr_query<FIND_COMPRESS><<<grid, TPB, 0, s>>>(h->P, h->n, pairs, q, answers_out, d); } break;
        default: { CC_PROF("k_incr_query", s); k_incr_query<FIND_NAIVE><<<grid, TPB, 0, s>>>(h->P, h->n, pairs, q, answers_out, d); } break;
    }
    return from_cuda(cudaGetLastError());
}

cc_status cc_incr_labels(cc_incr *h, uint32_t *labels_out, void *stream) {
    if (!h) return CC_ERR_INVALID;
    if (h->n == 0) return CC_OK;
    if (!labels_out || !aligned(labels_out, 4)) return CC_ERR_INVALID;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        CC_PROF("k_incr_labels", s);
        k_incr_labels<<<grid_for(di, h->n, TPB), TPB, 0, s>>>(h->P, h->n, labels_out, make_dev(di, h->n));
    }
    return from_cuda(cudaGetLastError());
}

uint32_t cc_incr_num_vertices(const cc_incr *h) { return h ? h->n : 0; }

cc_status cc_incr_destroy(cc_incr *h) {
    if (!h) return CC_OK;
    cudaError_t e = cudaSuccess;
    if (h->P) e = cudaFree(h->P);
    for (uint32_t *p : {h->hooks, h->prev}) {
        if (!p) continue;
        const cudaError_t e2 = cudaFree(p);
        if (e == cudaSuccess) e = e2;
    }
    delete h;
    return from_cuda(e);
}

}  // extern "C"
