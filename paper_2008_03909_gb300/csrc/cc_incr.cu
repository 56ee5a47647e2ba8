// cc_incr.cu -- batch-incremental connectivity (Section 3.5, Algorithm 3,
// Appendix B.4).  A handle keeps the union-find parent array P resident in
// device memory.  Initialize runs static connectivity on the base graph
// into P; each batch's inserts are Unions (the handle's union-find engine)
// and its queries compare the roots of both endpoints.  Inserts and queries
// are separate kernels on one stream, so a query sees every earlier insert
// (the phase-concurrent setting of Section 3.5, type 3).
#include "cc_internal.h"

using namespace ccg;

struct cc_incr {
    int device;
    uint32_t n;
    uint32_t *P;
    cc_finish_opt fo;
    uint32_t *hooks;   // UF-Hooks: the resident hooks array (all free after the base graph)
};

namespace {

constexpr unsigned TPB = 256;

__global__ void __launch_bounds__(256, 8) k_incr_iota(uint32_t *P, uint32_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        P[i] = (uint32_t)i;
}

// Insert(u, v) = Union(u, v) for every pair; four pairs per thread step so
// their parent loads overlap.
template <class E>
__global__ void __launch_bounds__(256, 8) k_incr_insert(uint32_t *P, uint32_t n, const uint32_t *pairs, uint64_t k, Dev d) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < k; i0 += 4 * stride) {
        uint32_t u[4], v[4], pu[4], pv[4];
        bool ok[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint64_t i = i0 + j * stride;
            ok[j] = i < k;
            u[j] = ok[j] ? __ldcs(pairs + 2 * i) : 0;
            v[j] = ok[j] ? __ldcs(pairs + 2 * i + 1) : 0;
            if (ok[j] && (u[j] >= n || v[j] >= n)) { atomicOr(d.err, ERR_BAD_EDGE); ok[j] = false; }
        }
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

// IsConnected(u, v): Find(u) == Find(v) with the handle's find option.
template <int FIND>
__global__ void __launch_bounds__(256, 8) k_incr_query(uint32_t *P, uint32_t n, const uint32_t *pairs, uint64_t q, uint8_t *ans, Dev d) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < q;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = __ldcs(pairs + 2 * i), v = __ldcs(pairs + 2 * i + 1);
        if (u >= n || v >= n) {
            atomicOr(d.err, ERR_BAD_EDGE);
            ans[i] = 0;
            continue;
        }
        uint32_t pu = ld_rel(P + u), pv = ld_rel(P + v);
        if (pu == pv) { ans[i] = 1; continue; }
        uint32_t ru = find_from<FIND>(P, u, pu, d);
        uint32_t rv = find_from<FIND>(P, v, pv, d);
        ans[i] = ru == rv;
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
    if (fo.kind != CC_FINISH_UF_REM_CAS && fo.kind != CC_FINISH_UF_ASYNC && fo.kind != CC_FINISH_UF_HOOKS &&
        fo.kind != CC_FINISH_UF_EARLY)
        return CC_ERR_UNSUPPORTED;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cc_incr *h = new cc_incr{di->device, n, nullptr, fo, nullptr};
    if (n > 0) {
        cudaError_t e = cudaMalloc(&h->P, (size_t)n * 4);
        if (e == cudaSuccess && fo.kind == CC_FINISH_UF_HOOKS) {
            e = cudaMalloc(&h->hooks, (size_t)n * 4);
            if (e == cudaSuccess) e = cudaMemsetAsync(h->hooks, 0xFF, (size_t)n * 4, s);
        }
        if (e != cudaSuccess) {
            if (h->P) cudaFree(h->P);
            if (h->hooks) cudaFree(h->hooks);
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
    const unsigned grid = grid_for(di, (k + 3) / 4, TPB);
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
    const unsigned grid = grid_for(di, q, TPB);
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
    if (h->hooks) {
        const cudaError_t e2 = cudaFree(h->hooks);
        if (e == cudaSuccess) e = e2;
    }
    delete h;
    return from_cuda(e);
}

}  // extern "C"
