// cc_probe.cu -- the MapEdges and GatherEdges primitives (Section 4,
// "Comparison with MapEdges and GatherEdges", Table 8): for every vertex, a
// reduction over its incident edges.  MapEdges reads every edge and counts
// it (the cost of reading the graph and writing one value per vertex);
// GatherEdges reads, for every edge, the value of an n-sized array at the
// neighbour (the indirect read every exact connectivity algorithm performs
// per edge).  They measure this GPU's floors for those two access patterns.
#include "cc_internal.h"

using namespace ccg;

namespace {

constexpr unsigned TPB = 256;

// Per-vertex reduction of the light path: MODE 0 counts the edges read,
// MODE 1 sums x at the neighbours.
template <int MODE>
struct ProbeEdge {
    const uint32_t *x;
    uint32_t acc;
    __device__ __forceinline__ void apply4(uint32_t, const uint32_t (&v)[4], const bool (&ok)[4]) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) acc += MODE == 0 ? 1u : x[v[j]];
    }
};

// The light path's reduction when the warp walks its 32 vertices' edges
// together (warp_light_edges): each edge adds into its source's slot of
// the warp's shared-memory sums (sums[u - base], vertices base .. base+31).
template <int MODE>
struct ProbeFlat {
    const uint32_t *x;
    uint32_t *sums;
    uint64_t base;
    __device__ __forceinline__ void apply4(uint32_t u, const uint32_t (&v)[4], const bool (&ok)[4]) {
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) acc += MODE == 0 ? 1u : x[v[j]];
        if (ok[0]) atomicAdd(sums + (uint32_t)(u - base), acc);
    }
    __device__ __forceinline__ void apply4u(const uint32_t (&u)[4], const uint32_t (&v)[4], const bool (&ok)[4]) {
        uint32_t val[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) val[j] = ok[j] ? (MODE == 0 ? 1u : x[v[j]]) : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (ok[j]) atomicAdd(sums + (uint32_t)(u[j] - base), val[j]);
    }
};

// MODE 0: MapEdges, out[v] = #edges read; MODE 1: GatherEdges,
// out[v] = sum of x[w] over neighbours w (mod 2^32).  The edges of the
// vertices of degree <= LIGHT_MAX are walked by the warp together
// (warp_light_edges); heavier vertices are zeroed here and reduced in
// chunks by k_probe_chunks.
template <typename OffT, int MODE>
__global__ void __launch_bounds__(256, 8) k_probe_bin(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                                                      const uint32_t *x, uint32_t *out, ChunkRef *chunks,
                                                      uint32_t *nchunks, uint64_t cap, Dev d) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    __shared__ uint32_t sums_all[TPB];
    uint32_t *sums = sums_all + (threadIdx.x & ~31u);
    for (uint64_t base = warp * 32; base < n; base += nw * 32) {
        const uint64_t v = base + lane;
        uint64_t b = 0, e = 0;
        if (v < n) vertex_range(I, (uint32_t)v, m, b, e, d);
        const uint64_t deg = e - b;
        const uint32_t nc = deg > LIGHT_MAX ? (uint32_t)((deg + CHUNK - 1) / CHUNK) : 0;
        const uint32_t slot = warp_append_full(nchunks, nc);
        if (nc) write_chunks(chunks, cap, slot, nc, (uint32_t)v, d);
        sums[lane] = 0;
        __syncwarp();
        ProbeFlat<MODE> f{x, sums, base};
        warp_light_edges((uint32_t)v, b, nc ? 0u : (uint32_t)deg, A, n, f, d);
        __syncwarp();
        if (v < n) out[v] = sums[lane];
        __syncwarp();
    }
}

template <typename OffT, int MODE>
__global__ void __launch_bounds__(256, 8) k_probe_chunks(const OffT *I, const uint32_t *A, uint32_t n, uint64_t m,
                                                         const uint32_t *x, uint32_t *out, const ChunkRef *chunks,
                                                         const uint32_t *nchunks, uint64_t cap, Dev d) {
    const int lane = threadIdx.x & 31;
    const uint32_t total = (uint32_t)((uint64_t)*nchunks < cap ? (uint64_t)*nchunks : cap);
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t c = warp; c < total; c += nwarps) {
        const ChunkRef cr = chunks[c];
        uint64_t b, e;
        vertex_range(I, cr.u, m, b, e, d);
        const uint64_t cb = b + (uint64_t)cr.c * CHUNK;
        const uint64_t ce = cb + CHUNK < e ? cb + CHUNK : e;
        ProbeEdge<MODE> f{x, 0u};
        warp_chunk_edges(cr.u, cb, ce, A, n, f, d);
        uint32_t acc = f.acc;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) atomicAdd(out + cr.u, acc);
    }
}

// Random sectors: word draw64(seed, i) * words / 2^64 of x for i < count,
// eight independent loads in flight per thread, summed mod 2^32 into *out.
// Each load touches one 32-byte sector at a position no neighbouring load
// shares: on an array larger than L2 this is the device's rate for the
// access that the k-out picks make (one random sector per pick).
__global__ void __launch_bounds__(256, 8) k_probe_sectors(const uint32_t *x, uint64_t words, uint64_t count,
                                                          uint64_t seed, uint32_t *out) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t acc = 0;
    for (uint64_t i0 = tid * 8; i0 < count; i0 += stride * 8) {
        uint32_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            v[j] = i0 + j < count ? ld_stream(x + __umul64hi(draw64(seed, i0 + j), words)) : 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) acc += v[j];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

template <typename OffT, int MODE>
cc_status run_probe(const void *offsets, const uint32_t *edges, uint32_t n, uint64_t m, const uint32_t *x,
                    uint32_t *out, cudaStream_t s) {
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    const Dev d = make_dev(di, n);
    const OffT *I = static_cast<const OffT *>(offsets);
    Scratch sc;
    const uint64_t cap = chunk_capacity(n, m);
    const size_t oc = sc.reserve(cap * sizeof(ChunkRef)), on = sc.reserve(4);
    cc_status st = sc.alloc(s);
    if (st != CC_OK) return st;
    cudaError_t e = cudaMemsetAsync(sc.at<uint32_t>(on), 0, 4, s);
    if (e != cudaSuccess) return from_cuda(e);
    const unsigned gv = grid_for(di, n, TPB), gc = grid_for(di, (uint64_t)1 << 40, TPB);
    {
        CC_PROF(MODE ? "k_gather_edges_bin" : "k_map_edges_bin", s);
        k_probe_bin<OffT, MODE><<<gv, TPB, 0, s>>>(I, edges, n, m, x, out, sc.at<ChunkRef>(oc), sc.at<uint32_t>(on),
                                                   cap, d);
    }
    {
        CC_PROF(MODE ? "k_gather_edges_chunks" : "k_map_edges_chunks", s);
        k_probe_chunks<OffT, MODE><<<gc, TPB, 0, s>>>(I, edges, n, m, x, out, sc.at<ChunkRef>(oc),
                                                      sc.at<uint32_t>(on), cap, d);
    }
    return from_cuda(cudaGetLastError());
}

}  // namespace

extern "C" {

cc_status cc_random_sectors(const uint32_t *x, uint64_t words, uint64_t count, uint64_t seed, uint32_t *out,
                            void *stream) {
    if (!x || !out || !aligned(x, 4) || !aligned(out, 4) || (words == 0 && count > 0)) return CC_ERR_INVALID;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(out, 0, 4, s);
    if (e != cudaSuccess) return from_cuda(e);
    if (count == 0) return CC_OK;
    {
        CC_PROF("k_probe_sectors", s);
        k_probe_sectors<<<grid_for(di, (count + 7) / 8, TPB), TPB, 0, s>>>(x, words, count, seed, out);
    }
    return from_cuda(cudaGetLastError());
}

cc_status cc_map_edges(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                       uint32_t *out, void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK || n == 0) return st;
    if (!out || !aligned(out, 4)) return CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return offsets_u64 ? run_probe<uint64_t, 0>(offsets, edges, n, m, nullptr, out, s)
                       : run_probe<uint32_t, 0>(offsets, edges, n, m, nullptr, out, s);
}

cc_status cc_gather_edges(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m,
                          const uint32_t *x, uint32_t *out, void *stream) {
    cc_status st = check_graph(offsets, offsets_u64, edges, n, m);
    if (st != CC_OK || n == 0) return st;
    if (!out || !x || !aligned(out, 4) || !aligned(x, 4)) return CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return offsets_u64 ? run_probe<uint64_t, 1>(offsets, edges, n, m, x, out, s)
                       : run_probe<uint32_t, 1>(offsets, edges, n, m, x, out, s);
}

}  // extern "C"
