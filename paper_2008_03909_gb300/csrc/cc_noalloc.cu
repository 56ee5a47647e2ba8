// cc_noalloc.cu -- an IdentifyFrequent entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need
// the frequent label: a latency-critical serving loop where cudaMalloc /
// cudaFree would synchronise the device and stall other work, a host
// callback or driver hook where runtime allocation calls are not allowed,
// or a process whose device memory is entirely reserved by another
// allocator.  cc_identify_frequent_noalloc serves them: its count scratch
// is a file-scope device array of fixed size, reserved when the library is
// loaded, so the call itself only enqueues a memset and kernels.
//
// The scratch is shared by every call on a device and keeps the contents of
// the last call; each call zeroes the part it uses before counting.  Calls
// whose work overlaps on the GPU (different streams without ordering) race
// on it and must not be issued.
#include "cc_internal.h"

using namespace ccg;

namespace {

constexpr unsigned TPB = 256;

static __device__ __align__(256) uint32_t g_noalloc_counts[CC_NOALLOC_MAX_LABELS];
static __device__ __align__(256) unsigned long long g_noalloc_key;

struct NoAllocScratch {
    uint32_t *counts = nullptr;
    unsigned long long *key = nullptr;
};

// Device addresses of the scratch arrays in the current device's context
// (host code cannot use the arrays' names as addresses).  They are looked
// up on every call rather than cached: a context that was torn down and
// created again (cudaDeviceReset) places the arrays at new addresses, and
// the lookup is a host-side table read that allocates nothing.  The first
// lookup on a device loads the library's device code there, so that first
// call belongs before any stream capture.
cc_status noalloc_scratch(NoAllocScratch *out) {
    void *c = nullptr, *k = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&c, g_noalloc_counts);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&k, g_noalloc_key);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return CC_ERR_CUDA;
    }
    out->counts = static_cast<uint32_t *>(c);
    out->key = static_cast<unsigned long long *>(k);
    return CC_OK;
}

// Count every label (labels >= n are flagged and skipped) with the same
// register heavy-hitter scheme as the allocating path.
__global__ void __launch_bounds__(256, 8) k_na_count(const uint32_t *L, uint32_t n, uint32_t *cnt, Dev d) {
    LabelCounter lc;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t l = L[i];
        if (l >= n) atomicOr(d.err, ERR_BAD_EDGE);
        else lc.add(cnt, l);
    }
    lc.flush(cnt);
}

// Arg-max with ties to the smallest label: max of (count << 32 | ~label).
__global__ void __launch_bounds__(256, 8) k_na_argmax(const uint32_t *cnt, uint32_t n, unsigned long long *key) {
    __shared__ unsigned long long red[8];
    unsigned long long best = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t c = cnt[i];
        unsigned long long k2 = c ? (((unsigned long long)c << 32) | (uint32_t)~(uint32_t)i) : 0ull;
        best = k2 > best ? k2 : best;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        best = y > best ? y : best;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) best = red[w] > best ? red[w] : best;
        if (best) atomicMax(key, best);
    }
}

__global__ void k_na_result(const unsigned long long *key, uint32_t *lmax) {
    unsigned long long k = *key;
    *lmax = k ? ~(uint32_t)(k & 0xFFFFFFFFull) : NONE;
}

}  // namespace

extern "C" cc_status cc_identify_frequent_noalloc(const uint32_t *labels, uint32_t n, uint32_t *lmax_out,
                                                  void *stream) {
    if (!lmax_out || (n > 0 && !labels)) return CC_ERR_INVALID;
    if (n > CC_NOALLOC_MAX_LABELS) return CC_ERR_INVALID;
    if (!aligned(lmax_out, 4) || (labels && !aligned(labels, 4))) return CC_ERR_INVALID;
    NoAllocScratch scr;
    cc_status st = noalloc_scratch(&scr);
    if (st != CC_OK) return st;
    const NoAllocScratch *sc = &scr;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Dev d = make_dev(di, n);
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemsetAsync(sc->counts, 0, (size_t)n * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc->key, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return from_cuda(e);
    const unsigned grid = grid_for(di, n, TPB);
    if (n > 0) {
        k_na_count<<<grid, TPB, 0, s>>>(labels, n, sc->counts, d);
        k_na_argmax<<<grid, TPB, 0, s>>>(sc->counts, n, sc->key);
    }
    k_na_result<<<1, 1, 0, s>>>(sc->key, lmax_out);
    return from_cuda(cudaGetLastError());
}
