// cc_internal.h -- host-side helpers shared by the library's translation
// units (not part of the public ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "connectit_gb.h"
#include "cc_device.cuh"

namespace ccg {

// Per-device facts the launches need.
struct DeviceInfo {
    int device = -1;
    int sms = 0;
    uint32_t *err = nullptr;   // device address of the sticky error word
};

// Info for the current device (initialised once per device, thread safe).
// Returns nullptr if the CUDA runtime fails.
const DeviceInfo *device_info();

// Iteration cap for one device loop on a graph of n vertices, and the cap on
// rounds of the host-driven round loops (SV, LT, BFS levels).
uint64_t loop_cap(uint64_t n);
uint32_t round_cap();

inline Dev make_dev(const DeviceInfo *di, uint64_t n) { return Dev{di->err, loop_cap(n)}; }

// CUDA error -> status (an allocation failure is CC_ERR_OOM, anything else,
// e.g. an earlier sticky fault, CC_ERR_CUDA).
cc_status from_cuda(cudaError_t e);

// Grid for a loop over `work` items with `threads` per block, capped at a
// few waves (kernels grid-stride beyond that).
inline unsigned grid_for(const DeviceInfo *di, uint64_t work, unsigned threads, unsigned waves = 8) {
    uint64_t b = (work + threads - 1) / threads;
    uint64_t cap = (uint64_t)di->sms * waves;
    if (b > cap) b = cap;
    if (b == 0) b = 1;
    return (unsigned)b;
}

// One stream-ordered scratch block carved into aligned pieces.
class Scratch {
  public:
    // Reserve `bytes` (256-byte aligned); returns the offset.
    size_t reserve(size_t bytes) {
        size_t off = total_;
        total_ += (bytes + 255) & ~size_t(255);
        return off;
    }
    cc_status alloc(cudaStream_t s) {
        if (total_ == 0) return CC_OK;
        cudaError_t e = cudaMallocAsync(&base_, total_, s);
        if (e != cudaSuccess) {
            base_ = nullptr;
            return from_cuda(e);
        }
        stream_ = s;
        return CC_OK;
    }
    template <typename T>
    T *at(size_t off) const { return reinterpret_cast<T *>(static_cast<char *>(base_) + off); }
    void release() {
        if (base_) cudaFreeAsync(base_, stream_);
        base_ = nullptr;
    }
    ~Scratch() { release(); }
    size_t total() const { return total_; }

  private:
    size_t total_ = 0;
    void *base_ = nullptr;
    cudaStream_t stream_ = nullptr;
};

// Degree statistics of a graph for the selector's features: sum and sum
// of squares of the degrees, counts of degree 0, 1, 2, 3..16 and > 64, the
// edges at vertices of degree > 64, and the highest degree (key
// deg << 32 | ~v: ties to the smallest vertex).
struct FeatStats {
    unsigned long long sum_deg, cnt[5], edges_gt64, maxkey, sum_deg2;
};

// Control block of one call, in device memory.
struct Ctl {
    uint32_t nchunks;
    uint32_t nlight;
    uint32_t changed;
    uint32_t minv;
    uint32_t nfront[2];
    uint32_t last_round;
    uint32_t lmax;
    uint32_t ndefer;
    unsigned long long key;
    unsigned long long edges;
    unsigned long long mf[2];
    unsigned long long ldd_explored;   // LDD: frontier edges of the rounds so far
    uint32_t ldd_pull;                 // LDD: 1 while the rounds run bottom-up
    uint32_t ldd_push_nf;              // LDD: the frontier size the top-down kernels see (0 bottom-up)
    uint32_t ldd_done;                 // LDD: blocks of the frontier pass done (the last one decides)
    uint32_t ldd_minc[2];              // LDD: smallest centre id of the frontier, by parity (as nfront)
    uint32_t guess;                    // k-out: sampled guess of L_max the fused binning used
    uint32_t rebin;                    // 1 when the exact L_max differs from the guess
    unsigned long long nonroots;       // k-out fused pass: vertices whose root is not themselves
    unsigned long long steps;          // k-out fused pass: parent steps walked by its compression
    uint32_t sel_class;                // selected path: the chosen class
    uint32_t skip;                     // selected path: 1 when the default finish must not run
    unsigned long long gcount;         // k-out fused pass: non-roots under the L_max guess
    uint32_t fallback;                 // 1 when the guess holds no majority (labels counted in full)
    uint32_t stats_done;               // selected path: blocks of k_degree_stats done
    uint32_t kout_span;                // k-out first pass: vertex spans taken so far
    uint32_t spans[2][2];              // dynamic spans of the k-out mid compression [0] and fused count [1]: taken, done
};

// Launch accounting: one scope per kernel launch.  Counts every launch and,
// while profiling is enabled, brackets it with CUDA events on its stream.
class LaunchScope {
  public:
    LaunchScope(const char *name, cudaStream_t s);
    ~LaunchScope();

  private:
    const char *name_;
    cudaStream_t s_;
    cudaEvent_t e0_ = nullptr, e1_ = nullptr;
};
#define CC_CAT2(a, b) a##b
#define CC_CAT(a, b) CC_CAT2(a, b)
#define CC_PROF(name, stream) ::ccg::LaunchScope CC_CAT(cc_prof_, __LINE__)(name, stream)

// The min-label finishes that need not be monotone (cc_minlabel.cu): the
// Liu-Tarjan framework's variants, Stergiou's algorithm, label propagation.
// They run on the candidate lists the binning pass built (candidates: the
// vertices with edges whose sampled label is not the frequent one).
struct MinLabelIn {
    const void *I;
    bool offsets_u64;
    const uint32_t *A;
    uint32_t n;
    uint64_t m;
    uint32_t *P;                            // sampled labels in, canonical labels out
    const uint32_t *lmax_p;                 // device: the frequent sampled label, or null
    const uint32_t *light, *nlight;         // device: candidates of degree <= LIGHT_MAX
    const ChunkRef *chunks;                 // device: CHUNK-edge pieces of the heavier candidates
    const uint32_t *nchunks;
    uint64_t chunk_cap;
    const unsigned long long *cand_edges;   // device: edges out of the candidates
};
cc_status minlabel_finish(const MinLabelIn &in, const cc_finish_opt &fo, const DeviceInfo *di, const Dev &d,
                          cudaStream_t s, uint32_t *rounds_out);

// Validation shared by the entry points (host side, synchronous).
inline bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
cc_status check_graph(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m);
cc_status check_sample(const cc_sample_opt &s);
cc_status check_finish(const cc_finish_opt &f);

}  // namespace ccg
