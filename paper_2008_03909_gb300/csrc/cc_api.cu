// cc_api.cu -- library-wide pieces of the C ABI: the per-device sticky
// error word, device facts, option defaults and validation, status strings.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cc_internal.h"

namespace ccg {

// Sticky device error word: kernels OR CC_DEVERR_* bits into it instead of
// trapping; cc_device_error() reads and clears it.
__device__ uint32_t g_cc_err;

namespace {
std::mutex g_mu;
DeviceInfo g_info[64];
std::atomic<uint64_t> g_cap_override{0};
}  // namespace

const DeviceInfo *device_info() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    DeviceInfo &di = g_info[dev];
    if (di.device == dev) return &di;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return nullptr;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cc_err) != cudaSuccess) return nullptr;
    // Keep freed scratch in the device's default pool across calls so that
    // stream-ordered allocation stays cheap after the first call.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    di.sms = sms;
    di.err = static_cast<uint32_t *>(p);
    di.device = dev;
    return &di;
}

uint64_t loop_cap(uint64_t n) {
    uint64_t o = g_cap_override.load();
    return o ? o : 2 * n + 1024;
}

uint32_t round_cap() {
    uint64_t o = g_cap_override.load();
    return o ? (uint32_t)(o < 4096 ? o : 4096) : 4096u;
}

cc_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return CC_OK;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
}

cc_status check_graph(const void *offsets, int offsets_u64, const uint32_t *edges, uint32_t n, uint64_t m) {
    if (n == 0xFFFFFFFFu) return CC_ERR_INVALID;   // 0xFFFFFFFF is reserved as "none"
    if (n == 0) return CC_OK;
    if (!offsets) return CC_ERR_INVALID;
    if (m > 0 && !edges) return CC_ERR_INVALID;
    // naturally aligned elements (the kernels never assume more than this)
    if (reinterpret_cast<uintptr_t>(offsets) % (offsets_u64 ? 8 : 4) != 0) return CC_ERR_INVALID;
    if (edges && reinterpret_cast<uintptr_t>(edges) % 4 != 0) return CC_ERR_INVALID;
    if (!offsets_u64 && m > 0xFFFFFFFFull) return CC_ERR_INVALID;
    return CC_OK;
}

cc_status check_sample(const cc_sample_opt &s) {
    if (s.kind < CC_SAMPLE_NONE || s.kind > CC_SAMPLE_LDD) return CC_ERR_INVALID;
    if (s.kind == CC_SAMPLE_KOUT && (s.k < 1 || s.k > 64)) return CC_ERR_INVALID;
    if (s.kind == CC_SAMPLE_BFS && (s.bfs_tries < 1 || s.bfs_tries > 1024)) return CC_ERR_INVALID;
    if (s.kind == CC_SAMPLE_LDD && !(s.ldd_beta > 0.0f && s.ldd_beta <= 64.0f)) return CC_ERR_INVALID;
    if (s.freq_samples > 4096) return CC_ERR_INVALID;
    if (s.kout_rule > CC_KOUT_PURE) return CC_ERR_INVALID;
    return CC_OK;
}

cc_status check_finish(const cc_finish_opt &f) {
    if (f.kind < CC_FINISH_UF_REM_CAS || f.kind > CC_FINISH_LABEL_PROP) return CC_ERR_INVALID;
    if (f.find < CC_FIND_NAIVE || f.find > CC_FIND_COMPRESS) return CC_ERR_INVALID;
    if (f.splice < CC_SPLICE_SPLIT_ONE || f.splice > CC_SPLICE_ATOMIC) return CC_ERR_INVALID;
    // Rem's Compress option is FindNaive / Split / Halve (FindCompress with
    // SpliceAtomic is incorrect: the counter-example in the appendix on
    // Rem's algorithm)
    if (f.kind == CC_FINISH_UF_REM_CAS && f.find == CC_FIND_COMPRESS) return CC_ERR_INVALID;
    if (f.kind != CC_FINISH_LIU_TARJAN) return f.lt_rules == 0 ? CC_OK : CC_ERR_INVALID;
    // the sixteen Liu-Tarjan variants
    const int conn = f.lt_rules & 3;
    if (f.lt_rules & ~31) return CC_ERR_INVALID;
    if (conn == 3) return CC_ERR_INVALID;
    if (conn == CC_LT_CONNECT && !(f.lt_rules & CC_LT_ALTER)) return CC_ERR_INVALID;   // Connect needs Alter
    if (conn == CC_LT_EXTENDED && (f.lt_rules & CC_LT_ROOTUP)) return CC_ERR_INVALID;
    return CC_OK;
}

namespace {
std::atomic<uint64_t> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
struct Pending {
    const char *name;
    cudaEvent_t e0, e1;
};
std::vector<Pending> g_pending;
std::map<std::string, std::pair<uint64_t, double>> g_totals;

void resolve_pending_locked() {
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.e1) == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess) {
            auto &t = g_totals[p.name];
            t.first += 1;
            t.second += ms;
        }
        cudaEventDestroy(p.e0);
        cudaEventDestroy(p.e1);
    }
    g_pending.clear();
    (void)cudaGetLastError();
}
}  // namespace

LaunchScope::LaunchScope(const char *name, cudaStream_t s) : name_(name), s_(s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_prof_on.load(std::memory_order_relaxed)) {
        if (cudaEventCreate(&e0_) == cudaSuccess && cudaEventCreate(&e1_) == cudaSuccess) {
            cudaEventRecord(e0_, s_);
        } else {
            (void)cudaGetLastError();
            e0_ = e1_ = nullptr;
        }
    }
}

LaunchScope::~LaunchScope() {
    if (!e0_ || !e1_) return;
    cudaEventRecord(e1_, s_);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending.push_back(Pending{name_, e0_, e1_});
    if (g_pending.size() > 4096) resolve_pending_locked();
}

}  // namespace ccg

using namespace ccg;

// The kernel whose image cc_binary_version reports (every kernel of the
// library is built for the same single target).
static __global__ void k_version_probe() {}

extern "C" {

void cc_default_opts(cc_sample_opt *sample, cc_finish_opt *finish) {
    if (sample) {
        sample->kind = CC_SAMPLE_KOUT;
        sample->k = 2;
        sample->bfs_tries = 3;
        sample->ldd_beta = 0.2f;
        sample->seed = 1;
        sample->freq_samples = 0;
        sample->kout_rule = CC_KOUT_HYBRID;
    }
    if (finish) {
        finish->kind = CC_FINISH_UF_REM_CAS;
        finish->find = CC_FIND_NAIVE;
        finish->splice = CC_SPLICE_SPLIT_ONE;
        finish->lt_rules = 0;
    }
}

cc_status cc_device_error(void *stream, uint32_t *bits_out) {
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t bits = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, di->err, sizeof(bits), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(di->err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    if (bits_out) *bits_out = bits;
    if (bits & CC_DEVERR_NONCONVERGED) return CC_ERR_NONCONVERGED;
    if (bits & (CC_DEVERR_BAD_EDGE | CC_DEVERR_BAD_OFFSETS)) return CC_ERR_BAD_INPUT;
    return CC_OK;
}

void cc_set_iteration_cap(uint64_t cap) { g_cap_override.store(cap); }

void cc_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    resolve_pending_locked();
    if (on) g_totals.clear();
    g_prof_on.store(on != 0);
}

int cc_profile_read(cc_kernel_time *out, int max) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    resolve_pending_locked();
    int i = 0;
    for (auto &kv : g_totals) {
        if (out && i < max) {
            std::memset(out[i].name, 0, sizeof(out[i].name));
            std::strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
            out[i].launches = kv.second.first;
            out[i].ms = kv.second.second;
        }
        ++i;
    }
    return i;
}

uint64_t cc_launch_count(void) { return g_launches.load(); }

const char *cc_status_str(cc_status s) {
    switch (s) {
        case CC_OK: return "ok";
        case CC_ERR_INVALID: return "invalid argument";
        case CC_ERR_OOM: return "out of device memory";
        case CC_ERR_CUDA: return "CUDA runtime error";
        case CC_ERR_NONCONVERGED: return "device loop reached its iteration or time cap";
        case CC_ERR_BAD_INPUT: return "edge id >= n or malformed offsets";
        case CC_ERR_UNSUPPORTED: return "unsupported option combination";
    }
    return "unknown status";
}

const char *cc_version(void) { return "connectit-gb300 0.1 (sm_103a)"; }

cc_status cc_binary_version(int *version_out) {
    if (!version_out) return CC_ERR_INVALID;
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, (const void *)k_version_probe);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return from_cuda(e);
    }
    *version_out = a.binaryVersion;
    return CC_OK;
}

}  // extern "C"
