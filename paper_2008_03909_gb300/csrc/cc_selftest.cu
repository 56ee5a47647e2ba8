// cc_selftest.cu -- checks of the library's bounded waits that need no
// fault: a cooperative launch whose blocks meet at the grid barrier a few
// times, optionally with one block that leaves without arriving.  The
// others then give up after the wait limit, record ERR_NONCONVERGED and
// leave; the context stays usable.
#include "cc_internal.h"

using namespace ccg;

namespace {

__global__ void k_barrier_selftest(GridBar *bar, int skip_block, uint64_t limit_ns, uint32_t *passed, Dev d) {
    if ((int)blockIdx.x == skip_block) return;   // never arrives
    for (int r = 0; r < 3; ++r)
        if (!grid_sync(bar, d, limit_ns)) return;
    if (threadIdx.x == 0) atomicAdd(passed, 1u);
}

}  // namespace

extern "C" cc_status cc_selftest_grid_barrier(int skip_block, uint32_t wait_ms, uint32_t *blocks_passed_out,
                                              void *stream) {
    if (wait_ms < 1 || wait_ms > 4000 || !blocks_passed_out) return CC_ERR_INVALID;
    const DeviceInfo *di = device_info();
    if (!di) return CC_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    const size_t o_bar = sc.reserve(sizeof(GridBar)), o_pass = sc.reserve(4);
    cc_status st = sc.alloc(s);
    if (st != CC_OK) return st;
    GridBar *bar = sc.at<GridBar>(o_bar);
    uint32_t *passed = sc.at<uint32_t>(o_pass);
    cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(passed, 0, 4, s);
    if (e != cudaSuccess) return from_cuda(e);
    Dev d = make_dev(di, 1);
    uint64_t limit = (uint64_t)wait_ms * 1000000ull;
    unsigned grid = (unsigned)di->sms;
    void *args[] = {&bar, &skip_block, &limit, &passed, &d};
    {
        CC_PROF("k_barrier_selftest", s);
        e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, grid, 128, args, 0, s);
    }
    if (e != cudaSuccess) return from_cuda(e);
    e = cudaMemcpyAsync(blocks_passed_out, passed, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    return cc_device_error(stream, nullptr);
}
