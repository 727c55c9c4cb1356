// isax_selftest.cu - checks of the library's failure handling that make no GPU
// fault.  Every wait in the library's kernels is bounded: after its limit the
// kernel records that it gave up and returns, and the host reports
// ISAX_ERR_TIMEOUT.  These entry points let a test make such waits run out on
// purpose, on barriers that nothing else uses and with no copy in flight, and
// let it mark the next queries as timed out on the host side, so the status
// path of every query entry point can be checked.
#include <atomic>
#include <string>

#include "isax_common.cuh"
#include "isax_kernels_util.cuh"

namespace isax {

// One CTA waits on its own mbarrier (arrival count 1): the barrier completes
// only if the kernel arrives on it itself (arrive != 0); no bulk copy is ever
// issued, so nothing is in flight when the wait gives up.
__global__ void __launch_bounds__(32) mbar_wait_selftest_kernel(uint32_t max_polls, uint32_t arrive,
                                                                 uint32_t* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        if (arrive) mbar_arrive(&bar);
        *status = mbar_wait_bounded(&bar, 0, max_polls) ? 0u : 1u;
    }
}

// The grid barrier of the binning step, expecting `expected` arrivals from a
// cooperative grid: with expected > gridDim.x it can never be met.
__global__ void __launch_bounds__(128) grid_barrier_selftest_kernel(uint32_t* count, uint32_t expected,
                                                                    uint32_t max_polls, uint32_t* status) {
    __shared__ int ok;
    const bool met = grid_barrier(count, expected, max_polls, &ok);
    if (threadIdx.x == 0 && !met) atomicOr(status, 1u);
}

// Host side: the next `pending` control blocks read after a query report a
// wait that gave up.
static std::atomic<int> g_inject_timeouts{0};

uint32_t injected_query_flags() {
    int v = g_inject_timeouts.load();
    while (v > 0) {
        if (g_inject_timeouts.compare_exchange_weak(v, v - 1)) return QF_STALLED;
    }
    return 0u;
}

static uint32_t run_status_kernel(cudaStream_t st, uint32_t* dev_words, bool coop, int ctas,
                                  uint32_t expected, uint32_t max_polls, uint32_t arrive) {
    ISAX_CUDA_TRY(cudaMemsetAsync(dev_words, 0, 2 * sizeof(uint32_t), st));
    if (coop) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)ctas);
        cfg.blockDim = dim3(128);
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ISAX_LAUNCH("grid_barrier_selftest", st);
        ISAX_CUDA_TRY(cudaLaunchKernelEx(&cfg, grid_barrier_selftest_kernel, dev_words, expected, max_polls,
                                         dev_words + 1));
    } else {
        ISAX_LAUNCH("mbar_wait_selftest", st);
        mbar_wait_selftest_kernel<<<1, 32, 0, st>>>(max_polls, arrive, dev_words + 1);
        ISAX_CUDA_TRY(cudaGetLastError());
    }
    uint32_t status = 0;
    ISAX_CUDA_TRY(cudaMemcpyAsync(&status, dev_words + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    return status;
}

}  // namespace isax

using namespace isax;

extern "C" isax_status isax_selftest_wait(int32_t kind, int32_t satisfied, int32_t max_polls, void* cuda_stream) {
    set_error(ISAX_OK, "");
    if (kind != 0 && kind != 1) {
        set_error(ISAX_ERR_INVALID_ARG, "kind must be 0 (mbarrier) or 1 (grid barrier)");
        return ISAX_ERR_INVALID_ARG;
    }
    if (max_polls < 1 || max_polls > (1 << 24)) {
        set_error(ISAX_ERR_INVALID_ARG, "max_polls must be in [1, 2^24]");
        return ISAX_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint32_t* words = nullptr;
    try {
        words = static_cast<uint32_t*>(dev_alloc(2 * sizeof(uint32_t), st));
        uint32_t status;
        if (kind == 0) {
            status = run_status_kernel(st, words, false, 1, 0, (uint32_t)max_polls, satisfied ? 1u : 0u);
        } else {
            const int ctas = 4;  // a small cooperative grid, all resident
            status = run_status_kernel(st, words, true, ctas, (uint32_t)(satisfied ? ctas : ctas + 1),
                                       (uint32_t)max_polls, 0u);
        }
        dev_free(words, st);
        words = nullptr;
        if (status) {
            set_error(ISAX_ERR_TIMEOUT, kind == 0 ? "the mbarrier wait gave up" : "the grid barrier gave up");
            return ISAX_ERR_TIMEOUT;
        }
        return ISAX_OK;
    } catch (const Error& e) {
        if (words) dev_free(words, st);
        set_error(e.st, e.msg);
        return e.st;
    }
}

extern "C" isax_status isax_debug_inject_timeout(int32_t queries) {
    set_error(ISAX_OK, "");
    if (queries < 0) {
        set_error(ISAX_ERR_INVALID_ARG, "queries must be >= 0");
        return ISAX_ERR_INVALID_ARG;
    }
    g_inject_timeouts.store(queries);
    return ISAX_OK;
}
