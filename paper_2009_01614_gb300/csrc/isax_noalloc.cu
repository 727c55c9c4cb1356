// isax_noalloc.cu - an exact k-NN query entry point that never allocates.
//
// Some callers cannot allocate device memory while they answer a query: a
// host runtime that owns every byte of the GPU through its own pool and treats
// any allocation behind its back as a bug, or a latency-critical serving thread
// for which cudaMalloc / cudaMallocAsync can block on the driver or on other
// streams.  For them, isax_query_knn_noalloc runs the
// same query kernels as isax_query_knn on scratch that lives in one
// file-scope device array, fixed in size when the library is loaded and kept by
// every GPU that loads it until the process exits.
//
// Host code must not use the array's name as a device address (on the host it
// is only a stand-in).  Once per device, with that device current, the first
// call looks the real address up with cudaGetSymbolAddress and caches it; make
// that first call before any stream capture begins.  All calls share the one
// array and it keeps the previous call's contents, so each call resets what
// must start cleared (the control block and the top-k slots, before the
// kernels; the first kernel clears the bins).  Two calls whose kernels overlap on the
// GPU would race on the array; calls are serialised by a process-wide lock and
// each returns only after its results are copied out, so calls through this
// entry point never overlap.
#include <string.h>

#include <mutex>
#include <string>

#include "isax_common.cuh"

namespace isax {

namespace noalloc {
namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr uint32_t MAX_LEAVES = ISAX_NOALLOC_MAX_LEAVES;
constexpr uint32_t MAX_WORK = 2 * MAX_LEAVES;  // scan items: leaves + series / 128 (the scan's piece)
constexpr uint32_t MAX_CAND = ISAX_NOALLOC_MAX_CANDIDATES;
constexpr uint32_t MAX_SURV = ISAX_NOALLOC_MAX_SURVIVORS;

// byte offsets of the scratch pieces inside the array
constexpr size_t OFF_Q = 0;
constexpr size_t OFF_TABLE = align256(OFF_Q + sizeof(float) * MAX_LEN);
constexpr size_t OFF_LEAF_LB = align256(OFF_TABLE + sizeof(float) * W * MAX_CARD);
constexpr size_t OFF_WORK = align256(OFF_LEAF_LB + sizeof(float) * MAX_LEAVES);
constexpr size_t OFF_BIN_COUNT = align256(OFF_WORK + sizeof(uint2) * MAX_WORK);
constexpr size_t OFF_BIN_CURSOR = align256(OFF_BIN_COUNT + sizeof(uint32_t) * NBINS);
constexpr size_t OFF_TOPK = align256(OFF_BIN_CURSOR + sizeof(uint32_t) * NBINS);
constexpr size_t OFF_CAND_KEY = align256(OFF_TOPK + sizeof(unsigned long long) * MAX_K);
constexpr size_t OFF_CAND_POS = align256(OFF_CAND_KEY + sizeof(unsigned long long) * MAX_CAND);
constexpr size_t OFF_CTL = align256(OFF_CAND_POS + sizeof(uint32_t) * MAX_CAND);
constexpr size_t OFF_OUT_IDX = align256(OFF_CTL + sizeof(QCtl));
constexpr size_t OFF_OUT_DIST = align256(OFF_OUT_IDX + sizeof(int64_t) * MAX_K);
constexpr size_t OFF_SURV = align256(OFF_OUT_DIST + sizeof(float) * MAX_K);
constexpr size_t TOTAL = align256(OFF_SURV + sizeof(uint2) * MAX_SURV);
static_assert(TOTAL == ISAX_NOALLOC_SCRATCH_BYTES, "scratch size must match isax.h");

static __device__ __align__(256) unsigned char g_scratch[TOTAL];

std::mutex g_mu;                 // one call at a time in this process
void* g_addr[64] = {};           // device address of g_scratch, per device

// device address of the array on the current device (looked up once)
unsigned char* scratch_on(int dev) {
    if (dev < 0 || dev >= 64) throw Error{ISAX_ERR_INVALID_ARG, "device ordinal out of range"};
    if (!g_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            throw Error{ISAX_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") +
                                           cudaGetErrorString(e)};
        g_addr[dev] = p;
    }
    return static_cast<unsigned char*>(g_addr[dev]);
}

QueryScratch scratch_view(unsigned char* base) {
    QueryScratch s{};
    s.q = reinterpret_cast<float*>(base + OFF_Q);
    s.table = reinterpret_cast<float*>(base + OFF_TABLE);
    s.leaf_lb = reinterpret_cast<float*>(base + OFF_LEAF_LB);
    s.work = reinterpret_cast<uint2*>(base + OFF_WORK);
    s.work_cap = MAX_WORK;
    s.bin_count = reinterpret_cast<uint32_t*>(base + OFF_BIN_COUNT);
    s.bin_cursor = reinterpret_cast<uint32_t*>(base + OFF_BIN_CURSOR);
    s.topk = reinterpret_cast<unsigned long long*>(base + OFF_TOPK);
    s.cand_key = reinterpret_cast<unsigned long long*>(base + OFF_CAND_KEY);
    s.cand_pos = reinterpret_cast<uint32_t*>(base + OFF_CAND_POS);
    s.cand_cap = MAX_CAND;
    s.ctl = reinterpret_cast<QCtl*>(base + OFF_CTL);
    s.out_idx = reinterpret_cast<int64_t*>(base + OFF_OUT_IDX);
    s.out_dist = reinterpret_cast<float*>(base + OFF_OUT_DIST);
    s.surv = reinterpret_cast<uint2*>(base + OFF_SURV);
    s.surv_cap = MAX_SURV;
    return s;
}

void fail(isax_status st, const std::string& msg) { throw Error{st, msg}; }

}  // namespace
}  // namespace noalloc
}  // namespace isax

using namespace isax;

extern "C" isax_status isax_query_knn_noalloc(const isax_index* cix, const float* q, int32_t k,
                                              uint32_t mem_flags, int64_t* out_idx,
                                              float* out_dist, isax_query_stats* stats,
                                              void* cuda_stream) {
    set_error(ISAX_OK, "");
    int prev = -1;
    bool switched = false;
    try {
        using namespace noalloc;
        if (!cix) fail(ISAX_ERR_INVALID_ARG, "index is NULL");
        if (!q || !out_idx || !out_dist) fail(ISAX_ERR_INVALID_ARG, "NULL query or output");
        if (mem_flags & ~(uint32_t)(ISAX_MEM_INPUT_DEVICE | ISAX_MEM_OUTPUT_DEVICE))
            fail(ISAX_ERR_INVALID_ARG, "unknown mem_flags bits");
        if (k < 1 || k > ISAX_MAX_K || (int64_t)k > cix->d.N)
            fail(ISAX_ERR_INVALID_ARG, "k must be in [1, min(N, 1024)]");
        if (cix->d.L > (int64_t)MAX_LEAVES || work_items_cap(cix->d.L, cix->d.N) > (int64_t)MAX_WORK)
            fail(ISAX_ERR_INVALID_ARG,
                 "index has " + std::to_string(cix->d.L) + " leaves and " + std::to_string(cix->d.N) +
                 " series; the allocation-free query supports at most " + std::to_string(MAX_LEAVES) +
                 " leaves and leaves + series / 128 <= " + std::to_string(MAX_WORK) +
                 " (use isax_query_knn)");
        isax_index* ix = const_cast<isax_index*>(cix);
        std::lock_guard<std::mutex> lk(g_mu);
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != ix->device) {
            ISAX_CUDA_TRY(cudaSetDevice(ix->device));
            switched = true;
        }
        cudaStream_t st = (cudaStream_t)cuda_stream;
        const QueryScratch s = scratch_view(scratch_on(ix->device));
        const int n = ix->d.n;
        ISAX_CUDA_TRY(cudaMemsetAsync(s.ctl, 0, sizeof(QCtl), st));
        ISAX_CUDA_TRY(cudaMemsetAsync(s.topk, 0xFF, sizeof(unsigned long long) * MAX_K, st));
        const cudaMemcpyKind kin = (mem_flags & ISAX_MEM_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                       : cudaMemcpyHostToDevice;
        ISAX_CUDA_TRY(cudaMemcpyAsync(s.q, q, sizeof(float) * n, kin, st));
        launch_query_on_scratch(ix, s, k, st);
        QCtl c;
        ISAX_CUDA_TRY(cudaMemcpyAsync(&c, s.ctl, sizeof(QCtl), cudaMemcpyDeviceToHost, st));
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
        c.flags |= injected_query_flags();
        if (c.flags & QF_NONFINITE) fail(ISAX_ERR_INVALID_ARG, "query contains a non-finite value");
        if (c.flags & QF_STALLED) {
            empty_survivors(s, st);
            ISAX_CUDA_TRY(cudaStreamSynchronize(st));
            fail(ISAX_ERR_TIMEOUT, "a bounded wait of the query gave up");
        }
        if (c.flags & QF_OVERFLOW)
            fail(ISAX_ERR_OOM, c.surv_count > MAX_SURV
                 ? "more than " + std::to_string(MAX_SURV) + " series passed the lower bound: the "
                   "allocation-free scratch is too small for this query (use isax_query_knn)"
                 : "the query kept more than " + std::to_string(MAX_CAND) +
                   " candidates for its final FP64 ordering: the allocation-free scratch is too "
                   "small for this query (use isax_query_knn)");
        if (c.flags & QF_SHORT) fail(ISAX_ERR_INTERNAL, "fewer than k candidates survived");
        const cudaMemcpyKind kout = (mem_flags & ISAX_MEM_OUTPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                         : cudaMemcpyDeviceToHost;
        ISAX_CUDA_TRY(cudaMemcpyAsync(out_idx, s.out_idx, sizeof(int64_t) * k, kout, st));
        ISAX_CUDA_TRY(cudaMemcpyAsync(out_dist, s.out_dist, sizeof(float) * k, kout, st));
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
        if (stats) {
            stats->leaves_total = ix->d.L;
            stats->leaves_queued = (int64_t)c.leaves_queued;
            stats->leaves_scanned = (int64_t)c.leaves_scanned;
            stats->series_lb = (int64_t)c.series_lb;
            stats->series_refined = (int64_t)c.refined_total;
            stats->approx_series = (int64_t)c.approx_series;
            stats->candidates = (int64_t)c.cand_total;
            stats->window = (int64_t)c.window;
            stats->approx_leaf = c.approx_leaf;
            stats->reruns = 0;
            stats->ed_floats = (int64_t)c.ed_floats;
        }
        if (switched) cudaSetDevice(prev);
        return ISAX_OK;
    } catch (const Error& e) {
        if (switched) cudaSetDevice(prev);
        set_error(e.st, e.msg);
        return e.st;
    } catch (...) {
        if (switched) cudaSetDevice(prev);
        set_error(ISAX_ERR_INTERNAL, "unexpected exception");
        return ISAX_ERR_INTERNAL;
    }
}
