// isax_api.cu - the C ABI: argument validation, error reporting, device
// selection, allocator hooks.  Every compute step runs in the kernels of
// isax_build.cu and isax_query.cu.
#include <math.h>
#include <string.h>

#include <mutex>
#include <string>

#include "isax_common.cuh"
#include "isax_tc.cuh"

namespace isax {

static thread_local std::string g_last_error;

void set_error(isax_status st, const std::string& msg) {
    (void)st;
    g_last_error = msg;
}

// ---------------------------------------------------------------- allocator
static isax_alloc_fn g_alloc = nullptr;
static isax_free_fn g_free = nullptr;
static void* g_ctx = nullptr;
static std::mutex g_pool_mu;
static bool g_pool_ready[64] = {};

// default: the device's default stream-ordered memory pool, told to keep
// freed memory (repeated builds then reuse it instead of remapping)
static void prepare_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64 || g_pool_ready[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_ready[dev] = true;
}

void* dev_alloc(size_t bytes, cudaStream_t st) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (g_alloc) {
        p = g_alloc(bytes, st, g_ctx);
        if (!p) throw Error{ISAX_ERR_OOM, "allocator hook returned NULL for " + std::to_string(bytes) + " bytes"};
        return p;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    prepare_pool(dev);
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        throw Error{ISAX_ERR_OOM, "cudaMallocAsync(" + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e)};
    }
    return p;
}

void trim_pool(int dev) {
    cudaMemPool_t pool;
    ISAX_CUDA_TRY(cudaDeviceGetDefaultMemPool(&pool, dev));
    ISAX_CUDA_TRY(cudaMemPoolTrimTo(pool, 0));
}

void dev_free(void* p, cudaStream_t st) {
    if (!p) return;
    if (g_free) {
        g_free(p, st, g_ctx);
        return;
    }
    cudaFreeAsync(p, st);
}

// ---------------------------------------------------------------- helpers
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) ISAX_CUDA_TRY(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <typename F>
static isax_status guarded(F&& f) {
    g_last_error.clear();
    try {
        f();
        return ISAX_OK;
    } catch (const Error& e) {
        g_last_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return ISAX_ERR_OOM;
    } catch (...) {
        g_last_error = "unexpected exception";
        return ISAX_ERR_INTERNAL;
    }
}

static void check(bool ok, const std::string& msg) {
    if (!ok) throw Error{ISAX_ERR_INVALID_ARG, msg};
}

static void check_series_shape(int64_t N, int32_t n) {
    check(N >= 1, "N must be >= 1");
    check(N <= (int64_t)0xfffffffeLL, "N must be < 2^32 - 1");
    check(n >= ISAX_W && n <= ISAX_MAX_LEN && n % ISAX_W == 0,
          "n must be a multiple of 16 in [16, 4096]");
}

static void check_card(int32_t card) {
    check(card >= 2 && card <= 256 && (card & (card - 1)) == 0,
          "cardinality must be a power of two in [2, 256]");
}

static void fill_stats(isax_query_stats* st, const isax_index* ix, const QCtl& c, int reruns) {
    if (!st) return;
    st->leaves_total = ix->d.L;
    st->leaves_queued = (int64_t)c.leaves_queued;
    st->leaves_scanned = (int64_t)c.leaves_scanned;
    st->series_lb = (int64_t)c.series_lb;
    st->series_refined = (int64_t)c.refined_total;
    st->approx_series = (int64_t)c.approx_series;
    st->candidates = (int64_t)c.cand_total;
    st->window = (int64_t)c.window;
    st->approx_leaf = c.approx_leaf;
    st->reruns = reruns;
    st->ed_floats = (int64_t)c.ed_floats;
}

// one query read from q_src (a device address); the results go to the caller's
// outputs
static void run_one(isax_index* ix, const float* q_src, int32_t k, uint32_t mem_flags, int64_t* out_idx,
                    float* out_dist, isax_query_stats* stats, cudaStream_t st, int mode = QUERY_MESSI) {
    QCtl c;
    int reruns = 0;
    query_device(ix, k, &c, &reruns, st, mode, out_idx, out_dist, (mem_flags & ISAX_MEM_OUTPUT_DEVICE) != 0,
                 q_src);
    fill_stats(stats, ix, c, reruns);
}

}  // namespace isax

using namespace isax;

static isax_status query_knn_mode(const isax_index* cix, const float* q, int32_t k, uint32_t mem_flags,
                           int64_t* out_idx, float* out_dist, isax_query_stats* stats,
                           void* cuda_stream, int mode) {
    return guarded([&] {
        check(cix != nullptr, "index is NULL");
        check(q != nullptr && out_idx != nullptr && out_dist != nullptr, "NULL query or output");
        check((mem_flags & ~(uint32_t)(ISAX_MEM_INPUT_DEVICE | ISAX_MEM_OUTPUT_DEVICE)) == 0,
              "unknown mem_flags bits");
        check(k >= 1 && k <= ISAX_MAX_K && (int64_t)k <= cix->d.N, "k must be in [1, min(N, 1024)]");
        isax_index* ix = const_cast<isax_index*>(cix);
        DeviceGuard dg(ix->device);
        std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(ix->mu));
        cudaStream_t st = (cudaStream_t)cuda_stream;
        // the query's first kernel reads a device query where it is; a host
        // query is first placed in the index's mapped block
        const float* q_src = q;
        if (!(mem_flags & ISAX_MEM_INPUT_DEVICE)) {
            ensure_query_mail(ix);
            memcpy(ix->mail->q, q, sizeof(float) * ix->d.n);
            q_src = ix->mail_dev->q;
        }
        run_one(ix, q_src, k, mem_flags, out_idx, out_dist, stats, st, mode);
    });
}

extern "C" {

isax_status isax_set_allocator(isax_alloc_fn alloc_fn, isax_free_fn free_fn, void* ctx) {
    return guarded([&] {
        check((alloc_fn == nullptr) == (free_fn == nullptr), "set both hooks or neither");
        g_alloc = alloc_fn;
        g_free = free_fn;
        g_ctx = ctx;
    });
}

isax_status isax_build_index(const float* series, int64_t N, int32_t n, const isax_build_params* p,
                             void* cuda_stream, isax_index** out) {
    return guarded([&] {
        check(out != nullptr, "out is NULL");
        *out = nullptr;
        isax_build_params prm = {ISAX_W, 256, 2000, 0u};
        if (p) prm = *p;
        check(series != nullptr, "series is NULL");
        check_series_shape(N, n);
        check(prm.w == ISAX_W, "w must be 16");
        check_card(prm.cardinality);
        check(prm.leaf_size >= 1, "leaf_size must be >= 1");
        check((prm.mem_flags & ~(uint32_t)(ISAX_MEM_INPUT_DEVICE | ISAX_BUILD_ROWS_HOST |
                                           ISAX_BUILD_ROWS_IN_PLACE | ISAX_BUILD_SPLIT_BALANCED)) == 0,
              "unknown mem_flags bits");
        check(!(prm.mem_flags & ISAX_BUILD_ROWS_IN_PLACE) || (prm.mem_flags & ISAX_MEM_INPUT_DEVICE),
              "ISAX_BUILD_ROWS_IN_PLACE needs device-resident series (ISAX_MEM_INPUT_DEVICE)");
        check(!((prm.mem_flags & ISAX_BUILD_ROWS_IN_PLACE) && (prm.mem_flags & ISAX_BUILD_ROWS_HOST)),
              "ISAX_BUILD_ROWS_IN_PLACE and ISAX_BUILD_ROWS_HOST exclude each other");
        check(aligned16(series), "series must be 16-byte aligned");
        cudaStream_t st = (cudaStream_t)cuda_stream;
        *out = build_index_impl(series, N, n, prm.cardinality, prm.leaf_size, prm.mem_flags, st);
    });
}

isax_status isax_query_knn(const isax_index* cix, const float* q, int32_t k, uint32_t mem_flags,
                           int64_t* out_idx, float* out_dist, isax_query_stats* stats,
                           void* cuda_stream) {
    return query_knn_mode(cix, q, k, mem_flags, out_idx, out_dist, stats, cuda_stream, QUERY_MESSI);
}

isax_status isax_query_knn_flat(const isax_index* cix, const float* q, int32_t k, uint32_t mem_flags,
                                int64_t* out_idx, float* out_dist, isax_query_stats* stats,
                                void* cuda_stream) {
    return query_knn_mode(cix, q, k, mem_flags, out_idx, out_dist, stats, cuda_stream, QUERY_FLAT);
}

isax_status isax_query_knn_batch(const isax_index* cix, const float* Q, int32_t B, int32_t k,
                                 uint32_t mem_flags, int64_t* out_idx, float* out_dist,
                                 isax_query_stats* stats, void* cuda_stream) {
    return guarded([&] {
        check(cix != nullptr, "index is NULL");
        check(B >= 0, "B must be >= 0");
        check(B == 0 || (Q != nullptr && out_idx != nullptr && out_dist != nullptr),
              "NULL queries or outputs");
        check((mem_flags & ~(uint32_t)(ISAX_MEM_INPUT_DEVICE | ISAX_MEM_OUTPUT_DEVICE)) == 0,
              "unknown mem_flags bits");
        check(k >= 1 && k <= ISAX_MAX_K && (int64_t)k <= cix->d.N, "k must be in [1, min(N, 1024)]");
        isax_index* ix = const_cast<isax_index*>(cix);
        DeviceGuard dg(ix->device);
        std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(ix->mu));
        cudaStream_t st = (cudaStream_t)cuda_stream;
        const int n = ix->d.n;
        const cudaMemcpyKind kin = (mem_flags & ISAX_MEM_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                       : cudaMemcpyHostToDevice;
        if (B == 0) return;
        (void)n;
        (void)kin;
        struct Ctx {
            const isax_index* ix;
            isax_query_stats* stats;
        } ctx{ix, stats};
        auto fill = [](void* p, int b, const QCtl& c, int reruns) {
            Ctx* cx = static_cast<Ctx*>(p);
            if (cx->stats) fill_stats(cx->stats + b, cx->ix, c, reruns);
        };
        query_batch_device(ix, Q, B, k, mem_flags, out_idx, out_dist, fill, &ctx, st);
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    });
}

void isax_free_index(isax_index* ix) {
    if (!ix) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ix->device);
    cudaDeviceSynchronize();
    free_index_arrays(ix, 0);
    cudaDeviceSynchronize();
    delete static_cast<std::mutex*>(ix->mu);
    delete ix;
    if (prev >= 0) cudaSetDevice(prev);
}

const char* isax_last_error(void) { return g_last_error.c_str(); }

isax_status isax_get_index_info(const isax_index* ix, isax_index_info* info) {
    return guarded([&] {
        check(ix != nullptr && info != nullptr, "NULL argument");
        info->N = ix->d.N;
        info->n = ix->d.n;
        info->w = ISAX_W;
        info->cardinality = ix->d.card;
        info->leaf_size = ix->d.leaf_size;
        info->leaves = ix->d.L;
        info->max_leaf = ix->max_leaf;
        info->device = ix->device;
        info->device_bytes = ix->bytes;
        info->maxabs = ix->d.maxabs;
    });
}

isax_status isax_trim_memory(int32_t device) {
    return guarded([&] {
        int count = 0;
        ISAX_CUDA_TRY(cudaGetDeviceCount(&count));
        check(device >= 0 && device < count, "device ordinal out of range");
        DeviceGuard dg(device);
        ISAX_CUDA_TRY(cudaDeviceSynchronize());
        trim_pool(device);
    });
}

isax_status isax_index_export(const isax_index* ix, uint8_t* sax, uint32_t* orig_id,
                              uint32_t* leaf_begin, uint8_t* envelope, float* breakpoints) {
    return guarded([&] {
        check(ix != nullptr, "index is NULL");
        DeviceGuard dg(ix->device);
        const DevIndex& d = ix->d;
        if (sax) ISAX_CUDA_TRY(cudaMemcpy(sax, d.sax, (size_t)d.N * 16, cudaMemcpyDeviceToHost));
        if (orig_id)
            ISAX_CUDA_TRY(cudaMemcpy(orig_id, d.orig, (size_t)d.N * 4, cudaMemcpyDeviceToHost));
        if (leaf_begin)
            ISAX_CUDA_TRY(cudaMemcpy(leaf_begin, d.leaf_begin, ((size_t)d.L + 1) * 4, cudaMemcpyDeviceToHost));
        if (envelope)
            ISAX_CUDA_TRY(cudaMemcpy(envelope, d.env, (size_t)d.L * 32, cudaMemcpyDeviceToHost));
        if (breakpoints)
            ISAX_CUDA_TRY(cudaMemcpy(breakpoints, d.bp + 1, (size_t)(d.card - 1) * 4, cudaMemcpyDeviceToHost));
    });
}

isax_status isax_summarize(const float* series, int64_t N, int32_t n, int32_t cardinality,
                           uint32_t mem_flags, uint8_t* out_sax, float* out_paa, void* cuda_stream) {
    return guarded([&] {
        check(series != nullptr, "series is NULL");
        check_series_shape(N, n);
        check_card(cardinality);
        check((mem_flags & ~(uint32_t)(ISAX_MEM_INPUT_DEVICE | ISAX_MEM_OUTPUT_DEVICE)) == 0,
              "unknown mem_flags bits");
        check(aligned16(series), "series must be 16-byte aligned");
        check(!(mem_flags & ISAX_MEM_OUTPUT_DEVICE) || !out_sax || aligned16(out_sax),
              "device out_sax must be 16-byte aligned");
        summarize_impl(series, N, n, cardinality, mem_flags, out_sax, out_paa, (cudaStream_t)cuda_stream);
    });
}

isax_status isax_prepare_bf16(isax_index* ix, void* cuda_stream) {
    return guarded([&] {
        check(ix != nullptr, "index is NULL");
        DeviceGuard dg(ix->device);
        std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(ix->mu));
        cudaStream_t st = (cudaStream_t)cuda_stream;
        prepare_tc(ix, st);
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    });
}

isax_status isax_query_knn_batch_bf16(const isax_index* cix, const float* Q, int32_t B, int32_t k,
                                      uint32_t mem_flags, int64_t* out_idx, float* out_dist,
                                      isax_query_stats* stats, void* cuda_stream) {
    return guarded([&] {
        check(cix != nullptr, "index is NULL");
        check(B >= 0, "B must be >= 0");
        check(B == 0 || (Q != nullptr && out_idx != nullptr && out_dist != nullptr),
              "NULL queries or outputs");
        check((mem_flags & ~(uint32_t)(ISAX_MEM_INPUT_DEVICE | ISAX_MEM_OUTPUT_DEVICE)) == 0,
              "unknown mem_flags bits");
        check(k >= 1 && k <= ISAX_MAX_K && (int64_t)k <= cix->d.N, "k must be in [1, min(N, 1024)]");
        check(cix->d.n % 64 == 0 && cix->d.n <= 2048,
              "the BF16 filter needs n to be a multiple of 64 and at most 2048");
        check(!(mem_flags & ISAX_MEM_INPUT_DEVICE) || aligned16(Q), "device queries must be 16-byte aligned");
        isax_index* ix = const_cast<isax_index*>(cix);
        DeviceGuard dg(ix->device);
        std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(ix->mu));
        cudaStream_t st = (cudaStream_t)cuda_stream;
        if (B == 0) return;
        struct Ctx {
            const isax_index* ix;
            isax_query_stats* stats;
        } ctx{ix, stats};
        auto fill = [](void* p, int b, const QCtl& c, int reruns) {
            Ctx* cx = static_cast<Ctx*>(p);
            if (cx->stats) fill_stats(cx->stats + b, cx->ix, c, reruns);
        };
        query_batch_tc(ix, Q, B, k, mem_flags, out_idx, out_dist, fill, &ctx, st);
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    });
}

int32_t isax_checks_enabled(void) {
#ifdef ISAX_CHECKS
    return 1;
#else
    return 0;
#endif
}

isax_status isax_check_word(uint32_t* out) {
    return guarded([&] {
        check(out != nullptr, "out is NULL");
        *out = take_check_word_build() | take_check_word_query();
    });
}

isax_status isax_exact_d2(const isax_index* cix, const float* Q, int32_t B, int32_t k, uint32_t mem_flags,
                          const int64_t* idx, double* out_d2, void* cuda_stream) {
    return guarded([&] {
        check(cix != nullptr, "index is NULL");
        check(B >= 0 && k >= 1 && k <= ISAX_MAX_K, "B must be >= 0 and k in [1, 1024]");
        check(B == 0 || (Q != nullptr && idx != nullptr && out_d2 != nullptr), "NULL queries, rows or output");
        check((mem_flags & ~(uint32_t)(ISAX_MEM_INPUT_DEVICE | ISAX_MEM_OUTPUT_DEVICE)) == 0,
              "unknown mem_flags bits");
        if (B == 0) return;
        isax_index* ix = const_cast<isax_index*>(cix);
        DeviceGuard dg(ix->device);
        std::lock_guard<std::mutex> lk(*static_cast<std::mutex*>(ix->mu));
        cudaStream_t st = (cudaStream_t)cuda_stream;
        const size_t qb = sizeof(float) * (size_t)B * ix->d.n, ib = sizeof(int64_t) * (size_t)B * k,
                     ob = sizeof(double) * (size_t)B * k;
        const bool in_dev = (mem_flags & ISAX_MEM_INPUT_DEVICE) != 0, out_dev = (mem_flags & ISAX_MEM_OUTPUT_DEVICE) != 0;
        // host inputs and outputs go through device staging
        struct Tmp {
            void* p = nullptr;
            cudaStream_t st;
            ~Tmp() { if (p) dev_free(p, st); }
        } tq{nullptr, st}, ti{nullptr, st}, to{nullptr, st};
        const float* dq = Q;
        const int64_t* di = idx;
        double* dout = out_d2;
        if (!in_dev) {
            tq.p = dev_alloc(qb, st);
            ti.p = dev_alloc(ib, st);
            ISAX_CUDA_TRY(cudaMemcpyAsync(tq.p, Q, qb, cudaMemcpyHostToDevice, st));
            ISAX_CUDA_TRY(cudaMemcpyAsync(ti.p, idx, ib, cudaMemcpyHostToDevice, st));
            dq = static_cast<const float*>(tq.p);
            di = static_cast<const int64_t*>(ti.p);
        }
        if (!out_dev) {
            to.p = dev_alloc(ob, st);
            dout = static_cast<double*>(to.p);
        }
        exact_d2_device(ix, dq, B, k, di, dout, st);
        if (!out_dev) ISAX_CUDA_TRY(cudaMemcpyAsync(out_d2, dout, ob, cudaMemcpyDeviceToHost, st));
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    });
}

isax_status isax_tc_selftest(const uint16_t* a, const uint16_t* b, int32_t n_cols, float* d,
                             void* cuda_stream) {
    return guarded([&] {
        check(a && b && d, "NULL pointer");
        check(n_cols >= 16 && n_cols <= 256 && n_cols % 16 == 0,
              "n_cols must be a multiple of 16 in [16, 256]");
        check(aligned16(a) && aligned16(b), "a and b must be 16-byte aligned");
        tc_selftest(a, b, n_cols, d, (cudaStream_t)cuda_stream);
    });
}

}  // extern "C"
