// isax_serve.cu - a resident query server: several indexes stay in device
// memory and exact k-NN requests for any of them are admitted, as they arrive,
// into a fixed set of in-flight slots (continuous batching: a request never
// waits for a batch to form or to drain, only for a free slot and for
// candidate-buffer memory).  Each slot owns device scratch sized for the
// largest index, a stream, pinned staging buffers and the captured query
// graphs of every (index, k) it has served; its per-query state (the k best,
// the candidate window, the control block) stays on the device.  A host thread
// runs the loop: admit queued requests FIFO while a slot is free and the
// request's candidate buffer fits the memory budget, poll the slots' completion
// events, rerun a query whose candidate buffer overflowed with a buffer four
// times larger (once the budget allows), and publish results.  Every query runs
// the single-query kernels (Section III, MESSI query answering), so its answer
// does not depend on what else is in flight.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "isax_common.cuh"

namespace isax {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// candidate entries reserved for a k-NN request (12 bytes each; a query that
// keeps more reruns with four times the room): the approximate answer's rows,
// which all take a slot, and room for the refined rows near the k-th best
static uint32_t serve_cand_cap(int k, int leaf_size) {
    return approx_rows_max(leaf_size, k) + 4096u + 256u * (uint32_t)k;
}

struct ServeRequest {
    uint64_t tag = 0;
    int32_t coll = 0;
    int32_t k = 1;
    double t_submit = 0;
    std::vector<float> q;
};

struct ServeResult {
    uint64_t tag = 0;
    int32_t coll = 0, k = 0, status = 0, reruns = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    QCtl ctl{};
    std::vector<int64_t> idx;
    std::vector<float> dist;
};

struct ServeSlot {
    QueryScratch qs{};
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    float* h_q = nullptr;       // pinned staging
    QCtl* h_ctl = nullptr;
    int64_t* h_idx = nullptr;
    float* h_dist = nullptr;
    std::map<const isax_index*, void*> graphs;
    bool busy = false;
    bool wants_room = false;    // overflowed; waiting for budget to rerun
    ServeRequest req;
    size_t reserved = 0;        // budget bytes held by the current request
    uint32_t need_cap = 0;
    uint32_t need_surv = 0;     // survivor entries needed after a survivor overflow
    double t_start = 0;
    int reruns = 0;
};

}  // namespace isax

struct isax_server {
    int device = 0;
    int nslots = 16;
    size_t budget = 256ull << 20;
    std::vector<isax_index*> colls;
    std::vector<isax::ServeSlot*> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<isax::ServeRequest> pending;
    std::deque<isax::ServeResult> done;
    std::thread loop;
    bool started = false;
    bool stop = false;
    size_t reserved = 0;
    uint64_t submitted = 0, completed = 0;
    int in_flight = 0, max_in_flight = 0;
    std::string error;
};

namespace isax {

static void slot_free(ServeSlot* sl) {
    if (sl->st) cudaStreamSynchronize(sl->st);
    for (auto& kv : sl->graphs) query_graphs_delete(kv.second);
    sl->graphs.clear();
    free_query_scratch_struct(sl->qs, sl->st);
    if (sl->st) cudaStreamSynchronize(sl->st);
    if (sl->h_q) cudaFreeHost(sl->h_q);
    if (sl->h_ctl) cudaFreeHost(sl->h_ctl);
    if (sl->h_idx) cudaFreeHost(sl->h_idx);
    if (sl->h_dist) cudaFreeHost(sl->h_dist);
    if (sl->done) cudaEventDestroy(sl->done);
    if (sl->st) cudaStreamDestroy(sl->st);
    delete sl;
}

static void server_setup(isax_server* s) {
    int64_t L = 1, Nmax = 1;
    int n = 16, card = 2, leaf = 1;
    for (isax_index* ix : s->colls) {
        L = std::max<int64_t>(L, ix->d.L);
        leaf = std::max(leaf, (int)ix->d.leaf_size);
        Nmax = std::max<int64_t>(Nmax, ix->d.N);
        n = std::max(n, (int)ix->d.n);
        card = std::max(card, (int)ix->d.card);
    }
    // all slots or none: a failure frees the slots made so far
    try {
        for (int i = 0; i < s->nslots; ++i) {
            ServeSlot* sl = new ServeSlot();
            s->slots.push_back(sl);
            ISAX_CUDA_TRY(cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking));
            ISAX_CUDA_TRY(cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming));
            alloc_query_scratch_for(L, Nmax, n, card, serve_cand_cap(1, leaf), default_surv_cap(Nmax), sl->qs,
                                    sl->st);
            ISAX_CUDA_TRY(cudaMallocHost((void**)&sl->h_q, sizeof(float) * n));
            ISAX_CUDA_TRY(cudaMallocHost((void**)&sl->h_ctl, sizeof(QCtl)));
            ISAX_CUDA_TRY(cudaMallocHost((void**)&sl->h_idx, sizeof(int64_t) * MAX_K));
            ISAX_CUDA_TRY(cudaMallocHost((void**)&sl->h_dist, sizeof(float) * MAX_K));
            ISAX_CUDA_TRY(cudaStreamSynchronize(sl->st));
        }
    } catch (...) {
        for (ServeSlot* sl : s->slots) slot_free(sl);
        s->slots.clear();
        throw;
    }
}

// The scan of a served query runs on num_sms / SERVE_SCAN_SHARE CTAs, so the
// scans of requests in flight on other slots can run beside it.
constexpr int SERVE_SCAN_SHARE = 2;

// the query's kernels, then its control block and answer copied to the slot's
// pinned staging, then the completion event
static void slot_launch(isax_server* s, ServeSlot* sl) {
    isax_index* ix = s->colls[sl->req.coll];
    if (sl->qs.cand_cap < sl->need_cap || sl->qs.surv_cap < sl->need_surv) {
        for (auto& kv : sl->graphs) query_graphs_clear(kv.second);  // they hold the old buffers
        if (sl->qs.cand_cap < sl->need_cap) grow_query_candidates(sl->qs, sl->need_cap, sl->st);
        if (sl->qs.surv_cap < sl->need_surv) grow_query_survivors(sl->qs, sl->need_surv, sl->st);
    }
    void*& g = sl->graphs[ix];
    if (!g) g = query_graphs_new();
    launch_query_graph_ext(ix, sl->qs, g, sl->req.k, sl->st, SERVE_SCAN_SHARE);
    ISAX_CUDA_TRY(cudaMemcpyAsync(sl->h_ctl, sl->qs.ctl, sizeof(QCtl), cudaMemcpyDeviceToHost, sl->st));
    ISAX_CUDA_TRY(cudaMemcpyAsync(sl->h_idx, sl->qs.out_idx, sizeof(int64_t) * sl->req.k,
                                  cudaMemcpyDeviceToHost, sl->st));
    ISAX_CUDA_TRY(cudaMemcpyAsync(sl->h_dist, sl->qs.out_dist, sizeof(float) * sl->req.k,
                                  cudaMemcpyDeviceToHost, sl->st));
    ISAX_CUDA_TRY(cudaEventRecord(sl->done, sl->st));
}

static void slot_start(isax_server* s, ServeSlot* sl, ServeRequest&& r, size_t bytes) {
    sl->req = std::move(r);
    sl->reserved = bytes;
    sl->need_cap = serve_cand_cap(sl->req.k, s->colls[sl->req.coll]->d.leaf_size);
    sl->need_surv = 0;
    sl->reruns = 0;
    sl->wants_room = false;
    sl->busy = true;
    sl->t_start = now_s();
    isax_index* ix = s->colls[sl->req.coll];
    memcpy(sl->h_q, sl->req.q.data(), sizeof(float) * ix->d.n);
    ISAX_CUDA_TRY(cudaMemcpyAsync(sl->qs.q, sl->h_q, sizeof(float) * ix->d.n, cudaMemcpyHostToDevice, sl->st));
    slot_launch(s, sl);
}

static void publish(isax_server* s, ServeSlot* sl, int status) {
    ServeResult res;
    res.tag = sl->req.tag;
    res.coll = sl->req.coll;
    res.k = sl->req.k;
    res.status = status;
    res.reruns = sl->reruns;
    res.t_submit = sl->req.t_submit;
    res.t_start = sl->t_start;
    res.t_done = now_s();
    res.ctl = *sl->h_ctl;
    if (status == ISAX_OK) {
        res.idx.assign(sl->h_idx, sl->h_idx + sl->req.k);
        res.dist.assign(sl->h_dist, sl->h_dist + sl->req.k);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->done.push_back(std::move(res));
    s->reserved -= sl->reserved;
    s->in_flight -= 1;
    s->completed += 1;
    sl->busy = false;
    sl->reserved = 0;
    s->cv_done.notify_all();
}

static void server_loop(isax_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        bool progress = false;
        // completions
        for (ServeSlot* sl : s->slots) {
            if (!sl->busy) continue;
            if (sl->wants_room) {
                // an overflowed query: rerun once its larger buffer fits the budget
                const size_t extra = ((size_t)sl->need_cap - sl->reserved / 12) * 12;
                bool ok = false;
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    if (s->reserved + extra <= s->budget || s->in_flight == 1) {
                        s->reserved += extra;
                        ok = true;
                    }
                }
                if (ok) {
                    sl->reserved += extra;
                    sl->wants_room = false;
                    sl->reruns += 1;
                    try {
                        slot_launch(s, sl);
                    } catch (const Error& err) {
                        {
                            std::lock_guard<std::mutex> lk(s->mu);
                            s->error = err.msg;
                        }
                        publish(s, sl, err.st);
                    }
                    progress = true;
                }
                continue;
            }
            const cudaError_t e = cudaEventQuery(sl->done);
            if (e == cudaErrorNotReady) continue;
            progress = true;
            if (e != cudaSuccess) {
                cudaGetLastError();
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->error = cudaGetErrorString(e);
                }
                publish(s, sl, ISAX_ERR_CUDA);
                continue;
            }
            QCtl& c = *sl->h_ctl;
            c.flags |= injected_query_flags();
            if (c.flags & QF_NONFINITE) {
                publish(s, sl, ISAX_ERR_INVALID_ARG);
            } else if (c.flags & QF_STALLED) {
                empty_survivors(sl->qs, sl->st);
                publish(s, sl, ISAX_ERR_TIMEOUT);
            } else if ((c.flags & QF_OVERFLOW) && sl->reruns < 4) {
                const uint64_t N = (uint64_t)s->colls[sl->req.coll]->d.N;
                if (c.cand_total > sl->qs.cand_cap) {
                    const uint64_t want = std::max<uint64_t>((uint64_t)c.cand_total * 2, (uint64_t)sl->need_cap * 4);
                    sl->need_cap = (uint32_t)std::min<uint64_t>(want, N + 16);
                }
                if (c.surv_count > sl->qs.surv_cap)
                    sl->need_surv = (uint32_t)std::min<uint64_t>(
                        std::max<uint64_t>((uint64_t)c.surv_count * 2, (uint64_t)sl->qs.surv_cap * 4), N + 16);
                sl->wants_room = true;
            } else if (c.flags & (QF_OVERFLOW | QF_SHORT)) {
                publish(s, sl, ISAX_ERR_INTERNAL);
            } else {
                publish(s, sl, ISAX_OK);
            }
        }
        // admission: FIFO, a free slot and room in the candidate budget
        for (;;) {
            ServeSlot* free_slot = nullptr;
            for (ServeSlot* sl : s->slots)
                if (!sl->busy) {
                    free_slot = sl;
                    break;
                }
            if (!free_slot) break;
            ServeRequest r;
            size_t bytes = 0;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->pending.empty()) break;
                bytes = (size_t)serve_cand_cap(s->pending.front().k,
                                               s->colls[s->pending.front().coll]->d.leaf_size) * 12;
                if (s->reserved + bytes > s->budget && s->in_flight > 0) break;
                r = std::move(s->pending.front());
                s->pending.pop_front();
                s->reserved += bytes;
                s->in_flight += 1;
                s->max_in_flight = std::max(s->max_in_flight, s->in_flight);
            }
            try {
                slot_start(s, free_slot, std::move(r), bytes);
            } catch (const Error& err) {
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->error = err.msg;
                }
                *free_slot->h_ctl = QCtl{};
                publish(s, free_slot, err.st);
            }
            progress = true;
        }
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop && s->pending.empty() && s->in_flight == 0) break;
            if (!progress) {
                if (s->in_flight == 0)
                    s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
                else
                    s->cv_work.wait_for(lk, std::chrono::microseconds(20));
            }
        }
    }
}

}  // namespace isax

using namespace isax;

extern "C" {

isax_status isax_server_create(const isax_server_params* p, isax_server** out) {
    if (!out) return ISAX_ERR_INVALID_ARG;
    *out = nullptr;
    isax_server* s = new isax_server();
    if (p) {
        if (p->slots < 0 || p->slots > 256 || p->candidate_budget < 0) {
            delete s;
            return ISAX_ERR_INVALID_ARG;
        }
        if (p->slots > 0) s->nslots = p->slots;
        if (p->candidate_budget > 0) s->budget = (size_t)p->candidate_budget;
    }
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return ISAX_ERR_CUDA;
    }
    *out = s;
    return ISAX_OK;
}

isax_status isax_server_add_collection(isax_server* s, isax_index* ix, int32_t* id) {
    if (!s || !ix) return ISAX_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->started || ix->device != s->device) return ISAX_ERR_INVALID_ARG;
    s->colls.push_back(ix);
    if (id) *id = (int32_t)s->colls.size() - 1;
    return ISAX_OK;
}

isax_status isax_server_submit(isax_server* s, int32_t collection, const float* q, int32_t k, uint64_t tag) {
    if (!s || !q) return ISAX_ERR_INVALID_ARG;
    if (collection < 0 || collection >= (int32_t)s->colls.size()) return ISAX_ERR_INVALID_ARG;
    isax_index* ix = s->colls[collection];
    if (k < 1 || k > ISAX_MAX_K || (int64_t)k > ix->d.N) return ISAX_ERR_INVALID_ARG;
    ServeRequest r;
    r.tag = tag;
    r.coll = collection;
    r.k = k;
    r.q.assign(q, q + ix->d.n);
    r.t_submit = now_s();
    std::unique_lock<std::mutex> lk(s->mu);
    if (!s->started) {
        // the slots are sized for the collections added so far
        lk.unlock();
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(s->device);
        try {
            server_setup(s);
        } catch (const Error& e) {
            if (prev >= 0) cudaSetDevice(prev);
            std::lock_guard<std::mutex> lk2(s->mu);
            s->error = e.msg;
            return e.st;
        }
        if (prev >= 0) cudaSetDevice(prev);
        lk.lock();
        s->started = true;
        s->loop = std::thread(server_loop, s);
    }
    s->pending.push_back(std::move(r));
    s->submitted += 1;
    s->cv_work.notify_one();
    return ISAX_OK;
}

int32_t isax_server_poll(isax_server* s, isax_server_result* out, int64_t* idx, float* dist, int32_t max,
                         int32_t stride, int32_t wait_ms) {
    if (!s || max < 0 || (max > 0 && !out) || stride < 0) return -1;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
    int32_t m = 0;
    while (m < max && !s->done.empty()) {
        ServeResult& r = s->done.front();
        if (idx && (int32_t)r.k > stride) break;
        isax_server_result& o = out[m];
        memset(&o, 0, sizeof(o));
        o.tag = r.tag;
        o.collection = r.coll;
        o.k = r.k;
        o.status = r.status;
        o.reruns = r.reruns;
        o.submit_s = r.t_submit;
        o.start_s = r.t_start;
        o.done_s = r.t_done;
        o.stats.leaves_total = s->colls[r.coll]->d.L;
        o.stats.leaves_queued = (int64_t)r.ctl.leaves_queued;
        o.stats.leaves_scanned = (int64_t)r.ctl.leaves_scanned;
        o.stats.series_lb = (int64_t)r.ctl.series_lb;
        o.stats.series_refined = (int64_t)r.ctl.refined_total;
        o.stats.approx_series = (int64_t)r.ctl.approx_series;
        o.stats.candidates = (int64_t)r.ctl.cand_total;
        o.stats.window = (int64_t)r.ctl.window;
        o.stats.approx_leaf = r.ctl.approx_leaf;
        o.stats.reruns = r.reruns;
        o.stats.ed_floats = (int64_t)r.ctl.ed_floats;
        if (idx && r.status == ISAX_OK) memcpy(idx + (size_t)m * stride, r.idx.data(), sizeof(int64_t) * r.k);
        if (dist && r.status == ISAX_OK) memcpy(dist + (size_t)m * stride, r.dist.data(), sizeof(float) * r.k);
        s->done.pop_front();
        ++m;
    }
    return m;
}

isax_status isax_server_get_info(isax_server* s, isax_server_info* info) {
    if (!s || !info) return ISAX_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    info->collections = (int32_t)s->colls.size();
    info->slots = s->nslots;
    info->queued = (int64_t)s->pending.size();
    info->in_flight = s->in_flight;
    info->max_in_flight = s->max_in_flight;
    info->reserved_bytes = (int64_t)s->reserved;
    info->budget_bytes = (int64_t)s->budget;
    info->submitted = (int64_t)s->submitted;
    info->completed = (int64_t)s->completed;
    return ISAX_OK;
}

double isax_server_clock(void) { return now_s(); }

void isax_server_destroy(isax_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->loop.joinable()) s->loop.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (ServeSlot* sl : s->slots) slot_free(sl);
    cudaDeviceSynchronize();
    if (prev >= 0) cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
