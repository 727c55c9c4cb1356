// isax_common.cuh - shared definitions of the sm_103a iSAX k-NN library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/isax.h"

namespace isax {

constexpr int W = ISAX_W;          // segments (the paper fixes w = 16)
constexpr int MAX_CARD = 256;      // 8-bit symbols
constexpr int MAX_K = ISAX_MAX_K;
constexpr int MAX_LEN = ISAX_MAX_LEN;
constexpr int ROOT_BITS = W;       // root key: first bit of each of the 16 segments

constexpr int NBINS = 256;         // leaf ordering bins (lower bound / threshold)
constexpr int APPROX_NEIGHBORS = 2; // leaves on each side of the descent leaf in the approximate answer
// rows of the approximate answer at most (its leaves, widened until they hold k
// rows): a query's first candidate slots
inline uint32_t approx_rows_max(int leaf_size, int k) {
    return (uint32_t)((2 * APPROX_NEIGHBORS + 1) * leaf_size + k);
}
constexpr uint64_t EMPTY_SLOT = ~0ull;

// ---------------------------------------------------------------- errors
struct Error {
    isax_status st;
    std::string msg;
};

void set_error(isax_status st, const std::string& msg);

#define ISAX_CUDA_TRY(expr)                                                         \
    do {                                                                            \
        cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess)                                                      \
            throw ::isax::Error{ISAX_ERR_CUDA, std::string(#expr) + ": " +          \
                                                   cudaGetErrorString(e_)};          \
    } while (0)

// ---------------------------------------------------------------- checked build
// Compiled with -DISAX_CHECKS, kernels verify the invariants their memory
// accesses rely on (positions and rows inside the collection, list entries
// inside their capacity, leaf ranges in order) and record a failed one as a bit
// of a device word (one per translation unit), which isax_check_word() reads
// and clears.  The access itself goes ahead as in the normal build, where the
// checks compile to nothing.
enum : uint32_t {
    CHK_SCAN_ITEM = 0,     // a scan work item outside the collection or longer than a piece
    CHK_SCAN_CAND = 1,     // a pass-2 row outside its piece
    CHK_REFINE_ROW = 2,    // a survivor's row outside the collection
    CHK_APPROX_RANGE = 3,  // the approximate answer's positions outside the collection
    CHK_FINAL_ROW = 4,     // a final-ordering candidate's row outside the collection
    CHK_LEAF_RANGE = 5,    // a leaf whose first position is after its end
    CHK_BUILD_ID = 6,      // a leaf-order position holding an original row >= N
    CHK_WORK_COUNT = 7,    // a work list longer than its capacity without the overflow flag
};
#ifdef ISAX_CHECKS
static __device__ unsigned int g_check_word = 0;
#define ISAX_CHECK(cond, bit)                                              \
    do {                                                                   \
        if (!(cond)) atomicOr(&::isax::g_check_word, 1u << (unsigned)(bit)); \
    } while (0)
// this translation unit's word, read and cleared
static inline uint32_t take_check_word_here() {
    uint32_t v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_check_word, sizeof(v)) != cudaSuccess) return 0xFFFFFFFFu;
    cudaMemcpyToSymbol(g_check_word, &z, sizeof(z));
    return v;
}
#else
#define ISAX_CHECK(cond, bit) \
    do {                      \
    } while (0)
static inline uint32_t take_check_word_here() { return 0; }
#endif
uint32_t take_check_word_query();  // isax_query.cu
uint32_t take_check_word_build();  // isax_build.cu

// ---------------------------------------------------------------- tracing
// Counts a launch; with profiling on, brackets it with CUDA events on `st`.
class KernelScope {
   public:
    KernelScope(const char* name, cudaStream_t st);
    ~KernelScope();
    KernelScope(const KernelScope&) = delete;
    KernelScope& operator=(const KernelScope&) = delete;

   private:
    const char* name_;
    cudaStream_t st_;
    void* e0_ = nullptr;
    void* e1_ = nullptr;
};
#define ISAX_LAUNCH(name, st) ::isax::KernelScope isax_ks_##__LINE__(name, st)
bool profiling_on();               // per-kernel event timing enabled
void count_launches(int kernels);  // launches made by replaying a captured graph

// ---------------------------------------------------------------- allocator
void* dev_alloc(size_t bytes, cudaStream_t st);  // throws Error{OOM}
void dev_free(void* p, cudaStream_t st);

// ---------------------------------------------------------------- index
// Device view of an index, passed by value to kernels.
struct DevIndex {
    int64_t N;
    int32_t n, card, cbits, keybits, leaf_size;
    int64_t L;                    // leaves
    const float* x;               // [N][n] rows: in leaf order, or the caller's rows in their
                                  // original order when rows_in_place
    const uint4* sax;             // [N] 16 symbols per series, leaf order
    const uint32_t* orig;         // [N] original row of each position
    const uint32_t* leaf_begin;   // [L+1]
    const uint4* env;             // [L][2]: min symbols, max symbols
    const unsigned long long* leaf_key;  // [L] key of the first series of each leaf
    const float* bp;              // [card+1] breakpoints: -inf, beta_1 .. beta_{card-1}, +inf
    float maxabs;                 // max |x| over the collection
    int32_t rows_in_place;        // x is the caller's array, indexed by original id
    // balanced-split tree (ISAX_BUILD_SPLIT_BALANCED only, else null): node g is
    // {first child, split segment} when internal (children g' and g'+1), {-1 - leaf, -1}
    // when a leaf; tree_root[key] is the node of the root child with that 16-bit key, -1
    // if none
    const int2* tree;
    const int32_t* tree_root;
};

// row of x that holds the series at leaf-order position pos
__device__ __forceinline__ uint32_t row_at(const DevIndex& ix, int64_t pos) {
    return ix.rows_in_place ? ix.orig[pos] : (uint32_t)pos;
}
// original id of the series in row r of x
__device__ __forceinline__ uint32_t id_of_row(const DevIndex& ix, uint32_t r) {
    return ix.rows_in_place ? r : ix.orig[r];
}

// Per-query control block (device).
struct QCtl {
    unsigned long long qkey;
    int32_t descent_leaf;
    int32_t approx_leaf;   // approximate answer: leaves [approx_leaf, approx_end)
    int32_t approx_end;
    uint8_t qsym[16];      // query symbols
    uint32_t work_count;   // scan work items (pieces of the queued leaves)
    uint32_t cand_count;   // candidate appends attempted (may exceed capacity)
    uint32_t cand_base;    // candidate slots [0, cand_base) hold the approximate answer's rows
    uint32_t surv_count;   // series whose bound passed (appended; may exceed capacity)
    uint32_t window;       // candidates re-ranked in FP64
    uint32_t flags;        // QF_* bits
    float thr_lb0;         // bound threshold the work list was binned with
    float thr_scan;        // squared-bound threshold of the series scan (from the approximate answer)
    uint32_t grid_sync;    // arrivals at the binning step's grid barrier
    uint32_t cand_total, pad0;  // candidate appends and
    unsigned long long refined_total;  // series refined, saved by q_finalize (which clears the live counts)
    float qpaa[16];        // query PAA (fp32, as used by the bound table)
    double E;              // sqrt(n) * (eps_x + eps_q): PAA rounding slack
    double delta;          // relative error bound of an fp32 squared distance
    unsigned long long series_lb, series_refined, leaves_scanned, leaves_queued, approx_series;
    unsigned long long ed_floats;  // row floats read by the refinement (abandoned rows: the chunks read)
    uint32_t scan_done;    // scan CTAs whose survivors are all in the list
    uint32_t pad1;
    // fp32 factors of the pruning limits, each rounded up from its FP64 value:
    // 1 + 5 delta, 1 + 8 delta, 1 + 3 delta, E, (1 + 24 u)(1 + 1e-12)
    float f_lb, f_ab, f_win, f_E, f_sq, pad2[3];
};

enum : uint32_t {
    QF_NONFINITE = 1u,  // query holds NaN or Inf
    QF_OVERFLOW = 2u,   // candidate buffer overflowed: rerun with more room
    QF_SHORT = 4u,      // fewer than k candidates reached the end (internal error)
    QF_STALLED = 8u,    // a bounded wait on a bulk copy gave up (internal error)
};

// Device scratch of one in-flight query.
struct QueryScratch {
    float* q;                      // [n]
    float* table;                  // [16][card] lower-bound table
    float* leaf_lb;                // [L]
    uint2* work;                   // [work_cap] scan items {first row, rows | leaf-start bit 31},
                                   // ordered by bin
    uint32_t work_cap;
    uint32_t* bin_count;           // [NBINS]
    uint32_t* bin_cursor;          // [NBINS]
    unsigned long long* topk;      // [MAX_K] packed (fp32 d2 bits << 32 | orig)
    unsigned long long* cand_key;  // [cap]
    uint32_t* cand_pos;            // [cap]
    uint32_t cand_cap;
    uint2* surv;                   // [surv_cap] series that passed the bound: {row of x + 1, bound
                                   // bits}; a slot with .x == 0 is empty (slots start empty, and
                                   // the refinement of a single query empties each one it takes)
    uint32_t surv_cap;
    QCtl* ctl;
    int64_t* out_idx;              // [MAX_K]
    float* out_dist;               // [MAX_K]
};

// A mapped page-locked block per index for its single queries: before a launch
// the host writes the query's source and output pointers (and, for a query in
// host memory, its values); the query's first kernel reads the query from
// there, and its last writes the answer to the caller's device outputs and
// leaves the control block (and the answer for host outputs) here, so a query
// needs no copies of its own around its kernels.
struct QMail {
    const float* q_src;   // device address of the query: the caller's array, or q below
    int64_t* out_idx;     // the caller's device outputs, or null (answer only below)
    float* out_dist;
    uint64_t pad;
    QCtl ctl;             // the control block as the query ended
    int64_t idx[MAX_K];
    float dist[MAX_K];
    float q[MAX_LEN];
};

}  // namespace isax

struct isax_index;

namespace isax {

// Host-side entry points (defined in the .cu files); they throw Error.
isax_index* build_index_impl(const float* series, int64_t N, int n, int card, int leaf_size,
                             uint32_t mem_flags, cudaStream_t st);
void summarize_impl(const float* series, int64_t N, int n, int card, uint32_t mem_flags,
                    uint8_t* out_sax, float* out_paa, cudaStream_t st);
// query strategies: MESSI (leaf pruning, leaves in bound order) and the ParIS
// flat scan (every series of the SAX array bounded, storage order)
enum : int { QUERY_MESSI = 0, QUERY_FLAT = 1 };
// One query on the index's own scratch, its n values read from q_src (a device
// address; null: already in the scratch); the control block is copied to
// *ctl_out and, when given, the answer to out_idx / out_dist (device pointers
// if out_device).
void query_device(isax_index* ix, int k, QCtl* ctl_out, int* reruns, cudaStream_t st,
                  int mode = QUERY_MESSI, int64_t* out_idx = nullptr, float* out_dist = nullptr,
                  bool out_device = false, const float* q_src = nullptr);
// the index's mapped block, allocated on first use
void ensure_query_mail(isax_index* ix);
typedef void (*isax_query_stats_fill)(void* ctx, int b, const QCtl& c, int reruns);
void query_batch_device(isax_index* ix, const float* Q, int B, int k, uint32_t mem_flags,
                        int64_t* out_idx, float* out_dist, isax_query_stats_fill fill,
                        void* fill_ctx, cudaStream_t st);
void free_index_arrays(isax_index* ix, cudaStream_t st);
// scan_share: the query's scan runs on num_sms / scan_share CTAs (1: every SM;
// more leaves room for the scans of concurrent queries)
void launch_query_on_scratch(isax_index* ix, const QueryScratch& s, int k, cudaStream_t st,
                             int mode = QUERY_MESSI, int scan_share = 1, QMail* mail = nullptr);
void alloc_query_scratch(isax_index* ix, uint32_t cand_cap, uint32_t surv_cap, cudaStream_t st,
                         bool keep_query = false);
uint32_t default_surv_cap(int64_t N);  // survivor entries of a fresh query scratch
void launch_breakpoints(int card, float* bp, cudaStream_t st);
// test hook: QF_STALLED for the next queries whose control block the host reads (isax_selftest.cu)
uint32_t injected_query_flags();
// batched query kernels (query b of the batch owns scratch ss[b])
void launch_bq_prep(isax_index* ix, const QueryScratch* ss, int B, int k, int neighbors,
                    cudaStream_t st);
void launch_bq_approx(isax_index* ix, const QueryScratch* ss, int B, int k, int neighbors,
                      cudaStream_t st);
void launch_bq_pairs(isax_index* ix, const QueryScratch* ss, int B, int k, uint32_t* leaf_count,
                     uint32_t* mask, cudaStream_t st);
void launch_bq_fill(isax_index* ix, int B, const uint32_t* mask, const uint32_t* leaf_off,
                    uint32_t* pairs, cudaStream_t st);
void launch_bq_recheck(isax_index* ix, const QueryScratch* ss, int k, const uint4* cand,
                       const uint32_t* cand_count, uint32_t cap, cudaStream_t st);
void launch_bq_finalize(isax_index* ix, const QueryScratch* ss, int B, int k, cudaStream_t st);
// FP64 squared distances, definition order, of rows idx[b][j] to queries Q[b] (device arrays)
void exact_d2_device(isax_index* ix, const float* Q, int B, int k, const int64_t* idx, double* out,
                     cudaStream_t st);
// scratch and captured graphs for the resident query server (isax_serve.cu)
int64_t work_items_cap(int64_t L, int64_t N);
void alloc_query_scratch_for(int64_t L, int64_t N, int n, int card, uint32_t cand_cap, uint32_t surv_cap,
                             QueryScratch& q, cudaStream_t st);
void grow_query_candidates(QueryScratch& q, uint32_t cand_cap, cudaStream_t st);
void grow_query_survivors(QueryScratch& q, uint32_t surv_cap, cudaStream_t st);
void empty_survivors(const QueryScratch& q, cudaStream_t st);
void free_query_scratch_struct(QueryScratch& q, cudaStream_t st);
void* query_graphs_new();
void query_graphs_delete(void* g);
void query_graphs_clear(void* g);
void launch_query_graph_ext(isax_index* ix, const QueryScratch& qs, void* g, int k, cudaStream_t st,
                            int scan_share = 1);
// the tensor-core filtered batch (isax_tc.cu)
void prepare_tc(isax_index* ix, cudaStream_t st);
void query_batch_tc(isax_index* ix, const float* Q, int B, int k, uint32_t mem_flags, int64_t* out_idx,
                    float* out_dist, isax_query_stats_fill fill, void* fill_ctx, cudaStream_t st);
void free_tc_state(isax_index* ix, cudaStream_t st);
void launch_summarize(const float* x, int64_t N, int n, int card, const float* bp,
                      uint4* sax, unsigned long long* keys, uint32_t* ids, float* paa_out,
                      unsigned int* maxabs_bits, unsigned int* nonfinite, int num_sms,
                      cudaStream_t st, uint32_t id_base = 0);

}  // namespace isax

// the opaque handle of the C ABI
struct isax_index {
    int device;
    int num_sms;
    isax::DevIndex d;
    int32_t max_leaf;
    int64_t bytes;
    // owned device arrays
    float* x;
    uint4* sax;
    uint32_t* orig;
    uint32_t* leaf_begin;
    uint4* env;
    unsigned long long* leaf_key;
    float* bp;
    int2* tree;          // balanced-split tree nodes (null for the round-robin split)
    int32_t* tree_root;  // [2^16]
    uint32_t* inv;       // row of x of each original row (built on first use; leaf-order rows only)
    int64_t tree_nodes;
    // query scratch (one in-flight query)
    isax::QueryScratch qs;
    void* mu;      // std::mutex*
    void* graphs;  // captured query launch sequences (isax_query.cu)
    void* pool;    // extra query slots for concurrent batches (isax_query.cu)
    void* tc;      // BF16 copy and batch scratch of the tensor-core filter (isax_tc.cu)
    bool rows_host;  // x is pinned host memory (ISAX_BUILD_ROWS_HOST)
    bool rows_in_place;  // x holds the rows in the input's order, read by original row
    bool rows_borrowed;  // ... and is the caller's device array (ISAX_BUILD_ROWS_IN_PLACE), not owned
    isax::QMail* mail;      // the single queries' mapped block (host address), or null
    isax::QMail* mail_dev;  // its device address
};
