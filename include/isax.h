/*
 * isax.h - C ABI of the GB300 exact Euclidean k-NN engine over in-memory
 * data-series collections, driven by an iSAX index (Peng, Fatourou, Palpanas,
 * "Data Series Indexing Gone Parallel": ParIS / ParIS+ / MESSI).
 *
 * All compute runs in sm_103a CUDA kernels; these entry points only validate
 * arguments, move buffers and launch.  Every call is stream-ordered on the
 * given CUDA stream (a cudaStream_t passed as void*, NULL = legacy default
 * stream) and returns after its results are in the caller's buffers.
 *
 * Pointers are "host" or "device" as the mem_flags bits say; device pointers
 * must belong to the device the index lives on.  Float arrays must be 16-byte
 * aligned (torch and cudaMalloc allocations are).  On any error a call returns
 * a non-zero isax_status, leaves its outputs unspecified, leaks nothing, and
 * isax_last_error() describes the failure (per calling thread).
 */
#ifndef ISAX_H
#define ISAX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum isax_status {
    ISAX_OK = 0,
    ISAX_ERR_INVALID_ARG = 1, /* bad size, pointer, flag, or non-finite input */
    ISAX_ERR_OOM = 2,         /* a device allocation failed */
    ISAX_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    ISAX_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    ISAX_ERR_INTERNAL = 5     /* an internal consistency check failed */
} isax_status;

#define ISAX_W 16          /* segments per series: the paper fixes w = 16 (Section III) */
#define ISAX_MAX_K 1024    /* largest k a query accepts */
#define ISAX_MAX_LEN 4096  /* largest series length n */

/* mem_flags bits */
#define ISAX_MEM_INPUT_DEVICE 1u  /* input series / queries are device pointers */
#define ISAX_MEM_OUTPUT_DEVICE 2u /* output arrays are device pointers */
/* build only: after the build, keep the leaf-ordered series in pinned HOST memory
 * and free their device copy; the SAX words, ids, leaf boundaries and envelopes
 * stay in device memory.  Queries then compute every lower bound on the GPU and
 * read the rows they refine over the CPU-GPU link (the paper's sketch of a GPU
 * design with the raw data in host memory, Section V).  The build itself still
 * stages the rows in device memory. */
#define ISAX_BUILD_ROWS_HOST 4u
/* build only, with ISAX_MEM_INPUT_DEVICE: the index keeps a pointer to the
 * caller's device array `series` and reads the rows there, by original row
 * index, for the rest of its life; it copies none of them.  This is the paper's
 * in-memory layout (Section III: the raw series stay in the RawData array and
 * each leaf holds the series' iSAX words and pointers into it, Section II).
 * The array must stay allocated and unchanged until isax_free_index; the index
 * owns only its SAX words, ids, leaf boundaries and envelopes.  Without this
 * flag the build copies the rows into leaf order and the caller may free
 * `series` when the call returns.  Not combinable with ISAX_BUILD_ROWS_HOST. */
#define ISAX_BUILD_ROWS_IN_PLACE 8u
/* build only: form the leaves by ADS+ node splitting (Section II, ADS+ Index)
 * instead of the default round-robin split.  The root has one child per 16-bit
 * key (the first bit of every segment); a node holding more than leaf_size
 * series splits on the segment whose next bit divides its first leaf_size + 1
 * series (in row order, i.e. as if the series were inserted one by one) most
 * evenly, the lowest segment on a tie; children take the node's series in row
 * order, child 0 (bit 0) first.  A node whose 16 segments are all at full
 * cardinality is not split (a leaf of identical words may exceed leaf_size).
 * The leaves are those of that tree in depth-first order, empty ones dropped; a
 * query's approximate-answer leaf is the one its word descends to.  Slower to
 * build (one pass over the collection per tree level); combinable with every
 * other build flag. */
#define ISAX_BUILD_SPLIT_BALANCED 16u

typedef struct isax_build_params {
    int32_t w;           /* segments; must be ISAX_W (16) */
    int32_t cardinality; /* symbols per segment: power of two in [2, 256] (256 = 8-bit SAX) */
    int32_t leaf_size;   /* leaf capacity, >= 1 (runs of identical keys are cut into pieces of this size) */
    uint32_t mem_flags;  /* ISAX_MEM_INPUT_DEVICE if `series` is a device pointer;
                            ISAX_BUILD_ROWS_HOST to keep the rows in host memory;
                            ISAX_BUILD_ROWS_IN_PLACE to read them in the caller's array;
                            ISAX_BUILD_SPLIT_BALANCED for ADS+ node splitting */
} isax_build_params;

typedef struct isax_query_stats {
    int64_t leaves_total;     /* leaves in the index (each gets an envelope bound) */
    int64_t leaves_queued;    /* leaves whose bound did not exceed the approximate BSF */
    int64_t leaves_scanned;   /* queued leaves whose series were bounded (all queued ones) */
    int64_t series_lb;        /* series lower bounds computed */
    int64_t series_refined;   /* exact distances computed (approximate leaf included) */
    int64_t approx_series;    /* series of the approximate-answer leaves (all refined) */
    int64_t candidates;       /* refined series kept for the final ordering */
    int64_t window;           /* candidates re-ranked in FP64 */
    int32_t approx_leaf;      /* leaf used for the approximate answer */
    int32_t reruns;           /* reruns after a candidate-buffer overflow */
    int64_t ed_floats;        /* row values read for exact distances (early abandoning stops a
                                 row before its end; on the BF16 path, the fp32 re-checks) */
} isax_query_stats;

typedef struct isax_index_info {
    int64_t N;             /* series */
    int32_t n;             /* series length */
    int32_t w;             /* segments (16) */
    int32_t cardinality;   /* symbols per segment */
    int32_t leaf_size;     /* leaf capacity */
    int64_t leaves;        /* leaves */
    int32_t max_leaf;      /* largest leaf */
    int32_t device;        /* CUDA device ordinal */
    int64_t device_bytes;  /* device memory held by the index */
    float maxabs;          /* max |x| over the collection (bounds fp32 PAA error) */
} isax_index_info;

typedef struct isax_index isax_index;

/*
 * Device allocator hooks.  alloc returns NULL on failure; both are called with
 * the stream of the calling entry point.  Default: cudaMallocAsync /
 * cudaFreeAsync from the device's default memory pool.
 */
typedef void* (*isax_alloc_fn)(size_t bytes, void* cuda_stream, void* ctx);
typedef void (*isax_free_fn)(void* ptr, void* cuda_stream, void* ctx);

/* Install allocator hooks for indexes built afterwards (NULL, NULL restores
 * the default).  Not thread-safe against concurrent builds. */
isax_status isax_set_allocator(isax_alloc_fn alloc_fn, isax_free_fn free_fn, void* ctx);

/* The default pool keeps the memory of freed indexes and scratch for reuse.
 * isax_trim_memory synchronises `device` and hands that cached memory back to
 * the driver (the memory of live indexes stays).  Useful before a large build
 * whose allocation the cached pieces cannot serve.  No effect on memory from
 * allocator hooks.  Errors: ISAX_ERR_INVALID_ARG (device), ISAX_ERR_CUDA. */
isax_status isax_trim_memory(int32_t device);

/*
 * isax_build_index - summarise a collection and build its iSAX index
 * (Section II, iSAX Representation and ADS+ Index; Section III, MESSI index
 * construction, Stages 1-2).
 *
 *   series  [N][n] fp32, row-major; borrowed for the call only unless
 *           ISAX_BUILD_ROWS_IN_PLACE.  A device input is copied into leaf
 *           order; a host input is copied to the device in chunks, each
 *           summarised as soon as it lands, and the copy (in the input's
 *           order, read by row) is the index's row store.
 *   N       1 .. 2^32-2 series.
 *   n       length, a multiple of 16 in [16, ISAX_MAX_LEN].
 *   p       parameters (see isax_build_params); NULL = {16, 256, 2000, 0}.
 *   out     receives the new index (NULL on error).
 *
 * Steps, all on the GPU: PAA of w segments and SAX symbols against N(0,1)
 * breakpoints; a stable radix sort of the bit-plane-interleaved iSAX keys
 * (first bit of every segment first: the root subtree of Section III); leaves
 * cut top-down from the sorted keys (with ISAX_BUILD_SPLIT_BALANCED: a sort by
 * root key, then ADS+ node splitting one tree level at a time); rows and SAX
 * words gathered into leaf order; per-leaf min/max symbol envelopes.
 * Errors: ISAX_ERR_INVALID_ARG (sizes, flags, null pointers, misaligned
 * pointer, a non-finite value anywhere in `series`), ISAX_ERR_OOM, ISAX_ERR_CUDA.
 */
isax_status isax_build_index(const float* series, int64_t N, int32_t n, const isax_build_params* p,
                             void* cuda_stream, isax_index** out);

/*
 * isax_query_knn - exact k nearest neighbours of one query under Euclidean
 * distance (Section II, Similarity Search; k = 1 is the paper's NN query),
 * answered with MESSI's strategy (Section III, MESSI Approach): approximate
 * answer from the query's own leaf, leaf pruning by envelope lower bounds,
 * leaves processed in lower-bound order, series lower bounds, then real
 * distances with early abandoning, BSF updates.
 *
 *   q        [n] fp32 query (host or device per ISAX_MEM_INPUT_DEVICE).
 *   k        1 .. min(N, ISAX_MAX_K).
 *   out_idx  [k] int64: 0-based rows of the original `series`, ascending by
 *            (distance, row); ties go to the lower row.
 *   out_dist [k] fp32 Euclidean distances (not squared), each the FP64
 *            distance rounded to fp32.
 *   stats    optional per-query counters (NULL to skip).
 * The answer equals the brute-force scan of the definition: distances are
 * re-ranked in FP64 wherever fp32 cannot order them.  Calls on the same index
 * are serialised internally.  Errors: ISAX_ERR_INVALID_ARG (k, pointers,
 * non-finite query), ISAX_ERR_CUDA, ISAX_ERR_OOM.
 */
isax_status isax_query_knn(const isax_index* ix, const float* q, int32_t k, uint32_t mem_flags,
                           int64_t* out_idx, float* out_dist, isax_query_stats* stats,
                           void* cuda_stream);

/*
 * isax_query_knn_batch - B queries Q[B][n]; row b's answer, in out_idx[b][k]
 * and out_dist[b][k], equals isax_query_knn on Q[b].  stats: NULL or [B].
 * Fewer than 8 queries run concurrently on per-query stream slots; larger
 * batches run in chunks, each step of the query launched once for the whole
 * chunk (Section III's query strategy, per query); queries whose survivors or
 * candidates overflow their room run again in a second pass with more room.  The
 * device scratch (up to 12 GB, and 6 GB for the second pass when one is needed,
 * sized to fit) is allocated on first use and kept until isax_free_index.  Errors as isax_query_knn, plus ISAX_ERR_TIMEOUT if a
 * bounded wait of the scan gave up.
 */
isax_status isax_query_knn_batch(const isax_index* ix, const float* Q, int32_t B, int32_t k,
                                 uint32_t mem_flags, int64_t* out_idx, float* out_dist,
                                 isax_query_stats* stats, void* cuda_stream);

/* Release an index and its device memory (NULL is a no-op). */
void isax_free_index(isax_index* ix);

/* Description of the last error on the calling thread ("" if none). */
const char* isax_last_error(void);

/* Sizes of an index. */
isax_status isax_get_index_info(const isax_index* ix, isax_index_info* info);

/*
 * isax_index_export - copy the index's internal arrays to host buffers (any
 * may be NULL): sax [N][16] symbols in leaf order, orig_id [N] original row of
 * each leaf-order position, leaf_begin [leaves+1] first position of each leaf,
 * envelope [leaves][32] (16 min symbols then 16 max symbols), breakpoints
 * [cardinality-1] the fp32 N(0,1) quantiles used for the symbols.
 */
isax_status isax_index_export(const isax_index* ix, uint8_t* sax, uint32_t* orig_id,
                              uint32_t* leaf_begin, uint8_t* envelope, float* breakpoints);

/*
 * isax_summarize - the build's summarisation step alone (Section II: PAA over
 * w = 16 equal segments, then the SAX symbol of each segment mean).
 *   series [N][n] fp32 (host or device per ISAX_MEM_INPUT_DEVICE)
 *   out_sax [N][16] uint8 symbols, out_paa [N][16] fp32 segment means (either
 *   may be NULL; host or device per ISAX_MEM_OUTPUT_DEVICE).
 */
isax_status isax_summarize(const float* series, int64_t N, int32_t n, int32_t cardinality,
                           uint32_t mem_flags, uint8_t* out_sax, float* out_paa, void* cuda_stream);

/*
 * isax_exact_d2 - FP64 squared Euclidean distances of given series of the
 * collection to given queries, each summed with the definition's order
 * (Section II, Similarity Search: the distance of the NN problem; elements in
 * ascending order, every difference, square and sum rounded to FP64 on its
 * own, no fused multiply-add).  out_d2[b][j] = d^2(Q[b], series idx[b][j]).
 * These are the values the brute-force definition orders by, so the answers
 * of row shards of one collection (each an exact k-NN of its own rows) merge
 * exactly when ordered by (out_d2, global row): two rows of different shards
 * whose fp32 distances tie are still put in their exact order.
 *   Q      [B][n] fp32, idx [B][k] int64 original rows (host or device per
 *          ISAX_MEM_INPUT_DEVICE); out_d2 [B][k] (host or device per
 *          ISAX_MEM_OUTPUT_DEVICE).  A row outside [0, N) gives NaN.
 * The first call on an index whose rows are in leaf order builds the map from
 * original row to leaf position (4 N bytes, kept until isax_free_index).
 * Synchronises cuda_stream.  Errors: ISAX_ERR_INVALID_ARG, ISAX_ERR_OOM,
 * ISAX_ERR_CUDA.
 */
isax_status isax_exact_d2(const isax_index* ix, const float* Q, int32_t B, int32_t k, uint32_t mem_flags,
                          const int64_t* idx, double* out_d2, void* cuda_stream);

/* ------------------------------------------------------------ allocation-free query */

#define ISAX_NOALLOC_MAX_LEAVES 524288u       /* largest index (in leaves) it serves */
#define ISAX_NOALLOC_MAX_CANDIDATES 262144u   /* fp32 near-tie candidates it can hold */
#define ISAX_NOALLOC_MAX_SURVIVORS 1048576u   /* series passing the lower bound it can hold */
#define ISAX_NOALLOC_SCRATCH_BYTES 22075648u  /* its fixed device scratch (about 21 MiB) */

/*
 * isax_query_knn_noalloc - the same exact k-NN query as isax_query_knn (same
 * arguments, same answers) for callers that must not allocate device memory
 * while they query: a runtime that owns all GPU memory through its own pool, or
 * a latency-critical serving thread for which an allocation can stall on the
 * driver.  The paper has no counterpart; it is a deployment feature.
 *
 * Its scratch is one device array built into the library, of
 * ISAX_NOALLOC_SCRATCH_BYTES, held by every GPU that loads the library until
 * the process exits.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and each clears what
 * must start at zero; calls are serialised inside the library and return after
 * their results are copied out, because two queries running at once on the GPU
 * would race on the shared array.
 * Limits and errors: ISAX_ERR_INVALID_ARG for an index with more than
 * ISAX_NOALLOC_MAX_LEAVES leaves or with leaves + N / 128 above twice that
 * (and as isax_query_knn); ISAX_ERR_OOM when
 * more than ISAX_NOALLOC_MAX_SURVIVORS series pass the lower bound of the
 * approximate answer, or the query keeps more than ISAX_NOALLOC_MAX_CANDIDATES
 * candidates for its final FP64 ordering (refined series that were within fp32
 * error of the k-th best when refined); isax_query_knn would rerun with larger
 * buffers, this entry point cannot.  It calls no allocation routine.
 */
isax_status isax_query_knn_noalloc(const isax_index* ix, const float* q, int32_t k,
                                   uint32_t mem_flags, int64_t* out_idx, float* out_dist,
                                   isax_query_stats* stats, void* cuda_stream);

/*
 * isax_query_knn_flat - the same exact k-NN query (same arguments, same
 * answers) answered the ParIS way instead of MESSI's (Section III, ParIS+ query
 * answering): after the approximate answer, the lower bound of EVERY series in
 * the SAX array is computed, in storage order, and the series it does not prune
 * are refined; no leaf is pruned by its envelope and leaves are not visited in
 * bound order.  Kept to measure what MESSI's leaf pruning and ordering buy.
 */
isax_status isax_query_knn_flat(const isax_index* ix, const float* q, int32_t k, uint32_t mem_flags,
                                int64_t* out_idx, float* out_dist, isax_query_stats* stats,
                                void* cuda_stream);

/* ------------------------------------------------------------ BF16-filtered batch */

/*
 * isax_query_knn_batch_bf16 - exact k-NN of B queries, the same answers as
 * isax_query_knn_batch (same arguments and layouts), for large batches.  The
 * paper refines by computing real distances one series at a time (Section III,
 * MESSI Approach); here the distances of a whole batch to the series of the
 * leaves that the envelope bound does not prune are first computed on the
 * tensor cores as ||x||^2 + ||q||^2 - 2 bf16(x).bf16(q) with FP32 accumulation,
 * and used only as a filter: a series is dropped only when that value minus a
 * rigorous bound on its rounding error (about 4.07 in squared-distance units for
 * z-normalised series of length 256) exceeds an upper bound of the query's k-th
 * best squared distance.  Every other series is re-checked with the exact fp32
 * distance of the single-query path, and the k best are ordered as there (FP64
 * where fp32 cannot separate them).  Each leaf's rows are read once per group of
 * up to 128 queries that need them (up to 65536 / (2 n) for n > 256).
 *   Requires n % 64 == 0 and n <= 2048 (else ISAX_ERR_INVALID_ARG).  The first call builds a
 *   BF16 copy of the collection (2 N n bytes of device memory, held until the
 *   index is freed; isax_prepare_bf16 builds it ahead of time).  Batches run in
 *   passes of up to 4096 queries; per pass it holds about
 *   B (4 L + 50 KB) bytes of scratch (L = leaves).  A query whose candidate
 *   window overflows is answered again by the single-query path (stats.reruns).
 *   ISAX_ERR_TIMEOUT if a bounded wait inside the filter gave up.
 */
isax_status isax_query_knn_batch_bf16(const isax_index* ix, const float* Q, int32_t B, int32_t k,
                                      uint32_t mem_flags, int64_t* out_idx, float* out_dist,
                                      isax_query_stats* stats, void* cuda_stream);

/* Build the BF16 copy used by isax_query_knn_batch_bf16 now (synchronises
 * cuda_stream).  ISAX_ERR_INVALID_ARG when n % 64 != 0, n > 2048, or values are
 * too large for the error bound (|x| >= 1e15). */
isax_status isax_prepare_bf16(isax_index* ix, void* cuda_stream);

/* ------------------------------------------------------------ resident query server */

/*
 * A resident query server (the paper has no counterpart; it serves the
 * single-query path of Section III to many clients).  Several indexes stay in
 * device memory; requests for any of them are admitted, as they arrive, into a
 * fixed set of in-flight slots (continuous batching: no batch has to form or
 * drain).  A request is admitted, in arrival order, when a slot is free and its
 * candidate buffer (12 bytes x (4096 + 256 k) entries) fits the memory budget
 * beside those of the requests in flight; a query whose buffer overflows is
 * rerun with four times the room once the budget allows.  Each request runs
 * the single-query kernels on its slot's own stream, scratch and captured
 * graphs, so its answer is the one isax_query_knn returns for it alone.  A host
 * thread inside the library runs the loop; the calls below are thread-safe.
 */
typedef struct isax_server isax_server;

typedef struct isax_server_params {
    int32_t slots;             /* requests in flight at most (1..256; 0: 16) */
    int64_t candidate_budget;  /* bytes of candidate buffers in flight (0: 256 MiB) */
} isax_server_params;

typedef struct isax_server_result {
    uint64_t tag;              /* the caller's tag from isax_server_submit */
    int32_t collection;        /* id from isax_server_add_collection */
    int32_t k;
    int32_t status;            /* ISAX_OK, or the error of this request */
    int32_t reruns;            /* reruns after a candidate overflow */
    double submit_s;           /* times on isax_server_clock(): submitted, */
    double start_s;            /* admitted into a slot, */
    double done_s;             /* answer copied back */
    isax_query_stats stats;
} isax_server_result;

typedef struct isax_server_info {
    int32_t collections, slots;
    int64_t queued;            /* submitted, not yet admitted */
    int32_t in_flight, max_in_flight;
    int64_t reserved_bytes, budget_bytes;
    int64_t submitted, completed;
} isax_server_info;

/* A server on the current device (params may be NULL for the defaults). */
isax_status isax_server_create(const isax_server_params* params, isax_server** out);

/* Add a collection before the first submit (the slots are sized for the
 * collections added by then).  The index stays owned by the caller and must
 * outlive the server; it must live on the server's device.  *id = 0, 1, ... */
isax_status isax_server_add_collection(isax_server* s, isax_index* ix, int32_t* id);

/* Queue one exact k-NN request: q is a HOST array of the collection's series
 * length n (copied before the call returns), 1 <= k <= min(N, 1024).  Returns
 * at once; the result is collected with isax_server_poll. */
isax_status isax_server_submit(isax_server* s, int32_t collection, const float* q, int32_t k,
                               uint64_t tag);

/* Up to max finished results, oldest first, waiting up to wait_ms for the
 * first one.  Result i's answer goes to idx[i * stride .. + k) and
 * dist[i * stride .. + k) (host arrays; either may be NULL; a result with
 * k > stride stays queued).  Returns the number of results, -1 on bad
 * arguments. */
int32_t isax_server_poll(isax_server* s, isax_server_result* out, int64_t* idx, float* dist,
                         int32_t max, int32_t stride, int32_t wait_ms);

/* Queue lengths, slots in use, budget in use. */
isax_status isax_server_get_info(isax_server* s, isax_server_info* info);

/* Seconds on the server's (monotonic) clock, for request timestamps. */
double isax_server_clock(void);

/* Finish every queued and in-flight request, then release the server. */
void isax_server_destroy(isax_server* s);

/* ------------------------------------------------------------ tensor-core check */

/*
 * isax_tc_selftest - one tile of the tensor-core contraction used by the
 * BF16-filtered batch path, exposed to check the machinery on its own (the
 * paper has no counterpart): d[i][j] = sum_t a[i][t] * b[j][t] accumulated in
 * FP32, for i < 128, j < n_cols, t < 256.
 *   a [128][256] and b [n_cols][256] BF16 bit patterns in device memory,
 *   16-byte aligned, row-major; d [128][n_cols] fp32 device output.
 *   n_cols: a multiple of 16 in [16, 256] (else ISAX_ERR_INVALID_ARG).
 * Synchronises cuda_stream; ISAX_ERR_TIMEOUT if a bounded wait gave up.
 */
isax_status isax_tc_selftest(const uint16_t* a, const uint16_t* b, int32_t n_cols, float* d,
                             void* cuda_stream);

/* ------------------------------------------------------------ failure checks */

/* 1 if the library was compiled with -DISAX_CHECKS (bounds-checked kernels),
 * else 0.  The paper has no counterpart. */
int32_t isax_checks_enabled(void);

/*
 * isax_check_word - in a bounds-checked build: the invariants that kernels
 * found violated since the last call, one bit each (row or position outside
 * the collection, a scan work item longer than a piece or past the end, a
 * survivor's or candidate's row outside the collection, a leaf range out of
 * order, ...), then cleared.  0 means every checked access stayed in range.
 * Always 0 in the normal build.  Call it with no query or build in flight.
 */
isax_status isax_check_word(uint32_t* out);

/*
 * isax_selftest_wait - make one of the library's bounded device waits run out
 * on purpose, to check its failure path without a GPU fault (the paper has no
 * counterpart).  kind 0: a one-warp kernel waits on its own mbarrier, which
 * completes only if satisfied != 0 (the kernel then arrives on it first); no
 * copy is in flight.  kind 1: a cooperative grid of 4 CTAs meets at the
 * binning step's grid barrier, expecting 4 arrivals if satisfied != 0 and 5
 * (never reached) otherwise.  Each wait polls at most max_polls times (1 ..
 * 2^24).  Returns ISAX_OK when the wait completed, ISAX_ERR_TIMEOUT when it gave
 * up; the device stays usable either way.  Synchronises cuda_stream.
 */
isax_status isax_selftest_wait(int32_t kind, int32_t satisfied, int32_t max_polls, void* cuda_stream);

/*
 * isax_debug_inject_timeout - test hook: the next `queries` query control
 * blocks that the host reads back (single, batch, BF16 batch, allocation-free
 * and served queries alike) report a bounded device wait that gave up, so each
 * entry point's handling of it (ISAX_ERR_TIMEOUT) can be checked without a wait
 * running out.  0 cancels.  The paper has no counterpart.
 */
isax_status isax_debug_inject_timeout(int32_t queries);

/* ------------------------------------------------------------ tracing */

typedef struct isax_kernel_time {
    char name[48];     /* kernel name */
    int64_t launches;  /* timed launches */
    double total_ms;   /* summed CUDA-event duration on the launching stream */
} isax_kernel_time;

/* Time later kernel launches of this library with a pair of CUDA events
 * recorded on each launch's stream (clears earlier records): mode 1 every
 * kernel (queries then launch kernel by kernel instead of replaying their
 * captured CUDA graph), mode 2 the index-build kernels only, 0 stop timing.
 * Timing adds two event records per timed launch. */
isax_status isax_profile(int32_t mode);

/* Per-kernel totals of the timed launches (waits for their events).  Fills at
 * most max entries of out (out may be NULL) and returns the number of distinct
 * kernels. */
int32_t isax_profile_report(isax_kernel_time* out, int32_t max);

/* Kernels this library has launched in this process (always counted). */
uint64_t isax_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* ISAX_H */
