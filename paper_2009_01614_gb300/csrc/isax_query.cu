// isax_query.cu - exact k-NN query answering on the GPU, following MESSI's
// query strategy (Section III, MESSI Approach; lower-bound and real-distance
// calculations are its two hot loops).  A single query is four launches:
//
//   q_front       query PAA, SAX symbols and key; the lower-bound table
//                 T[i][s] = (n/w) dist(qpaa_i, region s)^2 in fp32; the leaf the
//                 query's key descends to and the real distances of its rows
//                 (the approximate answer: the first BSF); the envelope lower
//                 bound of every leaf.
//   q_leaf_bin    the leaves the BSF does not prune, counted into bins of
//                 bound / BSF and listed bin by bin: a work list of leaf pieces
//                 in ascending lower-bound order (MESSI's priority queues).
//   q_scan_refine the pieces dealt to the warps in that order; each warp streams
//                 its pieces' 16-byte SAX words through a ring of shared-memory
//                 stages filled by bulk copies and bounds them against the table
//                 in shared memory; survivors {row of x, bound} go to a list.
//                 Warps with no piece left take survivors from the list, skip
//                 those whose bound now exceeds the k-th best and compute real
//                 distances; the k best so far live in a sorted array updated
//                 by an atomicMin cascade.
//   q_finalize    candidates within fp32 error of the k-th best re-ranked in
//                 FP64 (ties by lower row), distances rounded to fp32.
//
// Batches of queries (bq_*) run the same steps with the scan and the
// refinement as separate launches over all queries of a chunk.
//
// Rows.  The rows are either copied into leaf order by the build (row of x =
// leaf-order position) or read in the caller's array, where each leaf refers
// to its series by original row (the paper's leaves hold pointers into the raw
// data array): row_at() maps a position to its row of x, id_of_row() a row of
// x to the original id.  Survivors and candidates carry rows of x.
//
// Exactness.  Bounds are pruned only with the slack of a rigorous fp32 error
// analysis: a series is pruned only if its bound proves its exact distance
// exceeds (1 + 5 delta) times the current k-th best, where delta bounds the
// relative error of an fp32 squared distance and E bounds the PAA rounding
// error.  Every series whose fp32 distance lies within (1 + 3 delta) of the
// final k-th best is kept as a candidate and re-ranked in FP64 with the same
// left-to-right sum as the definition, so the indices equal the brute-force
// answer's.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "isax_common.cuh"
#include "isax_kernels_util.cuh"

namespace isax {

// ---------------------------------------------------------------- helpers

// squared lower-bound threshold: prune iff bound > this (see file comment)
__device__ float lb_threshold(unsigned long long kth, double delta, double E) {
    if (kth == EMPTY_SLOT) return INFINITY;
    double t = (double)key_d2(kth);
    double r = sqrt(t * (1.0 + 5.0 * delta)) + E;
    double lb = r * r * (1.0 + 24.0 * 0x1p-24) * (1.0 + 1e-12);
    return __double2float_ru(lb);
}

__device__ __forceinline__ int bin_of(float lb, float thr) {
    if (!(thr > 0.0f) || isinf(thr)) return 0;
    int b = (int)(sqrtf(lb / thr) * (float)NBINS);
    return b < 0 ? 0 : (b >= NBINS ? NBINS - 1 : b);
}


// one refined series (by one thread): update the k best, keep as candidate
__device__ void consider(const QueryScratch& s, int k, unsigned long long key, uint32_t pos,
                         double delta) {
    unsigned long long kth = ld_volatile_u64(&s.topk[k - 1]);
    if (key < kth) {
        topk_insert(s.topk, k, key);
        kth = ld_volatile_u64(&s.topk[k - 1]);
    }
    bool keep = kth == EMPTY_SLOT ||
                (double)key_d2(key) <= (double)key_d2(kth) * (1.0 + 3.0 * delta);
    if (keep) {
        // slots [0, cand_base) hold the approximate answer's rows (written in place)
        uint32_t i = s.ctl->cand_base + atomicAdd(&s.ctl->cand_count, 1u);
        if (i < s.cand_cap) {
            s.cand_key[i] = key;
            s.cand_pos[i] = pos;
        }
    }
}

// abandon a partial sum only above (1 + 8 delta) * k-th best: the full fp32
// distance then exceeds the candidate window (1 + 3 delta) for sure
__device__ __forceinline__ float abandon_limit(unsigned long long kth, double delta) {
    if (kth == EMPTY_SLOT) return INFINITY;
    return __double2float_ru((double)key_d2(kth) * (1.0 + 8.0 * delta));
}

// The fp32 factors of the limits below, each rounded up from its FP64 value
// (written once per query with the control block).
__device__ __forceinline__ void set_limit_factors(QCtl* c, double delta, double E) {
    c->f_lb = __double2float_ru(1.0 + 5.0 * delta);
    c->f_ab = __double2float_ru(1.0 + 8.0 * delta);
    c->f_win = __double2float_ru(1.0 + 3.0 * delta);
    c->f_E = __double2float_ru(E);
    c->f_sq = __double2float_ru((1.0 + 24.0 * 0x1p-24) * (1.0 + 1e-12));
}

// A k-th best's three limits in fp32, every operation rounded up from values
// that are themselves upper bounds, so each is at least the FP64 expression it
// stands for: thr >= lb_threshold (a bound above it is pruned), lim >=
// abandon_limit (a partial distance above it is abandoned), win >= the
// candidate window (1 + 3 delta) k-th best.  Larger limits prune, abandon and
// drop less, so the answer stays exact; FP64 arithmetic in every refining warp
// would load the GPU's few FP64 units.
__device__ __forceinline__ void limits_f32(const QCtl* c, unsigned long long kth, float& thr, float& lim,
                                           float& win) {
    if (kth == EMPTY_SLOT) {
        thr = lim = win = INFINITY;
        return;
    }
    const float t = key_d2(kth);
    const float r = __fadd_ru(__fsqrt_ru(__fmul_ru(t, c->f_lb)), c->f_E);
    thr = __fmul_ru(__fmul_ru(r, r), c->f_sq);
    lim = __fmul_ru(t, c->f_ab);
    win = __fmul_ru(t, c->f_win);
}

// squared distance of a row to the query, one warp, fixed order: every lane
// sums its elements left to right with fma, then a butterfly over lanes.
// n = 128 * NV: lane holds float4 p*32+lane.  Early abandon every 256 floats.
template <int NV>
__device__ __forceinline__ float warp_d2_vec(const float4* __restrict__ xr, const float4 (&qv)[NV],
                                             float abandon, bool& abandoned, int& nread) {
    const int lane = threadIdx.x & 31;
    float acc = 0.0f;
    abandoned = false;
    nread = NV * 128;
    if constexpr (NV <= 2) {
        float4 v[NV];
#pragma unroll
        for (int p = 0; p < NV; ++p) v[p] = ld_stream(xr + p * 32 + lane);
#pragma unroll
        for (int p = 0; p < NV; ++p) {
            float d;
            d = v[p].x - qv[p].x; acc = fmaf(d, d, acc);
            d = v[p].y - qv[p].y; acc = fmaf(d, d, acc);
            d = v[p].z - qv[p].z; acc = fmaf(d, d, acc);
            d = v[p].w - qv[p].w; acc = fmaf(d, d, acc);
        }
        return warp_sum_f(acc);
    } else {
#pragma unroll
    for (int p = 0; p < NV; p += 2) {
        float4 v0 = ld_stream(xr + p * 32 + lane);
        float4 v1 = ld_stream(xr + (p + 1) * 32 + lane);
        float d;
        d = v0.x - qv[p].x; acc = fmaf(d, d, acc);
        d = v0.y - qv[p].y; acc = fmaf(d, d, acc);
        d = v0.z - qv[p].z; acc = fmaf(d, d, acc);
        d = v0.w - qv[p].w; acc = fmaf(d, d, acc);
        d = v1.x - qv[p + 1].x; acc = fmaf(d, d, acc);
        d = v1.y - qv[p + 1].y; acc = fmaf(d, d, acc);
        d = v1.z - qv[p + 1].z; acc = fmaf(d, d, acc);
        d = v1.w - qv[p + 1].w; acc = fmaf(d, d, acc);
        if (p + 2 < NV) {
            float part = warp_sum_f(acc);
            if (part > abandon) {
                abandoned = true;
                nread = (p + 2) * 128;
                return part;
            }
        }
    }
    return warp_sum_f(acc);
    }
}

// any n: lane sums elements lane, lane+32, ...; abandon check every 8 full rounds
__device__ __forceinline__ float warp_d2_gen(const float* __restrict__ xr, const float* __restrict__ q,
                                             int n, float abandon, bool& abandoned, int& nread) {
    const int lane = threadIdx.x & 31;
    float acc = 0.0f;
    abandoned = false;
    nread = n;
    for (int t = 0; 32 * t < n; ++t) {
        int j = 32 * t + lane;
        if (j < n) {
            float d = xr[j] - __ldg(q + j);
            acc = fmaf(d, d, acc);
        }
        if ((t & 7) == 7 && 32 * (t + 1) < n) {
            float part = warp_sum_f(acc);
            if (part > abandon) {
                abandoned = true;
                nread = 32 * (t + 1);
                return part;
            }
        }
    }
    return warp_sum_f(acc);
}

// nread: the row's floats read (fewer than n when abandoned)
template <int NV>
__device__ __forceinline__ float warp_d2(const DevIndex& ix, int64_t r, const float4 (&qv)[NV ? NV : 1],
                                         const float* q, float abandon, bool& abandoned, int& nread) {
    if constexpr (NV > 0) {
        return warp_d2_vec<NV>(reinterpret_cast<const float4*>(ix.x + r * ix.n), qv, abandon,
                               abandoned, nread);
    } else {
        return warp_d2_gen(ix.x + r * ix.n, q, ix.n, abandon, abandoned, nread);
    }
}

template <int NV>
__device__ __forceinline__ void load_q(const float* q, float4 (&qv)[NV ? NV : 1]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int p = 0; p < (NV ? NV : 1); ++p)
        qv[p] = NV ? reinterpret_cast<const float4*>(q)[p * 32 + lane] : make_float4(0, 0, 0, 0);
}

// series lower bound for any cardinality: 16 table lookups (row stride card)
// summed in segment order; the 256-symbol scan has its own form (lb_word256)
__device__ __forceinline__ float series_lb(uint4 w, const float* __restrict__ tab, int card) {
    float lb = 0.0f;
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < W; ++i) {
        uint32_t s = (words[i >> 2] >> (8 * (i & 3))) & 255u;
        lb += tab[i * card + s];
    }
    return lb;
}

// work items of the scan: a queued leaf is cut into pieces of at most LB_PIECE
// rows, item = {first row, rows | 1 << 31 on the leaf's first piece}
constexpr int LB_PIECE = 128;
__device__ __forceinline__ uint32_t leaf_pieces(const DevIndex& ix, int64_t l) {
    const uint32_t size = ix.leaf_begin[l + 1] - ix.leaf_begin[l];
    return (size + LB_PIECE - 1) / LB_PIECE;
}
// the pieces of the leaf holding positions [b, e)
__device__ __forceinline__ void put_pieces_of(const QueryScratch& s, uint32_t b, uint32_t e, uint32_t at,
                                              uint32_t n_pieces, uint32_t cap) {
    for (uint32_t ch = 0; ch < n_pieces && at + ch < cap; ++ch) {
        const uint32_t r = b + ch * LB_PIECE;
        const uint32_t rows = e - r < (uint32_t)LB_PIECE ? e - r : (uint32_t)LB_PIECE;
        s.work[at + ch] = make_uint2(r, rows | (ch == 0 ? 0x80000000u : 0u));
    }
}
__device__ __forceinline__ void put_pieces(const DevIndex& ix, const QueryScratch& s, int64_t l, uint32_t at,
                                           uint32_t n_pieces, uint32_t cap) {
    const uint32_t b = (uint32_t)ix.leaf_begin[l], e = (uint32_t)ix.leaf_begin[l + 1];
    for (uint32_t ch = 0; ch < n_pieces && at + ch < cap; ++ch) {
        const uint32_t r = b + ch * LB_PIECE;
        const uint32_t rows = e - r < (uint32_t)LB_PIECE ? e - r : (uint32_t)LB_PIECE;
        s.work[at + ch] = make_uint2(r, rows | (ch == 0 ? 0x80000000u : 0u));
    }
}

// ---------------------------------------------------------------- q_prep
constexpr int PREP_THREADS = 256;

// Balanced-split index: the leaf a word descends to (root child of its 16-bit
// key, then at each node the child of the word's next bit on the node's split
// segment), or -1 when no series has that root key.
__device__ int32_t tree_leaf(const DevIndex& ix, const int* qsym) {
    unsigned root = 0;
    for (int i = 0; i < W; ++i) root = (root << 1) | ((unsigned)(qsym[i] >> (ix.cbits - 1)) & 1u);
    int32_t g = ix.tree_root[root];
    if (g < 0) return -1;
    int bits[W];
    for (int i = 0; i < W; ++i) bits[i] = 1;
    for (int depth = 0; depth <= W * 8; ++depth) {
        const int2 t = ix.tree[g];
        if (t.x < 0) return -1 - t.x;
        const int sg = t.y;
        if (sg < 0 || sg >= W || bits[sg] >= ix.cbits) return -1;
        const int b = (qsym[sg] >> (ix.cbits - 1 - bits[sg])) & 1;
        ++bits[sg];
        g = t.x + b;
    }
    return -1;
}

// One query's preparation by one CTA of PREP_THREADS threads; `neighbors`
// leaves on each side of the descent leaf join the approximate answer.
__device__ __forceinline__ void q_prep_body(const DevIndex& ix, const QueryScratch& s, int k,
                                            int neighbors) {
    __shared__ float bp[MAX_CARD + 1];
    __shared__ float qv[MAX_LEN];
    __shared__ float qpaa[W];
    __shared__ int qsym[W];
    __shared__ float red[32];
    __shared__ unsigned bad;
    __shared__ unsigned cnt_s;
    __shared__ unsigned long long key_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = ix.n, m = n / W, card = ix.card;
    for (int i = tid; i <= card; i += PREP_THREADS) bp[i] = ix.bp[i];
    for (int j = tid; j < n; j += PREP_THREADS) qv[j] = s.q[j];
    if (tid == 0) {
        bad = 0;
        cnt_s = 0;
    }
    // reset the per-query state left by the previous query
    for (int i = tid; i < k; i += PREP_THREADS) s.topk[i] = EMPTY_SLOT;
    for (int i = tid; i < NBINS; i += PREP_THREADS) {
        s.bin_count[i] = 0;
        s.bin_cursor[i] = 0;
    }
    __syncthreads();
    float amax = 0.0f;
    for (int j = tid; j < n; j += PREP_THREADS) amax = fmaxf(amax, fabsf(qv[j]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, off));
    if (lane == 0) red[warp] = amax;
    if (tid < W) {
        float sum = 0.0f;
        for (int j = 0; j < m; ++j) sum += qv[tid * m + j];
        const float p = sum / (float)m;
        qpaa[tid] = p;
        qsym[tid] = symbol_of(p, bp, card);
        if (!isfinite(p)) atomicOr(&bad, 1u);
    }
    __syncthreads();
    // lower-bound table T[i][s] = m * dist(qpaa_i, [bp[s], bp[s+1]))^2
    const float mf = (float)m;
    for (int e = tid; e < W * card; e += PREP_THREADS) {
        const int i = e / card, sym = e - i * card;
        const float lo = bp[sym], hi = bp[sym + 1], v = qpaa[i];
        const float d = v < lo ? lo - v : (v >= hi ? v - hi : 0.0f);
        s.table[e] = (d * d) * mf;
    }

    if (tid == 0) {
        unsigned long long key = 0;
        for (int pl = 0; pl < 4; ++pl) {
            const int b = ix.cbits - 1 - pl;
            unsigned plane = 0;
            for (int i = 0; i < W; ++i)
                plane = (plane << 1) | (b >= 0 ? ((unsigned)(qsym[i] >> b) & 1u) : 0u);
            key = (key << 16) | plane;
        }
        key_s = key;
    }
    __syncthreads();
    // descent: the last leaf whose first key <= the query key.  Keys are
    // sorted: count the samples at stride `step` that are <= key, then count
    // inside the one stride that holds the boundary.  A balanced-split index
    // keeps only the root key (the top 16 bits) in leaf_key: the search finds
    // the last leaf of the query's root child, and the tree descent below
    // refines it.
    const unsigned long long key = ix.tree ? (key_s & 0xFFFF000000000000ull) : key_s;
    const int64_t L = ix.L;
    const int64_t step = (L + PREP_THREADS - 1) / PREP_THREADS;
    const int64_t si = (int64_t)tid * step;
    const int c1 = __syncthreads_count(si < L && ix.leaf_key[si] <= key);
    const int64_t lo = c1 > 0 ? (int64_t)(c1 - 1) * step : 0;
    const int64_t hi = lo + step < L ? lo + step : L;
    unsigned cnt = 0;
    for (int64_t j = lo + tid; j < hi; j += PREP_THREADS) cnt += ix.leaf_key[j] <= key ? 1u : 0u;
    if (cnt) atomicAdd(&cnt_s, cnt);
    __syncthreads();
    if (tid == 0) {
        float qmax = 0.0f;
        for (int i = 0; i < PREP_THREADS / 32; ++i) qmax = fmaxf(qmax, red[i]);
        QCtl* c = s.ctl;
        c->qkey = key;
        const int64_t ub = lo + cnt_s;
        int64_t dl = ub > 0 ? ub - 1 : 0;
        if (ix.tree) {
            const int32_t t = tree_leaf(ix, qsym);
            if (t >= 0 && t < L) dl = t;
        }
        // approximate-answer range: that leaf and its APPROX_NEIGHBORS neighbours on
        // each side in key order (the nearest iSAX words), widened until it holds
        // >= k series
        int64_t a0 = dl - neighbors > 0 ? dl - neighbors : 0;
        int64_t a1 = dl + 1 + neighbors < L ? dl + 1 + neighbors : L;
        int64_t tot = (int64_t)ix.leaf_begin[a1] - ix.leaf_begin[a0];
        while (tot < k) {
            if (a1 < L) {
                tot += (int64_t)ix.leaf_begin[a1 + 1] - ix.leaf_begin[a1];
                ++a1;
            } else if (a0 > 0) {
                --a0;
                tot += (int64_t)ix.leaf_begin[a0 + 1] - ix.leaf_begin[a0];
            } else {
                break;
            }
        }
        c->approx_series = (unsigned long long)tot;
        c->descent_leaf = (int32_t)dl;
        c->approx_leaf = (int32_t)a0;
        c->approx_end = (int32_t)a1;
        c->work_count = 0;
        c->cand_count = 0;
        c->cand_base = 0;
        c->surv_count = 0;
        c->scan_done = 0;
        c->window = 0;
        c->flags = bad ? QF_NONFINITE : 0u;
        c->thr_lb0 = INFINITY;
        const double u = 0x1p-24;
        const double eps_x = 1.01 * (m + 1) * u * (double)ix.maxabs;
        const double eps_q = 1.01 * (m + 1) * u * (double)qmax;
        c->E = sqrt((double)n) * (eps_x + eps_q) * (1.0 + 1e-9);
        c->delta = (double)((n + 31) / 32 + 16) * u;
        set_limit_factors(c, c->delta, c->E);
        c->series_lb = 0;
        c->series_refined = 0;
        c->ed_floats = 0;
        c->leaves_scanned = 0;
        c->leaves_queued = 0;
        for (int i = 0; i < W; ++i) {
            c->qsym[i] = (uint8_t)qsym[i];
            c->qpaa[i] = qpaa[i];
        }

    }
}

__global__ void __launch_bounds__(PREP_THREADS) q_prep_kernel(DevIndex ix, QueryScratch s, int k) {
    q_prep_body(ix, s, k, APPROX_NEIGHBORS);
}
// a batch: query blockIdx.y
__global__ void __launch_bounds__(PREP_THREADS) bq_prep_kernel(DevIndex ix, const QueryScratch* ss,
                                                                int k, int neighbors) {
    q_prep_body(ix, ss[blockIdx.y], k, neighbors);
}

// ---------------------------------------------------------------- q_approx
template <int NV>
__device__ __forceinline__ void q_approx_body(const DevIndex& ix, const QueryScratch& s, int k) {
    const QCtl* c = s.ctl;
    if (c->flags & QF_NONFINITE) return;
    const int lane = threadIdx.x & 31;
    float4 qv[NV ? NV : 1];
    load_q<NV>(s.q, qv);
    const int64_t b = ix.leaf_begin[c->approx_leaf], e = ix.leaf_begin[c->approx_end];
    const double delta = c->delta;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long refined = 0;
    for (int64_t p = b + gw; p < e; p += nw) {
        bool ab;
        int nread;
        const uint32_t r = row_at(ix, p);
        const float d2 = warp_d2<NV>(ix, r, qv, s.q, INFINITY, ab, nread);
        if (lane == 0) {
            const unsigned long long kth = ld_volatile_u64(&s.topk[k - 1]);
            if (kth == EMPTY_SLOT || (double)d2 <= (double)key_d2(kth) * (1.0 + 3.0 * delta))
                consider(s, k, pack_key(d2, ix.orig[p]), r, delta);
        }
        ++refined;
    }
    if (lane == 0 && refined) {
        atomicAdd(&s.ctl->series_refined, refined);
        atomicAdd(&s.ctl->ed_floats, refined * (unsigned long long)ix.n);
    }
}
template <int NV>
__global__ void __launch_bounds__(256) q_approx_kernel(DevIndex ix, QueryScratch s, int k) {
    q_approx_body<NV>(ix, s, k);
}
template <int NV>
__global__ void __launch_bounds__(256) bq_approx_kernel(DevIndex ix, const QueryScratch* ss, int k) {
    q_approx_body<NV>(ix, ss[blockIdx.y], k);
}

// ---------------------------------------------------------------- q_leaf_lb
// Envelope bound of every leaf from the breakpoints and the query PAA: per
// segment the table entry of the envelope edge nearer the query (the same
// fp32 expression as the table), 0 when the query's symbol lies inside.
__device__ __forceinline__ void q_leaf_lb_body(const DevIndex& ix, const QueryScratch& s, int k) {
    __shared__ float bp[MAX_CARD + 1];
    __shared__ uint32_t hist[NBINS];
    __shared__ float thr_s;
    const QCtl* c = s.ctl;
    if (c->flags & QF_NONFINITE) return;
    const int card = ix.card;
    for (int i = threadIdx.x; i <= card; i += blockDim.x) bp[i] = ix.bp[i];
    for (int i = threadIdx.x; i < NBINS; i += blockDim.x) hist[i] = 0;
    if (threadIdx.x == 0) thr_s = lb_threshold(ld_volatile_u64(&s.topk[k - 1]), c->delta, c->E);
    __syncthreads();
    float qp[W];
    int qs[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
        qp[i] = c->qpaa[i];
        qs[i] = c->qsym[i];
    }
    const float mf = (float)(ix.n / W);
    const int64_t a0 = c->approx_leaf, a1 = c->approx_end;
    const float thr = thr_s;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < ix.L;
         l += (int64_t)gridDim.x * blockDim.x) {
        const uint4 mn = ix.env[2 * l], mx = ix.env[2 * l + 1];
        const uint32_t wn[4] = {mn.x, mn.y, mn.z, mn.w}, wx[4] = {mx.x, mx.y, mx.z, mx.w};
        float lb = 0.0f;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int lo = (wn[i >> 2] >> (8 * (i & 3))) & 255, hi = (wx[i >> 2] >> (8 * (i & 3))) & 255;
            if (qs[i] < lo) {
                const float d = bp[lo] - qp[i];
                lb += (d * d) * mf;
            } else if (qs[i] > hi) {
                const float d = qp[i] - bp[hi + 1];
                lb += (d * d) * mf;
            }
        }
        s.leaf_lb[l] = lb;
        if (!(l >= a0 && l < a1) && lb <= thr) atomicAdd(&hist[bin_of(lb, thr)], leaf_pieces(ix, l));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NBINS; i += blockDim.x)
        if (hist[i]) atomicAdd(&s.bin_count[i], hist[i]);
}
__global__ void __launch_bounds__(256) q_leaf_lb_kernel(DevIndex ix, QueryScratch s, int k) {
    q_leaf_lb_body(ix, s, k);
}
// the same for a batch of queries, grid.y = query
__global__ void __launch_bounds__(256) bq_leaf_lb_kernel(DevIndex ix, const QueryScratch* ss, int k) {
    q_leaf_lb_body(ix, ss[blockIdx.y], k);
}

// ---------------------------------------------------------------- q_leaf_scatter
__device__ __forceinline__ void q_leaf_scatter_body(const DevIndex& ix, const QueryScratch& s, int k) {
    __shared__ uint32_t off[NBINS];
    __shared__ uint32_t scratch[32];
    __shared__ float thr_s;
    QCtl* c = s.ctl;
    if (c->flags & QF_NONFINITE) return;
    uint32_t tot;
    uint32_t o = block_excl_scan<uint32_t>(s.bin_count[threadIdx.x], 0u, OpAdd<uint32_t>(), scratch, &tot);
    off[threadIdx.x] = o;
    if (threadIdx.x == 0) thr_s = lb_threshold(ld_volatile_u64(&s.topk[k - 1]), c->delta, c->E);
    __syncthreads();
    const float thr = thr_s;
    const int64_t a0 = c->approx_leaf, a1 = c->approx_end;
    uint32_t mine = 0;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < ix.L;
         l += (int64_t)gridDim.x * blockDim.x) {
        if (l >= a0 && l < a1) continue;
        const float lb = s.leaf_lb[l];
        if (lb <= thr) {
            const int b = bin_of(lb, thr);
            const uint32_t nch = leaf_pieces(ix, l);
            const uint32_t p = off[b] + atomicAdd(&s.bin_cursor[b], nch);
            put_pieces(ix, s, l, p, nch, tot < s.work_cap ? tot : s.work_cap);
            ++mine;
        }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) mine += __shfl_xor_sync(FULL, mine, o2);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&c->leaves_queued, (unsigned long long)mine);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->work_count = tot < s.work_cap ? tot : s.work_cap;
        if (tot > s.work_cap) atomicOr(&c->flags, QF_OVERFLOW);
        c->thr_lb0 = thr;
        c->thr_scan = thr;
    }
}
__global__ void __launch_bounds__(NBINS) q_leaf_scatter_kernel(DevIndex ix, QueryScratch s, int k) {
    q_leaf_scatter_body(ix, s, k);
}
__global__ void __launch_bounds__(NBINS) bq_leaf_scatter_kernel(DevIndex ix, const QueryScratch* ss, int k) {
    q_leaf_scatter_body(ix, ss[blockIdx.y], k);
}

// ---------------------------------------------------------------- q_flat_list
// The ParIS way of answering (Section III, ParIS+ query answering: the lower
// bound of every series in the SAX array, then the real distance of those it
// does not prune): every leaf goes on the work list, in storage order, with
// bound 0 and all in the first bin, so the scan bounds every series and never
// stops early nor skips a leaf.  The approximate-answer leaves stay out.
__global__ void __launch_bounds__(256) q_flat_list_kernel(DevIndex ix, QueryScratch s, int k) {
    QCtl* c = s.ctl;
    if (c->flags & QF_NONFINITE) return;
    const int lane = threadIdx.x & 31;
    const int64_t a0 = c->approx_leaf, a1 = c->approx_end;
    // a warp lists 32 consecutive leaves with one append
    for (int64_t l0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; l0 < ix.L;
         l0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = l0 + lane;
        const bool take = l < ix.L && !(l >= a0 && l < a1);
        const uint32_t nch = take ? leaf_pieces(ix, l) : 0u;
        uint32_t incl = nch;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += v;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        const unsigned leaves = __popc(__ballot_sync(FULL, take));
        uint32_t base = 0;
        if (lane == 0 && total) {
            base = atomicAdd(&c->work_count, total);
            atomicAdd(&c->leaves_queued, (unsigned long long)leaves);
        }
        base = __shfl_sync(FULL, base, 0);
        if (nch) put_pieces(ix, s, l, base + incl - nch, nch, 0xFFFFFFFFu);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->thr_lb0 = 0.0f;
        c->thr_scan = lb_threshold(ld_volatile_u64(&s.topk[k - 1]), c->delta, c->E);
    }
}

// ---------------------------------------------------------------- refinement helpers
constexpr int SR_BATCH = 8;  // refined distances per k-best update

// squared distances of two rows (second one optional) with all loads issued first
template <int NV>
__device__ __forceinline__ void warp_d2_two(const DevIndex& ix, int64_t r0, int64_t r1, bool two,
                                            const float4 (&qv)[NV], float& d0, float& d1) {
    const int lane = threadIdx.x & 31;
    const float4* x0 = reinterpret_cast<const float4*>(ix.x + r0 * ix.n);
    const float4* x1 = reinterpret_cast<const float4*>(ix.x + (two ? r1 : r0) * ix.n);
    float4 v0[NV], v1[NV];
#pragma unroll
    for (int p = 0; p < NV; ++p) {
        v0[p] = ld_stream(x0 + p * 32 + lane);
        v1[p] = two ? ld_stream(x1 + p * 32 + lane) : v0[p];
    }
    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
    for (int p = 0; p < NV; ++p) {
        float d;
        d = v0[p].x - qv[p].x; a0 = fmaf(d, d, a0);
        d = v0[p].y - qv[p].y; a0 = fmaf(d, d, a0);
        d = v0[p].z - qv[p].z; a0 = fmaf(d, d, a0);
        d = v0[p].w - qv[p].w; a0 = fmaf(d, d, a0);
        d = v1[p].x - qv[p].x; a1 = fmaf(d, d, a1);
        d = v1[p].y - qv[p].y; a1 = fmaf(d, d, a1);
        d = v1[p].z - qv[p].z; a1 = fmaf(d, d, a1);
        d = v1[p].w - qv[p].w; a1 = fmaf(d, d, a1);
    }
    d0 = warp_sum_f(a0);
    d1 = warp_sum_f(a1);
}

// squared distances of up to four rows (keep mask, warp-uniform), every load
// issued before any arithmetic; the same fp32 order as warp_d2_vec
template <int NV>
__device__ __forceinline__ void warp_d2_four(const DevIndex& ix, const uint2 (&e)[4], unsigned keep,
                                             const float4 (&qv)[NV], float (&d)[4]) {
    const int lane = threadIdx.x & 31;
    float4 v[4][NV];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (keep & (1u << t)) {
            const float4* x = reinterpret_cast<const float4*>(ix.x + (int64_t)e[t].x * ix.n);
#pragma unroll
            for (int p = 0; p < NV; ++p) v[t][p] = ld_stream(x + p * 32 + lane);
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        float a = 0.0f;
        if (keep & (1u << t)) {
#pragma unroll
            for (int p = 0; p < NV; ++p) {
                float dd;
                dd = v[t][p].x - qv[p].x; a = fmaf(dd, dd, a);
                dd = v[t][p].y - qv[p].y; a = fmaf(dd, dd, a);
                dd = v[t][p].z - qv[p].z; a = fmaf(dd, dd, a);
                dd = v[t][p].w - qv[p].w; a = fmaf(dd, dd, a);
            }
        }
        d[t] = warp_sum_f(a);
    }
}

// ---------------------------------------------------------------- q_front
// The query's preparation, approximate answer and leaf bounds in one launch
// (MESSI query answering, Section III: the approximate answer from the query's
// own leaf seeds the BSF; every leaf's envelope bound then decides whether the
// leaf is visited).  Every CTA computes the query's PAA, symbols and key and
// searches the descent leaf itself, with q_prep's expressions and search, so all
// CTAs find the same approximate-answer leaves; the grid's threads bound every
// leaf's envelope into leaf_lb (q_leaf_lb's expression) while its warps refine
// the approximate-answer rows, FR_ROWS rows per warp with one k-best update per
// warp.  CTA 0 writes the control block and the lower-bound table.  The k best,
// the candidate count and the refined count start each query cleared: the
// previous query's q_finalize leaves them so, and a new scratch is allocated so.
constexpr int FR_THREADS = 512, FR_WARPS = FR_THREADS / 32, FR_ROWS = 4, FR_LEAVES = 4, FR_KEYS = 4;

template <int NV>
__global__ void __launch_bounds__(FR_THREADS, 1) q_front_kernel(DevIndex ix, QueryScratch s, int k, int neighbors,
                                                              const QMail* mail) {
    __shared__ float bp[MAX_CARD + 1];
    __shared__ __align__(16) float qv[MAX_LEN];  // read as float4 below
    __shared__ float qpaa[W];
    __shared__ int qsym[W];
    __shared__ float red[FR_WARPS];
    __shared__ unsigned bad, cnt_s;
    __shared__ unsigned long long key_s;
    __shared__ int64_t range_s[2], spec_s[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = ix.n, m = n / W, card = ix.card;
    const bool lead = blockIdx.x == 0;
    // the envelopes of this thread's first FR_LEAVES leaves and the descent's
    // sample key do not depend on the query: they are brought into L2 (and the
    // sample read) first, while the query is read and summarised
    const int64_t L = ix.L;
    const int64_t stride = (int64_t)gridDim.x * FR_THREADS;
    const int64_t lfirst = (int64_t)blockIdx.x * FR_THREADS + tid;
#pragma unroll
    for (int u = 0; u < FR_LEAVES; ++u) {
        const int64_t l = lfirst + u * stride;
        if (l < L && (l & 3) == 0) prefetch_l2(ix.env + 2 * l);  // one 128-byte line per four leaves
    }
    const int64_t step = (L + FR_THREADS - 1) / FR_THREADS;
    const int64_t si = (int64_t)tid * step;
    const unsigned long long sample = si < L ? ix.leaf_key[si] : ~0ull;
    __shared__ const float* qsrc;
    if (tid == 0) {
        bad = 0;
        cnt_s = 0;
        // the query: where the index's mapped block says (CTA 0 also leaves it in
        // the scratch for the later kernels), else already in the scratch
        qsrc = mail ? mail->q_src : s.q;
    }
    for (int i = tid; i <= card; i += FR_THREADS) bp[i] = ix.bp[i];
    __syncthreads();
    for (int j = tid; j < n; j += FR_THREADS) {
        const float v = qsrc[j];
        qv[j] = v;
        if (lead && mail) s.q[j] = v;
    }
    if (lead) {
        // the binning step's counters and grid barrier start at zero
        for (int i = tid; i < NBINS; i += FR_THREADS) {
            s.bin_count[i] = 0;
            s.bin_cursor[i] = 0;
        }
        if (tid == 0) s.ctl->grid_sync = 0;
    }
    __syncthreads();
    float amax = 0.0f;
    for (int j = tid; j < n; j += FR_THREADS) amax = fmaxf(amax, fabsf(qv[j]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, off));
    if (lane == 0) red[warp] = amax;
    if (tid < W) {
        float sum = 0.0f;
        for (int j = 0; j < m; ++j) sum += qv[tid * m + j];
        const float p = sum / (float)m;
        qpaa[tid] = p;
        qsym[tid] = symbol_of(p, bp, card);
        if (!isfinite(p)) atomicOr(&bad, 1u);
    }
    __syncthreads();
    const float mf = (float)m;
    if (lead) {
        // lower-bound table T[i][s] = m * dist(qpaa_i, [bp[s], bp[s+1]))^2
        for (int e = tid; e < W * card; e += FR_THREADS) {
            const int i = e / card, sym = e - i * card;
            const float lo = bp[sym], hi = bp[sym + 1], v = qpaa[i];
            const float d = v < lo ? lo - v : (v >= hi ? v - hi : 0.0f);
            s.table[e] = (d * d) * mf;
        }
    }
    if (tid == 0) {
        unsigned long long key = 0;
        for (int pl = 0; pl < 4; ++pl) {
            const int b = ix.cbits - 1 - pl;
            unsigned plane = 0;
            for (int i = 0; i < W; ++i)
                plane = (plane << 1) | (b >= 0 ? ((unsigned)(qsym[i] >> b) & 1u) : 0u);
            key = (key << 16) | plane;
        }
        key_s = key;
    }
    __syncthreads();
    const unsigned long long key = ix.tree ? (key_s & 0xFFFF000000000000ull) : key_s;
    {
        // envelope bound of this thread's leaves (q_leaf_lb's expression); the
        // query's PAA and symbols are read from shared memory
        // FR_LEAVES leaves at a time, their envelopes all loaded before any bound
        for (int64_t l0 = lfirst; l0 < L; l0 += FR_LEAVES * stride) {
            uint4 mn[FR_LEAVES], mx[FR_LEAVES];
#pragma unroll
            for (int u = 0; u < FR_LEAVES; ++u) {
                const int64_t l = l0 + u * stride;
                if (l < L) {
                    mn[u] = ix.env[2 * l];
                    mx[u] = ix.env[2 * l + 1];
                }
            }
            // one leaf at a time through a short loop body (its code is fetched
            // once per query: a long unrolled body costs more in instruction
            // fetch than it saves); a segment inside the envelope adds +0, so
            // the sum is the per-segment expression's in segment order
#pragma unroll 1
            for (int u = 0; u < FR_LEAVES; ++u) {
                const int64_t l = l0 + u * stride;
                if (l >= L) break;
                uint4 a = mn[0], z = mx[0];
#pragma unroll
                for (int v = 1; v < FR_LEAVES; ++v)
                    if (u == v) {
                        a = mn[v];
                        z = mx[v];
                    }
                float lb = 0.0f;
#pragma unroll 1
                for (int g = 0; g < 4; ++g) {
                    const uint32_t wn = g == 0 ? a.x : g == 1 ? a.y : g == 2 ? a.z : a.w;
                    const uint32_t wx = g == 0 ? z.x : g == 1 ? z.y : g == 2 ? z.z : z.w;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int i = 4 * g + b;
                        const int lo = (wn >> (8 * b)) & 255, hi = (wx >> (8 * b)) & 255;
                        const int qsi = qsym[i];
                        const float qp = qpaa[i];
                        const float d = qsi < lo ? bp[lo] - qp : (qsi > hi ? qp - bp[hi + 1] : 0.0f);
                        lb += (d * d) * mf;
                    }
                }
                s.leaf_lb[l] = lb;
            }
        }
    }
    // descent: the last leaf whose first key <= the query key (q_prep's search).
    // The keys of the boundary's stride are read all at once, and with each key
    // the first positions of the leaves `neighbors` before and `neighbors` + 1
    // after it: the thread holding the descent leaf then knows the approximate
    // range's extent without another read.
    const int c1 = __syncthreads_count(si < L && sample <= key);
    const int64_t lo = c1 > 0 ? (int64_t)(c1 - 1) * step : 0;
    const int64_t hi = lo + step < L ? lo + step : L;
    if (tid == 0) spec_s[0] = spec_s[1] = -1;
    unsigned cnt = 0;
    int64_t mj[FR_KEYS];
    uint32_t mb0[FR_KEYS], mb1[FR_KEYS];
#pragma unroll
    for (int u = 0; u < FR_KEYS; ++u) mj[u] = -1;  // a thread past the stride holds no key
    for (int64_t j0 = lo + tid; j0 < hi; j0 += FR_KEYS * FR_THREADS) {
        unsigned long long kv[FR_KEYS];
#pragma unroll
        for (int u = 0; u < FR_KEYS; ++u) {
            const int64_t j = j0 + u * FR_THREADS;
            mj[u] = j;
            if (j < hi) {
                kv[u] = ix.leaf_key[j];
                const int64_t x0 = j - neighbors > 0 ? j - neighbors : 0;
                const int64_t x1 = j + 1 + neighbors < L ? j + 1 + neighbors : L;
                mb0[u] = ix.leaf_begin[x0];
                mb1[u] = ix.leaf_begin[x1];
            }
        }
#pragma unroll
        for (int u = 0; u < FR_KEYS; ++u) cnt += (mj[u] < hi && kv[u] <= key) ? 1u : 0u;
    }
    if (cnt) atomicAdd(&cnt_s, cnt);
    __syncthreads();
    {
        // the holder of the descent leaf publishes its range's extent
        const int64_t ub = lo + cnt_s;
        const int64_t dl = ub > 0 ? ub - 1 : 0;
        if (hi - lo <= (int64_t)FR_KEYS * FR_THREADS) {
#pragma unroll
            for (int u = 0; u < FR_KEYS; ++u)
                if (mj[u] == dl && dl >= lo && dl < hi) {
                    spec_s[0] = mb0[u];
                    spec_s[1] = mb1[u];
                }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const int64_t ub = lo + cnt_s;
        int64_t dl = ub > 0 ? ub - 1 : 0;
        bool known = spec_s[0] >= 0;  // the range's extent was read with the keys
        if (ix.tree) {
            const int32_t t = tree_leaf(ix, qsym);
            if (t >= 0 && t < L && t != dl) {
                dl = t;
                known = false;
            }
        }
        int64_t a0 = dl - neighbors > 0 ? dl - neighbors : 0;
        int64_t a1 = dl + 1 + neighbors < L ? dl + 1 + neighbors : L;
        int64_t b0 = known ? spec_s[0] : (int64_t)ix.leaf_begin[a0];
        int64_t b1 = known ? spec_s[1] : (int64_t)ix.leaf_begin[a1];
        int64_t tot = b1 - b0;
        while (tot < k) {
            if (a1 < L) {
                ++a1;
                b1 = ix.leaf_begin[a1];
            } else if (a0 > 0) {
                --a0;
                b0 = ix.leaf_begin[a0];
            } else {
                break;
            }
            tot = b1 - b0;
        }
        range_s[0] = b0;
        range_s[1] = b1;
        if (lead) {
            float qmax = 0.0f;
            for (int i = 0; i < FR_WARPS; ++i) qmax = fmaxf(qmax, red[i]);
            QCtl* c = s.ctl;
            c->qkey = key;
            c->approx_series = (unsigned long long)tot;
            c->cand_base = (uint32_t)tot;  // candidate slots of the approximate rows, by position
            c->descent_leaf = (int32_t)dl;
            c->approx_leaf = (int32_t)a0;
            c->approx_end = (int32_t)a1;
            c->work_count = 0;
            c->surv_count = 0;
            c->scan_done = 0;
            c->window = 0;
            c->flags = bad ? QF_NONFINITE : 0u;
            c->thr_lb0 = INFINITY;
            c->thr_scan = INFINITY;
            const double u = 0x1p-24;
            const double eps_x = 1.01 * (m + 1) * u * (double)ix.maxabs;
            const double eps_q = 1.01 * (m + 1) * u * (double)qmax;
            c->E = sqrt((double)n) * (eps_x + eps_q) * (1.0 + 1e-9);
            c->delta = (double)((n + 31) / 32 + 16) * u;
            set_limit_factors(c, c->delta, c->E);
            c->series_lb = 0;
            c->ed_floats = (unsigned long long)tot * (unsigned long long)n;  // the approximate rows, read whole
            c->leaves_scanned = 0;
            c->leaves_queued = 0;
            for (int i = 0; i < W; ++i) {
                c->qsym[i] = (uint8_t)qsym[i];
                c->qpaa[i] = qpaa[i];
            }
        }
    }
    __syncthreads();
    if (bad) return;  // a non-finite query: CTA 0 has flagged it
    // approximate answer: the rows of the approximate-answer leaves, FR_ROWS
    // consecutive positions per warp at a time
    const int64_t b = range_s[0], e = range_s[1];
    ISAX_CHECK(0 <= b && b <= e && e <= ix.N, CHK_APPROX_RANGE);
    constexpr int NQ = NV ? NV : 1;
    float4 qr[NQ];
#pragma unroll
    for (int p = 0; p < NQ; ++p)
        qr[p] = NV ? reinterpret_cast<const float4*>(qv)[p * 32 + lane] : make_float4(0, 0, 0, 0);
    const int64_t gw = (int64_t)blockIdx.x * FR_WARPS + warp, nw = (int64_t)gridDim.x * FR_WARPS;
    unsigned long long refined = 0;
    for (int64_t p0 = b + gw * FR_ROWS; p0 < e; p0 += nw * FR_ROWS) {
        const int R = e - p0 < FR_ROWS ? (int)(e - p0) : FR_ROWS;
        uint2 rw[4];
        uint32_t my_id = 0, my_row = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t p = p0 + (t < R ? t : 0);
            rw[t] = make_uint2(row_at(ix, p), 0u);
        }
        if (lane < R) {
            my_id = ix.orig[p0 + lane];
            my_row = rw[0].x;
#pragma unroll
            for (int t = 1; t < 4; ++t)
                if (lane == t) my_row = rw[t].x;
        }
        float d[4];
        if constexpr (NV > 0 && NV <= 2) {
            warp_d2_four<NQ>(ix, rw, (1u << R) - 1u, qr, d);
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                bool ab;
                int nread;
                d[t] = t < R ? warp_d2<NV>(ix, (int64_t)rw[t].x, qr, s.q, INFINITY, ab, nread) : 0.0f;
            }
        }
        float my_d2 = d[0];
#pragma unroll
        for (int t = 1; t < 4; ++t)
            if (lane == t) my_d2 = d[t];
        // the k best: for k = 1 one atomicMin per row (its result is not needed);
        // for larger k the rows under the current k-th best go through the
        // insertion cascade.  Every approximate row is a candidate for the final
        // ordering, in the slot of its position (q_finalize keeps those within
        // the final window).
        const unsigned long long my_key = pack_key(my_d2, my_id);
        if (k == 1) {
            if (lane < R) atomicMin(&s.topk[0], my_key);
        } else {
            unsigned long long kth = 0;
            if (lane == 0) kth = ld_volatile_u64(&s.topk[k - 1]);
            kth = __shfl_sync(FULL, kth, 0);
            if (lane < R && my_key < kth) topk_insert(s.topk, k, my_key);
        }
        if (lane < R) {
            const int64_t slot = p0 + lane - b;
            if (slot < (int64_t)s.cand_cap) {
                s.cand_key[slot] = my_key;
                s.cand_pos[slot] = my_row;
            }
        }
        refined += (unsigned long long)R;
    }
    if (lane == 0 && refined) atomicAdd(&s.ctl->series_refined, refined);
}

// ---------------------------------------------------------------- q_leaf_bin
// The leaves the approximate answer does not prune, listed bin by bin of
// bound / BSF (MESSI's priority queues): a cooperative launch of G CTAs.  Each
// CTA counts its leaves' pieces into the bins, the counts are summed over the
// grid, and after a grid barrier every CTA places its leaves' pieces at their
// bin's offset (the work list of q_leaf_lb + q_leaf_scatter, in one launch).
// The barrier waits at most GRID_WAIT polls; a barrier that gives up flags the
// query QF_STALLED and the list is left empty.
constexpr int BIN_THREADS = 512, BIN_LEAVES = 4;
constexpr uint32_t GRID_WAIT = 1u << 22;

__global__ void __launch_bounds__(BIN_THREADS) q_leaf_bin_kernel(DevIndex ix, QueryScratch s, int k) {
    __shared__ uint32_t hist[NBINS];
    __shared__ uint32_t off[NBINS];
    __shared__ uint32_t scratch[32];
    __shared__ float thr_s;
    __shared__ int ok_s;
    QCtl* c = s.ctl;
    const int tid = threadIdx.x;
    const uint32_t flags = c->flags;
    const int64_t a0 = c->approx_leaf, a1 = c->approx_end;
    for (int i = tid; i < NBINS; i += BIN_THREADS) hist[i] = 0;
    if (tid == 0) thr_s = lb_threshold(ld_volatile_u64(&s.topk[k - 1]), c->delta, c->E);
    __syncthreads();
    const float thr = thr_s;
    const bool skip = (flags & QF_NONFINITE) != 0;
    const int64_t L = ix.L, stride = (int64_t)gridDim.x * BIN_THREADS;
    const int64_t first = (int64_t)blockIdx.x * BIN_THREADS + tid;
    // BIN_LEAVES leaves at a time, all loads issued first: bound (bin, or -1 when
    // the leaf is not queued) and pieces; the first group stays in registers for
    // the placement after the barrier
    int bin0[BIN_LEAVES];
    uint32_t nch0[BIN_LEAVES], b0[BIN_LEAVES], e0[BIN_LEAVES];
    auto load_group = [&](int64_t l0, int (&bn)[BIN_LEAVES], uint32_t (&nc)[BIN_LEAVES], uint32_t (&b)[BIN_LEAVES],
                          uint32_t (&e)[BIN_LEAVES]) {
        float lb[BIN_LEAVES];
#pragma unroll
        for (int u = 0; u < BIN_LEAVES; ++u) {
            const int64_t l = l0 + u * stride;
            if (l < L) {
                lb[u] = s.leaf_lb[l];
                b[u] = ix.leaf_begin[l];
                e[u] = ix.leaf_begin[l + 1];
            }
        }
#pragma unroll
        for (int u = 0; u < BIN_LEAVES; ++u) {
            const int64_t l = l0 + u * stride;
            ISAX_CHECK(l >= L || b[u] < e[u], CHK_LEAF_RANGE);
            const bool q = l < L && !(l >= a0 && l < a1) && lb[u] <= thr;
            bn[u] = q ? bin_of(lb[u], thr) : -1;
            nc[u] = q ? (e[u] - b[u] + LB_PIECE - 1) / LB_PIECE : 0u;
        }
    };
    if (!skip) {
        for (int64_t l0 = first; l0 < L; l0 += BIN_LEAVES * stride) {
            int bn[BIN_LEAVES];
            uint32_t nc[BIN_LEAVES], b[BIN_LEAVES], e[BIN_LEAVES];
            load_group(l0, bn, nc, b, e);
#pragma unroll
            for (int u = 0; u < BIN_LEAVES; ++u) {
                if (bn[u] >= 0) atomicAdd(&hist[bn[u]], nc[u]);
                if (l0 == first) {
                    bin0[u] = bn[u];
                    nch0[u] = nc[u];
                    b0[u] = b[u];
                    e0[u] = e[u];
                }
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < NBINS; i += BIN_THREADS)
        if (hist[i]) atomicAdd(&s.bin_count[i], hist[i]);
    // grid barrier: every CTA's counts are in bin_count
    const bool met = grid_barrier(&c->grid_sync, gridDim.x, GRID_WAIT, &ok_s);
    if (!met && tid == 0) atomicOr(&c->flags, QF_STALLED);
    if (!met || skip) {
        if (blockIdx.x == 0 && tid == 0) c->work_count = 0;
        return;
    }
    uint32_t tot;
    const uint32_t cnt = tid < NBINS ? ld_volatile_u32(&s.bin_count[tid]) : 0u;
    const uint32_t o = block_excl_scan<uint32_t>(cnt, 0u, OpAdd<uint32_t>(), scratch, &tot);
    if (tid < NBINS) off[tid] = o;
    __syncthreads();
    const uint32_t cap = tot < s.work_cap ? tot : s.work_cap;
    uint32_t mine = 0;
    for (int64_t l0 = first; l0 < L; l0 += BIN_LEAVES * stride) {
        int bn[BIN_LEAVES];
        uint32_t nc[BIN_LEAVES], b[BIN_LEAVES], e[BIN_LEAVES];
        if (l0 == first) {
#pragma unroll
            for (int u = 0; u < BIN_LEAVES; ++u) {
                bn[u] = bin0[u];
                nc[u] = nch0[u];
                b[u] = b0[u];
                e[u] = e0[u];
            }
        } else {
            load_group(l0, bn, nc, b, e);
        }
#pragma unroll
        for (int u = 0; u < BIN_LEAVES; ++u) {
            if (bn[u] < 0) continue;
            const uint32_t p = off[bn[u]] + atomicAdd(&s.bin_cursor[bn[u]], nc[u]);
            put_pieces_of(s, b[u], e[u], p, nc[u], cap);
            ++mine;
        }
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) mine += __shfl_xor_sync(FULL, mine, o2);
    if ((tid & 31) == 0 && mine) atomicAdd(&c->leaves_queued, (unsigned long long)mine);
    if (blockIdx.x == 0 && tid == 0) {
        c->work_count = cap;
        if (tot > s.work_cap) atomicOr(&c->flags, QF_OVERFLOW);
        c->thr_lb0 = thr;
        c->thr_scan = thr;
    }
}

// ---------------------------------------------------------------- refinement inside the scan
// MESSI's workers compute a series' real distance as soon as its lower bound
// falls below the BSF, in the same pass over the queued leaves (Section III).
// Here the scan warps publish their survivors into the list as the separate
// refinement would read them, and a warp with no piece left turns to refining.
// The list is cut into chunks of RQ_CHUNK slots dealt to the CTAs in turn
// (chunk j to CTA j mod G); a CTA's warps take its slots RQ_UNIT at a time from
// a shared-memory counter, and wait (bounded) until each slot is filled, or the
// scan is over in every CTA and the slot lies past the last survivor.  Each
// slot taken goes back empty, so the list starts the next query empty.  A
// survivor whose bound exceeds the threshold of the current k-th best is
// skipped without reading its row; the others get the fp32 distance of the
// separate refinement (the same order of sums).
constexpr uint32_t RQ_WAIT = 1u << 21;      // polls of one slot before the wait gives up
constexpr uint32_t RQ_CHUNK = 64;           // list slots per chunk
constexpr uint32_t RQ_UNIT = 8;             // slots a warp takes at once
constexpr int RQ_KT_LANE = RQ_UNIT < 32 ? (int)RQ_UNIT : 0;  // the lane that reads the k-th best
static_assert(RQ_UNIT <= 32 && RQ_CHUNK % RQ_UNIT == 0, "a unit is at most a warp's lanes and divides a chunk");
constexpr uint32_t RQ_ROW = 1024;           // bytes of a row of n = 256
constexpr uint32_t RQ_BAR_WAIT = 1u << 22;  // bounded wait on a staged row copy
constexpr int RQ_DEPTH = 3;                 // pairs of rows in flight per warp (n = 256)

// squared distance of a row to the query (n = 128 * nv, query read through
// the read-only cache): warp_d2_vec's order and early abandon
__device__ __forceinline__ float warp_d2_v4q(const float4* __restrict__ xr, const float4* __restrict__ q, int nv,
                                             float abandon, bool& abandoned, int& nread) {
    const int lane = threadIdx.x & 31;
    float acc = 0.0f;
    abandoned = false;
    nread = nv * 128;
    for (int p = 0; p < nv; p += 2) {
        const bool two = p + 1 < nv;
        const float4 v0 = ld_stream(xr + p * 32 + lane);
        const float4 v1 = two ? ld_stream(xr + (p + 1) * 32 + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q0 = __ldg(q + p * 32 + lane);
        float d;
        d = v0.x - q0.x; acc = fmaf(d, d, acc);
        d = v0.y - q0.y; acc = fmaf(d, d, acc);
        d = v0.z - q0.z; acc = fmaf(d, d, acc);
        d = v0.w - q0.w; acc = fmaf(d, d, acc);
        if (two) {
            const float4 q1 = __ldg(q + (p + 1) * 32 + lane);
            d = v1.x - q1.x; acc = fmaf(d, d, acc);
            d = v1.y - q1.y; acc = fmaf(d, d, acc);
            d = v1.z - q1.z; acc = fmaf(d, d, acc);
            d = v1.w - q1.w; acc = fmaf(d, d, acc);
        }
        if (p + 2 < nv) {
            const float part = warp_sum_f(acc);
            if (part > abandon) {
                abandoned = true;
                nread = (p + 2) * 128;
                return part;
            }
        }
    }
    return warp_sum_f(acc);
}

// The refining phase of one warp of CTA `cta` of G.  fz: the CTA's shared
// words [the scan is over everywhere, polling token, units taken].  A warp
// takes RQ_UNIT slots at a time (one lane each); their kept rows queue in the
// lanes and are refined in turn.  HALF (n = 256, rows in device memory): each
// pair of rows is staged whole in the warp's own copy ring (free once its scan
// is done: wbuf, 6 KB = RQ_DEPTH buffers of two rows, with its barriers wbar,
// whose next waits have the parities in the bits of `par`) by asynchronous
// copies, RQ_DEPTH pairs in flight, and the query is read from its copy q_sm
// in shared memory.
template <bool HALF>
__device__ __forceinline__ void q_refine_claimed(const DevIndex& ix, const QueryScratch& s, int k, uint32_t cta,
                                                 uint32_t G, uint32_t* fz, unsigned char* wbuf, uint64_t* wbar,
                                                 uint32_t par, const float* q_sm) {
    QCtl* c = s.ctl;
    const int lane = threadIdx.x & 31;
    const uint64_t cap = s.surv_cap;
    const float4* q4 = reinterpret_cast<const float4*>(s.q);  // read through the read-only cache
    unsigned long long kth = 0ull;
    float thr = INFINITY, lim = INFINITY, win = INFINITY;
    unsigned long long n_ref = 0, n_floats = 0;
    float my_d2 = INFINITY;
    uint32_t my_pos = 0;
    int nb = 0;
    auto flush = [&]() {
        if (nb == 0) return;
        if (lane < nb && my_d2 <= win) consider(s, k, pack_key(my_d2, id_of_row(ix, my_pos)), my_pos, c->delta);
        __syncwarp();
        nb = 0;
    };
    auto push = [&](float d2, uint32_t r) {
        if (lane == nb) {
            my_d2 = d2;
            my_pos = r;
        }
        ++nb;
        if (nb == SR_BATCH) flush();
    };
    bool stalled = false;
    bool end = false;    // no later slot of this CTA can be filled
    uint32_t qrow = 0;   // lane t < RQ_UNIT: the row of the unit's slot t
    unsigned qm = 0;     // the unit's slots still to refine (warp-uniform)
    // The next unit of slots is claimed and its slots' first reads issued one
    // unit ahead (claim), so their latency passes while the rows before them
    // are refined; take() then waits for what is still missing.
    uint32_t nx_p = 0;              // the claimed unit (warp-uniform)
    uint2 nx_e = make_uint2(0u, 0u);  // lane t < RQ_UNIT: its slot's first read
    unsigned long long nx_kt = 0;   // lane RQ_KT_LANE: the k-th best, read with them
    auto slot_of = [&](uint32_t p) {
        return ((uint64_t)(p / (RQ_CHUNK / RQ_UNIT)) * G + cta) * RQ_CHUNK +
               (uint64_t)RQ_UNIT * (p % (RQ_CHUNK / RQ_UNIT)) + (uint64_t)lane;
    };
    auto claim = [&]() {
        uint32_t p = 0;
        if (lane == 0) p = atomicAdd(&fz[2], 1u);
        nx_p = __shfl_sync(FULL, p, 0);
        const uint64_t i = slot_of(nx_p);
        nx_e = lane < RQ_UNIT && i < cap ? ld_volatile_u2(&s.surv[i]) : make_uint2(0u, 0u);
        if (lane == RQ_KT_LANE) nx_kt = ld_volatile_u64(&s.topk[k - 1]);
    };
    // the claimed unit: lane t < RQ_UNIT waits for its slot (none: past the
    // list's end), empties it, and keeps its row unless the bound of the
    // current k-th best skips it; then the unit after it is claimed
    auto take = [&]() {
        uint2 e = nx_e;
        bool none = true;
        if (lane < RQ_UNIT) {
            const uint64_t i = slot_of(nx_p);
            none = i >= cap;  // past the list's room: never filled (the overflow rerun answers)
            uint32_t nap = 64;
            for (uint32_t poll = 0; !none && !e.x; ++poll) {
                if (*(volatile uint32_t*)&fz[0]) {
                    // the scan is over everywhere: every survivor is in the list
                    __threadfence();
                    e = ld_volatile_u2(&s.surv[i]);
                    if (e.x) break;
                    none = true;
                    if (i < (uint64_t)ld_volatile_u32(&c->surv_count)) stalled = true;  // a counted slot left empty
                    break;
                }
                if (poll >= RQ_WAIT) {
                    stalled = true;
                    none = true;
                    break;
                }
                // one thread of the CTA at a time looks at the scan's end
                if (atomicCAS(&fz[1], 0u, 1u) == 0u) {
                    if (ld_acquire_u32(&c->scan_done) >= G) {
                        __threadfence_block();
                        *(volatile uint32_t*)&fz[0] = 1u;
                    }
                    atomicExch(&fz[1], 0u);
                }
                __nanosleep(nap);
                if (nap < 1024u) nap <<= 1;
                e = ld_volatile_u2(&s.surv[i]);
            }
            if (!none) s.surv[i] = make_uint2(0u, 0u);  // back empty for the next query
        }
        end = __any_sync(FULL, (lane < RQ_UNIT && none) || stalled);
        const unsigned long long kt = __shfl_sync(FULL, nx_kt, RQ_KT_LANE);
        if (kt != kth || kth == 0ull) {
            kth = kt;
            limits_f32(c, kt, thr, lim, win);
        }
        qrow = e.x - 1u;
        qm = __ballot_sync(FULL, lane < RQ_UNIT && !none && __uint_as_float(e.y) <= thr);
        if (!end) claim();
    };
    // the next row to refine (mask bit t of the unit, row in lane t), taking
    // units until one has a kept row or the list ends; false when none is left
    auto next_row = [&](uint32_t& r) -> bool {
        while (qm == 0u && !end) take();
        if (qm == 0u) return false;
        const int t = __ffs(qm) - 1;
        qm &= qm - 1u;
        r = __shfl_sync(FULL, qrow, t);
        ISAX_CHECK(r < (uint64_t)ix.N, CHK_REFINE_ROW);
        return true;
    };
    claim();
    if constexpr (HALF) {
        const unsigned char* xb = reinterpret_cast<const unsigned char*>(ix.x);
        uint32_t pr0[RQ_DEPTH], pr1[RQ_DEPTH];  // each buffer's rows
        unsigned pm[RQ_DEPTH];                   // and which of the two it holds
        uint32_t pending = 0;                    // buffers whose copies are not yet waited for
        // The rows come in through the load path, 16 bytes per lane (a single
        // engine per SM issuing 1 KB bulk copies for every warp moves rows at
        // about half the rate of the warps' own loads); each barrier then counts
        // the 32 lanes' arrivals once their copies have landed.
        if (lane == 0) {
            for (int t = 0; t < RQ_DEPTH; ++t) {
                mbar_inval(&wbar[t]);
                mbar_init(&wbar[t], 32);
            }
            mbar_fence_init();
        }
        __syncwarp();
        par = 0u;
        // the next (up to) two rows into buffer b, copied whole
        auto fill = [&](int b) {
            pm[b] = 0u;
            if (next_row(pr0[b])) pm[b] |= 1u;
            if (next_row(pr1[b])) pm[b] |= 2u;
            if (!pm[b]) return;
            unsigned char* dst = wbuf + b * 2 * RQ_ROW + lane * 16;
            if (pm[b] & 1u) {
                const unsigned char* src = xb + (int64_t)pr0[b] * RQ_ROW + lane * 16;
                cp_async16(dst, src);
                cp_async16(dst + RQ_ROW / 2, src + RQ_ROW / 2);
            }
            if (pm[b] & 2u) {
                const unsigned char* src = xb + (int64_t)pr1[b] * RQ_ROW + lane * 16;
                cp_async16(dst + RQ_ROW, src);
                cp_async16(dst + RQ_ROW + RQ_ROW / 2, src + RQ_ROW / 2);
            }
            cp_async_arrive(&wbar[b]);
            pending |= 1u << b;
        };
#pragma unroll
        for (int b = 0; b < RQ_DEPTH; ++b) fill(b);
        // buffers in turn (the order they were filled in), each refilled once done
        while (pending && !stalled) {
#pragma unroll
            for (int b = 0; b < RQ_DEPTH; ++b) {
                if (!(pending & (1u << b)) || stalled) continue;
                if (!__all_sync(FULL, mbar_wait_bounded(&wbar[b], (par >> b) & 1u, RQ_BAR_WAIT))) {
                    stalled = true;
                    continue;
                }
                par ^= 1u << b;
                pending &= ~(1u << b);
                // the distances of the buffer's rows: every lane its two float4
                // of each row (the first half's, then the second half's), then
                // the butterfly, as warp_d2_vec<2>
                const float4 q0 = reinterpret_cast<const float4*>(q_sm)[lane];
                const float4 q1 = reinterpret_cast<const float4*>(q_sm)[32 + lane];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    if (!(pm[b] & (1u << t))) continue;
                    const float4* row = reinterpret_cast<const float4*>(wbuf + b * 2 * RQ_ROW + t * RQ_ROW);
                    const float4 v0 = row[lane], v1 = row[32 + lane];
                    float a = 0.0f, d;
                    d = v0.x - q0.x; a = fmaf(d, d, a);
                    d = v0.y - q0.y; a = fmaf(d, d, a);
                    d = v0.z - q0.z; a = fmaf(d, d, a);
                    d = v0.w - q0.w; a = fmaf(d, d, a);
                    d = v1.x - q1.x; a = fmaf(d, d, a);
                    d = v1.y - q1.y; a = fmaf(d, d, a);
                    d = v1.z - q1.z; a = fmaf(d, d, a);
                    d = v1.w - q1.w; a = fmaf(d, d, a);
                    ++n_ref;
                    n_floats += 256;
                    push(warp_sum_f(a), t ? pr1[b] : pr0[b]);
                }
                __syncwarp();  // every lane is done with the buffer before it is refilled
                fill(b);
            }
        }
        // after a wait that gave up: the copies still in flight land before the
        // ring is left (bounded)
        if (lane == 0)
            for (int t = 0; t < RQ_DEPTH; ++t)
                if (pending & (1u << t)) mbar_wait_bounded(&wbar[t], (par >> t) & 1u, RQ_BAR_WAIT);
        __syncwarp();
    } else {
        const float4* x4 = reinterpret_cast<const float4*>(ix.x);
        const bool vec = ix.n % 128 == 0;
        uint32_t r;
        while (!stalled && next_row(r)) {
            bool ab;
            int nread;
            const float d2 = vec ? warp_d2_v4q(x4 + (int64_t)r * (ix.n / 4), q4, ix.n / 128, lim, ab, nread)
                                 : warp_d2_gen(ix.x + (int64_t)r * ix.n, s.q, ix.n, lim, ab, nread);
            ++n_ref;
            n_floats += (unsigned long long)nread;
            if (!ab) push(d2, r);
        }
    }
    flush();
    if (lane == 0 && n_ref) {
        atomicAdd(&c->series_refined, n_ref);
        atomicAdd(&c->ed_floats, n_floats);
    }
    if (stalled) atomicOr(&c->flags, QF_STALLED);
}

// ---------------------------------------------------------------- q_series_lb
// The lower-bound scan (MESSI's lower-bound calculations).  Work item i of the
// list (a piece of at most LB_PIECE rows of a queued leaf, in ascending leaf
// bound for MESSI, storage order for the flat scan) belongs to CTA i mod G,
// whose warps take its items in list order from a shared-memory counter.  Each
// warp streams its pieces' 16-byte SAX words through a private ring of
// LB_STAGES shared-memory stages filled by bulk copies (the TMA engine,
// completion counted on one mbarrier per stage), LB_STAGES - 1 pieces ahead of
// the one it bounds, so HBM sees many copies in flight while the warp works
// from shared memory; the first copies start before the table is staged.  A
// series is bounded from the table (in shared memory, 1 KB-aligned rows)
// against the threshold the approximate answer set: the first 8 segments
// first, then 4 more and the last 4, each step only while some lane of the
// warp is still under the threshold (the sum runs in segment order either way,
// so the bound is the same).  Survivors {row of x, bound} are buffered per warp
// and appended with one atomic per batch.
constexpr int LB_THREADS = 1024;
constexpr int LB_WARPS = LB_THREADS / 32;
constexpr int LB_STAGES = 3;
constexpr int LB_PER_LANE = LB_PIECE / 32;
constexpr int LB_BUF = 48;     // survivors buffered per warp before one global append
constexpr uint32_t LB_WAIT = 1u << 22;  // bounded wait on a stage's copy
// The first LB_TAB_BYTES of the scan's shared memory: for 8-bit symbols the byte
// table [16][256] (4 KB), then the breakpoints and the query PAA; for smaller
// cardinalities the fp32 table [16][card] (at most 8 KB)
constexpr size_t LB_TAB_BYTES = 8192;
constexpr size_t LB_BP_OFF = 4096, LB_QPAA_OFF = LB_BP_OFF + sizeof(float) * (MAX_CARD + 4);
static_assert(LB_QPAA_OFF + sizeof(float) * W <= LB_TAB_BYTES, "byte table, breakpoints and PAA fit the region");
static_assert(sizeof(float) * W * (MAX_CARD / 2) <= LB_TAB_BYTES, "the fp32 table of cardinality <= 128 fits");
constexpr size_t LB_RING_BYTES = (size_t)LB_WARPS * LB_STAGES * LB_PIECE * sizeof(uint4);
// the scan's counters and flags (next item, each warp's last survivors and the
// CTA's base, the refinement's words), then the query for the n = 256
// refinement (16-byte aligned)
constexpr int LB_WORDS = LB_WARPS + 8;
constexpr size_t LB_Q_BYTES = 256 * sizeof(float);
constexpr size_t LB_SMEM = 1024 + LB_TAB_BYTES + LB_RING_BYTES + sizeof(uint64_t) * LB_WARPS * LB_STAGES +
                           sizeof(uint2) * LB_WARPS * (LB_STAGES + LB_BUF) + (size_t)LB_WARPS * LB_PIECE +
                           sizeof(uint32_t) * LB_WORDS + LB_Q_BYTES;
static_assert((LB_TAB_BYTES + LB_RING_BYTES + sizeof(uint64_t) * LB_WARPS * LB_STAGES +
               sizeof(uint2) * LB_WARPS * (LB_STAGES + LB_BUF) + (size_t)LB_WARPS * LB_PIECE +
               sizeof(uint32_t) * LB_WORDS) % 16 == 0 && LB_WORDS >= LB_WARPS + 6,
              "the query's copy in shared memory is 16-byte aligned after the scan's words");
static_assert(LB_SMEM <= 227 * 1024, "the scan's shared memory exceeds a CTA's limit");
static_assert(LB_STAGES >= RQ_DEPTH && LB_STAGES * LB_PIECE * sizeof(uint4) >= RQ_DEPTH * 2 * RQ_ROW,
              "a warp's ring and barriers hold the refinement's pairs of rows in flight");
constexpr uint32_t LB_QMAX = 255;  // byte-table units of the threshold
constexpr int LB_REFINERS = 4;  // warps per CTA that refine from the start of a fused launch
constexpr int LB_EAGER = 8;     // survivors a scanning warp buffers before it publishes them (fused)
static_assert(LB_REFINERS >= 0 && LB_REFINERS < LB_WARPS, "at least one warp scans");

template <int OFF>
__device__ __forceinline__ float lds_f32(uint32_t addr) {
    float x;
    asm("ld.shared.f32 %0, [%1+%2];" : "=f"(x) : "r"(addr), "n"(OFF));
    return x;
}
template <int OFF>
__device__ __forceinline__ uint32_t lds_u8(uint32_t addr) {
    uint32_t x;
    asm("ld.shared.u8 %0, [%1+%2];" : "=r"(x) : "r"(addr), "n"(OFF));
    return x;
}
// byte-table units of the 4 segments held by word Q of the SAX word, summed:
// the byte table's rows are 256 bytes and its base is 256-aligned, so one byte
// permute puts a symbol in the low byte of the table's address and the row
// offset is the load's immediate
template <int Q>
__device__ __forceinline__ uint32_t lb8_word(uint32_t v, uint32_t tab8_sa) {
    return lds_u8<(4 * Q + 0) * 256>(__byte_perm(v, tab8_sa, 0x7650u)) +
           lds_u8<(4 * Q + 1) * 256>(__byte_perm(v, tab8_sa, 0x7651u)) +
           lds_u8<(4 * Q + 2) * 256>(__byte_perm(v, tab8_sa, 0x7652u)) +
           lds_u8<(4 * Q + 3) * 256>(__byte_perm(v, tab8_sa, 0x7653u));
}
// the fp32 lower bound of an 8-bit SAX word, every table entry formed as the
// query's table is: T[i][s] = m * dist(qpaa_i, [bp[s], bp[s+1]))^2, summed in
// segment order
__device__ __forceinline__ float lb_exact256(uint4 w, const float* bp, const float* qpaa, float mf) {
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    float lb = 0.0f;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint32_t sym = (words[i >> 2] >> (8 * (i & 3))) & 255u;
        const float lo = bp[sym], hi = bp[sym + 1], v = qpaa[i];
        const float d = v < lo ? lo - v : (v >= hi ? v - hi : 0.0f);
        lb += (d * d) * mf;
    }
    return lb;
}

// One query's scan by G CTAs, this one being number cta (item i belongs to CTA
// i mod G).  REFINE > 0: every warp appends its own last survivors, the CTA
// then counts itself done in the control block (scan_done), and the warps go
// on to refine survivors (q_refine_claimed; REFINE == 2: rows of n = 256 staged
// by bulk copies); REFINE == 0: the CTA appends its warps' last survivors at
// once.
template <int CARD, int REFINE>
__device__ __forceinline__ void q_series_lb_body(const DevIndex& ix, const QueryScratch& s, int k, uint32_t cta,
                                                 uint32_t G) {
    extern __shared__ unsigned char lb_smem_raw[];
    QCtl* c = s.ctl;
    unsigned char* sm = lb_smem_raw + ((1024u - (smem_u32(lb_smem_raw) & 1023u)) & 1023u);
    float* tab = reinterpret_cast<float*>(sm);                      // fp32 table (cardinality < 256)
    unsigned char* tab8 = sm;                                       // byte table (8-bit symbols)
    float* bp_s = reinterpret_cast<float*>(sm + LB_BP_OFF);         // breakpoints (8-bit symbols)
    float* qpaa_s = reinterpret_cast<float*>(sm + LB_QPAA_OFF);     // query PAA (8-bit symbols)
    uint4* ring = reinterpret_cast<uint4*>(sm + LB_TAB_BYTES);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + LB_TAB_BYTES + LB_RING_BYTES);
    uint2* metas = reinterpret_cast<uint2*>(bars + LB_WARPS * LB_STAGES);
    uint2* bufs = metas + LB_WARPS * LB_STAGES;
    uint8_t* cand1 = reinterpret_cast<uint8_t*>(bufs + LB_WARPS * LB_BUF);  // [LB_WARPS][LB_PIECE]
    uint32_t* next_p = reinterpret_cast<uint32_t*>(cand1 + LB_WARPS * LB_PIECE);
    uint32_t* wcnt = next_p + 1;  // [LB_WARPS + 1]: each warp's last survivors, then the CTA's base
    // REFINE: warps done scanning, the scan over everywhere, polling token, slot units taken
    uint32_t* fz = wcnt + LB_WARPS + 1;
    float* q_sm = reinterpret_cast<float*>(next_p + LB_WORDS);  // REFINE == 2: the query (n = 256)
    const int card = ix.card;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // REFINE: the last LB_REFINERS warps refine from the start instead of scanning
    constexpr int SW = REFINE > 0 ? LB_WARPS - LB_REFINERS : LB_WARPS;
    const bool scans = warp < SW;
    uint4* wring = ring + (size_t)warp * LB_STAGES * LB_PIECE;
    uint64_t* wbar = bars + warp * LB_STAGES;
    uint2* wmeta = metas + warp * LB_STAGES;
    // everything the start needs is loaded at once: the flags, the item count,
    // this warp's first LB_STAGES items of the CTA (items warp * LB_STAGES + t,
    // read within the list's capacity and used only if below the count), the
    // threshold and the table
    const uint32_t flags = c->flags;
    const uint32_t count = c->work_count;
    const float thr = c->thr_scan;  // set with the work list, from the approximate answer
    uint2 e[LB_STAGES];
#pragma unroll
    for (int t = 0; t < LB_STAGES; ++t) {
        const size_t i = cta + (size_t)(warp * LB_STAGES + t) * G;
        e[t] = lane == 0 && scans && i < s.work_cap ? s.work[i] : make_uint2(0u, 0u);
    }
    // the table's inputs: the breakpoints and the query PAA (8-bit symbols), or
    // the query's fp32 table (smaller cardinalities)
    constexpr int TV = (W * MAX_CARD / 2 / 4 + LB_THREADS - 1) / LB_THREADS;
    float4 tv[TV];
    float bpv = 0.0f, qpv = 0.0f;
    if constexpr (CARD == 256) {
        if (threadIdx.x <= MAX_CARD) bpv = ix.bp[threadIdx.x];
        if (threadIdx.x < W) qpv = c->qpaa[threadIdx.x];
    } else {
        const float4* tsrc = reinterpret_cast<const float4*>(s.table);
        const int nv = W * card / 4;
#pragma unroll
        for (int t = 0; t < TV; ++t) {
            const int i = threadIdx.x + t * LB_THREADS;
            if (i < nv) tv[t] = tsrc[i];
        }
    }
    if (flags & QF_NONFINITE) return;
    const uint32_t mine = count > cta ? (count - cta + G - 1) / G : 0u;  // this CTA's items
    // lane 0 starts the copy of a piece into stage st
    auto issue = [&](uint32_t st, uint2 p) {
        const uint32_t rows = p.y & 0x7FFFFFFFu;
        wmeta[st] = p;
        mbar_arrive_expect_tx(&wbar[st], rows * (uint32_t)sizeof(uint4));
        // the SAX words are read once: first out of L2, so they pass by the
        // lines the survivors' refinement reads (its list, rows and query)
        if (rows)
            bulk_load_hint(wring + st * LB_PIECE, ix.sax + p.x, rows * (uint32_t)sizeof(uint4), &wbar[st],
                           l2_evict_first());
    };
    // the warp's own stage barriers, then its first LB_STAGES - 1 pieces; the
    // last of its first LB_STAGES is held until a stage frees up
    uint32_t issued = 0;
    const uint32_t j0 = warp * LB_STAGES;
    if (lane == 0) {
#pragma unroll
        for (int t = 0; t < LB_STAGES; ++t) mbar_init(&wbar[t], 1);
        mbar_fence_init();
#pragma unroll
        for (int t = 0; t + 1 < LB_STAGES; ++t)
            if (scans && j0 + t < mine) issue(t, e[t]);
    }
#pragma unroll
    for (int t = 0; t + 1 < LB_STAGES; ++t) issued += scans && j0 + t < mine ? 1u : 0u;
    uint2 pend = e[LB_STAGES - 1];
    bool pend_ok = scans && j0 + LB_STAGES - 1 < mine;
    const float mf = (float)(ix.n / W);
    if constexpr (CARD == 256) {
        if (threadIdx.x <= MAX_CARD) bp_s[threadIdx.x] = bpv;
        if (threadIdx.x < W) qpaa_s[threadIdx.x] = qpv;
        __syncthreads();
        // the byte table: q[i][s] = floor(T[i][s] * 255 / thr), at most 255, with T
        // the query table's fp32 entry; the scale and the product are rounded
        // down (and the scale shrunk by 2^-20), so q * thr / 255 <= T.  A row
        // whose units sum to more than 255 has a true bound >= 256 thr / 255,
        // whose fp32 sum of 16 entries exceeds thr: it would be pruned.  A
        // threshold that is not a positive finite number gives zeros: every row
        // goes on to the fp32 bound.
        const bool scaled = thr > 0.0f && thr < INFINITY;
        const float inv = scaled ? __fmul_rd(__fdiv_rd((float)LB_QMAX, thr), 1.0f - 0x1p-20f) : 0.0f;
        uint32_t packed = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int e = threadIdx.x * 4 + b;
            const int i = e >> 8, sym = e & 255;
            const float lo = bp_s[sym], hi = bp_s[sym + 1], v = qpaa_s[i];
            const float d = v < lo ? lo - v : (v >= hi ? v - hi : 0.0f);
            const float T = (d * d) * mf;
            const float qf = __fmul_rd(T, inv);
            const uint32_t q = qf >= (float)LB_QMAX ? LB_QMAX : (uint32_t)qf;
            packed |= q << (8 * b);
        }
        reinterpret_cast<uint32_t*>(tab8)[threadIdx.x] = packed;
        static_assert(LB_THREADS * 4 == W * MAX_CARD, "one 4-entry word of the byte table per thread");
    } else {
        float4* tdst = reinterpret_cast<float4*>(tab);
        const int nv = W * card / 4;
#pragma unroll
        for (int t = 0; t < TV; ++t) {
            const int i = threadIdx.x + t * LB_THREADS;
            if (i < nv) tdst[i] = tv[t];
        }
    }
    if (threadIdx.x == 0) {
        *next_p = SW * LB_STAGES;  // the items after the scanning warps' first ones go by claim
        fz[0] = fz[1] = fz[2] = fz[3] = 0u;
    }
    if (REFINE == 2 && threadIdx.x < 64)
        reinterpret_cast<float4*>(q_sm)[threadIdx.x] = reinterpret_cast<const float4*>(s.q)[threadIdx.x];
    __syncthreads();
    // the warp's next item of the CTA into `pend` (claimed in list order)
    auto claim = [&]() -> bool {
        uint32_t j = 0;
        if (lane == 0) j = atomicAdd(next_p, 1u);
        j = __shfl_sync(FULL, j, 0);
        if (lane == 0 && j < mine) pend = s.work[cta + (size_t)j * G];
        return j < mine;
    };
    const uint32_t tab8_sa = smem_u32(tab8);
    uint8_t* wcand = cand1 + warp * LB_PIECE;
    uint2* buf = bufs + warp * LB_BUF;
    int nbuf = 0;  // warp-uniform
    // the buffered survivors go to the global list in one append, each as
    // {row of x + 1, bound} in one 8-byte store (the position is translated
    // here, once per batch)
    auto drain = [&]() {
        if (nbuf == 0) return;
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&c->surv_count, (uint32_t)nbuf);
        base = __shfl_sync(FULL, base, 0);
        __syncwarp();
        for (int t = lane; t < nbuf; t += 32)
            if (base + t < s.surv_cap) s.surv[base + t] = make_uint2(row_at(ix, buf[t].x) + 1u, buf[t].y);
        __syncwarp();
        nbuf = 0;
    };
    // a kept row: appended to the warp's buffer as {position, bound}
    auto keep_rows = [&](bool keep, uint32_t pos, float lb) {
        const unsigned m = __ballot_sync(FULL, keep);
        // the row id is read when the buffer is appended: start bringing it in
        if (keep && ix.rows_in_place) prefetch_l2(ix.orig + pos);
        if (m) {
            if (nbuf + 32 > LB_BUF) drain();
            if (keep) buf[nbuf + __popc(m & ((1u << lane) - 1u))] = make_uint2(pos, __float_as_uint(lb));
            nbuf += __popc(m);
            __syncwarp();
        }
    };
    unsigned long long n_lb = 0, n_leaves = 0;
    bool stalled = false;
    uint32_t done = 0;  // warp-uniform, like issued and pend_ok
    for (;;) {
        if (pend_ok) {
            // the stage of piece `issued` held piece issued - LB_STAGES, already bounded
            if (lane == 0) issue(issued % LB_STAGES, pend);
            ++issued;
            pend_ok = claim();
        }
        if (done == issued) break;
        const uint32_t st = done % LB_STAGES;
        if (!__all_sync(FULL, mbar_wait_bounded(&wbar[st], (done / LB_STAGES) & 1u, LB_WAIT))) {
            stalled = true;
            break;
        }
        const uint2 p = wmeta[st];
        const uint32_t rows = p.y & 0x7FFFFFFFu, pos0 = p.x;
        ISAX_CHECK(rows <= (uint32_t)LB_PIECE && (uint64_t)pos0 + rows <= (uint64_t)ix.N, CHK_SCAN_ITEM);
        if (lane == 0) {
            n_lb += rows;
            n_leaves += p.y >> 31;
        }
        const uint4* src = wring + st * LB_PIECE;
        uint4 w[LB_PER_LANE];
#pragma unroll
        for (int j = 0; j < LB_PER_LANE; ++j) {
            const uint32_t r = j * 32 + lane;
            w[j] = r < rows ? src[r] : make_uint4(0u, 0u, 0u, 0u);
        }
        if constexpr (CARD == 256) {
            // pass 1, byte units: the first 8 segments of every row of the lane at
            // once, then per row the rest, 4 segments at a time, while some lane
            // of the warp is still at or under 255 units; rows still there after
            // all 16 segments are listed for pass 2
            uint32_t part[LB_PER_LANE];
#pragma unroll
            for (int j = 0; j < LB_PER_LANE; ++j) part[j] = lb8_word<0>(w[j].x, tab8_sa) + lb8_word<1>(w[j].y, tab8_sa);
            uint32_t ncand = 0;  // warp-uniform
#pragma unroll
            for (int j = 0; j < LB_PER_LANE; ++j) {
                const uint32_t r = j * 32 + lane;
                const bool ok = r < rows;
                uint32_t u = part[j];
                if (!__any_sync(FULL, ok && u <= LB_QMAX)) continue;
                u += lb8_word<2>(w[j].z, tab8_sa);
                if (!__any_sync(FULL, ok && u <= LB_QMAX)) continue;
                u += lb8_word<3>(w[j].w, tab8_sa);
                const bool cand = ok && u <= LB_QMAX;
                const unsigned m = __ballot_sync(FULL, cand);
                if (cand) wcand[ncand + __popc(m & ((1u << lane) - 1u))] = (uint8_t)r;
                ncand += __popc(m);
            }
            // pass 2: the fp32 bound of the listed rows (their words are still
            // in the stage), one per lane
            __syncwarp();
            for (uint32_t c0 = 0; c0 < ncand; c0 += 32) {
                const bool mine_c = c0 + lane < ncand;
                const uint32_t r = mine_c ? wcand[c0 + lane] : 0u;
                ISAX_CHECK(!mine_c || r < rows, CHK_SCAN_CAND);
                const float lb = mine_c ? lb_exact256(src[r], bp_s, qpaa_s, mf) : INFINITY;
                keep_rows(mine_c && lb <= thr, pos0 + r, lb);
            }
        } else {
#pragma unroll
            for (int j = 0; j < LB_PER_LANE; ++j) {
                const uint32_t r = j * 32 + lane;
                const float lb = series_lb(w[j], tab, card);
                keep_rows(r < rows && lb <= thr, pos0 + r, lb);
            }
        }
        ++done;
        __syncwarp();  // every lane is done with the stage before it is refilled
        // REFINE: survivors go to the list soon after they are found, for the
        // warps refining meanwhile
        if (REFINE > 0 && nbuf >= LB_EAGER) drain();
    }
    if (stalled) {
        // a copy never completed: flag the query and wait (bounded) for the
        // other copies still in flight into this warp's stages before leaving
        if (lane == 0) {
            atomicOr(&c->flags, QF_STALLED);
            for (uint32_t t = done + 1; t < issued; ++t)
                mbar_wait_bounded(&wbar[t % LB_STAGES], (t / LB_STAGES) & 1u, LB_WAIT);
        }
        __syncwarp();
    }
    if constexpr (REFINE > 0) {
        // the warp's last survivors, then the warp counts itself done; the CTA's
        // last warp counts the CTA done once every warp's survivors are visible
        // (each warp's fence before its count, the last one's fence after it)
        drain();
        if (lane == 0) {
            __threadfence();
            if (atomicAdd(&fz[0], 1u) == (uint32_t)LB_WARPS - 1u) {
                __threadfence();
                atomicAdd(&c->scan_done, 1u);
            }
        }
        __syncwarp();
    } else {
        // the warps' last survivors go to the list in one append for the whole CTA
        // (thousands of warps finish at about the same time: one counter update per
        // CTA instead of one per warp)
        if (lane == 0) wcnt[warp] = (uint32_t)nbuf;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int i = 0; i < LB_WARPS; ++i) tot += wcnt[i];
            wcnt[LB_WARPS] = tot ? atomicAdd(&c->surv_count, tot) : 0u;
        }
        __syncthreads();
        uint32_t base = wcnt[LB_WARPS];
        for (int i = 0; i < warp; ++i) base += wcnt[i];
        for (int t = lane; t < nbuf; t += 32)
            if (base + t < s.surv_cap) s.surv[base + t] = make_uint2(row_at(ix, buf[t].x) + 1u, buf[t].y);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n_lb += __shfl_xor_sync(FULL, n_lb, off);
    if (lane == 0) {
        if (n_lb) atomicAdd(&c->series_lb, n_lb);
        if (n_leaves) atomicAdd(&c->leaves_scanned, n_leaves);
    }
    if constexpr (REFINE > 0) {
        // the warp's ring and barriers go on staging rows: stage t's next wait
        // has the parity of the copies it has completed
        uint32_t par = 0;
#pragma unroll
        for (int t = 0; t < LB_STAGES; ++t)
            par |= ((issued > (uint32_t)t ? (issued - 1u - t) / LB_STAGES + 1u : 0u) & 1u) << t;
        if (!stalled)
            q_refine_claimed<REFINE == 2>(ix, s, k, cta, G, fz + 1, reinterpret_cast<unsigned char*>(wring), wbar,
                                          par, q_sm);
    }
}
// a single query's scan and refinement (one CTA per SM, cooperative launch:
// a refining warp may wait on any CTA's survivors)
template <int CARD, int REFINE>
__global__ void __launch_bounds__(LB_THREADS, 1) q_scan_refine_kernel(DevIndex ix, QueryScratch s, int k) {
    q_series_lb_body<CARD, REFINE>(ix, s, k, blockIdx.x, gridDim.x);
}
// a batch of queries: CTA j runs task j = {query, part | parts << 16}, the
// parts of a query sized to its number of work items
template <int CARD>
__global__ void __launch_bounds__(LB_THREADS, 1) bq_series_lb_kernel(DevIndex ix, const QueryScratch* ss,
                                                                     const uint2* __restrict__ tasks, int k) {
    const uint2 t = tasks[blockIdx.x];
    q_series_lb_body<CARD, 0>(ix, ss[t.x], k, t.y & 0xFFFFu, t.y >> 16);
}

// the scan kernels' shared-memory limit, raised once per device (before any
// capture: scratch allocation calls this too)
void prepare_scan_kernel(int device) {
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) device = -1;
    static bool done[64] = {};
    if (device >= 0 && device < 64 && done[device]) return;
    ISAX_CUDA_TRY(cudaFuncSetAttribute(q_scan_refine_kernel<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)LB_SMEM));
    ISAX_CUDA_TRY(cudaFuncSetAttribute(q_scan_refine_kernel<256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)LB_SMEM));
    ISAX_CUDA_TRY(cudaFuncSetAttribute(q_scan_refine_kernel<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)LB_SMEM));
    ISAX_CUDA_TRY(cudaFuncSetAttribute(q_scan_refine_kernel<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)LB_SMEM));
    ISAX_CUDA_TRY(cudaFuncSetAttribute(bq_series_lb_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)LB_SMEM));
    ISAX_CUDA_TRY(cudaFuncSetAttribute(bq_series_lb_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)LB_SMEM));
    if (device >= 0 && device < 64) done[device] = true;
}

// ---------------------------------------------------------------- q_refine
// survivor slot i as {row of x, bound} (a slot holds row + 1)
__device__ __forceinline__ uint2 surv_get(const QueryScratch& s, uint32_t i) {
    uint2 e = s.surv[i];
    e.x -= 1u;
    return e;
}
// Real distances of the survivors (MESSI's real distance calculations), in the
// order the scan found them: warp w takes survivor quads w, w + W, ... (W
// warps in the grid).  Before each quad the warp reads the current k-th best
// (lane 0, broadcast: the skip and early-abandon decisions are warp-uniform);
// a survivor whose bound now exceeds it is skipped without reading its row.
// Distances are computed with the same fp32 order as every other refinement
// and fed to the k best in batches of SR_BATCH.
constexpr int RF_THREADS = 256;

// gw / nw: this warp and the warps that share the query's survivors
template <int NV>
__device__ __forceinline__ void q_refine_body(const DevIndex& ix, const QueryScratch& s, int k, uint32_t gw,
                                              uint32_t nw) {
    QCtl* c = s.ctl;
    if (c->flags & QF_NONFINITE) return;
    const int lane = threadIdx.x & 31;
    constexpr int NQ = NV ? NV : 1;
    float4 qv[NQ];
    load_q<NV>(s.q, qv);
    const uint32_t found = c->surv_count;
    const uint32_t total = found < s.surv_cap ? found : s.surv_cap;
    unsigned long long kth = 0ull;  // cached k-th best and the limits derived from it
    float thr = INFINITY, lim = INFINITY, win = INFINITY;
    unsigned long long n_ref = 0, n_floats = 0;
    float my_d2 = INFINITY;
    uint32_t my_pos = 0;
    int nb = 0;
    // the window filter uses the cached k-th best (never below the current one);
    // consider() decides with a fresh value
    auto flush = [&]() {
        if (nb == 0) return;
        if (lane < nb && my_d2 <= win) consider(s, k, pack_key(my_d2, id_of_row(ix, my_pos)), my_pos, c->delta);
        __syncwarp();
        nb = 0;
    };
    auto push = [&](float d2, uint32_t r) {
        if (lane == nb) {
            my_d2 = d2;
            my_pos = r;
        }
        ++nb;
        if (nb == SR_BATCH) flush();
    };
    // the k-th best and the next four survivors are read one round ahead, so
    // their latency overlaps the current distances
    unsigned long long kt_next = 0;
    if (lane == 0) kt_next = ld_volatile_u64(&s.topk[k - 1]);
    uint2 nx[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) nx[t] = 4 * gw + t < total ? surv_get(s, 4 * gw + t) : make_uint2(0u, 0x7f800000u);
    for (uint32_t i = 4 * gw; i < total; i += 4 * nw) {
        __syncwarp();
        const unsigned long long kt = __shfl_sync(FULL, kt_next, 0);
        if (lane == 0) kt_next = ld_volatile_u64(&s.topk[k - 1]);
        if (kt != kth || kth == 0ull) {
            kth = kt;
            limits_f32(c, kt, thr, lim, win);
        }
        uint2 e[4];
        unsigned keep = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            e[t] = nx[t];
            if (i + t < total && __uint_as_float(e[t].y) <= thr) keep |= 1u << t;
            ISAX_CHECK(!(keep & (1u << t)) || e[t].x < (uint64_t)ix.N, CHK_REFINE_ROW);
        }
        const uint32_t in = i + 4 * nw;
#pragma unroll
        for (int t = 0; t < 4; ++t) nx[t] = in + t < total ? surv_get(s, in + t) : make_uint2(0u, 0x7f800000u);
        if (!keep) continue;
        if constexpr (NV > 0 && NV <= 2) {
            float d[4];
            warp_d2_four<NQ>(ix, e, keep, qv, d);
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (keep & (1u << t)) {
                    ++n_ref;
                    n_floats += (unsigned long long)ix.n;
                    push(d[t], e[t].x);
                }
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (keep & (1u << t)) {
                    bool ab;
                    int nread;
                    const float d0 = warp_d2<NV>(ix, (int64_t)e[t].x, qv, s.q, lim, ab, nread);
                    ++n_ref;
                    n_floats += (unsigned long long)nread;
                    if (!ab) push(d0, e[t].x);
                }
        }
    }
    flush();
    if (lane == 0 && n_ref) {
        atomicAdd(&c->series_refined, n_ref);
        atomicAdd(&c->ed_floats, n_floats);
    }
}
// a batch of queries: CTA j runs task j = {query, part | parts << 16}, the
// parts of a query sharing its survivors
template <int NV>
__global__ void __launch_bounds__(RF_THREADS, 3) bq_refine_kernel(DevIndex ix, const QueryScratch* ss,
                                                                  const uint2* __restrict__ tasks, int k) {
    const uint2 t = tasks[blockIdx.x];
    constexpr uint32_t WPB = RF_THREADS / 32;
    q_refine_body<NV>(ix, ss[t.x], k, (t.y & 0xFFFFu) * WPB + (threadIdx.x >> 5), (t.y >> 16) * WPB);
}

// n = 256 (two float4 per lane): every row in two halves of 128 floats.  The
// first halves of a quad of survivors are read one round ahead; their partial
// distances then decide each row (a partial above (1 + 8 delta) times the k-th
// best puts the full fp32 distance outside the candidate window: the row is
// abandoned and its second half never read), and the second halves of the kept
// rows are read together with the next quad's first halves, so a round still
// costs one memory latency.  A row's distance is its lanes' sums over both
// halves, then the butterfly: warp_d2_vec<2>'s value.
__device__ __forceinline__ void q_refine_half_body(const DevIndex& ix, const QueryScratch& s, int k, uint32_t gw,
                                                   uint32_t nw) {
    QCtl* c = s.ctl;
    if (c->flags & QF_NONFINITE) return;
    const int lane = threadIdx.x & 31;
    float4 qv[2];
    load_q<2>(s.q, qv);
    const uint32_t found = c->surv_count;
    const uint32_t total = found < s.surv_cap ? found : s.surv_cap;
    unsigned long long kth = 0ull;
    float thr = INFINITY, lim = INFINITY, win = INFINITY;
    unsigned long long n_ref = 0, n_floats = 0;
    float my_d2 = INFINITY;
    uint32_t my_pos = 0;
    int nb = 0;
    auto flush = [&]() {
        if (nb == 0) return;
        if (lane < nb && my_d2 <= win) consider(s, k, pack_key(my_d2, id_of_row(ix, my_pos)), my_pos, c->delta);
        __syncwarp();
        nb = 0;
    };
    auto push = [&](float d2, uint32_t r) {
        if (lane == nb) {
            my_d2 = d2;
            my_pos = r;
        }
        ++nb;
        if (nb == SR_BATCH) flush();
    };
    unsigned long long kt_next = 0;
    if (lane == 0) kt_next = ld_volatile_u64(&s.topk[k - 1]);
    auto refresh = [&]() {
        const unsigned long long kt = __shfl_sync(FULL, kt_next, 0);
        if (lane == 0) kt_next = ld_volatile_u64(&s.topk[k - 1]);
        if (kt != kth || kth == 0ull) {
            kth = kt;
            limits_f32(c, kt, thr, lim, win);
        }
    };
    const float4* x4 = reinterpret_cast<const float4*>(ix.x);
    uint2 nx[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) nx[t] = 4 * gw + t < total ? surv_get(s, 4 * gw + t) : make_uint2(0u, 0x7f800000u);
    // the quad at index i: its rows and the ones the bound does not skip; the
    // next quad's survivors are read meanwhile
    auto take = [&](uint32_t i, uint2 (&e)[4], unsigned& keep) {
        keep = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            e[t] = nx[t];
            if (i + t < total && __uint_as_float(e[t].y) <= thr) keep |= 1u << t;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) nx[t] = i + 4 * nw + t < total ? surv_get(s, i + 4 * nw + t) : make_uint2(0u, 0x7f800000u);
    };
    uint32_t i = 4 * gw;
    uint2 eA[4];
    unsigned keepA = 0;
    float4 hA[4];
    refresh();
    take(i, eA, keepA);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        ISAX_CHECK(!(keepA & (1u << t)) || eA[t].x < (uint64_t)ix.N, CHK_REFINE_ROW);
        if (keepA & (1u << t)) hA[t] = ld_stream(x4 + (int64_t)eA[t].x * 64 + lane);
    }
    while (i < total) {
        // partial distances of the quad's first halves
        float a[4];
        unsigned keep2 = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            a[t] = 0.0f;
            if (keepA & (1u << t)) {
                float d;
                d = hA[t].x - qv[0].x; a[t] = fmaf(d, d, a[t]);
                d = hA[t].y - qv[0].y; a[t] = fmaf(d, d, a[t]);
                d = hA[t].z - qv[0].z; a[t] = fmaf(d, d, a[t]);
                d = hA[t].w - qv[0].w; a[t] = fmaf(d, d, a[t]);
                ++n_ref;
                n_floats += 128;
                if (warp_sum_f(a[t]) <= lim) keep2 |= 1u << t;
            }
        }
        // the next quad, then one round of reads: the kept rows' second halves
        // and the next quad's first halves
        const uint32_t iB = i + 4 * nw;
        uint2 eB[4];
        unsigned keepB = 0;
        refresh();
        if (iB < total) take(iB, eB, keepB);
        float4 sA[4], hB[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            ISAX_CHECK(!(keepB & (1u << t)) || eB[t].x < (uint64_t)ix.N, CHK_REFINE_ROW);
            if (keep2 & (1u << t)) sA[t] = ld_stream(x4 + (int64_t)eA[t].x * 64 + 32 + lane);
            if (keepB & (1u << t)) hB[t] = ld_stream(x4 + (int64_t)eB[t].x * 64 + lane);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (keep2 & (1u << t)) {
                float d;
                d = sA[t].x - qv[1].x; a[t] = fmaf(d, d, a[t]);
                d = sA[t].y - qv[1].y; a[t] = fmaf(d, d, a[t]);
                d = sA[t].z - qv[1].z; a[t] = fmaf(d, d, a[t]);
                d = sA[t].w - qv[1].w; a[t] = fmaf(d, d, a[t]);
                n_floats += 128;
                push(warp_sum_f(a[t]), eA[t].x);
            }
        }
        i = iB;
        keepA = keepB;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            eA[t] = eB[t];
            hA[t] = hB[t];
        }
    }
    flush();
    if (lane == 0 && n_ref) {
        atomicAdd(&c->series_refined, n_ref);
        atomicAdd(&c->ed_floats, n_floats);
    }
}
__global__ void __launch_bounds__(RF_THREADS, 2) bq_refine_half_kernel(DevIndex ix, const QueryScratch* ss,
                                                                       const uint2* __restrict__ tasks, int k) {
    const uint2 t = tasks[blockIdx.x];
    constexpr uint32_t WPB = RF_THREADS / 32;
    q_refine_half_body(ix, ss[t.x], k, (t.y & 0xFFFFu) * WPB + (threadIdx.x >> 5), (t.y >> 16) * WPB);
}

// ---------------------------------------------------------------- q_finalize
constexpr int FIN_THREADS = 1024, FIN_WARPS = FIN_THREADS / 32, FIN_CAP = 2 * FIN_THREADS, FIN_UNROLL = 8;

__device__ __forceinline__ bool key_greater(unsigned long long a, uint32_t ia, unsigned long long b,
                                            uint32_t ib) {
    return a > b || (a == b && ia > ib);
}

// FP64 squared distance with the definition's order: sum_j (x_j - q_j)^2, j
// ascending, no fused multiply-add.  Lanes form the rounded FP64 squares of 32
// elements at a time in parallel (staged in `buf`, 32 doubles of this warp);
// lane 0 then adds them in order, so the sum is the same sequence of FP64
// additions as the definition.
__device__ __forceinline__ double warp_d2_fp64_seq(const float* __restrict__ xr,
                                                   const float* __restrict__ q, int n,
                                                   double* buf) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int t = 0; t < n; t += 32) {
        double sq = 0.0;
        if (t + lane < n) {
            const double d = __dsub_rn((double)xr[t + lane], (double)q[t + lane]);
            sq = __dmul_rn(d, d);
        }
        buf[lane] = sq;
        __syncwarp();
        if (lane == 0) {
            const int cnt = n - t < 32 ? n - t : 32;
#pragma unroll 8
            for (int l = 0; l < cnt; ++l) acc = __dadd_rn(acc, buf[l]);
        }
        __syncwarp();
    }
    return __shfl_sync(FULL, acc, 0);
}

// FP64 squared distance summed lane-parallel (each lane left to right over its
// elements, then a butterfly): the value returned for rows whose order is
// already decided.
__device__ __forceinline__ double warp_d2_fp64_tree(const float* __restrict__ xr,
                                                    const float* __restrict__ q, int n) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int j = lane; j < n; j += 32) {
        const double d = __dsub_rn((double)xr[j], (double)q[j]);
        acc = __dadd_rn(acc, __dmul_rn(d, d));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(FULL, acc, off));
    return acc;
}

__device__ __forceinline__ void bitonic_sort_smem(unsigned long long* sk, uint32_t* sid, int P) {
    const int tid = threadIdx.x;
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < P / 2; t += FIN_THREADS) {
                const int a = 2 * t - (t & (stride - 1));
                const int b = a + stride;
                const bool asc = (a & size) == 0;
                if (key_greater(sk[a], sid[a], sk[b], sid[b]) == asc) {
                    const unsigned long long tk = sk[a];
                    sk[a] = sk[b];
                    sk[b] = tk;
                    const uint32_t ti = sid[a];
                    sid[a] = sid[b];
                    sid[b] = ti;
                }
            }
            __syncthreads();
        }
    }
}

// Candidates within (1 + 3 delta) of the final k-th best (the window) are
// re-ranked in FP64 by (d2, row).  One filter pass stages the window; a window
// larger than the stage is processed in rounds, merging a running top-k.
__device__ __forceinline__ void q_finalize_body(const DevIndex& ix, const QueryScratch& s, int k) {
    __shared__ unsigned long long sk[FIN_CAP];
    __shared__ uint32_t sid[FIN_CAP];
    __shared__ uint32_t stage[FIN_THREADS];
    __shared__ unsigned long long stage_key[FIN_THREADS];
    __shared__ double sqbuf[FIN_WARPS][32];
    __shared__ int nst, ambiguous;
    QCtl* c = s.ctl;
    // the control block's words and the k-th best are read together
    const uint32_t flags = c->flags;
    const unsigned long long kth = s.topk[k - 1];
    const double delta = c->delta;
    const uint32_t cand_base = c->cand_base, cand_count = c->cand_count;
    if (flags & QF_NONFINITE) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (kth == EMPTY_SLOT) {
        if (tid == 0) c->flags |= QF_SHORT;
        return;
    }
    const double bound = (double)key_d2(kth) * (1.0 + 3.0 * delta);
    const uint32_t attempted = cand_base + cand_count;
    const uint32_t M = attempted < s.cand_cap ? attempted : s.cand_cap;
    const int n = ix.n;
    if (tid == 0) nst = 0;
    __syncthreads();
    // one pass over all candidates (FIN_UNROLL per thread at a time, all read
    // first): count the window, stage it if it fits
    for (uint32_t i0 = tid; i0 < M; i0 += FIN_UNROLL * FIN_THREADS) {
        unsigned long long key[FIN_UNROLL];
#pragma unroll
        for (int u = 0; u < FIN_UNROLL; ++u) {
            const uint32_t i = i0 + u * FIN_THREADS;
            key[u] = i < M ? s.cand_key[i] : EMPTY_SLOT;
        }
#pragma unroll
        for (int u = 0; u < FIN_UNROLL; ++u) {
            const uint32_t i = i0 + u * FIN_THREADS;
            if (i < M && (double)key_d2(key[u]) <= bound) {
                const int p = atomicAdd(&nst, 1);
                if (p < FIN_THREADS) {
                    stage[p] = s.cand_pos[i];
                    stage_key[p] = key[u];
                    ISAX_CHECK(stage[p] < (uint64_t)ix.N, CHK_FINAL_ROW);
                }
            }
        }
    }
    if (tid == 0) ambiguous = 0;
    __syncthreads();
    const int window = nst;
    int cnt = 0;
    bool done = false;
    if (window == k) {
        // The window holds exactly the k best: only their order is in question.
        // Sorted by fp32 (d2, row), it is the FP64 order as well when every
        // two neighbours are more than 3 delta apart (each FP64 value is within
        // delta of its fp32 value); then a warp-parallel FP64 sum gives the
        // returned distance.  Otherwise the sequential definition decides.
        for (int t = tid; t < window; t += FIN_THREADS) {
            sk[t] = stage_key[t];
            sid[t] = stage[t];
        }
        int P = 1;
        while (P < window) P <<= 1;
        for (int t = window + tid; t < P; t += FIN_THREADS) {
            sk[t] = EMPTY_SLOT;
            sid[t] = 0xffffffffu;
        }
        __syncthreads();
        bitonic_sort_smem(sk, sid, P);
        for (int t = tid; t + 1 < window; t += FIN_THREADS)
            if ((double)key_d2(sk[t + 1]) <= (double)key_d2(sk[t]) * (1.0 + 3.0 * delta)) ambiguous = 1;
        __syncthreads();
        if (!ambiguous) {
            for (int e = warp; e < window; e += FIN_WARPS) {
                const uint32_t pos = sid[e];
                const double d = warp_d2_fp64_tree(ix.x + (int64_t)pos * n, s.q, n);
                if (lane == 0) {
                    s.out_idx[e] = (int64_t)(uint32_t)sk[e];
                    s.out_dist[e] = __double2float_rn(sqrt(d));
                }
            }
            cnt = k;
            done = true;
        }
        __syncthreads();
    }
    if (done) {
    } else if (window <= FIN_THREADS) {
        for (int e = warp; e < window; e += FIN_WARPS) {
            const uint32_t pos = stage[e];
            const double d = warp_d2_fp64_seq(ix.x + (int64_t)pos * n, s.q, n, sqbuf[warp]);
            if (lane == 0) {
                sk[e] = (unsigned long long)__double_as_longlong(d);
                sid[e] = id_of_row(ix, pos);
            }
        }
        int P = 1;
        while (P < window) P <<= 1;
        for (int t = window + tid; t < P; t += FIN_THREADS) {
            sk[t] = EMPTY_SLOT;
            sid[t] = 0xffffffffu;
        }
        __syncthreads();
        bitonic_sort_smem(sk, sid, P);
        cnt = window < k ? window : k;
    } else {
        // large window (many exact ties): rounds of FIN_THREADS candidates
        for (uint32_t base = 0; base < M; base += FIN_THREADS) {
            __syncthreads();
            if (tid == 0) nst = 0;
            __syncthreads();
            const uint32_t i = base + tid;
            if (i < M && (double)key_d2(s.cand_key[i]) <= bound) stage[atomicAdd(&nst, 1)] = s.cand_pos[i];
            __syncthreads();
            const int added = nst;
            if (added == 0) continue;
            for (int e = warp; e < added; e += FIN_WARPS) {
                const uint32_t pos = stage[e];
                const double d = warp_d2_fp64_seq(ix.x + (int64_t)pos * n, s.q, n, sqbuf[warp]);
                if (lane == 0) {
                    sk[cnt + e] = (unsigned long long)__double_as_longlong(d);
                    sid[cnt + e] = id_of_row(ix, pos);
                }
            }
            const int total = cnt + added;
            int P = 1;
            while (P < total) P <<= 1;
            for (int t = total + tid; t < P; t += FIN_THREADS) {
                sk[t] = EMPTY_SLOT;
                sid[t] = 0xffffffffu;
            }
            __syncthreads();
            bitonic_sort_smem(sk, sid, P);
            cnt = total < k ? total : k;
        }
    }
    if (!done && tid < cnt) {
        s.out_idx[tid] = (int64_t)sid[tid];
        s.out_dist[tid] = __double2float_rn(sqrt(__longlong_as_double((long long)sk[tid])));
    }
    if (tid == 0) {
        c->window = (uint32_t)window;
        if (cnt < k) c->flags |= QF_SHORT;
        if (attempted > s.cand_cap || c->surv_count > s.surv_cap) c->flags |= QF_OVERFLOW;
    }
}
// After the answer: the totals the host reads are saved and the state the next
// query's q_front accumulates into is cleared (the k best, the candidate and
// refined counts), so a query's first kernel needs no clearing step of its own.
__device__ __forceinline__ void q_finalize_epilogue(const QueryScratch& s, int k) {
    __syncthreads();  // every thread is done reading the k best
    QCtl* c = s.ctl;
    if (threadIdx.x == 0) {
        c->cand_total = c->cand_base + c->cand_count;
        c->refined_total = c->series_refined;
        c->cand_count = 0;
        c->series_refined = 0;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) s.topk[i] = EMPTY_SLOT;
}
// the index's mapped block: the control block as the query ended, the answer,
// and the answer again in the caller's device outputs (oi, od: read from the
// block when the kernel started) if it named them
__device__ __forceinline__ void q_finalize_mail(const QueryScratch& s, int k, QMail* mail, int64_t* oi,
                                                float* od) {
    __syncthreads();  // the answer and the saved totals are written
    static_assert(FIN_THREADS >= MAX_K, "one thread per answer");
    if ((int)threadIdx.x < k) {
        const int t = threadIdx.x;
        const int64_t i = s.out_idx[t];
        const float d = s.out_dist[t];
        mail->idx[t] = i;
        mail->dist[t] = d;
        if (oi) oi[t] = i;
        if (od) od[t] = d;
    }
    static_assert(sizeof(QCtl) % sizeof(unsigned long long) == 0, "the control block is copied in 8-byte words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(s.ctl);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&mail->ctl);
    for (int t = threadIdx.x; t < (int)(sizeof(QCtl) / sizeof(unsigned long long)); t += blockDim.x) dst[t] = src[t];
}
__global__ void __launch_bounds__(FIN_THREADS, 1) q_finalize_kernel(DevIndex ix, QueryScratch s, int k, QMail* mail) {
    // the caller's output pointers are read from host memory now, so the read
    // has landed when the answer is ready
    int64_t* oi = nullptr;
    float* od = nullptr;
    if (mail && (int)threadIdx.x < k) {
        oi = mail->out_idx;
        od = mail->out_dist;
    }
    q_finalize_body(ix, s, k);
    q_finalize_epilogue(s, k);
    if (mail) q_finalize_mail(s, k, mail, oi, od);
}
__global__ void __launch_bounds__(FIN_THREADS, 1) bq_finalize_kernel(DevIndex ix, const QueryScratch* ss,
                                                                   int k) {
    q_finalize_body(ix, ss[blockIdx.y], k);
    q_finalize_epilogue(ss[blockIdx.y], k);
}

// ---------------------------------------------------------------- exact FP64 distances
// FP64 squared distance of given series to given queries with the definition's
// order (elements ascending, each difference, square and sum rounded on its
// own, no fused multiply-add), the value the brute-force definition computes.
// Merging the answers of row shards by it orders them exactly as the whole
// collection's brute force does.  One warp per (query, result); inv maps an
// original row to its row of x (null when x is in the original order).
constexpr int XD_WARPS = 8;
__global__ void __launch_bounds__(XD_WARPS * 32) exact_d2_kernel(DevIndex ix, const uint32_t* __restrict__ inv,
                                                                 const float* __restrict__ Q, int B, int k,
                                                                 const int64_t* __restrict__ idx,
                                                                 double* __restrict__ out) {
    __shared__ double buf[XD_WARPS][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * XD_WARPS + warp;
    if (t >= (int64_t)B * k) return;  // warp-uniform
    const int64_t b = t / k;
    const int64_t id = idx[t];
    double d = __longlong_as_double(0x7ff8000000000000ll);  // NaN for a row outside [0, N)
    if (id >= 0 && id < ix.N) {
        const int64_t row = inv ? (int64_t)inv[id] : id;
        d = warp_d2_fp64_seq(ix.x + row * ix.n, Q + b * ix.n, ix.n, buf[warp]);
    }
    if (lane == 0) out[t] = d;
}

// inv[orig[p]] = p: the row of x of every original row, for indexes that hold
// their rows in leaf order
__global__ void __launch_bounds__(256) inverse_perm_kernel(const uint32_t* __restrict__ orig, int64_t N,
                                                           uint32_t* __restrict__ inv) {
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (int64_t)gridDim.x * blockDim.x)
        inv[orig[p]] = (uint32_t)p;
}

// ================================================================ batched kernels
// Kernels of the batched path with the tensor-core filter (the contraction
// itself is in isax_tc.cu).  Query b of a batch owns scratch ss[b].

// (leaf, query) pairs that the leaf envelope bound does not prune, against
// each query's threshold after its approximate answer; a query's own
// approximate-answer leaves are left out (already refined exactly).
// Lane = query, warp = leaf: one ballot per (leaf, 32 queries), stored in
// mask[l * G + g] (G = ceil(B / 32) query groups); the pairs of every leaf are
// counted, and per query the leaves and series it keeps.  The bound is the
// single-query path's fp32 expression without branches: per segment at most
// one of (beta_lo - paa) and (paa - beta_hi+1) is positive, and the other
// clamps to +0, so the sum takes the same values in the same order.
constexpr int BP_WARPS = 8;
constexpr int BP_LEAVES = 256;  // leaves per CTA

__global__ void __launch_bounds__(BP_WARPS * 32) bq_pairs_kernel(
    DevIndex ix, const QueryScratch* ss, int B, int k, uint32_t* __restrict__ leaf_count,
    uint32_t* __restrict__ mask) {
    __shared__ float bp[MAX_CARD + 1];
    __shared__ unsigned long long part_l[BP_WARPS][32], part_s[BP_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = gridDim.y;
    const int b = blockIdx.y * 32 + lane;
    for (int i = threadIdx.x; i <= ix.card; i += blockDim.x) bp[i] = ix.bp[i];
    float qp[W];
    float thr = -1.0f;  // a negative threshold takes no leaf
    int64_t a0 = 0, a1 = 0;
    if (b < B) {
        const QCtl* c = ss[b].ctl;
        if (!(c->flags & QF_NONFINITE)) {
            thr = lb_threshold(ld_volatile_u64(&ss[b].topk[k - 1]), c->delta, c->E);
            a0 = c->approx_leaf;
            a1 = c->approx_end;
        }
#pragma unroll
        for (int i = 0; i < W; ++i) qp[i] = c->qpaa[i];
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) qp[i] = 0.0f;
    }
    __syncthreads();
    const float mf = (float)(ix.n / W);
    const int64_t l0 = (int64_t)blockIdx.x * BP_LEAVES;
    const int64_t l1 = l0 + BP_LEAVES < ix.L ? l0 + BP_LEAVES : ix.L;
    unsigned long long my_leaves = 0, my_series = 0;
    for (int64_t l = l0 + warp; l < l1; l += BP_WARPS) {
        const uint4 mn = ix.env[2 * l], mx = ix.env[2 * l + 1];
        const uint32_t wn[4] = {mn.x, mn.y, mn.z, mn.w}, wx[4] = {mx.x, mx.y, mx.z, mx.w};
        float lb = 0.0f;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const int lo = (wn[i >> 2] >> (8 * (i & 3))) & 255, hi = (wx[i >> 2] >> (8 * (i & 3))) & 255;
            const float d = fmaxf(bp[lo] - qp[i], 0.0f) + fmaxf(qp[i] - bp[hi + 1], 0.0f);
            lb += (d * d) * mf;
        }
        const bool take = lb <= thr && !(l >= a0 && l < a1);
        const unsigned m = __ballot_sync(FULL, take);
        if (lane == 0) {
            mask[l * G + blockIdx.y] = m;
            if (m) atomicAdd(&leaf_count[l], (uint32_t)__popc(m));
        }
        if (take) {
            ++my_leaves;
            my_series += ix.leaf_begin[l + 1] - ix.leaf_begin[l];
        }
    }
    part_l[warp][lane] = my_leaves;
    part_s[warp][lane] = my_series;
    __syncthreads();
    if (warp == 0 && b < B) {
        unsigned long long tl = 0, ts = 0;
        for (int w = 0; w < BP_WARPS; ++w) {
            tl += part_l[w][lane];
            ts += part_s[w][lane];
        }
        if (tl) {
            atomicAdd(&ss[b].ctl->leaves_queued, tl);
            atomicAdd(&ss[b].ctl->series_lb, ts);
        }
    }
}

// the queries of every leaf, ascending, at leaf_off[l] onwards: one warp per
// leaf, lanes over query groups, offsets by a warp scan of the group counts
__global__ void __launch_bounds__(256) bq_fill_kernel(int64_t L, int G, const uint32_t* __restrict__ mask,
                                                      const uint32_t* __restrict__ leaf_off,
                                                      uint32_t* __restrict__ pairs) {
    const int lane = threadIdx.x & 31;
    const int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (l >= L) return;
    uint32_t base = leaf_off[l];
    for (int g0 = 0; g0 < G; g0 += 32) {
        const int g = g0 + lane;
        uint32_t m = g < G ? mask[l * G + g] : 0u;
        const uint32_t c = (uint32_t)__popc(m);
        uint32_t incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += v;
        }
        uint32_t o = base + incl - c;
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            pairs[o++] = (uint32_t)(g * 32 + bit);
        }
        base += __shfl_sync(FULL, incl, 31);
    }
}

// Exact fp32 check of the rows the tensor-core filter kept: one warp per
// (row, query) record {position, query, filtered d2 bits, its error bound
// bits}.  A record whose filtered distance minus its bound already exceeds the
// query's current k-th best (with the fp32 slack) cannot be among the k best
// and is skipped; the others take the single-query path's refinement (same
// fp32 summation, same candidate window).
template <int NV>
__global__ void __launch_bounds__(256) bq_recheck_kernel(DevIndex ix, const QueryScratch* ss, int k,
                                                         const uint4* __restrict__ cand,
                                                         const uint32_t* __restrict__ cand_count,
                                                         uint32_t cap) {
    const int lane = threadIdx.x & 31;
    const uint32_t total = *cand_count;
    const uint32_t M = total < cap ? total : cap;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < M; i += nw) {
        const uint4 r = cand[i];
        const QueryScratch& s = ss[r.y];
        const double delta = s.ctl->delta;
        // one k-th best for the whole warp: lane 0 may still be finishing the
        // previous record's update, and the skip and early-abandon decisions
        // below must be warp-uniform (the distance is a warp reduction)
        __syncwarp();
        unsigned long long kth = 0;
        if (lane == 0) kth = ld_volatile_u64(&s.topk[k - 1]);
        kth = __shfl_sync(FULL, kth, 0);
        if (kth != EMPTY_SLOT && (double)__uint_as_float(r.z) - (double)__uint_as_float(r.w) >
                                     (double)key_d2(kth) * (1.0 + 5.0 * delta))
            continue;
        float4 qv[NV ? NV : 1];
        load_q<NV>(s.q, qv);
        bool ab;
        int nread;
        const uint32_t row = row_at(ix, r.x);
        const float d2 = warp_d2<NV>(ix, (int64_t)row, qv, s.q, abandon_limit(kth, delta), ab, nread);
        if (lane == 0) {
            atomicAdd(&s.ctl->series_refined, 1ull);
            atomicAdd(&s.ctl->ed_floats, (unsigned long long)nread);
            if (!ab) {
                const unsigned long long kk = ld_volatile_u64(&s.topk[k - 1]);
                if (kk == EMPTY_SLOT || (double)d2 <= (double)key_d2(kk) * (1.0 + 3.0 * delta))
                    consider(s, k, pack_key(d2, ix.orig[r.x]), row, delta);
            }
        }
    }
}

// ================================================================ host side
void free_query_scratch_struct(QueryScratch& q, cudaStream_t st);
static void free_scratch(QueryScratch& q, cudaStream_t st) { free_query_scratch_struct(q, st); }
void free_query_scratch_struct(QueryScratch& q, cudaStream_t st) {
    void* ptrs[] = {q.q, q.table, q.leaf_lb, q.work, q.bin_count, q.bin_cursor, q.topk,
                    q.cand_key, q.cand_pos, q.ctl, q.out_idx, q.out_dist, q.surv};
    for (void* p : ptrs)
        if (p) dev_free(p, st);
    q = QueryScratch{};
}

// scratch for queries on any index with at most L leaves, series length n and
// cardinality card
// scan work items of an index: at most one per leaf plus one per LB_PIECE series
int64_t work_items_cap(int64_t L, int64_t N) { return L + (N + LB_PIECE - 1) / LB_PIECE + 1; }

void alloc_query_scratch_for(int64_t L, int64_t N, int n, int card, uint32_t cand_cap, uint32_t surv_cap,
                             QueryScratch& q, cudaStream_t st) {
    prepare_scan_kernel(-1);
    q.q = static_cast<float*>(dev_alloc(sizeof(float) * n, st));
    q.table = static_cast<float*>(dev_alloc(sizeof(float) * W * card, st));
    q.leaf_lb = static_cast<float*>(dev_alloc(sizeof(float) * L, st));
    q.work_cap = (uint32_t)work_items_cap(L, N);
    q.work = static_cast<uint2*>(dev_alloc(sizeof(uint2) * q.work_cap, st));
    q.bin_count = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * NBINS, st));
    q.bin_cursor = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * NBINS, st));
    q.topk = static_cast<unsigned long long*>(dev_alloc(sizeof(unsigned long long) * MAX_K, st));
    q.cand_cap = cand_cap;
    q.cand_key = static_cast<unsigned long long*>(dev_alloc(sizeof(unsigned long long) * cand_cap, st));
    q.cand_pos = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * cand_cap, st));
    q.ctl = static_cast<QCtl*>(dev_alloc(sizeof(QCtl), st));
    q.out_idx = static_cast<int64_t*>(dev_alloc(sizeof(int64_t) * MAX_K, st));
    q.out_dist = static_cast<float*>(dev_alloc(sizeof(float) * MAX_K, st));
    q.surv_cap = surv_cap;
    q.surv = static_cast<uint2*>(dev_alloc(sizeof(uint2) * surv_cap, st));
    // a query starts with its k best empty, its counts at zero and its survivor
    // slots empty (each query's kernels leave them so for the next one)
    ISAX_CUDA_TRY(cudaMemsetAsync(q.surv, 0, sizeof(uint2) * surv_cap, st));
    ISAX_CUDA_TRY(cudaMemsetAsync(q.ctl, 0, sizeof(QCtl), st));
    ISAX_CUDA_TRY(cudaMemsetAsync(q.topk, 0xFF, sizeof(unsigned long long) * MAX_K, st));
}

uint32_t default_surv_cap(int64_t N) { return (uint32_t)std::max<int64_t>(1, std::min<int64_t>(N, 1 << 21)); }

static void alloc_scratch(const DevIndex& d, uint32_t cand_cap, uint32_t surv_cap, QueryScratch& q,
                          cudaStream_t st) {
    alloc_query_scratch_for(d.L, d.N, d.n, d.card, cand_cap, surv_cap, q, st);
}

// a larger survivor buffer (the old contents are dropped)
void grow_query_survivors(QueryScratch& q, uint32_t surv_cap, cudaStream_t st) {
    if (q.surv) dev_free(q.surv, st);
    q.surv = nullptr;
    q.surv_cap = 0;
    q.surv = static_cast<uint2*>(dev_alloc(sizeof(uint2) * surv_cap, st));
    q.surv_cap = surv_cap;
    ISAX_CUDA_TRY(cudaMemsetAsync(q.surv, 0, sizeof(uint2) * surv_cap, st));
}

// every survivor slot empty again: after a query whose refinement gave up a
// wait, slots it never took may still be filled
void empty_survivors(const QueryScratch& q, cudaStream_t st) {
    if (q.surv && q.surv_cap) ISAX_CUDA_TRY(cudaMemsetAsync(q.surv, 0, sizeof(uint2) * q.surv_cap, st));
}

// a larger candidate buffer (the old contents are dropped)
void grow_query_candidates(QueryScratch& q, uint32_t cand_cap, cudaStream_t st) {
    if (q.cand_key) dev_free(q.cand_key, st);
    if (q.cand_pos) dev_free(q.cand_pos, st);
    q.cand_key = nullptr;
    q.cand_pos = nullptr;
    q.cand_cap = 0;
    q.cand_key = static_cast<unsigned long long*>(dev_alloc(sizeof(unsigned long long) * cand_cap, st));
    q.cand_pos = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * cand_cap, st));
    q.cand_cap = cand_cap;
}

// The query's kernel sequence, captured once per k into a CUDA graph and
// replayed with one launch (while per-kernel tracing is off).  Graphs hold the
// scratch pointers, so they are dropped whenever the scratch is reallocated.
struct QueryGraphs {
    cudaStream_t capture = nullptr;
    std::map<int, cudaGraphExec_t> exec;
    int kernels_per_query = 0;
    void clear() {
        for (auto& kv : exec) cudaGraphExecDestroy(kv.second);
        exec.clear();
    }
    ~QueryGraphs() {
        clear();
        if (capture) cudaStreamDestroy(capture);
    }
};

// Extra scratch sets that let the queries of a batch run concurrently, each
// on its own stream.
constexpr int BATCH_SLOTS = 8;
struct QuerySlot {
    QueryScratch qs{};
    QueryGraphs graphs;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};
struct PlainBatch;
static void free_plain_batch(PlainBatch* pb, cudaStream_t st);
struct SlotPool {
    PlainBatch* plain[2] = {nullptr, nullptr};  // scratch of the batched path: normal and large tier
    std::vector<QuerySlot*> slots;
    QCtl* host_ctl = nullptr;  // pinned: one control block per query of a batch
    size_t host_cap = 0;
    int64_t* host_idx = nullptr;  // pinned staging for host outputs (a D2H copy into
    float* host_dist = nullptr;   // pageable memory would serialise the streams)
    size_t host_out_cap = 0;
};

static void free_slot_pool(isax_index* ix, cudaStream_t st) {
    SlotPool* p = static_cast<SlotPool*>(ix->pool);
    if (!p) return;
    for (PlainBatch*& pb : p->plain)
        if (pb) free_plain_batch(pb, st);
    for (QuerySlot* sl : p->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        free_scratch(sl->qs, st);
        sl->graphs.clear();
        if (sl->done) cudaEventDestroy(sl->done);
        if (sl->stream) cudaStreamDestroy(sl->stream);
        delete sl;
    }
    if (p->host_ctl) cudaFreeHost(p->host_ctl);
    if (p->host_idx) cudaFreeHost(p->host_idx);
    if (p->host_dist) cudaFreeHost(p->host_dist);
    delete p;
    ix->pool = nullptr;
}

void free_query_scratch(isax_index* ix, cudaStream_t st) { free_scratch(ix->qs, st); }

static void drop_query_graphs(isax_index* ix) {
    if (ix->graphs) static_cast<QueryGraphs*>(ix->graphs)->clear();
}

// A new scratch for the index's own queries; the old one (if any) is freed only
// once the new one is allocated, so a failed allocation leaves the index as it
// was.  keep_query: the query already in the old scratch moves to the new one.
void alloc_query_scratch(isax_index* ix, uint32_t cand_cap, uint32_t surv_cap, cudaStream_t st,
                         bool keep_query) {
    QueryScratch fresh{};
    try {
        alloc_scratch(ix->d, cand_cap, surv_cap, fresh, st);
        if (keep_query && ix->qs.q)
            ISAX_CUDA_TRY(cudaMemcpyAsync(fresh.q, ix->qs.q, sizeof(float) * ix->d.n, cudaMemcpyDeviceToDevice, st));
    } catch (...) {
        free_scratch(fresh, st);
        throw;
    }
    drop_query_graphs(ix);
    free_query_scratch(ix, st);
    ix->qs = fresh;
}

void free_index_arrays(isax_index* ix, cudaStream_t st) {
    if (ix->graphs) {
        delete static_cast<QueryGraphs*>(ix->graphs);
        ix->graphs = nullptr;
    }
    free_slot_pool(ix, st);
    free_tc_state(ix, st);
    free_query_scratch(ix, st);
    if (ix->rows_host && ix->x) {
        cudaStreamSynchronize(st);
        cudaFreeHost(ix->x);
        ix->x = nullptr;
    }
    if (ix->rows_borrowed) ix->x = nullptr;  // the caller's array
    if (ix->mail) {
        cudaFreeHost(ix->mail);
        ix->mail = nullptr;
        ix->mail_dev = nullptr;
    }
    void* ptrs[] = {ix->x, ix->sax, ix->orig, ix->leaf_begin, ix->env, ix->leaf_key, ix->bp,
                    ix->tree, ix->tree_root, ix->inv};
    for (void* p : ptrs)
        if (p) dev_free(p, st);
    ix->x = nullptr;
    ix->sax = nullptr;
    ix->orig = nullptr;
    ix->leaf_begin = nullptr;
    ix->env = nullptr;
    ix->leaf_key = nullptr;
    ix->bp = nullptr;
    ix->tree = nullptr;
    ix->tree_root = nullptr;
    ix->inv = nullptr;
}

namespace {

template <int NV>
void launch_query_kernels(isax_index* ix, const QueryScratch& s, int k, cudaStream_t st, int mode,
                          int scan_share, QMail* mail) {
    const DevIndex& d = ix->d;
    // the query's share of the SMs (all of them, or a part when queries run side by side)
    const unsigned grid = (unsigned)std::max(1, ix->num_sms / std::max(1, scan_share));
    {
        ISAX_LAUNCH("q_front", st);
        q_front_kernel<NV><<<grid, FR_THREADS, 0, st>>>(d, s, k, APPROX_NEIGHBORS, mail);
    }
    const unsigned lb_blocks = (unsigned)std::min<int64_t>((d.L + 255) / 256, (int64_t)ix->num_sms * 8);
    if (mode == QUERY_FLAT) {
        ISAX_LAUNCH("q_flat_list", st);
        q_flat_list_kernel<<<lb_blocks, 256, 0, st>>>(d, s, k);
    } else {
        // cooperative: its CTAs meet at a grid barrier, so all of them must be resident
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(BIN_THREADS);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        ISAX_LAUNCH("q_leaf_bin", st);
        ISAX_CUDA_TRY(cudaLaunchKernelEx(&cfg, q_leaf_bin_kernel, d, s, k));
    }
    {
        // one CTA per SM (its warps' copy rings take most of the SM's shared
        // memory); cooperative: a refining warp waits on other CTAs' survivors
        prepare_scan_kernel(ix->device);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(LB_THREADS);
        cfg.dynamicSmemBytes = LB_SMEM;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        // n = 256 with the rows in device memory: rows staged in shared memory
        // by the warps' asynchronous copies; otherwise (rows in host memory too)
        // read by the warps' own loads
        const bool half = NV == 2 && !ix->rows_host;
        ISAX_LAUNCH("q_scan_refine", st);
        if (d.card == 256) {
            if (half) ISAX_CUDA_TRY(cudaLaunchKernelEx(&cfg, q_scan_refine_kernel<256, 2>, d, s, k));
            else ISAX_CUDA_TRY(cudaLaunchKernelEx(&cfg, q_scan_refine_kernel<256, 1>, d, s, k));
        } else {
            if (half) ISAX_CUDA_TRY(cudaLaunchKernelEx(&cfg, q_scan_refine_kernel<0, 2>, d, s, k));
            else ISAX_CUDA_TRY(cudaLaunchKernelEx(&cfg, q_scan_refine_kernel<0, 1>, d, s, k));
        }
    }
    {
        ISAX_LAUNCH("q_finalize", st);
        q_finalize_kernel<<<1, FIN_THREADS, 0, st>>>(d, s, k, mail);
    }
    ISAX_CUDA_TRY(cudaGetLastError());
}

}  // namespace

// The query's kernels on the given scratch (the index's own, or the
// allocation-free entry point's built-in array).
void launch_query_on_scratch(isax_index* ix, const QueryScratch& s, int k, cudaStream_t st, int mode,
                             int scan_share, QMail* mail) {
    const int n = ix->d.n;
    if (n % 128 == 0) {
        switch (n / 128) {
            case 1: return launch_query_kernels<1>(ix, s, k, st, mode, scan_share, mail);
            case 2: return launch_query_kernels<2>(ix, s, k, st, mode, scan_share, mail);
            case 4: return launch_query_kernels<4>(ix, s, k, st, mode, scan_share, mail);
            case 8: return launch_query_kernels<8>(ix, s, k, st, mode, scan_share, mail);
            default: break;
        }
    }
    launch_query_kernels<0>(ix, s, k, st, mode, scan_share, mail);
}

// One exact k-NN query; q is already in ix->qs.q.  Results land in
// ix->qs.out_idx / out_dist; the control block is copied to *ctl_out.
// launch the query's kernels on st: replay of a captured graph, or direct
// launches while per-kernel tracing is on
static void launch_query_graph(isax_index* ix, const QueryScratch& qs, QueryGraphs* g, int k,
                               cudaStream_t st, int mode = QUERY_MESSI, int scan_share = 1,
                               QMail* mail = nullptr) {
    if (profiling_on()) {
        launch_query_on_scratch(ix, qs, k, st, mode, scan_share, mail);
        return;
    }
    const int key = k | (mode << 16) | (scan_share << 20);
    auto it = g->exec.find(key);
    if (it == g->exec.end()) {
        if (!g->capture) ISAX_CUDA_TRY(cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking));
        ISAX_CUDA_TRY(cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t graph = nullptr;
        try {
            launch_query_on_scratch(ix, qs, k, g->capture, mode, scan_share, mail);
        } catch (...) {
            cudaStreamEndCapture(g->capture, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        ISAX_CUDA_TRY(cudaStreamEndCapture(g->capture, &graph));
        size_t nodes = 0;
        cudaGraphGetNodes(graph, nullptr, &nodes);
        g->kernels_per_query = (int)nodes;
        cudaGraphExec_t exec = nullptr;
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        ISAX_CUDA_TRY(e);
        if (g->exec.size() >= 8) g->clear();
        it = g->exec.emplace(key, exec).first;
    }
    ISAX_CUDA_TRY(cudaGraphLaunch(it->second, st));
    count_launches(g->kernels_per_query);
}

// captured query graphs for callers outside this file (one cache per index and scratch)
void* query_graphs_new() { return new QueryGraphs(); }
void query_graphs_delete(void* g) { delete static_cast<QueryGraphs*>(g); }
void query_graphs_clear(void* g) { static_cast<QueryGraphs*>(g)->clear(); }
void launch_query_graph_ext(isax_index* ix, const QueryScratch& qs, void* g, int k, cudaStream_t st,
                            int scan_share) {
    launch_query_graph(ix, qs, static_cast<QueryGraphs*>(g), k, st, QUERY_MESSI, scan_share);
}

static void launch_query_index(isax_index* ix, int k, cudaStream_t st, int mode) {
    if (!ix->graphs) ix->graphs = new QueryGraphs();
    launch_query_graph(ix, ix->qs, static_cast<QueryGraphs*>(ix->graphs), k, st, mode, 1, ix->mail_dev);
}

void ensure_query_mail(isax_index* ix) {
    if (ix->mail) return;
    QMail* h = nullptr;
    ISAX_CUDA_TRY(cudaHostAlloc((void**)&h, sizeof(QMail), cudaHostAllocMapped));
    void* dv = nullptr;
    const cudaError_t e = cudaHostGetDevicePointer(&dv, h, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(h);
        ISAX_CUDA_TRY(e);
    }
    memset(h, 0, sizeof(QMail));
    ix->mail = h;
    ix->mail_dev = static_cast<QMail*>(dv);
}

void query_device(isax_index* ix, int k, QCtl* ctl_out, int* reruns, cudaStream_t st, int mode,
                  int64_t* out_idx, float* out_dist, bool out_device, const float* q_src) {
    *reruns = 0;
    ensure_query_mail(ix);
    // the mapped block names where the query is read and the answer written;
    // the query's kernels leave the control block there
    QMail* m = ix->mail;
    m->q_src = q_src ? q_src : ix->qs.q;
    m->out_idx = out_device ? out_idx : nullptr;
    m->out_dist = out_device ? out_dist : nullptr;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    for (int attempt = 0;; ++attempt) {
        launch_query_index(ix, k, st, mode);
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
        *ctl_out = m->ctl;
        ctl_out->flags |= injected_query_flags();
        if (ctl_out->flags & QF_NONFINITE) throw Error{ISAX_ERR_INVALID_ARG, "query contains a non-finite value"};
        if (ctl_out->flags & QF_STALLED) {
            empty_survivors(ix->qs, st);
            ISAX_CUDA_TRY(cudaStreamSynchronize(st));
            throw Error{ISAX_ERR_TIMEOUT, "a bounded wait of the query gave up"};
        }
        if (ctl_out->flags & QF_OVERFLOW) {
            if (attempt >= 3) throw Error{ISAX_ERR_INTERNAL, "candidate buffer kept overflowing"};
            const uint64_t N = (uint64_t)ix->d.N;
            uint64_t want_c = ix->qs.cand_cap, want_s = ix->qs.surv_cap;
            if (ctl_out->cand_total > ix->qs.cand_cap)
                want_c = std::min<uint64_t>(std::max<uint64_t>((uint64_t)ctl_out->cand_total * 2,
                                                               (uint64_t)ix->qs.cand_cap * 4), N);
            if (ctl_out->surv_count > ix->qs.surv_cap)
                want_s = std::min<uint64_t>(std::max<uint64_t>((uint64_t)ctl_out->surv_count * 2,
                                                               (uint64_t)ix->qs.surv_cap * 4), N);
            alloc_query_scratch(ix, (uint32_t)want_c, (uint32_t)want_s, st, true);  // q moves along
            if (!q_src) m->q_src = ix->qs.q;  // the query now sits in the new scratch
            ++*reruns;
            continue;
        }
        if (ctl_out->flags & QF_SHORT) throw Error{ISAX_ERR_INTERNAL, "fewer than k candidates survived"};
        if (!out_device) {
            if (out_idx) memcpy(out_idx, m->idx, sizeof(int64_t) * k);
            if (out_dist) memcpy(out_dist, m->dist, sizeof(float) * k);
        }
        return;
    }
}

// B queries, up to BATCH_SLOTS at a time on their own streams (each query's
// answer is the single-query answer: same kernels, own scratch).  Queries
// whose candidate buffer overflowed are rerun one by one afterwards.
static void query_batch_slots(isax_index* ix, const float* Q, int B, int k, uint32_t mem_flags,
                              int64_t* out_idx, float* out_dist, isax_query_stats_fill fill,
                              void* fill_ctx, cudaStream_t st) {
    const int n = ix->d.n;
    const int S = B < BATCH_SLOTS ? B : BATCH_SLOTS;
    if (!ix->pool) ix->pool = new SlotPool();
    SlotPool* pool = static_cast<SlotPool*>(ix->pool);
    while ((int)pool->slots.size() < S) {
        // a slot joins the pool only once all of it is allocated
        QuerySlot* sl = new QuerySlot();
        try {
            ISAX_CUDA_TRY(cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking));
            ISAX_CUDA_TRY(cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming));
            alloc_scratch(ix->d, ix->qs.cand_cap, ix->qs.surv_cap, sl->qs, st);
        } catch (...) {
            free_scratch(sl->qs, st);
            if (sl->done) cudaEventDestroy(sl->done);
            if (sl->stream) cudaStreamDestroy(sl->stream);
            delete sl;
            throw;
        }
        pool->slots.push_back(sl);
    }
    if (pool->host_cap < (size_t)B) {
        if (pool->host_ctl) cudaFreeHost(pool->host_ctl);
        pool->host_ctl = nullptr;
        pool->host_cap = 0;
        ISAX_CUDA_TRY(cudaMallocHost((void**)&pool->host_ctl, sizeof(QCtl) * (size_t)B));
        pool->host_cap = (size_t)B;
    }
    const bool host_out = !(mem_flags & ISAX_MEM_OUTPUT_DEVICE);
    if (host_out && pool->host_out_cap < (size_t)B * k) {
        if (pool->host_idx) cudaFreeHost(pool->host_idx);
        if (pool->host_dist) cudaFreeHost(pool->host_dist);
        pool->host_idx = nullptr;
        pool->host_dist = nullptr;
        pool->host_out_cap = 0;
        ISAX_CUDA_TRY(cudaMallocHost((void**)&pool->host_idx, sizeof(int64_t) * (size_t)B * k));
        ISAX_CUDA_TRY(cudaMallocHost((void**)&pool->host_dist, sizeof(float) * (size_t)B * k));
        pool->host_out_cap = (size_t)B * k;
    }
    int64_t* dst_idx = host_out ? pool->host_idx : out_idx;
    float* dst_dist = host_out ? pool->host_dist : out_dist;
    // the slots' work starts after everything already queued on st
    cudaEvent_t start;
    ISAX_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    ISAX_CUDA_TRY(cudaEventRecord(start, st));
    for (int i = 0; i < S; ++i) ISAX_CUDA_TRY(cudaStreamWaitEvent(pool->slots[i]->stream, start, 0));
    cudaEventDestroy(start);
    const cudaMemcpyKind kin = (mem_flags & ISAX_MEM_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                   : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = (mem_flags & ISAX_MEM_OUTPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                     : cudaMemcpyDeviceToHost;
    for (int b = 0; b < B; ++b) {
        QuerySlot* sl = pool->slots[b % S];
        const cudaStream_t ss = sl->stream;
        ISAX_CUDA_TRY(cudaMemcpyAsync(sl->qs.q, Q + (size_t)b * n, sizeof(float) * n, kin, ss));
        launch_query_graph(ix, sl->qs, &sl->graphs, k, ss);
        ISAX_CUDA_TRY(cudaMemcpyAsync(&pool->host_ctl[b], sl->qs.ctl, sizeof(QCtl),
                                      cudaMemcpyDeviceToHost, ss));
        ISAX_CUDA_TRY(cudaMemcpyAsync(dst_idx + (size_t)b * k, sl->qs.out_idx, sizeof(int64_t) * k,
                                      kout, ss));
        ISAX_CUDA_TRY(cudaMemcpyAsync(dst_dist + (size_t)b * k, sl->qs.out_dist, sizeof(float) * k,
                                      kout, ss));
    }
    for (int i = 0; i < S; ++i) {
        ISAX_CUDA_TRY(cudaEventRecord(pool->slots[i]->done, pool->slots[i]->stream));
        ISAX_CUDA_TRY(cudaStreamWaitEvent(st, pool->slots[i]->done, 0));
    }
    for (int i = 0; i < S; ++i) ISAX_CUDA_TRY(cudaStreamSynchronize(pool->slots[i]->stream));
    if (host_out) {
        memcpy(out_idx, pool->host_idx, sizeof(int64_t) * (size_t)B * k);
        memcpy(out_dist, pool->host_dist, sizeof(float) * (size_t)B * k);
    }
    bool nonfinite = false;
    for (int b = 0; b < B; ++b) {
        QCtl c = pool->host_ctl[b];
        c.flags |= injected_query_flags();
        int reruns = 0;
        if (c.flags & QF_NONFINITE) {
            nonfinite = true;
            continue;
        }
        if (c.flags & QF_STALLED) {
            for (int i = 0; i < S; ++i) empty_survivors(pool->slots[i]->qs, st);
            ISAX_CUDA_TRY(cudaStreamSynchronize(st));
            throw Error{ISAX_ERR_TIMEOUT, "a bounded wait of the query gave up"};
        }
        if (c.flags & (QF_OVERFLOW | QF_SHORT)) {
            ISAX_CUDA_TRY(cudaMemcpyAsync(ix->qs.q, Q + (size_t)b * n, sizeof(float) * n, kin, st));
            query_device(ix, k, &c, &reruns, st);
            ISAX_CUDA_TRY(cudaMemcpyAsync(out_idx + (size_t)b * k, ix->qs.out_idx, sizeof(int64_t) * k,
                                          kout, st));
            ISAX_CUDA_TRY(cudaMemcpyAsync(out_dist + (size_t)b * k, ix->qs.out_dist, sizeof(float) * k,
                                          kout, st));
            ISAX_CUDA_TRY(cudaStreamSynchronize(st));
            reruns += 1;
        }
        if (fill) fill(fill_ctx, b, c, reruns);
    }
    if (nonfinite) throw Error{ISAX_ERR_INVALID_ARG, "a query contains a non-finite value"};
}

// a launcher instantiated for the row length: NV float4 per lane (n / 128), 0 = generic
#define ISAX_NV_DISPATCH(n, CALL)                 \
    do {                                          \
        switch ((n) % 128 == 0 ? (n) / 128 : 0) { \
            case 1: CALL(1); break;               \
            case 2: CALL(2); break;               \
            case 4: CALL(4); break;               \
            case 8: CALL(8); break;               \
            default: CALL(0); break;              \
        }                                         \
    } while (0)

// ---------------------------------------------------------------- batched plain path
// A batch answered chunk by chunk with one launch per step for the whole chunk:
// the same per-query kernels as isax_query_knn, on per-query scratch carved
// from one allocation.  Preparation, approximate answer and leaf bounds run
// with grid.y = query.  The scan and the refinement run as task lists built on
// the host from the queries' counts: a query gets one scan CTA per PB_SCAN_ITEMS
// work items (item i to its part i mod P) and one refinement CTA per
// PB_REFINE_SURV survivors, so the chunk's scans stream the SAX words of all
// its queries in one long launch, balanced however skewed the queries are.
// Each query has the single
// query's worst-case room for work items, and room for PB_SURV survivors and
// PB_CAND candidates (tier 0).  The queries that overflow one are answered again
// together, in a second pass with 8x and 4x the room (tier 1); one that overflows
// that too is answered alone.  A chunk holds as many queries as fit in the
// tier's byte budget (at most PB_MAX_CHUNK).
constexpr int PB_MAX_CHUNK = 1024;
constexpr size_t PB_BYTES[2] = {(size_t)12 << 30, (size_t)6 << 30};
constexpr uint32_t PB_SURV = 1u << 21;        // survivors per query (tier 0)
constexpr uint32_t PB_CAND = 1u << 18;        // candidates per query (tier 0)
constexpr uint32_t PB_SURV_MULT[2] = {1, 8}, PB_CAND_MULT[2] = {1, 4};
constexpr uint32_t PB_SCAN_ITEMS = 1024;       // work items per scan task
constexpr uint32_t PB_REFINE_SURV = 4096;      // survivors per refinement task
constexpr uint32_t PB_MAX_PARTS = 1024;        // tasks per query and step

struct PlainBatch {
    int cap = 0, n = 0, card = 0;
    uint32_t surv_cap = 0;
    int64_t L = 0, N = 0;
    float* q = nullptr;                   // [cap][n]
    float* table = nullptr;               // [cap][16][card]
    float* leaf_lb = nullptr;             // [cap][L]
    uint2* work = nullptr;                // [cap][PB_WORK]
    uint32_t* bins = nullptr;             // [cap][2][NBINS]
    unsigned long long* topk = nullptr;   // [cap][MAX_K]
    unsigned long long* cand_key = nullptr;  // [cap][PB_CAND]
    uint32_t* cand_pos = nullptr;         // [cap][PB_CAND]
    uint2* surv = nullptr;                // [cap][PB_SURV]
    QCtl* ctl = nullptr;                  // [cap]
    int64_t* out_idx = nullptr;           // [cap][MAX_K]
    float* out_dist = nullptr;            // [cap][MAX_K]
    QueryScratch* ss = nullptr;           // [cap] device copy of the per-query views
    uint2* tasks_scan = nullptr;          // [cap * PB_MAX_PARTS] {query, part | parts << 16}
    uint2* tasks_refine = nullptr;        // [cap * PB_MAX_PARTS]
    QCtl* h_ctl = nullptr;                // pinned [cap]
    uint2* h_tasks_scan = nullptr;        // pinned staging of the task lists
    uint2* h_tasks_refine = nullptr;
};

static void free_plain_batch(PlainBatch* pb, cudaStream_t st) {
    if (!pb) return;
    cudaStreamSynchronize(st);
    void* ptrs[] = {pb->q, pb->table, pb->leaf_lb, pb->work, pb->bins, pb->topk, pb->cand_key, pb->cand_pos,
                    pb->surv, pb->ctl, pb->out_idx, pb->out_dist, pb->ss, pb->tasks_scan, pb->tasks_refine};
    for (void* p : ptrs)
        if (p) dev_free(p, st);
    if (pb->h_ctl) cudaFreeHost(pb->h_ctl);
    if (pb->h_tasks_scan) cudaFreeHost(pb->h_tasks_scan);
    if (pb->h_tasks_refine) cudaFreeHost(pb->h_tasks_refine);
    delete pb;
}

static PlainBatch* ensure_plain_batch(isax_index* ix, cudaStream_t st, int tier) {
    SlotPool* pool = static_cast<SlotPool*>(ix->pool);
    const DevIndex& d = ix->d;
    PlainBatch*& slot = pool->plain[tier];
    if (slot && slot->n == d.n && slot->card == d.card && slot->L == d.L && slot->N == d.N) return slot;
    if (slot) free_plain_batch(slot, st);
    slot = nullptr;
    PlainBatch* pb = new PlainBatch();
    const uint32_t work_cap = (uint32_t)work_items_cap(d.L, d.N);
    const uint32_t surv_cap = (uint32_t)std::min<int64_t>((int64_t)PB_SURV * PB_SURV_MULT[tier], d.N);
    const uint32_t cand_cap = (uint32_t)std::min<int64_t>((int64_t)PB_CAND * PB_CAND_MULT[tier], d.N + 16);
    const size_t per_query = sizeof(uint2) * (work_cap + (size_t)surv_cap) + sizeof(float) * (size_t)d.L +
                             12 * (size_t)cand_cap + sizeof(float) * (d.n + W * d.card) + 16 * MAX_K + 4096;
    const size_t C = (size_t)std::max<int64_t>(
        8, std::min<int64_t>(PB_MAX_CHUNK, (int64_t)(PB_BYTES[tier] / per_query)));
    try {
        pb->cap = (int)C;
        pb->n = d.n;
        pb->card = d.card;
        pb->L = d.L;
        pb->N = d.N;
        pb->surv_cap = surv_cap;
        auto alloc = [&](size_t bytes) { return dev_alloc(bytes, st); };
        pb->q = static_cast<float*>(alloc(sizeof(float) * C * d.n));
        pb->table = static_cast<float*>(alloc(sizeof(float) * C * W * d.card));
        pb->leaf_lb = static_cast<float*>(alloc(sizeof(float) * C * (size_t)d.L));
        pb->work = static_cast<uint2*>(alloc(sizeof(uint2) * C * work_cap));
        pb->bins = static_cast<uint32_t*>(alloc(sizeof(uint32_t) * C * 2 * NBINS));
        pb->topk = static_cast<unsigned long long*>(alloc(sizeof(unsigned long long) * C * MAX_K));
        pb->cand_key = static_cast<unsigned long long*>(alloc(sizeof(unsigned long long) * C * cand_cap));
        pb->cand_pos = static_cast<uint32_t*>(alloc(sizeof(uint32_t) * C * cand_cap));
        pb->surv = static_cast<uint2*>(alloc(sizeof(uint2) * C * surv_cap));
        pb->ctl = static_cast<QCtl*>(alloc(sizeof(QCtl) * C));
        pb->out_idx = static_cast<int64_t*>(alloc(sizeof(int64_t) * C * MAX_K));
        pb->out_dist = static_cast<float*>(alloc(sizeof(float) * C * MAX_K));
        pb->ss = static_cast<QueryScratch*>(alloc(sizeof(QueryScratch) * C));
        pb->tasks_scan = static_cast<uint2*>(alloc(sizeof(uint2) * C * PB_MAX_PARTS));
        pb->tasks_refine = static_cast<uint2*>(alloc(sizeof(uint2) * C * PB_MAX_PARTS));
        ISAX_CUDA_TRY(cudaMallocHost((void**)&pb->h_ctl, sizeof(QCtl) * C));
        ISAX_CUDA_TRY(cudaMallocHost((void**)&pb->h_tasks_scan, sizeof(uint2) * C * PB_MAX_PARTS));
        ISAX_CUDA_TRY(cudaMallocHost((void**)&pb->h_tasks_refine, sizeof(uint2) * C * PB_MAX_PARTS));
        std::vector<QueryScratch> hs(C);
        for (size_t b = 0; b < C; ++b) {
            QueryScratch& v = hs[b];
            v.q = pb->q + b * d.n;
            v.table = pb->table + b * W * d.card;
            v.leaf_lb = pb->leaf_lb + b * (size_t)d.L;
            v.work = pb->work + b * work_cap;
            v.work_cap = work_cap;
            v.bin_count = pb->bins + b * 2 * NBINS;
            v.bin_cursor = v.bin_count + NBINS;
            v.topk = pb->topk + b * MAX_K;
            v.cand_key = pb->cand_key + b * cand_cap;
            v.cand_pos = pb->cand_pos + b * cand_cap;
            v.cand_cap = cand_cap;
            v.surv = pb->surv + b * surv_cap;
            v.surv_cap = surv_cap;
            v.ctl = pb->ctl + b;
            v.out_idx = pb->out_idx + b * MAX_K;
            v.out_dist = pb->out_dist + b * MAX_K;
        }
        ISAX_CUDA_TRY(cudaMemcpyAsync(pb->ss, hs.data(), sizeof(QueryScratch) * C, cudaMemcpyHostToDevice, st));
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    } catch (...) {
        free_plain_batch(pb, st);
        throw;
    }
    slot = pb;
    return pb;
}

// the task list of one step: each query's parts, from its count of units
static uint32_t make_tasks(const QCtl* ctl, int C, uint2* tasks, bool scan, uint32_t surv_cap) {
    uint32_t T = 0;
    for (int b = 0; b < C; ++b) {
        const QCtl& c = ctl[b];
        if (c.flags & (QF_NONFINITE | QF_OVERFLOW | QF_STALLED)) continue;  // answered again alone
        if (!scan && c.surv_count > surv_cap) continue;                      // likewise
        const uint64_t units = scan ? c.work_count : c.surv_count;
        if (units == 0) continue;
        const uint64_t per = scan ? PB_SCAN_ITEMS : PB_REFINE_SURV;
        const uint32_t P = (uint32_t)std::min<uint64_t>(PB_MAX_PARTS, (units + per - 1) / per);
        for (uint32_t p = 0; p < P; ++p) tasks[T++] = make_uint2((uint32_t)b, p | (P << 16));
    }
    return T;
}

template <int NV>
static void launch_plain_chunk(isax_index* ix, PlainBatch* pb, int C, int k, cudaStream_t st) {
    const DevIndex& d = ix->d;
    const QueryScratch* ss = pb->ss;
    launch_bq_prep(ix, ss, C, k, APPROX_NEIGHBORS, st);
    launch_bq_approx(ix, ss, C, k, APPROX_NEIGHBORS, st);
    const unsigned lb_blocks = (unsigned)std::min<int64_t>((d.L + 255) / 256, (int64_t)ix->num_sms * 8);
    {
        ISAX_LAUNCH("bq_leaf_lb", st);
        bq_leaf_lb_kernel<<<dim3(lb_blocks, C), 256, 0, st>>>(d, ss, k);
    }
    {
        ISAX_LAUNCH("bq_leaf_scatter", st);
        bq_leaf_scatter_kernel<<<dim3(lb_blocks, C), NBINS, 0, st>>>(d, ss, k);
    }
    ISAX_CUDA_TRY(cudaMemcpyAsync(pb->h_ctl, pb->ctl, sizeof(QCtl) * (size_t)C, cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    const uint32_t Ts = make_tasks(pb->h_ctl, C, pb->h_tasks_scan, true, 0);
    if (Ts) {
        ISAX_CUDA_TRY(cudaMemcpyAsync(pb->tasks_scan, pb->h_tasks_scan, sizeof(uint2) * Ts, cudaMemcpyHostToDevice, st));
        prepare_scan_kernel(ix->device);
        ISAX_LAUNCH("bq_series_lb", st);
        if (d.card == 256)
            bq_series_lb_kernel<256><<<Ts, LB_THREADS, LB_SMEM, st>>>(d, ss, pb->tasks_scan, k);
        else
            bq_series_lb_kernel<0><<<Ts, LB_THREADS, LB_SMEM, st>>>(d, ss, pb->tasks_scan, k);
    }
    ISAX_CUDA_TRY(cudaMemcpyAsync(pb->h_ctl, pb->ctl, sizeof(QCtl) * (size_t)C, cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    const uint32_t Tr = make_tasks(pb->h_ctl, C, pb->h_tasks_refine, false, pb->surv_cap);
    if (Tr) {
        ISAX_CUDA_TRY(cudaMemcpyAsync(pb->tasks_refine, pb->h_tasks_refine, sizeof(uint2) * Tr,
                                      cudaMemcpyHostToDevice, st));
        ISAX_LAUNCH("bq_refine", st);
        if (NV == 2)
            bq_refine_half_kernel<<<Tr, RF_THREADS, 0, st>>>(d, ss, pb->tasks_refine, k);
        else
            bq_refine_kernel<NV><<<Tr, RF_THREADS, 0, st>>>(d, ss, pb->tasks_refine, k);
    }
    launch_bq_finalize(ix, ss, C, k, st);
    ISAX_CUDA_TRY(cudaGetLastError());
}

// Batches of at least PLAIN_BATCH_MIN queries take the chunked path; smaller
// ones run their single-query graphs concurrently on stream slots.
constexpr int PLAIN_BATCH_MIN = 8;

void query_batch_device(isax_index* ix, const float* Q, int B, int k, uint32_t mem_flags,
                        int64_t* out_idx, float* out_dist, isax_query_stats_fill fill,
                        void* fill_ctx, cudaStream_t st) {
    if (B < PLAIN_BATCH_MIN)
        return query_batch_slots(ix, Q, B, k, mem_flags, out_idx, out_dist, fill, fill_ctx, st);
    if (!ix->pool) ix->pool = new SlotPool();
    const int n = ix->d.n;
    const cudaMemcpyKind kin = (mem_flags & ISAX_MEM_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                   : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = (mem_flags & ISAX_MEM_OUTPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                     : cudaMemcpyDeviceToHost;
    bool nonfinite = false;
    // tier 0 takes every query in order; tier 1 the ones that overflowed tier 0
    std::vector<int> todo(B), next;
    for (int b = 0; b < B; ++b) todo[b] = b;
    for (int tier = 0; tier < 2 && !todo.empty(); ++tier) {
        PlainBatch* pb = ensure_plain_batch(ix, st, tier);
        const int T = (int)todo.size();
        for (int c0 = 0; c0 < T; c0 += pb->cap) {
            const int C = std::min(pb->cap, T - c0);
            const bool contiguous = todo[c0 + C - 1] - todo[c0] == C - 1;
            if (contiguous) {
                ISAX_CUDA_TRY(cudaMemcpyAsync(pb->q, Q + (size_t)todo[c0] * n, sizeof(float) * (size_t)C * n, kin, st));
            } else {
                for (int i = 0; i < C; ++i)
                    ISAX_CUDA_TRY(cudaMemcpyAsync(pb->q + (size_t)i * n, Q + (size_t)todo[c0 + i] * n,
                                                  sizeof(float) * n, kin, st));
            }
#define ISAX_CALL(NV) launch_plain_chunk<NV>(ix, pb, C, k, st)
            ISAX_NV_DISPATCH(n, ISAX_CALL);
#undef ISAX_CALL
            ISAX_CUDA_TRY(cudaMemcpyAsync(pb->h_ctl, pb->ctl, sizeof(QCtl) * (size_t)C, cudaMemcpyDeviceToHost, st));
            if (contiguous) {
                const size_t g0 = (size_t)todo[c0];
                ISAX_CUDA_TRY(cudaMemcpy2DAsync(out_idx + g0 * k, sizeof(int64_t) * k, pb->out_idx,
                                                sizeof(int64_t) * MAX_K, sizeof(int64_t) * k, C, kout, st));
                ISAX_CUDA_TRY(cudaMemcpy2DAsync(out_dist + g0 * k, sizeof(float) * k, pb->out_dist,
                                                sizeof(float) * MAX_K, sizeof(float) * k, C, kout, st));
            } else {
                for (int i = 0; i < C; ++i) {
                    const size_t g = (size_t)todo[c0 + i];
                    ISAX_CUDA_TRY(cudaMemcpyAsync(out_idx + g * k, pb->out_idx + (size_t)i * MAX_K,
                                                  sizeof(int64_t) * k, kout, st));
                    ISAX_CUDA_TRY(cudaMemcpyAsync(out_dist + g * k, pb->out_dist + (size_t)i * MAX_K,
                                                  sizeof(float) * k, kout, st));
                }
            }
            ISAX_CUDA_TRY(cudaStreamSynchronize(st));
            for (int i = 0; i < C; ++i) {
                const int b = todo[c0 + i];
                QCtl c = pb->h_ctl[i];
                c.flags |= injected_query_flags();
                int reruns = tier;
                if (c.flags & QF_NONFINITE) {
                    nonfinite = true;
                    continue;
                }
                if (c.flags & QF_STALLED) throw Error{ISAX_ERR_TIMEOUT, "a bulk copy of the lower-bound scan never completed"};
                if (c.flags & (QF_OVERFLOW | QF_SHORT)) {
                    if (tier == 0) {
                        next.push_back(b);  // answered again with more room
                        continue;
                    }
                    // even the larger room was too small: answer it alone
                    const size_t g = (size_t)b;
                    ISAX_CUDA_TRY(cudaMemcpyAsync(ix->qs.q, Q + g * n, sizeof(float) * n, kin, st));
                    int more = 0;
                    query_device(ix, k, &c, &more, st);
                    ISAX_CUDA_TRY(cudaMemcpyAsync(out_idx + g * k, ix->qs.out_idx, sizeof(int64_t) * k, kout, st));
                    ISAX_CUDA_TRY(cudaMemcpyAsync(out_dist + g * k, ix->qs.out_dist, sizeof(float) * k, kout, st));
                    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
                    reruns += 1 + more;
                }
                if (fill) fill(fill_ctx, b, c, reruns);
            }
        }
        todo.swap(next);
        next.clear();
    }
    if (nonfinite) throw Error{ISAX_ERR_INVALID_ARG, "a query contains a non-finite value"};
}

// ---------------------------------------------------------------- exact FP64 distances (host)
void exact_d2_device(isax_index* ix, const float* Q, int B, int k, const int64_t* idx, double* out,
                     cudaStream_t st) {
    if (!ix->rows_in_place && !ix->inv) {
        uint32_t* inv = static_cast<uint32_t*>(dev_alloc(sizeof(uint32_t) * (size_t)ix->d.N, st));
        ISAX_LAUNCH("inverse_perm", st);
        inverse_perm_kernel<<<ix->num_sms * 8, 256, 0, st>>>(ix->d.orig, ix->d.N, inv);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            dev_free(inv, st);
            ISAX_CUDA_TRY(e);
        }
        ix->inv = inv;
        ix->bytes += (int64_t)sizeof(uint32_t) * ix->d.N;
    }
    const int64_t T = (int64_t)B * k;
    if (T == 0) return;
    ISAX_LAUNCH("exact_d2", st);
    exact_d2_kernel<<<(unsigned)((T + XD_WARPS - 1) / XD_WARPS), XD_WARPS * 32, 0, st>>>(
        ix->d, ix->rows_in_place ? nullptr : ix->inv, Q, B, k, idx, out);
    ISAX_CUDA_TRY(cudaGetLastError());
}

// ---------------------------------------------------------------- batched launchers
void launch_bq_prep(isax_index* ix, const QueryScratch* ss, int B, int k, int neighbors,
                    cudaStream_t st) {
    ISAX_LAUNCH("bq_prep", st);
    bq_prep_kernel<<<dim3(1, B), PREP_THREADS, 0, st>>>(ix->d, ss, k, neighbors);
    ISAX_CUDA_TRY(cudaGetLastError());
}

template <int NV>
static void launch_bq_approx_nv(isax_index* ix, const QueryScratch* ss, int B, int k, int blocks,
                                cudaStream_t st) {
    ISAX_LAUNCH("bq_approx", st);
    bq_approx_kernel<NV><<<dim3(blocks, B), 256, 0, st>>>(ix->d, ss, k);
}

template <int NV>
static void launch_bq_recheck_nv(isax_index* ix, const QueryScratch* ss, int k, const uint4* cand,
                                 const uint32_t* cand_count, uint32_t cap, cudaStream_t st) {
    ISAX_LAUNCH("bq_recheck", st);
    bq_recheck_kernel<NV><<<ix->num_sms * 8, 256, 0, st>>>(ix->d, ss, k, cand, cand_count, cap);
}

void launch_bq_approx(isax_index* ix, const QueryScratch* ss, int B, int k, int neighbors,
                      cudaStream_t st) {
    const int per_query = (int)std::min<int64_t>(
        16, std::max<int64_t>(1, ((int64_t)(2 * neighbors + 1) * ix->d.leaf_size + 63) / 64));
#define ISAX_CALL(NV) launch_bq_approx_nv<NV>(ix, ss, B, k, per_query, st)
    ISAX_NV_DISPATCH(ix->d.n, ISAX_CALL);
#undef ISAX_CALL
    ISAX_CUDA_TRY(cudaGetLastError());
}

void launch_bq_pairs(isax_index* ix, const QueryScratch* ss, int B, int k, uint32_t* leaf_count,
                     uint32_t* mask, cudaStream_t st) {
    const dim3 grid((unsigned)((ix->d.L + BP_LEAVES - 1) / BP_LEAVES), (unsigned)((B + 31) / 32));
    ISAX_LAUNCH("bq_pairs", st);
    bq_pairs_kernel<<<grid, BP_WARPS * 32, 0, st>>>(ix->d, ss, B, k, leaf_count, mask);
    ISAX_CUDA_TRY(cudaGetLastError());
}

void launch_bq_fill(isax_index* ix, int B, const uint32_t* mask, const uint32_t* leaf_off,
                    uint32_t* pairs, cudaStream_t st) {
    const int64_t L = ix->d.L;
    ISAX_LAUNCH("bq_fill", st);
    bq_fill_kernel<<<(unsigned)((L * 32 + 255) / 256), 256, 0, st>>>(L, (B + 31) / 32, mask, leaf_off, pairs);
    ISAX_CUDA_TRY(cudaGetLastError());
}

void launch_bq_recheck(isax_index* ix, const QueryScratch* ss, int k, const uint4* cand,
                       const uint32_t* cand_count, uint32_t cap, cudaStream_t st) {
#define ISAX_CALL(NV) launch_bq_recheck_nv<NV>(ix, ss, k, cand, cand_count, cap, st)
    ISAX_NV_DISPATCH(ix->d.n, ISAX_CALL);
#undef ISAX_CALL
    ISAX_CUDA_TRY(cudaGetLastError());
}

void launch_bq_finalize(isax_index* ix, const QueryScratch* ss, int B, int k, cudaStream_t st) {
    ISAX_LAUNCH("bq_finalize", st);
    bq_finalize_kernel<<<dim3(1, B), FIN_THREADS, 0, st>>>(ix->d, ss, k);
    ISAX_CUDA_TRY(cudaGetLastError());
}

uint32_t take_check_word_query() { return take_check_word_here(); }

}  // namespace isax
