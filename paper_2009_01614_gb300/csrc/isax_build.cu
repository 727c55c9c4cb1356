// isax_build.cu - index construction on the GPU (Section II: PAA, iSAX symbols,
// ADS+ tree; Section III: MESSI's two-stage in-memory build).
//
// MESSI computes the iSAX summaries of RawData chunks and appends them to one
// iSAX buffer per root subtree (Stage 1), then builds every root subtree
// independently (Stage 2).  On the GPU the same result comes from:
//   summarize  - one warp per series: PAA of 16 segments, SAX symbols, and a
//                bit-plane-interleaved key whose top 16 bits are the root key
//                (first bit of every segment);
//   radix sort - a stable LSD sort of (key, row) pairs (one launch per 8-bit
//                digit, decoupled look-back): the per-root buffers become
//                contiguous runs, and inside a run series are ordered by
//                their next bits, so every iSAX node is a contiguous range;
//   leaves     - a node becomes a leaf once it holds <= leaf_size series; a
//                node splits on the next key bit (round-robin over segments),
//                decided for every adjacent pair from its common-prefix length
//                and a sliding-window maximum (no pointer tree is built);
//                or, with ISAX_BUILD_SPLIT_BALANCED, the ADS+ split itself: a
//                sort by root key, then one pass per tree level that splits
//                every overflowing node on its most balanced segment;
//   permute    - rows and SAX words gathered into leaf order (with the rows
//                kept in input order, the sort's last pass places the SAX
//                words and row ids itself);
//   envelopes  - per-leaf min/max symbol of every segment.
#include <algorithm>
#include <mutex>
#include <vector>

#include "isax_common.cuh"
#include "isax_kernels_util.cuh"

namespace isax {

// ============================================================== breakpoints
// Phi^{-1}(p) for p in (0, 1/2): Acklam's rational approximation
// (P. J. Acklam, "An algorithm for computing the inverse normal cumulative
// distribution function", 2003), then Halley steps on Phi(x) = erfc(-x/sqrt2)/2.
__device__ double inv_norm_lower(double p) {
    const double a1 = -3.969683028665376e+01, a2 = 2.209460984245205e+02,
                 a3 = -2.759285104469687e+02, a4 = 1.383577518672690e+02,
                 a5 = -3.066479806614716e+01, a6 = 2.506628277459239e+00;
    const double b1 = -5.447609879822406e+01, b2 = 1.615858368580409e+02,
                 b3 = -1.556989798598866e+02, b4 = 6.680131188771972e+01,
                 b5 = -1.328068155288572e+01;
    const double c1 = -7.784894002430293e-03, c2 = -3.223964580411365e-01,
                 c3 = -2.400758277161838e+00, c4 = -2.549732539343734e+00,
                 c5 = 4.374664141464968e+00, c6 = 2.938163982698783e+00;
    const double d1 = 7.784695709041462e-03, d2 = 3.224671290700398e-01,
                 d3 = 2.445134137142996e+00, d4 = 3.754408661907416e+00;
    double x;
    if (p < 0.02425) {
        double q = sqrt(-2.0 * log(p));
        x = (((((c1 * q + c2) * q + c3) * q + c4) * q + c5) * q + c6) /
            ((((d1 * q + d2) * q + d3) * q + d4) * q + 1.0);
    } else {
        double q = p - 0.5, r = q * q;
        x = (((((a1 * r + a2) * r + a3) * r + a4) * r + a5) * r + a6) * q /
            (((((b1 * r + b2) * r + b3) * r + b4) * r + b5) * r + 1.0);
    }
    const double sqrt2pi = 2.5066282746310002;
    for (int it = 0; it < 3; ++it) {
        double e = 0.5 * erfc(-x * 0.70710678118654752440) - p;
        double u = e * sqrt2pi * exp(0.5 * x * x);
        x = x - u / (1.0 + 0.5 * x * u);
    }
    return x;
}

// bp[0..card] = {-inf, beta_1 .. beta_{card-1}, +inf}, beta_t = Phi^{-1}(t/card)
// rounded to fp32; antisymmetric by construction, beta_{card/2} = 0.
__global__ void breakpoints_kernel(int card, float* bp) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > card) return;
    float v;
    if (t == 0)
        v = -INFINITY;
    else if (t == card)
        v = INFINITY;
    else if (2 * t == card)
        v = 0.0f;
    else {
        int tl = 2 * t < card ? t : card - t;
        double x = inv_norm_lower((double)tl / (double)card);
        v = __double2float_rn(2 * t < card ? x : -x);
    }
    bp[t] = v;
}

void launch_breakpoints(int card, float* bp, cudaStream_t st) {
    ISAX_LAUNCH("breakpoints", st);
    breakpoints_kernel<<<(card + 1 + 255) / 256, 256, 0, st>>>(card, bp);
    ISAX_CUDA_TRY(cudaGetLastError());
}

// ============================================================== summarize
// key: bit-plane-interleaved symbols, most significant plane first, segment 0
// at the top of each 16-bit plane; planes beyond cbits (or beyond 4) are 0.
__device__ __forceinline__ unsigned long long planes_to_key(int sym, bool active, int cbits) {
    unsigned long long key = 0;
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) {
        int b = cbits - 1 - pl;
        unsigned m = __ballot_sync(FULL, active && b >= 0 && ((sym >> (b < 0 ? 0 : b)) & 1));
        key = (key << 16) | (unsigned long long)(__brev(m & 0xffffu) >> 16);
    }
    return key;
}

// Symbol lookup in constant time.  The breakpoints of any cardinality <= 256
// lie in (-4, 4) and are at least 0.0098 apart, more than the 1/128 width of
// the cells of a grid over [-4, 4); the grid stores, for each cell start g,
// #{beta_t <= g}, so a value in the cell adds at most the next breakpoint.
// The result is exactly #{beta_t <= v} (the definition symbol_of computes).
constexpr int SYM_CELLS = 1024;

__device__ __forceinline__ float cell_start(int c) { return -4.0f + (float)c * 0.0078125f; }

__device__ __forceinline__ void build_symbol_grid(const float* bp, int card, uint8_t* grid) {
    for (int c = threadIdx.x; c < SYM_CELLS; c += blockDim.x)
        grid[c] = (uint8_t)symbol_of(cell_start(c), bp, card);
}

__device__ __forceinline__ int symbol_fast(float v, const float* bp, const uint8_t* grid, int card) {
    if (!(v >= -4.0f)) return 0;  // below every breakpoint (and NaN)
    if (v >= 4.0f) return card - 1;
    int c = (int)floorf((v + 4.0f) * 128.0f);  // off by at most one: fixed below
    c = c < 0 ? 0 : (c > SYM_CELLS - 1 ? SYM_CELLS - 1 : c);
    if (c < SYM_CELLS - 1 && cell_start(c + 1) <= v) ++c;
    if (c > 0 && cell_start(c) > v) --c;
    int s = grid[c];
    if (bp[s + 1] <= v) ++s;  // bp[card] = +inf
    return s;
}

// Series length NLEN in {128, 256, 512, 1024, 2048}; a warp takes ROWS (1 or 2)
// series per round.  Each lane loads NLEN/128 float4 of every row (all loads
// issued before any use); a segment is F = NLEN/64 consecutive float4 held by
// F consecutive lanes.  Segment sum: x+y+z+w per lane, then an xor tree over
// the F lanes.  Then lane L owns (row L/16, segment L%16): its PAA = sum *
// (16/NLEN) (exact scaling) and its symbol, computed once.
template <int NLEN, int ROWS>
__global__ void __launch_bounds__(256, (NLEN <= 256 ? 6 : NLEN <= 1024 ? 4 : 2))
summarize_vec_kernel(
    const float4* __restrict__ x, int64_t N, int card, int cbits, const float* __restrict__ bp_g,
    uint8_t* __restrict__ sax, unsigned long long* __restrict__ keys, uint32_t* __restrict__ ids,
    float* __restrict__ paa_out, unsigned* maxabs_bits, unsigned* nonfinite, uint32_t id_base) {
    constexpr int F = NLEN / 64;
    constexpr int PASSES = NLEN / 128;
    constexpr int SPP = 32 / F;
    constexpr float INV_M = 16.0f / (float)NLEN;
    __shared__ float bp[MAX_CARD + 1];
    __shared__ uint8_t grid[SYM_CELLS];
    __shared__ float red_max[32];
    __shared__ unsigned red_bad;
    for (int i = threadIdx.x; i <= card; i += blockDim.x) bp[i] = bp_g[i];
    if (threadIdx.x == 0) red_bad = 0;
    __syncthreads();
    build_symbol_grid(bp, card, grid);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int myrow = lane >> 4, myseg = lane & 15;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float amax = 0.0f;
    bool bad = false;
    for (int64_t base = gw * ROWS; base < N; base += nw * ROWS) {
        float4 v[ROWS][PASSES];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const float4* xr = x + (base + r) * (NLEN / 4);
            const bool ok = base + r < N;
#pragma unroll
            for (int p = 0; p < PASSES; ++p)
                v[r][p] = ok ? ld_stream(xr + p * 32 + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float mysum = 0.0f;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
#pragma unroll
            for (int p = 0; p < PASSES; ++p) {
                float s = ((v[r][p].x + v[r][p].y) + v[r][p].z) + v[r][p].w;
                amax = fmaxf(amax, fmaxf(fmaxf(fabsf(v[r][p].x), fabsf(v[r][p].y)),
                                         fmaxf(fabsf(v[r][p].z), fabsf(v[r][p].w))));
#pragma unroll
                for (int off = 1; off < F; off <<= 1) s += __shfl_xor_sync(FULL, s, off);
                const int src = ((myseg - p * SPP) & (SPP - 1)) * F;
                const float t = __shfl_sync(FULL, s, src);
                if (myrow == r && myseg / SPP == p) mysum = t;
            }
        }
        const int64_t row = base + myrow;
        const bool valid = myrow < ROWS && row < N;
        const float paa = mysum * INV_M;
        const int sym = symbol_fast(paa, bp, grid, card);
        bad |= valid && !isfinite(paa);
        unsigned long long key = 0;
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) {
            const int b = cbits - 1 - pl;
            const unsigned m = __ballot_sync(FULL, valid && b >= 0 && ((sym >> (b < 0 ? 0 : b)) & 1));
            key = (key << 16) | (unsigned long long)(__brev((m >> (16 * myrow)) & 0xffffu) >> 16);
        }
        if (valid) {
            sax[row * W + myseg] = (uint8_t)sym;
            if (paa_out) paa_out[row * W + myseg] = paa;
            if (myseg == 0) {
                if (keys) keys[row] = key;
                if (ids) ids[row] = id_base + (uint32_t)row;
            }
        }
    }
    // block reductions -> one atomic per block
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, off));
    if (lane == 0) red_max[threadIdx.x >> 5] = amax;
    if (bad) atomicOr(&red_bad, 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red_max[i]);
        atomicMax(maxabs_bits, __float_as_uint(m));
        if (red_bad) atomicOr(nonfinite, 1u);
    }
}

// Any n (multiple of 16): a half-warp per series, one lane per segment summing
// its m values left to right; PAA = sum / m.
__global__ void __launch_bounds__(256) summarize_generic_kernel(
    const float* __restrict__ x, int64_t N, int n, int card, int cbits,
    const float* __restrict__ bp_g, uint8_t* __restrict__ sax, unsigned long long* __restrict__ keys,
    uint32_t* __restrict__ ids, float* __restrict__ paa_out, unsigned* maxabs_bits,
    unsigned* nonfinite, uint32_t id_base) {
    __shared__ float bp[MAX_CARD + 1];
    __shared__ float red_max[32];
    __shared__ unsigned red_bad;
    for (int i = threadIdx.x; i <= card; i += blockDim.x) bp[i] = bp_g[i];
    if (threadIdx.x == 0) red_bad = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int seg = lane & 15, half = lane >> 4;
    const int m = n / W;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float amax = 0.0f;
    bool bad = false;
    for (int64_t pair = gw; pair * 2 < N; pair += nw) {
        const int64_t row = pair * 2 + half;
        const bool valid = row < N;
        int sym = 0;
        float paa = 0.0f;
        if (valid) {
            const float* p = x + row * n + seg * m;
            float s = 0.0f;
            for (int j = 0; j < m; ++j) {
                float v = p[j];
                s += v;
                amax = fmaxf(amax, fabsf(v));
            }
            paa = s / (float)m;
            sym = symbol_of(paa, bp, card);
            bad |= !isfinite(paa);
        }
        unsigned long long key = 0;
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) {
            int b = cbits - 1 - pl;
            unsigned mk = __ballot_sync(FULL, valid && b >= 0 && ((sym >> (b < 0 ? 0 : b)) & 1));
            unsigned mine = (mk >> (16 * half)) & 0xffffu;
            key = (key << 16) | (unsigned long long)(__brev(mine) >> 16);
        }
        if (valid) {
            sax[row * W + seg] = (uint8_t)sym;
            if (paa_out) paa_out[row * W + seg] = paa;
            if (seg == 0) {
                if (keys) keys[row] = key;
                if (ids) ids[row] = id_base + (uint32_t)row;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, off));
    if (lane == 0) red_max[threadIdx.x >> 5] = amax;
    if (bad) atomicOr(&red_bad, 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmaxf(mm, red_max[i]);
        atomicMax(maxabs_bits, __float_as_uint(mm));
        if (red_bad) atomicOr(nonfinite, 1u);
    }
}

void launch_summarize(const float* x, int64_t N, int n, int card, const float* bp, uint4* sax,
                      unsigned long long* keys, uint32_t* ids, float* paa_out,
                      unsigned* maxabs_bits, unsigned* nonfinite, int num_sms, cudaStream_t st,
                      uint32_t id_base) {
    int cbits = 0;
    while ((1 << cbits) < card) ++cbits;
    const int threads = 256;
    const int64_t want = (N + 15) / 16;  // up to two rows per warp
    // persistent grid: as many blocks as are resident at once
    auto grid_of = [&](const void* fn) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess ||
            per_sm < 1)
            per_sm = 4;
        return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * per_sm));
    };
    uint8_t* s8 = reinterpret_cast<uint8_t*>(sax);
    const float4* x4 = reinterpret_cast<const float4*>(x);
    ISAX_LAUNCH("summarize", st);
#define ISAX_SUM_CASE(L, R)                                                                    \
    case L:                                                                                    \
        summarize_vec_kernel<L, R><<<grid_of((const void*)summarize_vec_kernel<L, R>),         \
                                     threads, 0, st>>>(x4, N, card, cbits, bp, s8, keys, ids,  \
                                                       paa_out, maxabs_bits, nonfinite, id_base); \
        break;
    switch (n) {
        ISAX_SUM_CASE(128, 2)
        ISAX_SUM_CASE(256, 2)
        ISAX_SUM_CASE(512, 2)
        ISAX_SUM_CASE(1024, 1)
        ISAX_SUM_CASE(2048, 1)
        default:
            summarize_generic_kernel<<<grid_of((const void*)summarize_generic_kernel), threads, 0,
                                       st>>>(x, N, n, card, cbits, bp, s8, keys,
                                                                 ids, paa_out, maxabs_bits,
                                                                 nonfinite, id_base);
    }
#undef ISAX_SUM_CASE
    ISAX_CUDA_TRY(cudaGetLastError());
}

// ============================================================== exclusive scan
constexpr int SC_THREADS = 256, SC_ITEMS = 16, SC_TILE = SC_THREADS * SC_ITEMS;

__global__ void __launch_bounds__(SC_THREADS) scan_reduce_kernel(const uint32_t* __restrict__ in,
                                                                  int64_t len,
                                                                  uint32_t* __restrict__ sums) {
    __shared__ uint32_t scratch[32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j)
        if (base + j < len) s += in[base + j];
    uint32_t tot;
    block_excl_scan<uint32_t>(s, 0u, OpAdd<uint32_t>(), scratch, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single block: exclusive scan of nb block sums in place; sums[nb] = total
__global__ void __launch_bounds__(1024) scan_sums_kernel(uint32_t* sums, int64_t nb) {
    __shared__ uint32_t scratch[32];
    const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = (int64_t)threadIdx.x * per, b1 = std::min<int64_t>(b0 + per, nb);
    uint32_t s = 0;
    for (int64_t i = b0; i < b1; ++i) s += sums[i];
    uint32_t tot;
    uint32_t off = block_excl_scan<uint32_t>(s, 0u, OpAdd<uint32_t>(), scratch, &tot);
    for (int64_t i = b0; i < b1; ++i) {
        uint32_t v = sums[i];
        sums[i] = off;
        off += v;
    }
    if (threadIdx.x == 0) sums[nb] = tot;
}

__global__ void __launch_bounds__(SC_THREADS) scan_apply_kernel(const uint32_t* in, uint32_t* out,
                                                                 int64_t len,
                                                                 const uint32_t* __restrict__ sums) {
    __shared__ uint32_t scratch[32];
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    uint32_t v[SC_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        v[j] = base + j < len ? in[base + j] : 0u;
        s += v[j];
    }
    uint32_t tot;
    uint32_t off = block_excl_scan<uint32_t>(s, 0u, OpAdd<uint32_t>(), scratch, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        if (base + j < len) out[base + j] = off;
        off += v[j];
    }
}

// out[i] = sum_{j<i} in[i] for i < len; out may alias in.  `sums` needs
// ceil(len / SC_TILE) + 1 entries; the total lands in sums[ceil(len/SC_TILE)].
static void exclusive_scan(const uint32_t* in, uint32_t* out, int64_t len, uint32_t* sums,
                           cudaStream_t st) {
    if (len <= 0) {
        ISAX_CUDA_TRY(cudaMemsetAsync(sums, 0, sizeof(uint32_t), st));
        return;
    }
    int64_t nb = (len + SC_TILE - 1) / SC_TILE;
    {
    ISAX_LAUNCH("scan_reduce", st);
    scan_reduce_kernel<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, len, sums);
    }
    {
    ISAX_LAUNCH("scan_sums", st);
    scan_sums_kernel<<<1, 1024, 0, st>>>(sums, nb);
    }
    {
    ISAX_LAUNCH("scan_apply", st);
    scan_apply_kernel<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, out, len, sums);
    }
    ISAX_CUDA_TRY(cudaGetLastError());
}

static int64_t scan_sums_len(int64_t len) { return (len + SC_TILE - 1) / SC_TILE + 1; }

// ============================================================== radix sort
// Stable LSD radix sort of (64-bit key, 32-bit row) pairs, 8-bit digits.  Per
// pass: per-tile digit histograms, an exclusive scan over (digit, tile), then
// a scatter in which every warp ranks its elements with ballots over the digit
// bits (stable: element order inside a tile is warp, item, lane).
constexpr int RS_THREADS = 256, RS_ITEMS = 8, RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void __launch_bounds__(RS_THREADS) rs_hist_kernel(
    const unsigned long long* __restrict__ keys, int64_t N, int shift, uint32_t* __restrict__ hist,
    int64_t tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        const int64_t idx = base + i;
        if (idx < N) atomicAdd(&h[(unsigned)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// One tile of RS_TILE pairs per block.  Ranks are computed per warp with
// ballots over the digit bits (stable: tile order is warp, item, lane); the
// tile is first reordered by digit in shared memory, then written out so that
// consecutive threads write consecutive positions of each digit's run.
__global__ void __launch_bounds__(RS_THREADS) rs_scatter_kernel(
    const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin,
    unsigned long long* __restrict__ kout, uint32_t* __restrict__ vout, int64_t N, int shift,
    const uint32_t* __restrict__ offsets, int64_t tiles) {
    __shared__ uint32_t cnt[RS_WARPS][256];
    __shared__ uint32_t tile_off[256];
    __shared__ uint32_t dstart[256];
    __shared__ uint32_t scratch[32];
    __shared__ unsigned long long skey[RS_TILE];
    __shared__ uint32_t sval[RS_TILE];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    tile_off[threadIdx.x] = offsets[(int64_t)threadIdx.x * tiles + blockIdx.x];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
    const int wbase = warp * (RS_ITEMS * 32);
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long k[RS_ITEMS];
    uint32_t local[RS_ITEMS];
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        const int64_t idx = tbase + wbase + it * 32 + lane;
        const bool valid = idx < N;
        k[it] = valid ? kin[idx] : 0ull;
        const unsigned d = (unsigned)(k[it] >> shift) & 255u;
        unsigned peers = __ballot_sync(FULL, valid);
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const unsigned bb = __ballot_sync(FULL, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == leader) {
            old = cnt[warp][d];
            cnt[warp][d] = old + __popc(peers);
        }
        old = __shfl_sync(FULL, old, leader < 0 ? 0 : leader);
        local[it] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    {   // per digit: exclusive prefix over warps, then the tile-local start of each digit
        const int d = threadIdx.x;
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t t = cnt[w][d];
            cnt[w][d] = sum;
            sum += t;
        }
        uint32_t tot;
        dstart[d] = block_excl_scan<uint32_t>(sum, 0u, OpAdd<uint32_t>(), scratch, &tot);
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        const int64_t idx = tbase + wbase + it * 32 + lane;
        if (idx < N) {
            const unsigned d = (unsigned)(k[it] >> shift) & 255u;
            const uint32_t lp = dstart[d] + cnt[warp][d] + local[it];
            skey[lp] = k[it];
            sval[lp] = vin[idx];
        }
    }
    __syncthreads();
    const int64_t rem = N - tbase;
    const int valid_count = rem < RS_TILE ? (int)rem : RS_TILE;
    for (int i = threadIdx.x; i < valid_count; i += RS_THREADS) {
        const unsigned long long key = skey[i];
        const unsigned d = (unsigned)(key >> shift) & 255u;
        const uint32_t gpos = tile_off[d] + (uint32_t)(i - dstart[d]);
        kout[gpos] = key;
        vout[gpos] = sval[i];
    }
}

// ---------------------------------------------------------- one-sweep passes
// The same stable LSD sort with a single launch per digit, after the
// decoupled look-back of Merrill and Garland's single-pass prefix scan as
// Adinets and Merrill's Onesweep applies it to radix sorting: the digit
// histograms of all passes come from one read of the keys, and in a pass each
// CTA takes the next tile by ticket, ranks it, publishes its per-digit counts,
// then adds up its predecessors' counts walking back until a tile whose
// inclusive prefix is already published, and publishes its own.  A (tile,
// digit) status word holds a 2-bit state over a 30-bit count (N < 2^30).
constexpr int OS_THREADS = 1024, OS_ITEMS = 8, OS_TILE = OS_THREADS * OS_ITEMS;
constexpr int OS_CTAS = 1;  // resident per SM
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr uint32_t OS_AGG = 1u << 30, OS_INC = 2u << 30, OS_COUNT = OS_AGG - 1u;
constexpr uint32_t OS_WAIT = 1u << 20;  // polls of one predecessor's status before the wait gives up
constexpr int OS_LOOK = 16;             // predecessors' status words read at once in the look-back
// keys, rows in tile order, rows as loaded (the ranking's digit masks use the keys' room first)
constexpr size_t OS_SMEM = (size_t)OS_TILE * (sizeof(unsigned long long) + 2 * sizeof(uint32_t));
static_assert(OS_WARPS * 256 * sizeof(uint32_t) <= OS_TILE * sizeof(unsigned long long), "masks fit the keys' room");
constexpr int OS_HIST_THREADS = 256, OS_HIST_UNROLL = 4;

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// hist[p][d] += the keys whose digit p (bits shift0 + 8p ..) is d
__global__ void __launch_bounds__(OS_HIST_THREADS) os_hist_kernel(const unsigned long long* __restrict__ keys,
                                                                  int64_t N, int shift0, int passes,
                                                                  uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[8 * 256];
    for (int i = threadIdx.x; i < 8 * 256; i += OS_HIST_THREADS) h[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * OS_HIST_THREADS;
    for (int64_t i0 = (int64_t)blockIdx.x * OS_HIST_THREADS + threadIdx.x; i0 < N; i0 += stride * OS_HIST_UNROLL) {
        unsigned long long k[OS_HIST_UNROLL];
#pragma unroll
        for (int u = 0; u < OS_HIST_UNROLL; ++u) {
            const int64_t i = i0 + u * stride;
            k[u] = i < N ? keys[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < OS_HIST_UNROLL; ++u) {
            if (i0 + u * stride >= N) break;
            for (int p = 0; p < passes; ++p)
                atomicAdd(&h[p * 256 + ((unsigned)(k[u] >> (shift0 + 8 * p)) & 255u)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * 256; i += OS_HIST_THREADS)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One digit pass.  ghist: this pass's digit histogram over all keys; status:
// tiles x 256 words, zero before the pass; ticket: zero before the pass;
// err: set when a look-back wait gave up (the output is then not sorted).
// sax_dst (the last pass of a build whose rows stay in input order, else
// null): each pair's SAX word sax_src[row] and its row id also go to the
// pair's final position in sax_dst / orig_dst, the random 16-byte gathers
// overlapping the pass instead of running as a launch of their own.
// The tile's digit counts are taken and published as soon as its keys are in,
// and the first 256 threads (one digit each) walk back while the other warps
// rank their keys; the walk reads OS_LOOK predecessors' words at a time, so
// that a run of tiles that have published only their own counts costs one
// round trip per OS_LOOK of them.
__global__ void __launch_bounds__(OS_THREADS, OS_CTAS) os_scatter_kernel(
    const unsigned long long* __restrict__ kin, const uint32_t* __restrict__ vin,
    unsigned long long* __restrict__ kout, uint32_t* __restrict__ vout, int64_t N, int shift,
    const uint32_t* __restrict__ ghist, uint32_t* status, uint32_t* ticket, unsigned* err,
    const uint4* __restrict__ sax_src, uint4* __restrict__ sax_dst, uint32_t* __restrict__ orig_dst) {
    extern __shared__ __align__(16) unsigned char os_smem[];
    unsigned long long* skey = reinterpret_cast<unsigned long long*>(os_smem);
    uint32_t* sval = reinterpret_cast<uint32_t*>(skey + OS_TILE);
    uint32_t* sval_in = sval + OS_TILE;
    uint32_t* masks = reinterpret_cast<uint32_t*>(os_smem);  // [warp][digit] lanes, while ranking
    __shared__ uint32_t cnt[OS_WARPS][256];  // warp's count, then its digit's tile-local start
    __shared__ uint32_t hist[256];           // the tile's digit counts
    __shared__ uint32_t dpos[256];           // output position of the tile's element i of digit d: dpos[d] + i
    __shared__ unsigned long long scratch[32];
    __shared__ uint32_t s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    for (int i = threadIdx.x; i < OS_WARPS * 256; i += OS_THREADS) {
        (&cnt[0][0])[i] = 0;
        masks[i] = 0;
    }
    if (threadIdx.x < 256) hist[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t t = s_tile;
    const int64_t tbase = (int64_t)t * OS_TILE;
    const int valid = (int)(N - tbase < OS_TILE ? N - tbase : OS_TILE);
    // the tile's rows come into shared memory meanwhile (16-byte pieces, the
    // ragged end one by one)
    {
        const int whole = valid / 4;
        for (int c = threadIdx.x; c < whole; c += OS_THREADS) cp_async16(sval_in + 4 * c, vin + tbase + 4 * c);
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int i = whole * 4 + threadIdx.x; i < valid; i += OS_THREADS) sval_in[i] = vin[tbase + i];
    }
    const int wbase = warp * (OS_ITEMS * 32);
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long k[OS_ITEMS];
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const int i = wbase + it * 32 + lane;
        k[it] = i < valid ? kin[tbase + i] : 0ull;
    }
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it)
        if (wbase + it * 32 + lane < valid) atomicAdd(&hist[(unsigned)(k[it] >> shift) & 255u], 1u);
    __syncthreads();
    // ranks inside the warp: the lanes of an item with the same digit find one
    // another through the warp's digit mask (tile order is warp, item, lane:
    // stable)
    uint32_t local[OS_ITEMS];
    auto rank = [&]() {
        uint32_t* wm = masks + warp * 256;
#pragma unroll
        for (int it = 0; it < OS_ITEMS; ++it) {
            const bool ok = wbase + it * 32 + lane < valid;
            const unsigned d = (unsigned)(k[it] >> shift) & 255u;
            if (ok) atomicOr(&wm[d], 1u << lane);
            __syncwarp();
            const unsigned peers = ok ? wm[d] : 0u;
            __syncwarp();
            const int leader = ok ? __ffs(peers) - 1 : lane;
            uint32_t old = 0;
            if (ok && lane == leader) {
                old = cnt[warp][d];
                cnt[warp][d] = old + __popc(peers);
                wm[d] = 0u;
            }
            old = __shfl_sync(FULL, old, leader);
            local[it] = old + __popc(peers & lt);
            __syncwarp();
        }
    };
    uint32_t tot = 0, gh = 0, before = 0;
    if (threadIdx.x < 256) {
        // the tile's count of digit d published at once, then the digit's
        // elements in the tiles before this one
        const int d = threadIdx.x;
        tot = hist[d];
        uint32_t* mine = status + (size_t)t * 256 + d;
        st_relaxed_u32(mine, (t == 0 ? OS_INC : OS_AGG) | tot);
        gh = ghist[d];
        int64_t j = (int64_t)t - 1;
        uint32_t polls = 0;
        while (j >= 0) {
            uint32_t w[OS_LOOK];
#pragma unroll
            for (int u = 0; u < OS_LOOK; ++u)
                w[u] = j - u >= 0 ? ld_relaxed_u32(status + (size_t)(j - u) * 256 + d) : OS_INC;
            bool done = false;
            int used = 0;  // words taken, in order, up to the first not yet published
#pragma unroll
            for (int u = 0; u < OS_LOOK; ++u) {
                if (done || used < u) continue;
                if (!(w[u] & (OS_AGG | OS_INC))) continue;
                before += w[u] & OS_COUNT;
                used = u + 1;
                if (w[u] & OS_INC) done = true;
            }
            if (done) break;
            j -= used;
            if (used == 0) {
                if (++polls >= OS_WAIT) {
                    atomicOr(err, 1u);
                    break;
                }
                __nanosleep(32);
            }
        }
        if (t > 0) st_relaxed_u32(mine, OS_INC | (before + tot));
        rank();
    } else {
        rank();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // the digits' starts: in the whole pass (from the histogram) and in the tile
    // (one scan of both, packed: a tile's counts sum to at most OS_TILE)
    unsigned long long all;
    const unsigned long long ex = block_excl_scan<unsigned long long>(
        threadIdx.x < 256 ? ((unsigned long long)gh << 32) | tot : 0ull, 0ull, OpAdd<unsigned long long>(), scratch,
        &all);
    if (threadIdx.x < 256) {
        const int d = threadIdx.x;
        uint32_t run = (uint32_t)ex;  // each warp's first position of digit d in the tile
#pragma unroll
        for (int w = 0; w < OS_WARPS; ++w) {
            const uint32_t c = cnt[w][d];
            cnt[w][d] = run;
            run += c;
        }
        dpos[d] = (uint32_t)(ex >> 32) + before - (uint32_t)ex;
    }
    __syncthreads();
    // the tile reordered by digit in shared memory
#pragma unroll
    for (int it = 0; it < OS_ITEMS; ++it) {
        const int i = wbase + it * 32 + lane;
        if (i < valid) {
            const uint32_t lp = cnt[warp][(unsigned)(k[it] >> shift) & 255u] + local[it];
            skey[lp] = k[it];
            sval[lp] = sval_in[i];
        }
    }
    __syncthreads();
    // written out so that consecutive threads write consecutive positions of
    // each digit's run
    if (sax_dst) {
        // (the gathers of all the thread's pairs issued before any store)
        uint4 w[OS_ITEMS];
#pragma unroll
        for (int u = 0; u < OS_ITEMS; ++u) {
            const int i = threadIdx.x + u * OS_THREADS;
            if (i < valid) w[u] = sax_src[sval[i]];
        }
#pragma unroll
        for (int u = 0; u < OS_ITEMS; ++u) {
            const int i = threadIdx.x + u * OS_THREADS;
            if (i < valid) {
                const unsigned long long key = skey[i];
                const uint32_t gpos = dpos[(unsigned)(key >> shift) & 255u] + (uint32_t)i, row = sval[i];
                kout[gpos] = key;
                vout[gpos] = row;
                sax_dst[gpos] = w[u];
                orig_dst[gpos] = row;
            }
        }
        return;
    }
    for (int i = threadIdx.x; i < valid; i += OS_THREADS) {
        const unsigned long long key = skey[i];
        const uint32_t gpos = dpos[(unsigned)(key >> shift) & 255u] + (uint32_t)i;
        kout[gpos] = key;
        vout[gpos] = sval[i];
    }
}

// ============================================================== leaf formation
__device__ __forceinline__ int lcp_bits(unsigned long long a, unsigned long long b, int keybits) {
    int l = (a == b) ? 64 : __clzll((long long)(a ^ b));
    return l < keybits ? l : keybits;
}

// c[i] = common prefix of keys i-1, i (c[0] = 0); a[j] = common prefix of keys
// j and j+L (the whole window j..j+L shares it, the keys being sorted).
__global__ void lf_lcp_kernel(const unsigned long long* __restrict__ keys, int64_t N, int64_t L,
                              int keybits, uint8_t* __restrict__ c, uint8_t* __restrict__ a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long ki = keys[i];
        c[i] = (uint8_t)(i == 0 ? 0 : lcp_bits(keys[i - 1], ki, keybits));
        if (i + L < N) a[i] = (uint8_t)lcp_bits(ki, keys[i + L], keybits);
    }
}

// prefix max P and suffix max S of a[] inside consecutive blocks of L entries
// (van Herk / Gil-Werman sliding-window maximum)
constexpr int LF_THREADS = 256, LF_ITEMS = 8;

// P[e] = max a[b0 .. e] and S[e] = max a[e .. b1 - 1] inside each block [b0, b1)
// of L positions: a warp per block, LF_ITEMS consecutive positions per lane and
// a warp max-scan per chunk of 32 x LF_ITEMS (no block barrier).
__global__ void __launch_bounds__(LF_THREADS) lf_blockmax_kernel(const uint8_t* __restrict__ a,
                                                                  int64_t NA, int64_t L,
                                                                  uint8_t* __restrict__ P,
                                                                  uint8_t* __restrict__ S) {
    constexpr int CH = 32 * LF_ITEMS;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t blk = gw; blk * L < NA; blk += nw) {
        const int64_t b0 = blk * L, b1 = std::min(b0 + L, NA);
        uint32_t carry = 0;
        for (int64_t c0 = b0; c0 < b1; c0 += CH) {
            const int64_t t0 = c0 + (int64_t)lane * LF_ITEMS;
            uint32_t run[LF_ITEMS];
            uint32_t m = 0;
#pragma unroll
            for (int j = 0; j < LF_ITEMS; ++j) {
                if (t0 + j < b1) m = max(m, (uint32_t)a[t0 + j]);
                run[j] = m;
            }
            const uint32_t inc = warp_incl_scan<uint32_t>(m, OpMax<uint32_t>());
            uint32_t before = __shfl_up_sync(FULL, inc, 1);
            if (lane == 0) before = 0;
            const uint32_t tot = __shfl_sync(FULL, inc, 31);
#pragma unroll
            for (int j = 0; j < LF_ITEMS; ++j)
                if (t0 + j < b1) P[t0 + j] = (uint8_t)max(carry, max(before, run[j]));
            carry = max(carry, tot);
        }
        carry = 0;
        for (int64_t c1 = b1; c1 > b0; c1 -= CH) {
            // position e = c1 - 1 - (lane * ITEMS + j), walking right to left
            const int64_t t1 = c1 - 1 - (int64_t)lane * LF_ITEMS;
            uint32_t run[LF_ITEMS];
            uint32_t m = 0;
#pragma unroll
            for (int j = 0; j < LF_ITEMS; ++j) {
                const int64_t e = t1 - j;
                if (e >= b0 && e >= c1 - CH) m = max(m, (uint32_t)a[e]);
                run[j] = m;
            }
            const uint32_t inc = warp_incl_scan<uint32_t>(m, OpMax<uint32_t>());
            uint32_t before = __shfl_up_sync(FULL, inc, 1);
            if (lane == 0) before = 0;
            const uint32_t tot = __shfl_sync(FULL, inc, 31);
#pragma unroll
            for (int j = 0; j < LF_ITEMS; ++j) {
                const int64_t e = t1 - j;
                if (e >= b0 && e >= c1 - CH) S[e] = (uint8_t)max(carry, max(before, run[j]));
            }
            carry = max(carry, tot);
        }
    }
}

// A boundary (new leaf) starts at position i when the node that holds both
// i-1 and i splits: always at the root (common prefix < 16 bits); below the
// root when that node, the run of keys sharing c[i] bits around i, holds more
// than L series, i.e. some window of L+1 consecutive keys containing i-1 and
// i shares c[i] bits: max(a[i-L .. i-1]) >= c[i].
// 1 if series i starts a leaf: the first series, a new root key, or a split
// at depth ci (the common prefix with the previous series) that the window of
// L series ending at i - 1 does not cover (its common prefix M is >= ci).
// P / S: prefix / suffix maxima of a inside blocks of L (N < 2^32: 32-bit
// index arithmetic, one division).
__device__ __forceinline__ uint32_t leaf_start_flag(const uint8_t* __restrict__ c, const uint8_t* __restrict__ P,
                                                    const uint8_t* __restrict__ S, uint32_t i, uint32_t N,
                                                    uint32_t L, int keybits) {
    if (i == 0) return 1u;
    const int ci = c[i];
    if (ci < ROOT_BITS) return 1u;
    if (ci >= keybits) return 0u;
    const uint32_t NA = N > L ? N - L : 0u;
    if (NA == 0) return 0u;  // M = 0 < ci
    const uint32_t lo = i > L ? i - L : 0u;
    const uint32_t hi = i - 1 < NA - 1 ? i - 1 : NA - 1;
    if (lo > hi) return 0u;
    const uint32_t q = lo / L, r = lo - q * L;
    int M;
    if (hi < (q + 1) * L)  // lo and hi in one block
        M = r == 0 ? P[hi] : S[lo];
    else
        M = max(S[lo], P[hi]);
    return M >= ci ? 1u : 0u;
}

// Leaf starts in two passes over tiles of LF_TILE series (LF_PER consecutive
// series per thread): the number of starts of each tile, then (after a scan of
// those counts) the starts themselves, written in order.
constexpr int LF_PER = 16, LF_TILE = 256 * LF_PER;
__global__ void __launch_bounds__(256) lf_count_kernel(const uint8_t* __restrict__ c, const uint8_t* __restrict__ P,
                                                       const uint8_t* __restrict__ S, int64_t N, int64_t L,
                                                       int keybits, uint32_t* __restrict__ tile_count) {
    __shared__ uint32_t scratch[32];
    const int64_t i0 = (int64_t)blockIdx.x * LF_TILE + (int64_t)threadIdx.x * LF_PER;
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < LF_PER; ++j)
        if (i0 + j < N) n += leaf_start_flag(c, P, S, (uint32_t)(i0 + j), (uint32_t)N, (uint32_t)L, keybits);
    uint32_t tot;
    block_excl_scan<uint32_t>(n, 0u, OpAdd<uint32_t>(), scratch, &tot);
    if (threadIdx.x == 0) tile_count[blockIdx.x] = tot;
}
__global__ void __launch_bounds__(256) lf_emit_kernel(const uint8_t* __restrict__ c, const uint8_t* __restrict__ P,
                                                      const uint8_t* __restrict__ S, int64_t N, int64_t L,
                                                      int keybits, const uint32_t* __restrict__ tile_off,
                                                      uint32_t* __restrict__ starts, uint32_t count) {
    __shared__ uint32_t scratch[32];
    const int64_t i0 = (int64_t)blockIdx.x * LF_TILE + (int64_t)threadIdx.x * LF_PER;
    uint32_t f = 0;  // bit j: series i0 + j starts a leaf
#pragma unroll
    for (int j = 0; j < LF_PER; ++j)
        if (i0 + j < N && leaf_start_flag(c, P, S, (uint32_t)(i0 + j), (uint32_t)N, (uint32_t)L, keybits))
            f |= 1u << j;
    uint32_t tot;
    uint32_t o = tile_off[blockIdx.x] + block_excl_scan<uint32_t>(__popc(f), 0u, OpAdd<uint32_t>(), scratch, &tot);
    for (; f; f &= f - 1u) starts[o++] = (uint32_t)(i0 + __ffs(f) - 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) starts[count] = (uint32_t)N;
}

// leaves over capacity (only runs of identical keys) are cut into pieces of L
__global__ void lf_pieces_kernel(const uint32_t* __restrict__ starts, uint32_t L0, int64_t L,
                                 uint32_t* __restrict__ pieces) {
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < L0;
         l += (int64_t)gridDim.x * blockDim.x) {
        int64_t sz = (int64_t)starts[l + 1] - starts[l];
        pieces[l] = (uint32_t)((sz + L - 1) / L);
    }
}

__global__ void lf_expand_kernel(const uint32_t* __restrict__ starts, const uint32_t* __restrict__ poff,
                                 uint32_t L0, int64_t L, int64_t N, uint32_t* __restrict__ leaf_begin,
                                 uint32_t nleaves) {
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < L0;
         l += (int64_t)gridDim.x * blockDim.x) {
        int64_t s0 = starts[l], s1 = starts[l + 1];
        uint32_t o = poff[l];
        for (int64_t p = s0; p < s1; p += L) leaf_begin[o++] = (uint32_t)p;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) leaf_begin[nleaves] = (uint32_t)N;
}

// ============================================================== permute, envelopes
// Rows, SAX words and original ids gathered into leaf order.  Rows move through
// the TMA engine: thread 0 of each CTA gathers a batch of rows (16 KB) into one
// of PM_STAGES shared-memory stages with bulk copies completed on the stage's
// mbarrier, then writes the whole batch - contiguous in the output - with one
// bulk store, refilling the stage once that store has read it.  Up to
// PM_STAGES batches are in flight per CTA.  The other threads copy the SAX
// words and ids.  Waits are bounded: on a timeout the kernel flags `err`,
// waits (bounded) for its copies in flight, and returns.
constexpr int PM_THREADS = 128, PM_STAGES = 4, PM_STAGE_BYTES = 16384;
constexpr uint32_t PM_MAX_TRIES = 1u << 24;

__global__ void __launch_bounds__(PM_THREADS) permute_kernel(const float* __restrict__ x, int n,
                                                             const uint32_t* __restrict__ ids,
                                                             int64_t N, float* __restrict__ xp,
                                                             const uint4* __restrict__ sax_in,
                                                             uint4* __restrict__ sax_out,
                                                             uint32_t* __restrict__ orig,
                                                             unsigned* err) {
    extern __shared__ __align__(1024) unsigned char pm_stage[];
    __shared__ __align__(8) uint64_t bar[PM_STAGES];
    const uint32_t rowbytes = (uint32_t)n * 4u;
    const int B = (int)(PM_STAGE_BYTES / rowbytes) > 0 ? (int)(PM_STAGE_BYTES / rowbytes) : 1;
    // contiguous output range of this CTA, in whole batches
    const int64_t nbatch_all = (N + B - 1) / B;
    const int64_t per = (nbatch_all + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = std::min<int64_t>((int64_t)blockIdx.x * per * B, N);
    const int64_t r1 = std::min<int64_t>(r0 + per * B, N);
    if (threadIdx.x == 0) {
        for (int st = 0; st < PM_STAGES; ++st) mbar_init(&bar[st], 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int64_t nb = (r1 - r0 + B - 1) / B;
        auto issue = [&](int64_t b) {
            const int st = (int)(b % PM_STAGES);
            const int64_t rb = r0 + b * B;
            const int rows = (int)std::min<int64_t>(B, r1 - rb);
            unsigned char* dst = pm_stage + (size_t)st * PM_STAGE_BYTES;
            mbar_arrive_expect_tx(&bar[st], (uint32_t)rows * rowbytes);
#pragma unroll 4
            for (int i = 0; i < rows; ++i) {
                const uint32_t src = ids[rb + i];
                bulk_load(dst + (size_t)i * rowbytes, x + (int64_t)src * n, rowbytes, &bar[st]);
            }
        };
        const int64_t pro = nb < PM_STAGES ? nb : PM_STAGES;
        for (int64_t b = 0; b < pro; ++b) issue(b);
        int64_t done = 0;
        for (int64_t b = 0; b < nb; ++b) {
            const int st = (int)(b % PM_STAGES);
            const uint32_t parity = (uint32_t)((b / PM_STAGES) & 1);
            if (!mbar_wait_bounded(&bar[st], parity, PM_MAX_TRIES)) {
                atomicOr(err, 1u);
                break;
            }
            done = b + 1;
            fence_proxy_async_smem();
            const int64_t rb = r0 + b * B;
            const int rows = (int)std::min<int64_t>(B, r1 - rb);
            bulk_store(xp + rb * n, pm_stage + (size_t)st * PM_STAGE_BYTES, (uint32_t)rows * rowbytes);
            bulk_commit();
            if (b + PM_STAGES < nb) {
                bulk_wait_read_all();
                issue(b + PM_STAGES);
            }
        }
        // loads issued but not awaited (only after a timeout): bounded wait
        const int64_t issued = nb < done + PM_STAGES ? nb : done + PM_STAGES;
        for (int64_t b = done; b < issued; ++b)
            mbar_wait_bounded(&bar[b % PM_STAGES], (uint32_t)((b / PM_STAGES) & 1), PM_MAX_TRIES);
        bulk_wait_all();
    } else {
        for (int64_t r = r0 + threadIdx.x - 1; r < r1; r += PM_THREADS - 1) {
            const uint32_t src = ids[r];
            sax_out[r] = sax_in[src];
            orig[r] = src;
        }
    }
}

// SAX words and original ids alone into leaf order, for an index that reads
// the caller's rows in place: thread per position.
__global__ void __launch_bounds__(256) permute_sax_kernel(const uint32_t* __restrict__ ids, int64_t N,
                                                         const uint4* __restrict__ sax_in,
                                                         uint4* __restrict__ sax_out,
                                                         uint32_t* __restrict__ orig) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t src = ids[r];
        ISAX_CHECK(src < (uint64_t)N, CHK_BUILD_ID);
        sax_out[r] = sax_in[src];
        orig[r] = src;
    }
}

// The same gather with plain 16-byte loads and stores, one warp per row, for
// an index whose rows live in host memory: the output (and the input, when it
// is host memory) is reached over the CPU-GPU link, where many independent
// small requests in flight keep the link busy.
__global__ void __launch_bounds__(256) permute_plain_kernel(const float* __restrict__ x, int n,
                                                           const uint32_t* __restrict__ ids, int64_t N,
                                                           float* __restrict__ xp,
                                                           const uint4* __restrict__ sax_in,
                                                           uint4* __restrict__ sax_out,
                                                           uint32_t* __restrict__ orig) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nv = n / 4;
    for (int64_t r = gw; r < N; r += nw) {
        const uint32_t src = ids[r];
        const float4* s4 = reinterpret_cast<const float4*>(x + (int64_t)src * n);
        float4* d4 = reinterpret_cast<float4*>(xp + r * n);
        for (int i = lane; i < nv; i += 32) d4[i] = s4[i];
        if (lane == 0) {
            sax_out[r] = sax_in[src];
            orig[r] = src;
        }
    }
}

__device__ __forceinline__ uint4 vmin4(uint4 a, uint4 b) {
    return make_uint4(__vminu4(a.x, b.x), __vminu4(a.y, b.y), __vminu4(a.z, b.z), __vminu4(a.w, b.w));
}
__device__ __forceinline__ uint4 vmax4(uint4 a, uint4 b) {
    return make_uint4(__vmaxu4(a.x, b.x), __vmaxu4(a.y, b.y), __vmaxu4(a.z, b.z), __vmaxu4(a.w, b.w));
}
__device__ __forceinline__ uint4 shfl_xor_u4(uint4 v, int off) {
    return make_uint4(__shfl_xor_sync(FULL, v.x, off), __shfl_xor_sync(FULL, v.y, off),
                      __shfl_xor_sync(FULL, v.z, off), __shfl_xor_sync(FULL, v.w, off));
}

// one warp per leaf: byte-wise min and max of the members' symbols
__global__ void __launch_bounds__(256) envelope_kernel(const uint4* __restrict__ sax,
                                                       const uint32_t* __restrict__ leaf_begin,
                                                       int64_t L,
                                                       const unsigned long long* __restrict__ keys,
                                                       uint4* __restrict__ env,
                                                       unsigned long long* __restrict__ leaf_key,
                                                       unsigned long long key_mask,
                                                       uint32_t* __restrict__ max_leaf) {
    __shared__ uint32_t big[8];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t biggest = 0;  // the largest leaf this warp saw (one atomic per block at the end)
    for (int64_t l = gw; l < L; l += nw) {
        const uint32_t b = leaf_begin[l], e = leaf_begin[l + 1];
        ISAX_CHECK(b < e, CHK_LEAF_RANGE);
        uint4 mn = make_uint4(FULL, FULL, FULL, FULL), mx = make_uint4(0, 0, 0, 0);
        // four words per lane in flight
        uint32_t r = b + lane;
        for (; r + 96 < e; r += 128) {
            const uint4 s0 = sax[r], s1 = sax[r + 32], s2 = sax[r + 64], s3 = sax[r + 96];
            mn = vmin4(vmin4(mn, s0), vmin4(s1, vmin4(s2, s3)));
            mx = vmax4(vmax4(mx, s0), vmax4(s1, vmax4(s2, s3)));
        }
        for (; r < e; r += 32) {
            const uint4 s = sax[r];
            mn = vmin4(mn, s);
            mx = vmax4(mx, s);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            mn = vmin4(mn, shfl_xor_u4(mn, off));
            mx = vmax4(mx, shfl_xor_u4(mx, off));
        }
        if (lane == 0) {
            env[2 * l] = mn;
            env[2 * l + 1] = mx;
            leaf_key[l] = keys[b] & key_mask;
        }
        biggest = max(biggest, e - b);
    }
    if (lane == 0) big[threadIdx.x >> 5] = biggest;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t m = 0;
        for (int w = 0; w < 8; ++w) m = max(m, big[w]);
        if (m) atomicMax(max_leaf, m);
    }
}


// ============================================================== balanced-split leaves
// ADS+ node splitting (Section II, ADS+ Index), built one tree level at a time
// over the whole collection.  Positions are grouped by node, each node's
// series in row order.  A level decides, for every node holding more than
// leaf_size series, the segment whose next bit divides its first leaf_size + 1
// series most evenly (what a node filled one series at a time sees when it
// first overflows), then partitions every such node stably by that bit, child
// 0 first.  Node state: first position, size, bits taken on each segment
// (4-bit fields), tree node id.
constexpr unsigned long long BL_BITS1 = 0x1111111111111111ull;  // one bit on every segment

__device__ __forceinline__ int bl_nib(unsigned long long bits, int g) {
    return (int)(bits >> (4 * g)) & 15;
}

// flags[i] = 1 where a run of equal root keys (the key's top 16 bits) starts
__global__ void bl_root_flags_kernel(const unsigned long long* __restrict__ keys, int64_t N,
                                     uint32_t* __restrict__ flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || (keys[i] >> 48) != (keys[i - 1] >> 48)) ? 1u : 0u;
}

// level 0: node j is run j of the root-key order
__global__ void bl_root_nodes_kernel(const unsigned long long* __restrict__ keys,
                                     const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos,
                                     int64_t N, uint32_t* __restrict__ elem_node,
                                     uint32_t* __restrict__ nstart, int32_t* __restrict__ root) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = pos[i] + flags[i] - 1u;
        elem_node[i] = j;
        if (flags[i]) {
            nstart[j] = (uint32_t)i;
            root[keys[i] >> 48] = (int32_t)j;
        }
    }
}

__global__ void bl_root_fill_kernel(const uint32_t* __restrict__ nstart, int64_t nodes, int64_t N,
                                    uint32_t* __restrict__ ncnt, unsigned long long* __restrict__ nbits,
                                    uint32_t* __restrict__ ngid) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nodes;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t e = j + 1 < nodes ? nstart[j + 1] : (uint32_t)N;
        ncnt[j] = e - nstart[j];
        nbits[j] = BL_BITS1;
        ngid[j] = (uint32_t)j;
    }
}

// warp per node: the split segment of every node over capacity (-1: no split,
// also when all 16 segments are at full cardinality)
__global__ void __launch_bounds__(256) bl_decide_kernel(const uint4* __restrict__ sax,
                                                        const uint32_t* __restrict__ nstart,
                                                        const uint32_t* __restrict__ ncnt,
                                                        const unsigned long long* __restrict__ nbits,
                                                        int64_t nodes, uint32_t cap, int cbits,
                                                        int32_t* __restrict__ seg,
                                                        uint32_t* __restrict__ split) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = gw; j < nodes; j += nw) {
        int best = -1;
        if (ncnt[j] > cap) {
            const unsigned long long bits = nbits[j];
            const uint32_t b = nstart[j], m = cap + 1u;
            int sh[16];
            uint32_t ones[16];
#pragma unroll
            for (int g = 0; g < 16; ++g) {
                const int nb = bl_nib(bits, g);
                sh[g] = nb < cbits ? cbits - 1 - nb : -1;
                ones[g] = 0;
            }
            for (uint32_t p = lane; p < m; p += 32) {
                const uint4 v = sax[b + p];
                const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int g = 0; g < 16; ++g) {
                    const uint32_t sym = (wd[g >> 2] >> (8 * (g & 3))) & 255u;
                    ones[g] += sh[g] >= 0 ? (sym >> sh[g]) & 1u : 0u;
                }
            }
            long long best_bal = 0;
#pragma unroll
            for (int g = 0; g < 16; ++g) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) ones[g] += __shfl_xor_sync(FULL, ones[g], off);
                const long long bal = llabs(2LL * (long long)ones[g] - (long long)m);
                if (sh[g] >= 0 && (best < 0 || bal < best_bal)) {
                    best = g;
                    best_bal = bal;
                }
            }
        }
        if (lane == 0) {
            seg[j] = best;
            split[j] = best >= 0 ? 1u : 0u;
        }
    }
}

// zf[i] = 1 unless position i is in a splitting node and its next bit there is 1
__global__ void bl_bit_kernel(const uint4* __restrict__ sax, const uint32_t* __restrict__ elem_node,
                              const int32_t* __restrict__ seg, const unsigned long long* __restrict__ nbits,
                              int64_t N, int cbits, uint32_t* __restrict__ zf) {
    const uint8_t* s8 = reinterpret_cast<const uint8_t*>(sax);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = elem_node[i];
        const int s = seg[j];
        uint32_t f = 1u;
        if (s >= 0) {
            const uint32_t sym = s8[i * 16 + s];
            f = ((sym >> (cbits - 1 - bl_nib(nbits[j], s))) & 1u) ^ 1u;
        }
        zf[i] = f;
    }
}

// the next level's nodes: a splitting node j becomes its children at j + spos[j]
// (bit 0) and the one after (bit 1); the tree records the split
__global__ void bl_nodes_kernel(int64_t nodes, const uint32_t* __restrict__ nstart,
                                const uint32_t* __restrict__ ncnt, const unsigned long long* __restrict__ nbits,
                                const uint32_t* __restrict__ ngid, const int32_t* __restrict__ seg,
                                const uint32_t* __restrict__ spos, const uint32_t* __restrict__ Z,
                                const uint32_t* __restrict__ ztot, int64_t N, uint32_t next_gid,
                                uint32_t* __restrict__ nstart2, uint32_t* __restrict__ ncnt2,
                                unsigned long long* __restrict__ nbits2, uint32_t* __restrict__ ngid2,
                                int2* __restrict__ tree) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nodes;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t o = (uint32_t)j + spos[j];
        const int s = seg[j];
        if (s < 0) {
            nstart2[o] = nstart[j];
            ncnt2[o] = ncnt[j];
            nbits2[o] = nbits[j];
            ngid2[o] = ngid[j];
            continue;
        }
        const uint32_t st = nstart[j], c = ncnt[j], e = st + c;
        const uint32_t zeros = (e < N ? Z[e] : *ztot) - Z[st];
        const unsigned long long nb = nbits[j] + (1ull << (4 * s));
        const uint32_t g0 = next_gid + 2u * spos[j];
        tree[ngid[j]] = make_int2((int)g0, s);
        nstart2[o] = st;
        ncnt2[o] = zeros;
        nbits2[o] = nb;
        ngid2[o] = g0;
        nstart2[o + 1] = st + zeros;
        ncnt2[o + 1] = c - zeros;
        nbits2[o + 1] = nb;
        ngid2[o + 1] = g0 + 1u;
    }
}

// stable partition of every splitting node by its bit; the rest stay in place
__global__ void bl_scatter_kernel(int64_t N, const uint4* __restrict__ sax_a, const uint32_t* __restrict__ id_a,
                                  const uint32_t* __restrict__ en_a, const int32_t* __restrict__ seg,
                                  const uint32_t* __restrict__ nstart, const uint32_t* __restrict__ ncnt,
                                  const uint32_t* __restrict__ spos, const uint32_t* __restrict__ zf,
                                  const uint32_t* __restrict__ Z, const uint32_t* __restrict__ ztot,
                                  uint4* __restrict__ sax_b, uint32_t* __restrict__ id_b,
                                  uint32_t* __restrict__ en_b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t j = en_a[i];
        const int s = seg[j];
        const uint32_t o = j + spos[j];
        int64_t dst = i;
        uint32_t nn = o;
        if (s >= 0) {
            const uint32_t st = nstart[j], e = st + ncnt[j];
            const uint32_t zs = Z[st], zeros = (e < N ? Z[e] : *ztot) - zs, zb = Z[i] - zs;
            if (zf[i]) {
                dst = (int64_t)st + zb;
            } else {
                dst = (int64_t)st + zeros + ((uint32_t)i - st - zb);
                nn = o + 1u;
            }
        }
        sax_b[dst] = sax_a[i];
        id_b[dst] = id_a[i];
        en_b[dst] = nn;
    }
}

__global__ void bl_leaf_flags_kernel(const uint32_t* __restrict__ ncnt, int64_t nodes,
                                     uint32_t* __restrict__ nonempty) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nodes;
         j += (int64_t)gridDim.x * blockDim.x)
        nonempty[j] = ncnt[j] > 0 ? 1u : 0u;
}

// the final nodes are the leaves in depth-first order; the empty ones are
// dropped and a descent that ends in one continues to the next leaf kept
__global__ void bl_leaves_kernel(int64_t nodes, const uint32_t* __restrict__ nstart,
                                 const uint32_t* __restrict__ ncnt, const uint32_t* __restrict__ ngid,
                                 const uint32_t* __restrict__ li, uint32_t L, int64_t N,
                                 uint32_t* __restrict__ leaf_begin, int2* __restrict__ tree) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nodes;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t l = li[j];
        if (ncnt[j] > 0) leaf_begin[l] = nstart[j];
        tree[ngid[j]] = make_int2(-1 - (int)(l < L ? l : L - 1u), -1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) leaf_begin[L] = (uint32_t)N;
}

// ============================================================== orchestration
namespace {

// Host-to-device copies on a stream of their own, each followed by an event
// that the build's stream waits for, so summarising one chunk overlaps the copy
// of the next.  The destructor waits for every copy issued: the host source is
// the caller's and is only borrowed for the call.
struct ChunkCopier {
    cudaStream_t main;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    explicit ChunkCopier(cudaStream_t st) : main(st) {
        ISAX_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        ISAX_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        // the copies start after what the build has queued (the destination's allocation)
        ISAX_CUDA_TRY(cudaEventRecord(ev, main));
        ISAX_CUDA_TRY(cudaStreamWaitEvent(cs, ev, 0));
    }
    void copy(void* dst, const void* src, size_t bytes) {
        ISAX_CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs));
        ISAX_CUDA_TRY(cudaEventRecord(ev, cs));
        ISAX_CUDA_TRY(cudaStreamWaitEvent(main, ev, 0));
    }
    ~ChunkCopier() {
        if (cs) {
            cudaStreamSynchronize(cs);
            cudaStreamDestroy(cs);
        }
        if (ev) cudaEventDestroy(ev);
    }
    ChunkCopier(const ChunkCopier&) = delete;
    ChunkCopier& operator=(const ChunkCopier&) = delete;
};

struct TempPool {
    cudaStream_t st;
    std::vector<void*> ptrs;
    template <typename T>
    T* get(size_t count) {
        void* p = dev_alloc(std::max<size_t>(count, 1) * sizeof(T), st);
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    void release(void* p) {
        auto it = std::find(ptrs.begin(), ptrs.end(), p);
        if (it != ptrs.end()) {
            dev_free(p, st);
            ptrs.erase(it);
        }
    }
    ~TempPool() {
        for (void* p : ptrs) dev_free(p, st);
    }
};

inline unsigned grid_for(int64_t work, int per_block, int num_sms, int max_per_sm = 16) {
    int64_t b = (work + per_block - 1) / per_block;
    int64_t cap = (int64_t)num_sms * max_per_sm;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

uint32_t read_u32(const uint32_t* p, cudaStream_t st) {
    uint32_t v = 0;
    ISAX_CUDA_TRY(cudaMemcpyAsync(&v, p, sizeof v, cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    return v;
}

// Stable LSD radix sort of (key, row) pairs on `passes` 8-bit digits, the
// lowest at bit `shift0`; the sorted pairs end in kA / vA.  One-sweep passes
// for N < 2^30, else three-phase ones.  A look-back wait that gave up sets
// *err and ends the build here, before anything reads the unsorted rows.
// With sax_dst, a one-sweep sort's last pass also writes sax_dst[i] =
// sax_src[vA[i]] and orig_dst[i] = vA[i]; returns whether it did.
bool radix_sort(unsigned long long*& kA, uint32_t*& vA, unsigned long long*& kB, uint32_t*& vB, int64_t N,
                int shift0, int passes, TempPool& tmp, cudaStream_t st, unsigned* err, int num_sms,
                const uint4* sax_src = nullptr, uint4* sax_dst = nullptr, uint32_t* orig_dst = nullptr) {
    if (N <= 0 || passes <= 0) return false;
    if (N < ((int64_t)1 << 30) && passes <= 8) {
        const int64_t tiles = (N + OS_TILE - 1) / OS_TILE;
        const size_t words = (size_t)passes * 256 + (size_t)passes + (size_t)passes * tiles * 256;
        uint32_t* ws = tmp.get<uint32_t>(words);
        uint32_t* hist = ws;
        uint32_t* tickets = ws + (size_t)passes * 256;
        uint32_t* status = tickets + passes;
        ISAX_CUDA_TRY(cudaMemsetAsync(ws, 0, words * sizeof(uint32_t), st));
        {
            ISAX_LAUNCH("os_hist", st);
            os_hist_kernel<<<grid_for(N, OS_HIST_THREADS * OS_HIST_UNROLL, num_sms, 8), OS_HIST_THREADS, 0, st>>>(
                kA, N, shift0, passes, hist);
        }
        {
            // the pass's shared memory (above the default limit), once per device
            // (setting it again is harmless)
            static bool attr_done[64] = {};
            int dev = -1;
            if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
            if (dev < 0 || dev >= 64 || !attr_done[dev]) {
                ISAX_CUDA_TRY(cudaFuncSetAttribute(os_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)OS_SMEM));
                if (dev >= 0 && dev < 64) attr_done[dev] = true;
            }
        }
        for (int pass = 0; pass < passes; ++pass) {
            ISAX_LAUNCH("os_scatter", st);
            const bool last = pass + 1 == passes;
            os_scatter_kernel<<<(unsigned)tiles, OS_THREADS, OS_SMEM, st>>>(
                kA, vA, kB, vB, N, shift0 + 8 * pass, hist + (size_t)pass * 256, status + (size_t)pass * tiles * 256,
                tickets + pass, err, sax_src, last ? sax_dst : nullptr, orig_dst);
            ISAX_CUDA_TRY(cudaGetLastError());
            std::swap(kA, kB);
            std::swap(vA, vB);
        }
        tmp.release(ws);
        if (read_u32(err, st)) throw Error{ISAX_ERR_TIMEOUT, "a look-back wait of the radix sort gave up"};
        return sax_dst != nullptr;
    }
    const int64_t tiles = (N + RS_TILE - 1) / RS_TILE;
    uint32_t* hist = tmp.get<uint32_t>((size_t)256 * tiles);
    uint32_t* sums = tmp.get<uint32_t>(scan_sums_len(256 * tiles));
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = shift0 + 8 * pass;
        {
        ISAX_LAUNCH("rs_hist", st);
        rs_hist_kernel<<<(unsigned)tiles, RS_THREADS, 0, st>>>(kA, N, shift, hist, tiles);
        }
        exclusive_scan(hist, hist, 256 * tiles, sums, st);
        {
        ISAX_LAUNCH("rs_scatter", st);
        rs_scatter_kernel<<<(unsigned)tiles, RS_THREADS, 0, st>>>(kA, vA, kB, vB, N, shift, hist, tiles);
        }
        ISAX_CUDA_TRY(cudaGetLastError());
        std::swap(kA, kB);
        std::swap(vA, vB);
    }
    tmp.release(hist);
    tmp.release(sums);
    return false;
}

// Leaves of the round-robin split, cut top-down from the sorted keys kA; fills
// ix->leaf_begin and returns the number of leaves.
uint32_t round_robin_leaves(isax_index* ix, TempPool& tmp, const unsigned long long* kA, int64_t N,
                            int leaf_size, int keybits, int num_sms, cudaStream_t st) {
    const int64_t Lc = leaf_size;
    const int64_t NA = N > Lc ? N - Lc : 0;
    uint8_t* c = tmp.get<uint8_t>(N);
    uint8_t* a = tmp.get<uint8_t>(NA);
    uint8_t* P = tmp.get<uint8_t>(NA);
    uint8_t* S = tmp.get<uint8_t>(NA);
    const int64_t tiles = (N + LF_TILE - 1) / LF_TILE;
    uint32_t* tcount = tmp.get<uint32_t>(tiles);
    uint32_t* toff = tmp.get<uint32_t>(tiles);
    uint32_t* sums = tmp.get<uint32_t>(scan_sums_len(tiles));
    {
    ISAX_LAUNCH("lf_lcp", st);
    lf_lcp_kernel<<<grid_for(N, 256, num_sms), 256, 0, st>>>(kA, N, Lc, keybits, c, a);
    }
    if (NA > 0) {
        ISAX_LAUNCH("lf_blockmax", st);
        int64_t nblk = (NA + Lc - 1) / Lc;
        lf_blockmax_kernel<<<(unsigned)std::min<int64_t>((nblk + LF_THREADS / 32 - 1) / (LF_THREADS / 32),
                                                         (int64_t)num_sms * 8),
                             LF_THREADS, 0, st>>>(a, NA, Lc, P, S);
    }
    {
    ISAX_LAUNCH("lf_count", st);
    lf_count_kernel<<<(unsigned)tiles, 256, 0, st>>>(c, P, S, N, Lc, keybits, tcount);
    }
    exclusive_scan(tcount, toff, tiles, sums, st);
    ISAX_CUDA_TRY(cudaGetLastError());
    uint32_t L0 = 0;
    ISAX_CUDA_TRY(cudaMemcpyAsync(&L0, sums + (scan_sums_len(tiles) - 1), sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    uint32_t* starts = tmp.get<uint32_t>((size_t)L0 + 1);
    {
    ISAX_LAUNCH("lf_emit", st);
    lf_emit_kernel<<<(unsigned)tiles, 256, 0, st>>>(c, P, S, N, Lc, keybits, toff, starts, L0);
    }
    uint32_t* pieces = tmp.get<uint32_t>(L0);
    uint32_t* poff = tmp.get<uint32_t>(L0);
    uint32_t* psums = tmp.get<uint32_t>(scan_sums_len(L0));
    {
    ISAX_LAUNCH("lf_pieces", st);
    lf_pieces_kernel<<<grid_for(L0, 256, num_sms), 256, 0, st>>>(starts, L0, Lc, pieces);
    }
    exclusive_scan(pieces, poff, L0, psums, st);
    uint32_t L = 0;
    ISAX_CUDA_TRY(cudaMemcpyAsync(&L, psums + (scan_sums_len(L0) - 1), sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    ix->leaf_begin = static_cast<uint32_t*>(dev_alloc(((size_t)L + 1) * sizeof(uint32_t), st));
    {
    ISAX_LAUNCH("lf_expand", st);
    lf_expand_kernel<<<grid_for(L0, 256, num_sms), 256, 0, st>>>(starts, poff, L0, Lc, N,
                                                                  ix->leaf_begin, L);
    }
    ISAX_CUDA_TRY(cudaGetLastError());
    for (void* p : {(void*)c, (void*)a, (void*)P, (void*)S, (void*)tcount, (void*)toff,
                    (void*)sums, (void*)starts, (void*)pieces, (void*)poff, (void*)psums})
        tmp.release(p);
    return L;
}

// Leaves of ADS+ node splitting: sorts (kA, vA) by root key, then splits level
// by level; vA ends holding the rows in leaf order.  Fills ix->leaf_begin,
// ix->tree, ix->tree_root, ix->tree_nodes and returns the number of leaves.
uint32_t balanced_leaves(isax_index* ix, TempPool& tmp, const uint4* sax_tmp, unsigned long long*& kA,
                         unsigned long long*& kB, uint32_t*& vA, uint32_t*& vB, int64_t N, int cbits,
                         int leaf_size, int num_sms, cudaStream_t st, unsigned* sort_err) {
    radix_sort(kA, vA, kB, vB, N, 48, 2, tmp, st, sort_err, num_sms);  // the root key: top 16 bits

    const unsigned g_n = grid_for(N, 256, num_sms);
    uint32_t* zf = tmp.get<uint32_t>(N);
    uint32_t* Z = tmp.get<uint32_t>(N);
    uint32_t* zsums = tmp.get<uint32_t>(scan_sums_len(N));
    const uint32_t* ztot = zsums + (scan_sums_len(N) - 1);
    {
    ISAX_LAUNCH("bl_root", st);
    bl_root_flags_kernel<<<g_n, 256, 0, st>>>(kA, N, zf);
    }
    exclusive_scan(zf, Z, N, zsums, st);
    const int64_t n0 = read_u32(ztot, st);

    uint4* sax_a = tmp.get<uint4>(N);
    uint4* sax_b = tmp.get<uint4>(N);
    uint32_t* en_a = tmp.get<uint32_t>(N);
    uint32_t* en_b = tmp.get<uint32_t>(N);
    uint32_t* nstart = tmp.get<uint32_t>(n0);
    uint32_t* ncnt = tmp.get<uint32_t>(n0);
    unsigned long long* nbits = tmp.get<unsigned long long>(n0);
    uint32_t* ngid = tmp.get<uint32_t>(n0);
    ix->tree_root = static_cast<int32_t*>(dev_alloc(((size_t)1 << 16) * sizeof(int32_t), st));
    ISAX_CUDA_TRY(cudaMemsetAsync(ix->tree_root, 0xFF, ((size_t)1 << 16) * sizeof(int32_t), st));
    int64_t tcap = n0 + 2 * (N / ((int64_t)leaf_size + 1) + 1) + 1024;
    ix->tree = static_cast<int2*>(dev_alloc((size_t)tcap * sizeof(int2), st));
    {
    ISAX_LAUNCH("bl_root", st);
    permute_sax_kernel<<<num_sms * 8, 256, 0, st>>>(vA, N, sax_tmp, sax_a, vB);
    bl_root_nodes_kernel<<<g_n, 256, 0, st>>>(kA, zf, Z, N, en_a, nstart, ix->tree_root);
    bl_root_fill_kernel<<<grid_for(n0, 256, num_sms), 256, 0, st>>>(nstart, n0, N, ncnt, nbits, ngid);
    }
    ISAX_CUDA_TRY(cudaGetLastError());

    int64_t nodes = n0;
    int64_t next_gid = n0;
    // a path adds one bit to one segment per level: at most 16 (cbits - 1) levels split
    for (int level = 0;; ++level) {
        if (level > 16 * cbits) throw Error{ISAX_ERR_CUDA, "balanced split: too many tree levels"};
        int32_t* seg = tmp.get<int32_t>(nodes);
        uint32_t* split = tmp.get<uint32_t>(nodes);
        uint32_t* spos = tmp.get<uint32_t>(nodes);
        uint32_t* ssums = tmp.get<uint32_t>(scan_sums_len(nodes));
        {
        ISAX_LAUNCH("bl_decide", st);
        bl_decide_kernel<<<grid_for(nodes, 8, num_sms), 256, 0, st>>>(sax_a, nstart, ncnt, nbits, nodes,
                                                                    (uint32_t)leaf_size, cbits, seg, split);
        }
        exclusive_scan(split, spos, nodes, ssums, st);
        const int64_t S = read_u32(ssums + (scan_sums_len(nodes) - 1), st);
        if (S == 0) {
            for (void* p : {(void*)seg, (void*)split, (void*)spos, (void*)ssums}) tmp.release(p);
            break;
        }
        if (next_gid + 2 * S > tcap) {
            const int64_t nc = std::max(next_gid + 2 * S, 2 * tcap);
            int2* t = static_cast<int2*>(dev_alloc((size_t)nc * sizeof(int2), st));
            ISAX_CUDA_TRY(cudaMemcpyAsync(t, ix->tree, (size_t)next_gid * sizeof(int2), cudaMemcpyDeviceToDevice, st));
            dev_free(ix->tree, st);
            ix->tree = t;
            tcap = nc;
        }
        {
        ISAX_LAUNCH("bl_split", st);
        bl_bit_kernel<<<g_n, 256, 0, st>>>(sax_a, en_a, seg, nbits, N, cbits, zf);
        }
        exclusive_scan(zf, Z, N, zsums, st);
        const int64_t nodes2 = nodes + S;
        uint32_t* nstart2 = tmp.get<uint32_t>(nodes2);
        uint32_t* ncnt2 = tmp.get<uint32_t>(nodes2);
        unsigned long long* nbits2 = tmp.get<unsigned long long>(nodes2);
        uint32_t* ngid2 = tmp.get<uint32_t>(nodes2);
        {
        ISAX_LAUNCH("bl_split", st);
        bl_nodes_kernel<<<grid_for(nodes, 256, num_sms), 256, 0, st>>>(
            nodes, nstart, ncnt, nbits, ngid, seg, spos, Z, ztot, N, (uint32_t)next_gid, nstart2, ncnt2,
            nbits2, ngid2, ix->tree);
        bl_scatter_kernel<<<g_n, 256, 0, st>>>(N, sax_a, vA, en_a, seg, nstart, ncnt, spos, zf, Z, ztot,
                                               sax_b, vB, en_b);
        }
        ISAX_CUDA_TRY(cudaGetLastError());
        std::swap(sax_a, sax_b);
        std::swap(vA, vB);
        std::swap(en_a, en_b);
        for (void* p : {(void*)seg, (void*)split, (void*)spos, (void*)ssums, (void*)nstart, (void*)ncnt,
                        (void*)nbits, (void*)ngid})
            tmp.release(p);
        nstart = nstart2;
        ncnt = ncnt2;
        nbits = nbits2;
        ngid = ngid2;
        nodes = nodes2;
        next_gid += 2 * S;
    }

    // (the tree may hold more nodes than series: empty leaves)
    uint32_t* nonempty = tmp.get<uint32_t>(nodes);
    uint32_t* li = tmp.get<uint32_t>(nodes);
    uint32_t* lsums = tmp.get<uint32_t>(scan_sums_len(nodes));
    {
    ISAX_LAUNCH("bl_leaves", st);
    bl_leaf_flags_kernel<<<grid_for(nodes, 256, num_sms), 256, 0, st>>>(ncnt, nodes, nonempty);
    }
    exclusive_scan(nonempty, li, nodes, lsums, st);
    const uint32_t L = read_u32(lsums + (scan_sums_len(nodes) - 1), st);
    ix->leaf_begin = static_cast<uint32_t*>(dev_alloc(((size_t)L + 1) * sizeof(uint32_t), st));
    {
    ISAX_LAUNCH("bl_leaves", st);
    bl_leaves_kernel<<<grid_for(nodes, 256, num_sms), 256, 0, st>>>(nodes, nstart, ncnt, ngid, li, L, N,
                                                                     ix->leaf_begin, ix->tree);
    }
    ISAX_CUDA_TRY(cudaGetLastError());
    ix->tree_nodes = next_gid;
    for (void* p : {(void*)zf, (void*)Z, (void*)zsums, (void*)sax_a, (void*)sax_b, (void*)en_a, (void*)en_b,
                    (void*)nstart, (void*)ncnt, (void*)nbits, (void*)ngid, (void*)nonempty, (void*)li,
                    (void*)lsums})
        tmp.release(p);
    return L;
}

}  // namespace

void free_index_arrays(isax_index* ix, cudaStream_t st);


isax_index* build_index_impl(const float* series, int64_t N, int n, int card, int leaf_size,
                             uint32_t mem_flags, cudaStream_t st) {
    int dev = 0;
    ISAX_CUDA_TRY(cudaGetDevice(&dev));
    int num_sms = 0;
    ISAX_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));

    isax_index* ix = new isax_index();
    ix->device = dev;
    ix->num_sms = num_sms;
    ix->mu = new std::mutex();
    // a host buffer this build page-locked, unlocked again when the build ends
    struct HostReg {
        void* p = nullptr;
        cudaStream_t st = nullptr;
        ~HostReg() {
            if (p) {
                cudaStreamSynchronize(st);
                cudaHostUnregister(p);
            }
        }
    } host_reg;
    host_reg.st = st;
    try {
        int cbits = 0;
        while ((1 << cbits) < card) ++cbits;
        const int keybits = 16 * std::min(cbits, 4);
        TempPool tmp{st, {}};

        const float* xin = series;
        const bool rows_host = (mem_flags & ISAX_BUILD_ROWS_HOST) != 0;
        const bool in_place = (mem_flags & ISAX_BUILD_ROWS_IN_PLACE) != 0;
        // host input copied to the device in chunks, each summarised as soon as it has
        // landed; that copy, in the input's order, is the index's row store (read by row)
        const bool chunked_host = !(mem_flags & ISAX_MEM_INPUT_DEVICE) && !rows_host;
        if (chunked_host) {
            ix->x = static_cast<float*>(dev_alloc((size_t)N * n * sizeof(float), st));
            ix->rows_in_place = true;
            xin = ix->x;
        } else if (!(mem_flags & ISAX_MEM_INPUT_DEVICE)) {
            if (rows_host) {
                // read in place over the CPU-GPU link: page-lock it for the build if the
                // caller has not (nothing of the collection is staged in device memory)
                cudaPointerAttributes at{};
                cudaError_t e = cudaPointerGetAttributes(&at, series);
                if (e != cudaSuccess) cudaGetLastError();
                if (e != cudaSuccess || at.type == cudaMemoryTypeUnregistered) {
                    ISAX_CUDA_TRY(cudaHostRegister(const_cast<float*>(series), (size_t)N * n * sizeof(float),
                                                   cudaHostRegisterDefault));
                    host_reg.p = const_cast<float*>(series);
                }
                void* dp = nullptr;
                ISAX_CUDA_TRY(cudaHostGetDevicePointer(&dp, const_cast<float*>(series), 0));
                xin = static_cast<const float*>(dp);
            }
        }

        // breakpoints + summaries
        ix->bp = static_cast<float*>(dev_alloc((card + 1) * sizeof(float), st));
        launch_breakpoints(card, ix->bp, st);
        uint4* sax_tmp = tmp.get<uint4>(N);
        unsigned long long* kA = tmp.get<unsigned long long>(N);
        unsigned long long* kB = tmp.get<unsigned long long>(N);
        uint32_t* vA = tmp.get<uint32_t>(N);
        uint32_t* vB = tmp.get<uint32_t>(N);
        // maxabs bits, nonfinite, max_leaf, permutation wait gave up, sort wait gave up
        unsigned* misc = tmp.get<unsigned>(5);
        ISAX_CUDA_TRY(cudaMemsetAsync(misc, 0, 5 * sizeof(unsigned), st));
        if (chunked_host) {
            ChunkCopier cp(st);
            float* xd = ix->x;
            const int64_t R = std::max<int64_t>(1, ((int64_t)1 << 30) / ((int64_t)n * 4));  // ~1 GB chunks
            for (int64_t r0 = 0; r0 < N; r0 += R) {
                const int64_t rows = std::min<int64_t>(R, N - r0);
                cp.copy(xd + r0 * n, series + r0 * n, (size_t)rows * n * sizeof(float));
                launch_summarize(xd + r0 * n, rows, n, card, ix->bp, sax_tmp + r0, kA + r0, vA + r0, nullptr,
                                 misc, misc + 1, num_sms, st, (uint32_t)r0);
            }
        } else {
            launch_summarize(xin, N, n, card, ix->bp, sax_tmp, kA, vA, nullptr, misc, misc + 1, num_sms,
                             st);
        }

        // leaves: the round-robin split of the sorted keys, or ADS+ node splitting
        // (the index's SAX words and row ids: when the rows stay in input order,
        // the sort's last pass puts them in leaf order itself)
        const bool balanced = (mem_flags & ISAX_BUILD_SPLIT_BALANCED) != 0;
        ix->sax = static_cast<uint4*>(dev_alloc((size_t)N * sizeof(uint4), st));
        ix->orig = static_cast<uint32_t*>(dev_alloc((size_t)N * sizeof(uint32_t), st));
        uint32_t L = 0;
        bool sax_placed = false;
        if (balanced) {
            L = balanced_leaves(ix, tmp, sax_tmp, kA, kB, vA, vB, N, cbits, leaf_size, num_sms, st, misc + 4);
        } else {
            const bool gather = in_place || chunked_host;
            sax_placed = radix_sort(kA, vA, kB, vB, N, 64 - keybits, keybits / 8, tmp, st, misc + 4, num_sms,
                                    gather ? sax_tmp : nullptr, gather ? ix->sax : nullptr,
                                    gather ? ix->orig : nullptr);
            L = round_robin_leaves(ix, tmp, kA, N, leaf_size, keybits, num_sms, st);
        }

        // permute rows and SAX words into leaf order
        if (in_place || chunked_host) {
            // the rows stay in the input's order (the caller's array, or the device copy
            // of a host input), read by original id
            if (in_place) {
                ix->x = const_cast<float*>(series);
                ix->rows_in_place = true;
                ix->rows_borrowed = true;
            }
            if (!sax_placed) {
                ISAX_LAUNCH("permute_sax", st);
                permute_sax_kernel<<<num_sms * 8, 256, 0, st>>>(vA, N, sax_tmp, ix->sax, ix->orig);
            }
        } else if (rows_host) {
            // leaf-ordered rows in pinned host memory (unified addressing: the host
            // pointer is valid on the device)
            float* xh = nullptr;
            ISAX_CUDA_TRY(cudaMallocHost((void**)&xh, (size_t)N * n * sizeof(float)));
            ix->x = xh;
            ix->rows_host = true;
            ISAX_LAUNCH("permute_plain", st);
            permute_plain_kernel<<<num_sms * 8, 256, 0, st>>>(xin, n, vA, N, ix->x, sax_tmp, ix->sax,
                                                              ix->orig);
        } else {
            ix->x = static_cast<float*>(dev_alloc((size_t)N * n * sizeof(float), st));
            const size_t pm_smem = (size_t)PM_STAGES * PM_STAGE_BYTES;
            ISAX_CUDA_TRY(cudaFuncSetAttribute(permute_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)pm_smem));
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, permute_kernel, PM_THREADS, pm_smem) !=
                    cudaSuccess || per_sm < 1)
                per_sm = 1;
            ISAX_LAUNCH("permute", st);
            permute_kernel<<<num_sms * per_sm, PM_THREADS, pm_smem, st>>>(xin, n, vA, N, ix->x, sax_tmp,
                                                                         ix->sax, ix->orig, misc + 3);
        }
        ISAX_CUDA_TRY(cudaGetLastError());

        // envelopes
        ix->env = static_cast<uint4*>(dev_alloc((size_t)L * 2 * sizeof(uint4), st));
        ix->leaf_key = static_cast<unsigned long long*>(
            dev_alloc((size_t)L * sizeof(unsigned long long), st));
        {
        ISAX_LAUNCH("envelope", st);
        envelope_kernel<<<grid_for(L, 8, num_sms, 8), 256, 0, st>>>(
            ix->sax, ix->leaf_begin, L, kA, ix->env, ix->leaf_key,
            balanced ? 0xFFFF000000000000ull : ~0ull, misc + 2);
        ISAX_CUDA_TRY(cudaGetLastError());
        }

        unsigned hm[5];
        ISAX_CUDA_TRY(cudaMemcpyAsync(hm, misc, sizeof hm, cudaMemcpyDeviceToHost, st));
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
        if (hm[1]) throw Error{ISAX_ERR_INVALID_ARG, "series contains a non-finite value"};
        if (hm[3]) throw Error{ISAX_ERR_TIMEOUT, "a bulk-copy wait of the permutation gave up"};
        if (hm[4]) throw Error{ISAX_ERR_TIMEOUT, "a look-back wait of the radix sort gave up"};
        float maxabs;
        memcpy(&maxabs, &hm[0], sizeof maxabs);

        DevIndex& d = ix->d;
        d.N = N;
        d.n = n;
        d.card = card;
        d.cbits = cbits;
        d.keybits = keybits;
        d.leaf_size = leaf_size;
        d.L = L;
        d.x = ix->x;
        d.sax = ix->sax;
        d.orig = ix->orig;
        d.leaf_begin = ix->leaf_begin;
        d.env = ix->env;
        d.leaf_key = ix->leaf_key;
        d.bp = ix->bp;
        d.maxabs = maxabs;
        d.rows_in_place = ix->rows_in_place ? 1 : 0;
        d.tree = ix->tree;
        d.tree_root = ix->tree_root;
        ix->max_leaf = (int32_t)hm[2];
        ix->bytes = (int64_t)N * n * 4 + N * 16 + N * 4 + ((int64_t)L + 1) * 4 + (int64_t)L * 40 +
                    (card + 1) * 4;
        if (rows_host || in_place) ix->bytes -= (int64_t)N * n * 4;
        if (balanced) ix->bytes += ix->tree_nodes * 8 + ((int64_t)1 << 16) * 4;
        alloc_query_scratch(ix, (uint32_t)std::min<int64_t>(N, 1 << 20), default_surv_cap(N), st);
    } catch (...) {
        free_index_arrays(ix, st);
        delete static_cast<std::mutex*>(ix->mu);
        delete ix;
        throw;
    }
    return ix;
}

// ---------------------------------------------------------------- summarize alone
void summarize_impl(const float* series, int64_t N, int n, int card, uint32_t mem_flags,
                    uint8_t* out_sax, float* out_paa, cudaStream_t st) {
    int dev = 0, num_sms = 0;
    ISAX_CUDA_TRY(cudaGetDevice(&dev));
    ISAX_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    TempPool tmp{st, {}};
    const float* xin = series;
    if (!(mem_flags & ISAX_MEM_INPUT_DEVICE)) {
        float* xd = tmp.get<float>((size_t)N * n);
        ISAX_CUDA_TRY(cudaMemcpyAsync(xd, series, (size_t)N * n * sizeof(float),
                                      cudaMemcpyHostToDevice, st));
        xin = xd;
    }
    const bool out_dev = mem_flags & ISAX_MEM_OUTPUT_DEVICE;
    float* bp = tmp.get<float>(card + 1);
    launch_breakpoints(card, bp, st);
    uint4* sax = (out_dev && out_sax) ? reinterpret_cast<uint4*>(out_sax) : tmp.get<uint4>(N);
    float* paa = nullptr;
    if (out_paa) paa = out_dev ? out_paa : tmp.get<float>((size_t)N * W);
    unsigned* misc = tmp.get<unsigned>(2);
    ISAX_CUDA_TRY(cudaMemsetAsync(misc, 0, 2 * sizeof(unsigned), st));
    launch_summarize(xin, N, n, card, bp, sax, nullptr, nullptr, paa, misc, misc + 1, num_sms, st);
    if (!out_dev) {
        if (out_sax)
            ISAX_CUDA_TRY(cudaMemcpyAsync(out_sax, sax, (size_t)N * W, cudaMemcpyDeviceToHost, st));
        if (out_paa)
            ISAX_CUDA_TRY(cudaMemcpyAsync(out_paa, paa, (size_t)N * W * sizeof(float),
                                          cudaMemcpyDeviceToHost, st));
    }
    unsigned hm[2];
    ISAX_CUDA_TRY(cudaMemcpyAsync(hm, misc, sizeof hm, cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    if (hm[1]) throw Error{ISAX_ERR_INVALID_ARG, "series contains a non-finite value"};
}

uint32_t take_check_word_build() { return take_check_word_here(); }

}  // namespace isax
