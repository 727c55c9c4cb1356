// isax_tc.cu - tensor-core (tcgen05) contraction machinery for the batched,
// BF16-filtered exact k-NN path.  BF16 operands staged in shared memory in the
// 128-byte-swizzled K-major layout (the A side by TMA tensor copies), one
// elected thread issues tcgen05.mma (kind::f16, FP32 accumulate) into TMEM,
// completion is committed to an mbarrier, and the epilogue warps read the
// accumulator rows back with tcgen05.ld.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "isax_common.cuh"
#include "isax_kernels_util.cuh"
#include "isax_tc.cuh"

namespace isax {

// ---------------------------------------------------------------- host: tensor maps
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mu;

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    std::lock_guard<std::mutex> lk(g_encode_mu);
    if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            throw Error{ISAX_ERR_CUDA, "cuTensorMapEncodeTiled is not available"};
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    return g_encode;
}

// rows x cols BF16 matrix (row-major), boxes of 64 elements x box_rows rows,
// 128-byte swizzle, rows past the end read as zeros
static void make_tmap_bf16_box(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols,
                               uint32_t box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_KATOM, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        throw Error{ISAX_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
}
static void make_tmap_bf16_rows(CUtensorMap* tm, const void* base, uint64_t rows, uint32_t box_rows) {
    make_tmap_bf16_box(tm, base, rows, TC_K, box_rows);
}
static void make_tmap_bf16(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols) {
    make_tmap_bf16_box(tm, base, rows, cols, TC_M);
}

// ---------------------------------------------------------------- device: tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem desc] . B[smem desc]^T, BF16 in, FP32 accumulate
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// arrive on `bar` once every tcgen05 operation issued so far by this thread completes
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// this warp's 32 TMEM lanes x 32 consecutive FP32 columns starting at taddr
__device__ __forceinline__ void tc_ld_x32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// this warp's 32 TMEM lanes x 16 consecutive FP32 columns starting at taddr
__device__ __forceinline__ void tc_ld_x16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* tm, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(smem_dst)),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset (unused when swizzled, K-major)
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

// byte offset of the 16-byte chunk `ch` (8 BF16, k = 8 ch .. 8 ch + 7) of row j in a
// tile of `rows` rows stored as 4 K-atoms of 64 elements, 128-byte swizzled
__device__ __forceinline__ uint32_t sw128_offset(int j, int ch, int rows) {
    const int ka = ch >> 3, c = ch & 7;
    return (uint32_t)(ka * (rows / 8) * 1024 + (j >> 3) * 1024 + (j & 7) * 128 + ((c ^ (j & 7)) << 4));
}

// ---------------------------------------------------------------- self test
// D[128][N] = A[128][256] . B[N][256]^T: A by TMA, B stored by the threads,
// 16 MMAs of K = 16, accumulator read back by the 4 warps.
__global__ void __launch_bounds__(128) tc_selftest_kernel(const __grid_constant__ CUtensorMap tmA,
                                                          const uint4* __restrict__ B, int N,
                                                          float* __restrict__ D, unsigned* err) {
    extern __shared__ unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // swizzled tiles start on a 1024-byte boundary (dynamic size has 1 KB of slack)
    unsigned char* sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    unsigned char* As = sm;
    unsigned char* Bs = sm + TC_M * TC_K * 2;
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;
    if (warp == 0) tmem_alloc(&tmem_base, ncols);
    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        mbar_fence_init();
    }
    for (int c = tid; c < N * (TC_K / 8); c += blockDim.x) {
        const int j = c / (TC_K / 8), ch = c % (TC_K / 8);
        *reinterpret_cast<uint4*>(Bs + sw128_offset(j, ch, N)) = B[(size_t)j * (TC_K / 8) + ch];
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar_load, TC_M * TC_K * 2);
        for (int ka = 0; ka < TC_K / TC_KATOM; ++ka)
            tma_load_2d(As + ka * TC_M * TC_KATOM * 2, &tmA, ka * TC_KATOM, 0, &bar_load);
        if (!mbar_wait_bounded(&bar_load, 0, 1u << 24)) {
            atomicOr(err, 1u);
        } else {
            tc_fence_after();
            const uint32_t idesc = tc_idesc_bf16(TC_M, N);
            for (int s = 0; s < TC_K / 16; ++s) {
                const int ka = s >> 2, kk = s & 3;
                const uint64_t ad = sdesc_sw128(smem_u32(As) + ka * TC_M * TC_KATOM * 2 + kk * 32);
                const uint64_t bd = sdesc_sw128(smem_u32(Bs) + ka * N * TC_KATOM * 2 + kk * 32);
                tc_mma_f16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
            }
            tc_commit(&bar_mma);
        }
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bar_mma, 0, 1u << 24);
    tc_fence_after();
    if (ok) {
        for (int c0 = 0; c0 < N; c0 += 32) {
            float v[32];
            tc_ld_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            const int row = warp * 32 + lane;
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (c0 + i < N) D[(size_t)row * N + c0 + i] = v[i];
        }
    } else if (lane == 0) {
        atomicOr(err, 2u);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
}

void tc_selftest(const void* A, const void* B, int N, float* D, cudaStream_t st) {
    CUtensorMap tm;
    make_tmap_bf16_rows(&tm, A, TC_M, TC_M);
    unsigned* err = static_cast<unsigned*>(dev_alloc(sizeof(unsigned), st));
    ISAX_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
    const size_t smem = 1024 + (size_t)TC_M * TC_K * 2 + (size_t)N * TC_K * 2;
    ISAX_CUDA_TRY(cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    {
        ISAX_LAUNCH("tc_selftest", st);
        tc_selftest_kernel<<<1, 128, smem, st>>>(tm, static_cast<const uint4*>(B), N, D, err);
        ISAX_CUDA_TRY(cudaGetLastError());
    }
    unsigned h = 0;
    ISAX_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    dev_free(err, st);
    if (h) throw Error{ISAX_ERR_TIMEOUT, "tensor-core self test: a wait gave up (" + std::to_string(h) + ")"};
}

// ================================================================ BF16 filter
// Batched exact k-NN with the refinement's distance computation moved to the
// tensor cores as a filter:
//   d~2(x, q) = ||x||^2 + ||q||^2 - 2 bf16(x) . bf16(q)   (FP32 accumulate)
// is within E(x, q) of the exact squared distance (bound below), so a row can
// be among a query's k best only if d~2 - E <= (an upper bound of the k-th
// best squared distance).  Those rows are re-checked with the exact fp32
// distance of the single-query path and the k best are ordered as there
// (FP64 only within fp32 error of each other): the answers are the exact ones.
//
// Work is leaf-major: every leaf that the envelope bound leaves to a set of
// queries is contracted once against all of them (up to TF_NQ per work item),
// so the leaf's rows are read once per batch instead of once per query.
//
// Error bound.  With u = 2^-24, u_b = 2^-8 (BF16 unit roundoff), X >= ||x||,
// Q >= ||q||: rounding x and q to BF16 moves x.q by at most (2 u_b + u_b^2) X Q;
// the tensor-core FP32 sum of the exact BF16 products is taken to err by at
// most n 2^-21 sum|x_i q_i| (four times the truncating-summation bound, which
// leaves room for the hardware's internal alignment); the squared norms
// (FP64 sums rounded to fp32), their fp32 sum and the final fma add at most
// 4 u (X^2 + Q^2) + 2.01 u (1 + u_b)^2 X Q.  Hence
//   E = [2 (2 u_b + u_b^2) + 2 n 2^-21 (1 + u_b)^2 + 2.01 u (1 + u_b)^2] X Q
//       + 4 u (X^2 + Q^2),
// evaluated in FP64 with X the largest row norm of the leaf and Q the query
// norm, both rounded up (about 4.07 for z-normalised series of length 256).

constexpr int TF_NQ = 256;           // queries per work item (MMA N, at most)
constexpr int TF_STAGES = 5;         // A ring: one 128-row x 64-element K-atom each
constexpr int TF_EPI_WARPS = 8;      // epilogue warps (two per TMEM lane quarter)
constexpr int TF_GATHER_WARPS = 4;   // warps that fill the B tile
constexpr int TF_THREADS = (TF_EPI_WARPS + TF_GATHER_WARPS + 2) * 32;  // + TMA warp + MMA warp
constexpr int TF_SLOTS = 4;          // work-item descriptors in flight
constexpr uint32_t TF_ATOM_BYTES = TC_M * TC_KATOM * 2;
constexpr uint32_t TF_B_BYTES = 131072;  // the B tile: up to TF_NQ queries x n BF16 (<= 128 KB)
constexpr uint32_t TF_TMEM_COLS = 2 * TF_NQ;  // two accumulators
constexpr uint32_t TF_WAIT = 1u << 22;  // bounded mbarrier waits
constexpr int TF_QCAP = 4096;        // per-query candidate window entries
constexpr int TF_MAX_B = 4096;       // queries per pass
constexpr int TC_APPROX_NEIGHBORS = 2;  // approximate answer: descent leaf +- 2 leaves

static size_t smem_tf() { return 1024 + (size_t)TF_B_BYTES + (size_t)TF_STAGES * TF_ATOM_BYTES; }

// queries per work item for series length n: the B tile (nq x n BF16) fits 128 KB
static int tf_nq_max(int n) {
    int q = (int)TF_B_BYTES / (2 * n);
    q = q > TF_NQ ? TF_NQ : q;
    return q & ~15;
}

struct TcView {
    const uint32_t* leaf_begin;
    const float* xn;           // [N] squared row norms (fp32), leaf order
    const float* leaf_xnorm;   // [L] largest row norm of the leaf, rounded up
    const uint4* items;        // work items {leaf, first pair, queries, 0}
    const uint32_t* n_items;
    uint32_t* claim;
    const uint32_t* pairs;     // query of each pair, grouped by leaf
    const uint16_t* qb;        // [B][n] BF16 queries
    const float4* qc;          // [B] {squared norm (fp32), norm rounded up, upper bound of the
                               //      k-th best squared distance after the approximate answer, 0}
    unsigned long long* utop;  // [B][MAX_K] k smallest upper bounds d~2 + E (packed with the position)
    uint4* cand;               // kept rows {position, query, d~2 bits, E bits}
    uint32_t* cand_count;
    uint32_t cand_cap;
    uint32_t* err;
    int n, k;
    double c_xq, c_sq;
};

__device__ __forceinline__ void tf_fail(volatile int* abort_flag, uint32_t* err, uint32_t code) {
    *abort_flag = 1;
    atomicOr(err, code);
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// warp-uniform bounded wait
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity) {
    return __all_sync(FULL, mbar_wait_bounded(bar, parity, TF_WAIT));
}

// Roles (TF_THREADS = 448):
//   warps 0-7   epilogue: read the accumulators back and keep the rows that pass;
//   warps 8-11  gather: the item's queries into the B tile (cp.async, 128-byte
//               swizzled K-major) as soon as the previous item's MMAs retire,
//               and its per-column limits into one of two limit buffers;
//   warp 12     claims work items (TF_SLOTS descriptor slots ahead) and streams
//               the leaf's rows through the A ring with TMA, across items;
//   warp 13     issues the MMAs (one thread), accumulators alternating between
//               two TMEM buffers, and releases the B tile when its MMAs complete.
// Every hand-off is an mbarrier with a bounded wait; a wait that gives up sets
// the error word and every role leaves its loop (no CTA-wide barrier inside).
__global__ void __launch_bounds__(TF_THREADS, 1)
    tc_filter_kernel(const __grid_constant__ CUtensorMap tmX, TcView v) {
    extern __shared__ unsigned char sm_raw[];
    __shared__ __align__(8) uint64_t full[TF_STAGES], empty[TF_STAGES], accf[2], acce[2];
    __shared__ __align__(8) uint64_t itemf[TF_SLOTS], iteme[TF_SLOTS], bfull, bempty, cfull[2], cempty[2], fin;
    __shared__ uint4 item_s[TF_SLOTS];     // {leaf, first pair, queries, first row}
    __shared__ uint32_t item_le[TF_SLOTS];  // one past the leaf's last row
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_s;
    __shared__ float lim_s[2][TF_NQ], eu_s[2][TF_NQ], qn_s[2][TF_NQ];
    __shared__ unsigned int ku_s[2][TF_NQ];
    __shared__ uint32_t qid_s[2][TF_NQ];
    unsigned char* sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    const int n = v.n, k = v.k;
    const int katoms = n / TC_KATOM;
    unsigned char* Bs = sm;
    unsigned char* As = sm + TF_B_BYTES;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) tmem_alloc(&tmem_base, TF_TMEM_COLS);
    if (threadIdx.x == 0) {
        for (int i = 0; i < TF_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&acce[i], TF_EPI_WARPS);
            mbar_init(&cfull[i], TF_GATHER_WARPS);
            mbar_init(&cempty[i], TF_EPI_WARPS);
        }
        mbar_init(&bfull, TF_GATHER_WARPS);
        mbar_init(&bempty, 1);
        for (int i = 0; i < TF_SLOTS; ++i) {
            mbar_init(&itemf[i], 1);
            mbar_init(&iteme[i], TF_EPI_WARPS + TF_GATHER_WARPS + 1);
        }
        mbar_init(&fin, 1);
        abort_s = 0;
        mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr int W_GATHER = TF_EPI_WARPS, W_PROD = TF_EPI_WARPS + TF_GATHER_WARPS, W_MMA = W_PROD + 1;

    if (warp == W_PROD) {
        // ------------------------------------------------ scheduler + TMA producer
        if (lane == 0) {
            uint32_t p_it = 0;
            for (uint32_t i = 0;; ++i) {
                const uint32_t slot = i % TF_SLOTS, ph = (i / TF_SLOTS) & 1u;
                if (!mbar_wait_bounded(&iteme[slot], ph ^ 1u, TF_WAIT)) {
                    tf_fail(&abort_s, v.err, 1u);
                    break;
                }
                const uint32_t idx = atomicAdd(v.claim, 1u);
                uint4 it = idx < *v.n_items ? v.items[idx] : make_uint4(0u, 0u, 0u, 0u);
                uint32_t it_le = 0;
                if (it.z != 0) {
                    it.w = v.leaf_begin[it.x];
                    it_le = v.leaf_begin[it.x + 1];
                }
                item_s[slot] = it;
                item_le[slot] = it_le;
                mbar_arrive(&itemf[slot]);
                if (it.z == 0 || abort_s) break;
                const int64_t lb = it.w, le = it_le;
                const int tiles = (int)((le - lb + TC_M - 1) / TC_M);
                bool ok = true;
                for (int t = 0; t < tiles && ok; ++t) {
                    for (int ka = 0; ka < katoms; ++ka, ++p_it) {
                        const uint32_t st = p_it % TF_STAGES, sph = (p_it / TF_STAGES) & 1u;
                        if (abort_s || !mbar_wait_bounded(&empty[st], sph ^ 1u, TF_WAIT)) {
                            tf_fail(&abort_s, v.err, 2u);
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(&full[st], TF_ATOM_BYTES);
                        tma_load_2d(As + st * TF_ATOM_BYTES, &tmX, ka * TC_KATOM,
                                    (int)(lb + (int64_t)t * TC_M), &full[st]);
                    }
                }
                if (!ok) break;
            }
            // copies still in flight (after an abort) land before the CTA exits
            for (uint32_t i = p_it > TF_STAGES ? p_it - TF_STAGES : 0; i < p_it; ++i)
                mbar_wait_bounded(&full[i % TF_STAGES], (i / TF_STAGES) & 1u, TF_WAIT);
        }
    } else if (warp == W_MMA) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t m_it = 0, m_t = 0;
            for (uint32_t i = 0;; ++i) {
                const uint32_t slot = i % TF_SLOTS, ph = (i / TF_SLOTS) & 1u;
                if (!mbar_wait_bounded(&itemf[slot], ph, TF_WAIT)) {
                    tf_fail(&abort_s, v.err, 4u);
                    break;
                }
                const uint4 it = item_s[slot];
                const uint32_t it_le = item_le[slot];
                mbar_arrive(&iteme[slot]);
                if (it.z == 0 || abort_s) break;
                const int n16 = (int)((it.z + 15u) & ~15u);
                const int64_t lb = it.w, le = it_le;
                const int tiles = (int)((le - lb + TC_M - 1) / TC_M);
                if (!mbar_wait_bounded(&bfull, i & 1u, TF_WAIT)) {
                    tf_fail(&abort_s, v.err, 8u);
                    break;
                }
                tc_fence_after();
                const uint32_t idesc = tc_idesc_bf16(TC_M, n16);
                const uint32_t bs = smem_u32(Bs);
                bool ok = true;
                for (int t = 0; t < tiles && ok; ++t, ++m_t) {
                    const uint32_t a = m_t & 1u, aph = (m_t >> 1) & 1u;
                    if (!mbar_wait_bounded(&acce[a], aph ^ 1u, TF_WAIT)) {
                        tf_fail(&abort_s, v.err, 16u);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dcol = tmem + a * (uint32_t)TF_NQ;
                    for (int ka = 0; ka < katoms; ++ka, ++m_it) {
                        const uint32_t st = m_it % TF_STAGES, sph = (m_it / TF_STAGES) & 1u;
                        if (!mbar_wait_bounded(&full[st], sph, TF_WAIT)) {
                            tf_fail(&abort_s, v.err, 32u);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t abase = smem_u32(As + st * TF_ATOM_BYTES);
                        const uint32_t bbase = bs + (uint32_t)(ka * n16 * 128);
#pragma unroll
                        for (int kk = 0; kk < TC_KATOM / 16; ++kk)
                            tc_mma_f16(dcol, sdesc_sw128(abase + kk * 32), sdesc_sw128(bbase + kk * 32), idesc,
                                       (ka | kk) ? 1u : 0u);
                        tc_commit(&empty[st]);
                    }
                    if (ok) tc_commit(&accf[a]);
                }
                if (!ok) break;
                tc_commit(&bempty);  // the B tile is free once these MMAs complete
            }
            // every MMA issued has completed before TMEM is released
            tc_commit(&fin);
            mbar_wait_bounded(&fin, 0, TF_WAIT);
        }
    } else if (warp >= W_GATHER) {
        // ------------------------------------------------ gather warps
        const int gt = threadIdx.x - W_GATHER * 32;  // 0 .. 127
        const int cpr = n / 8;                        // 16-byte chunks per query row
        for (uint32_t i = 0;; ++i) {
            const uint32_t slot = i % TF_SLOTS, ph = (i / TF_SLOTS) & 1u;
            if (!warp_wait(&itemf[slot], ph)) {
                if (lane == 0) tf_fail(&abort_s, v.err, 64u);
                break;
            }
            const uint4 it = item_s[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&iteme[slot]);
            if (__any_sync(FULL, it.z == 0 || abort_s)) break;  // warp-uniform exit
            const uint32_t s = i & 1u, u = i >> 1;
            const uint32_t leaf = it.x, q0 = it.y, nq = it.z;
            const int n16 = (int)((nq + 15u) & ~15u);
            // the limit buffer s is free once the epilogue of the item two back is done
            if (!warp_wait(&cempty[s], (u & 1u) ^ 1u)) {
                if (lane == 0) tf_fail(&abort_s, v.err, 128u);
                break;
            }
            // query ids of this warp's rows (g, g + 4, ...; lane r holds row g + 4 r) and
            // the per-column limits, before the B tile is free
            const int gw = warp - W_GATHER;
            uint32_t myq[TF_NQ / (TF_GATHER_WARPS * 32)];
#pragma unroll
            for (int h = 0; h < TF_NQ / (TF_GATHER_WARPS * 32); ++h) {
                const int jr = gw + TF_GATHER_WARPS * (lane + 32 * h);
                myq[h] = jr < (int)nq ? v.pairs[q0 + jr] : 0u;
            }
            for (int j = gt; j < n16; j += TF_GATHER_WARPS * 32) {
                if (j < (int)nq) {
                    const uint32_t b = v.pairs[q0 + j];
                    const float4 qc = v.qc[b];
                    const unsigned long long ku = ld_volatile_u64(&v.utop[(size_t)b * MAX_K + k - 1]);
                    double ub = (double)qc.z;
                    if (ku != EMPTY_SLOT) ub = fmin(ub, (double)key_d2(ku));
                    const double X = (double)v.leaf_xnorm[leaf], Q = (double)qc.y;
                    const double E = (v.c_xq * X * Q + v.c_sq * (X * X + Q * Q)) * (1.0 + 1e-9);
                    qid_s[s][j] = b;
                    qn_s[s][j] = qc.x;
                    lim_s[s][j] = __double2float_ru(ub + E);
                    eu_s[s][j] = __double2float_ru(E);
                    ku_s[s][j] = ku == EMPTY_SLOT ? 0x7f800000u : (unsigned)(ku >> 32);
                } else {
                    qn_s[s][j] = 0.0f;  // padding columns: a limit no value passes
                    lim_s[s][j] = -INFINITY;
                }
            }
            // the B tile is free once the previous item's MMAs have completed; every
            // copy is then issued without waiting
            if (i > 0 && !warp_wait(&bempty, (i - 1) & 1u)) {
                if (lane == 0) tf_fail(&abort_s, v.err, 128u);
                break;
            }
#pragma unroll
            for (int h = 0; h < TF_NQ / (TF_GATHER_WARPS * 32); ++h) {
                for (int r = 0; r < 32; ++r) {
                    const int j = gw + TF_GATHER_WARPS * (r + 32 * h);
                    if (j >= n16) break;
                    const uint32_t b = __shfl_sync(FULL, myq[h], r);
                    for (int ch = lane; ch < cpr; ch += 32) {
                        unsigned char* dst = Bs + sw128_offset(j, ch, n16);
                        if (j < (int)nq)
                            cp_async16(dst, v.qb + (size_t)b * n + ch * 8);
                        else
                            *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
            }
            cp_async_wait_all();
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&cfull[s]);
                mbar_arrive(&bfull);
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps
        // warp w reads TMEM lanes 32 (w % 4) .. +31 (its rows), column groups of
        // 16 alternating between the two warps of a quarter
        const int qd = warp & 3, half = warp >> 2;
        uint32_t e_t = 0;
        for (uint32_t i = 0;; ++i) {
            const uint32_t slot = i % TF_SLOTS, ph = (i / TF_SLOTS) & 1u;
            if (!warp_wait(&itemf[slot], ph)) {
                if (lane == 0) tf_fail(&abort_s, v.err, 256u);
                break;
            }
            const uint4 it = item_s[slot];
            const uint32_t it_le = item_le[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&iteme[slot]);
            if (__any_sync(FULL, it.z == 0 || abort_s)) break;  // warp-uniform exit
            const uint32_t s = i & 1u, u = i >> 1;
            const uint32_t nq = it.z;
            const int n16 = (int)((nq + 15u) & ~15u);
            const int64_t lb = it.w, le = it_le;
            const int tiles = (int)((le - lb + TC_M - 1) / TC_M);
            if (!warp_wait(&cfull[s], u & 1u)) {  // this item's limits are in place
                if (lane == 0) tf_fail(&abort_s, v.err, 512u);
                break;
            }
            const float* lim = lim_s[s];
            const float* qn = qn_s[s];
            const int groups = n16 / 16;
            const int row = qd * 32 + lane;
            int64_t pos = lb + row;
            float xr = pos < le ? v.xn[pos] : INFINITY;
            bool ok = true;
            for (int t = 0; t < tiles; ++t, ++e_t) {
                const uint32_t a = e_t & 1u, aph = (e_t >> 1) & 1u;
                const bool valid = pos < le;
                // the next tile's row norm, loaded while this tile is consumed
                const int64_t pn = pos + TC_M;
                const float xr_next = pn < le ? v.xn[pn] : INFINITY;
                if (!warp_wait(&accf[a], aph)) {
                    if (lane == 0) tf_fail(&abort_s, v.err, 1024u);
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int g = half; g < groups; g += 2) {
                    float acc[16];
                    __syncwarp();  // converge after the divergent updates below
                    tc_ld_x16(tmem + a * (uint32_t)TF_NQ + (uint32_t)(g * 16) + ((uint32_t)(qd * 32) << 16), acc);
                    // fast test of the 16 columns; rows past the leaf carry +inf
                    unsigned pm = 0;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const int j = g * 16 + c;
                        const float dt = fmaf(-2.0f, acc[c], xr + qn[j]);
                        pm |= (dt <= lim[j] ? 1u : 0u) << c;
                    }
                    if (!valid) pm = 0;
                    if (__any_sync(FULL, pm != 0) == 0) continue;
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        const int j = g * 16 + c;
                        if (j >= (int)nq) break;
                        const float dt = fmaf(-2.0f, acc[c], xr + qn[j]);
                        const bool pass = (pm >> c) & 1u;
                        const unsigned m = __ballot_sync(FULL, pass);
                        if (m == 0) continue;
                        const int leader = __ffs(m) - 1;
                        uint32_t base = 0;
                        if (lane == leader) base = atomicAdd(v.cand_count, (uint32_t)__popc(m));
                        base = __shfl_sync(FULL, base, leader);
                        if (pass) {
                            const uint32_t slot_c = base + (uint32_t)__popc(m & ((1u << lane) - 1u));
                            const float eu = eu_s[s][j];
                            const uint32_t qb_id = qid_s[s][j];
                            if (slot_c < v.cand_cap)
                                v.cand[slot_c] = make_uint4((uint32_t)pos, qb_id, __float_as_uint(dt),
                                                            __float_as_uint(eu));
                            const float up = __fadd_ru(dt, eu);
                            if (__float_as_uint(up) < ku_s[s][j]) {
                                unsigned long long* slots = v.utop + (size_t)qb_id * MAX_K;
                                topk_insert(slots, k, pack_key(up, (uint32_t)pos));
                                const unsigned long long kk = ld_volatile_u64(&slots[k - 1]);
                                if (kk != EMPTY_SLOT) atomicMin(&ku_s[s][j], (unsigned)(kk >> 32));
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[a]);
                pos = pn;
                xr = xr_next;
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(&cempty[s]);  // this item's limits are no longer read
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, TF_TMEM_COLS);
}

// BF16 copy of the collection (leaf order), fp32 squared row norms, and the
// largest row norm of every leaf (rounded up).  One CTA per leaf, one warp per row.
__global__ void __launch_bounds__(256) tc_prepare_kernel(const float* __restrict__ x,
                                                         const uint32_t* __restrict__ row_of,
                                                         const uint32_t* __restrict__ leaf_begin, int n,
                                                         uint16_t* __restrict__ xb, float* __restrict__ xn,
                                                         float* __restrict__ leaf_xnorm, unsigned* bad) {
    __shared__ double wmax[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t l = blockIdx.x;
    const int64_t lb = leaf_begin[l], le = leaf_begin[l + 1];
    double mymax = 0.0;
    for (int64_t r = lb + warp; r < le; r += 8) {
        // rows in leaf order, or the caller's rows gathered by original id
        const float4* xr = reinterpret_cast<const float4*>(x + (int64_t)(row_of ? row_of[r] : (uint32_t)r) * n);
        uint2* dst = reinterpret_cast<uint2*>(xb + r * n);
        double acc = 0.0;
        for (int i = lane; i < n / 4; i += 32) {
            const float4 f = ld_stream(xr + i);
            acc += (double)f.x * f.x + (double)f.y * f.y + (double)f.z * f.z + (double)f.w * f.w;
            const __nv_bfloat162 h0 = __floats2bfloat162_rn(f.x, f.y), h1 = __floats2bfloat162_rn(f.z, f.w);
            dst[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
        if (lane == 0) xn[r] = __double2float_rn(acc);
        mymax = fmax(mymax, acc);
    }
    if (lane == 0) wmax[warp] = mymax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < 8; ++i) m = fmax(m, wmax[i]);
        const float X = __double2float_ru(sqrt(m) * (1.0 + 1e-12));
        leaf_xnorm[l] = X;
        if (!(X < 1e18f)) atomicOr(bad, 1u);
    }
}

// per query of the batch (after its approximate answer): BF16 copy, and
// {squared norm (fp32), norm rounded up, upper bound of the k-th best squared
// distance: the approximate answer's k-th fp32 value times (1 + 5 delta)}
__global__ void __launch_bounds__(256) tc_qprep_kernel(const QueryScratch* __restrict__ ss, int B, int n,
                                                       int k, uint16_t* __restrict__ qb,
                                                       float4* __restrict__ qc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 8 + warp;
    if (b >= B) return;
    const QueryScratch& s = ss[b];
    const float4* qr = reinterpret_cast<const float4*>(s.q);
    uint2* dst = reinterpret_cast<uint2*>(qb + (size_t)b * n);
    double acc = 0.0;
    for (int i = lane; i < n / 4; i += 32) {
        const float4 f = qr[i];
        acc += (double)f.x * f.x + (double)f.y * f.y + (double)f.z * f.z + (double)f.w * f.w;
        const __nv_bfloat162 h0 = __floats2bfloat162_rn(f.x, f.y), h1 = __floats2bfloat162_rn(f.z, f.w);
        dst[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL, acc, off);
    if (lane == 0) {
        const unsigned long long kth = s.topk[k - 1];
        const float ub = kth == EMPTY_SLOT ? INFINITY
                                           : __double2float_ru((double)key_d2(kth) * (1.0 + 5.0 * s.ctl->delta));
        qc[b] = make_float4(__double2float_rn(acc), __double2float_ru(sqrt(acc) * (1.0 + 1e-12)), ub, 0.0f);
    }
}

// one CTA: exclusive scan of the per-leaf pair counts (pair offsets) and of the
// per-leaf work items (ceil(count / nq_max), the leaf's queries split evenly),
// writing the items.  misc[0] = items, misc[1] = pairs.
__global__ void __launch_bounds__(1024) bq_items_kernel(const uint32_t* __restrict__ leaf_count, int64_t L,
                                                        int nq_max, uint32_t* __restrict__ leaf_off,
                                                        uint4* __restrict__ items, uint32_t items_cap,
                                                        uint32_t* misc) {
    __shared__ uint32_t scr0[32], scr1[32];
    const int64_t per = (L + blockDim.x - 1) / blockDim.x;
    const int64_t l0 = (int64_t)threadIdx.x * per, l1 = l0 + per < L ? l0 + per : L;
    uint32_t sc = 0, sch = 0;
    for (int64_t l = l0; l < l1; ++l) {
        const uint32_t c = leaf_count[l];
        sc += c;
        sch += (c + nq_max - 1) / nq_max;
    }
    uint32_t tot_c, tot_ch;
    uint32_t oc = block_excl_scan<uint32_t>(sc, 0u, OpAdd<uint32_t>(), scr0, &tot_c);
    uint32_t och = block_excl_scan<uint32_t>(sch, 0u, OpAdd<uint32_t>(), scr1, &tot_ch);
    for (int64_t l = l0; l < l1; ++l) {
        const uint32_t c = leaf_count[l];
        leaf_off[l] = oc;
        const uint32_t nch = (c + nq_max - 1) / nq_max;
        for (uint32_t ch = 0; ch < nch; ++ch, ++och) {
            const uint32_t a = (uint32_t)((uint64_t)c * ch / nch), e = (uint32_t)((uint64_t)c * (ch + 1) / nch);
            if (och < items_cap) items[och] = make_uint4((uint32_t)l, oc + a, e - a, 0u);
        }
        oc += c;
    }
    if (threadIdx.x == 0) {
        misc[0] = tot_ch < items_cap ? tot_ch : items_cap;
        misc[1] = tot_c;
        leaf_off[L] = tot_c;
    }
}

// ================================================================ host side
struct TcState {
    // per index: BF16 copy of the collection
    uint16_t* xb = nullptr;        // [N][n]
    float* xn = nullptr;           // [N]
    float* leaf_xnorm = nullptr;   // [L]
    CUtensorMap tmap;
    uint32_t* leaf_count = nullptr;   // [L]
    uint32_t* leaf_off = nullptr;     // [L+1]
    uint32_t* mask = nullptr;         // [L][ceil(Bcap / 32)] pair ballots
    uint32_t* misc = nullptr;         // [0] items [1] pairs [2] claim [3] kept rows [4] error bits
    uint32_t* host_misc = nullptr;    // pinned copy of misc
    uint4* cand = nullptr;            // kept rows
    uint32_t cand_cap = 0;
    // per batch (grown on demand)
    int Bcap = 0;
    float* q = nullptr;
    float* table = nullptr;
    uint32_t* bins = nullptr;
    unsigned long long* topk = nullptr;
    unsigned long long* cand_key = nullptr;
    uint32_t* cand_pos = nullptr;
    QCtl* ctl = nullptr;
    int64_t* out_idx = nullptr;
    float* out_dist = nullptr;
    QueryScratch* ss = nullptr;
    uint16_t* qb = nullptr;
    float4* qc = nullptr;
    unsigned long long* utop = nullptr;
    uint32_t* pairs = nullptr;
    uint4* items = nullptr;
    uint32_t items_cap = 0;
    QCtl* host_ctl = nullptr;      // pinned
    int64_t* host_idx = nullptr;   // pinned [Bcap][MAX_K]
    float* host_dist = nullptr;
};

static void free_batch(TcState* t, cudaStream_t st) {
    void* ptrs[] = {t->q, t->table, t->bins, t->topk, t->cand_key, t->cand_pos, t->ctl, t->out_idx,
                    t->out_dist, t->ss, t->qb, t->qc, t->utop, t->pairs, t->items, t->mask};
    for (void* p : ptrs)
        if (p) dev_free(p, st);
    if (t->host_ctl) cudaFreeHost(t->host_ctl);
    if (t->host_idx) cudaFreeHost(t->host_idx);
    if (t->host_dist) cudaFreeHost(t->host_dist);
    t->q = t->table = nullptr;
    t->bins = t->cand_pos = t->pairs = nullptr;
    t->topk = t->cand_key = t->utop = nullptr;
    t->ctl = nullptr;
    t->out_idx = nullptr;
    t->out_dist = nullptr;
    t->qc = nullptr;
    t->ss = nullptr;
    t->qb = nullptr;
    t->items = nullptr;
    t->mask = nullptr;
    t->items_cap = 0;
    t->host_ctl = nullptr;
    t->host_idx = nullptr;
    t->host_dist = nullptr;
    t->Bcap = 0;
}

void free_tc_state(isax_index* ix, cudaStream_t st) {
    TcState* t = static_cast<TcState*>(ix->tc);
    if (!t) return;
    free_batch(t, st);
    void* ptrs[] = {t->xb, t->xn, t->leaf_xnorm, t->leaf_count, t->leaf_off, t->misc, t->cand};
    for (void* p : ptrs)
        if (p) dev_free(p, st);
    if (t->host_misc) cudaFreeHost(t->host_misc);
    delete t;
    ix->tc = nullptr;
}

template <typename T>
static T* dalloc(size_t count, cudaStream_t st) {
    return static_cast<T*>(dev_alloc(sizeof(T) * (count ? count : 1), st));
}

// the BF16 copy of the collection, built once per index
static TcState* ensure_tc(isax_index* ix, cudaStream_t st) {
    if (ix->tc) return static_cast<TcState*>(ix->tc);
    const DevIndex& d = ix->d;
    if (d.n % TC_KATOM != 0 || d.n > 2048)
        throw Error{ISAX_ERR_INVALID_ARG,
                    "the BF16 filter needs a series length that is a multiple of 64 and at most 2048"};
    if (!(d.maxabs < 1e15f))
        throw Error{ISAX_ERR_INVALID_ARG, "values too large for the BF16 filter's error bound"};
    TcState* t = new TcState();
    ix->tc = t;
    try {
        t->xb = dalloc<uint16_t>((size_t)d.N * d.n, st);
        t->xn = dalloc<float>((size_t)d.N, st);
        t->leaf_xnorm = dalloc<float>((size_t)d.L, st);
        t->leaf_count = dalloc<uint32_t>((size_t)d.L, st);
        t->leaf_off = dalloc<uint32_t>((size_t)d.L + 1, st);
        t->misc = dalloc<uint32_t>(8, st);
        ISAX_CUDA_TRY(cudaMallocHost((void**)&t->host_misc, sizeof(uint32_t) * 8));
        ISAX_CUDA_TRY(cudaMemsetAsync(t->misc, 0, sizeof(uint32_t) * 8, st));
        {
            ISAX_LAUNCH("tc_prepare", st);
            tc_prepare_kernel<<<(unsigned)d.L, 256, 0, st>>>(ix->x, d.rows_in_place ? d.orig : nullptr,
                                                             ix->leaf_begin, d.n, t->xb, t->xn,
                                                             t->leaf_xnorm, t->misc + 4);
            ISAX_CUDA_TRY(cudaGetLastError());
        }
        ISAX_CUDA_TRY(cudaMemcpyAsync(t->host_misc, t->misc, sizeof(uint32_t) * 8, cudaMemcpyDeviceToHost, st));
        ISAX_CUDA_TRY(cudaStreamSynchronize(st));
        if (t->host_misc[4])
            throw Error{ISAX_ERR_INVALID_ARG, "row norms too large for the BF16 filter's error bound"};
        make_tmap_bf16(&t->tmap, t->xb, (uint64_t)d.N, (uint64_t)d.n);
    } catch (...) {
        free_tc_state(ix, st);
        throw;
    }
    return t;
}

static void ensure_batch_alloc(TcState* t, const isax_index* ix, int B, cudaStream_t st);
// batch scratch for B queries: all of it, or (on a failed allocation) none
static void ensure_batch(TcState* t, const isax_index* ix, int B, cudaStream_t st) {
    if (t->Bcap >= B) return;
    free_batch(t, st);
    try {
        ensure_batch_alloc(t, ix, B, st);
    } catch (...) {
        free_batch(t, st);
        throw;
    }
}
static void ensure_batch_alloc(TcState* t, const isax_index* ix, int B, cudaStream_t st) {
    const DevIndex& d = ix->d;
    const size_t Bs = (size_t)B;
    t->q = dalloc<float>(Bs * d.n, st);
    t->table = dalloc<float>(Bs * W * d.card, st);
    t->bins = dalloc<uint32_t>(Bs * 2 * NBINS, st);
    t->topk = dalloc<unsigned long long>(Bs * MAX_K, st);
    t->cand_key = dalloc<unsigned long long>(Bs * TF_QCAP, st);
    t->cand_pos = dalloc<uint32_t>(Bs * TF_QCAP, st);
    t->ctl = dalloc<QCtl>(Bs, st);
    t->out_idx = dalloc<int64_t>(Bs * MAX_K, st);
    t->out_dist = dalloc<float>(Bs * MAX_K, st);
    t->ss = dalloc<QueryScratch>(Bs, st);
    t->qb = dalloc<uint16_t>(Bs * d.n, st);
    t->qc = dalloc<float4>(Bs, st);
    t->utop = dalloc<unsigned long long>(Bs * MAX_K, st);
    t->pairs = dalloc<uint32_t>(Bs * (size_t)d.L, st);
    t->mask = dalloc<uint32_t>((size_t)d.L * ((Bs + 31) / 32), st);
    const int nq = tf_nq_max(d.n);
    t->items_cap = (uint32_t)std::min<uint64_t>((uint64_t)d.L * (1 + (Bs + nq - 1) / nq), 0xffffffffull);
    t->items = dalloc<uint4>(t->items_cap, st);
    ISAX_CUDA_TRY(cudaMallocHost((void**)&t->host_ctl, sizeof(QCtl) * Bs));
    ISAX_CUDA_TRY(cudaMallocHost((void**)&t->host_idx, sizeof(int64_t) * Bs * MAX_K));
    ISAX_CUDA_TRY(cudaMallocHost((void**)&t->host_dist, sizeof(float) * Bs * MAX_K));
    std::vector<QueryScratch> hs(Bs);
    for (size_t b = 0; b < Bs; ++b) {
        QueryScratch& q = hs[b];
        q.q = t->q + b * d.n;
        q.table = t->table + b * W * d.card;
        q.leaf_lb = nullptr;
        q.work = nullptr;
        q.bin_count = t->bins + b * 2 * NBINS;
        q.bin_cursor = q.bin_count + NBINS;
        q.topk = t->topk + b * MAX_K;
        q.cand_key = t->cand_key + b * TF_QCAP;
        q.cand_pos = t->cand_pos + b * TF_QCAP;
        q.cand_cap = TF_QCAP;
        q.ctl = t->ctl + b;
        q.out_idx = t->out_idx + b * MAX_K;
        q.out_dist = t->out_dist + b * MAX_K;
    }
    ISAX_CUDA_TRY(cudaMemcpyAsync(t->ss, hs.data(), sizeof(QueryScratch) * Bs, cudaMemcpyHostToDevice, st));
    ISAX_CUDA_TRY(cudaMemsetAsync(t->ctl, 0, sizeof(QCtl) * Bs, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));  // hs goes out of scope
    t->Bcap = B;
}

static void ensure_cand(TcState* t, uint32_t cap, cudaStream_t st) {
    if (t->cand_cap >= cap) return;
    if (t->cand) dev_free(t->cand, st);
    t->cand = nullptr;
    t->cand_cap = 0;
    t->cand = dalloc<uint4>(cap, st);
    t->cand_cap = cap;
}

// E = c_xq X Q + c_sq (X^2 + Q^2)  (see the error bound at the top of this part)
static void tc_bound_constants(int n, double* c_xq, double* c_sq) {
    const double u = 0x1p-24, ub = 0x1p-8;
    const double g = (1.0 + ub) * (1.0 + ub);
    *c_xq = 2.0 * (2.0 * ub + ub * ub) + 2.0 * n * 0x1p-21 * g + 2.01 * u * g;
    *c_sq = 4.0 * u;
}

// one pass of at most TF_MAX_B queries, already in t->q; false if the kept-row
// buffer overflowed (nothing is valid then)
static bool run_pass(isax_index* ix, TcState* t, int B, int k, cudaStream_t st) {
    const DevIndex& d = ix->d;
    const int nq = tf_nq_max(d.n);
    launch_bq_prep(ix, t->ss, B, k, TC_APPROX_NEIGHBORS, st);
    launch_bq_approx(ix, t->ss, B, k, TC_APPROX_NEIGHBORS, st);
    {
        ISAX_LAUNCH("tc_qprep", st);
        tc_qprep_kernel<<<(B + 7) / 8, 256, 0, st>>>(t->ss, B, d.n, k, t->qb, t->qc);
        ISAX_CUDA_TRY(cudaGetLastError());
    }
    ISAX_CUDA_TRY(cudaMemsetAsync(t->utop, 0xff, sizeof(unsigned long long) * (size_t)B * MAX_K, st));
    ISAX_CUDA_TRY(cudaMemsetAsync(t->leaf_count, 0, sizeof(uint32_t) * d.L, st));
    ISAX_CUDA_TRY(cudaMemsetAsync(t->misc, 0, sizeof(uint32_t) * 8, st));
    launch_bq_pairs(ix, t->ss, B, k, t->leaf_count, t->mask, st);
    {
        ISAX_LAUNCH("bq_items", st);
        bq_items_kernel<<<1, 1024, 0, st>>>(t->leaf_count, d.L, nq, t->leaf_off, t->items, t->items_cap,
                                            t->misc);
        ISAX_CUDA_TRY(cudaGetLastError());
    }
    launch_bq_fill(ix, B, t->mask, t->leaf_off, t->pairs, st);
    TcView v;
    v.leaf_begin = ix->leaf_begin;
    v.xn = t->xn;
    v.leaf_xnorm = t->leaf_xnorm;
    v.items = t->items;
    v.n_items = t->misc + 0;
    v.claim = t->misc + 2;
    v.pairs = t->pairs;
    v.qb = t->qb;
    v.qc = t->qc;
    v.utop = t->utop;
    v.cand = t->cand;
    v.cand_count = t->misc + 3;
    v.cand_cap = t->cand_cap;
    v.err = t->misc + 4;
    v.n = d.n;
    v.k = k;
    tc_bound_constants(d.n, &v.c_xq, &v.c_sq);
    const size_t smem = smem_tf();
    {
        static bool attr[64] = {};
        if (ix->device < 0 || ix->device >= 64 || !attr[ix->device]) {
            ISAX_CUDA_TRY(cudaFuncSetAttribute(tc_filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem_tf()));
            if (ix->device >= 0 && ix->device < 64) attr[ix->device] = true;
        }
        ISAX_LAUNCH("tc_filter", st);
        tc_filter_kernel<<<ix->num_sms, TF_THREADS, smem, st>>>(t->tmap, v);
        ISAX_CUDA_TRY(cudaGetLastError());
    }
    launch_bq_recheck(ix, t->ss, k, t->cand, t->misc + 3, t->cand_cap, st);
    launch_bq_finalize(ix, t->ss, B, k, st);
    ISAX_CUDA_TRY(cudaMemcpyAsync(t->host_misc, t->misc, sizeof(uint32_t) * 8, cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaMemcpyAsync(t->host_ctl, t->ctl, sizeof(QCtl) * B, cudaMemcpyDeviceToHost, st));
    ISAX_CUDA_TRY(cudaStreamSynchronize(st));
    if (t->host_misc[4])
        throw Error{ISAX_ERR_TIMEOUT, "tensor-core filter: a bounded wait gave up (" +
                                          std::to_string(t->host_misc[4]) + ")"};
    return t->host_misc[3] <= t->cand_cap;
}

void prepare_tc(isax_index* ix, cudaStream_t st) { ensure_tc(ix, st); }

void query_batch_tc(isax_index* ix, const float* Q, int B, int k, uint32_t mem_flags, int64_t* out_idx,
                    float* out_dist, isax_query_stats_fill fill, void* fill_ctx, cudaStream_t st) {
    TcState* t = ensure_tc(ix, st);
    const int n = ix->d.n;
    const int P = std::max(1, std::min<int>(TF_MAX_B, (int)std::min<int64_t>(B, (1ll << 29) / std::max<int64_t>(ix->d.L, 1))));
    ensure_batch(t, ix, std::min(B, P), st);
    if (!t->cand) ensure_cand(t, 1u << 22, st);
    const cudaMemcpyKind kin = (mem_flags & ISAX_MEM_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                   : cudaMemcpyHostToDevice;
    const bool dev_out = (mem_flags & ISAX_MEM_OUTPUT_DEVICE) != 0;
    bool nonfinite = false;
    for (int b0 = 0; b0 < B; b0 += P) {
        const int Bp = std::min(P, B - b0);
        for (int attempt = 0;; ++attempt) {
            ISAX_CUDA_TRY(cudaMemcpyAsync(t->q, Q + (size_t)b0 * n, sizeof(float) * (size_t)Bp * n, kin, st));
            if (run_pass(ix, t, Bp, k, st)) break;
            if (attempt >= 3) throw Error{ISAX_ERR_INTERNAL, "tensor-core filter kept too many rows"};
            const uint64_t want = std::min<uint64_t>((uint64_t)t->host_misc[3] * 2, 0xffffffffull);
            ensure_cand(t, (uint32_t)want, st);
        }
        // outputs: row b of the [Bp][MAX_K] result arrays holds query b0 + b
        if (dev_out) {
            ISAX_CUDA_TRY(cudaMemcpy2DAsync(out_idx + (size_t)b0 * k, sizeof(int64_t) * k, t->out_idx,
                                            sizeof(int64_t) * MAX_K, sizeof(int64_t) * k, Bp,
                                            cudaMemcpyDeviceToDevice, st));
            ISAX_CUDA_TRY(cudaMemcpy2DAsync(out_dist + (size_t)b0 * k, sizeof(float) * k, t->out_dist,
                                            sizeof(float) * MAX_K, sizeof(float) * k, Bp,
                                            cudaMemcpyDeviceToDevice, st));
        } else {
            ISAX_CUDA_TRY(cudaMemcpy2DAsync(t->host_idx, sizeof(int64_t) * k, t->out_idx,
                                            sizeof(int64_t) * MAX_K, sizeof(int64_t) * k, Bp,
                                            cudaMemcpyDeviceToHost, st));
            ISAX_CUDA_TRY(cudaMemcpy2DAsync(t->host_dist, sizeof(float) * k, t->out_dist,
                                            sizeof(float) * MAX_K, sizeof(float) * k, Bp,
                                            cudaMemcpyDeviceToHost, st));
            ISAX_CUDA_TRY(cudaStreamSynchronize(st));
            memcpy(out_idx + (size_t)b0 * k, t->host_idx, sizeof(int64_t) * (size_t)Bp * k);
            memcpy(out_dist + (size_t)b0 * k, t->host_dist, sizeof(float) * (size_t)Bp * k);
        }
        const cudaMemcpyKind kout = dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        for (int b = 0; b < Bp; ++b) {
            QCtl c = t->host_ctl[b];
            c.flags |= injected_query_flags();
            int reruns = 0;
            if (c.flags & QF_NONFINITE) {
                nonfinite = true;
                continue;
            }
            if (c.flags & QF_STALLED) throw Error{ISAX_ERR_TIMEOUT, "a bounded wait of the query gave up"};
            c.leaves_scanned = c.leaves_queued;
            if (c.flags & (QF_OVERFLOW | QF_SHORT)) {
                // this query's candidate window overflowed: answer it alone
                ISAX_CUDA_TRY(cudaMemcpyAsync(ix->qs.q, Q + (size_t)(b0 + b) * n, sizeof(float) * n, kin, st));
                query_device(ix, k, &c, &reruns, st);
                ISAX_CUDA_TRY(cudaMemcpyAsync(out_idx + (size_t)(b0 + b) * k, ix->qs.out_idx,
                                              sizeof(int64_t) * k, kout, st));
                ISAX_CUDA_TRY(cudaMemcpyAsync(out_dist + (size_t)(b0 + b) * k, ix->qs.out_dist,
                                              sizeof(float) * k, kout, st));
                ISAX_CUDA_TRY(cudaStreamSynchronize(st));
                reruns += 1;
            }
            if (fill) fill(fill_ctx, b0 + b, c, reruns);
        }
    }
    if (nonfinite) throw Error{ISAX_ERR_INVALID_ARG, "a query contains a non-finite value"};
}

}  // namespace isax
