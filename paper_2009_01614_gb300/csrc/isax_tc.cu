// isax_tc.cu - tensor-core (tcgen05) contraction machinery for the batched,
// BF16-filtered exact k-NN path.  BF16 operands staged in shared memory in the
// 128-byte-swizzled K-major layout (the A side by TMA tensor copies), one
// elected thread issues tcgen05.mma (kind::f16, FP32 accumulate) into TMEM,
// completion is committed to an mbarrier, and the epilogue warps read the
// accumulator rows back with tcgen05.ld.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>

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

// rows x 256 BF16 matrix (row pitch 512 B), boxes of 64 elements x box_rows rows,
// 128-byte swizzle, rows past the end read as zeros
void make_tmap_bf16_rows(CUtensorMap* tm, const void* base, uint64_t rows, uint32_t box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)TC_K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)TC_K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_KATOM, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        throw Error{ISAX_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
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

}  // namespace isax
