// isax_kernels_util.cuh - small device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "isax_common.cuh"

namespace isax {

constexpr unsigned FULL = 0xffffffffu;

// streaming 16-byte load that does not allocate in L1 (data read once)
__device__ __forceinline__ float4 ld_stream(const float4* p) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint4 ld_stream_u4(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// streaming store (evict-first)
__device__ __forceinline__ void st_stream(float4* p, float4 v) {
    asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// bring the line holding p into L2 ahead of a later read
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *(volatile const unsigned long long*)p;
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
    return *(volatile const uint32_t*)p;
}
__device__ __forceinline__ uint2 ld_volatile_u2(const uint2* p) {
    uint2 v;
    asm volatile("ld.volatile.global.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

// packed (fp32 value bits << 32 | id): for non-negative values the integer
// order is the (value, id) order
__device__ __forceinline__ unsigned long long pack_key(float d2, uint32_t id) {
    return ((unsigned long long)__float_as_uint(d2) << 32) | id;
}
__device__ __forceinline__ float key_d2(unsigned long long key) {
    return __uint_as_float((uint32_t)(key >> 32));
}

// insert key into the ascending array slots[0..k): each step puts the smaller
// value in the slot and carries the larger one down; values only decrease, so
// after all concurrent cascades the array holds the k smallest keys, sorted.
__device__ inline void topk_insert(unsigned long long* slots, int k, unsigned long long key) {
    int j = 0;
    while (j < k && ld_volatile_u64(&slots[j]) <= key) ++j;
    for (; j < k; ++j) {
        unsigned long long old = atomicMin(&slots[j], key);
        if (old == EMPTY_SLOT) return;
        if (old > key) key = old;
    }
}

// symbol of v: number of breakpoints beta_t <= v, by binary search over
// bp[0..card] = {-inf, beta_1, ..., beta_{card-1}, +inf} (bp in shared memory)
__device__ __forceinline__ int symbol_of(float v, const float* bp, int card) {
    int s = 0;
    for (int step = card >> 1; step > 0; step >>= 1)
        if (bp[s + step] <= v) s += step;
    return s;
}

// ---------------------------------------------------------------- bulk copies (TMA engine)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// arrive once and expect `bytes` more transaction bytes in the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// arrive once (no transaction bytes)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// bounded wait for phase `parity` of a barrier; false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t max_tries) {
    for (uint32_t i = 0; i < max_tries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// global -> shared, completion counted on `bar` (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// an L2 policy that marks the lines a load brings in as the first to evict
// (data read once, streamed past the working set of the reads around it)
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// bulk_load with an L2 cache policy
__device__ __forceinline__ void bulk_load_hint(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar,
                                               unsigned long long policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
// an mbarrier's memory may be initialised again once no operation uses it
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// 16 bytes global -> shared by this thread (through L2, not L1), asynchronously
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
// one arrival on `bar` once this thread's earlier cp.async copies have landed
// (the barrier's expected count covers it: no increment)
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// shared -> global in the calling thread's bulk group
__device__ __forceinline__ void bulk_store(void* dst, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the calling thread's committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a cooperative launch (all CTAs resident): every CTA
// arrives once on *count, which the caller has cleared before the launch, and
// then waits until `expected` arrivals are seen, polling at most max_polls
// times.  Returns false (in every thread of the CTA) when the wait gave up.
// Called by every thread of every CTA; writes before it are visible after it.
__device__ __forceinline__ bool grid_barrier(uint32_t* count, uint32_t expected, uint32_t max_polls, int* ok_smem) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        bool ok = false;
        for (uint32_t i = 0; i < max_polls; ++i) {
            if (ld_acquire_u32(count) >= expected) {
                ok = true;
                break;
            }
            __nanosleep(64);
        }
        *ok_smem = ok ? 1 : 0;
    }
    __syncthreads();
    return *ok_smem != 0;
}

template <typename T>
struct OpAdd {
    __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
};
template <typename T>
struct OpMax {
    __device__ __forceinline__ T operator()(T a, T b) const { return a > b ? a : b; }
};

// inclusive warp scan
template <typename T, typename Op>
__device__ __forceinline__ T warp_incl_scan(T v, Op op) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        T t = __shfl_up_sync(FULL, v, off);
        if (lane >= off) v = op(v, t);
    }
    return v;
}

// exclusive block scan (blockDim.x a multiple of 32, <= 1024); `scratch` holds
// 32 elements of shared memory; returns the exclusive prefix and the total.
// Must be called by every thread; ends with a __syncthreads.
template <typename T, typename Op>
__device__ __forceinline__ T block_excl_scan(T v, T identity, Op op, T* scratch, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(v, op);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? scratch[lane] : identity;
        w = warp_incl_scan(w, op);
        scratch[lane] = w;
    }
    __syncthreads();
    T before = warp > 0 ? scratch[warp - 1] : identity;
    T excl_in_warp = __shfl_up_sync(FULL, inc, 1);
    if (lane == 0) excl_in_warp = identity;
    T res = op(before, excl_in_warp);
    *total = scratch[nw - 1];
    __syncthreads();
    return res;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

}  // namespace isax
