// isax_tc.cuh - shapes and descriptors of the tensor-core contraction.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace isax {

constexpr int TC_M = 128;     // rows per MMA tile (TMEM lanes)
constexpr int TC_K = 256;     // series length handled by the contraction (K)
constexpr int TC_KATOM = 64;  // BF16 elements per 128-byte swizzle atom row

// instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B BF16, both
// K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

void tc_selftest(const void* A, const void* B, int N, float* D, cudaStream_t st);

}  // namespace isax
