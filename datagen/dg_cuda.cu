/*
 * dg_cuda.cu - device build of the seeded input generator (dg_core.h).  One
 * thread per row; every FP64 operation goes through a __d*_rn intrinsic so no
 * multiply-add is fused, which makes each row bit-identical to the host build.
 * Used to fill large collections directly in device memory.
 */
#include <cuda_runtime.h>

#include "dg_core.h"

template <int NMAX>
__global__ void __launch_bounds__(128) dg_rows_kernel(int kind, uint64_t seed, int64_t row0,
                                                      int64_t count, int n, float* out) {
    double buf[NMAX];
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    float* o = out + (size_t)r * (size_t)n;
    if (kind == 0)
        dg_random_walk_row(seed, (uint64_t)(row0 + r), n, buf, o);
    else
        dg_sinusoid_row(seed, (uint64_t)(row0 + r), n, buf, o);
}

template <int NMAX>
static cudaError_t dg_launch(int kind, uint64_t seed, int64_t row0, int64_t count, int n,
                             float* out, cudaStream_t st) {
    const int tpb = 128;
    int64_t blocks = (count + tpb - 1) / tpb;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    if (blocks == 0) return cudaSuccess;
    dg_rows_kernel<NMAX><<<(unsigned)blocks, tpb, 0, st>>>(kind, seed, row0, count, n, out);
    return cudaGetLastError();
}

static int dg_dispatch(int kind, uint64_t seed, int64_t row0, int64_t count, int n, float* out,
                       void* stream) {
    if (n < 1 || n > DG_MAX_N || count < 0 || !out) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (n <= 256)
        e = dg_launch<256>(kind, seed, row0, count, n, out, st);
    else if (n <= 1024)
        e = dg_launch<1024>(kind, seed, row0, count, n, out, st);
    else
        e = dg_launch<DG_MAX_N>(kind, seed, row0, count, n, out, st);
    return e == cudaSuccess ? 0 : 100 + (int)e;
}

extern "C" int dg_cuda_random_walks(uint64_t seed, int64_t row0, int64_t count, int n,
                                    float* d_out, void* stream) {
    return dg_dispatch(0, seed, row0, count, n, d_out, stream);
}

extern "C" int dg_cuda_sinusoids(uint64_t seed, int64_t row0, int64_t count, int n, float* d_out,
                                 void* stream) {
    return dg_dispatch(1, seed, row0, count, n, d_out, stream);
}
