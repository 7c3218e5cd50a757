// FMA-rate probe of the FP64 and FP32 pipes (the ALU roofs of the fast solves).
//
// Every thread keeps NCH independent accumulators and advances each one by one
// fused multiply-add per round, x <- x * a + b, for `iters` rounds: NCH independent
// dependency chains per thread hide the FMA latency, so with enough threads per SM
// the issue rate of the FMA pipe is the limit. With a = 1 - 2^-20 the values settle
// towards b / (1 - a) and stay finite; the sums are written out so that nothing is
// optimised away. The rate is 2 * NCH * iters * threads / kernel time (one FMA = two
// floating-point operations), timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cqprobe.h"

namespace {

constexpr int NCH = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T a, T b, int iters, T *__restrict__ out) {
    T x[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) x[k] = (T)(threadIdx.x + 1 + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < NCH; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < NCH; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int blocks, int threads, int iters, void *out, double *rate, cudaStream_t s) {
    const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1024.0);
    T *o = static_cast<T *>(out);
    k_fma_chains<T><<<blocks, threads, 0, s>>>(a, b, iters, o);        // warm-up
    if (cudaGetLastError() != cudaSuccess) return -3;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -3;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return -3;
    }
    int st = 0;
    float ms = 0.0f;
    if (cudaEventRecord(e0, s) != cudaSuccess) st = -3;
    if (!st) k_fma_chains<T><<<blocks, threads, 0, s>>>(a, b, iters, o);
    if (!st && cudaGetLastError() != cudaSuccess) st = -3;
    if (!st && cudaEventRecord(e1, s) != cudaSuccess) st = -3;
    if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = -3;
    if (!st && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = -3;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    if (!(ms > 0.0f)) return -3;
    *rate = 2.0 * NCH * (double)iters * (double)blocks * (double)threads / (ms * 1e-3);
    return 0;
}

}  // namespace

extern "C" int cq_probe_fma_rate(int32_t prec, int32_t blocks, int32_t threads, int32_t iters, void *out_dev,
                                 double *flops_per_s, void *stream) {
    if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 || iters < 1 || !out_dev || !flops_per_s)
        return -1;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == 0) return run<double>(blocks, threads, iters, out_dev, flops_per_s, s);
    if (prec == 1) return run<float>(blocks, threads, iters, out_dev, flops_per_s, s);
    return -1;
}
