// Device arithmetic-rate probe: the FP64 fused multiply-add rate of this GPU, measured rather
// than taken from a datasheet, as the denominator for the kernels that FP64 arithmetic bounds
// (the FP64 step and the shape-vector solve).  Not part of the method.
//
// Every thread runs kChains (16) independent FMA chains x <- x * a + b for `iters` iterations, so
// the FP64 pipe never waits on a dependency once a few warps per SM are resident; the grid is
// blocks_per_sm CTAs of 256 threads on every SM.  Each CTA writes one sum to `sink` so the
// compiler keeps the work.
#include <cuda_runtime.h>

#include <string>

#include "mlbm_internal.h"

namespace mlbm {
namespace {

constexpr int kChains = 16;
constexpr int kRateThreads = 256;

__global__ void __launch_bounds__(kRateThreads) fma64_rate_kernel(int64_t iters, double a, double b,
                                                                 double *__restrict__ sink) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * (threadIdx.x + 1) + c;
#pragma unroll 4
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    __shared__ double red[kRateThreads / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRateThreads / 32; ++w) t += red[w];
        sink[blockIdx.x] = t;
    }
}

}  // namespace
}  // namespace mlbm

using namespace mlbm;

extern "C" {

int mlbm_fp64_fma_rate(int64_t iters, int blocks_per_sm, double *sink, int64_t sink_len, void *stream,
                       double *flops) {
    set_error("");
    if (iters <= 0 || blocks_per_sm <= 0 || !sink || !flops) return fail(MLBM_EINVAL, "bad argument");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(MLBM_ECUDA, "no usable CUDA device");
    }
    const int64_t blocks = (int64_t)blocks_per_sm * sms;
    if (blocks > sink_len || blocks > (1 << 30))
        return fail(MLBM_EINVAL, "sink holds " + std::to_string(sink_len) + " doubles, the probe needs " +
                                     std::to_string(blocks));
    fma64_rate_kernel<<<(int)blocks, kRateThreads, 0, (cudaStream_t)stream>>>(iters, 0.9999999, 1e-7, sink);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MLBM_ECUDA, std::string("FMA rate probe launch: ") + cudaGetErrorString(e));
    *flops = 2.0 * kChains * (double)iters * (double)kRateThreads * (double)blocks;
    return MLBM_OK;
}

}  // extern "C"
