// libmgq FP32 arithmetic probe: the measured FP32 FMA peak that the
// ALU-bound kernels (force, heat bath, overrelaxation) are compared with.
#include "mgq_internal.h"

namespace mgq {

// 8 independent chains of packed FMAs (16 FMAs per iteration); the chains'
// values are combined into *sink only by thread 0 of block 0 when the
// combination is negative, which it never is for these inputs, so that no
// launch writes memory but the compiler cannot remove the chains.
__global__ void __launch_bounds__(256) k_fma_probe(int iters, float* sink) {
    float2 acc[8];
    const float2 a = make_float2(0.999999f, 0.999998f), b = make_float2(1e-7f, 2e-7f);
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = make_float2(1.0f + k * 1e-3f + threadIdx.x * 1e-6f, 0.5f + k * 1e-3f);
#pragma unroll 4
    for (int i = 0; i < iters; i++)
#pragma unroll
        for (int k = 0; k < 8; k++) acc[k] = __ffma2_rn(acc[k], a, b);
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; k++) s += acc[k].x + acc[k].y;
    if (s < 0.0f) sink[0] = s;
}

}  // namespace mgq

using namespace mgq;

extern "C" {

uint64_t mgq_fma_probe(int iters, float* sink, void* stream) {
    if (iters < 1 || !sink) return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    const int blocks = 4 * sms;
    k_fma_probe<<<blocks, 256, 0, as_stream(stream)>>>(iters, sink);
    if (cudaGetLastError() != cudaSuccess) return 0;
    return (uint64_t)blocks * 256ull * (uint64_t)iters * 32ull;
}

}  // extern "C"
