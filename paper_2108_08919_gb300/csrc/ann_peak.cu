// FP32 fused multiply-add throughput of this GPU, measured: the denominator of the pair passes'
// roofline (they are bound by plain FP32 issue, not by HBM or the tensor cores).
//
// Every thread runs NACC independent FMA chains (the dependent latency is hidden by the chains and
// the resident warps) for `iters` iterations; the grid holds every SM at full occupancy.  Two
// forms: the scalar FFMA and the two-lane FFMA2 (one instruction for two lanes), so that the
// rate the pipes sustain is measured whichever form the pair passes issue.  The chains'
// results are stored only when they equal a value they never reach, so no work is removed.
#include "../../include/ann.h"

#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kAcc = 8;

template <bool PAIR>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, float a, float c, float *sink)
{
    float2 acc[kAcc];
#pragma unroll
    for (int k = 0; k < kAcc; k++) acc[k] = make_float2((float)(threadIdx.x + k), (float)(blockIdx.x - k));
    const float2 av = make_float2(a, a), cv = make_float2(c, c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kAcc; k++) {
            if (PAIR) {
                acc[k] = __ffma2_rn(acc[k], av, cv);
            } else {
                acc[k].x = fmaf(acc[k].x, a, c);
                acc[k].y = fmaf(acc[k].y, a, c);
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kAcc; k++) s += acc[k].x + acc[k].y;
    if (s == 1234.5678f) sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int ann_fp32_fma_peak(void *stream, double *tflops_scalar, double *tflops_pair, int32_t *sms)
{
    if (!tflops_scalar || !tflops_pair) return ANN_ERR_INVALID_ARG;
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<false>, kThreads, 0)) {
        cudaGetLastError();
        return ANN_ERR_CUDA;
    }
    if (sms) *sms = nsm;
    const int blocks = nsm * (per_sm > 0 ? per_sm : 1);
    const int iters = 16384;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, sizeof(float) * (size_t)blocks * kThreads);
    if (!e) e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    double out[2] = {0.0, 0.0};
    for (int form = 0; form < 2 && !e; form++) {
        float best = 0.f;
        for (int rep = 0; rep < 4 && !e; rep++) {   // the first launch warms up, the best of the rest counts
            e = cudaEventRecord(e0, s);
            if (!e) {
                if (form == 0) k_fma_chains<false><<<blocks, kThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
                else k_fma_chains<true><<<blocks, kThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
                e = cudaGetLastError();
            }
            if (!e) e = cudaEventRecord(e1, s);
            if (!e) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
            if (!e && rep > 0 && (best == 0.f || ms < best)) best = ms;
        }
        // 2 flops per lane FMA, 2 lanes per accumulator (scalar form: two chains)
        const double flops = 2.0 * 2.0 * kAcc * (double)iters * blocks * kThreads;
        if (!e && best > 0.f) out[form] = flops / (best * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e) {
        cudaGetLastError();
        return ANN_ERR_CUDA;
    }
    *tflops_scalar = out[0];
    *tflops_pair = out[1];
    return ANN_OK;
}
