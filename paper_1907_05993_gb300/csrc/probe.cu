// Measurement helper (no counterpart in the paper): an FP32 fused-multiply-add
// throughput probe, the denominator of the ALU roofline of the ROI
// cross-correlation.  Each thread runs 8 independent chains of packed FP32x2
// FMAs (the instruction the FFT butterflies and smoothing passes use), so the
// FMA pipes stay busy without memory traffic.
#include "internal.cuh"

namespace {

__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, float seed, float *out)
{
    float2 acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = make_float2(seed + (float)(threadIdx.x + j), seed - (float)j);
    const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = __ffma2_rn(acc[j], m, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += acc[j].x + acc[j].y;
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace

extern "C" int hrebsd_probe_fp32_fma(hrebsd_ctx *ctx, int iters, double *flops, void *stream)
{
    if (!ctx || iters < 1 || !flops) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    const int blocks = ctx->num_sms * 8, threads = 256;
    void *scratch = nullptr;
    if ((e = hr_ws(ctx, 15, (size_t)blocks * threads * sizeof(float), &scratch))) return e;
    fma_probe_kernel<<<blocks, threads, 0, hr_stream(stream)>>>(iters, 1.0f, (float *)scratch);
    HR_LAUNCHED(ctx);
    *flops = (double)blocks * threads * iters * 8 * 2 * 2;   // 8 chains x 2 lanes x (mul + add)
    return HREBSD_OK;
}
