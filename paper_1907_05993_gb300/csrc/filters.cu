// f2: pattern preprocessing for real scans (Section 3.2-3.3): Gaussian
// low-/high-pass filtering, static and dynamic background correction, and the
// shift and zoom/shrink correction about the pattern centre.  The paper names
// these steps without their kernels; the library uses Gaussian filters of
// radius ceil(3 sigma) with normalised weights and replicated borders (the
// family of the demons smoothing), division by the scan's mean pattern
// (static) and by the pattern's own blur (dynamic), and a Keys cubic resample
// for the affine correction.  One pass over the images per call; everything
// is FP32 with FP32 accumulation.
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int kMaxFilterRadius = 96;

struct FilterTaps {
    int r;
    float t[2 * kMaxFilterRadius + 1];
};

bool make_taps(float sigma, FilterTaps *f)
{
    if (!(sigma >= 0.0f)) return false;
    if (sigma == 0.0f) {
        f->r = 0;
        f->t[0] = 1.0f;
        return true;
    }
    const int r = (int)ceil(3.0 * (double)sigma);
    if (r > kMaxFilterRadius) return false;
    double s = 0.0, w[2 * kMaxFilterRadius + 1];
    for (int k = -r; k <= r; ++k) s += (w[k + r] = exp(-(double)k * k / (2.0 * (double)sigma * sigma)));
    f->r = r;
    for (int k = 0; k <= 2 * r; ++k) f->t[k] = (float)(w[k] / s);
    return true;
}

// along x (dx = 1) or y (dx = 0), replicated borders; one thread per output
__global__ void blur_pass_kernel(const float *__restrict__ in, float *__restrict__ out, int n, int H, int W, int dx,
                                 FilterTaps f)
{
    const size_t plane = (size_t)H * W, total = (size_t)n * plane;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t img = idx / plane;
        const int rem = (int)(idx - img * plane), y = rem / W, x = rem - y * W;
        const float *p = in + img * plane;
        float acc = 0.0f;
        if (dx) {
            const float *row = p + (size_t)y * W;
            for (int k = -f.r; k <= f.r; ++k) acc = fmaf(f.t[k + f.r], __ldg(row + min(max(x + k, 0), W - 1)), acc);
        } else {
            for (int k = -f.r; k <= f.r; ++k)
                acc = fmaf(f.t[k + f.r], __ldg(p + (size_t)min(max(y + k, 0), H - 1) * W + x), acc);
        }
        out[idx] = acc;
    }
}

__global__ void sub_kernel(const float *a, const float *b, float *out, size_t total)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

// out = a / d (d per pixel, or the [H][W] plane d broadcast over images when bcast); |d| < 1e-12 -> 0
__global__ void div_kernel(const float *a, const float *d, float *out, size_t total, size_t plane, int bcast)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const float dv = d[bcast ? i % plane : i];
        out[i] = fabsf(dv) >= 1e-12f ? a[i] / dv : 0.0f;
    }
}

__global__ void mean_pattern_kernel(const float *__restrict__ in, int n, size_t plane, float *out)
{
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < plane; p += (size_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += in[(size_t)i * plane + p];
        out[p] = (float)(s / n);
    }
}

__device__ __forceinline__ void keys4(float t, float *wt)
{
    const float a = -0.5f;
    const float s0 = t + 1.0f, s1 = t, s2 = 1.0f - t, s3 = 2.0f - t;
    wt[0] = ((a * s0 - 5.0f * a) * s0 + 8.0f * a) * s0 - 4.0f * a;
    wt[1] = ((a + 2.0f) * s1 - (a + 3.0f)) * s1 * s1 + 1.0f;
    wt[2] = ((a + 2.0f) * s2 - (a + 3.0f)) * s2 * s2 + 1.0f;
    wt[3] = ((a * s3 - 5.0f * a) * s3 + 8.0f * a) * s3 - 4.0f * a;
}

// out(x) = in(pc + (x - pc - t) / s), index coordinates, Keys cubic, replicated borders
__global__ void shift_zoom_kernel(const float *__restrict__ in, int n, int H, int W, const float *__restrict__ shift,
                                  const float *__restrict__ zoom, float pcx, float pcy, float *__restrict__ out)
{
    const size_t plane = (size_t)H * W, total = (size_t)n * plane;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t img = idx / plane;
        const int rem = (int)(idx - img * plane), yo = rem / W, xo = rem - yo * W;
        const float tx = shift ? shift[img * 2] : 0.0f, ty = shift ? shift[img * 2 + 1] : 0.0f;
        const float s = zoom ? zoom[img] : 1.0f;
        const float x = pcx + ((float)xo - pcx - tx) / s, y = pcy + ((float)yo - pcy - ty) / s;
        const float fx0 = floorf(x), fy0 = floorf(y);
        const int x0 = (int)fx0, y0 = (int)fy0;
        float wx[4], wy[4];
        keys4(x - fx0, wx);
        keys4(y - fy0, wy);
        const float *M = in + img * plane;
        float acc = 0.0f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const float *row = M + (size_t)min(max(y0 - 1 + m, 0), H - 1) * W;
            float r = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) r = fmaf(wx[k], __ldg(row + min(max(x0 - 1 + k, 0), W - 1)), r);
            acc = fmaf(wy[m], r, acc);
        }
        out[idx] = acc;
    }
}

int grid_of(hrebsd_ctx *ctx, size_t total)
{
    size_t g = (total + 255) / 256, cap = (size_t)ctx->num_sms * 16;
    return (int)(g < cap ? (g ? g : 1) : cap);
}

// blur of n images into out via tmp (x pass into tmp, y pass into out)
int blur_into(hrebsd_ctx *ctx, const float *in, float *tmp, float *out, int n, int H, int W, const FilterTaps &f,
              cudaStream_t st)
{
    const size_t total = (size_t)n * H * W;
    blur_pass_kernel<<<grid_of(ctx, total), 256, 0, st>>>(in, tmp, n, H, W, 1, f);
    HR_LAUNCHED(ctx);
    blur_pass_kernel<<<grid_of(ctx, total), 256, 0, st>>>(tmp, out, n, H, W, 0, f);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

enum { WS_F0 = 16, WS_F1 = 17, WS_F2 = 18 };

}  // namespace

extern "C" int hrebsd_bandpass_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, float sigma_lp,
                                     float sigma_hp, float *out, void *stream)
{
    FilterTaps lp, hp;
    if (!ctx || n < 0 || H < 1 || W < 1 || !make_taps(sigma_lp, &lp) || !make_taps(sigma_hp, &hp))
        return HREBSD_EINVAL;
    if (n == 0) return HREBSD_OK;
    if (!in || !out) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    const size_t total = (size_t)n * H * W;
    void *t0, *t1, *t2;
    if ((e = hr_ws(ctx, WS_F0, total * 4, &t0)) || (e = hr_ws(ctx, WS_F1, total * 4, &t1)) ||
        (e = hr_ws(ctx, WS_F2, total * 4, &t2)))
        return e;
    cudaStream_t st = hr_stream(stream);
    hr_prof_begin(ctx, st);
    if ((e = blur_into(ctx, in, (float *)t0, (float *)t1, n, H, W, lp, st))) return e;   // t1 = low-pass
    if (hp.r > 0 || sigma_hp > 0.0f) {
        if ((e = blur_into(ctx, in, (float *)t0, (float *)t2, n, H, W, hp, st))) return e;   // t2 = G_hp * in
        sub_kernel<<<grid_of(ctx, total), 256, 0, st>>>((const float *)t1, (const float *)t2, out, total);
        HR_LAUNCHED(ctx);
    } else {
        HR_CHECK(cudaMemcpyAsync(out, t1, total * 4, cudaMemcpyDeviceToDevice, st));
    }
    hr_prof_end(ctx, PROF_PRE, st);
    return HREBSD_OK;
}

extern "C" int hrebsd_mean_pattern(hrebsd_ctx *ctx, const float *in, int n, int H, int W, float *out, void *stream)
{
    if (!ctx || n < 1 || H < 1 || W < 1 || !in || !out) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    cudaStream_t st = hr_stream(stream);
    hr_prof_begin(ctx, st);
    mean_pattern_kernel<<<grid_of(ctx, (size_t)H * W), 256, 0, st>>>(in, n, (size_t)H * W, out);
    hr_prof_end(ctx, PROF_PRE, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

extern "C" int hrebsd_background_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, const float *static_bg,
                                       float sigma_dyn, float *out, void *stream)
{
    FilterTaps f;
    if (!ctx || n < 0 || H < 1 || W < 1 || !make_taps(sigma_dyn, &f)) return HREBSD_EINVAL;
    if (n == 0) return HREBSD_OK;
    if (!in || !out) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    const size_t total = (size_t)n * H * W, plane = (size_t)H * W;
    void *t0, *t1, *t2;
    if ((e = hr_ws(ctx, WS_F0, total * 4, &t0)) || (e = hr_ws(ctx, WS_F1, total * 4, &t1)) ||
        (e = hr_ws(ctx, WS_F2, total * 4, &t2)))
        return e;
    cudaStream_t st = hr_stream(stream);
    hr_prof_begin(ctx, st);
    const float *cur = in;
    if (static_bg) {
        div_kernel<<<grid_of(ctx, total), 256, 0, st>>>(in, static_bg, (float *)t2, total, plane, 1);
        HR_LAUNCHED(ctx);
        cur = (const float *)t2;
    }
    if (sigma_dyn > 0.0f) {
        if ((e = blur_into(ctx, cur, (float *)t0, (float *)t1, n, H, W, f, st))) return e;
        div_kernel<<<grid_of(ctx, total), 256, 0, st>>>(cur, (const float *)t1, out, total, plane, 0);
        HR_LAUNCHED(ctx);
    } else if (cur != out) {
        HR_CHECK(cudaMemcpyAsync(out, cur, total * 4, cudaMemcpyDeviceToDevice, st));
    }
    hr_prof_end(ctx, PROF_PRE, st);
    return HREBSD_OK;
}

extern "C" int hrebsd_shift_zoom_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, const float *shift,
                                       const float *zoom, const hrebsd_geometry *g, float *out, void *stream)
{
    if (!ctx || !g || n < 0 || H < 1 || W < 1) return HREBSD_EINVAL;
    if (n == 0) return HREBSD_OK;
    if (!in || !out || in == out) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    const size_t total = (size_t)n * H * W;
    cudaStream_t st = hr_stream(stream);
    hr_prof_begin(ctx, st);
    shift_zoom_kernel<<<grid_of(ctx, total), 256, 0, st>>>(in, n, H, W, shift, zoom, (float)(g->xstar * W - 0.5),
                                                           (float)(g->ystar * H - 0.5), out);
    hr_prof_end(ctx, PROF_PRE, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}
