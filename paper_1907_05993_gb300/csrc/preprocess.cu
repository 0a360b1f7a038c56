// a1: static background correction + normalisation, and the 2x2 pyramid.
//
// Section 2 normalises every pattern to zero mean before correlation and
// Section 3.3 corrects the background before registration.  One CTA owns one
// pattern and streams it four times (moments, mean, variance, output); the
// pattern (at most a few hundred KB) stays in L2 between the passes, so HBM
// sees one read and one write per pixel.
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int kPreThreads = 512;

struct QuadricInverse {
    double ginv[36];   // inverse Gram matrix of the basis {1, x, y, x^2, xy, y^2}
};

__device__ __forceinline__ void basis6(float x, float y, float *phi)
{
    phi[0] = 1.0f;
    phi[1] = x;
    phi[2] = y;
    phi[3] = x * x;
    phi[4] = x * y;
    phi[5] = y * y;
}

// Block-wide sum of `n` doubles per thread (n <= 6); result broadcast.
template <int NV>
__device__ void block_sum(double (&v)[NV], double *red /* [32][NV] */)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < NV; ++k) red[wid * NV + k] = v[k];
    __syncthreads();
    if (wid == 0) {
        for (int k = 0; k < NV; ++k) {
            double t = lane < nw ? red[lane * NV + k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) red[k] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = red[k];
    __syncthreads();
}

__global__ void __launch_bounds__(kPreThreads) preprocess_kernel(const float *__restrict__ in, float *out, int H,
                                                                 int W, int flat, QuadricInverse qi)
{
    __shared__ double red[32 * 6];
    __shared__ float coef[6];
    __shared__ int ok_flag;
    const size_t base = (size_t)blockIdx.x * H * W;
    const float *img = in + base;
    const int n = H * W;
    const float sx = 2.0f / W, sy = 2.0f / H;

    // Sums are taken in FP32 over chunks of kChunk pixels of one thread and the chunk sums added in
    // FP64: the quadric's coefficients come out of a poorly conditioned 6 x 6 system and the
    // normalised values are small differences of O(1) numbers, so plain FP32 sums of ~128 terms
    // would move the output by ~1e-4 (thousands of units in the last place).
    constexpr int kChunk = 8;
    // pass 1: quadric moments b_k = sum phi_k I
    if (flat) {
        double d[6] = {0, 0, 0, 0, 0, 0};
        for (int p0 = threadIdx.x; p0 < n; p0 += kChunk * blockDim.x) {
            float acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                const int p = p0 + c * blockDim.x;
                if (p < n) {
                    int i = p / W, j = p - i * W;
                    float phi[6];
                    basis6(fmaf((float)j + 0.5f, sx, -1.0f), fmaf((float)i + 0.5f, sy, -1.0f), phi);
                    float v = img[p];
#pragma unroll
                    for (int k = 0; k < 6; ++k) acc[k] = fmaf(phi[k], v, acc[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) d[k] += (double)acc[k];
        }
        block_sum<6>(d, red);
        if (threadIdx.x == 0) {
            for (int r = 0; r < 6; ++r) {
                double c = 0.0;
                for (int k = 0; k < 6; ++k) c += qi.ginv[r * 6 + k] * d[k];
                coef[r] = (float)c;
            }
            ok_flag = 1;
        }
        __syncthreads();
        // the division is skipped when the fitted surface is not positive everywhere
        int bad = 0;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            int i = p / W, j = p - i * W;
            float phi[6];
            basis6(fmaf((float)j + 0.5f, sx, -1.0f), fmaf((float)i + 0.5f, sy, -1.0f), phi);
            float fit = 0.0f;
#pragma unroll
            for (int k = 0; k < 6; ++k) fit = fmaf(coef[k], phi[k], fit);
            bad |= !(fit > 0.0f);
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) ok_flag = 0;
        __syncthreads();
    }
    const bool use_fit = flat && ok_flag;

    auto value = [&](int p) -> float {
        float v = img[p];
        if (use_fit) {
            int i = p / W, j = p - i * W;
            float phi[6];
            basis6(fmaf((float)j + 0.5f, sx, -1.0f), fmaf((float)i + 0.5f, sy, -1.0f), phi);
            float fit = 0.0f;
#pragma unroll
            for (int k = 0; k < 6; ++k) fit = fmaf(coef[k], phi[k], fit);
            v = v / fit;
        }
        return v;
    };

    // pass 2: mean
    double m[1] = {0.0};
    for (int p0 = threadIdx.x; p0 < n; p0 += kChunk * blockDim.x) {
        float s = 0.0f;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
            const int p = p0 + c * blockDim.x;
            if (p < n) s += value(p);
        }
        m[0] += (double)s;
    }
    block_sum<1>(m, red);
    const double mean = m[0] / n;
    // pass 3: variance about the mean; the mean as a pair hi + lo of FP32 values, so that the
    // subtraction from the quotient (both near 1, exact for the hi part) keeps the mean's precision
    double v2[1] = {0.0};
    const float meanf = (float)mean, meanlo = (float)(mean - (double)meanf);
    for (int p0 = threadIdx.x; p0 < n; p0 += kChunk * blockDim.x) {
        float ss = 0.0f;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
            const int p = p0 + c * blockDim.x;
            if (p < n) {
                float d = (value(p) - meanf) - meanlo;
                ss = fmaf(d, d, ss);
            }
        }
        v2[0] += (double)ss;
    }
    block_sum<1>(v2, red);
    const double sd = sqrt(v2[0] / n);
    const float inv = (sd > 0.0 && sd > 1e-6 * fabs(mean)) ? (float)(1.0 / sd) : 0.0f;
    // pass 4: output (in and out may alias: every pixel is read before it is written by the same thread)
    float *o = out + base;
    for (int p = threadIdx.x; p < n; p += blockDim.x) o[p] = ((value(p) - meanf) - meanlo) * inv;
}

__global__ void reduce2_kernel(const float *__restrict__ in, float *__restrict__ out, int n, int H, int W)
{
    const int h = H >> 1, w = W >> 1;
    const size_t total = (size_t)n * h * w;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        size_t img = idx / ((size_t)h * w);
        int rem = (int)(idx - img * h * w);
        int i = rem / w, j = rem - i * w;
        const float *p = in + img * H * W + (size_t)(2 * i) * W + 2 * j;
        float2 a = *reinterpret_cast<const float2 *>(p);
        float2 b = *reinterpret_cast<const float2 *>(p + W);
        out[idx] = 0.25f * ((a.x + a.y) + (b.x + b.y));
    }
}

int quadric_inverse(int H, int W, QuadricInverse *qi)
{
    double G[36] = {0};
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double x = (j + 0.5) / W * 2.0 - 1.0, y = (i + 0.5) / H * 2.0 - 1.0;
            double phi[6] = {1.0, x, y, x * x, x * y, y * y};
            for (int k = 0; k < 6; ++k)
                for (int l = 0; l < 6; ++l) G[k * 6 + l] += phi[k] * phi[l];
        }
    // Gauss-Jordan inversion with partial pivoting
    double A[6][12];
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 12; ++c) A[r][c] = c < 6 ? G[r * 6 + c] : (c - 6 == r);
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (fabs(A[piv][c]) < 1e-300) return -1;
        for (int k = 0; k < 12; ++k) {
            double t = A[c][k];
            A[c][k] = A[piv][k];
            A[piv][k] = t;
        }
        double d = A[c][c];
        for (int k = 0; k < 12; ++k) A[c][k] /= d;
        for (int r = 0; r < 6; ++r)
            if (r != c) {
                double f = A[r][c];
                for (int k = 0; k < 12; ++k) A[r][k] -= f * A[c][k];
            }
    }
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) qi->ginv[r * 6 + c] = A[r][c + 6];
    return 0;
}

}  // namespace

// Launch the 2x2 box-mean reduction of n images [n][H][W] -> [n][H/2][W/2].
int hr_launch_reduce2(hrebsd_ctx *ctx, const float *in, float *out, int n, int H, int W, cudaStream_t st)
{
    size_t total = (size_t)n * (H / 2) * (W / 2);
    if (total == 0) return HREBSD_OK;
    int blocks = (int)((total + 255) / 256);
    int cap = ctx->num_sms * 16;
    if (blocks > cap) blocks = cap;
    hr_prof_begin(ctx, st);
    reduce2_kernel<<<blocks, 256, 0, st>>>(in, out, n, H, W);
    hr_prof_end(ctx, PROF_DEMONS_AUX, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

extern "C" int hrebsd_preprocess_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, int flat, float *out,
                                       void *stream)
{
    if (!ctx || n < 0 || H < 2 || W < 2) return HREBSD_EINVAL;
    if (n == 0) return HREBSD_OK;
    if (!in || !out) return HREBSD_EINVAL;
    int st = hr_set_device(ctx);
    if (st) return st;
    QuadricInverse qi;
    if (flat && quadric_inverse(H, W, &qi)) return HREBSD_EINVAL;
    if (!flat)
        for (double &g : qi.ginv) g = 0.0;
    hr_prof_begin(ctx, hr_stream(stream));
    preprocess_kernel<<<n, kPreThreads, 0, hr_stream(stream)>>>(in, out, H, W, flat, qi);
    hr_prof_end(ctx, PROF_PRE, hr_stream(stream));
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

// Box mean of f x f blocks: [n][H][W] -> [n][H/f][W/f] (the pyramid level
// log2(f) in one pass; used to build the inputs and targets of the learned
// initialiser at the 64x64 level).
namespace {
__global__ void downsample_kernel(const float *__restrict__ in, float *__restrict__ out, int n, int H, int W, int f)
{
    const int h = H / f, w = W / f;
    const size_t total = (size_t)n * h * w;
    const float s = 1.0f / (float)(f * f);
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t img = idx / ((size_t)h * w);
        const int rem = (int)(idx - img * h * w), i = rem / w, j = rem - i * w;
        const float *p = in + img * H * W + (size_t)(i * f) * W + j * f;
        float acc = 0.0f;
        for (int a = 0; a < f; ++a)
            for (int b = 0; b < f; ++b) acc += p[(size_t)a * W + b];
        out[idx] = acc * s;
    }
}
}  // namespace

extern "C" int hrebsd_downsample_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, int f, float *out,
                                       void *stream)
{
    if (!ctx || n < 0 || f < 1 || H % f || W % f) return HREBSD_EINVAL;
    if (n == 0) return HREBSD_OK;
    if (!in || !out) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    size_t total = (size_t)n * (H / f) * (W / f);
    int grid = (int)((total + 255) / 256);
    if (grid > ctx->num_sms * 16) grid = ctx->num_sms * 16;
    hr_prof_begin(ctx, hr_stream(stream));
    downsample_kernel<<<grid, 256, 0, hr_stream(stream)>>>(in, out, n, H, W, f);
    hr_prof_end(ctx, PROF_PRE, hr_stream(stream));
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

// Displacement field between pyramid resolutions (learned initialiser): planar
// [B][2][h][w] -> [B][2][h2][w2], values rescaled to the new pixel unit.
// Shrinking by f: box mean of f x f blocks / f.  Growing by f: bilinear sample
// at x_c = (x_f + 0.5) / f - 0.5 (clamped to the image) times f, which for f = 2
// is the prolongation between registration levels (Section 1).
namespace {
__device__ __forceinline__ float bilinear_plane(const float *__restrict__ M, int h, int w, float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    const int x0 = min((int)x, max(w - 2, 0)), y0 = min((int)y, max(h - 2, 0));
    const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
    const float fx = x - (float)x0, fy = y - (float)y0;
    const float a = M[y0 * w + x0], b = M[y0 * w + x1], c = M[y1 * w + x0], d = M[y1 * w + x1];
    const float top = fmaf(fx, b, (1.0f - fx) * a), bot = fmaf(fx, d, (1.0f - fx) * c);
    return fmaf(fy, bot, (1.0f - fy) * top);
}

__global__ void field_resample_kernel(const float *__restrict__ in, int B, int h, int w, float *__restrict__ out,
                                      int h2, int w2)
{
    const size_t total = (size_t)B * 2 * h2 * w2;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t plane = idx / ((size_t)h2 * w2);   // b * 2 + component
        const int rem = (int)(idx - plane * h2 * w2), i = rem / w2, j = rem - i * w2;
        const float *src = in + plane * h * w;
        float v;
        if (h2 <= h) {
            const int f = h / h2;
            float acc = 0.0f;
            for (int a = 0; a < f; ++a)
                for (int b = 0; b < f; ++b) acc += src[(size_t)(i * f + a) * w + j * f + b];
            v = acc / (float)(f * f) / (float)f;
        } else {
            const int f = h2 / h;
            const float inv = 1.0f / (float)f;
            v = (float)f * bilinear_plane(src, h, w, ((float)j + 0.5f) * inv - 0.5f, ((float)i + 0.5f) * inv - 0.5f);
        }
        out[idx] = v;
    }
}

bool pow2_ratio(int a, int b)   // a = b * 2^k, k >= 0
{
    if (a < b || a % b) return false;
    const int r = a / b;
    return (r & (r - 1)) == 0;
}
}  // namespace

extern "C" int hrebsd_field_resample(hrebsd_ctx *ctx, const float *in, int B, int h, int w, float *out, int h2, int w2,
                                     void *stream)
{
    if (!ctx || B < 0 || h < 1 || w < 1 || h2 < 1 || w2 < 1) return HREBSD_EINVAL;
    const bool shrink = h2 <= h;
    if (shrink ? !(pow2_ratio(h, h2) && pow2_ratio(w, w2) && h / h2 == w / w2)
               : !(pow2_ratio(h2, h) && pow2_ratio(w2, w) && h2 / h == w2 / w))
        return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!in || !out) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    const size_t total = (size_t)B * 2 * h2 * w2;
    int grid = (int)((total + 255) / 256);
    if (grid > ctx->num_sms * 16) grid = ctx->num_sms * 16;
    hr_prof_begin(ctx, hr_stream(stream));
    field_resample_kernel<<<grid, 256, 0, hr_stream(stream)>>>(in, B, h, w, out, h2, w2);
    hr_prof_end(ctx, PROF_CNN, hr_stream(stream));
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}
