// a1: static background correction + normalisation, and the 2x2 pyramid.
//
// Section 2 normalises every pattern to zero mean before correlation and
// Section 3.3 corrects the background before registration.  One CTA owns one
// pattern: it reads it for the background moments, divides it by the fitted
// quadric once (float-float) writing the quotient less a constant to the
// output, then reads that back for the variance and the normalised output;
// the pattern (at most a few hundred KB) stays in L2 between the passes, so
// HBM sees about one read and one write per pixel.
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

// Unevaluated sums hi + lo of two FP32 values ("float-float", ~48 bits): the
// background quadric and the quotient pattern / quadric are evaluated in this
// precision, because the normalised output is a difference of two numbers near
// one divided by a standard deviation near 0.1, so plain FP32 would carry a
// smooth error pattern of ~10 units in the last place of the output.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_from_double(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

// exact sum of two floats (Knuth's two-sum)
__device__ __forceinline__ ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = two_sum(a.hi, b.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return two_sum(s.hi, lo);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);   // exact error of the product
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return two_sum(p, e);
}

// coordinate (2 k + 1 - n) / n in [-1, 1] of pixel k of n as hi + lo
__device__ __forceinline__ ff pixel_coord(int k, int n)
{
    const float num = (float)(2 * k + 1 - n), den = (float)n;   // exact integers
    const float h = __fdiv_rn(num, den);
    const float l = __fdiv_rn(__fmaf_rn(-h, den, num), den);   // the residual num - h n is exact
    return {h, l};
}

constexpr int kMaxDim = 1536;   // largest H and W of the background fit (per-row and per-column terms in shared memory)

__global__ void __launch_bounds__(kPreThreads) preprocess_kernel(const float *__restrict__ in, float *out, int H,
                                                                 int W, int flat, QuadricInverse qi)
{
    __shared__ double red[32 * 6];
    __shared__ double coef[6];
    __shared__ float2 rowA[kMaxDim], rowB[kMaxDim];   // per row: c0 + c2 y + c5 y^2 and c1 + c4 y (hi, lo)
    __shared__ float2 colX[kMaxDim];                  // per column: x (hi, lo)
    __shared__ float rowY[kMaxDim];                   // per row: y (the correctly rounded FP32 coordinate)
    const size_t base = (size_t)blockIdx.x * H * W;
    const float *img = in + base;
    const int n = H * W;

    // Sums are taken in FP32 over chunks of kChunk pixels of one thread and the chunk sums added in
    // FP64: the quadric's coefficients come out of a poorly conditioned 6 x 6 system, and plain FP32
    // sums of ~128 terms would move the output by ~1e-4.
    constexpr int kChunk = 8;
    if (flat) {   // the pixel coordinates, once per row and column
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            const ff x = pixel_coord(j, W);
            colX[j] = make_float2(x.hi, x.lo);
        }
        for (int i = threadIdx.x; i < H; i += blockDim.x) rowY[i] = pixel_coord(i, H).hi;
        __syncthreads();
    }
    // pass 1: quadric moments b_k = sum phi_k I (basis at the correctly rounded pixel coordinates);
    // b_0 is the pattern's sum
    double total = 0.0;
    if (flat) {
        double d[6] = {0, 0, 0, 0, 0, 0};
        for (int p0 = threadIdx.x; p0 < n; p0 += kChunk * blockDim.x) {
            float acc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                const int p = p0 + c * blockDim.x;
                if (p < n) {
                    const int i = p / W, j = p - i * W;
                    float phi[6];
                    basis6(colX[j].x, rowY[i], phi);
                    const float v = img[p];
#pragma unroll
                    for (int k = 0; k < 6; ++k) acc[k] = fmaf(phi[k], v, acc[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) d[k] += (double)acc[k];
        }
        block_sum<6>(d, red);
        total = d[0];
        if (threadIdx.x == 0) {
            for (int r = 0; r < 6; ++r) {
                double c = 0.0;
                for (int k = 0; k < 6; ++k) c += qi.ginv[r * 6 + k] * d[k];
                coef[r] = c;
            }
        }
        __syncthreads();
        // per-row parts of the quadric in FP64, kept as hi + lo
        for (int i = threadIdx.x; i < H; i += blockDim.x) {
            const double y = (2.0 * i + 1.0 - H) / H;
            const ff A = ff_from_double(coef[0] + y * (coef[2] + y * coef[5]));
            const ff Bc = ff_from_double(coef[1] + y * coef[4]);
            rowA[i] = make_float2(A.hi, A.lo);
            rowB[i] = make_float2(Bc.hi, Bc.lo);
        }
        __syncthreads();
    }
    const ff C = flat ? ff_from_double(coef[3]) : ff{0.0f, 0.0f};

    // the quadric at pixel p as hi + lo: A(y) + x (B(y) + x c3)
    auto fit_at = [&](int p) -> ff {
        const int i = p / W, j = p - i * W;
        const ff x = {colX[j].x, colX[j].y};
        const ff A = {rowA[i].x, rowA[i].y}, Bc = {rowB[i].x, rowB[i].y};
        return ff_add(A, ff_mul(x, ff_add(Bc, ff_mul(x, C))));
    };
    // the division is skipped when the fitted surface is not positive at every pixel (checked on the
    // FP32 value of the quadric, whose sign differs from the hi + lo one only within rounding of zero)
    bool use_fit = flat;
    if (flat) {
        bool bad = false;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int i = p / W, j = p - i * W;
            const float x = colX[j].x;
            bad |= !(fmaf(x, fmaf(x, C.hi, rowB[i].x), rowA[i].x) > 0.0f);
        }
        use_fit = !__syncthreads_or(bad);
    }

    // the pattern divided by the quadric, as hi + lo: q ~ v / f (within 2 units of the last place,
    // from the correctly rounded reciprocal), the remainder v - q f.hi exact by fma, then the
    // correction (remainder - q f.lo) / f; with the division by f.hi a product with the same
    // reciprocal (its error lands ~2^-24 below the correction, itself ~2^-24 below q)
    auto value = [&](int p) -> ff {
        const float v = img[p];
        if (!use_fit) return {v, 0.0f};
        const ff f = fit_at(p);
        const float rf = __frcp_rn(f.hi);
        const float q = __fmul_rn(v, rf);
        float r = __fmaf_rn(-q, f.hi, v);
        r = __fmaf_rn(-q, f.lo, r);
        return two_sum(q, __fmul_rn(r, rf));
    };
    // pass 2: the quotient less K (1 for the background-divided pattern, whose values lie near one;
    // the mean intensity, rounded, for the raw one), d = (q.hi - K) + q.lo in FP32: the leading part
    // cancels before rounding, so d keeps the float-float accuracy of q and the mean of d is small; d
    // is stored in the output (the pattern is read before it is overwritten, by the same thread) and
    // summed for the mean
    if (!flat) {   // the raw pattern's sum for K
        double t[1] = {0.0};
        for (int p0 = threadIdx.x; p0 < n; p0 += kChunk * blockDim.x) {
            float sv = 0.0f;
#pragma unroll
            for (int c = 0; c < kChunk; ++c) {
                const int p = p0 + c * blockDim.x;
                if (p < n) sv += img[p];
            }
            t[0] += (double)sv;
        }
        block_sum<1>(t, red);
        total = t[0];
    }
    const float K = use_fit ? 1.0f : (float)(total / n);
    float *o = out + base;
    double m[1] = {0.0};
    for (int p0 = threadIdx.x; p0 < n; p0 += kChunk * blockDim.x) {
        float sd = 0.0f;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
            const int p = p0 + c * blockDim.x;
            if (p < n) {
                const ff q = value(p);
                const float d = __fadd_rn(__fsub_rn(q.hi, K), q.lo);
                o[p] = d;
                sd += d;
            }
        }
        m[0] += (double)sd;
    }
    block_sum<1>(m, red);
    const double mean_d = m[0] / n, mean = mean_d + (double)K;
    const float md = (float)mean_d;
    // pass 3: variance about the mean
    double v2[1] = {0.0};
    for (int p0 = threadIdx.x; p0 < n; p0 += kChunk * blockDim.x) {
        float ss = 0.0f;
#pragma unroll
        for (int c = 0; c < kChunk; ++c) {
            const int p = p0 + c * blockDim.x;
            if (p < n) {
                const float d = __fsub_rn(o[p], md);
                ss = fmaf(d, d, ss);
            }
        }
        v2[0] += (double)ss;
    }
    block_sum<1>(v2, red);
    const double sdv = sqrt(v2[0] / n);
    const float inv = (sdv > 0.0 && sdv > 1e-6 * fabs(mean)) ? (float)(1.0 / sdv) : 0.0f;
    // pass 4: output
    for (int p = threadIdx.x; p < n; p += blockDim.x) o[p] = __fsub_rn(o[p], md) * inv;
}

// One pyramid level down: the 2x2 box mean, floor(H/2) x floor(W/2) (an odd
// last row or column takes no part).  VEC: H and W even, so every pair of
// neighbours starts on an 8-byte boundary and is read as one float2.
template <bool VEC>
__global__ void reduce2_kernel(const float *__restrict__ in, float *__restrict__ out, int n, int H, int W)
{
    const int h = H >> 1, w = W >> 1;
    const size_t total = (size_t)n * h * w;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        size_t img = idx / ((size_t)h * w);
        int rem = (int)(idx - img * h * w);
        int i = rem / w, j = rem - i * w;
        const float *p = in + img * H * W + (size_t)(2 * i) * W + 2 * j;
        float2 a, b;
        if (VEC) {
            a = *reinterpret_cast<const float2 *>(p);
            b = *reinterpret_cast<const float2 *>(p + W);
        } else {
            a = make_float2(p[0], p[1]);
            b = make_float2(p[W], p[W + 1]);
        }
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
    if (H % 2 == 0 && W % 2 == 0 && ((uintptr_t)in & 7) == 0)
        reduce2_kernel<true><<<blocks, 256, 0, st>>>(in, out, n, H, W);
    else
        reduce2_kernel<false><<<blocks, 256, 0, st>>>(in, out, n, H, W);
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
    if (flat && (H > kMaxDim || W > kMaxDim)) return HREBSD_EINVAL;
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
