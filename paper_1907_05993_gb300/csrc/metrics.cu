// Structural similarity of the demons-warped reference and the test pattern
// (Section 3.1, Fig. 3: SSIM is the quality measure of the demons-only
// method, which has no correlation peak).  SSIM of Wang et al. (2004) with an
// 11 x 11 Gaussian window of sigma 1.5 (normalised), C1 = (0.01 L)^2,
// C2 = (0.03 L)^2, L = max - min of the test pattern, averaged over the window
// centres whose window lies inside the image.  The warped reference is
// M(x - u(x)) with the clamped bilinear sampling of the registration.
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int R5 = 5, K11 = 2 * R5 + 1, T = 32, E = T + 2 * R5;   // window radius, tile of centres, tile + halo

__device__ __forceinline__ float bilinear_ref(const float *__restrict__ M, int h, int w, float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    const int x0 = min((int)x, w - 2), y0 = min((int)y, h - 2);
    const float fx = x - (float)x0, fy = y - (float)y0;
    const float *p = M + (size_t)y0 * w + x0;
    const float top = fmaf(fx, p[1], (1.0f - fx) * p[0]);
    const float bot = fmaf(fx, p[w + 1], (1.0f - fx) * p[w]);
    return fmaf(fy, bot, (1.0f - fy) * top);
}

// range L = max - min of each test pattern (one CTA per pair)
__global__ void range_kernel(const float *__restrict__ test, int HW, float *L)
{
    const float *t = test + (size_t)blockIdx.x * HW;
    float lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < HW; i += blockDim.x) {
        lo = fminf(lo, t[i]);
        hi = fmaxf(hi, t[i]);
    }
    __shared__ float slo[32], shi[32];
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        slo[threadIdx.x >> 5] = lo;
        shi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)blockDim.x / 32; ++k) {
            lo = fminf(lo, slo[k]);
            hi = fmaxf(hi, shi[k]);
        }
        L[blockIdx.x] = hi - lo;
    }
}

// One CTA per (pair, 32 x 32 tile of window centres).
__global__ void __launch_bounds__(256) ssim_tile_kernel(const float *__restrict__ ref, const int32_t *__restrict__ ref_idx,
                                                        const float *__restrict__ test, const float *__restrict__ field,
                                                        int H, int W, int tiles_x, const float *__restrict__ L,
                                                        double *sum)
{
    extern __shared__ float ssim_smem[];
    float(*sa)[E][E + 1] = reinterpret_cast<float(*)[E][E + 1]>(ssim_smem);                 // [5][E][E + 1]
    float(*sh)[E][T + 1] = reinterpret_cast<float(*)[E][T + 1]>(ssim_smem + 5 * E * (E + 1));   // [5][E][T + 1]
    __shared__ float g[K11];
    __shared__ double red[8];
    const int b = blockIdx.y, tid = threadIdx.x;
    const int cy0 = R5 + (blockIdx.x / tiles_x) * T, cx0 = R5 + (blockIdx.x % tiles_x) * T;
    const size_t plane = (size_t)H * W;
    const float *M = ref + (size_t)(ref_idx ? ref_idx[b] : 0) * plane;
    const float *Y = test + (size_t)b * plane;
    const float *ux = field ? field + (size_t)b * 2 * plane : nullptr;
    if (tid < K11) {
        const float d = (float)(tid - R5);
        g[tid] = expf(-d * d / (2.0f * 1.5f * 1.5f));
    }
    __syncthreads();
    if (tid == 0) {
        float s = 0.0f;
        for (int k = 0; k < K11; ++k) s += g[k];
        for (int k = 0; k < K11; ++k) g[k] /= s;
    }
    for (int i = tid; i < E * E; i += blockDim.x) {
        const int ly = i / E, lx = i - ly * E;
        const int gy = min(cy0 - R5 + ly, H - 1), gx = min(cx0 - R5 + lx, W - 1);
        const size_t o = (size_t)gy * W + gx;
        const float x = ux ? bilinear_ref(M, H, W, (float)gx - ux[o], (float)gy - ux[plane + o]) : M[o];
        const float y = Y[o];
        sa[0][ly][lx] = x;
        sa[1][ly][lx] = y;
        sa[2][ly][lx] = x * x;
        sa[3][ly][lx] = y * y;
        sa[4][ly][lx] = x * y;
    }
    __syncthreads();
    for (int i = tid; i < E * T; i += blockDim.x) {
        const int ly = i / T, lx = i - ly * T;
        float acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        for (int j = 0; j < K11; ++j)
            for (int k = 0; k < 5; ++k) acc[k] = fmaf(g[j], sa[k][ly][lx + j], acc[k]);
        for (int k = 0; k < 5; ++k) sh[k][ly][lx] = acc[k];
    }
    __syncthreads();
    const float Lb = L[b], C1 = (0.01f * Lb) * (0.01f * Lb), C2 = (0.03f * Lb) * (0.03f * Lb);
    double part = 0.0;
    for (int i = tid; i < T * T; i += blockDim.x) {
        const int ly = i / T, lx = i - ly * T;
        const int cy = cy0 + ly, cx = cx0 + lx;
        if (cy > H - 1 - R5 || cx > W - 1 - R5) continue;
        float m[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        for (int j = 0; j < K11; ++j)
            for (int k = 0; k < 5; ++k) m[k] = fmaf(g[j], sh[k][ly + j][lx], m[k]);
        const float mx = m[0], my = m[1];
        const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
        part += (double)(((2.0f * mx * my + C1) * (2.0f * sxy + C2)) /
                         ((mx * mx + my * my + C1) * (sxx + syy + C2)));
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)blockDim.x / 32; ++k) t += red[k];
        atomicAdd(sum + b, t);
    }
}

constexpr size_t kSsimSmem = sizeof(float) * 5 * (E * (E + 1) + E * (T + 1));

__global__ void ssim_finish_kernel(double *sum, int B, double count)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) sum[b] /= count;
}

}  // namespace

extern "C" int hrebsd_ssim_warped(hrebsd_ctx *ctx, const float *ref, const int32_t *ref_idx, const float *test,
                                  const float *field, int B, int H, int W, double *ssim, void *stream)
{
    if (!ctx || B < 0 || H < K11 || W < K11) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!ref || !test || !ssim) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    void *Lbuf = nullptr;
    if ((e = hr_ws(ctx, 14, (size_t)B * sizeof(float), &Lbuf))) return e;
    cudaStream_t st = hr_stream(stream);
    hr_prof_begin(ctx, st);
    HR_CHECK(cudaMemsetAsync(ssim, 0, (size_t)B * sizeof(double), st));
    range_kernel<<<B, 256, 0, st>>>(test, H * W, (float *)Lbuf);
    HR_LAUNCHED(ctx);
    const int tiles_x = (W - 2 * R5 + T - 1) / T, tiles_y = (H - 2 * R5 + T - 1) / T;
    static int configured = -1;
    if (configured != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(ssim_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSsimSmem));
        configured = ctx->device;
    }
    ssim_tile_kernel<<<dim3(tiles_x * tiles_y, B), 256, kSsimSmem, st>>>(ref, ref_idx, test, field, H, W, tiles_x,
                                                                        (const float *)Lbuf, ssim);
    HR_LAUNCHED(ctx);
    ssim_finish_kernel<<<(B + 255) / 256, 256, 0, st>>>(ssim, B, (double)(H - 2 * R5) * (W - 2 * R5));
    hr_prof_end(ctx, PROF_XCF, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}
