// a6: remap of the reference pattern by R_finite (Section 2, Eq. 12).
//
// Output pixel x' (test frame) looks up the reference at the gnomonic
// projection of R^T r', r' = (x' - xpc, y' - ypc, Z*): the reference point
// that Eq. 2 maps onto x' under the pure rotation R.  The value is a Keys
// (1981) cubic convolution (a = -0.5) over 4x4 reference pixels with
// replicated borders.  One thread per output pixel of a row; each CTA of a
// persistent grid walks an equal run of consecutive rows of all pairs; the
// references (a few grains) are gathered through the read-only path and stay
// in L2, so HBM traffic is the 4 B written per pixel.
#include "internal.cuh"

namespace {

__device__ __forceinline__ void keys_weights(float t, float *wt)
{
    // taps at offsets -1, 0, 1, 2 of the floor sample; t in [0, 1)
    const float a = -0.5f;
    const float s0 = t + 1.0f, s1 = t, s2 = 1.0f - t, s3 = 2.0f - t;
    wt[0] = ((a * s0 - 5.0f * a) * s0 + 8.0f * a) * s0 - 4.0f * a;
    wt[1] = ((a + 2.0f) * s1 - (a + 3.0f)) * s1 * s1 + 1.0f;
    wt[2] = ((a + 2.0f) * s2 - (a + 3.0f)) * s2 * s2 + 1.0f;
    wt[3] = ((a * s3 - 5.0f * a) * s3 + 8.0f * a) * s3 - 4.0f * a;
}

// A CTA walks a contiguous run of output rows (row = pair x H + i, all index
// arithmetic 32-bit), threads along the row; R^T of a pair is converted to
// FP32 registers once, when the run enters the pair.  Pixels whose 4 x 4
// footprint lies inside the reference read it without clamping; the others
// clamp every tap (the same values, since the clamp only acts outside).
__global__ void __launch_bounds__(256) remap_kernel(const float *__restrict__ ref, const int32_t *__restrict__ ref_idx,
                                                    const double *__restrict__ Rf, int B, int H, int W, float xpc,
                                                    float ypc, float zs, unsigned rows_per_cta, float *__restrict__ out)
{
    const unsigned total = (unsigned)B * (unsigned)H;
    const unsigned r0 = blockIdx.x * rows_per_cta;
    const unsigned r1 = min(total, r0 + rows_per_cta);
    const size_t plane = (size_t)H * W;
    int bcur = -1;
    float r[9];
    const float *M = ref;
    for (unsigned row = r0; row < r1; ++row) {
        const int b = (int)(row / (unsigned)H), i = (int)(row - (unsigned)b * H);
        if (b != bcur) {   // uniform across the CTA
            const double *R = Rf + (size_t)b * 9;
#pragma unroll
            for (int k = 0; k < 9; ++k) r[k] = (float)__ldg(R + k);
            M = ref + (size_t)__ldg(ref_idx + b) * plane;
            bcur = b;
        }
        float *orow = out + (size_t)b * plane + (size_t)i * W;
        const float dy = (float)i + 0.5f - ypc;
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            const float dx = (float)j + 0.5f - xpc;
            // v = R^T r'
            const float v0 = fmaf(r[0], dx, fmaf(r[3], dy, r[6] * zs));
            const float v1 = fmaf(r[1], dx, fmaf(r[4], dy, r[7] * zs));
            const float v2 = fmaf(r[2], dx, fmaf(r[5], dy, r[8] * zs));
            const float iv = zs / v2;
            const float x = fmaf(v0, iv, xpc - 0.5f), y = fmaf(v1, iv, ypc - 0.5f);
            const float fx0 = floorf(x), fy0 = floorf(y);
            const int x0 = (int)fx0, y0 = (int)fy0;
            float wx[4], wy[4];
            keys_weights(x - fx0, wx);
            keys_weights(y - fy0, wy);
            float acc = 0.0f;
            if (x0 >= 1 && x0 <= W - 3 && y0 >= 1 && y0 <= H - 3) {
                const float *p = M + (y0 - 1) * W + (x0 - 1);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    float rr = 0.0f;
#pragma unroll
                    for (int k = 0; k < 4; ++k) rr = fmaf(wx[k], __ldg(p + m * W + k), rr);
                    acc = fmaf(wy[m], rr, acc);
                }
            } else {
                int cx[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) cx[k] = min(max(x0 - 1 + k, 0), W - 1);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float *rowp = M + min(max(y0 - 1 + m, 0), H - 1) * W;
                    float rr = 0.0f;
#pragma unroll
                    for (int k = 0; k < 4; ++k) rr = fmaf(wx[k], __ldg(rowp + cx[k]), rr);
                    acc = fmaf(wy[m], rr, acc);
                }
            }
            orow[j] = acc;
        }
    }
}

}  // namespace

extern "C" int hrebsd_remap(hrebsd_ctx *ctx, const float *ref, const int32_t *ref_idx, const double *R_finite, int B,
                            int H, int W, const hrebsd_geometry *g, float *remapped, void *stream)
{
    if (!ctx || !g || B < 0 || H < 2 || W < 2) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!ref || !ref_idx || !R_finite || !remapped) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    const long long rows = (long long)B * H;
    if (rows > 0x7fffffffLL || (long long)H * W > 0x7fffffffLL) return HREBSD_EINVAL;
    const int threads = W >= 256 ? 256 : (W + 31) / 32 * 32;
    const long long cap = (long long)ctx->num_sms * (2048 / threads);   // resident CTAs
    hr_prof_begin(ctx, hr_stream(stream));
    const unsigned grid = (unsigned)(rows < cap ? rows : cap);
    const unsigned per = (unsigned)((rows + grid - 1) / grid);   // rows of one CTA's run
    remap_kernel<<<grid, threads, 0, hr_stream(stream)>>>(ref, ref_idx, R_finite, B, H, W, (float)(g->xstar * W),
                                                          (float)(g->ystar * H), (float)(g->zstar * W), per,
                                                          remapped);
    hr_prof_end(ctx, PROF_REMAP, hr_stream(stream));
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}
