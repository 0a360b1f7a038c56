// Seeded synthetic Kikuchi patterns on the GPU (input generator only).
//
// Same recipe as synth/kikuchi.py: per pixel the sum of Gaussian band
// profiles exp(-theta^2/(2 theta_B^2)) over 25 planes, times a quadratic
// background, scaled to a mean of `counts`, then the Cornish-Fisher
// approximation of a Poisson draw from SplitMix64 counters.  The per-plane
// geometry (unit normal, Bragg angle, amplitude) comes from the host.  Band
// arithmetic is FP32 here and FP64 in numpy, so the two agree to rounding;
// the random counters are identical.
#include <cuda_runtime.h>
#include <stdint.h>

#define NPLANE 25

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t key, uint64_t ctr)
{
    return (double)(mix64(key + ctr * 0x632BE59BD9B4E019ull) >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void __launch_bounds__(512) kikuchi_kernel(const float *__restrict__ planes, const uint64_t *__restrict__ keys,
                                                      int H, int W, float xpc, float ypc, float zs, float counts,
                                                      int noise, int background, float *__restrict__ out)
{
    __shared__ float pl[NPLANE * 5];
    __shared__ double red[16];
    const int img = blockIdx.x;
    for (int i = threadIdx.x; i < NPLANE * 5; i += blockDim.x) pl[i] = planes[(size_t)img * NPLANE * 5 + i];
    __syncthreads();
    float *o = out + (size_t)img * H * W;
    double acc = 0.0;
    for (int p = threadIdx.x; p < H * W; p += blockDim.x) {
        const int i = p / W, j = p - i * W;
        float dx = (float)j + 0.5f - xpc, dy = (float)i + 0.5f - ypc;
        float inv = rsqrtf(dx * dx + dy * dy + zs * zs);
        float d0 = dx * inv, d1 = dy * inv, d2 = zs * inv;
        float bands = 0.0f;
#pragma unroll 5
        for (int k = 0; k < NPLANE; ++k) {
            const float *q = pl + 5 * k;
            float s = fminf(fmaxf(q[0] * d0 + q[1] * d1 + q[2] * d2, -1.0f), 1.0f);
            float th = asinf(s);
            bands += q[4] * __expf(-(th * th) / (2.0f * q[3] * q[3]));
        }
        float bg = 1.0f;
        if (background) {
            float xd = ((float)j + 0.5f) / W * 2.0f - 1.0f, yd = ((float)i + 0.5f) / H * 2.0f - 1.0f;
            bg = 1.0f - 0.3f * (xd * xd + yd * yd) + 0.05f * yd;
        }
        float v = bg * (1.0f + 0.5f * bands);
        o[p] = v;
        acc += v;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    const float scale = (float)((double)counts * H * W / tot);
    const uint64_t key = keys[img];
    for (int p = threadIdx.x; p < H * W; p += blockDim.x) {
        float lam = o[p] * scale;
        if (noise) {
            double u1 = 1.0 - uniform01(key, 2ull * p), u2 = uniform01(key, 2ull * p + 1);
            float z = (float)(sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
            lam = fmaxf(rintf(lam + sqrtf(lam) * z + (z * z - 1.0f) / 6.0f), 0.0f);
        }
        o[p] = lam;
    }
}

extern "C" int synth_kikuchi(const float *planes, const uint64_t *keys, int n, int H, int W, float xpc, float ypc,
                             float zs, float counts, int noise, int background, float *out, void *stream)
{
    if (n <= 0) return 0;
    kikuchi_kernel<<<n, 512, 0, (cudaStream_t)stream>>>(planes, keys, H, W, xpc, ypc, zs, counts, noise, background, out);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
