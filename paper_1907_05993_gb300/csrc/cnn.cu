// a10 (project addition, no counterpart in the paper): learned initialiser of
// the coarse demons field.  A 4-level U-Net (3x3 convolutions, 16-32-64-128
// channels, max-pool, nearest up-sampling, skip concatenations, 1x1 head)
// maps the 64x64 reference/test pair to the 2-channel field at that level.
// Training (MSE, Adam) and inference run on this library's kernels:
// implicit-GEMM convolutions on BF16 tensor cores with FP32 accumulation
// (cnn_kernels.cuh), and small element-wise kernels below.
#include <math.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <vector>

#include "cnn_kernels.cuh"
#include "cnn_tc.cuh"

#include "internal.cuh"

using namespace hr_cnn;

namespace {

constexpr int NCONV = 14;
struct LayerDef {
    int cin, cout, res;   // res: spatial size at batch-level 64
};
// forward order: e1a e1b e2a e2b e3a e3b ba bb d3a d3b d2a d2b d1a d1b
constexpr LayerDef kLayers[NCONV] = {{2, 16, 64},   {16, 16, 64},  {16, 32, 32}, {32, 32, 32}, {32, 64, 16},
                                     {64, 64, 16},  {64, 128, 8},  {128, 128, 8}, {192, 64, 16}, {64, 64, 16},
                                     {96, 32, 32},  {32, 32, 32},  {48, 16, 64}, {16, 16, 64}};
constexpr int HEAD_CIN = 16, HEAD_COUT = 2;

// Output channels per CTA of the TMA + tensor-memory convolution at an image
// size (the tiled weight copy is laid out for it).
int tma_bn(int res)
{
    return res >= 64 ? TmaGeom<64>::BN : res >= 32 ? TmaGeom<32>::BN : res >= 16 ? TmaGeom<16>::BN : TmaGeom<8>::BN;
}

__host__ __device__ inline int pad16(int c) { return (c + 15) / 16 * 16; }

// Grid of the per-image element-wise kernels: x covers `per` items of one
// image in blocks of 256, y walks the images.
dim3 grid2(int per, int N)
{
    return dim3((unsigned)((per + 255) / 256), (unsigned)(N < 65535 ? (N > 0 ? N : 1) : 65535));
}

// ------------------------------------------------------------------ element-wise kernels
// Input of the network from preprocessed patterns: box mean of f x f blocks
// (f = H / 64) of ref[ref_idx[b]] and test[b] -> NHWC BF16, channels (ref, test, 0...).
__device__ __forceinline__ void store_input_pixel(bf16 *o, float r, float t)
{
    __nv_bfloat162 v[8];
    v[0] = __floats2bfloat162_rn(r, t);
#pragma unroll
    for (int k = 1; k < 8; ++k) v[k] = __floats2bfloat162_rn(0.0f, 0.0f);
    uint4 *dst = reinterpret_cast<uint4 *>(o);
    dst[0] = *reinterpret_cast<const uint4 *>(&v[0]);
    dst[1] = *reinterpret_cast<const uint4 *>(&v[4]);
}

__global__ void pack_patterns_kernel(const float *ref, const float *test, const int32_t *ref_idx, int B, int H, int W,
                                     bf16 *x)
{
    const int f = H / 64;
    const float s = 1.0f / (float)(f * f);
    for (int b = blockIdx.y; b < B; b += gridDim.y)
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < 4096; p += gridDim.x * blockDim.x) {
            const int yy = p / 64, xx = p % 64;
            const float *r = ref + (size_t)ref_idx[b] * H * W, *t = test + (size_t)b * H * W;
            float sr = 0.0f, st = 0.0f;
            for (int dy = 0; dy < f; ++dy)
                for (int dx = 0; dx < f; ++dx) {
                    const size_t o = (size_t)(yy * f + dy) * W + xx * f + dx;
                    sr += r[o];
                    st += t[o];
                }
            store_input_pixel(x + ((size_t)b * 4096 + p) * 16, sr * s, st * s);
        }
}

// NCHW BF16 [B][2][64][64] -> NHWC BF16 padded to 16 channels.
__global__ void pack_nchw_kernel(const bf16 *in, int B, bf16 *x)
{
    for (int b = blockIdx.y; b < B; b += gridDim.y)
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < 4096; p += gridDim.x * blockDim.x) {
            const size_t i = (size_t)b * 8192 + p;
            store_input_pixel(x + ((size_t)b * 4096 + p) * 16, __bfloat162float(in[i]), __bfloat162float(in[i + 4096]));
        }
}

// 2x2 max-pool of NHWC BF16 (stride xs, offset xo, C channels, C and xs, xo
// multiples of 8) -> dense [N][h/2][w/2][C] plus the argmax (0..3, first
// maximum in row-major order of the 2x2 window).  One thread per 8 channels.
__global__ void maxpool_kernel(const bf16 *x, int xs, int xo, int C, int N, int H, int W, bf16 *y, uint8_t *arg)
{
    const int h = H / 2, w = W / 2, C8 = C / 8, per = h * w * C8;
    for (int n = blockIdx.y; n < N; n += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
            const int c8 = i % C8, q = i / C8, xx = q % w, yy = q / w;
            uint4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                v[k] = *reinterpret_cast<const uint4 *>(
                    x + ((size_t)(n * H + 2 * yy + k / 2) * W + 2 * xx + k % 2) * xs + xo + c8 * 8);
            uint4 out;
            uint8_t am[8];
            const bf16 *e0 = reinterpret_cast<const bf16 *>(&v[0]);
            bf16 *eo = reinterpret_cast<bf16 *>(&out);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float best = -INFINITY;
                int bi = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float t = __bfloat162float(e0[k * 8 + e]);
                    if (t > best) {
                        best = t;
                        bi = k;
                    }
                }
                eo[e] = __float2bfloat16_rn(best);
                am[e] = (uint8_t)bi;
            }
            const size_t o = ((size_t)n * h * w + q) * C + c8 * 8;
            *reinterpret_cast<uint4 *>(y + o) = out;
            *reinterpret_cast<uint2 *>(arg + o) = *reinterpret_cast<const uint2 *>(am);
        }
}

// d_in[p][c] (FP32, dense [N][H][W][C]) = routed dy from the pool + skip gradient (stride ss, offset so).
__global__ void maxpool_bwd_kernel(const float *dy, const uint8_t *arg, int C, int N, int H, int W, const float *skip,
                                   int ss, int so, float *dx)
{
    const size_t total = (size_t)N * H * W * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int xx = (int)(q % W), yy = (int)((q / W) % H), n = (int)(q / ((size_t)W * H));
        const size_t pi = ((size_t)(n * (H / 2) + yy / 2) * (W / 2) + xx / 2) * C + c;
        const int k = (yy & 1) * 2 + (xx & 1);
        float v = arg[pi] == k ? dy[pi] : 0.0f;
        if (skip) v += skip[q * ss + so + c];
        dx[i] = v;
    }
}

// Nearest up-sampling x2 of dense [N][h][w][C] BF16 into y (stride ys, offset
// yo; C, ys, yo multiples of 8).  One thread per 8 channels.
__global__ void up2_kernel(const bf16 *x, int C, int N, int h, int w, bf16 *y, int ys, int yo)
{
    const int H = 2 * h, W = 2 * w, C8 = C / 8, per = H * W * C8;
    for (int n = blockIdx.y; n < N; n += gridDim.y)
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
            const int c8 = i % C8, q = i / C8, xx = q % W, yy = q / W;
            const uint4 v = *reinterpret_cast<const uint4 *>(x + ((size_t)(n * h + yy / 2) * w + xx / 2) * C + c8 * 8);
            *reinterpret_cast<uint4 *>(y + ((size_t)n * H * W + q) * ys + yo + c8 * 8) = v;
        }
}

// Adjoint of up2: dx[N][h][w][C] = sum of the 4 children of dy (stride ys, offset yo).
__global__ void up2_bwd_kernel(const float *dy, int ys, int yo, int C, int N, int h, int w, float *dx)
{
    const int W = 2 * w;
    const size_t total = (size_t)N * h * w * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const size_t q = i / C;
        const int xx = (int)(q % w), yy = (int)((q / w) % h), n = (int)(q / ((size_t)w * h));
        float s = 0.0f;
        for (int k = 0; k < 4; ++k) s += dy[((size_t)(n * 2 * h + 2 * yy + k / 2) * W + 2 * xx + k % 2) * ys + yo + c];
        dx[i] = s;
    }
}

// dpre (BF16 dense [P][C]) = dpost (FP32, stride ds, offset do) * (out > 0), out BF16 (stride os, offset oo).
__global__ void relu_bwd_kernel(const float *dpost, int ds, int dof, const bf16 *out, int os, int oo, int C, size_t P,
                                bf16 *dpre)
{
    const size_t total = P * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i / C;
        const int c = (int)(i % C);
        const float g = __bfloat162float(out[p * os + oo + c]) > 0.0f ? dpost[p * ds + dof + c] : 0.0f;
        dpre[i] = __float2bfloat16_rn(g);
    }
}

// The ReLU backward, the bias gradient and the planar copies of the tcgen05 weight gradients in one
// pass: dpre[p][c] = BF16(dpost[p][c] if out[p][c] > 0 else 0) (dense [P][C]); db[c] += sum_p dpre[p][c];
// dk[c][q] = dpre[q + s_k][c] (s_k = +1, 0, -1; zero past the row ends).  A block walks tiles of 64
// pixels x 32 channels (with the two halo pixels; C, ds, dof, os and oo multiples of 8; P a multiple
// of 64), keeps its bias sums in registers and adds them to db once (few atomics per address).
__global__ void __launch_bounds__(256) relu_bwd_planar_kernel(const float *dpost, int ds, int dof, const bf16 *out,
                                                              int os, int oo, int C, int P, int res, bf16 *dpre,
                                                              bf16 *d0, bf16 *d1, bf16 *d2, float *db)
{
    __shared__ unsigned short tile[66][34];
    __shared__ float bsum[64][33];
    const int c0 = blockIdx.y * 32, t = threadIdx.x;
    float part[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // channels c0 + (t & 3) * 8 + j of this thread's centre pixels
    unsigned short *dk[3] = {reinterpret_cast<unsigned short *>(d0), reinterpret_cast<unsigned short *>(d1),
                             reinterpret_cast<unsigned short *>(d2)};
    for (int tq = blockIdx.x; tq < P / 64; tq += gridDim.x) {
        const int q0 = tq * 64;
        for (int i = t; i < 66 * 4; i += 256) {   // 66 pixels x 4 groups of 8 channels
            const int r = i >> 2, g = i & 3, q = q0 - 1 + r, c = c0 + g * 8;
            __align__(16) unsigned short h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (q >= 0 && q < P && c < C) {
                const uint4 ov = *reinterpret_cast<const uint4 *>(out + (size_t)q * os + oo + c);
                const float4 g0 = *reinterpret_cast<const float4 *>(dpost + (size_t)q * ds + dof + c);
                const float4 g1 = *reinterpret_cast<const float4 *>(dpost + (size_t)q * ds + dof + c + 4);
                const bf16 *ob = reinterpret_cast<const bf16 *>(&ov);
                const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const bf16 bv = __float2bfloat16_rn(__bfloat162float(ob[j]) > 0.0f ? gv[j] : 0.0f);
                    h[j] = *reinterpret_cast<const unsigned short *>(&bv);
                }
                if (r >= 1 && r <= 64) {   // a centre pixel: dpre and the bias sums
                    *reinterpret_cast<uint4 *>(dpre + (size_t)q * C + c) = *reinterpret_cast<const uint4 *>(h);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const unsigned short u = h[j];
                        part[j] += __bfloat162float(*reinterpret_cast<const bf16 *>(&u));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) tile[r][g * 8 + j] = h[j];
        }
        __syncthreads();
        for (int i = t; i < 3 * 32 * 8; i += 256) {   // (copy, channel, 8-pixel group)
            const int k = i / 256, c = (i >> 3) & 31, g = i & 7;
            if (c0 + c >= C) continue;
            const int sft = 1 - k;
            __align__(16) unsigned short h[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int jj = g * 8 + j, x = (q0 + jj) % res;
                h[j] = (x + sft >= 0 && x + sft < res) ? tile[jj + 1 + sft][c] : (unsigned short)0;
            }
            *reinterpret_cast<uint4 *>(dk[k] + (size_t)(c0 + c) * P + q0 + g * 8) = *reinterpret_cast<const uint4 *>(h);
        }
        __syncthreads();   // the tile is read before the next one is written
    }
    // a thread's centre pixels all lie in its channel group t & 3: reduce over the 64 threads of each group
#pragma unroll
    for (int j = 0; j < 8; ++j) bsum[t >> 2][(t & 3) * 8 + j] = part[j];
    __syncthreads();
    if (t < 32 && c0 + t < C) {
        float s = 0.0f;
        for (int k = 0; k < 64; ++k) s += bsum[k][t];
        atomicAdd(db + c0 + t, s);
    }
}

// db[o] += sum_p dpre[p][o]
__global__ void bias_grad_kernel(const bf16 *dpre, int C, size_t P, float *db)
{
    __shared__ float part[256];
    const int c = threadIdx.x % C, lane_rows = blockDim.x / C;
    float s = 0.0f;
    if ((int)threadIdx.x < lane_rows * C)
        for (size_t p = (size_t)blockIdx.x * lane_rows + threadIdx.x / C; p < P; p += (size_t)gridDim.x * lane_rows)
            s += __bfloat162float(dpre[p * C + c]);
    part[threadIdx.x] = s;
    __syncthreads();
    if ((int)threadIdx.x < C) {
        float t = 0.0f;
        for (int r = 0; r < lane_rows; ++r) t += part[r * C + threadIdx.x];
        atomicAdd(db + threadIdx.x, t);
    }
}

// 1x1 head: out[b][o][y][x] (FP32 planar) = bias[o] + sum_c w[o][c] d1[p][c]
__global__ void head_fwd_kernel(const bf16 *d1, const bf16 *w, const float *bias, int N, float *out)
{
    static_assert(HEAD_CIN == 16, "two 16-byte loads per pixel");
    for (int n = blockIdx.y; n < N; n += gridDim.y)
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < 4096; p += gridDim.x * blockDim.x) {
            const uint4 *src = reinterpret_cast<const uint4 *>(d1 + ((size_t)n * 4096 + p) * HEAD_CIN);
            uint4 v[2] = {src[0], src[1]};
            const bf16 *e = reinterpret_cast<const bf16 *>(v);
            float a0 = bias[0], a1 = bias[1];
#pragma unroll
            for (int c = 0; c < HEAD_CIN; ++c) {
                const float t = __bfloat162float(e[c]);
                a0 = fmaf(__bfloat162float(w[c]), t, a0);
                a1 = fmaf(__bfloat162float(w[HEAD_CIN + c]), t, a1);
            }
            out[(size_t)n * 8192 + p] = a0;
            out[(size_t)n * 8192 + 4096 + p] = a1;
        }
}

// MSE gradient and loss: dout = 2 (pred - target) / count; loss += sum d^2 / count.
__global__ void mse_kernel(const float *pred, const float *target, size_t count, float *dout, float *loss)
{
    __shared__ float red[256];
    float s = 0.0f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float d = pred[i] - target[i];
        dout[i] = 2.0f * d / (float)count;
        s = fmaf(d, d, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / (float)count);
}

// Head backward: dd1[p][c] = sum_o w[o][c] dout[o][p]; dw[o][c] += sum_p dout[o][p] d1[p][c]; db[o] += sum_p dout.
__global__ void head_bwd_kernel(const float *dout, const bf16 *d1, const bf16 *w, int N, float *dd1, float *dw,
                                float *db)
{
    __shared__ float red[256][HEAD_COUT * (HEAD_CIN + 1)];
    float acc[HEAD_COUT * (HEAD_CIN + 1)];
    for (int k = 0; k < HEAD_COUT * (HEAD_CIN + 1); ++k) acc[k] = 0.0f;
    const size_t total = (size_t)N * 4096;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / 4096, p = i % 4096;
        const float g0 = dout[b * 8192 + p], g1 = dout[b * 8192 + 4096 + p];
        for (int c = 0; c < HEAD_CIN; ++c) {
            const float v = __bfloat162float(d1[i * HEAD_CIN + c]);
            dd1[i * HEAD_CIN + c] = __bfloat162float(w[c]) * g0 + __bfloat162float(w[HEAD_CIN + c]) * g1;
            acc[c] = fmaf(g0, v, acc[c]);
            acc[HEAD_CIN + 1 + c] = fmaf(g1, v, acc[HEAD_CIN + 1 + c]);
        }
        acc[HEAD_CIN] += g0;
        acc[2 * HEAD_CIN + 1] += g1;
    }
    for (int k = 0; k < HEAD_COUT * (HEAD_CIN + 1); ++k) red[threadIdx.x][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < HEAD_COUT * (HEAD_CIN + 1)) {
        float s = 0.0f;
        for (int t = 0; t < (int)blockDim.x; ++t) s += red[t][threadIdx.x];
        const int o = threadIdx.x / (HEAD_CIN + 1), c = threadIdx.x % (HEAD_CIN + 1);
        if (c < HEAD_CIN) atomicAdd(dw + o * HEAD_CIN + c, s);
        else atomicAdd(db + o, s);
    }
}

// Adam (Kingma & Ba) on FP32 master weights, bias-corrected step size lr_t.
__global__ void adam_kernel(float *w, const float *g, float *m, float *v, size_t n, float lr_t, float b1, float b2,
                            float eps)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr_t * mi / (sqrtf(vi) + eps);
    }
}

// FP32 master weights are kept in the forward layout [co][tap][cinp] (channels
// padded to 16; the padded entries see zero inputs, so their gradients are zero
// and they stay at zero).  -> BF16 copy of the same layout, and the BF16
// input-gradient layout [ci][tap'][co] with tap' = 8 - tap (the flipped
// kernel with input and output channels exchanged); the tensor-memory tile
// layouts of the forward kernel (wt) and of the input-gradient kernel (wtd:
// output channel c, input channel o, tap 8 - tap; null where ci is not a
// multiple of its channel block).
__global__ void weights_to_bf16_kernel(const float *w, int ci, int co, int cinp, bf16 *wf, bf16 *wd, bf16 *wt, int bn,
                                       bf16 *wtd)
{
    const int total = co * 9 * cinp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c = i % cinp, tap = (i / cinp) % 9, o = i / (cinp * 9);
        const float v = c < ci ? w[i] : 0.0f;
        wf[i] = __float2bfloat16_rn(v);
        if (wd && c < ci) wd[((size_t)c * 9 + (8 - tap)) * co + o] = __float2bfloat16_rn(v);
        // tensor-memory path: [co / bn][cinp / 16][c % 16 / 8][tap][o % bn][c % 8]
        if (wt)
            wt[(((((size_t)(o / bn) * (cinp / 16) + c / 16) * 2 + (c % 16) / 8) * 9 + tap) * bn + o % bn) * 8 + c % 8] =
                __float2bfloat16_rn(v);
        if (wtd && c < ci)   // co is a multiple of 16
            wtd[(((((size_t)(c / bn) * (co / 16) + o / 16) * 2 + (o % 16) / 8) * 9 + (8 - tap)) * bn + c % bn) * 8 + o % 8] =
                __float2bfloat16_rn(v);
    }
}

__global__ void cast_bf16_kernel(const float *w, int n, bf16 *out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = __float2bfloat16_rn(w[i]);
}


int grid_for(hrebsd_ctx *ctx, size_t n)
{
    size_t g = (n + 255) / 256;
    size_t cap = (size_t)ctx->num_sms * 16;
    return (int)(g < cap ? (g ? g : 1) : cap);
}

}  // namespace

// ------------------------------------------------------------------ network object
struct hr_cnn_net {
    // parameters (FP32 master), gradients, Adam moments: one flat buffer each
    size_t n_params = 0;
    size_t w_off[NCONV + 1], b_off[NCONV + 1];   // index NCONV = head
    float *W = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    bf16 *wf[NCONV + 1] = {}, *wd[NCONV] = {}, *wt[NCONV] = {}, *wtd[NCONV] = {};
    int step = 0;
    // activations for a batch capacity
    int cap = 0;
    bf16 *x = nullptr;                              // [B][64][64][16]
    bf16 *act[NCONV] = {};                          // outputs (the ones not in concat buffers)
    bf16 *cat1 = nullptr, *cat2 = nullptr, *cat3 = nullptr;
    bf16 *pool[3] = {};
    uint8_t *parg[3] = {};
    float *out = nullptr, *dout = nullptr, *loss = nullptr;
    float *g_a = nullptr, *g_b = nullptr, *g_c = nullptr;   // FP32 gradient scratch (largest activation)
    float *g_cat = nullptr;                                 // FP32 gradient of a concat input
    bf16 *dpre = nullptr;
    bf16 *xT = nullptr, *dyS[3] = {};   // planar copies for the tcgen05 weight gradients
    std::vector<void *> allocs;
    size_t param_allocs = 0;   // allocations of the parameter block (kept when activations are regrown)
};

namespace {

int net_alloc(std::vector<void *> &allocs, size_t bytes, void **p)
{
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return HREBSD_ENOMEM;
    }
    allocs.push_back(*p);
    return HREBSD_OK;
}

void net_free_acts(hr_cnn_net *n)
{
    // activations are the allocations after the parameter block (its count recorded when it was made)
    const size_t keep = n->param_allocs;
    for (size_t i = keep; i < n->allocs.size(); ++i) cudaFree(n->allocs[i]);
    if (n->allocs.size() > keep) n->allocs.resize(keep);
    n->cap = 0;
}

int ensure_net(hrebsd_ctx *ctx)
{
    if (ctx->cnn) return HREBSD_OK;
    hr_cnn_net *n = new hr_cnn_net();
    size_t off = 0;
    for (int l = 0; l <= NCONV; ++l) {   // [co][9][cinp] + bias per conv, head [2][16] + bias
        const int co = l < NCONV ? kLayers[l].cout : HEAD_COUT;
        n->w_off[l] = off;
        off += l < NCONV ? (size_t)co * 9 * pad16(kLayers[l].cin) : (size_t)co * HEAD_CIN;
        n->b_off[l] = off;
        off += co;
    }
    n->n_params = off;
    int e;
    void *p;
    float **bufs[4] = {&n->W, &n->G, &n->M, &n->V};
    for (auto b : bufs) {
        if ((e = net_alloc(n->allocs, off * sizeof(float), &p))) { delete n; return e; }
        *b = (float *)p;
        HR_CHECK(cudaMemset(p, 0, off * sizeof(float)));
    }
    for (int l = 0; l <= NCONV; ++l) {
        const int ci = l < NCONV ? kLayers[l].cin : HEAD_CIN, co = l < NCONV ? kLayers[l].cout : HEAD_COUT;
        const size_t sz = l < NCONV ? (size_t)co * 9 * pad16(ci) : (size_t)co * ci;
        if ((e = net_alloc(n->allocs, sz * sizeof(bf16), &p))) { delete n; return e; }
        n->wf[l] = (bf16 *)p;
    }
    for (int l = 0; l < NCONV; ++l) {
        if ((e = net_alloc(n->allocs, (size_t)kLayers[l].cin * 9 * kLayers[l].cout * sizeof(bf16), &p))) { delete n; return e; }
        n->wd[l] = (bf16 *)p;
    }
    for (int l = 0; l < NCONV; ++l) {
        if ((e = net_alloc(n->allocs, (size_t)pad16(kLayers[l].cin) * 9 * kLayers[l].cout * sizeof(bf16), &p))) {
            delete n;
            return e;
        }
        n->wt[l] = (bf16 *)p;
    }
    for (int l = 1; l < NCONV; ++l) {   // the input gradients on tensor memory where the channel block divides ci
        if (kLayers[l].cin % tma_bn(kLayers[l].res)) continue;
        if ((e = net_alloc(n->allocs, (size_t)kLayers[l].cin * 9 * kLayers[l].cout * sizeof(bf16), &p))) {
            delete n;
            return e;
        }
        n->wtd[l] = (bf16 *)p;
    }
    n->param_allocs = n->allocs.size();
    ctx->cnn = n;
    return HREBSD_OK;
}

int ensure_acts(hrebsd_ctx *ctx, int B)
{
    hr_cnn_net *n = ctx->cnn;
    if (n->cap >= B) return HREBSD_OK;
    HR_CHECK(cudaDeviceSynchronize());
    net_free_acts(n);
    int e;
    void *p;
    const size_t px64 = (size_t)B * 4096;
#define NA(ptr, bytes)                                                        \
    do {                                                                      \
        if ((e = net_alloc(n->allocs, (bytes), &p))) return e;                \
        ptr = decltype(ptr)(p);                                               \
    } while (0)
    NA(n->x, px64 * 16 * sizeof(bf16));
    for (int l = 0; l < NCONV; ++l) {
        const size_t px = (size_t)B * kLayers[l].res * kLayers[l].res;
        NA(n->act[l], px * kLayers[l].cout * sizeof(bf16));
    }
    NA(n->cat1, px64 * 48 * sizeof(bf16));
    NA(n->cat2, px64 / 4 * 96 * sizeof(bf16));
    NA(n->cat3, px64 / 16 * 192 * sizeof(bf16));
    NA(n->pool[0], px64 / 4 * 16 * sizeof(bf16));
    NA(n->pool[1], px64 / 16 * 32 * sizeof(bf16));
    NA(n->pool[2], px64 / 64 * 64 * sizeof(bf16));
    NA(n->parg[0], px64 / 4 * 16);
    NA(n->parg[1], px64 / 16 * 32);
    NA(n->parg[2], px64 / 64 * 64);
    NA(n->out, px64 * 2 * sizeof(float));
    NA(n->dout, px64 * 2 * sizeof(float));
    NA(n->loss, sizeof(float));
    const size_t gmax = px64 * 48;   // largest activation (cat1) in elements
    NA(n->g_a, gmax * sizeof(float));
    NA(n->g_b, gmax * sizeof(float));
    NA(n->g_c, gmax * sizeof(float));
    NA(n->g_cat, gmax * sizeof(float));
    NA(n->dpre, gmax * sizeof(bf16));
    size_t xmax = 0, dmax = 0;   // the largest conv input (padded channels) and output, in elements
    for (int l = 0; l < NCONV; ++l) {
        const size_t px = (size_t)B * kLayers[l].res * kLayers[l].res;
        xmax = std::max(xmax, px * pad16(kLayers[l].cin));
        dmax = std::max(dmax, px * kLayers[l].cout);
    }
    NA(n->xT, xmax * sizeof(bf16));
    for (int k = 0; k < 3; ++k) NA(n->dyS[k], dmax * sizeof(bf16));
#undef NA
    n->cap = B;
    return HREBSD_OK;
}

int refresh_bf16(hrebsd_ctx *ctx, cudaStream_t st)
{
    hr_cnn_net *n = ctx->cnn;
    for (int l = 0; l < NCONV; ++l) {
        const int ci = kLayers[l].cin, co = kLayers[l].cout;
        weights_to_bf16_kernel<<<grid_for(ctx, (size_t)co * 9 * pad16(ci)), 256, 0, st>>>(
            n->W + n->w_off[l], ci, co, pad16(ci), n->wf[l], n->wd[l], n->wt[l], tma_bn(kLayers[l].res), n->wtd[l]);
        HR_LAUNCHED(ctx);
    }
    cast_bf16_kernel<<<1, 64, 0, st>>>(n->W + n->w_off[NCONV], HEAD_COUT * HEAD_CIN, n->wf[NCONV]);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

// One convolution launch.
// Persistent halo-tiled convolution when the shape has a variant (images of
// at least 16 x 16, cin <= 96 and the weights + two halos within 113 KB):
// returns 1 when there is none.
template <int CIN, int BN>
int launch_halo_t(hrebsd_ctx *ctx, const ConvArgs &a, cudaStream_t st)
{
    using G = HaloConv<CIN, BN>;
    static_assert(G::SMEM <= 113 * 1024, "halo variant too large");
    static int configured = -1, occ = 1;
    if (configured != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(conv3x3_halo_kernel<CIN, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)G::SMEM));
        HR_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv3x3_halo_kernel<CIN, BN>, 256, G::SMEM));
        if (occ < 1) occ = 1;
        configured = ctx->device;
    }
    const long long tiles = (long long)a.N * (a.H / G::TH) * (a.W / G::TW);
    const int cb = (a.cout + BN - 1) / BN;
    long long gx = (long long)ctx->num_sms * occ / cb;
    if (gx < 1) gx = 1;
    if (gx > tiles) gx = tiles;
    conv3x3_halo_kernel<CIN, BN><<<dim3((unsigned)gx, cb), 256, G::SMEM, st>>>(a);
    return HREBSD_OK;
}

// Halo tiles by TMA into tcgen05 MMAs (forward convolutions with BF16 output and
// the tiled weight copy).  Returns 1 when the shape is not covered.
template <int RES>
int launch_tma_t(hrebsd_ctx *ctx, const ConvArgs &a, const bf16 *wt, cudaStream_t st)
{
    using G = TmaGeom<RES>;
    constexpr int BN = G::BN;
    if (a.cout % BN || a.cout > 256) return 1;
    TmaConvArgs t;
    t.wt = wt;
    t.bias = a.bias;
    t.y = a.y_fp32 ? nullptr : reinterpret_cast<bf16 *>(a.y);
    t.yf = a.y_fp32 ? reinterpret_cast<float *>(a.y) : nullptr;
    t.ys = a.ys;
    t.yo = a.yo;
    t.relu = a.relu;
    t.cin = a.cin;
    t.cout = a.cout;
    t.N = a.N;
    // channels per box: the widest of 64, 32, 16 dividing cin that leaves room for 3 stages (else 2)
    t.cw = 0;
    for (int pass = 0; pass < 2 && !t.cw; ++pass) {
        for (int cw = 64; cw >= 16; cw /= 2) {
            if (a.cin % cw) continue;
            const size_t ab = ((size_t)G::PR * cw * 2 + 1023) / 1024 * 1024;
            const size_t st_b = (ab + (size_t)(cw / 16) * 9 * BN * 32 + 1023) / 1024 * 1024;
            if (st_b * (pass == 0 ? 3 : 2) <= 200 * 1024) {
                t.cw = cw;
                t.a_bytes = (int)ab;
                t.stage_bytes = (int)st_b;
                break;
            }
        }
    }
    if (!t.cw) return 1;
    t.nst = (int)((200 * 1024) / (size_t)t.stage_bytes);
    if (t.nst > 8) t.nst = 8;
    if (t.nst < 2) return 1;
    size_t smem = (size_t)t.nst * t.stage_bytes + 1024;   // + slack for 1024-byte alignment
    // at most 512 / TMEM CTAs per SM, so that tcgen05.alloc never waits
    const size_t cap = (size_t)(228 * 1024) / (size_t)(512 / G::TMEM + 1);
    if (smem + 2048 < cap) smem = cap - 2048 + 16;
    static int configured = -1;
    if (configured != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(conv3x3_tma_tc_kernel<RES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      210 * 1024));
        configured = ctx->device;
    }
    CUtensorMap tm;
    const uint64_t xs2 = (uint64_t)a.xs * 2;
    const uint64_t dims[4] = {(uint64_t)a.cin, (uint64_t)RES, (uint64_t)RES, (uint64_t)a.N};
    const uint64_t strides[3] = {xs2, xs2 * RES, xs2 * RES * RES};
    const uint32_t box[4] = {(uint32_t)t.cw, (uint32_t)G::Wp, (uint32_t)(G::Ht + 2), (uint32_t)G::TI};
    if (hr_encode_tmap_bf16_4d(&tm, a.x + a.xo, dims, strides, box, t.cw * 2)) {
        fprintf(stderr, "hrebsd: tensor map of a %dx%d x %d-channel convolution input refused\n", RES, RES, a.cin);
        return HREBSD_ECUDA;   // the tensor-memory path was asked for: no silent fallback
    }
    const long long tiles = (long long)((a.N + G::TI - 1) / G::TI) * (RES / G::Ht) * (a.cout / BN);
    if (tiles > 0x7fffffffLL) return 1;
    t.ntiles = (int)tiles;
    int per_sm = 512 / G::TMEM;
    const int by_smem = (int)((size_t)(228 * 1024) / (smem + 2048));
    if (by_smem < per_sm) per_sm = by_smem;
    const long long grid = tiles < (long long)ctx->num_sms * per_sm ? tiles : (long long)ctx->num_sms * per_sm;
    conv3x3_tma_tc_kernel<RES><<<(unsigned)grid, kTmaConvThreads, smem, st>>>(tm, t, ctx->d_err);
    return cudaGetLastError() == cudaSuccess ? HREBSD_OK : HREBSD_ECUDA;
}

int launch_tma_conv(hrebsd_ctx *ctx, const ConvArgs &a, const bf16 *wt, cudaStream_t st)
{
    if (!wt || !ctx->cnn_tc || a.H != a.W || a.N < 1 || a.cin % 16) return 1;
    if (a.xs % 8 || a.xo % 8 || a.ys % 8 || a.yo % 8) return 1;
    switch (a.H) {
    case 64: return launch_tma_t<64>(ctx, a, wt, st);
    case 32: return launch_tma_t<32>(ctx, a, wt, st);
    case 16: return launch_tma_t<16>(ctx, a, wt, st);
    case 8: return launch_tma_t<8>(ctx, a, wt, st);
    default: return 1;
    }
}

int launch_halo_conv(hrebsd_ctx *ctx, const ConvArgs &a, cudaStream_t st)
{
    if (a.H != a.W || a.H < 16 || a.H % 16 || a.N < 1) return 1;
    const int co = a.cout;
    const int bn = co % 64 == 0 ? 64 : (co % 32 == 0 ? 32 : (co % 16 == 0 ? 16 : 0));
    if (!bn) return 1;
#define HR_H(C, B) \
    if (a.cin == C && bn >= B) return launch_halo_t<C, B>(ctx, a, st)
    HR_H(16, 32);
    HR_H(16, 16);
    HR_H(32, 64);
    HR_H(32, 32);
    HR_H(32, 16);
    HR_H(48, 16);
    HR_H(64, 32);
    HR_H(64, 16);
    HR_H(96, 16);
#undef HR_H
    return 1;
}

int conv(hrebsd_ctx *ctx, const bf16 *x, int xs, int xo, int cin, const bf16 *w, const float *bias, int cout, void *y,
         int ys, int yo, int y_fp32, int relu, int N, int res, cudaStream_t st, const bf16 *wt = nullptr)
{
    ConvArgs a;
    a.x = x;
    a.xs = xs;
    a.xo = xo;
    a.cin = cin;
    a.w = w;
    a.bias = bias;
    a.cout = cout;
    a.y = y;
    a.ys = ys;
    a.yo = yo;
    a.y_fp32 = y_fp32;
    a.relu = relu;
    a.N = N;
    a.H = res;
    a.W = res;
    const int P = N * res * res;
    hr_prof_begin(ctx, st);
    int e = launch_tma_conv(ctx, a, wt, st);
    if (e == 1) e = launch_halo_conv(ctx, a, st);
    if (e == 1) {   // no halo variant for this shape: pipelined implicit GEMM
        // output-channel tile: the largest of 64, 32, 16 that divides cout
        const int bn = cout % 64 == 0 ? 64 : (cout % 32 == 0 ? 32 : 16);
        dim3 grid((P + 127) / 128, (cout + bn - 1) / bn);
#define HR_CONV(BN, KS)                                                                                           \
    do {                                                                                                          \
        constexpr size_t sm = conv_smem_bytes(BN, KS, 3);                                                         \
        static int configured = -1;                                                                              \
        if (configured != ctx->device) {                                                                          \
            HR_CHECK(cudaFuncSetAttribute(conv3x3_kernel<BN, KS, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                          (int)sm));                                                              \
            configured = ctx->device;                                                                             \
        }                                                                                                         \
        conv3x3_kernel<BN, KS, 3><<<grid, 256, sm, st>>>(a);                                                     \
    } while (0)
        if (bn == 64) HR_CONV(64, 2);
        else if (bn == 32) HR_CONV(32, 2);
        else HR_CONV(16, 4);
#undef HR_CONV
    } else if (e) {
        return e;
    }
    hr_prof_end(ctx, PROF_CNN, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

// Weight gradients on tcgen05 (planar copies, then the TMA-fed GEMM per tap); 1 = not applicable.
// dy_planar: n->dyS already holds dy's three shifted planar copies.
template <int NB>
int wgrad_tc_t(hrebsd_ctx *ctx, const bf16 *dy, int cout, const bf16 *x, int xs, int xo, int cin, float *dw, int N,
               int res, bool dy_planar, cudaStream_t st)
{
    hr_cnn_net *n = ctx->cnn;
    const int P = N * res * res;
    planar_shift_kernel<<<dim3((unsigned)((P + 63) / 64), (unsigned)((cin + 31) / 32)), 256, 0, st>>>(
        x, xs, xo, cin, P, res, nullptr, n->xT, nullptr);
    HR_LAUNCHED(ctx);
    if (!dy_planar) {
        planar_shift_kernel<<<dim3((unsigned)((P + 63) / 64), (unsigned)((cout + 31) / 32)), 256, 0, st>>>(
            dy, cout, 0, cout, P, res, n->dyS[0], n->dyS[1], n->dyS[2]);
        HR_LAUNCHED(ctx);
    }
    // planar [channel][image][pixel] as 4-D maps {pixels of an image, images, channels, 1}, 64-pixel boxes
    const uint64_t ip = (uint64_t)res * res * 2;
    const uint64_t dX[4] = {(uint64_t)res * res, (uint64_t)N, (uint64_t)cin, 1};
    const uint64_t sX[3] = {ip, (uint64_t)P * 2, (uint64_t)cin * P * 2};
    const uint32_t bX[4] = {64, 1, 128, 1};
    const uint64_t dD[4] = {(uint64_t)res * res, (uint64_t)N, (uint64_t)cout, 1};
    const uint64_t sD[3] = {ip, (uint64_t)P * 2, (uint64_t)cout * P * 2};
    const uint32_t bD[4] = {64, 1, (uint32_t)NB, 1};
    CUtensorMap tx, td[3];
    if (hr_encode_tmap_bf16_4d(&tx, n->xT, dX, sX, bX, 128)) return 1;
    for (int k = 0; k < 3; ++k)
        if (hr_encode_tmap_bf16_4d(&td[k], n->dyS[k], dD, sD, bD, 128)) return 1;
    WgradTcArgs a;
    a.dw = dw;
    a.cin = cin;
    a.cout = cout;
    a.res = res;
    a.ncb = (cin + 127) / 128;
    a.nob = cout / NB;
    a.ktiles = P / 64;
    const int items = a.ncb * a.nob;
    a.splits = ctx->num_sms / items;
    if (a.splits < 1) a.splits = 1;
    if (a.splits > a.ktiles) a.splits = a.ktiles;
    constexpr int STAGE = 128 * 128 + 9 * NB * 128;
    a.nst = (200 * 1024) / STAGE;
    if (a.nst > 8) a.nst = 8;
    const size_t smem = (size_t)a.nst * STAGE + 1024;   // + slack for 1024-byte alignment
    static int configured = -1;
    if (configured != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(conv3x3_wgrad_tc_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      210 * 1024));
        configured = ctx->device;
    }
    conv3x3_wgrad_tc_kernel<NB><<<(unsigned)(items * a.splits), kWgradThreads, smem, st>>>(tx, td[0], td[1], td[2], a,
                                                                                          ctx->d_err);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

bool wgrad_tc_ok(hrebsd_ctx *ctx, int cout, int res)
{
    return ctx->cnn_tc && ctx->cnn->xT && cout % 16 == 0 && (res == 8 || res == 16 || res == 32 || res == 64);
}

int wgrad(hrebsd_ctx *ctx, const bf16 *dy, int cout, const bf16 *x, int xs, int xo, int cin, float *dw, int N, int res,
          cudaStream_t st, bool dy_planar = false)
{
    hr_prof_begin(ctx, st);
    int e = 1;
    if (wgrad_tc_ok(ctx, cout, res))
        e = cout % 32 == 0 ? wgrad_tc_t<32>(ctx, dy, cout, x, xs, xo, cin, dw, N, res, dy_planar, st)
                           : wgrad_tc_t<16>(ctx, dy, cout, x, xs, xo, cin, dw, N, res, dy_planar, st);
    if (e == 1) {   // mma.sync over pixel chunks
        WgradArgs a;
        a.dy = dy;
        a.cout = cout;
        a.x = x;
        a.xs = xs;
        a.xo = xo;
        a.cin = cin;
        a.dw = dw;
        a.N = N;
        a.H = res;
        a.W = res;
        const int P = N * res * res;
        a.chunk = 2048;
        dim3 grid((P + a.chunk - 1) / a.chunk, 9 * ((cin + 63) / 64), (cout + 63) / 64);
        conv3x3_wgrad_kernel<<<grid, 128, 0, st>>>(a);
        HR_LAUNCHED(ctx);
    } else if (e) {
        return e;
    }
    hr_prof_end(ctx, PROF_CNN, st);
    return HREBSD_OK;
}

// Where each conv reads its input and writes its output: (buffer, channel stride, offset).
struct View {
    bf16 *p;
    int s, o;
};

void layer_views(hr_cnn_net *n, View *in, View *out)
{
    // e1a: x(16) -> act0 ; e1b: act0 -> cat1[32:48] ; e2a: pool0 -> act2 ; e2b: act2 -> cat2[64:96]
    // e3a: pool1 -> act4 ; e3b: act4 -> cat3[128:192] ; ba: pool2 -> act6 ; bb: act6 -> act7
    // d3a: cat3 -> act8 ; d3b: act8 -> act9 ; d2a: cat2 -> act10 ; d2b -> act11 ; d1a: cat1 -> act12 ; d1b -> act13
    in[0] = {n->x, 16, 0};
    out[0] = {n->act[0], 16, 0};
    in[1] = {n->act[0], 16, 0};
    out[1] = {n->cat1, 48, 32};
    in[2] = {n->pool[0], 16, 0};
    out[2] = {n->act[2], 32, 0};
    in[3] = {n->act[2], 32, 0};
    out[3] = {n->cat2, 96, 64};
    in[4] = {n->pool[1], 32, 0};
    out[4] = {n->act[4], 64, 0};
    in[5] = {n->act[4], 64, 0};
    out[5] = {n->cat3, 192, 128};
    in[6] = {n->pool[2], 64, 0};
    out[6] = {n->act[6], 128, 0};
    in[7] = {n->act[6], 128, 0};
    out[7] = {n->act[7], 128, 0};
    in[8] = {n->cat3, 192, 0};
    out[8] = {n->act[8], 64, 0};
    in[9] = {n->act[8], 64, 0};
    out[9] = {n->act[9], 64, 0};
    in[10] = {n->cat2, 96, 0};
    out[10] = {n->act[10], 32, 0};
    in[11] = {n->act[10], 32, 0};
    out[11] = {n->act[11], 32, 0};
    in[12] = {n->cat1, 48, 0};
    out[12] = {n->act[12], 16, 0};
    in[13] = {n->act[12], 16, 0};
    out[13] = {n->act[13], 16, 0};
}

int forward(hrebsd_ctx *ctx, int B, cudaStream_t st)
{
    hr_cnn_net *n = ctx->cnn;
    View in[NCONV], out[NCONV];
    layer_views(n, in, out);
    int e;
    auto run = [&](int l) {
        return conv(ctx, in[l].p, in[l].s, in[l].o, pad16(kLayers[l].cin), n->wf[l], n->W + n->b_off[l],
                    kLayers[l].cout, out[l].p, out[l].s, out[l].o, 0, 1, B, kLayers[l].res, st, n->wt[l]);
    };
    auto pool = [&](int k, const View &v, int C, int res) {
        maxpool_kernel<<<grid2(res * res / 4 * C / 8, B), 256, 0, st>>>(v.p, v.s, v.o, C, B, res, res, n->pool[k],
                                                                       n->parg[k]);
        return cudaGetLastError() == cudaSuccess ? (ctx->launches++, HREBSD_OK) : HREBSD_ECUDA;
    };
    auto up = [&](const bf16 *src, int C, int res, bf16 *dst, int ds) {
        up2_kernel<<<grid2(res * res * 4 * C / 8, B), 256, 0, st>>>(src, C, B, res, res, dst, ds, 0);
        return cudaGetLastError() == cudaSuccess ? (ctx->launches++, HREBSD_OK) : HREBSD_ECUDA;
    };
    if ((e = run(0)) || (e = run(1)) || (e = pool(0, out[1], 16, 64))) return e;
    if ((e = run(2)) || (e = run(3)) || (e = pool(1, out[3], 32, 32))) return e;
    if ((e = run(4)) || (e = run(5)) || (e = pool(2, out[5], 64, 16))) return e;
    if ((e = run(6)) || (e = run(7)) || (e = up(n->act[7], 128, 8, n->cat3, 192))) return e;
    if ((e = run(8)) || (e = run(9)) || (e = up(n->act[9], 64, 16, n->cat2, 96))) return e;
    if ((e = run(10)) || (e = run(11)) || (e = up(n->act[11], 32, 32, n->cat1, 48))) return e;
    if ((e = run(12)) || (e = run(13))) return e;
    hr_prof_begin(ctx, st);
    head_fwd_kernel<<<grid2(4096, B), 256, 0, st>>>(n->act[13], n->wf[NCONV], n->W + n->b_off[NCONV], B, n->out);
    hr_prof_end(ctx, PROF_CNN, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

// Backward of conv l given the FP32 gradient of its post-ReLU output (dpost,
// stride ds, offset do): weight and bias gradients, and (if dx != null) the FP32
// gradient of its input written dense with the input's channel count.
int conv_bwd(hrebsd_ctx *ctx, int l, const float *dpost, int ds, int dof, float *dx, int B, cudaStream_t st)
{
    hr_cnn_net *n = ctx->cnn;
    View in[NCONV], out[NCONV];
    layer_views(n, in, out);
    const LayerDef &L = kLayers[l];
    const size_t P = (size_t)B * L.res * L.res;
    int e;
    if (wgrad_tc_ok(ctx, L.cout, L.res)) {   // ReLU backward, bias gradient and dy's planar copies in one pass
        const size_t tiles = P / 64, cap = (size_t)ctx->num_sms * 4;
        relu_bwd_planar_kernel<<<dim3((unsigned)(tiles < cap ? tiles : cap), (unsigned)((L.cout + 31) / 32)), 256, 0,
                                 st>>>(
            dpost, ds, dof, out[l].p, out[l].s, out[l].o, L.cout, (int)P, L.res, n->dpre, n->dyS[0], n->dyS[1],
            n->dyS[2], n->G + n->b_off[l]);
        HR_LAUNCHED(ctx);
        if ((e = wgrad(ctx, n->dpre, L.cout, in[l].p, in[l].s, in[l].o, pad16(L.cin), n->G + n->w_off[l], B, L.res,
                       st, true)))
            return e;
    } else {
        relu_bwd_kernel<<<grid_for(ctx, P * L.cout), 256, 0, st>>>(dpost, ds, dof, out[l].p, out[l].s, out[l].o,
                                                                  L.cout, P, n->dpre);
        HR_LAUNCHED(ctx);
        if ((e = wgrad(ctx, n->dpre, L.cout, in[l].p, in[l].s, in[l].o, pad16(L.cin), n->G + n->w_off[l], B, L.res,
                       st)))
            return e;
        bias_grad_kernel<<<grid_for(ctx, P), 256, 0, st>>>(n->dpre, L.cout, P, n->G + n->b_off[l]);
        HR_LAUNCHED(ctx);
    }
    if (dx)
        return conv(ctx, n->dpre, L.cout, 0, L.cout, n->wd[l], nullptr, L.cin, dx, L.cin, 0, 1, 0, B, L.res, st,
                    n->wtd[l]);
    return HREBSD_OK;
}

int backward(hrebsd_ctx *ctx, int B, cudaStream_t st)
{
    hr_cnn_net *n = ctx->cnn;
    int e;
    float *dd = n->g_a;   // gradient of d1b's output [B*4096][16]
    hr_prof_begin(ctx, st);
    head_bwd_kernel<<<grid_for(ctx, (size_t)B * 4096), 256, 0, st>>>(n->dout, n->act[13], n->wf[NCONV], B, dd,
                                                                     n->G + n->w_off[NCONV], n->G + n->b_off[NCONV]);
    hr_prof_end(ctx, PROF_CNN, st);
    HR_LAUNCHED(ctx);
    const size_t p64 = (size_t)B * 4096, p32 = p64 / 4, p16 = p64 / 16;
    auto ub = [&](const float *src, int ss, int C, int res, float *dst) {   // res: coarse size
        up2_bwd_kernel<<<grid_for(ctx, (size_t)B * res * res * C), 256, 0, st>>>(src, ss, 0, C, B, res, res, dst);
        return cudaGetLastError() == cudaSuccess ? (ctx->launches++, HREBSD_OK) : HREBSD_ECUDA;
    };
    auto pb = [&](int k, const float *dp, int C, int res, const float *skip, int ss, int so, float *dst) {
        maxpool_bwd_kernel<<<grid_for(ctx, (size_t)B * res * res * C), 256, 0, st>>>(dp, n->parg[k], C, B, res, res,
                                                                                    skip, ss, so, dst);
        return cudaGetLastError() == cudaSuccess ? (ctx->launches++, HREBSD_OK) : HREBSD_ECUDA;
    };
    // decoder level 1 (64x64)
    if ((e = conv_bwd(ctx, 13, dd, 16, 0, n->g_b, B, st))) return e;               // -> d d1a.out
    if ((e = conv_bwd(ctx, 12, n->g_b, 16, 0, n->g_cat, B, st))) return e;         // -> d cat1 [32|16]
    if ((e = ub(n->g_cat, 48, 32, 32, n->g_a))) return e;                          // -> d d2b.out [p32][32]
    // keep d e1 (skip part of cat1) in g_cat (channels 32..47, stride 48)
    if ((e = conv_bwd(ctx, 11, n->g_a, 32, 0, n->g_b, B, st))) return e;           // -> d d2a.out
    float *dcat2 = n->g_c;
    if ((e = conv_bwd(ctx, 10, n->g_b, 32, 0, dcat2, B, st))) return e;            // -> d cat2 [64|32]
    if ((e = ub(dcat2, 96, 64, 16, n->g_a))) return e;                             // -> d d3b.out [p16][64]
    if ((e = conv_bwd(ctx, 9, n->g_a, 64, 0, n->g_b, B, st))) return e;            // -> d d3a.out
    float *dcat3 = n->dout + 0;   // reuse? no: dout is needed only before; use a slice of g_a after
    dcat3 = n->g_a + p16 * 64;    // g_a holds d d3b.out in its first p16*64 floats
    if ((e = conv_bwd(ctx, 8, n->g_b, 64, 0, dcat3, B, st))) return e;             // -> d cat3 [128|64]
    if ((e = ub(dcat3, 192, 128, 8, n->g_b))) return e;                            // -> d bb.out [p8][128]
    float *t1 = n->g_b + p16 / 4 * 128;
    if ((e = conv_bwd(ctx, 7, n->g_b, 128, 0, t1, B, st))) return e;              // -> d ba.out
    float *t2 = t1 + p16 / 4 * 128;
    if ((e = conv_bwd(ctx, 6, t1, 128, 0, t2, B, st))) return e;                   // -> d pool2 [p8][64]
    float *de3 = t2 + p16 / 4 * 64;
    if ((e = pb(2, t2, 64, 16, dcat3, 192, 128, de3))) return e;                   // d e3b.out = pool + skip
    float *t3 = de3 + p16 * 64;
    if ((e = conv_bwd(ctx, 5, de3, 64, 0, t3, B, st))) return e;                   // -> d e3a.out
    float *t4 = t3 + p16 * 64;
    if ((e = conv_bwd(ctx, 4, t3, 64, 0, t4, B, st))) return e;                    // -> d pool1 [p16][32]
    float *de2 = n->g_c + p32 * 96;   // g_c holds dcat2 [p32][96] first
    if ((e = pb(1, t4, 32, 32, dcat2, 96, 64, de2))) return e;                     // d e2b.out
    float *t5 = de2 + p32 * 32;
    if ((e = conv_bwd(ctx, 3, de2, 32, 0, t5, B, st))) return e;                   // -> d e2a.out
    float *t6 = t5 + p32 * 32;
    if ((e = conv_bwd(ctx, 2, t5, 32, 0, t6, B, st))) return e;                    // -> d pool0 [p32][16]
    float *de1 = n->g_a;   // free now
    if ((e = pb(0, t6, 16, 64, n->g_cat, 48, 32, de1))) return e;                  // d e1b.out
    if ((e = conv_bwd(ctx, 1, de1, 16, 0, n->g_b, B, st))) return e;               // -> d e1a.out
    if ((e = conv_bwd(ctx, 0, n->g_b, 16, 0, nullptr, B, st))) return e;
    (void)p64;
    return HREBSD_OK;
}

}  // namespace

// ------------------------------------------------------------------ ABI
extern "C" int hrebsd_cnn_init(hrebsd_ctx *ctx, const float *params_host, long long n_params)
{
    if (!ctx) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e || (e = ensure_net(ctx))) return e;
    hr_cnn_net *n = ctx->cnn;
    if (params_host) {
        if (n_params != (long long)n->n_params) return HREBSD_EINVAL;
        HR_CHECK(cudaMemcpy(n->W, params_host, n->n_params * sizeof(float), cudaMemcpyHostToDevice));
    }
    HR_CHECK(cudaMemset(n->M, 0, n->n_params * sizeof(float)));
    HR_CHECK(cudaMemset(n->V, 0, n->n_params * sizeof(float)));
    n->step = 0;
    if ((e = refresh_bf16(ctx, 0))) return e;
    HR_CHECK(cudaDeviceSynchronize());
    return HREBSD_OK;
}

extern "C" long long hrebsd_cnn_num_params(hrebsd_ctx *ctx)
{
    if (!ctx) return -1;
    if (hr_set_device(ctx) || ensure_net(ctx)) return -1;
    return (long long)ctx->cnn->n_params;
}

extern "C" int hrebsd_cnn_get_params(hrebsd_ctx *ctx, float *params_host, float *grads_host)
{
    if (!ctx || !ctx->cnn) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    HR_CHECK(cudaDeviceSynchronize());
    if (params_host) HR_CHECK(cudaMemcpy(params_host, ctx->cnn->W, ctx->cnn->n_params * 4, cudaMemcpyDeviceToHost));
    if (grads_host) HR_CHECK(cudaMemcpy(grads_host, ctx->cnn->G, ctx->cnn->n_params * 4, cudaMemcpyDeviceToHost));
    return HREBSD_OK;
}

extern "C" int hrebsd_cnn_get_state(hrebsd_ctx *ctx, float *m_host, float *v_host, int *step)
{
    if (!ctx || !ctx->cnn) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    HR_CHECK(cudaDeviceSynchronize());
    if (m_host) HR_CHECK(cudaMemcpy(m_host, ctx->cnn->M, ctx->cnn->n_params * 4, cudaMemcpyDeviceToHost));
    if (v_host) HR_CHECK(cudaMemcpy(v_host, ctx->cnn->V, ctx->cnn->n_params * 4, cudaMemcpyDeviceToHost));
    if (step) *step = ctx->cnn->step;
    return HREBSD_OK;
}

extern "C" int hrebsd_cnn_set_state(hrebsd_ctx *ctx, const float *m_host, const float *v_host, int step)
{
    if (!ctx || !m_host || !v_host || step < 0) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e || (e = ensure_net(ctx))) return e;
    HR_CHECK(cudaDeviceSynchronize());
    HR_CHECK(cudaMemcpy(ctx->cnn->M, m_host, ctx->cnn->n_params * 4, cudaMemcpyHostToDevice));
    HR_CHECK(cudaMemcpy(ctx->cnn->V, v_host, ctx->cnn->n_params * 4, cudaMemcpyHostToDevice));
    ctx->cnn->step = step;
    return HREBSD_OK;
}

// Model file of the learned initialiser (project format, little-endian):
//   bytes 0-7   magic "HRCNN001"
//   8-15        int64 number of parameters n
//   16-23       int64 Adam step count
//   then        float32 parameters [n], Adam first moments [n], second moments [n]
//   last 8      uint64 FNV-1a hash of every byte before it
// The hash makes a truncated or damaged file fail to load instead of loading
// wrong weights.  The file is written under a temporary name and renamed, so
// an interrupted save leaves an earlier file of that name intact.
namespace {

constexpr char kCnnMagic[8] = {'H', 'R', 'C', 'N', 'N', '0', '0', '1'};

uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h)
{
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ull;

}  // namespace

extern "C" int hrebsd_cnn_save(hrebsd_ctx *ctx, const char *path)
{
    if (!ctx || !ctx->cnn || !path || !*path) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    const hr_cnn_net *n = ctx->cnn;
    const size_t np = n->n_params, body = 24 + 3 * np * 4;
    std::vector<unsigned char> buf(body + 8);
    memcpy(buf.data(), kCnnMagic, 8);
    const int64_t hdr[2] = {(int64_t)np, (int64_t)n->step};
    memcpy(buf.data() + 8, hdr, 16);
    HR_CHECK(cudaDeviceSynchronize());
    HR_CHECK(cudaMemcpy(buf.data() + 24, n->W, np * 4, cudaMemcpyDeviceToHost));
    HR_CHECK(cudaMemcpy(buf.data() + 24 + np * 4, n->M, np * 4, cudaMemcpyDeviceToHost));
    HR_CHECK(cudaMemcpy(buf.data() + 24 + 2 * np * 4, n->V, np * 4, cudaMemcpyDeviceToHost));
    const uint64_t h = fnv1a(buf.data(), body, kFnvBasis);
    memcpy(buf.data() + body, &h, 8);
    std::vector<char> tmp(strlen(path) + 32);
    snprintf(tmp.data(), tmp.size(), "%s.tmp%ld", path, (long)getpid());
    FILE *f = fopen(tmp.data(), "wb");
    if (!f) return HREBSD_EIO;
    const bool ok = fwrite(buf.data(), 1, buf.size(), f) == buf.size();
    if (fclose(f) != 0 || !ok || rename(tmp.data(), path) != 0) {
        remove(tmp.data());
        return HREBSD_EIO;
    }
    return HREBSD_OK;
}

extern "C" int hrebsd_cnn_load(hrebsd_ctx *ctx, const char *path)
{
    if (!ctx || !path || !*path) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e || (e = ensure_net(ctx))) return e;
    hr_cnn_net *n = ctx->cnn;
    const size_t np = n->n_params, body = 24 + 3 * np * 4;
    FILE *f = fopen(path, "rb");
    if (!f) return HREBSD_EIO;
    std::vector<unsigned char> buf(body + 8);
    const size_t got = fread(buf.data(), 1, buf.size(), f);
    const int extra = fgetc(f);   // the file must end here
    fclose(f);
    if (got < 24 || memcmp(buf.data(), kCnnMagic, 8) != 0) return HREBSD_EFORMAT;
    int64_t hdr[2];
    memcpy(hdr, buf.data() + 8, 16);
    if (hdr[0] != (int64_t)np || hdr[1] < 0 || hdr[1] > 0x7fffffff) return HREBSD_EFORMAT;
    if (got != buf.size() || extra != EOF) return HREBSD_EFORMAT;
    uint64_t h;
    memcpy(&h, buf.data() + body, 8);
    if (h != fnv1a(buf.data(), body, kFnvBasis)) return HREBSD_EFORMAT;
    HR_CHECK(cudaDeviceSynchronize());
    HR_CHECK(cudaMemcpy(n->W, buf.data() + 24, np * 4, cudaMemcpyHostToDevice));
    HR_CHECK(cudaMemcpy(n->M, buf.data() + 24 + np * 4, np * 4, cudaMemcpyHostToDevice));
    HR_CHECK(cudaMemcpy(n->V, buf.data() + 24 + 2 * np * 4, np * 4, cudaMemcpyHostToDevice));
    n->step = (int)hdr[1];
    if ((e = refresh_bf16(ctx, 0))) return e;
    HR_CHECK(cudaDeviceSynchronize());
    return HREBSD_OK;
}

static int infer_common(hrebsd_ctx *ctx, int B, float *field, cudaStream_t st)
{
    int e = forward(ctx, B, st);
    if (e) return e;
    HR_CHECK(cudaMemcpyAsync(field, ctx->cnn->out, (size_t)B * 8192 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    return HREBSD_OK;
}

extern "C" int hrebsd_cnn_infer(hrebsd_ctx *ctx, const uint16_t *x_bf16, int B, float *field64, void *stream)
{
    if (!ctx || !ctx->cnn || B < 0) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!x_bf16 || !field64) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e || (e = ensure_acts(ctx, B))) return e;
    cudaStream_t st = hr_stream(stream);
    pack_nchw_kernel<<<grid2(4096, B), 256, 0, st>>>(reinterpret_cast<const bf16 *>(x_bf16), B,
                                                                     ctx->cnn->x);
    HR_LAUNCHED(ctx);
    return infer_common(ctx, B, field64, st);
}

extern "C" int hrebsd_cnn_infer_patterns(hrebsd_ctx *ctx, const float *ref, const float *test, const int32_t *ref_idx,
                                         int B, int H, int W, float *field64, void *stream)
{
    if (!ctx || !ctx->cnn || B < 0) return HREBSD_EINVAL;
    if (H != W || H < 64 || H % 64) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!ref || !test || !ref_idx || !field64) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e || (e = ensure_acts(ctx, B))) return e;
    cudaStream_t st = hr_stream(stream);
    pack_patterns_kernel<<<grid2(4096, B), 256, 0, st>>>(ref, test, ref_idx, B, H, W, ctx->cnn->x);
    HR_LAUNCHED(ctx);
    return infer_common(ctx, B, field64, st);
}

extern "C" int hrebsd_cnn_train_step(hrebsd_ctx *ctx, const uint16_t *x_bf16, const float *target, int B, float lr,
                                     float *loss_out, void *stream)
{
    if (!ctx || !ctx->cnn || B <= 0 || !x_bf16 || !target || !(lr >= 0.0f)) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e || (e = ensure_acts(ctx, B))) return e;
    hr_cnn_net *n = ctx->cnn;
    cudaStream_t st = hr_stream(stream);
    pack_nchw_kernel<<<grid2(4096, B), 256, 0, st>>>(reinterpret_cast<const bf16 *>(x_bf16), B, n->x);
    HR_LAUNCHED(ctx);
    if ((e = forward(ctx, B, st))) return e;
    HR_CHECK(cudaMemsetAsync(n->loss, 0, sizeof(float), st));
    HR_CHECK(cudaMemsetAsync(n->G, 0, n->n_params * sizeof(float), st));
    mse_kernel<<<grid_for(ctx, (size_t)B * 8192), 256, 0, st>>>(n->out, target, (size_t)B * 8192, n->dout, n->loss);
    HR_LAUNCHED(ctx);
    if ((e = backward(ctx, B, st))) return e;
    if (lr > 0.0f) {
        n->step++;
        const float b1 = 0.9f, b2 = 0.999f;
        const double bc1 = 1.0 - pow((double)b1, n->step), bc2 = 1.0 - pow((double)b2, n->step);
        const float lr_t = (float)(lr * sqrt(bc2) / bc1);
        // eps scaled so that the update equals lr m_hat / (sqrt(v_hat) + 1e-8)
        const float eps = (float)(1e-8 * sqrt(bc2));
        adam_kernel<<<grid_for(ctx, n->n_params), 256, 0, st>>>(n->W, n->G, n->M, n->V, n->n_params, lr_t, b1, b2, eps);
        HR_LAUNCHED(ctx);
        if ((e = refresh_bf16(ctx, st))) return e;
    }
    if (loss_out) HR_CHECK(cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
    return HREBSD_OK;
}

void hr_cnn_destroy(hrebsd_ctx *ctx)
{
    if (!ctx->cnn) return;
    for (void *p : ctx->cnn->allocs) cudaFree(p);
    delete ctx->cnn;
    ctx->cnn = nullptr;
}
