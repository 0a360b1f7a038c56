// Kernels of the learned initialiser (project addition; the paper has no
// learned part): a 4-level U-Net, 3x3 convolutions of 16-32-64-128 channels,
// BF16 operands on the tensor cores with FP32 accumulation.
//
// Activations are NHWC BF16 with the channel count padded to a multiple of
// 16; a tensor is (pointer, channel stride, channel offset), so a layer can
// write straight into its slice of a concatenation buffer.  3x3 weights are
// stored [cout][tap][cin] (K = tap * cin + c contiguous per output channel),
// the layout the B operand of mma.m16n8k16.row.col wants.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

typedef __nv_bfloat16 bf16;

namespace hr_cnn {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t &r0, uint32_t &r1, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t &r0, uint32_t &r1, const void *p)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(smem_u32(p)));
}

// D += A (16x16, row) * B (16x8, col), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

struct ConvArgs {
    const bf16 *x;       // input NHWC, channel stride xs, offset xo, cin channels
    int xs, xo, cin;     // cin multiple of 16
    const bf16 *w;       // [cout][9][cin]
    const float *bias;   // [cout] or null
    int cout;            // multiple of 8
    void *y;             // output NHWC, channel stride ys, offset yo
    int ys, yo;
    int y_fp32;          // 1: FP32 output, else BF16
    int relu;
    int N, H, W;
};

// Implicit-GEMM 3x3 convolution, stride 1, zero padding:
// y[p][o] = bias[o] + sum_{tap, c} x[p + off(tap)][c] w[o][tap][c], off = (ky-1, kx-1).
// CTA tile 64 pixels x 64 output channels, 4 warps of 16 pixels x 64 channels.
__global__ void __launch_bounds__(128) conv3x3_kernel(ConvArgs a)
{
    constexpr int LDA = 24;   // bf16 per shared row (16 + 8 padding: conflict-free ldmatrix)
    __shared__ __align__(16) bf16 sa[64 * LDA];
    __shared__ __align__(16) bf16 sb[64 * LDA];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.N * a.H * a.W;
    const int p0 = blockIdx.x * 64, o0 = blockIdx.y * 64;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    // this thread's load slots: pixel / output channel tid/2, half (8 channels) tid%2
    const int lp = p0 + (tid >> 1), half = tid & 1;
    int pn = 0, py = 0, px = 0;
    if (lp < P) {
        pn = lp / (a.H * a.W);
        const int rem = lp - pn * a.H * a.W;
        py = rem / a.W;
        px = rem - py * a.W;
    }
    const int lo = o0 + (tid >> 1);
    const int ncb = a.cin / 16;
    for (int tap = 0; tap < 9; ++tap) {
        const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
        const bool inside = lp < P && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
        const bf16 *xrow = a.x + ((size_t)(pn * a.H + yy) * a.W + xx) * a.xs + a.xo + half * 8;
        const bf16 *wrow = a.w + ((size_t)lo * 9 + tap) * a.cin + half * 8;
        for (int cb = 0; cb < ncb; ++cb) {
            uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
            if (inside) va = *reinterpret_cast<const uint4 *>(xrow + cb * 16);
            if (lo < a.cout) vb = *reinterpret_cast<const uint4 *>(wrow + cb * 16);
            *reinterpret_cast<uint4 *>(sa + (tid >> 1) * LDA + half * 8) = va;
            *reinterpret_cast<uint4 *>(sb + (tid >> 1) * LDA + half * 8) = vb;
            __syncthreads();
            uint32_t a0, a1, a2, a3;
            ldsm_x4(a0, a1, a2, a3, sa + (warp * 16 + (lane & 15)) * LDA + (lane >> 4) * 8);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                uint32_t b0, b1;
                ldsm_x2(b0, b1, sb + (j * 8 + (lane & 7)) * LDA + ((lane >> 3) & 1) * 8);
                mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
            }
            __syncthreads();
        }
    }
    // epilogue: rows (pixels) warp*16 + lane/4 (+8), columns j*8 + (lane%4)*2 (+1)
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
        const int p = p0 + warp * 16 + (lane >> 2) + hrow * 8;
        if (p >= P) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int o = o0 + j * 8 + (lane & 3) * 2;
            if (o >= a.cout) continue;
            float v0 = acc[j][hrow * 2], v1 = acc[j][hrow * 2 + 1];
            if (a.bias) {
                v0 += a.bias[o];
                v1 += a.bias[o + 1];
            }
            if (a.relu) {
                v0 = fmaxf(v0, 0.0f);
                v1 = fmaxf(v1, 0.0f);
            }
            const size_t off = (size_t)p * a.ys + a.yo + o;
            if (a.y_fp32) {
                float *y = reinterpret_cast<float *>(a.y);
                y[off] = v0;
                y[off + 1] = v1;
            } else {
                *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(a.y) + off) = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

struct WgradArgs {
    const bf16 *dy;      // [P][cout] (dense)
    int cout;            // multiple of 16
    const bf16 *x;       // conv input NHWC (stride xs, offset xo), cin channels
    int xs, xo, cin;
    float *dw;           // [cout][9][cin], accumulated with atomics
    int N, H, W;
    int chunk;           // pixels per CTA (multiple of 16)
};

// dw[o][tap][c] += sum_p dy[p][o] x[p + off(tap)][c] over this CTA's pixel chunk.
// grid (pixel chunks, 9 * cin/64 (rounded up), cout/64 (rounded up)); 4 warps,
// each 16 output channels x 64 input channels.
__global__ void __launch_bounds__(128) conv3x3_wgrad_kernel(WgradArgs a)
{
    constexpr int LD = 72;   // bf16 per shared row (64 + 8)
    __shared__ __align__(16) bf16 sdy[16 * LD];   // [16 pixels][64 couts]
    __shared__ __align__(16) bf16 sx[16 * LD];    // [16 pixels][64 cins]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.N * a.H * a.W;
    const int ncblk = (a.cin + 63) / 64;
    const int tap = blockIdx.y / ncblk, c0 = (blockIdx.y - tap * ncblk) * 64;
    const int o0 = blockIdx.z * 64;
    const int dyy = tap / 3 - 1, dxx = tap % 3 - 1;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
    const int pbeg = blockIdx.x * a.chunk, pend = min(P, pbeg + a.chunk);
    // load slots: pixel tid/8, 8 channels at (tid%8)*8
    const int lr = tid >> 3, lc = (tid & 7) * 8;
    for (int pb = pbeg; pb < pend; pb += 16) {
        const int p = pb + lr;
        uint4 vd = make_uint4(0, 0, 0, 0), vx = make_uint4(0, 0, 0, 0);
        if (p < pend) {
            if (o0 + lc < a.cout) vd = *reinterpret_cast<const uint4 *>(a.dy + (size_t)p * a.cout + o0 + lc);
            const int n = p / (a.H * a.W), rem = p - n * a.H * a.W;
            const int yy = rem / a.W + dyy, xx = rem % a.W + dxx;
            if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W && c0 + lc < a.cin)
                vx = *reinterpret_cast<const uint4 *>(a.x + ((size_t)(n * a.H + yy) * a.W + xx) * a.xs + a.xo + c0 + lc);
        }
        *reinterpret_cast<uint4 *>(sdy + lr * LD + lc) = vd;
        *reinterpret_cast<uint4 *>(sx + lr * LD + lc) = vx;
        __syncthreads();
        // A (16 couts x 16 pixels) = dy^T: transposed load of the [pixel][cout] tile
        uint32_t a0, a1, a2, a3;
        ldsm_x4_t(a0, a1, a2, a3, sdy + ((lane & 7) + ((lane >> 4) & 1) * 8) * LD + warp * 16 + ((lane >> 3) & 1) * 8);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t b0, b1;   // B (16 pixels x 8 cins): transposed load of the [pixel][cin] tile
            ldsm_x2_t(b0, b1, sx + ((lane & 7) + ((lane >> 3) & 1) * 8) * LD + j * 8);
            mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
        }
        __syncthreads();
    }
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
        const int o = o0 + warp * 16 + (lane >> 2) + hrow * 8;
        if (o >= a.cout) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = c0 + j * 8 + (lane & 3) * 2;
            if (c >= a.cin) continue;
            float *dst = a.dw + ((size_t)o * 9 + tap) * a.cin + c;
            atomicAdd(dst, acc[j][hrow * 2]);
            atomicAdd(dst + 1, acc[j][hrow * 2 + 1]);
        }
    }
}

}  // namespace hr_cnn
