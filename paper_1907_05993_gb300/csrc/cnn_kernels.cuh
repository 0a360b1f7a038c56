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

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros (the
// source address is then not read).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(smem)), "l"(gmem), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Implicit-GEMM 3x3 convolution, stride 1, zero padding:
// y[p][o] = bias[o] + sum_{tap, c} x[p + off(tap)][c] w[o][tap][c], off = (ky-1, kx-1).
// CTA tile: 128 output pixels (8 warps x 16) x BN output channels.  The K
// dimension (9 taps x cin) is walked in k-steps of 16 channels of one tap;
// KS k-steps form a pipeline stage whose A rows (the shifted input pixels,
// zero-filled outside the image) and B rows (weights) arrive by cp.async,
// STAGES stages in flight.
template <int BN, int KS, int STAGES>
__global__ void __launch_bounds__(256) conv3x3_kernel(ConvArgs a)
{
    constexpr int BM = 128, LD = 24;   // bf16 per shared row (16 + 8 padding: conflict-free ldmatrix)
    constexpr int A_EL = BM * LD, B_EL = BN * LD, STEP_EL = A_EL + B_EL, STAGE_EL = KS * STEP_EL;
    extern __shared__ __align__(16) unsigned char conv_smem[];
    bf16 *sm = reinterpret_cast<bf16 *>(conv_smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.N * a.H * a.W;
    const int p0 = blockIdx.x * BM, o0 = blockIdx.y * BN;
    // loader slots: A row tid/2 (a pixel), half tid%2 (8 channels); B row tid/2 for tid < 2 BN
    const int lp = p0 + (tid >> 1), half = tid & 1;
    int pn = 0, py = 0, px = 0;
    if (lp < P) {
        pn = lp / (a.H * a.W);
        const int rem = lp - pn * a.H * a.W;
        py = rem / a.W;
        px = rem - py * a.W;
    }
    const int lo = o0 + (tid >> 1);
    const int ncb = a.cin / 16, KT = 9 * ncb, nstage = (KT + KS - 1) / KS;
    auto load_stage = [&](int s) {
        bf16 *base = sm + (s % STAGES) * STAGE_EL;
#pragma unroll
        for (int j = 0; j < KS; ++j) {
            const int kt = s * KS + j;
            const int tap = kt / ncb, cb = kt - tap * ncb;
            const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
            const bool oka = kt < KT && lp < P && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const bf16 *srca = oka ? a.x + ((size_t)(pn * a.H + yy) * a.W + xx) * a.xs + a.xo + cb * 16 + half * 8 : a.x;
            cp_async16(base + j * STEP_EL + (tid >> 1) * LD + half * 8, srca, oka ? 16 : 0);
            if (tid < 2 * BN) {
                const bool okb = kt < KT && lo < a.cout;
                const bf16 *srcb = okb ? a.w + ((size_t)lo * 9 + tap) * a.cin + cb * 16 + half * 8 : a.w;
                cp_async16(base + j * STEP_EL + A_EL + (tid >> 1) * LD + half * 8, srcb, okb ? 16 : 0);
            }
        }
    };
    float acc[BN / 8][4];
#pragma unroll
    for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nstage) load_stage(s);
        cp_async_commit();
    }
    for (int s = 0; s < nstage; ++s) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();   // stage s is in shared memory; stage s - 1 is consumed by every warp
        if (s + STAGES - 1 < nstage) load_stage(s + STAGES - 1);
        cp_async_commit();
        const bf16 *base = sm + (s % STAGES) * STAGE_EL;
#pragma unroll
        for (int j = 0; j < KS; ++j) {
            const bf16 *sa = base + j * STEP_EL, *sb = sa + A_EL;
            uint32_t a0, a1, a2, a3;
            ldsm_x4(a0, a1, a2, a3, sa + (warp * 16 + (lane & 15)) * LD + (lane >> 4) * 8);
#pragma unroll
            for (int jn = 0; jn < BN / 8; ++jn) {
                uint32_t b0, b1;
                ldsm_x2(b0, b1, sb + (jn * 8 + (lane & 7)) * LD + ((lane >> 3) & 1) * 8);
                mma_bf16(acc[jn], a0, a1, a2, a3, b0, b1);
            }
        }
    }
    cp_async_wait<0>();
    // epilogue: rows (pixels) warp*16 + lane/4 (+8), columns jn*8 + (lane%4)*2 (+1)
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
        const int p = p0 + warp * 16 + (lane >> 2) + hrow * 8;
        if (p >= P) continue;
#pragma unroll
        for (int j = 0; j < BN / 8; ++j) {
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

// Shared-memory bytes of conv3x3_kernel<BN, KS, STAGES>.
constexpr size_t conv_smem_bytes(int bn, int ks, int stages) { return (size_t)stages * ks * (128 + bn) * 24 * 2; }

// Same convolution for images of at least 16 x 16 pixels, as a persistent
// kernel over spatial tiles of 8 rows x 16 columns of one image.  The CTA keeps
// all 9 taps of its BN weight rows in shared memory and double-buffers the
// (8 + 2) x (16 + 2)-pixel input halo of its tiles (zeros outside the image),
// so that every tap is an offset into the halo: the A fragments come from
// ldmatrix row addresses of the shifted pixels, with no per-tap copy.  Warp w
// computes image row w of the tile (16 pixels) x BN output channels.  Shared
// rows are padded by 16 bytes to an odd number of 16-byte units (conflict-free
// ldmatrix).
template <int CIN, int BN>
struct HaloConv {
    static constexpr int TH = 8, TW = 16, HH = TH + 2, HW = TW + 2, HPX = HH * HW;
    static constexpr int RB = 2 * CIN + 16;       // bytes per halo pixel
    static constexpr int WRB = 18 * CIN + 16;     // bytes per output channel (9 taps x CIN)
    static constexpr size_t W_BYTES = (size_t)BN * WRB;
    static constexpr size_t H_BYTES = (size_t)HPX * RB;
    static constexpr size_t SMEM = W_BYTES + 2 * H_BYTES;
};

template <int CIN, int BN>
__global__ void __launch_bounds__(256) conv3x3_halo_kernel(ConvArgs a)
{
    using G = HaloConv<CIN, BN>;
    extern __shared__ __align__(16) unsigned char halo_smem[];
    unsigned char *sw = halo_smem;
    unsigned char *const sh0 = halo_smem + G::W_BYTES;   // halo buffers sh0, sh0 + H_BYTES
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int res = a.H;   // square images, res % 16 == 0
    const int tx_n = res / G::TW, ty_n = res / G::TH, per_img = tx_n * ty_n;
    const long long tiles = (long long)a.N * per_img;
    const int o0 = blockIdx.y * BN;
    constexpr int CCH = CIN / 8;   // 16-byte chunks per pixel
    // weights of output channels o0 .. o0 + BN - 1, all taps
    for (int i = tid; i < BN * 9 * CCH; i += blockDim.x) {
        const int n = i / (9 * CCH), rem = i - n * 9 * CCH;
        const int o = o0 + n;
        const bool ok = o < a.cout;
        cp_async16(sw + n * G::WRB + rem * 16, ok ? a.w + ((size_t)o * 9 * CIN + rem * 8) : a.w, ok ? 16 : 0);
    }
    auto load_halo = [&](long long t, unsigned char *dst) {
        const int img = (int)(t / per_img), r = (int)(t - (long long)img * per_img);
        const int y0 = (r / tx_n) * G::TH - 1, x0 = (r % tx_n) * G::TW - 1;
        for (int i = tid; i < G::HPX * CCH; i += blockDim.x) {
            const int px = i / CCH, c = i - px * CCH;
            const int yy = y0 + px / G::HW, xx = x0 + px % G::HW;
            const bool ok = yy >= 0 && yy < res && xx >= 0 && xx < res;
            const bf16 *src = ok ? a.x + ((size_t)(img * res + yy) * res + xx) * a.xs + a.xo + c * 8 : a.x;
            cp_async16(dst + px * G::RB + c * 16, src, ok ? 16 : 0);
        }
    };
    long long t = blockIdx.x;
    if (t < tiles) load_halo(t, sh0);
    cp_async_commit();
    for (int it = 0; t < tiles; ++it, t += gridDim.x) {
        const long long tn = t + gridDim.x;
        if (tn < tiles) load_halo(tn, sh0 + ((it + 1) & 1) * G::H_BYTES);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const unsigned char *hb = sh0 + (it & 1) * G::H_BYTES;
        float acc[BN / 8][4];
#pragma unroll
        for (int j = 0; j < BN / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
        // lane's A row: pixel (warp, lane % 16) of the tile, channel half lane / 16
        const unsigned char *arow = hb + (warp * G::HW + (lane & 15)) * G::RB + (lane >> 4) * 16;
        const unsigned char *brow = sw + (lane & 7) * G::WRB + ((lane >> 3) & 1) * 16;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const unsigned char *ap = arow + ((tap / 3) * G::HW + tap % 3) * G::RB;
#pragma unroll
            for (int kb = 0; kb < CIN / 16; ++kb) {
                uint32_t a0, a1, a2, a3;
                ldsm_x4(a0, a1, a2, a3, ap + kb * 32);
#pragma unroll
                for (int jn = 0; jn < BN / 8; ++jn) {
                    uint32_t b0, b1;
                    ldsm_x2(b0, b1, brow + jn * 8 * G::WRB + (tap * CIN + kb * 16) * 2);
                    mma_bf16(acc[jn], a0, a1, a2, a3, b0, b1);
                }
            }
        }
        // epilogue: pixels (warp, lane / 4 (+8)), channels jn * 8 + (lane % 4) * 2 (+1)
        const int img = (int)(t / per_img), r = (int)(t - (long long)img * per_img);
        const int yy = (r / tx_n) * G::TH + warp, xb = (r % tx_n) * G::TW;
#pragma unroll
        for (int hrow = 0; hrow < 2; ++hrow) {
            const size_t p = (size_t)(img * res + yy) * res + xb + (lane >> 2) + hrow * 8;
#pragma unroll
            for (int j = 0; j < BN / 8; ++j) {
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
                const size_t off = p * a.ys + a.yo + o;
                if (a.y_fp32) {
                    float *y = reinterpret_cast<float *>(a.y);
                    *reinterpret_cast<float2 *>(y + off) = make_float2(v0, v1);
                } else {
                    *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(a.y) + off) =
                        __floats2bfloat162_rn(v0, v1);
                }
            }
        }
        __syncthreads();   // the halo buffer of this tile may be refilled
    }
    cp_async_wait<0>();
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

// Planar BF16 copies of an NHWC tensor (channel stride ss, offset so, C channels, P pixels of images
// res x res): dk[c][q] = src[q + s_k][c] with s_0 = +1, s_1 = 0, s_2 = -1, zero where x + s_k leaves
// the row [0, res); null outputs are skipped.  A block moves 64 pixels x 32 channels through a shared
// tile with one halo pixel on each side: 16-byte loads along channels (ss, so and C multiples of 8),
// 16-byte stores of 8 pixels along each output row (P a multiple of 64).
__global__ void __launch_bounds__(256) planar_shift_kernel(const bf16 *src, int ss, int so, int C, int P, int res,
                                                         bf16 *d0, bf16 *d1, bf16 *d2)
{
    __shared__ unsigned short tile[66][34];   // [pixel][channel]; row stride of 17 words
    const int q0 = blockIdx.x * 64, c0 = blockIdx.y * 32;
    for (int i = threadIdx.x; i < 66 * 4; i += 256) {   // 66 pixels x 4 groups of 8 channels
        const int r = i >> 2, g = i & 3, q = q0 - 1 + r, c = c0 + g * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (q >= 0 && q < P && c < C) v = *reinterpret_cast<const uint4 *>(src + (size_t)q * ss + so + c);
        const unsigned short *h = reinterpret_cast<const unsigned short *>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) tile[r][g * 8 + j] = h[j];
    }
    __syncthreads();
    unsigned short *out[3] = {reinterpret_cast<unsigned short *>(d0), reinterpret_cast<unsigned short *>(d1),
                              reinterpret_cast<unsigned short *>(d2)};
    for (int i = threadIdx.x; i < 3 * 32 * 8; i += 256) {   // (copy, channel, 8-pixel group)
        const int k = i / 256, c = (i >> 3) & 31, g = i & 7;
        if (!out[k] || c0 + c >= C) continue;
        const int sft = 1 - k;
        __align__(16) unsigned short h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int jj = g * 8 + j, x = (q0 + jj) % res;
            h[j] = (x + sft >= 0 && x + sft < res) ? tile[jj + 1 + sft][c] : (unsigned short)0;
        }
        *reinterpret_cast<uint4 *>(out[k] + (size_t)(c0 + c) * P + q0 + g * 8) = *reinterpret_cast<const uint4 *>(h);
    }
}

}  // namespace hr_cnn
