// 3x3 convolution on the fifth-generation tensor cores (tcgen05): the
// implicit GEMM of conv3x3_kernel (128 output pixels x BN output channels per
// CTA, K = 9 taps x cin walked in k-steps of 16 channels of one tap, STAGES
// cp.async stages of KS k-steps) with the MMAs issued by one thread from
// shared-memory descriptors into an FP32 accumulator in tensor memory.
//
// Shared layout of a k-step: the A rows (shifted input pixels) and B rows
// (weights) in the K-major core-matrix layout: row r, 8-channel group g at
// base + g * plane + 16 r (plane = rows x 16 bytes).  A stage is reused only
// after the MMAs that read it have completed (one mbarrier per stage, armed by
// tcgen05.commit).  Every wait is bounded; a wait that gives up sets the error
// flag and the CTA skips its epilogue.
#pragma once

#include "cnn_kernels.cuh"
#include "tc.cuh"

namespace hr_cnn {

template <int BN, int KS, int STAGES>
struct TcConv {
    static constexpr int BM = 128;
    static constexpr uint32_t A_PLANE = BM * 16, B_PLANE = BN * 16;
    static constexpr uint32_t STEP = 2 * A_PLANE + 2 * B_PLANE;   // one k-step: 16 channels of A and B
    static constexpr uint32_t STAGE = KS * STEP;
    static constexpr uint32_t SMEM = STAGES * STAGE;
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;      // power of two >= 32
};

template <int BN, int KS, int STAGES>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(ConvArgs a, int *err)
{
    using G = TcConv<BN, KS, STAGES>;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int P = a.N * a.H * a.W;
    const int p0 = blockIdx.x * G::BM, o0 = blockIdx.y * BN;
    // loader: A row tid (one output pixel), both 8-channel halves; B rows tid / 2 (half tid % 2) for tid < 2 BN
    const int lp = p0 + tid;
    int pn = 0, py = 0, px = 0;
    if (lp < P) {
        pn = lp / (a.H * a.W);
        const int rem = lp - pn * a.H * a.W;
        py = rem / a.W;
        px = rem - py * a.W;
    }
    const int lo = o0 + (tid >> 1), bhalf = tid & 1;
    const int ncb = a.cin / 16, KT = 9 * ncb, nstage = (KT + KS - 1) / KS;
    auto load_stage = [&](int s) {
        unsigned char *base = tc_smem + (s % STAGES) * G::STAGE;
#pragma unroll
        for (int j = 0; j < KS; ++j) {
            const int kt = s * KS + j;
            const int tap = kt / ncb, cb = kt - tap * ncb;
            const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
            const bool oka = kt < KT && lp < P && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            unsigned char *st = base + j * G::STEP;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const bf16 *src = oka ? a.x + ((size_t)(pn * a.H + yy) * a.W + xx) * a.xs + a.xo + cb * 16 + hh * 8 : a.x;
                cp_async16(st + hh * G::A_PLANE + tid * 16, src, oka ? 16 : 0);
            }
            if (tid < 2 * BN) {
                const bool okb = kt < KT && lo < a.cout;
                const bf16 *src = okb ? a.w + ((size_t)lo * 9 + tap) * a.cin + cb * 16 + bhalf * 8 : a.w;
                cp_async16(st + 2 * G::A_PLANE + bhalf * G::B_PLANE + (tid >> 1) * 16, src, okb ? 16 : 0);
            }
        }
    };
    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) hr_tma::mbar_init(&bar[i], 1);
        hr_tma::fence_mbar_init();
    }
    if (warp == 0) hr_tc::tmem_alloc(&tmem_base, G::TMEM_COLS);
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nstage) load_stage(s);
        cp_async_commit();
    }
    hr_tc::fence_before_sync();
    __syncthreads();
    hr_tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    constexpr uint32_t idesc = hr_tc::idesc_bf16(128, BN);
    bool ok = true;
    for (int s = 0; s < nstage; ++s) {
        cp_async_wait<STAGES - 2>();
        hr_tma::fence_proxy_async();   // this thread's cp.async data -> visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            hr_tc::fence_after_sync();
            const uint32_t sb = hr_tma::smem_u32(tc_smem + (s % STAGES) * G::STAGE);
#pragma unroll
            for (int j = 0; j < KS; ++j) {
                const uint32_t st = sb + j * G::STEP;
                hr_tc::mma_bf16(tb, hr_tc::smem_desc(st, G::A_PLANE, 128),
                                hr_tc::smem_desc(st + 2 * G::A_PLANE, G::B_PLANE, 128), idesc, (s | j) != 0);
            }
            hr_tc::commit(&bar[s % STAGES]);
        }
        // the buffer of stage s + STAGES - 1 was read by the MMAs of stage s - 1
        const int nx = s + STAGES - 1;
        if (nx < nstage) {
            if (s >= 1) ok = hr_tma::mbar_wait(&bar[(s - 1) % STAGES], ((s - 1) / STAGES) & 1) && ok;
            load_stage(nx);
        }
        cp_async_commit();
    }
    // the last commit covers every MMA of this CTA
    ok = hr_tma::mbar_wait(&bar[(nstage - 1) % STAGES], ((nstage - 1) / STAGES) & 1) && ok;
    ok = __syncthreads_and(ok);
    cp_async_wait<0>();
    hr_tc::fence_after_sync();
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        const int p = p0 + warp * 32 + (tid & 31);   // TMEM lane = A row = output pixel
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            hr_tc::ld16(tb + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (p < P) {
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const int o = o0 + c0 + i;
                    if (o >= a.cout) continue;
                    float v0 = v[i], v1 = v[i + 1];
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
                        *reinterpret_cast<float2 *>(reinterpret_cast<float *>(a.y) + off) = make_float2(v0, v1);
                    } else {
                        *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(a.y) + off) =
                            __floats2bfloat162_rn(v0, v1);
                    }
                }
            }
        }
    }
    hr_tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) hr_tc::tmem_dealloc(tb, G::TMEM_COLS);
}

// ------------------------------------------------------------------ halo tiles by TMA
// 3x3 convolution on tcgen05 with the input halo loaded once per tile.  The
// CTA computes a tile of TI images x Ht rows x all W columns of the output, for
// BN output channels.  The input window (Ht + 2 rows, W + 2 columns, zero
// outside the image) of each 8-channel group is one TMA box, stored as a flat
// run of pixels [image][row][column] of 16 bytes each ("plane").  In this
// flat order the input of tap (dy, dx) for the output at flat index q is at
// q + dy (W + 2) + dx, so the A operand of a tap is the plane's rows shifted by
// a constant: one shared-memory descriptor per (tap, 128-row block), no copy.
// Rows q whose column is W or W + 1 (or whose row lies past the tile) are
// computed but never stored.  The weights of a 16-channel chunk are laid out on
// the host side as [half][tap][BN][8] and arrive by one bulk copy.
//
// Roles: thread 0 issues the copies of chunk c into stage c % nst once the MMAs
// that read the stage before have completed (mbarrier `empty`, armed by
// tcgen05.commit); thread 32 waits for the copies (mbarrier `full`, transaction
// bytes), issues 9 x nM MMAs of 128 x BN x 16 into nM accumulators in tensor
// memory, and commits; after the last chunk all four warps read their TMEM
// lanes, add the bias, apply ReLU and store BF16.  Waits are bounded; a wait
// that gives up sets the error flag and the CTA skips its stores.
struct TmaConvArgs {
    const bf16 *wt;      // [cout / BN][cin / 16][2][9][BN][8]
    const float *bias;   // [cout] or null
    bf16 *y;             // output (NHWC, channel stride ys, offset yo)
    int ys, yo, relu;
    int cin, cout, N, res;
    int Ht, TI, nM, PR;  // tile rows, images per tile, 128-row MMA blocks, rows per plane
    int nst;             // pipeline stages in use (<= 3)
    int tmem_cols;
};

template <int BN>
__global__ void __launch_bounds__(128) conv3x3_tma_tc_kernel(const __grid_constant__ CUtensorMap tmX, TmaConvArgs a,
                                                            int *err)
{
    constexpr int MAXST = 3;
    constexpr uint32_t B_BYTES = 9 * BN * 32;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t full[MAXST], empty[MAXST], done;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunk = a.cin / 16, nst = a.nst;
    const int Wp = a.res + 2, Rimg = (a.Ht + 2) * Wp;
    const uint32_t A_PL = (uint32_t)a.PR * 16, STAGE = 2 * A_PL + B_BYTES;
    const uint32_t box_bytes = 16u * (uint32_t)(Rimg * a.TI);
    const int ncot = a.cout / BN, ty_tiles = a.res / a.Ht;
    const int cot = blockIdx.x % ncot, tile = blockIdx.x / ncot;
    const int n0 = (tile / ty_tiles) * a.TI, y0 = (tile % ty_tiles) * a.Ht;
    if (tid == 0) {
        for (int i = 0; i < nst; ++i) {
            hr_tma::mbar_init(&full[i], 1);
            hr_tma::mbar_init(&empty[i], 1);
        }
        hr_tma::mbar_init(&done, 1);
        hr_tma::fence_mbar_init();
    }
    if (warp == 0) hr_tc::tmem_alloc(&tmem_base, (uint32_t)a.tmem_cols);
    hr_tc::fence_before_sync();
    __syncthreads();
    hr_tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    bool ok = true;
    if (tid == 0) {
        const bf16 *wsrc = a.wt + (size_t)cot * nchunk * (B_BYTES / 2);
        for (int c = 0; c < nchunk; ++c) {
            const int s = c % nst, k = c / nst;
            if (k >= 1) ok = hr_tma::mbar_wait(&empty[s], (k - 1) & 1) && ok;
            unsigned char *base = tc_smem + s * STAGE;
            hr_tma::mbar_arrive_expect_tx(&full[s], 2 * box_bytes + B_BYTES);
            hr_tma::load_4d(base, &tmX, &full[s], c * 16, -1, y0 - 1, n0);
            hr_tma::load_4d(base + A_PL, &tmX, &full[s], c * 16 + 8, -1, y0 - 1, n0);
            hr_tma::load_bulk(base + 2 * A_PL, wsrc + (size_t)c * (B_BYTES / 2), B_BYTES, &full[s]);
        }
    } else if (tid == 32) {
        constexpr uint32_t idesc = hr_tc::idesc_bf16(128, BN);
        for (int c = 0; c < nchunk; ++c) {
            const int s = c % nst, k = c / nst;
            ok = hr_tma::mbar_wait(&full[s], k & 1) && ok;
            hr_tc::fence_after_sync();
            const uint32_t sa = hr_tma::smem_u32(tc_smem + s * STAGE), sb = sa + 2 * A_PL;
#pragma unroll 1
            for (int t = 0; t < 9; ++t) {
                const uint32_t off = (uint32_t)((t / 3) * Wp + t % 3) * 16;
                const uint64_t bdesc = hr_tc::smem_desc(sb + t * BN * 16, 9 * BN * 16, 128);
                for (int m = 0; m < a.nM; ++m)
                    hr_tc::mma_bf16(tb + (uint32_t)(m * BN), hr_tc::smem_desc(sa + m * 2048 + off, A_PL, 128), bdesc,
                                    idesc, (c | t) != 0);
            }
            hr_tc::commit(&empty[s]);
        }
        hr_tc::commit(&done);
    }
    ok = hr_tma::mbar_wait(&done, 0) && ok;
    ok = __syncthreads_and(ok);
    hr_tc::fence_after_sync();
    if (!ok) {
        if (tid == 0) {
            atomicExch(err, 1);
            // copies still in flight land before the CTA leaves (bounded)
            for (int c = nchunk - nst < 0 ? 0 : nchunk - nst; c < nchunk; ++c)
                (void)hr_tma::mbar_wait(&full[c % nst], (c / nst) & 1);
        }
    } else {
        const int o0 = cot * BN;
        for (int m = 0; m < a.nM; ++m) {
            const int q = m * 128 + warp * 32 + lane;
            const int nl = q / Rimg, rem = q - nl * Rimg, ty = rem / Wp, tx = rem - ty * Wp;
            const bool valid = nl < a.TI && ty < a.Ht && tx < a.res && n0 + nl < a.N;
            const size_t p = ((size_t)(n0 + nl) * a.res + (y0 + ty)) * a.res + tx;
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                hr_tc::ld16(tb + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * BN + c0), v);
                if (valid) {
                    __align__(16) __nv_bfloat162 o2[8];
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        float v0 = v[i], v1 = v[i + 1];
                        if (a.bias) {
                            v0 += a.bias[o0 + c0 + i];
                            v1 += a.bias[o0 + c0 + i + 1];
                        }
                        if (a.relu) {
                            v0 = fmaxf(v0, 0.0f);
                            v1 = fmaxf(v1, 0.0f);
                        }
                        o2[i / 2] = __floats2bfloat162_rn(v0, v1);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(a.y + p * a.ys + a.yo + o0 + c0);
                    dst[0] = *reinterpret_cast<const uint4 *>(&o2[0]);
                    dst[1] = *reinterpret_cast<const uint4 *>(&o2[4]);
                }
            }
        }
    }
    hr_tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) hr_tc::tmem_dealloc(tb, (uint32_t)a.tmem_cols);
}

}  // namespace hr_cnn
