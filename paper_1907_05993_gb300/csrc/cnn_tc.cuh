// 3x3 convolutions of the learned initialiser on the fifth-generation tensor
// cores (tcgen05): input halo tiles by TMA, MMAs issued by one thread from
// shared-memory descriptors into FP32 accumulators in tensor memory.
#pragma once

#include "cnn_kernels.cuh"
#include "tc.cuh"

namespace hr_cnn {

// ------------------------------------------------------------------ halo tiles by TMA
// 3x3 convolution on tcgen05 with the input halo loaded once per tile.  A tile
// is TI images x Ht rows x all W columns of the output, for BN output channels.
// The input window (Ht + 2 rows, W + 2 columns, zero outside the image) of CW
// channels (16, 32 or 64) is one TMA box, stored as a flat run of pixels
// [image][row][column] of CW x 2 bytes each in the matching 32/64/128-byte
// swizzled layout.  In this flat order the input of tap (dy, dx) for the output
// at flat index q is at q + dy (W + 2) + dx, so the A operand of a tap is the
// run shifted by a constant number of rows: one shared-memory descriptor per
// (tap, 128-row block, 16-channel step), no copy.  Rows q whose column is W or
// W + 1 (or that lie past the tile) are computed, never stored.  The weights of
// a 16-channel step are laid out on the host side as [half][tap][BN][8] (no
// swizzle) and arrive by one bulk copy with the box.
//
// Persistent and warp-specialised (320 threads, one CTA per SM): warp 0 lane 0
// streams (tile, box) copies through a ring of `nst` shared-memory stages;
// warp 1 lane 0 issues 9 x nM MMAs of 128 x BN x 16 per 16-channel step into
// one of two accumulators in tensor memory and releases each stage with
// tcgen05.commit; warps 2-9 read the finished accumulator (two warps per TMEM
// lane quadrant, alternate 128-row blocks), add the bias, apply ReLU, store
// BF16 and hand the accumulator back, so that the epilogue of one tile
// overlaps the MMAs of the next.  Every
// wait is bounded and also gives up when another role has given up; the CTA
// then stores nothing more and sets the error flag.
// Tile geometry per image size (compile-time, shared by host and kernel): Ht
// output rows of TI images per tile, BN output channels; NM 128-row MMA blocks
// cover the tile's last stored flat row; PR rows per box buffer cover the box
// and the furthest row an MMA reads; two accumulators of ACC TMEM columns.
template <int RES>
struct TmaGeom {
    static constexpr int Ht = RES >= 16 ? 16 : 8;
    static constexpr int TI = RES >= 16 ? 1 : 5;
    static constexpr int BN = RES >= 64 ? 16 : (RES >= 32 ? 32 : 64);
    static constexpr int Wp = RES + 2, Rimg = (Ht + 2) * Wp;
    static constexpr int QN = (TI - 1) * Rimg + (Ht - 1) * Wp + RES;
    static constexpr int NM = (QN + 127) / 128;
    static constexpr int ROWS = TI * Rimg > NM * 128 + 2 * Wp + 2 ? TI * Rimg : NM * 128 + 2 * Wp + 2;
    static constexpr int PR = (ROWS + 7) / 8 * 8;
    static constexpr int ACC = NM * BN <= 32 ? 32 : NM * BN <= 64 ? 64 : NM * BN <= 128 ? 128 : 256;
    static constexpr int TMEM = 2 * ACC;
    static constexpr int EM = (NM + 1) / 2;   // row blocks per epilogue warp
    static_assert(NM * BN <= 256 && RES % Ht == 0 && Wp <= 256 && Ht + 2 <= 256, "tile geometry");
};

struct TmaConvArgs {
    const bf16 *wt;      // [cout / BN][cin / 16][2][9][BN][8]
    const float *bias;   // [cout] or null
    bf16 *y;             // output (NHWC, channel stride ys, offset yo), or null when yf is set
    float *yf;           // FP32 output in the same layout (the input gradients), or null
    int ys, yo, relu;
    int cin, cout, N;
    int cw;              // channels per box (16, 32 or 64)
    int a_bytes;         // bytes of a box buffer (multiple of 1024)
    int stage_bytes;     // box buffer + weights of its 16-channel steps (multiple of 1024)
    int nst;             // shared-memory stages in the ring (<= 8)
    int ntiles;          // tiles x output-channel blocks
};

namespace tmaconv {

__device__ __forceinline__ bool wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    for (uint32_t i = 0; i < hr_tma::kSpinLimit; ++i) {
        if (hr_tma::mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && *abort) return false;
    }
    *abort = 1;
    return false;
}

struct Tile {
    int cot, n0, y0;
};
template <int RES>
__device__ __forceinline__ Tile tile_of(int t, int ncot)
{
    using G = TmaGeom<RES>;
    constexpr int ty_tiles = RES / G::Ht;
    const int sp = t / ncot;
    return Tile{t - sp * ncot, (sp / ty_tiles) * G::TI, (sp % ty_tiles) * G::Ht};
}

}  // namespace tmaconv

constexpr int kTmaConvThreads = 320;   // producer warp, MMA warp, 8 epilogue warps

template <int RES>
__global__ void __launch_bounds__(kTmaConvThreads, 1)
    conv3x3_tma_tc_kernel(const __grid_constant__ CUtensorMap tmX, TmaConvArgs a, int *err)
{
    using G = TmaGeom<RES>;
    constexpr int BN = G::BN, NM = G::NM, Wp = G::Wp, Rimg = G::Rimg;
    constexpr int MAXST = 8;
    constexpr uint32_t B_BYTES = 9 * BN * 32;   // weights of one 16-channel step
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ __align__(8) uint64_t full[MAXST], empty[MAXST], accf[2], acce[2], drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_s;
    __shared__ float bias_s[256];
    // swizzled boxes need 1024-byte aligned buffers: the host adds 1 KB of slack
    unsigned char *tc_smem = tc_smem_raw + ((1024u - (hr_tma::smem_u32(tc_smem_raw) & 1023u)) & 1023u);
    volatile int *abort = &abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ksub = a.cw / 16, nbox = a.cin / a.cw, nst = a.nst, ncot = a.cout / BN;
    const uint32_t RB = (uint32_t)a.cw * 2;   // bytes per pixel row of a box
    const uint32_t STAGE = (uint32_t)a.stage_bytes;
    const uint32_t box_bytes = RB * (uint32_t)(Rimg * G::TI);
    if (tid == 0) {
        for (int i = 0; i < nst; ++i) {
            hr_tma::mbar_init(&full[i], 1);
            hr_tma::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            hr_tma::mbar_init(&accf[i], 1);
            hr_tma::mbar_init(&acce[i], 8);
        }
        hr_tma::mbar_init(&drain, 1);
        abort_s = 0;
        hr_tma::fence_mbar_init();
    }
    for (int i = tid; i < a.cout; i += blockDim.x) bias_s[i] = a.bias ? a.bias[i] : 0.0f;
    if (warp == 1) hr_tc::tmem_alloc(&tmem_base, (uint32_t)G::TMEM);
    hr_tc::fence_before_sync();
    __syncthreads();
    hr_tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    if (warp == 0) {
        if (lane == 0) {   // producer
            int it = 0;
            for (int t = blockIdx.x; t < a.ntiles && !*abort; t += gridDim.x) {
                const tmaconv::Tile T = tmaconv::tile_of<RES>(t, ncot);
                const bf16 *wsrc = a.wt + (size_t)T.cot * (a.cin / 16) * (B_BYTES / 2);
                for (int c = 0; c < nbox; ++c, ++it) {
                    const int s = it % nst, k = it / nst;
                    if (k >= 1 && !tmaconv::wait(&empty[s], (k - 1) & 1, abort)) break;
                    unsigned char *base = tc_smem + s * STAGE;
                    hr_tma::mbar_arrive_expect_tx(&full[s], box_bytes + ksub * B_BYTES);
                    hr_tma::load_4d(base, &tmX, &full[s], c * a.cw, -1, T.y0 - 1, T.n0);
                    hr_tma::load_bulk(base + a.a_bytes, wsrc + (size_t)c * ksub * (B_BYTES / 2), ksub * B_BYTES,
                                      &full[s]);
                }
            }
            if (*abort) {   // copies still in flight land before the CTA leaves (bounded)
                for (int j = it - nst < 0 ? 0 : it - nst; j < it; ++j)
                    (void)hr_tma::mbar_wait(&full[j % nst], (j / nst) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc = hr_tc::idesc_bf16(128, BN);
            // descriptors are linear in the start address (field = address >> 4, no carry for
            // addresses below 256 KB): per stage one base, per MMA one add
            uint32_t toff[9];
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) toff[tap] = ((uint32_t)((tap / 3) * Wp + tap % 3) * RB) >> 4;
            const uint32_t mstep = (128u * RB) >> 4;
            int it = 0, i = 0;
            for (int t = blockIdx.x; t < a.ntiles && !*abort; t += gridDim.x, ++i) {
                const int b = i & 1, u = i >> 1;
                if (u >= 1 && !tmaconv::wait(&acce[b], (u - 1) & 1, abort)) break;
                hr_tc::fence_after_sync();
                const uint32_t d = tb + (uint32_t)(b * G::ACC);
                for (int c = 0; c < nbox; ++c, ++it) {
                    const int s = it % nst, k = it / nst;
                    if (!tmaconv::wait(&full[s], k & 1, abort)) break;
                    hr_tc::fence_after_sync();
                    const uint32_t sa = hr_tma::smem_u32(tc_smem + s * STAGE);
                    const uint64_t a0 = hr_tc::smem_desc_swz(sa, RB);
                    const uint64_t b0 = hr_tc::smem_desc(sa + (uint32_t)a.a_bytes, 9 * BN * 16, 128);
                    for (int kk = 0; kk < ksub; ++kk) {
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
                            const uint64_t at = a0 + (toff[tap] + 2u * kk);
                            const uint64_t bt = b0 + ((kk * B_BYTES + tap * BN * 16) >> 4);
                            const uint32_t acc = (c | kk | tap) != 0;
#pragma unroll
                            for (int m = 0; m < NM; ++m)
                                hr_tc::mma_bf16(d + (uint32_t)(m * BN), at + m * mstep, bt, idesc, acc);
                        }
                    }
                    hr_tc::commit(&empty[s]);
                }
                hr_tc::commit(&accf[b]);
            }
        }
    } else {   // epilogue: warps 2..9; TMEM lane quadrant warp % 4, 128-row blocks m = (warp - 2) / 4 (mod 2)
        const int quad = warp & 3, half = (warp - 2) >> 2;
        // the flat row -> pixel decode is the same for every tile: once per thread
        int prel[G::EM], pnl[G::EM];
#pragma unroll
        for (int j = 0; j < G::EM; ++j) {
            const int m = 2 * j + half;
            const int q = m * 128 + quad * 32 + lane;
            const int nl = q / Rimg, rem = q - nl * Rimg, ty = rem / Wp, tx = rem - ty * Wp;
            const bool ok = m < NM && nl < G::TI && ty < G::Ht && tx < RES;
            prel[j] = ok ? (nl * RES + ty) * RES + tx : -1;
            pnl[j] = nl;
        }
        int i = 0;
        for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++i) {
            const int b = i & 1, u = i >> 1;
            const bool got = tmaconv::wait(&accf[b], u & 1, abort);
            if (!__all_sync(0xffffffffu, got)) break;
            hr_tc::fence_after_sync();
            const tmaconv::Tile T = tmaconv::tile_of<RES>(t, ncot);
            const int o0 = T.cot * BN;
            const size_t pbase = ((size_t)T.n0 * RES + T.y0) * RES;
            const uint32_t d = tb + (uint32_t)(b * G::ACC) + ((uint32_t)(quad * 32) << 16);
#pragma unroll
            for (int j = 0; j < G::EM; ++j) {
                const int m = 2 * j + half;
                if (m >= NM) break;
                float v[BN];
#pragma unroll
                for (int c0 = 0; c0 < BN; c0 += 16) hr_tc::ld16_async(d + (uint32_t)(m * BN + c0), &v[c0]);
                hr_tc::wait_ld();
                if (prel[j] >= 0 && T.n0 + pnl[j] < a.N && a.yf) {   // FP32 output
                    float4 *dst = reinterpret_cast<float4 *>(a.yf + (pbase + prel[j]) * a.ys + a.yo + o0);
#pragma unroll
                    for (int c0 = 0; c0 < BN; c0 += 4) {
                        float4 o4 = make_float4(v[c0] + bias_s[o0 + c0], v[c0 + 1] + bias_s[o0 + c0 + 1],
                                                v[c0 + 2] + bias_s[o0 + c0 + 2], v[c0 + 3] + bias_s[o0 + c0 + 3]);
                        if (a.relu) {
                            o4.x = fmaxf(o4.x, 0.0f);
                            o4.y = fmaxf(o4.y, 0.0f);
                            o4.z = fmaxf(o4.z, 0.0f);
                            o4.w = fmaxf(o4.w, 0.0f);
                        }
                        dst[c0 / 4] = o4;
                    }
                } else if (prel[j] >= 0 && T.n0 + pnl[j] < a.N) {
                    uint4 *dst = reinterpret_cast<uint4 *>(a.y + (pbase + prel[j]) * a.ys + a.yo + o0);
#pragma unroll
                    for (int c0 = 0; c0 < BN; c0 += 8) {
                        __align__(16) __nv_bfloat162 o2[4];
#pragma unroll
                        for (int k = 0; k < 8; k += 2) {
                            float v0 = v[c0 + k] + bias_s[o0 + c0 + k], v1 = v[c0 + k + 1] + bias_s[o0 + c0 + k + 1];
                            if (a.relu) {
                                v0 = fmaxf(v0, 0.0f);
                                v1 = fmaxf(v1, 0.0f);
                            }
                            o2[k / 2] = __floats2bfloat162_rn(v0, v1);
                        }
                        dst[c0 / 8] = *reinterpret_cast<const uint4 *>(o2);
                    }
                }
            }
            hr_tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) hr_tma::mbar_arrive(&acce[b]);
        }
    }
    // an MMA thread that gave up may leave MMAs in flight: let them finish before TMEM is freed
    hr_tc::fence_before_sync();
    __syncthreads();
    if (*abort) {
        if (tid == 32) {
            hr_tc::commit(&drain);   // arrives once every MMA issued so far has completed
            (void)hr_tma::mbar_wait(&drain, 0);
        }
        if (tid == 0) atomicExch(err, 1);
        __syncthreads();
    }
    hr_tc::fence_after_sync();
    if (warp == 1) hr_tc::tmem_dealloc(tb, (uint32_t)G::TMEM);
}

}  // namespace hr_cnn

namespace hr_cnn {

// Weight gradients of a 3x3 convolution on tcgen05:
//   dw[o][tap][c] = sum_p dy[p][o] x[p + off(tap)][c] = sum_q dy[q - off(tap)][o] x[q][c],
// a GEMM per tap over the pixels q (K).  With K-major operands (the library's tested descriptor
// form) the pixels must be contiguous: the inputs come transposed to planar [channel][image][pixel]
// BF16 (xT, and dy in three copies shifted by +1, 0, -1 pixels along x with zeros past the row ends);
// the shift along y is the TMA coordinate (whole rows, 16-byte aligned; rows outside read zero).
// D[c][tap * NB + o] = A (128 input channels x 64 pixels) B_tap^T (NB output channels x 64 pixels),
// accumulated over the CTA's range of 64-pixel K tiles; the epilogue adds D into dw with atomics.
// Warp 0: TMA producer; warp 1: MMA issuer; warps 2-5: epilogue (TMEM lanes = input channels).
struct WgradTcArgs {
    float *dw;        // [cout][9][cin], accumulated
    int cin, cout, res;
    int ncb, nob;     // 128-channel input blocks, NB-channel output blocks
    int splits;       // K ranges per (input block, output block)
    int ktiles;       // 64-pixel K tiles in all images
    int nst;          // pipeline stages
};

constexpr int kWgradThreads = 192;

template <int NB>
__global__ void __launch_bounds__(kWgradThreads, 1)
    conv3x3_wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmD0,
                            const __grid_constant__ CUtensorMap tmD1, const __grid_constant__ CUtensorMap tmD2,
                            WgradTcArgs a, int *err)
{
    static_assert(NB % 16 == 0 && 9 * NB <= 512, "one output block of every tap in TMEM");
    constexpr int MAXST = 8;
    constexpr uint32_t A_BYTES = 128 * 128;      // 128 channels x 64 pixels BF16
    constexpr uint32_t B_BYTES = NB * 128;       // NB channels x 64 pixels BF16
    constexpr uint32_t STAGE = A_BYTES + 9 * B_BYTES;
    static_assert(STAGE % 1024 == 0, "1024-byte aligned stages (128-byte swizzle)");
    constexpr uint32_t TMEM_COLS = 9 * NB <= 256 ? 256 : 512;
    extern __shared__ __align__(1024) unsigned char wg_smem_raw[];
    __shared__ __align__(8) uint64_t full[MAXST], empty[MAXST], accf, drain;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_s;
    unsigned char *smem = wg_smem_raw + ((1024u - (hr_tma::smem_u32(wg_smem_raw) & 1023u)) & 1023u);
    volatile int *abort = &abort_s;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nst = a.nst;
    // this CTA's item: input block, output block, K range
    const int cb = blockIdx.x % a.ncb, rest = blockIdx.x / a.ncb, ob = rest % a.nob, sp = rest / a.nob;
    const int k0 = (int)((long long)sp * a.ktiles / a.splits), k1 = (int)((long long)(sp + 1) * a.ktiles / a.splits);
    const int tiles_per_img = a.res * a.res / 64;
    if (tid == 0) {
        for (int i = 0; i < nst; ++i) {
            hr_tma::mbar_init(&full[i], 1);
            hr_tma::mbar_init(&empty[i], 1);
        }
        hr_tma::mbar_init(&accf, 1);
        hr_tma::mbar_init(&drain, 1);
        abort_s = 0;
        hr_tma::fence_mbar_init();
    }
    if (warp == 1) hr_tc::tmem_alloc(&tmem_base, TMEM_COLS);
    hr_tc::fence_before_sync();
    __syncthreads();
    hr_tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    if (k1 > k0) {
        if (warp == 0) {
            if (lane == 0) {   // producer: per K tile the x tile and the 9 shifted dy tiles
                int it = 0;
                for (int kt = k0; kt < k1 && !*abort; ++kt, ++it) {
                    const int s = it % nst, k = it / nst;
                    if (k >= 1 && !tmaconv::wait(&empty[s], (k - 1) & 1, abort)) break;
                    unsigned char *base = smem + s * STAGE;
                    const int n = kt / tiles_per_img, p0 = (kt - n * tiles_per_img) * 64;
                    hr_tma::mbar_arrive_expect_tx(&full[s], STAGE);
                    hr_tma::load_4d(base, &tmX, &full[s], p0, n, cb * 128, 0);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int ty = tap / 3 - 1, tx = tap % 3 - 1;   // off(tap) = (ty, tx)
                        const CUtensorMap *tm = tx < 0 ? &tmD0 : (tx == 0 ? &tmD1 : &tmD2);
                        hr_tma::load_4d(base + A_BYTES + tap * B_BYTES, tm, &full[s], p0 - ty * a.res, n, ob * NB, 0);
                    }
                }
                if (*abort) {   // copies still in flight land before the CTA leaves (bounded)
                    for (int j = it - nst < 0 ? 0 : it - nst; j < it; ++j)
                        (void)hr_tma::mbar_wait(&full[j % nst], (j / nst) & 1);
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {   // MMA issuer: D += A B^T, 4 K steps of 16 pixels
                // the nine B tiles are consecutive rows of one K-major matrix (tap, output channel): one
                // MMA covers taps [0, T0) and, where 9 NB > 256, a second one taps [T0, 9)
                constexpr int T0 = 9 * NB <= 256 ? 9 : 256 / NB;
                constexpr uint32_t idesc0 = hr_tc::idesc_bf16(128, T0 * NB);
                constexpr uint32_t idesc1 = hr_tc::idesc_bf16(128, T0 < 9 ? (9 - T0) * NB : 16);
                static_assert((T0 * NB) % 16 == 0 && ((9 - T0) * NB) % 16 == 0, "MMA widths of 16-column steps");
                int it = 0;
                bool ok = true;
                for (int kt = k0; kt < k1 && !*abort; ++kt, ++it) {
                    const int s = it % nst, k = it / nst;
                    if (!tmaconv::wait(&full[s], k & 1, abort)) {
                        ok = false;
                        break;
                    }
                    hr_tc::fence_after_sync();
                    const uint32_t sa = hr_tma::smem_u32(smem + s * STAGE);
                    const uint64_t ad = hr_tc::smem_desc_swz(sa, 128);
                    const uint64_t bd0 = hr_tc::smem_desc_swz(sa + A_BYTES, 128);
                    const uint64_t bd1 = hr_tc::smem_desc_swz(sa + A_BYTES + T0 * B_BYTES, 128);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t acc = (kt > k0 || kk > 0) ? 1u : 0u;
                        hr_tc::mma_bf16(tb, ad + 2u * kk, bd0 + 2u * kk, idesc0, acc);
                        if (T0 < 9) hr_tc::mma_bf16(tb + (uint32_t)(T0 * NB), ad + 2u * kk, bd1 + 2u * kk, idesc1, acc);
                    }
                    hr_tc::commit(&empty[s]);
                }
                if (ok) hr_tc::commit(&accf);
            }
        } else {   // epilogue: warps 2-5, TMEM lane quadrant warp % 4 = 32 input channels
            const int quad = warp & 3;
            const bool got = tmaconv::wait(&accf, 0, abort);
            if (__all_sync(0xffffffffu, got)) {
                hr_tc::fence_after_sync();
                const int c = cb * 128 + quad * 32 + lane;
                for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
                    for (int j0 = 0; j0 < NB; j0 += 16) {
                        float v[16];
                        hr_tc::ld16(tb + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tap * NB + j0), v);
                        if (c < a.cin) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const int o = ob * NB + j0 + j;
                                if (o < a.cout) atomicAdd(a.dw + ((size_t)o * 9 + tap) * a.cin + c, v[j]);
                            }
                        }
                    }
                }
            }
        }
    }
    // an MMA thread that gave up may leave MMAs in flight: let them finish before TMEM is freed
    hr_tc::fence_before_sync();
    __syncthreads();
    if (*abort) {
        if (tid == 32) {
            hr_tc::commit(&drain);   // arrives once every MMA issued so far has completed
            (void)hr_tma::mbar_wait(&drain, 0);
        }
        if (tid == 0) atomicExch(err, 1);
        __syncthreads();
    }
    hr_tc::fence_after_sync();
    if (warp == 1) hr_tc::tmem_dealloc(tb, TMEM_COLS);
}

}  // namespace hr_cnn
