// a2-a4, a9: batched multi-resolution demons registration (Section 1, Eq. 1).
//
// Data layout (HBM): every buffer is pair-major.  Images are [B][h][w]
// FP32; the internal field buffers are [B][h][w] float2 (u_x, u_y
// interleaved), so that one 8-byte access moves both components and the two
// planes of every stencil run through packed FP32x2 FMAs.  The caller's
// field is the planar [B][2][h][w] of the ABI; only the last step writes it.
// The reference pyramid ([R][h][w], a few grains) is small and stays in L2;
// the per-pair test pyramid and the field buffers stream from HBM.
//
// One demons iteration u_{k+1} = G_f * (u_k + G_u * du(u_k)) is ONE fused
// kernel launch over every (active pair, tile) (tile shapes 64x64, 64x32,
// 32x32, 64x16, autotuned per level size).  The launch stores the
// unsmoothed field s_{k+1} = u_k + G_u * du(u_k) instead of u_{k+1}; the next
// launch recomputes u_{k+1} = G_f * s_{k+1} on the fly from a tile with a
// 2r halo (r the Gaussian radius).  This keeps the expensive part (warp +
// force) on a halo of r instead of 2r and saves a separate smoothing pass.
// Per pixel-iteration HBM sees the test image (4 B) and s (8 B) read and s
// (8 B) written; the bilinear gathers of the moving image hit the
// L2-resident reference pyramid.  The separable passes keep a sliding window
// of RUN + 2r samples per thread in registers (RUN outputs per thread) and
// use packed FP32x2 FMAs for the two field components.
//
// Border handling: every Gaussian pass has replicated borders.  The passes
// read s and du at clamped positions (plain path: clamped addresses; TMA
// path: clamped shared-memory indices on tiles that reach outside the image)
// and the test image's out-of-image values are those of the nearest in-image
// pixel; with that, every value the passes read at an in-image position is
// exact, and out-of-image values are never consumed by an in-image output.
//
// Uneven work (a9): pairs stop independently (stop rule on the SSD history).
// A small control kernel after each iteration compacts the list of active
// pairs; the iteration kernel is persistent (grid = SMs x resident CTAs) and
// walks the (active pair, tile) work list, so stopped pairs cost nothing.
#include <math.h>
#include <string.h>

#include <atomic>
#include <type_traits>

#include "internal.cuh"
#include "tma.cuh"

int hr_launch_reduce2(hrebsd_ctx *ctx, const float *in, float *out, int n, int H, int W, cudaStream_t st);

namespace {

constexpr int TX = 64;           // tile width (outputs)
constexpr int TY = 32;           // tile height
constexpr int RUN = 8;           // outputs per thread in a separable pass
constexpr int kIterThreads = 256;
constexpr int kMaxRad = 6;

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }
// Row stride (in float2) with an odd number of 16-byte slots, so that float4
// accesses of consecutive rows by consecutive threads hit distinct banks.
__host__ __device__ constexpr int pad_stride(int n) { return (n % 4 == 2) ? n : n + 2; }

struct Taps {
    float up[2 * kMaxRad + 1];   // G_u (update smoothing), centred at index RAD
    float f[2 * kMaxRad + 1];    // G_f (field smoothing)
};

struct IterArgs {
    const float *Ftest;      // test level images [B][h][w]
    const float *Mref;       // reference level images [R][h][w]
    const int *ref_idx;      // [B]
    const float2 *in;        // k == 0: u_0 [B][h][w]; k > 0: s_k
    float2 *out;             // s_{k+1}
    float *part;             // SSD partials [B][tiles]
    const int *active;       // active pair list
    const int *n_active;     // its length
    int *n_next_reset;       // counter of the next list, zeroed by this launch
    unsigned long long *px_count;   // tracing: pixel-iterations (NULL = off)
    int *err;                       // set to 1 when a bounded wait gives up
    int h, w, tiles_x, tiles;
    int in_is_s;
    float alpha2;
    Taps taps;
    // row sweep: texture over the level's reference images stacked as R x h rows of w (a CUDA array;
    // reference r's row y is texture row r h + y), 0 = plain loads from Mref
    unsigned long long mtex = 0;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Cell and weight of the clamped bilinear sample along one axis at the point
// q - u (q an integer pixel index, u the displacement; the warp M(x - u(x))).
// The point is split into integer and fraction from the displacement itself:
// with n = floor(-u) and f = -u - n the point is (q + n) + f, so the weight
// keeps the full FP32 precision of u instead of that of q - u (whose unit in
// the last place is 1.5e-5 px at q ~ 200, an error the iteration amplifies at
// weakly textured pixels).  Clamping the point to [0, m - 1]: the cell index
// is clamped to [0, m - 2], and the weight becomes 0 below the image and 1
// beyond it (exactly the clamped point's cell and weight).
__device__ __forceinline__ void warp_cell(int q, float u, int m, int &i, float &f)
{
    const float n = floorf(-u);
    const float fr = -u - n;                            // in [0, 1]
    const float x = (float)q + n;                       // integer-valued, exact
    const float xc = fminf(fmaxf(x, 0.0f), (float)(m - 2));
    f = __saturatef(fr + (x - xc));                     // fr inside, 0 / 1 when clamped
    i = (int)xc;
}

// warp_cell with the pixel index q and the largest cell index m - 2 given as
// floats (integer-valued, exact): the same cell and weight.
__device__ __forceinline__ void warp_cell_f(float q, float u, float m2, int &i, float &f)
{
    const float n = floorf(-u);
    const float fr = -u - n;
    const float x = q + n;
    const float xc = fminf(fmaxf(x, 0.0f), m2);
    f = __saturatef(fr + (x - xc));
    i = (int)xc;
}

// warp_cell_f with the cell index returned as a float (integer-valued, exact): the texture
// coordinate of the cell's four-texel gather.  Same cell and weight.
__device__ __forceinline__ void warp_cell_ff(float q, float u, float m2, float &xc, float &f)
{
    const float n = floorf(-u);
    const float fr = -u - n;
    const float x = q + n;
    xc = fminf(fmaxf(x, 0.0f), m2);
    f = __saturatef(fr + (x - xc));
}

// Bilinear sample of M at the point (qx - ux, qy - uy), clamped to the image;
// (1 - f) a + f b per axis, exact at the nodes.
__device__ __forceinline__ float warp_sample(const float *__restrict__ M, int h, int w, int qx, int qy, float ux,
                                             float uy)
{
    int x0, y0;
    float fx, fy;
    warp_cell(qx, ux, w, x0, fx);
    warp_cell(qy, uy, h, y0, fy);
    const float *p = M + y0 * w + x0;
    float a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + w), d = __ldg(p + w + 1);
    float top = fmaf(fx, b, (1.0f - fx) * a);
    float bot = fmaf(fx, d, (1.0f - fx) * c);
    return fmaf(fy, bot, (1.0f - fy) * top);
}

__device__ __forceinline__ float2 bilinear2_clamped(const float2 *__restrict__ M, int h, int w, float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    int x0 = min((int)x, w - 2);
    int y0 = min((int)y, h - 2);
    float fx = x - (float)x0, fy = y - (float)y0;
    const float2 *p = M + y0 * w + x0;
    float2 a = p[0], b = p[1], c = p[w], d = p[w + 1];
    float2 top = make_float2(fmaf(fx, b.x, (1.0f - fx) * a.x), fmaf(fx, b.y, (1.0f - fx) * a.y));
    float2 bot = make_float2(fmaf(fx, d.x, (1.0f - fx) * c.x), fmaf(fx, d.y, (1.0f - fx) * c.y));
    return make_float2(fmaf(fy, bot.x, (1.0f - fy) * top.x), fmaf(fy, bot.y, (1.0f - fy) * top.y));
}

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Two warp samples (the same arithmetic as warp_sample, each rounding step
// identical) with the interpolation done in packed FP32x2 operations.
// 1 - f is formed as fma(f, -1, 1), which rounds like the subtraction.
__device__ __forceinline__ float2 warp_sample_pair(const float *__restrict__ M, int h, int w, int qxa, int qya,
                                                   float2 ua, int qxb, int qyb, float2 ub)
{
    int xa0, ya0, xb0, yb0;
    float fxa, fya, fxb, fyb;
    warp_cell(qxa, ua.x, w, xa0, fxa);
    warp_cell(qya, ua.y, h, ya0, fya);
    warp_cell(qxb, ub.x, w, xb0, fxb);
    warp_cell(qyb, ub.y, h, yb0, fyb);
    const float2 fx = make_float2(fxa, fxb), fy = make_float2(fya, fyb);
    const float *pa = M + ya0 * w + xa0, *pb = M + yb0 * w + xb0;
    const float2 A = make_float2(__ldg(pa), __ldg(pb)), Bv = make_float2(__ldg(pa + 1), __ldg(pb + 1));
    const float2 C = make_float2(__ldg(pa + w), __ldg(pb + w)), D = make_float2(__ldg(pa + w + 1), __ldg(pb + w + 1));
    const float2 n1 = make_float2(-1.0f, -1.0f), one = make_float2(1.0f, 1.0f);
    const float2 omx = __ffma2_rn(fx, n1, one), omy = __ffma2_rn(fy, n1, one);
    const float2 top = __ffma2_rn(fx, Bv, __fmul2_rn(omx, A));
    const float2 bot = __ffma2_rn(fx, D, __fmul2_rn(omx, C));
    return __ffma2_rn(fy, bot, __fmul2_rn(omy, top));
}

template <int RAD, int TX_ = TX, int TY_ = TY>
struct Geo {
    static constexpr int BW = TX_ + 2 * RAD, BH = TY_ + 2 * RAD;       // u and du (T + r)
    static constexpr int BWP = round_up(BW, RUN), BHP = round_up(BH, RUN);
    static constexpr int AW = TX_ + 4 * RAD, AH = TY_ + 4 * RAD;       // s (T + 2r)
    static constexpr int AHP = BHP + 2 * RAD;                        // rows read by padded y-pass runs
    static constexpr int AST = pad_stride(BWP + 2 * RAD);            // s tile row stride (>= AW)
    static constexpr int XST = pad_stride(BWP);                      // x-pass of s row stride
    static constexpr int UST = BWP;                                  // u row stride
    static constexpr int DST = pad_stride(BWP);                      // du row stride
    static constexpr int XDST = pad_stride(TX_);                      // x-pass of du row stride
    static constexpr int FW = BW + 2, FH = BH + 2;                   // test image (T + r + 1)
    static constexpr int SA = (AHP * AST > BH * DST) ? AHP * AST : BH * DST;   // float2
    static constexpr int SX = (AHP * XST > BH * XDST) ? AHP * XST : BH * XDST; // float2
    static constexpr int SU = BHP * UST;                                        // float2
    static constexpr int SF = FH * FW;                                          // float
    static constexpr size_t BYTES = (size_t)(SA + SX + SU) * 8 + (size_t)SF * 4;
};

// Separable pass over a run of RUN outputs along a row (x pass) of float2
// data: out[o] = sum_k t[k] in[o + k], k = 0..2r.  `in` and `out` 16-byte aligned.
template <int RAD>
__device__ __forceinline__ void run_x(const float2 *in, float2 *out, const float2 (&t)[2 * RAD + 1])
{
    constexpr int NW = RUN + 2 * RAD;
    float2 win[NW];
    const float4 *in4 = reinterpret_cast<const float4 *>(in);
#pragma unroll
    for (int j = 0; j < NW / 2; ++j) {
        float4 v = in4[j];
        win[2 * j] = make_float2(v.x, v.y);
        win[2 * j + 1] = make_float2(v.z, v.w);
    }
    // tap-outer order: RUN independent accumulation chains per step (the sum
    // order of every output is still k = 0 .. 2r)
    float2 acc[RUN];
#pragma unroll
    for (int o = 0; o < RUN; ++o) acc[o] = __fmul2_rn(t[0], win[o]);
#pragma unroll
    for (int k = 1; k <= 2 * RAD; ++k)
#pragma unroll
        for (int o = 0; o < RUN; ++o) acc[o] = ffma2(t[k], win[o + k], acc[o]);
    float4 *out4 = reinterpret_cast<float4 *>(out);
#pragma unroll
    for (int o = 0; o < RUN; o += 2) out4[o / 2] = make_float4(acc[o].x, acc[o].y, acc[o + 1].x, acc[o + 1].y);
}

// Same along a column: in[j * stride], j = 0..RUN + 2r - 1 -> acc[o].
// run_x on a row whose columns outside [lo, hi] stand for the nearest of them
// (the window is read column by column through clamped indices; same sums).
template <int RAD>
__device__ __forceinline__ void run_x_clamped(const float2 *row, int c0, int lo, int hi, float2 *out,
                                              const float2 (&t)[2 * RAD + 1])
{
    constexpr int NW = RUN + 2 * RAD;
    float2 win[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) win[j] = row[min(max(c0 + j, lo), hi)];
    float2 acc[RUN];
#pragma unroll
    for (int o = 0; o < RUN; ++o) acc[o] = __fmul2_rn(t[0], win[o]);
#pragma unroll
    for (int k = 1; k <= 2 * RAD; ++k)
#pragma unroll
        for (int o = 0; o < RUN; ++o) acc[o] = ffma2(t[k], win[o + k], acc[o]);
    float4 *out4 = reinterpret_cast<float4 *>(out);
#pragma unroll
    for (int o = 0; o < RUN; o += 2) out4[o / 2] = make_float4(acc[o].x, acc[o].y, acc[o + 1].x, acc[o + 1].y);
}

template <int RAD>
__device__ __forceinline__ void run_y(const float2 *in, int stride, const float2 (&t)[2 * RAD + 1], float2 (&acc)[RUN])
{
    constexpr int NW = RUN + 2 * RAD;
    float2 win[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) win[j] = in[j * stride];
#pragma unroll
    for (int o = 0; o < RUN; ++o) acc[o] = __fmul2_rn(t[0], win[o]);
#pragma unroll
    for (int k = 1; k <= 2 * RAD; ++k)
#pragma unroll
        for (int o = 0; o < RUN; ++o) acc[o] = ffma2(t[k], win[o + k], acc[o]);
}

// One item of work: a tile of one active pair.
struct TileRef {
    int pair, tile, x0, y0;
};

template <int TX_ = TX, int TY_ = TY>
__device__ __forceinline__ TileRef tile_of(const IterArgs &a, long long item)
{
    TileRef t;
    t.pair = a.active[item / a.tiles];
    t.tile = (int)(item % a.tiles);
    t.x0 = (t.tile % a.tiles_x) * TX_;
    t.y0 = (t.tile / a.tiles_x) * TY_;
    return t;
}

// IN_S: the input is s (k > 0) and u = G_f * s is formed from an s tile with a
// 2r halo; otherwise the input is u itself (first iteration of a level).
// The input and test-image tiles of the NEXT item are loaded into registers
// while the current item is computed (register-staged prefetch), so their
// latency overlaps the passes instead of stalling the CTA.
template <int RAD, bool IN_S>
__global__ void __launch_bounds__(kIterThreads, 2) demons_iter_kernel(IterArgs a)
{
    using L = Geo<RAD>;
    constexpr int NT = kIterThreads;
    constexpr bool SMOOTH_IN = IN_S && RAD > 0;
    constexpr int IW = SMOOTH_IN ? L::AW : L::BW;     // input tile columns
    constexpr int IH = SMOOTH_IN ? L::AH : L::BH;     // input tile rows
    constexpr int IOFF = SMOOTH_IN ? 2 * RAD : RAD;   // input tile halo
    constexpr int IST = SMOOTH_IN ? L::AST : L::UST;  // its shared-memory row stride
    constexpr int NIN = IW * IH, NPI = (NIN + NT - 1) / NT;
    constexpr int NF = L::FW * L::FH, NPF = (NF + NT - 1) / NT;
    constexpr int NPTS = L::BW * L::BH;

    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sA = reinterpret_cast<float2 *>(smraw);   // s tile, later du
    float2 *sX = sA + L::SA;                          // x-pass results
    float2 *sU = sX + L::SX;                          // u on T + r
    float *sF = reinterpret_cast<float *>(sU + L::SU);   // test image on T + r + 1
    float2 *sIn = SMOOTH_IN ? sA : sU;
    __shared__ float red[NT / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 tf[2 * RAD + 1], tu[2 * RAD + 1];
#pragma unroll
    for (int k = 0; k <= 2 * RAD; ++k) {
        tf[k] = make_float2(a.taps.f[k], a.taps.f[k]);
        tu[k] = make_float2(a.taps.up[k], a.taps.up[k]);
    }
    const int n_active = *a.n_active;
    if (blockIdx.x == 0 && tid == 0) {
        *a.n_next_reset = 0;
        if (a.px_count) atomicAdd(a.px_count, (unsigned long long)n_active * a.h * a.w);
    }
    const long long work = (long long)n_active * a.tiles;
    const int h = a.h, w = a.w;
    const size_t plane = (size_t)h * w;

    float2 pin[NPI];
    float pf[NPF];
    auto fetch = [&](const TileRef &t) {
        const float2 *src = a.in + (size_t)t.pair * plane;
        const float *Fimg = a.Ftest + (size_t)t.pair * plane;
#pragma unroll
        for (int j = 0; j < NPI; ++j) {
            const int idx = tid + j * NT;
            if (idx < NIN) {
                const int r = idx / IW, c = idx - r * IW;
                const int gy = clampi(t.y0 - IOFF + r, 0, h - 1), gx = clampi(t.x0 - IOFF + c, 0, w - 1);
                pin[j] = __ldg(src + (size_t)gy * w + gx);
            }
        }
#pragma unroll
        for (int j = 0; j < NPF; ++j) {
            const int idx = tid + j * NT;
            if (idx < NF) {
                const int r = idx / L::FW, c = idx - r * L::FW;
                const int gy = clampi(t.y0 - RAD - 1 + r, 0, h - 1), gx = clampi(t.x0 - RAD - 1 + c, 0, w - 1);
                pf[j] = __ldg(Fimg + (size_t)gy * w + gx);
            }
        }
    };
    auto commit = [&]() {
#pragma unroll
        for (int j = 0; j < NPI; ++j) {
            const int idx = tid + j * NT;
            if (idx < NIN) {
                const int r = idx / IW, c = idx - r * IW;
                sIn[r * IST + c] = pin[j];
            }
        }
#pragma unroll
        for (int j = 0; j < NPF; ++j) {
            const int idx = tid + j * NT;
            if (idx < NF) sF[idx] = pf[j];
        }
    };

    long long item = blockIdx.x;
    if (item < work) {
        fetch(tile_of(a, item));
        commit();
    }
    for (; item < work; item += gridDim.x) {
        __syncthreads();   // the tiles of `item` are in shared memory
        const TileRef cur = tile_of(a, item);
        const long long next = item + gridDim.x;
        if (next < work) fetch(tile_of(a, next));   // in flight during this item
        const int x0 = cur.x0, y0 = cur.y0;
        const float *M = a.Mref + (size_t)__ldg(a.ref_idx + cur.pair) * plane;

        if (SMOOTH_IN) {
            // ---- u = G_f * s on T + r: x pass (rows of T + 2r), then y pass
            constexpr int NSX = L::BWP / RUN;
            for (int it = tid; it < NSX * L::AHP; it += NT) {
                const int seg = it / L::AHP, row = it - seg * L::AHP;
                run_x<RAD>(sA + row * L::AST + seg * RUN, sX + row * L::XST + seg * RUN, tf);
            }
            __syncthreads();
            constexpr int NSY = L::BHP / RUN;
            for (int it = tid; it < NSY * L::BWP; it += NT) {
                const int seg = it / L::BWP, col = it - seg * L::BWP;
                float2 acc[RUN];
                run_y<RAD>(sX + seg * RUN * L::XST + col, L::XST, tf, acc);
#pragma unroll
                for (int o = 0; o < RUN; ++o) sU[(seg * RUN + o) * L::UST + col] = acc[o];
            }
            __syncthreads();
        }

        // ---- warp + force at the clamped position of every point of T + r
        float ssd = 0.0f;
        float2 *sD = sA;
        auto force = [&](int idx, float2 &du, float &d2) {
            const int r = idx / L::BW, c = idx - r * L::BW;
            const int vy = y0 - RAD + r, vx = x0 - RAD + c;
            const int qy = clampi(vy, 0, h - 1), qx = clampi(vx, 0, w - 1);
            const int qly = qy - (y0 - RAD), qlx = qx - (x0 - RAD);
            const float2 u = sU[qly * L::UST + qlx];
            const float *fc = sF + (qly + 1) * L::FW + (qlx + 1);
            const int xl = qx > 0 ? -1 : 0, xr = qx < w - 1 ? 1 : 0;
            const int yl = qy > 0 ? -L::FW : 0, yr = qy < h - 1 ? L::FW : 0;
            const float gx = (fc[xr] - fc[xl]) * ((xr - xl) == 2 ? 0.5f : 1.0f);
            const float gy = (fc[yr] - fc[yl]) * ((yr - yl) == 2 * L::FW ? 0.5f : 1.0f);
            const float mw = warp_sample(M, h, w, qx, qy, u.x, u.y);
            const float d = mw - fc[0];
            const float den = fmaf(gx, gx, fmaf(gy, gy, a.alpha2 * d * d));
            const float t = den > 1e-9f ? __fdividef(d, den) : 0.0f;
            du = make_float2(t * gx, t * gy);
            const bool in_T = r >= RAD && r < RAD + TY && c >= RAD && c < RAD + TX && vy < h && vx < w;
            d2 = in_T ? d * d : 0.0f;
        };
        for (int i0 = tid; i0 < NPTS; i0 += 2 * NT) {
            const int i1 = i0 + NT;
            float2 du0, du1 = make_float2(0.0f, 0.0f);
            float e0, e1 = 0.0f;
            force(i0, du0, e0);
            if (i1 < NPTS) force(i1, du1, e1);
            sD[(i0 / L::BW) * L::DST + i0 % L::BW] = du0;
            if (i1 < NPTS) sD[(i1 / L::BW) * L::DST + i1 % L::BW] = du1;
            ssd += e0 + e1;
        }
        __syncthreads();
        // ---- G_u * du: x pass on rows of T + r, columns of T
        constexpr int NSXD = TX / RUN;
        for (int it = tid; it < NSXD * L::BH; it += NT) {
            const int seg = it / L::BH, row = it - seg * L::BH;
            run_x<RAD>(sD + row * L::DST + seg * RUN, sX + row * L::XDST + seg * RUN, tu);
        }
        __syncthreads();
        // ---- y pass, s_{k+1} = u_k + G_u * du on T
        float2 *dst = a.out + (size_t)cur.pair * plane;
        for (int it = tid; it < (TY / RUN) * TX; it += NT) {
            const int seg = it / TX, col = it - seg * TX;
            float2 acc[RUN];
            run_y<RAD>(sX + seg * RUN * L::XDST + col, L::XDST, tu, acc);
            const int gx = x0 + col;
#pragma unroll
            for (int o = 0; o < RUN; ++o) {
                const int gy = y0 + seg * RUN + o;
                if (gy < h && gx < w) {
                    const float2 u = sU[(seg * RUN + o + RAD) * L::UST + col + RAD];
                    dst[(size_t)gy * w + gx] = __fadd2_rn(u, acc[o]);
                }
            }
        }
        // ---- SSD partial of this tile; then the prefetched tiles go to shared memory
        for (int o = 16; o > 0; o >>= 1) ssd += __shfl_xor_sync(0xffffffffu, ssd, o);
        if (lane == 0) red[warp] = ssd;
        __syncthreads();
        if (tid == 0) {
            float t = 0.0f;
            for (int i = 0; i < NT / 32; ++i) t += red[i];
            a.part[(size_t)cur.pair * a.tiles + cur.tile] = t;
        }
        if (next < work) commit();
    }
}

// ---------------------------------------------------------------------------
// TMA-fed iteration (every iteration for r = 3, k > 0 for other radii; the
// first iteration of a level reads u_0 instead of s).  The s tile (T + 2r,
// padded) and the test image tile (T + r + 1, widened to 16-byte-aligned
// columns) arrive by bulk tensor copies issued by one thread, so the other
// threads spend no instructions on loads: the s copy for the next item is
// issued as soon as the x pass has consumed the current s tile, the
// test-image copy as soon as the force stage has consumed the current one.
// The copy fills out-of-image elements with zeros; on border tiles the x
// passes read s and du through clamped indices and the test image's
// out-of-image elements are filled from the nearest in-image ones (the
// clamped-address semantics of the plain path).  The force stage works on
// vertical runs of 4 pixels per thread with the gradient stencil and field
// read once per run.
template <int RAD, int TX_, int TY_>
struct GeoT {
    using L = Geo<RAD, TX_, TY_>;
    static constexpr int FOFF = 4 * ((RAD + 1 + 3) / 4);   // test-image halo, rounded to 16 bytes
    static constexpr int FWB = TX_ + 2 * FOFF;               // test-image tile columns
    static constexpr int FH = L::FH;
    static constexpr uint32_t S_BYTES = (uint32_t)L::AHP * L::AST * 8;
    static constexpr uint32_t F_BYTES = (uint32_t)FH * FWB * 4;
    static constexpr int S_OFF = 0;
    static constexpr int F_OFF = (int)round_up((int)S_BYTES, 128);
    static constexpr int X_OFF = F_OFF + (int)round_up((int)F_BYTES, 128);
    static constexpr int U_OFF = X_OFF + L::SX * 8;
    static constexpr int D_OFF = U_OFF + L::SU * 8;
    static constexpr size_t BYTES = (size_t)D_OFF + (size_t)L::BH * L::DST * 8;
};

// Replicate out-of-image rows, then columns, of a tile whose rows cover global
// [g0r, g0r + nr) and columns [g0c, g0c + nc) (element type T, row stride st).
template <typename T>
__device__ __forceinline__ void fix_rows(T *t, int st, int nr, int nc, int g0r, int nimg)
{
    const int top = max(0, -g0r), bot = max(0, g0r + nr - nimg);
    if (!(top | bot)) return;
    for (int idx = threadIdx.x; idx < (top + bot) * nc; idx += blockDim.x) {
        const int k = idx / nc, c = idx - k * nc;
        const int dr = k < top ? k : nr - bot + (k - top);
        const int sr = k < top ? top : nr - bot - 1;
        t[dr * st + c] = t[sr * st + c];
    }
}

template <typename T>
__device__ __forceinline__ void fix_cols(T *t, int st, int nr, int nc, int g0c, int nimg)
{
    const int left = max(0, -g0c), right = max(0, g0c + nc - nimg);
    if (!(left | right)) return;
    const int n = left + right;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        const int row = idx / n, k = idx - row * n;
        const int dc = k < left ? k : nc - right + (k - left);
        const int sc = k < left ? left : nc - right - 1;
        t[row * st + dc] = t[row * st + sc];
    }
}

// Replicate edges in one pass: every element of the tile outside the image
// (rows [g0r, g0r + nr) and columns [g0c, g0c + nc) in image coordinates)
// takes the value at the nearest in-image row and column.  Sources are
// in-image elements, which are never written, so no barrier is needed between
// rows and columns (the result equals fix_rows followed by fix_cols).
template <typename T>
__device__ __forceinline__ void fix_frame(T *t, int st, int nr, int nc, int g0r, int g0c, int himg, int wimg)
{
    const int top = max(0, -g0r), bot = max(0, g0r + nr - himg);
    const int left = max(0, -g0c), right = max(0, g0c + nc - wimg);
    const int rhi = nr - bot - 1, chi = nc - right - 1;
    const int n1 = (top + bot) * nc, ncol = left + right, n = n1 + (nr - top - bot) * ncol;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        int r, c;
        if (idx < n1) {
            const int k = idx / nc;
            c = idx - k * nc;
            r = k < top ? k : nr - bot + (k - top);
        } else {
            const int q = idx - n1, k = q / ncol, m = q - k * ncol;
            r = top + k;
            c = m < left ? m : nc - right + (m - left);
        }
        t[r * st + c] = t[min(max(r, top), rhi) * st + min(max(c, left), chi)];
    }
}

// IN_S: the input is s_k (u = G_f * s); false for the first iteration of a
// level, whose input is the prolonged field u_0 itself.
template <int RAD, int TX_, int TY_, int MINB, int NT_, int FR, bool IN_S = true>
__global__ void __launch_bounds__(NT_, MINB) demons_iter_tma_kernel(const __grid_constant__ CUtensorMap tmS,
                                                                             const __grid_constant__ CUtensorMap tmF,
                                                                             IterArgs a)
{
    using L = Geo<RAD, TX_, TY_>;
    using G = GeoT<RAD, TX_, TY_>;
    constexpr int NT = NT_;
    extern __shared__ __align__(1024) unsigned char smraw[];
    float2 *sS = reinterpret_cast<float2 *>(smraw + G::S_OFF);   // [AHP][AST]
    float *sF = reinterpret_cast<float *>(smraw + G::F_OFF);     // [FH][FWB]
    float2 *sX = reinterpret_cast<float2 *>(smraw + G::X_OFF);
    float2 *sU = reinterpret_cast<float2 *>(smraw + G::U_OFF);   // [BHP][UST]
    float2 *sD = reinterpret_cast<float2 *>(smraw + G::D_OFF);   // [BH][DST]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float red[NT / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 tf[2 * RAD + 1], tu[2 * RAD + 1];
#pragma unroll
    for (int k = 0; k <= 2 * RAD; ++k) {
        tf[k] = make_float2(a.taps.f[k], a.taps.f[k]);
        tu[k] = make_float2(a.taps.up[k], a.taps.up[k]);
    }
    const int n_active = *a.n_active;
    if (blockIdx.x == 0 && tid == 0) {
        *a.n_next_reset = 0;
        if (a.px_count) atomicAdd(a.px_count, (unsigned long long)n_active * a.h * a.w);
    }
    const long long work = (long long)n_active * a.tiles;
    const int h = a.h, w = a.w;
    const size_t plane = (size_t)h * w;
    if (tid == 0) {
        hr_tma::mbar_init(&bar[0], 1);
        hr_tma::mbar_init(&bar[1], 1);
        hr_tma::fence_mbar_init();
    }
    __syncthreads();
    auto issue_S = [&](const TileRef &t) {
        hr_tma::mbar_arrive_expect_tx(&bar[0], G::S_BYTES);
        hr_tma::load_3d(sS, &tmS, &bar[0], 2 * (t.x0 - 2 * RAD), t.y0 - 2 * RAD, t.pair);
    };
    auto issue_F = [&](const TileRef &t) {
        hr_tma::mbar_arrive_expect_tx(&bar[1], G::F_BYTES);
        hr_tma::load_3d(sF, &tmF, &bar[1], t.x0 - G::FOFF, t.y0 - RAD - 1, t.pair);
    };
    // The item's tile is decoded once, by thread 0 when it issues the item's copies, and read by
    // all threads from shared memory after the barrier that opens the item (thread 0 overwrites it
    // with the next item only after a later barrier of the current one).
    __shared__ TileRef s_tile;
    __shared__ int s_ref, s_border;
    long long item = blockIdx.x;
    TileRef tn;   // thread 0: the next item
    auto publish = [&](const TileRef &t) {
        s_tile = t;
        s_ref = __ldg(a.ref_idx + t.pair);
        // tiles whose s or test-image box reaches outside the image get their edges replicated
        s_border = t.x0 - 2 * RAD < 0 || t.x0 - 2 * RAD + L::AST > w || t.y0 - 2 * RAD < 0 ||
                   t.y0 - 2 * RAD + L::AHP > h || t.x0 - G::FOFF < 0 || t.x0 - G::FOFF + G::FWB > w ||
                   t.y0 - RAD - 1 < 0 || t.y0 - RAD - 1 + G::FH > h;
    };
    if (tid == 0 && item < work) {
        tn = tile_of<TX_, TY_>(a, item);
        publish(tn);
        issue_S(tn);
        issue_F(tn);
    }
    uint32_t phase = 0;
    // thread 0: the SSD partial of the previous item, summed from red[] after the barrier that
    // opens the next item (or the one after the loop), so no barrier closes an item
    int prev_pair = -1, prev_tile = 0;
    auto write_partial = [&]() {
        float t = 0.0f;
        for (int i = 0; i < NT / 32; ++i) t += red[i];
        a.part[(size_t)prev_pair * a.tiles + prev_tile] = t;
    };
    for (; item < work; item += gridDim.x) {
        const long long next = item + gridDim.x;
        bool ok = hr_tma::mbar_wait(&bar[0], phase);
        ok = hr_tma::mbar_wait(&bar[1], phase) && ok;
        if (!__syncthreads_and(ok)) {
            if (tid == 0) atomicExch(a.err, 1);
            return;
        }
        if (tid == 0 && prev_pair >= 0) write_partial();
        phase ^= 1u;
        const TileRef cur = s_tile;
        const int x0 = cur.x0, y0 = cur.y0;
        const float *M = a.Mref + (size_t)s_ref * plane;
        // ---- tiles that reach outside the image
        const bool border = s_border != 0;
        // (the test-image tile is read in the force stage: its out-of-image elements are filled
        // here, before the barrier that ends the x pass; the s tile is read only by the x pass,
        // which goes through clamped indices on border tiles; u_0 is read directly, so its tile
        // is filled too, followed by a barrier)
        if (border) {
            fix_frame(sF, G::FWB, G::FH, G::FWB, y0 - RAD - 1, x0 - G::FOFF, h, w);
            if constexpr (!IN_S) {
                fix_frame(sS, L::AST, L::AHP, L::AST, y0 - 2 * RAD, x0 - 2 * RAD, h, w);
                __syncthreads();
            }
        }
        // ---- u = G_f * s on T + r
        if constexpr (IN_S) {
            constexpr int NSX = L::BWP / RUN;
            if (!border) {
                for (int it = tid; it < NSX * L::AHP; it += NT) {
                    const int seg = it / L::AHP, row = it - seg * L::AHP;
                    run_x<RAD>(sS + row * L::AST + seg * RUN, sX + row * L::XST + seg * RUN, tf);
                }
            } else {   // s outside the image = s at the clamped position
                const int rlo = max(0, 2 * RAD - y0), rhi = L::AHP - 1 - max(0, y0 - 2 * RAD + L::AHP - h);
                const int clo = max(0, 2 * RAD - x0), chi = L::AST - 1 - max(0, x0 - 2 * RAD + L::AST - w);
                for (int it = tid; it < NSX * L::AHP; it += NT) {
                    const int seg = it / L::AHP, row = it - seg * L::AHP;
                    const int rs = min(max(row, rlo), rhi), c0 = seg * RUN;
                    if (c0 >= clo && c0 + RUN + 2 * RAD - 1 <= chi)
                        run_x<RAD>(sS + rs * L::AST + c0, sX + row * L::XST + c0, tf);
                    else
                        run_x_clamped<RAD>(sS + rs * L::AST, c0, clo, chi, sX + row * L::XST + c0, tf);
                }
            }
            __syncthreads();
            if (tid == 0 && next < work) {   // the s tile is consumed: fetch the next one
                tn = tile_of<TX_, TY_>(a, next);
                publish(tn);
                hr_tma::fence_proxy_async();
                issue_S(tn);
            }
        }
        // ---- (the y pass of G_f runs inside the force stage below, on each
        // thread's own column run; u on T + r is kept in sU for the last stage)

        // ---- warp + force on T + r, vertical runs of FR pixels (one column, FR
        // rows per thread; consecutive threads take consecutive columns, so the
        // moving-image gathers of a warp are row-contiguous and the shared-memory
        // accesses conflict-free).  Every run is computed the same way (no
        // divergent border path): the test-image tile has replicated borders, so
        // the central difference becomes the one-sided one at the image edge once
        // scaled by 1 instead of 1/2; du at points outside the image is computed
        // but never read (the x pass of du reads the clamped positions).  Rows of
        // the last group beyond T + r are computed from padding and discarded.
        float ssd = 0.0f;
        const int rows_in = min(TY_, h - y0);   // rows of T inside the image
        constexpr int NG = (L::BH + FR - 1) / FR;
        constexpr int FC = G::FOFF - RAD;   // test-image column of local column 0
        for (int it = tid; it < NG * L::BW; it += NT) {
            const int g = it / L::BW, c = it - g * L::BW;
            const int r0 = FR * g;
            const int vx = x0 - RAD + c, vy0 = y0 - RAD + r0;
            const bool colT = c >= RAD && c < RAD + TX_ && vx < w;
            // one-sided difference (scale 1) in the first and last column; columns outside the
            // image are computed from replicated data and discarded
            const float sx = (unsigned)(vx - 1) >= (unsigned)(w - 2) ? 1.0f : 0.5f;
            const float *fcol = sF + r0 * G::FWB + c + FC;   // test image, local rows r0 - 1 .. r0 + FR
            float fv[FR + 2], fl[FR], fr[FR];
#pragma unroll
            for (int j = 0; j < FR + 2; ++j) fv[j] = fcol[j * G::FWB];
#pragma unroll
            for (int i = 0; i < FR; ++i) {
                fl[i] = fcol[(i + 1) * G::FWB - 1];
                fr[i] = fcol[(i + 1) * G::FWB + 1];
            }
            float2 u[FR];
            if constexpr (!IN_S) {   // u_0 itself: the tile holds it with the same 2r halo as s
#pragma unroll
                for (int i = 0; i < FR; ++i) {
                    u[i] = sS[(r0 + i + RAD) * L::AST + c + RAD];
                    sU[(r0 + i) * L::UST + c] = u[i];
                }
            } else {   // y pass of G_f for rows r0 .. r0 + FR - 1 of column c (same sum order as run_y)
                static_assert(((L::BH + FR - 1) / FR) * FR <= L::BHP, "force runs stay inside sU");
                float2 win[FR + 2 * RAD];
#pragma unroll
                for (int j = 0; j < FR + 2 * RAD; ++j) win[j] = sX[(r0 + j) * L::XST + c];
#pragma unroll
                for (int i = 0; i < FR; ++i) u[i] = __fmul2_rn(tf[0], win[i]);
#pragma unroll
                for (int k = 1; k <= 2 * RAD; ++k)
#pragma unroll
                    for (int i = 0; i < FR; ++i) u[i] = ffma2(tf[k], win[i + k], u[i]);
#pragma unroll
                for (int i = 0; i < FR; ++i) sU[(r0 + i) * L::UST + c] = u[i];
            }
            // pixel pairs (i, i + 1) in packed FP32x2 arithmetic; every rounding step is the
            // scalar one (a - b as fma(b, -1, a), products and fmas in the same order)
            static_assert(FR % 2 == 0, "force runs are processed in pixel pairs");
            const float2 n1 = make_float2(-1.0f, -1.0f), sx2 = make_float2(sx, sx);
            const float2 al2 = make_float2(a.alpha2, a.alpha2);
#pragma unroll
            for (int i = 0; i < FR; i += 2) {
                const float2 mw = warp_sample_pair(M, h, w, vx, vy0 + i, u[i], vx, vy0 + i + 1, u[i + 1]);
                const int vya = vy0 + i, vyb = vya + 1;
                const float2 sy2 = make_float2((unsigned)(vya - 1) >= (unsigned)(h - 2) ? 1.0f : 0.5f,
                                               (unsigned)(vyb - 1) >= (unsigned)(h - 2) ? 1.0f : 0.5f);
                const float2 gx = __fmul2_rn(sx2, __ffma2_rn(make_float2(fl[i], fl[i + 1]), n1,
                                                             make_float2(fr[i], fr[i + 1])));
                const float2 gy = __fmul2_rn(sy2, __ffma2_rn(make_float2(fv[i], fv[i + 1]), n1,
                                                             make_float2(fv[i + 2], fv[i + 3])));
                const float2 d = __ffma2_rn(make_float2(fv[i + 1], fv[i + 2]), n1, mw);
                const float2 den = __ffma2_rn(gx, gx, __ffma2_rn(gy, gy, __fmul2_rn(__fmul2_rn(al2, d), d)));
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int r = r0 + i + j;
                    const float dj = j ? d.y : d.x, denj = j ? den.y : den.x;
                    const float t = denj > 1e-9f ? __fdividef(dj, denj) : 0.0f;
                    const float2 g = j ? make_float2(gx.y, gy.y) : make_float2(gx.x, gy.x);
                    if (L::BH % FR == 0 || r < L::BH) sD[r * L::DST + c] = __fmul2_rn(make_float2(t, t), g);
                    if (colT && (unsigned)(r - RAD) < (unsigned)rows_in) ssd = fmaf(dj, dj, ssd);
                }
            }
        }
        __syncthreads();
        if (tid == 0 && next < work) {   // the test-image tile (and u_0's) is consumed: fetch the next one
            if constexpr (!IN_S) {
                tn = tile_of<TX_, TY_>(a, next);
                publish(tn);
            }
            hr_tma::fence_proxy_async();
            if constexpr (!IN_S) issue_S(tn);
            issue_F(tn);
        }
        // ---- G_u * du: x pass on rows of T + r, columns of T.  du outside the image is du at the
        // clamped position: border tiles read rows and columns through clamped indices
        constexpr int NSXD = TX_ / RUN;
        if (!border) {
            for (int it = tid; it < NSXD * L::BH; it += NT) {
                const int seg = it / L::BH, row = it - seg * L::BH;
                run_x<RAD>(sD + row * L::DST + seg * RUN, sX + row * L::XDST + seg * RUN, tu);
            }
        } else {
            const int rlo = max(0, RAD - y0), rhi = L::BH - 1 - max(0, y0 - RAD + L::BH - h);
            const int clo = max(0, RAD - x0), chi = L::BW - 1 - max(0, x0 - RAD + L::BW - w);
            for (int it = tid; it < NSXD * L::BH; it += NT) {
                const int seg = it / L::BH, row = it - seg * L::BH;
                const int rs = min(max(row, rlo), rhi), c0 = seg * RUN;
                if (c0 >= clo && c0 + RUN + 2 * RAD - 1 <= chi)
                    run_x<RAD>(sD + rs * L::DST + c0, sX + row * L::XDST + c0, tu);
                else
                    run_x_clamped<RAD>(sD + rs * L::DST, c0, clo, chi, sX + row * L::XDST + c0, tu);
            }
        }
        __syncthreads();
        // ---- y pass, s_{k+1} = u_k + G_u * du on T
        float2 *dst = a.out + (size_t)cur.pair * plane;
        for (int it = tid; it < (TY_ / RUN) * TX_; it += NT) {
            const int seg = it / TX_, col = it - seg * TX_;
            float2 acc[RUN];
            run_y<RAD>(sX + seg * RUN * L::XDST + col, L::XDST, tu, acc);
            const int gx = x0 + col, gy0 = y0 + seg * RUN;
            if (gx < w) {
                const int nrow = h - gy0;   // rows of this run inside the image (may exceed RUN)
                float2 *p = dst + (size_t)gy0 * w + gx;
                const float2 *su = sU + (seg * RUN + RAD) * L::UST + col + RAD;
#pragma unroll
                for (int o = 0; o < RUN; ++o) {
                    if (o < nrow) p[(size_t)o * w] = __fadd2_rn(su[o * L::UST], acc[o]);
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) ssd += __shfl_xor_sync(0xffffffffu, ssd, o);
        if (lane == 0) red[warp] = ssd;
        if (tid == 0) {
            prev_pair = cur.pair;
            prev_tile = cur.tile;
        }
    }
    __syncthreads();
    if (tid == 0 && prev_pair >= 0) write_partial();
}

#include "demons_strip.cuh"
#include "demons_level.cuh"

struct CtrlArgs {
    const float *part;       // [B][tiles]
    double *hist;            // [B][hist_stride]
    const int *active;       // current list
    const int *n_active;
    int *next;               // next list
    int *n_next;
    int32_t *iters;          // [B][levels]
    int32_t *status;         // [B]
    int tiles, hist_stride, k, cap, window, level, levels;
    float tol;
};

// Stop rule of one level after iteration k (E_k complete in part[]).
__global__ void demons_control_kernel(CtrlArgs c)
{
    const int n = *c.n_active;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int p = c.active[i];
        double E = 0.0;
        const float *pp = c.part + (size_t)p * c.tiles;
        for (int t = 0; t < c.tiles; ++t) E += (double)pp[t];
        double *hh = c.hist + (size_t)p * c.hist_stride;
        hh[c.k] = E;
        int32_t *it = c.iters + (size_t)p * c.levels + c.level;
        if (!isfinite(E)) {
            *it = c.k;
            c.status[p] |= HREBSD_PAIR_NONFINITE;
        } else if (c.window > 0 && c.k >= c.window && (hh[c.k - c.window] - E) < (double)c.tol * hh[c.k - c.window]) {
            *it = c.k;
        } else if (c.k + 1 >= c.cap) {
            *it = c.cap;
            c.status[p] |= HREBSD_PAIR_CAPPED;
        } else {
            c.next[atomicAdd(c.n_next, 1)] = p;
        }
    }
}

// Final field of a level: u = u_0 when no update was applied, else G_f * s_n.
// PLANAR writes the ABI layout [B][2][h][w], otherwise interleaved float2.
template <int RAD, bool PLANAR>
__global__ void __launch_bounds__(256) demons_finalize_kernel(const float2 *u0, const float2 *s0, const float2 *s1,
                                                              const int32_t *iters, int levels, int level,
                                                              float *uout, int B, int h, int w, int tiles_x,
                                                              int tiles, Taps taps)
{
    constexpr int AW = TX + 2 * RAD, AH = TY + 2 * RAD;
    extern __shared__ __align__(16) unsigned char fin_smem[];
    float2 *sa = reinterpret_cast<float2 *>(fin_smem);   // [AH][AW]
    float2 *sx = sa + AW * AH;                            // [AH][TX]
    const size_t plane = (size_t)h * w;
    for (long long item = blockIdx.x; item < (long long)B * tiles; item += gridDim.x) {
        const int pair = (int)(item / tiles), tile = (int)(item % tiles);
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        const int n = iters[(size_t)pair * levels + level];
        const float2 *src = (n == 0 ? u0 : ((n & 1) ? s1 : s0)) + (size_t)pair * plane;
        auto put = [&](int gy, int gx, float2 v) {
            size_t g = (size_t)gy * w + gx;
            if (PLANAR) {
                uout[(size_t)pair * 2 * plane + g] = v.x;
                uout[(size_t)pair * 2 * plane + plane + g] = v.y;
            } else {
                reinterpret_cast<float2 *>(uout)[(size_t)pair * plane + g] = v;
            }
        };
        if (n == 0 || RAD == 0) {
            for (int idx = threadIdx.x; idx < TX * TY; idx += blockDim.x) {
                int gy = y0 + idx / TX, gx = x0 + idx % TX;
                if (gy < h && gx < w) put(gy, gx, src[(size_t)gy * w + gx]);
            }
            continue;
        }
        for (int idx = threadIdx.x; idx < AW * AH; idx += blockDim.x) {
            int ly = idx / AW, lx = idx - ly * AW;
            int gy = clampi(y0 - RAD + ly, 0, h - 1), gx = clampi(x0 - RAD + lx, 0, w - 1);
            sa[idx] = src[(size_t)gy * w + gx];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < AH * TX; idx += blockDim.x) {
            int ly = idx / TX, lx = idx - ly * TX;
            float2 acc = make_float2(0.0f, 0.0f);
            for (int k = 0; k <= 2 * RAD; ++k) acc = ffma2(make_float2(taps.f[k], taps.f[k]), sa[ly * AW + lx + k], acc);
            sx[idx] = acc;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < TX * TY; idx += blockDim.x) {
            int ly = idx / TX, lx = idx - ly * TX;
            int gy = y0 + ly, gx = x0 + lx;
            if (gy >= h || gx >= w) continue;
            float2 acc = make_float2(0.0f, 0.0f);
            for (int k = 0; k <= 2 * RAD; ++k) acc = ffma2(make_float2(taps.f[k], taps.f[k]), sx[(ly + k) * TX + lx], acc);
            put(gy, gx, acc);
        }
        __syncthreads();
    }
}

// The same final field for levels NT = 64, 128 or 256 pixels wide at the radius 3, as a sweep down
// the rows: one CTA of NT threads per pair (thread t owns column t).  Steps of 7 input rows are
// loaded into a double-buffered shared-memory block with replicated halo columns (one barrier per
// step); each thread's x pass of its column goes into a 7-row register window (row y in slot y mod 7,
// the first row fills every slot, rows past the bottom repeat the last row), and the y pass of the
// window gives output row y - 3.  Same taps in the same order as the tile kernel: the same values.
template <int NT, bool PLANAR>
__global__ void __launch_bounds__(NT) demons_finalize_sweep_kernel(const float2 *u0, const float2 *s0,
                                                                   const float2 *s1, const int32_t *iters,
                                                                   int levels, int level, float *uout, int B, int h,
                                                                   Taps taps)
{
    constexpr int RAD = 3, R = 2 * RAD + 1, HO = 4, RST = NT + 2 * HO;
    __shared__ __align__(16) float2 rows[2][R][RST];
    const int t = threadIdx.x;
    float2 tf[R];
#pragma unroll
    for (int k = 0; k < R; ++k) tf[k] = make_float2(taps.f[k], taps.f[k]);
    const size_t plane = (size_t)h * NT;
    const int nsteps = (h + RAD + R - 1) / R;   // input rows 0 .. h + 2 (past the bottom: row h - 1)
    int buf = 0;
    for (int pair = blockIdx.x; pair < B; pair += gridDim.x) {
        const int n = iters[(size_t)pair * levels + level];
        const float2 *src = (n == 0 ? u0 : ((n & 1) ? s1 : s0)) + (size_t)pair * plane;
        auto put = [&](int y, float2 v) {
            if (PLANAR) {
                uout[(size_t)pair * 2 * plane + (size_t)y * NT + t] = v.x;
                uout[(size_t)pair * 2 * plane + plane + (size_t)y * NT + t] = v.y;
            } else {
                reinterpret_cast<float2 *>(uout)[(size_t)pair * plane + (size_t)y * NT + t] = v;
            }
        };
        if (n == 0) {   // no update was applied: u_0 itself
            for (int y = 0; y < h; ++y) put(y, src[(size_t)y * NT + t]);
            continue;
        }
        float2 win[R];
        for (int k = 0; k < nsteps; ++k) {
            float2 (*rb)[RST] = rows[buf];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const float2 v = src[(size_t)min(R * k + i, h - 1) * NT + t];
                rb[i][HO + t] = v;
                if (t == 0)
#pragma unroll
                    for (int j = 1; j <= RAD; ++j) rb[i][HO - j] = v;
                if (t == NT - 1)
#pragma unroll
                    for (int j = 1; j <= RAD; ++j) rb[i][HO + NT - 1 + j] = v;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int y = R * k + i;
                float2 xa = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int j = 0; j < R; ++j) xa = ffma2(tf[j], rb[i][HO + t - RAD + j], xa);
                win[i] = xa;   // row y in slot y mod R = i
                if (y == 0) {
#pragma unroll
                    for (int j = 1; j < R; ++j) win[j] = xa;
                }
                const int yo = y - RAD;
                if (yo >= 0 && yo < h) {
                    // rows yo - 3 + j = y - 6 + j sit in slots (i + 1 + j) mod R
                    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
                    for (int j = 0; j < R; ++j) acc = ffma2(tf[j], win[(i + 1 + j) % R], acc);
                    put(yo, acc);
                }
            }
            buf ^= 1;
        }
    }
}

// Prolongation (Section 1): fine(x_f) = 2 * bilinear(coarse, (x_f + 0.5)/2 - 0.5), interleaved fields.
// The fine level is H x W, 2h x 2w or one more row/column where the size did not halve (the extra row or
// column samples past the coarse edge: the clamped edge value).  Each CTA walks an equal run of
// consecutive fine rows of all pairs (row = pair x H + i; the division per row, not per pixel), threads
// along the row, so consecutive threads write consecutive pixels.
__global__ void __launch_bounds__(256) prolong_kernel(const float2 *__restrict__ uc, float2 *__restrict__ uf, int B,
                                                      int h, int w, int H, int W, size_t rows_per_cta)
{
    const size_t total = (size_t)B * H;
    const size_t r0 = (size_t)blockIdx.x * rows_per_cta;
    const size_t r1 = r0 + rows_per_cta < total ? r0 + rows_per_cta : total;
    for (size_t r = r0; r < r1; ++r) {
        const int b = (int)(r / (unsigned)H), i = (int)(r - (size_t)b * H);
        const float y = ((float)i + 0.5f) * 0.5f - 0.5f;
        const float2 *ucb = uc + (size_t)b * h * w;
        float2 *row = uf + r * W;
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            const float x = ((float)j + 0.5f) * 0.5f - 0.5f;
            const float2 v = bilinear2_clamped(ucb, h, w, x, y);
            row[j] = make_float2(2.0f * v.x, 2.0f * v.y);
        }
    }
}

// Prolongation of B coarse fields (h x w) to the finer level's stored size H x W.
int launch_prolong(hrebsd_ctx *ctx, const float2 *uc, float2 *uf, int B, int h, int w, int H, int W, cudaStream_t st)
{
    const int threads = W >= 256 ? 256 : (W + 31) / 32 * 32;
    const size_t rows = (size_t)B * H, cap = (size_t)ctx->num_sms * (2048 / threads);
    const size_t grid = rows < cap ? rows : cap, per = (rows + grid - 1) / grid;
    hr_prof_begin(ctx, st);
    prolong_kernel<<<(unsigned)grid, threads, 0, st>>>(uc, uf, B, h, w, H, W, per);
    hr_prof_end(ctx, PROF_DEMONS_AUX, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

// Planar [B][2][h][w] -> interleaved [B][h][w] float2 (the optional initial field).
__global__ void interleave_kernel(const float *__restrict__ in, float2 *__restrict__ out, int B, int h, int w)
{
    const size_t plane = (size_t)h * w, total = (size_t)B * plane;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        size_t b = idx / plane, p = idx - b * plane;
        out[idx] = make_float2(in[b * 2 * plane + p], in[b * 2 * plane + plane + p]);
    }
}

__global__ void iota_kernel(int *a, int n, int *count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

template <int RAD, bool IN_S>
int launch_iter_t(hrebsd_ctx *ctx, const IterArgs &a, int max_items, cudaStream_t st)
{
    constexpr size_t smem = Geo<RAD>::BYTES;
    static int configured_dev = -1;
    static int occ = 0;
    if (configured_dev != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(demons_iter_kernel<RAD, IN_S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        HR_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, demons_iter_kernel<RAD, IN_S>, kIterThreads, smem));
        if (occ < 1) occ = 1;
        configured_dev = ctx->device;
    }
    int grid = ctx->num_sms * occ;
    if (grid > max_items) grid = max_items;
    if (grid < 1) grid = 1;
    hr_prof_begin(ctx, st);
    demons_iter_kernel<RAD, IN_S><<<grid, kIterThreads, smem, st>>>(a);
    hr_prof_end(ctx, PROF_ITER, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

template <int RAD>
int launch_iter(hrebsd_ctx *ctx, const IterArgs &a, int max_items, cudaStream_t st)
{
    return a.in_is_s ? launch_iter_t<RAD, true>(ctx, a, max_items, st) : launch_iter_t<RAD, false>(ctx, a, max_items, st);
}

template <int RAD, int TX_, int TY_, int MINB, int NT_, int FR, bool IN_S = true>
int launch_iter_tma(hrebsd_ctx *ctx, const CUtensorMap &tmS, const CUtensorMap &tmF, const IterArgs &a, int max_items,
                    cudaStream_t st)
{
    constexpr size_t smem = GeoT<RAD, TX_, TY_>::BYTES;
    static int configured_dev = -1;
    static int occ = 0;
    if (configured_dev != ctx->device) {
        auto k = demons_iter_tma_kernel<RAD, TX_, TY_, MINB, NT_, FR, IN_S>;
        HR_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HR_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, NT_, smem));
        if (occ < 1) occ = 1;
        configured_dev = ctx->device;
    }
    int grid = ctx->num_sms * occ;
    if (grid > max_items) grid = max_items;
    if (grid < 1) grid = 1;
    hr_prof_begin(ctx, st);
    demons_iter_tma_kernel<RAD, TX_, TY_, MINB, NT_, FR, IN_S><<<grid, NT_, smem, st>>>(tmS, tmF, a);
    hr_prof_end(ctx, PROF_ITER, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

// Tensor maps of one level for the TMA-fed iteration: the two s buffers
// (float2 [B][h][w] seen as FP32 [B][h][2w]) and the test images.
template <int RAD, int TX_, int TY_>
bool encode_level_maps(const float2 *s0, const float2 *s1, const float2 *u0, const float *ftest, int B, int h, int w,
                       CUtensorMap *tmS, CUtensorMap *tmF)
{
    using L = Geo<RAD, TX_, TY_>;
    using G = GeoT<RAD, TX_, TY_>;
    const uint64_t row2 = (uint64_t)w * 8, img2 = row2 * h, row1 = (uint64_t)w * 4, img1 = row1 * h;
    if (hr_encode_tmap_3d(&tmS[0], s0, 2ull * w, h, B, row2, img2, 2 * L::AST, L::AHP, 1)) return false;
    if (hr_encode_tmap_3d(&tmS[1], s1, 2ull * w, h, B, row2, img2, 2 * L::AST, L::AHP, 1)) return false;
    if (u0 && hr_encode_tmap_3d(&tmS[2], u0, 2ull * w, h, B, row2, img2, 2 * L::AST, L::AHP, 1)) return false;
    if (hr_encode_tmap_3d(tmF, ftest, w, h, B, row1, img1, G::FWB, G::FH, 1)) return false;
    return true;
}

// Tile shapes of the TMA-fed iteration (autotuned per level).  Every shape
// computes each output pixel with the same arithmetic in the same order, so
// the field does not depend on the choice; only the per-tile SSD partials
// (and hence the last bits of the level SSD) are grouped differently.  The
// extra shapes are compiled for the radius of sigma = 1 (r = 3); other radii
// use shape 0.
constexpr int kTileVariants = 8;
constexpr int kStripVariant = 5;   // the row sweep (demons_strip.cuh): one CTA per pair, whole rows
constexpr int kLoopVariant = 6;    // the row sweep with every iteration k >= 1 of a level in one launch
constexpr int kLevelVariant = 7;   // the whole level in shared memory (demons_level.cuh), <= 64 x 64
constexpr int kVarTX[kTileVariants] = {64, 32, 64, 64, 64, 256, 256, 64};
constexpr int kVarTY[kTileVariants] = {32, 32, 16, 32, 64, 256, 256, 64};
constexpr int kMinTX = 32, kMinTY = 16;   // smallest tile extents (size the per-tile SSD partials)
bool variant_ok(int rad, int v) { return v == 0 || (rad == 3 && v > 0 && v < kTileVariants); }
constexpr bool min_extents_ok()
{
    for (int v = 0; v < kTileVariants; ++v)
        if (kVarTX[v] < kMinTX || kVarTY[v] < kMinTY) return false;
    return TX >= kMinTX && TY >= kMinTY;
}
static_assert(min_extents_ok(), "kMinTX/kMinTY must not exceed any tile shape (the SSD partials are sized by them)");
static_assert(HREBSD_TILE_VARIANTS == kTileVariants, "tile variants");

// The row sweep covers levels 64, 128 or 256 pixels wide at the Gaussian radius 3 (its register
// windows are 2r + 1 = 7 rows, the rows of one step).
bool strip_ok(int rad, int w) { return rad == 3 && (w == 64 || w == 128 || w == 256); }

template <int NT, bool IN_S, bool LOOP, bool TEX>
int launch_strip_tt(hrebsd_ctx *ctx, const IterArgs &a, const strip::LoopArgs &c, int max_items, cudaStream_t st)
{
    using G = strip::Geo<3, NT>;
    static int configured_dev = -1;
    static int occ = 0;
    auto k = strip::demons_strip_kernel<3, NT, IN_S, LOOP, TEX>;
    if (configured_dev != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::BYTES));
        HR_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, NT, G::BYTES));
        if (occ < 1) occ = 1;
        configured_dev = ctx->device;
    }
    int grid = ctx->num_sms * occ;
    if (grid > max_items) grid = max_items;
    if (grid < 1) grid = 1;
    hr_prof_begin(ctx, st);
    k<<<grid, NT, G::BYTES, st>>>(a, c);
    hr_prof_end(ctx, PROF_ITER, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}
// The moving image by texture gathers when a.mtex is set, else by plain loads.
template <int NT, bool IN_S, bool LOOP>
int launch_strip_t(hrebsd_ctx *ctx, const IterArgs &a, const strip::LoopArgs &c, int max_items, cudaStream_t st)
{
    return a.mtex ? launch_strip_tt<NT, IN_S, LOOP, true>(ctx, a, c, max_items, st)
                  : launch_strip_tt<NT, IN_S, LOOP, false>(ctx, a, c, max_items, st);
}

// One iteration over the active pairs.  a.tiles must be 1 (one SSD partial per pair); a.in is s_k,
// or u_0 when !in_s.
int launch_strip(hrebsd_ctx *ctx, bool in_s, const IterArgs &a, int max_items, cudaStream_t st)
{
    const strip::LoopArgs c{};
    switch (a.w) {
    case 64: return in_s ? launch_strip_t<64, true, false>(ctx, a, c, max_items, st) : launch_strip_t<64, false, false>(ctx, a, c, max_items, st);
    case 128: return in_s ? launch_strip_t<128, true, false>(ctx, a, c, max_items, st) : launch_strip_t<128, false, false>(ctx, a, c, max_items, st);
    case 256: return in_s ? launch_strip_t<256, true, false>(ctx, a, c, max_items, st) : launch_strip_t<256, false, false>(ctx, a, c, max_items, st);
    default: return HREBSD_EINVAL;
    }
}

// Iterations 1 .. cap - 1 of a level in one launch for the pairs of a.active (the survivors of
// iteration 0), each ended by the stop rule in its CTA; a.in / a.out unused (s_k alternates between
// c.s0 and c.s1 as in the per-iteration launches).
int launch_strip_loop(hrebsd_ctx *ctx, const IterArgs &a, const strip::LoopArgs &c, int max_items, cudaStream_t st)
{
    switch (a.w) {
    case 64: return launch_strip_t<64, true, true>(ctx, a, c, max_items, st);
    case 128: return launch_strip_t<128, true, true>(ctx, a, c, max_items, st);
    case 256: return launch_strip_t<256, true, true>(ctx, a, c, max_items, st);
    default: return HREBSD_EINVAL;
    }
}

// The tile shape of a level: the tuned or pinned one, else the row sweep where it applies (the fastest
// shape measured at 64, 128 and 256 pixels wide), else shape 0.
int hr_tuned_variant(const hrebsd_ctx *ctx, int rad, int h, int w)
{
    for (const auto &t : ctx->tune)
        if (t.h == h && t.w == w) return variant_ok(rad, t.var) ? t.var : 0;
    return strip_ok(rad, w) ? kStripVariant : 0;
}

// The whole level in shared memory covers levels of at most 64 x 64 pixels at the Gaussian radius 3.
bool level_ok(int rad, int h, int w) { return rad == 3 && h <= lvl::MAXD && w <= lvl::MAXD; }

// One launch for a whole level of B pairs (pairs from the counter a.work, zeroed here).
int launch_level(hrebsd_ctx *ctx, const lvl::LevelArgs &a, cudaStream_t st)
{
    static int configured_dev = -1;
    static int occ = 0;
    auto k = lvl::demons_level_kernel<3>;
    if (configured_dev != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lvl::BYTES));
        HR_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, lvl::NT, lvl::BYTES));
        if (occ < 1) occ = 1;
        configured_dev = ctx->device;
    }
    int grid = ctx->num_sms * occ;
    if (grid > a.B) grid = a.B;
    if (grid < 1) grid = 1;
    HR_CHECK(cudaMemsetAsync(a.work, 0, sizeof(int), st));
    hr_prof_begin(ctx, st);
    k<<<grid, lvl::NT, lvl::BYTES, st>>>(a);
    hr_prof_end(ctx, PROF_ITER, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

// Pairs the loop form keeps resident at once (one CTA each) at a level w pixels wide.
template <int NT>
int strip_capacity_t(hrebsd_ctx *ctx)
{
    using G = strip::Geo<3, NT>;
    static int configured_dev = -1;
    static int occ = 0;
    if (configured_dev != ctx->device) {
        auto k = strip::demons_strip_kernel<3, NT, true, true, true>;   // the same resources without TEX
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::BYTES) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, NT, G::BYTES) != cudaSuccess)
            occ = 0;
        configured_dev = ctx->device;
    }
    return ctx->num_sms * occ;
}
int strip_capacity(hrebsd_ctx *ctx, int w)
{
    return w == 64 ? strip_capacity_t<64>(ctx) : w == 128 ? strip_capacity_t<128>(ctx) : w == 256 ? strip_capacity_t<256>(ctx) : 0;
}

// ---------------------------------------------------------------------------
// CUDA graph per pyramid level.  The launches of a level are captured once on
// a private stream and replayed on the caller's stream; the cache is keyed by
// every pointer, size and parameter the launches depend on.
bool hr_graph_usable(hrebsd_ctx *ctx, cudaStream_t st)
{
    if (!ctx->graphs || ctx->prof_on) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;   // the caller is capturing: launch into its graph
    }
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->cap_stream = nullptr;
        return false;
    }
    return true;
}

template <typename Emit>
int hr_graph_run(hrebsd_ctx *ctx, const hr_graph_key &key, cudaStream_t st, Emit &&emit)
{
    constexpr size_t kMaxGraphs = 32;
    hr_graph_entry *hit = nullptr;
    for (auto &g : ctx->graph_cache)
        if (!memcmp(&g.key, &key, sizeof key)) {
            hit = &g;
            break;
        }
    if (!hit) {
        const long long n0 = ctx->launches;
        HR_CHECK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int e = emit(ctx->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
        const long long nodes = ctx->launches - n0;
        ctx->launches = n0;
        if (e || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return e ? e : hr_cuda_error(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
        }
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return hr_cuda_error(ie, "cudaGraphInstantiate", __FILE__, __LINE__);
        if (ctx->graph_cache.size() >= kMaxGraphs) {
            size_t lru = 0;
            for (size_t i = 1; i < ctx->graph_cache.size(); ++i)
                if (ctx->graph_cache[i].last < ctx->graph_cache[lru].last) lru = i;
            cudaGraphExecDestroy(ctx->graph_cache[lru].exec);
            ctx->graph_cache.erase(ctx->graph_cache.begin() + lru);
        }
        ctx->graph_cache.push_back(hr_graph_entry{key, ex, nodes, 0});
        hit = &ctx->graph_cache.back();
    }
    hit->last = ++ctx->graph_clock;
    HR_CHECK(cudaGraphLaunch(hit->exec, st));
    ctx->launches += hit->nodes;
    return HREBSD_OK;
}

// Texture over the reference images of a level (R images of h x w, stacked as R h rows of w) for the
// row sweep's four-texel gathers, which read CUDA arrays only.  The context keeps one array per level
// width and grows it when a call needs more rows; every call first copies its references in, on its
// stream, so the array holds them when the level's launches run (calls on one context are serialised
// like its workspace).  *tex = 0 selects plain loads: option off, R h above the device's gather
// height, a stream that is being captured (no allocation or synchronisation inside a capture), or an
// array that could not be allocated.  Growing an array synchronises the device (the old one may be in
// use) and drops the cached graphs (their launches name the old texture).
int hr_ref_texture(hrebsd_ctx *ctx, const float *ref, int R, int h, int w, cudaStream_t st, unsigned long long *tex)
{
    *tex = 0;
    if (!ctx->tex_gather) return HREBSD_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return HREBSD_OK;
    }
    if (!ctx->tex_max_rows) {
        int mh = 0, mw = 0;
        HR_CHECK(cudaDeviceGetAttribute(&mh, cudaDevAttrMaxTexture2DGatherHeight, ctx->device));
        HR_CHECK(cudaDeviceGetAttribute(&mw, cudaDevAttrMaxTexture2DGatherWidth, ctx->device));
        ctx->tex_max_rows = mw >= 256 && mh > 0 ? mh : -1;
    }
    const long long rows = (long long)R * h;
    if (ctx->tex_max_rows < 0 || rows > ctx->tex_max_rows || w > 256) return HREBSD_OK;
    size_t mi = ctx->mtex.size();
    for (size_t i = 0; i < ctx->mtex.size(); ++i)
        if (ctx->mtex[i].w == w) mi = i;
    if (mi == ctx->mtex.size() || ctx->mtex[mi].rows < rows) {
        long long cap_rows = rows > 8LL * h ? rows : 8LL * h;   // room for 8 references from the start
        if (mi < ctx->mtex.size()) {
            const long long twice = 2LL * ctx->mtex[mi].rows;
            if (twice > cap_rows) cap_rows = twice;
            HR_CHECK(cudaDeviceSynchronize());
            for (auto &g : ctx->graph_cache) cudaGraphExecDestroy(g.exec);
            ctx->graph_cache.clear();
            cudaDestroyTextureObject(ctx->mtex[mi].tex);
            cudaFreeArray(ctx->mtex[mi].arr);
            ctx->mtex.erase(ctx->mtex.begin() + mi);
        }
        if (cap_rows > ctx->tex_max_rows) cap_rows = ctx->tex_max_rows;
        hr_mtex m{w, (int)cap_rows, nullptr, 0};
        const cudaChannelFormatDesc fd = cudaCreateChannelDesc<float>();
        if (cudaMallocArray(&m.arr, &fd, (size_t)w, (size_t)cap_rows, cudaArrayTextureGather) != cudaSuccess) {
            cudaGetLastError();
            return HREBSD_OK;
        }
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = m.arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        cudaTextureObject_t to = 0;
        const cudaError_t ce = cudaCreateTextureObject(&to, &rd, &td, nullptr);
        if (ce != cudaSuccess) {
            cudaFreeArray(m.arr);
            return hr_cuda_error(ce, "cudaCreateTextureObject", __FILE__, __LINE__);
        }
        m.tex = to;
        ctx->mtex.push_back(m);
        mi = ctx->mtex.size() - 1;
    }
    HR_CHECK(cudaMemcpy2DToArrayAsync(ctx->mtex[mi].arr, 0, 0, ref, (size_t)w * 4, (size_t)w * 4, (size_t)rows,
                                      cudaMemcpyDeviceToDevice, st));
    *tex = ctx->mtex[mi].tex;
    return HREBSD_OK;
}


#define HR_TMA_VARIANTS(RAD, CALL)                                                                                 \
    case 0: return CALL(RAD, 64, 32, 2, 256, 4);                                                                   \
    case 1: if (RAD == 3) return CALL(3, 32, 32, 3, 256, 4); break;                                                \
    case 2: if (RAD == 3) return CALL(3, 64, 16, 3, 256, 4); break;                                                \
    case 3: if (RAD == 3) return CALL(3, 64, 32, 2, 512, 4); break;                                                \
    case 4: if (RAD == 3) return CALL(3, 64, 64, 1, 768, 4); break;

// tmS: [3] (s0, s1 and, when u0 is given, the level's initial field).
bool encode_maps(int rad, int var, const float2 *s0, const float2 *s1, const float2 *u0, const float *ftest, int B,
                 int h, int w, CUtensorMap *tmS, CUtensorMap *tmF)
{
#define HR_ENC(R, X, Y, MB, NT, FR) encode_level_maps<R, X, Y>(s0, s1, u0, ftest, B, h, w, tmS, tmF)
    switch (rad) {
    case 1: return var == 0 && HR_ENC(1, 64, 32, 2, 256, 4);
    case 2: return var == 0 && HR_ENC(2, 64, 32, 2, 256, 4);
    case 3:
        switch (var) { HR_TMA_VARIANTS(3, HR_ENC) default: break; }
        return false;
    case 4: return var == 0 && HR_ENC(4, 64, 32, 2, 256, 4);
    case 5: return var == 0 && HR_ENC(5, 64, 32, 2, 256, 4);
    case 6: return var == 0 && HR_ENC(6, 64, 32, 2, 256, 4);
    default: return false;
    }
#undef HR_ENC
}

// in_s false (first iteration of a level, input u_0): compiled for radius 3 only.
int dispatch_iter_tma(hrebsd_ctx *ctx, int rad, int var, bool in_s, const CUtensorMap &tmS, const CUtensorMap &tmF,
                      const IterArgs &a, int max_items, cudaStream_t st)
{
    if (!in_s) {
#define HR_LT0(R, X, Y, MB, NT, FR) launch_iter_tma<R, X, Y, MB, NT, FR, false>(ctx, tmS, tmF, a, max_items, st)
        if (rad == 3) {
            switch (var) { HR_TMA_VARIANTS(3, HR_LT0) default: break; }
        }
#undef HR_LT0
        return HREBSD_EINVAL;
    }
#define HR_LT(R, X, Y, MB, NT, FR) launch_iter_tma<R, X, Y, MB, NT, FR>(ctx, tmS, tmF, a, max_items, st)
    switch (rad) {
    case 1: if (var == 0) return HR_LT(1, 64, 32, 2, 256, 4); break;
    case 2: if (var == 0) return HR_LT(2, 64, 32, 2, 256, 4); break;
    case 3:
        switch (var) { HR_TMA_VARIANTS(3, HR_LT) default: break; }
        break;
    case 4: if (var == 0) return HR_LT(4, 64, 32, 2, 256, 4); break;
    case 5: if (var == 0) return HR_LT(5, 64, 32, 2, 256, 4); break;
    case 6: if (var == 0) return HR_LT(6, 64, 32, 2, 256, 4); break;
    default: break;
    }
#undef HR_LT
    return HREBSD_EINVAL;
}

int dispatch_iter(hrebsd_ctx *ctx, int rad, const IterArgs &a, int max_items, cudaStream_t st)
{
    switch (rad) {
    case 0: return launch_iter<0>(ctx, a, max_items, st);
    case 1: return launch_iter<1>(ctx, a, max_items, st);
    case 2: return launch_iter<2>(ctx, a, max_items, st);
    case 3: return launch_iter<3>(ctx, a, max_items, st);
    case 4: return launch_iter<4>(ctx, a, max_items, st);
    case 5: return launch_iter<5>(ctx, a, max_items, st);
    case 6: return launch_iter<6>(ctx, a, max_items, st);
    default: return HREBSD_EINVAL;
    }
}

int dispatch_finalize(hrebsd_ctx *ctx, int rad, bool planar, const float2 *u0, const float2 *s0, const float2 *s1,
                      const int32_t *iters, int levels, int level, float *uout, int B, int h, int w, int tiles_x,
                      int tiles, const Taps &taps, cudaStream_t st)
{
    if (rad == 3 && (w == 64 || w == 128 || w == 256)) {   // the row sweep
        const int grid = B < ctx->num_sms * 8 ? B : ctx->num_sms * 8;
        hr_prof_begin(ctx, st);
#define HR_FSW(NT)                                                                                                 \
        if (planar) demons_finalize_sweep_kernel<NT, true><<<grid, NT, 0, st>>>(u0, s0, s1, iters, levels, level, \
                                                                                uout, B, h, taps);                 \
        else demons_finalize_sweep_kernel<NT, false><<<grid, NT, 0, st>>>(u0, s0, s1, iters, levels, level, uout, B, \
                                                                          h, taps)
        if (w == 64) HR_FSW(64);
        else if (w == 128) HR_FSW(128);
        else HR_FSW(256);
#undef HR_FSW
        hr_prof_end(ctx, PROF_DEMONS_AUX, st);
        HR_LAUNCHED(ctx);
        return HREBSD_OK;
    }
    long long items = (long long)B * tiles;
    int grid = (int)(items < ctx->num_sms * 8LL ? items : ctx->num_sms * 8LL);
    const size_t smem = (size_t)((TX + 2 * rad) * (TY + 2 * rad) + (TY + 2 * rad) * TX) * sizeof(float2);
    hr_prof_begin(ctx, st);
#define HR_FIN(R)                                                                                                  \
    do {                                                                                                           \
        auto kt = demons_finalize_kernel<R, true>;                                                                 \
        auto kf = demons_finalize_kernel<R, false>;                                                                \
        HR_CHECK(cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));                \
        HR_CHECK(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));                \
        if (planar) kt<<<grid, 256, smem, st>>>(u0, s0, s1, iters, levels, level, uout, B, h, w, tiles_x, tiles, taps); \
        else kf<<<grid, 256, smem, st>>>(u0, s0, s1, iters, levels, level, uout, B, h, w, tiles_x, tiles, taps);  \
    } while (0)
    switch (rad) {
    case 0: HR_FIN(0); break;
    case 1: HR_FIN(1); break;
    case 2: HR_FIN(2); break;
    case 3: HR_FIN(3); break;
    case 4: HR_FIN(4); break;
    case 5: HR_FIN(5); break;
    case 6: HR_FIN(6); break;
    default: return HREBSD_EINVAL;
    }
#undef HR_FIN
    hr_prof_end(ctx, PROF_DEMONS_AUX, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

enum { WS_TPYR = 0, WS_RPYR, WS_U0, WS_S0, WS_S1, WS_UOUT, WS_PART, WS_HIST, WS_LIST, WS_COUNT };

// Register B pairs (all buffers already offset to this chunk).
// Bytes of each workspace slot for B pairs (WS_* order).
void slot_bytes(int R, int B, int H, int W, const hrebsd_demons_params *p, size_t *bytes)
{
    const int L = p->levels;
    int cap_max = 0;
    for (int l = 0; l < L; ++l) cap_max = p->max_iters[l] > cap_max ? p->max_iters[l] : cap_max;
    size_t pyr_px = 0, rpyr_px = 0;
    for (int l = 1; l < L; ++l) {
        pyr_px += (size_t)B * (H >> l) * (W >> l);
        rpyr_px += (size_t)R * (H >> l) * (W >> l);
    }
    const size_t field_elems = (size_t)B * 2 * H * W;
    const int tiles0 = ((W + kMinTX - 1) / kMinTX) * ((H + kMinTY - 1) / kMinTY);
    bytes[WS_TPYR] = pyr_px * 4 + 16;
    bytes[WS_RPYR] = rpyr_px * 4 + 16;
    bytes[WS_U0] = field_elems * 4;
    bytes[WS_S0] = field_elems * 4;
    bytes[WS_S1] = field_elems * 4;
    bytes[WS_UOUT] = (L > 1 ? field_elems / 4 : 1) * 4;
    bytes[WS_PART] = (size_t)B * tiles0 * 4;
    bytes[WS_HIST] = (size_t)B * (cap_max + 1) * 8;
    bytes[WS_LIST] = ((size_t)2 * B + 64) * 4;
}

// Register B pairs (all buffers already offset to this chunk).  `given`
// (nullable) supplies the workspace slots; otherwise they come from the context.
int register_chunk(hrebsd_ctx *ctx, const float *ref, const float *test, const int32_t *ref_idx, int R, int B,
                   int H, int W, const hrebsd_demons_params *p, const float *init_field, float *field,
                   int32_t *iters, int32_t *status, cudaStream_t st, void *const *given = nullptr)
{
    const int L = p->levels;
    const int start = (p->start_level < 0 || p->start_level >= L) ? L - 1 : p->start_level;
    int cap_max = 0;
    for (int l = 0; l < L; ++l) cap_max = p->max_iters[l] > cap_max ? p->max_iters[l] : cap_max;
    const int rad = max(hr_gauss_radius(p->sigma_update), hr_gauss_radius(p->sigma_field));
    Taps taps;
    if (hr_gauss_taps(p->sigma_update, rad, taps.up) < 0 || hr_gauss_taps(p->sigma_field, rad, taps.f) < 0)
        return HREBSD_EINVAL;

    // workspace
    size_t pyr_px = 0, rpyr_px = 0;
    for (int l = 1; l < L; ++l) {
        pyr_px += (size_t)B * (H >> l) * (W >> l);
        rpyr_px += (size_t)R * (H >> l) * (W >> l);
    }
    const size_t field_elems = (size_t)B * 2 * H * W;
    const int tiles0 = ((W + TX - 1) / TX) * ((H + TY - 1) / TY);
    void *tpyr = nullptr, *rpyr = nullptr, *u0 = nullptr, *s0 = nullptr, *s1 = nullptr, *uout = nullptr;
    void *part = nullptr, *hist = nullptr, *lists = nullptr;
    int e;
    size_t sb[WS_COUNT];
    slot_bytes(R, B, H, W, p, sb);
    void **slot_ptr[WS_COUNT] = {&tpyr, &rpyr, &u0, &s0, &s1, &uout, &part, &hist, &lists};
    for (int k = 0; k < WS_COUNT; ++k) {
        if (given) *slot_ptr[k] = given[k];
        else if ((e = hr_ws(ctx, k, sb[k], slot_ptr[k]))) return e;
    }
    (void)pyr_px; (void)rpyr_px; (void)field_elems; (void)tiles0;
    int *list0 = (int *)lists, *list1 = list0 + B, *cnt = list1 + B;   // cnt[0], cnt[1]

    // pyramids (level pointers)
    const float *tl[8], *rl[8];
    tl[0] = test;
    rl[0] = ref;
    {
        float *tp = (float *)tpyr, *rp = (float *)rpyr;
        for (int l = 1; l < L; ++l) {
            int hp = H >> (l - 1), wp = W >> (l - 1);
            if ((e = hr_launch_reduce2(ctx, tl[l - 1], tp, B, hp, wp, st))) return e;
            if ((e = hr_launch_reduce2(ctx, rl[l - 1], rp, R, hp, wp, st))) return e;
            tl[l] = tp;
            rl[l] = rp;
            tp += (size_t)B * (H >> l) * (W >> l);
            rp += (size_t)R * (H >> l) * (W >> l);
        }
    }
    HR_CHECK(cudaMemsetAsync(iters, 0, sizeof(int32_t) * B * L, st));
    HR_CHECK(cudaMemsetAsync(status, 0, sizeof(int32_t) * B, st));
    {
        const int hs = H >> start, ws = W >> start;
        size_t n0 = (size_t)B * hs * ws;
        if (init_field) {
            int grid = (int)((n0 + 255) / 256);
            if (grid > ctx->num_sms * 16) grid = ctx->num_sms * 16;
            hr_prof_begin(ctx, st);
            interleave_kernel<<<grid, 256, 0, st>>>(init_field, (float2 *)u0, B, hs, ws);
            hr_prof_end(ctx, PROF_DEMONS_AUX, st);
            HR_LAUNCHED(ctx);
        } else {
            HR_CHECK(cudaMemsetAsync(u0, 0, n0 * sizeof(float2), st));
        }
    }

    for (int l = start; l >= 0; --l) {
        const int h = H >> l, w = W >> l;
        const int cap = p->max_iters[l];
        int var = hr_tuned_variant(ctx, rad, h, w);
        // the whole level in shared memory, one launch (needs at least one iteration)
        const bool use_level = var == kLevelVariant && level_ok(rad, h, w) && cap >= 1;
        if (var == kLevelVariant && !use_level) var = kStripVariant;
        const bool sweep_v = var == kStripVariant || var == kLoopVariant;
        const bool use_strip = sweep_v && strip_ok(rad, w) && !ctx->no_tma;
        if (sweep_v && !use_strip) var = 4;   // the row sweep does not cover this level: 64x64 tiles
        // the whole level after iteration 0 in one launch (needs the stop rule's history: cap > 1):
        // shape 6, or shape 5 when every pair has a CTA of its own, so that no pair waits for another
        // (more pairs than CTAs: per-iteration launches re-balance the uneven counts every iteration)
        const bool use_loop = use_strip && cap > 1 &&
                              (var == kLoopVariant || (var == kStripVariant && B <= strip_capacity(ctx, w)));
        // the row sweep's moving image through texture gathers (not in the allocation-free call)
        unsigned long long mtex = 0;
        if (use_strip && !given && (e = hr_ref_texture(ctx, rl[l], R, h, w, st, &mtex))) return e;
        CUtensorMap tmS[3], tmF;
        const bool use_tma = !use_level && !use_strip && rad > 0 && !ctx->no_tma && cap > 1 &&
                             encode_maps(rad, var, (const float2 *)s0, (const float2 *)s1, (const float2 *)u0, tl[l],
                                         B, h, w, tmS, &tmF);
        // The launches of one level: list reset, cap x (iteration, control) -- or, in the loop
        // form, iteration 0 and its control, then one launch for the rest --, finalize,
        // prolongation.  Replayed from a cached CUDA graph when possible.
        auto emit = [&](cudaStream_t st) -> int {
            int e2;
            if (use_level) {   // the whole level, final field included, in one launch
                lvl::LevelArgs a;
                a.Ftest = tl[l];
                a.Mref = rl[l];
                a.ref_idx = ref_idx;
                a.u0 = (const float2 *)u0;
                a.uout = l == 0 ? field : (float *)uout;
                a.hist = (double *)hist;
                a.iters = iters;
                a.status = status;
                a.work = cnt;
                a.px_count = hr_prof_pixiters(ctx);
                a.B = B;
                a.h = h;
                a.w = w;
                a.hist_stride = cap_max + 1;
                a.cap = cap;
                a.window = p->stop_window;
                a.level = l;
                a.levels = L;
                a.planar = l == 0;
                a.tol = p->stop_tol;
                a.alpha2 = p->alpha * p->alpha;
                a.taps = taps;
                if ((e2 = launch_level(ctx, a, st))) return e2;
                if (l > 0)   // to the finer level's stored size
                    return launch_prolong(ctx, (const float2 *)uout, (float2 *)u0, B, h, w, H >> (l - 1), W >> (l - 1), st);
                return HREBSD_OK;
            }
            hr_prof_begin(ctx, st);
            iota_kernel<<<(B + 255) / 256, 256, 0, st>>>(list0, B, cnt);
            hr_prof_end(ctx, PROF_DEMONS_AUX, st);
            HR_LAUNCHED(ctx);
            for (int k = 0; k < (use_loop ? 1 : cap); ++k) {
                const bool tma_k = !use_strip && use_tma && (k > 0 || rad == 3);
                const int tx = tma_k ? kVarTX[var] : TX, ty = tma_k ? kVarTY[var] : TY;
                const int tiles_x = use_strip ? 1 : (w + tx - 1) / tx;
                const int tiles = use_strip ? 1 : tiles_x * ((h + ty - 1) / ty);
                int *cur = (k & 1) ? list1 : list0, *nxt = (k & 1) ? list0 : list1;
                IterArgs a;
                a.Ftest = tl[l];
                a.Mref = rl[l];
                a.ref_idx = ref_idx;
                a.in = k == 0 ? (const float2 *)u0 : ((k & 1) ? (const float2 *)s1 : (const float2 *)s0);
                a.out = ((k + 1) & 1) ? (float2 *)s1 : (float2 *)s0;
                a.part = (float *)part;
                a.active = cur;
                a.n_active = cnt + (k & 1);
                a.n_next_reset = cnt + ((k + 1) & 1);
                a.h = h;
                a.w = w;
                a.tiles_x = tiles_x;
                a.tiles = tiles;
                a.in_is_s = k > 0;
                a.alpha2 = p->alpha * p->alpha;
                a.taps = taps;
                a.px_count = hr_prof_pixiters(ctx);
                a.err = ctx->d_err;
                a.mtex = use_strip ? mtex : 0;
                if (use_strip) e2 = launch_strip(ctx, k > 0, a, B, st);
                else if (tma_k) e2 = dispatch_iter_tma(ctx, rad, var, k > 0, k > 0 ? tmS[k & 1] : tmS[2], tmF, a, B * tiles, st);
                else e2 = dispatch_iter(ctx, rad, a, B * tiles, st);
                if (e2) return e2;
                CtrlArgs c;
                c.part = (const float *)part;
                c.hist = (double *)hist;
                c.active = cur;
                c.n_active = cnt + (k & 1);
                c.next = nxt;
                c.n_next = cnt + ((k + 1) & 1);
                c.iters = iters;
                c.status = status;
                c.tiles = tiles;
                c.hist_stride = cap_max + 1;
                c.k = k;
                c.cap = cap;
                c.window = p->stop_window;
                c.level = l;
                c.levels = L;
                c.tol = p->stop_tol;
                int cgrid = (B + 255) / 256;
                if (cgrid > ctx->num_sms * 4) cgrid = ctx->num_sms * 4;
                hr_prof_begin(ctx, st);
                demons_control_kernel<<<cgrid, 256, 0, st>>>(c);
                hr_prof_end(ctx, PROF_CTRL, st);
                HR_LAUNCHED(ctx);
            }
            if (use_loop) {   // iterations 1 .. cap - 1 of the survivors of iteration 0 (list1)
                IterArgs a;
                a.Ftest = tl[l];
                a.Mref = rl[l];
                a.ref_idx = ref_idx;
                a.in = nullptr;
                a.out = nullptr;
                a.part = (float *)part;
                a.active = list1;
                a.n_active = cnt + 1;
                a.n_next_reset = nullptr;
                a.h = h;
                a.w = w;
                a.tiles_x = 1;
                a.tiles = 1;
                a.in_is_s = 1;
                a.alpha2 = p->alpha * p->alpha;
                a.taps = taps;
                a.px_count = hr_prof_pixiters(ctx);
                a.err = ctx->d_err;
                a.mtex = mtex;
                strip::LoopArgs c;
                c.s0 = (float2 *)s0;
                c.s1 = (float2 *)s1;
                c.hist = (double *)hist;
                c.iters = iters;
                c.status = status;
                c.hist_stride = cap_max + 1;
                c.cap = cap;
                c.window = p->stop_window;
                c.level = l;
                c.levels = L;
                c.tol = p->stop_tol;
                c.work = cnt;   // list0's count, free after iteration 0: the loop's item counter
                HR_CHECK(cudaMemsetAsync(cnt, 0, sizeof(int), st));
                if ((e2 = launch_strip_loop(ctx, a, c, B, st))) return e2;
            }
            const int tiles_x = (w + TX - 1) / TX, tiles = tiles_x * ((h + TY - 1) / TY);
            float *dst = l == 0 ? field : (float *)uout;
            if ((e2 = dispatch_finalize(ctx, rad, l == 0, (const float2 *)u0, (const float2 *)s0, (const float2 *)s1,
                                        iters, L, l, dst, B, h, w, tiles_x, tiles, taps, st)))
                return e2;
            if (l > 0)   // to the finer level's stored size
                return launch_prolong(ctx, (const float2 *)uout, (float2 *)u0, B, h, w, H >> (l - 1), W >> (l - 1), st);
            return HREBSD_OK;
        };
        if (given || !hr_graph_usable(ctx, st)) {
            if ((e = emit(st))) return e;
            continue;
        }
        // graph key: everything the launches of this level depend on
        hr_graph_key key{};
        const void *kp[] = {ref_idx, tl[l], rl[l], u0, s0, s1, uout, part, hist, lists, iters, status, field,
                            ctx->d_err, (const void *)(uintptr_t)mtex};
        static_assert(sizeof(kp) / sizeof(kp[0]) <= sizeof(key.p) / sizeof(key.p[0]), "graph key");
        for (size_t i = 0; i < sizeof(kp) / sizeof(kp[0]); ++i) key.p[i] = kp[i];
        const int ki[] = {l, L, B, h, w, cap, cap_max, rad, var, (int)use_tma, p->stop_window, (int)use_strip,
                          (int)use_loop, (int)use_level};
        for (size_t i = 0; i < sizeof(ki) / sizeof(ki[0]); ++i) key.i[i] = ki[i];
        key.f[0] = p->alpha;
        key.f[1] = p->stop_tol;
        memcpy(&key.f[2], taps.up, sizeof(taps.up));
        memcpy(&key.f[2 + 2 * kMaxRad + 1], taps.f, sizeof(taps.f));
        if ((e = hr_graph_run(ctx, key, st, emit))) return e;
    }
    return HREBSD_OK;
}

int check_register_args(hrebsd_ctx *ctx, const float *ref, const float *test, const int32_t *ref_idx, int R, int B,
                        int H, int W, const hrebsd_demons_params *p, float *field, int32_t *iters,
                        int32_t *pair_status)
{
    if (!ctx || !p || B < 0 || R < 1) return HREBSD_EINVAL;
    if (p->levels < 1 || p->levels > 8) return HREBSD_EINVAL;
    const int L = p->levels;
    // level l is (H >> l) x (W >> l): floor halving, sizes that do not halve included
    if ((H >> (L - 1)) < 8 || (W >> (L - 1)) < 8) return HREBSD_EINVAL;
    for (int l = 0; l < L; ++l)
        if (p->max_iters[l] < 0 || p->max_iters[l] > 4096) return HREBSD_EINVAL;
    if (!(p->alpha >= 0.0f) || p->stop_window < 0) return HREBSD_EINVAL;
    if (hr_gauss_radius(p->sigma_update) > kMaxRad || hr_gauss_radius(p->sigma_field) > kMaxRad) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!ref || !test || !ref_idx || !field || !iters || !pair_status) return HREBSD_EINVAL;
    return HREBSD_OK;
}

}  // namespace

namespace {

// Synthetic inputs of the autotuner: striped images (a few plane waves, like
// Kikuchi bands) and a field of a small rotation about the image centre, so
// that the moving-image gathers have realistic offsets.
__global__ void tune_fill_kernel(float *img, int n_img, float2 *s0, float2 *s1, int n_field, int h, int w)
{
    const size_t plane = (size_t)h * w, total = (size_t)n_img * plane;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(idx / plane), y = (int)((idx % plane) / w), x = (int)(idx % w);
        const float xf = (float)x / (float)w, yf = (float)y / (float)h;
        float v = 0.0f;
        for (int k = 0; k < 6; ++k) {
            const float ang = 0.52f * (float)k + 0.11f * (float)(b % 7);
            v += cosf(37.0f * (cosf(ang) * xf + sinf(ang) * yf) + (float)k);
        }
        img[idx] = v;
        if (b < n_field) {
            const float cx = (float)x - 0.5f * (float)(w - 1), cy = (float)y - 0.5f * (float)(h - 1);
            const float2 u = make_float2(-0.03f * cy + 0.4f, 0.03f * cx - 0.3f);
            s0[idx] = u;
            s1[idx] = u;
        }
    }
}

enum { WS_TUNE_IMG = 9, WS_TUNE_S0, WS_TUNE_S1, WS_TUNE_PART, WS_TUNE_IDX };
constexpr int WS_TUNE_LOOP = 21;   // the loop form's history, counts and status

}  // namespace

extern "C" int hrebsd_set_tile_variant(hrebsd_ctx *ctx, int h, int w, int variant)
{
    if (!ctx || h < 1 || w < 1 || variant < -1 || variant >= kTileVariants) return HREBSD_EINVAL;
    for (size_t i = 0; i < ctx->tune.size(); ++i)
        if (ctx->tune[i].h == h && ctx->tune[i].w == w) {
            if (variant < 0) ctx->tune.erase(ctx->tune.begin() + i);
            else ctx->tune[i].var = variant;
            return HREBSD_OK;
        }
    if (variant >= 0) ctx->tune.push_back(hr_tune_entry{h, w, variant});
    return HREBSD_OK;
}

extern "C" int hrebsd_get_tile_variant(const hrebsd_ctx *ctx, int h, int w)
{
    if (!ctx) return HREBSD_EINVAL;
    for (const auto &t : ctx->tune)
        if (t.h == h && t.w == w) return t.var;
    return 0;
}

extern "C" int hrebsd_autotune(hrebsd_ctx *ctx, int B, int H, int W, const hrebsd_demons_params *p, float *ms_out,
                               void *stream)
{
    if (!ctx || !p || B < 1) return HREBSD_EINVAL;
    int e = check_register_args(ctx, (const float *)1, (const float *)1, (const int32_t *)1, 1, B, H, W, p,
                                (float *)1, (int32_t *)1, (int32_t *)1);
    if (e) return e;
    if ((e = hr_set_device(ctx))) return e;
    const int L = p->levels;
    const int rad = max(hr_gauss_radius(p->sigma_update), hr_gauss_radius(p->sigma_field));
    Taps taps;
    if (hr_gauss_taps(p->sigma_update, rad, taps.up) < 0 || hr_gauss_taps(p->sigma_field, rad, taps.f) < 0)
        return HREBSD_EINVAL;
    if (ms_out)
        for (int i = 0; i < L * kTileVariants; ++i) ms_out[i] = nanf("");
    if (rad == 0) return HREBSD_OK;   // no TMA-fed iteration at r = 0
    const int Bt = B < 2048 ? B : 2048;
    const size_t px0 = (size_t)H * W;
    const int tiles0 = ((W + kMinTX - 1) / kMinTX) * ((H + kMinTY - 1) / kMinTY);
    void *img, *s0, *s1, *part, *idx;
    if ((e = hr_ws(ctx, WS_TUNE_IMG, (Bt + 1) * px0 * 4, &img))) return e;
    if ((e = hr_ws(ctx, WS_TUNE_S0, Bt * px0 * 8, &s0))) return e;
    if ((e = hr_ws(ctx, WS_TUNE_S1, Bt * px0 * 8, &s1))) return e;
    if ((e = hr_ws(ctx, WS_TUNE_PART, (size_t)Bt * tiles0 * 4, &part))) return e;
    if ((e = hr_ws(ctx, WS_TUNE_IDX, ((size_t)2 * Bt + 4) * 4, &idx))) return e;
    constexpr int kLoopCap = 8;   // the loop form runs iterations 1 .. kLoopCap - 1 per timed launch
    void *lws;
    if ((e = hr_ws(ctx, WS_TUNE_LOOP, (size_t)Bt * (kLoopCap + 1) * 8 + (size_t)Bt * 8, &lws))) return e;
    double *lhist = (double *)lws;
    int32_t *liters = (int32_t *)(lhist + (size_t)Bt * (kLoopCap + 1)), *lstatus = liters + Bt;
    int32_t *ridx = (int32_t *)idx, *list = ridx + Bt, *cnt = list + Bt;
    cudaStream_t st = hr_stream(stream);
    const int prof = ctx->prof_on;
    ctx->prof_on = 0;   // tuning launches stay out of the trace
    cudaEvent_t ev[2];
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
        ctx->prof_on = prof;
        return hr_cuda_error(cudaGetLastError(), "cudaEventCreate", __FILE__, __LINE__);
    }
    auto run = [&]() -> int {
        HR_CHECK(cudaMemsetAsync(ridx, 0, (size_t)Bt * 4, st));
        iota_kernel<<<(Bt + 255) / 256, 256, 0, st>>>(list, Bt, cnt);
        HR_LAUNCHED(ctx);
        for (int l = 0; l < L; ++l) {
            const int h = H >> l, w = W >> l;
            float *ref = (float *)img, *test = ref + (size_t)h * w;   // image 0 is the reference
            tune_fill_kernel<<<ctx->num_sms * 8, 256, 0, st>>>((float *)img, Bt + 1, (float2 *)s0, (float2 *)s1,
                                                               Bt, h, w);
            HR_LAUNCHED(ctx);
            unsigned long long mtex = 0;   // the row sweep's moving image as in a registration
            if (strip_ok(rad, w)) {
                const int e3 = hr_ref_texture(ctx, ref, 1, h, w, st, &mtex);
                if (e3) return e3;
            }
            float best = 0.0f;
            int best_v = 0;
            for (int v = 0; v < kTileVariants; ++v) {
                if (!variant_ok(rad, v) || ctx->no_tma) continue;
                const bool lv = v == kLoopVariant;
                const bool sv = v == kStripVariant || lv;
                const bool vv = v == kLevelVariant;
                if (sv && !strip_ok(rad, w)) continue;
                if (vv && !level_ok(rad, h, w)) continue;
                CUtensorMap tmS[3], tmF;
                if (!sv && !vv && !encode_maps(rad, v, (const float2 *)s0, (const float2 *)s1, nullptr, test, Bt, h, w, tmS, &tmF))
                    continue;
                const int tiles_x = sv ? 1 : (w + kVarTX[v] - 1) / kVarTX[v];
                const int tiles = sv ? 1 : tiles_x * ((h + kVarTY[v] - 1) / kVarTY[v]);
                IterArgs a;
                a.Ftest = test;
                a.Mref = ref;
                a.ref_idx = ridx;
                a.part = (float *)part;
                a.active = list;
                a.n_active = cnt;
                a.n_next_reset = cnt + 1;
                a.px_count = nullptr;
                a.err = ctx->d_err;
                a.h = h;
                a.w = w;
                a.tiles_x = tiles_x;
                a.tiles = tiles;
                a.in_is_s = 1;
                a.alpha2 = p->alpha * p->alpha;
                a.taps = taps;
                a.mtex = sv ? mtex : 0;
                // 2 warm-up iterations, then the best of 3 timed batches of 4 (the loop form: one
                // warm-up launch, then the best of 3 launches of kLoopCap - 1 iterations each)
                constexpr int kWarm = 2, kBatch = 4, kRounds = 3;
                float ms = 0.0f;
                int k = 0;
                if (vv) {   // whole levels of kLoopCap iterations: one warm-up launch, then the best of 3
                    lvl::LevelArgs la;
                    la.Ftest = test;
                    la.Mref = ref;
                    la.ref_idx = ridx;
                    la.u0 = (const float2 *)s0;
                    la.uout = (float *)s1;
                    la.hist = lhist;
                    la.iters = liters;
                    la.status = lstatus;
                    la.work = cnt + 2;
                    la.px_count = nullptr;
                    la.B = Bt;
                    la.h = h;
                    la.w = w;
                    la.hist_stride = kLoopCap + 1;
                    la.cap = kLoopCap;
                    la.window = 0;
                    la.level = 0;
                    la.levels = 1;
                    la.planar = 0;
                    la.tol = 0.0f;
                    la.alpha2 = p->alpha * p->alpha;
                    la.taps = taps;
                    HR_CHECK(cudaMemsetAsync(lstatus, 0, (size_t)Bt * 4, st));
                    for (int rep = 0; rep <= kRounds; ++rep) {
                        HR_CHECK(cudaEventRecord(ev[0], st));
                        int e2 = launch_level(ctx, la, st);
                        if (e2) return e2;
                        HR_CHECK(cudaEventRecord(ev[1], st));
                        HR_CHECK(cudaEventSynchronize(ev[1]));
                        float t = 0.0f;
                        HR_CHECK(cudaEventElapsedTime(&t, ev[0], ev[1]));
                        t /= (float)kLoopCap;
                        if (rep == 1 || (rep > 1 && t < ms)) ms = t;
                    }
                }
                if (lv) {
                    strip::LoopArgs c;
                    c.s0 = (float2 *)s0;
                    c.s1 = (float2 *)s1;
                    c.hist = lhist;
                    c.iters = liters;
                    c.status = lstatus;
                    c.hist_stride = kLoopCap + 1;
                    c.cap = kLoopCap;
                    c.window = 0;   // no stop rule: every pair runs all iterations
                    c.level = 0;
                    c.levels = 1;
                    c.tol = 0.0f;
                    c.work = cnt + 2;
                    HR_CHECK(cudaMemsetAsync(lstatus, 0, (size_t)Bt * 4, st));
                    for (int rep = 0; rep <= kRounds; ++rep) {
                        HR_CHECK(cudaMemsetAsync(c.work, 0, sizeof(int), st));
                        HR_CHECK(cudaEventRecord(ev[0], st));
                        int e2 = launch_strip_loop(ctx, a, c, Bt, st);
                        if (e2) return e2;
                        HR_CHECK(cudaEventRecord(ev[1], st));
                        HR_CHECK(cudaEventSynchronize(ev[1]));
                        float t = 0.0f;
                        HR_CHECK(cudaEventElapsedTime(&t, ev[0], ev[1]));
                        t /= (float)(kLoopCap - 1);
                        if (rep == 1 || (rep > 1 && t < ms)) ms = t;
                    }
                }
                for (; !lv && !vv && k < kWarm; ++k) {
                    a.in = (k & 1) ? (const float2 *)s1 : (const float2 *)s0;
                    a.out = (k & 1) ? (float2 *)s0 : (float2 *)s1;
                    int e2 = sv ? launch_strip(ctx, true, a, Bt, st)
                                : dispatch_iter_tma(ctx, rad, v, true, tmS[k & 1], tmF, a, Bt * tiles, st);
                    if (e2) return e2;
                }
                for (int rep = 0; !lv && !vv && rep < kRounds; ++rep) {
                    HR_CHECK(cudaEventRecord(ev[0], st));
                    for (int j = 0; j < kBatch; ++j, ++k) {
                        a.in = (k & 1) ? (const float2 *)s1 : (const float2 *)s0;
                        a.out = (k & 1) ? (float2 *)s0 : (float2 *)s1;
                        int e2 = sv ? launch_strip(ctx, true, a, Bt, st)
                                    : dispatch_iter_tma(ctx, rad, v, true, tmS[k & 1], tmF, a, Bt * tiles, st);
                        if (e2) return e2;
                    }
                    HR_CHECK(cudaEventRecord(ev[1], st));
                    HR_CHECK(cudaEventSynchronize(ev[1]));
                    float t = 0.0f;
                    HR_CHECK(cudaEventElapsedTime(&t, ev[0], ev[1]));
                    t /= (float)kBatch;
                    if (rep == 0 || t < ms) ms = t;
                }
                if (ms_out) ms_out[l * kTileVariants + v] = ms;
                // shape 6 is timed but not chosen: its synthetic pairs all run the same number of
                // iterations, while on scan data a pair with many iterations holds its CTA alone
                // (shape 5 switches to the loop form by itself when every pair has a CTA)
                if (lv) continue;
                // Score = time x (1 + 1 % per halving of the tile area below 64 x 64): the
                // synthetic patterns (small, smooth displacements; every pair active) timed the
                // 64x32 and 64x64 shapes as a tie at 256x256 where the 64x64 one was 4 % faster
                // on the batched scan; a clearly faster small tile still wins.
                // Every shape but the level in shared memory (7) leaves the stop rule to a control
                // launch after each iteration, which this timing does not see: about 5 us per
                // iteration in the batched scan's launch list, added to their time.
                constexpr float kCtrlMs = 0.005f;
                const float extra = vv ? 0.0f : kCtrlMs;
                const float score = (ms + extra) *
                                    (1.0f + 0.01f * fmaxf(0.0f, log2f(4096.0f / (float)(kVarTX[v] * kVarTY[v]))));
                if (best_v == 0 && best == 0.0f) {
                    best = score;
                    best_v = v;
                } else if (score < best) {
                    best = score;
                    best_v = v;
                }
            }
            int e3 = hrebsd_set_tile_variant(ctx, h, w, best_v);
            if (e3) return e3;
        }
        return HREBSD_OK;
    };
    e = run();
    ctx->prof_on = prof;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e) return e;
    return hrebsd_device_error(ctx);
}

extern "C" int hrebsd_demons_register_batch(hrebsd_ctx *ctx, const float *ref, const float *test,
                                            const int32_t *ref_idx, int R, int B, int H, int W,
                                            const hrebsd_demons_params *p, const float *init_field, float *field,
                                            int32_t *iters, int32_t *pair_status, void *stream)
{
    int e = check_register_args(ctx, ref, test, ref_idx, R, B, H, W, p, field, iters, pair_status);
    if (e || B == 0) return e;
    const int L = p->levels;
    e = hr_set_device(ctx);
    if (e) return e;
    // pairs are processed in chunks so that the workspace stays bounded (~24 GB at 256x256)
    const size_t per_pair = (size_t)H * W * 4 * 2 * 4;   // u0, s0, s1 (+ pyramids), bytes
    size_t chunk = (size_t)24 << 30;
    chunk /= per_pair;
    if (chunk < 1) chunk = 1;
    const int start = (p->start_level < 0 || p->start_level >= L) ? L - 1 : p->start_level;
    cudaStream_t st = hr_stream(stream);
    for (int b0 = 0; b0 < B; b0 += (int)chunk) {
        int nb = (int)((size_t)(B - b0) < chunk ? (size_t)(B - b0) : chunk);
        const float *init = init_field ? init_field + (size_t)b0 * 2 * (H >> start) * (W >> start) : nullptr;
        e = register_chunk(ctx, ref, test + (size_t)b0 * H * W, ref_idx + b0, R, nb, H, W, p, init,
                           field + (size_t)b0 * 2 * H * W, iters + (size_t)b0 * L, pair_status + b0, st);
        if (e) return e;
    }
    return HREBSD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free registration.  Some callers cannot call cudaMalloc: hosts
// that enforce a fixed device-memory budget set up before they start, plugins
// whose host application owns the allocator, and latency-bound services where
// an allocation (which may synchronise the device) in the middle of a request
// is not allowed.  For them the workspace of the registration lives in one
// static device array of HREBSD_NOALLOC_SCRATCH_BYTES, which every process that
// loads this library holds on each device it uses until exit.  All calls share
// it and it keeps the previous call's contents: every slot is written before it
// is read (the initial field is zeroed or copied in explicitly), so nothing
// leaks from one call into the next, but calls that overlap on the GPU
// (different streams, or different host threads) race on the array and must be
// serialised by the caller.
namespace {

__device__ __align__(256) unsigned char hr_noalloc_scratch[HREBSD_NOALLOC_SCRATCH_BYTES];

// Device address of the array on the current device, looked up once per
// device (host code cannot use the symbol itself as a device address).  The
// cache entries are atomics: two host threads making the first call on a
// device at the same time both look the address up and store the same value.
int noalloc_scratch_address(int device, unsigned char **out)
{
    static std::atomic<unsigned char *> addr[256];
    if (device < 0 || device >= 256) return HREBSD_EINVAL;
    unsigned char *a = addr[device].load(std::memory_order_acquire);
    if (!a) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, hr_noalloc_scratch);
        if (e != cudaSuccess) return hr_cuda_error(e, "cudaGetSymbolAddress(hr_noalloc_scratch)", __FILE__, __LINE__);
        a = static_cast<unsigned char *>(p);
        addr[device].store(a, std::memory_order_release);
    }
    *out = a;
    return HREBSD_OK;
}

}  // namespace

extern "C" int hrebsd_demons_register_batch_noalloc(hrebsd_ctx *ctx, const float *ref, const float *test,
                                                    const int32_t *ref_idx, int R, int B, int H, int W,
                                                    const hrebsd_demons_params *p, const float *init_field,
                                                    float *field, int32_t *iters, int32_t *pair_status,
                                                    void *stream)
{
    int e = check_register_args(ctx, ref, test, ref_idx, R, B, H, W, p, field, iters, pair_status);
    if (e || B == 0) return e;
    size_t sb[WS_COUNT], off[WS_COUNT], total = 0;
    slot_bytes(R, B, H, W, p, sb);
    for (int k = 0; k < WS_COUNT; ++k) {
        off[k] = total;
        total += (sb[k] + 255) / 256 * 256;
    }
    if (total > (size_t)HREBSD_NOALLOC_SCRATCH_BYTES) return HREBSD_ESCRATCH;
    if ((e = hr_set_device(ctx))) return e;
    unsigned char *base = nullptr;
    if ((e = noalloc_scratch_address(ctx->device, &base))) return e;
    void *given[WS_COUNT];
    for (int k = 0; k < WS_COUNT; ++k) given[k] = base + off[k];
    ctx->no_events = 1;   // tracing would create CUDA events; skip it for this call
    e = register_chunk(ctx, ref, test, ref_idx, R, B, H, W, p, init_field, field, iters, pair_status,
                       hr_stream(stream), given);
    ctx->no_events = 0;
    return e;
}
