// Demons iteration as a vertical sweep over whole pattern rows (included by
// demons.cu; same arithmetic per pixel as the tile kernels, so the field is
// bit-identical to theirs).
//
// One CTA of NT = w threads owns one active pair of a level w pixels wide and
// walks down its rows in steps of R = 7 rows; thread t owns column t and warp
// v the 32 columns [32 v, 32 v + 32).  Per step:
//   x pass of G_f on the step's s rows, for the warp's own columns -> RX rows;
//   per column, in registers: the y pass of G_f over a rolling window of the
//     last 2r + 1 RX rows gives u (lagging the input by r rows); the bilinear
//     gathers of the moving image at x - u (with TEX one texture gather of the
//     cell's four pixels from a CUDA-array copy of the references, else four
//     loads) are issued for all R rows before any of them is used, then the
//     force of Eq. 1 (test-image rows staged in shared memory)  -> du rows;
//   one CTA barrier (the du rows' x pass reads r columns of the neighbouring
//     warps);
//   x pass of G_u on the du rows, for the warp's own columns     -> DX rows;
// and, at the start of the next step, per column: the y pass of G_u over a
// rolling window of DX rows, plus u, gives s_{k+1} (lagging by 2r rows),
// stored to HBM.  Everything but the du rows stays within a warp, so a step
// has a single CTA barrier (du rows alternate between two buffers).
// The separable passes read each input once per output in the vertical
// direction (register windows) and have no halo rows at all; the x passes
// read r halo columns on each side, which hold the row's edge values
// (replicated borders).  Rows outside the image repeat the edge row: the
// first row pushed into a window fills all of it, and after the last row the
// last DX row is pushed again.  A window of 2r + 1 = R rows keeps row y in
// slot y mod R, so its slots are compile-time indices in the unrolled row loop
// and nothing moves between registers.  The s and test-image rows of step
// k + 2 are requested by bulk copies (one per row, issued by 16 lanes of one
// warp, completion on an mbarrier that every thread waits on with a bounded
// wait) as soon as step k's barrier shows its buffer consumed.
namespace strip {

constexpr int R = 7;


template <int RAD, int NT>
struct Geo {
    static_assert(2 * RAD + 1 == R, "the register windows rotate with the step only for 2r + 1 = R");
    static_assert(RAD == 3, "rows with halo keep their data at a 16-byte boundary 4 elements in");
    static_assert(NT % 32 == 0 && NT >= 64 && NT / RUN == 4 * (NT / 32), "four x-pass runs per warp and row, two edge warps");
    static constexpr int HO = 4;                        // halo rows: data column c at index c + HO
    static constexpr int HST = NT + 10;                 // float2 stride of halo rows (odd 16-byte slots)
    static constexpr int XST = NT + 10;                 // float2 stride of RX / DX rows (the same)
    static constexpr int FR_ = R + 2;                   // test-image rows of a step
    static constexpr int FST = NT + 4;                  // float stride of test-image rows (odd 16-byte slots)
    static_assert((HST / 2) % 2 == 1 && (XST / 2) % 2 == 1 && (FST / 4) % 2 == 1, "odd numbers of 16-byte slots");
    static_assert((HST / 2) % 8 == 5 && (XST / 2) % 8 == 5, "the x-pass lane map below is conflict-free for 5 mod 8");
    static constexpr size_t S_OFF = 0;                                   // s rows [2][R][HST] float2
    static constexpr size_t F_OFF = S_OFF + (size_t)2 * R * HST * 8;     // test rows [2][FR_][FST] float
    static constexpr size_t D_OFF = F_OFF + (size_t)2 * FR_ * FST * 4;   // du rows [2][R][HST] float2
    static constexpr size_t X_OFF = D_OFF + (size_t)2 * R * HST * 8;     // RX rows [R][XST] float2
    static constexpr size_t Y_OFF = X_OFF + (size_t)R * XST * 8;         // DX rows [R][XST] float2
    static constexpr size_t BYTES = Y_OFF + (size_t)R * XST * 8;
    static constexpr uint32_t S_BYTES = (uint32_t)R * NT * 8;            // bytes of a step's s rows
    static constexpr uint32_t F_BYTES = (uint32_t)FR_ * NT * 4;          // ... and test-image rows
    static_assert(S_OFF % 16 == 0 && F_OFF % 16 == 0 && X_OFF % 16 == 0 && D_OFF % 16 == 0 && Y_OFF % 16 == 0,
                  "16-byte aligned regions");
};

// The bulk copies of step k of a pair into one buffer: s rows clamp(R k + i) (i < R) of the pair's
// plane sp (when copy_s) and test-image rows clamp(R k - r - 1 + i) (i < R + 2) of its plane fp, whole
// rows.  Called by every lane of one warp: lane 0 announces the bytes, then lanes 0 .. R - 1 copy the
// s rows and lanes R .. 2R + 1 the test rows.
template <int RAD, int NT>
__device__ __forceinline__ void issue_step(bool copy_s, const float2 *sp, const float *fp, int h, int k, float2 *sS,
                                           float *sF, uint64_t *bar, int lane)
{
    using G = Geo<RAD, NT>;
    if (lane == 0) hr_tma::mbar_arrive_expect_tx(bar, (copy_s ? G::S_BYTES : 0u) + G::F_BYTES);
    __syncwarp();
    if (lane < R) {
        if (copy_s) {
            hr_tma::fence_proxy_async();   // the buffer's previous contents were read by the generic proxy
            hr_tma::load_bulk(sS + lane * G::HST + G::HO, sp + (size_t)min(R * k + lane, h - 1) * NT, NT * 8, bar);
        }
    } else if (lane < R + G::FR_) {
        const int i = lane - R;
        hr_tma::fence_proxy_async();
        hr_tma::load_bulk(sF + i * G::FST, fp + (size_t)min(max(R * k - RAD - 1 + i, 0), h - 1) * NT, NT * 4, bar);
    }
}

// The whole level in one launch (the row sweep's LOOP form): every active pair iterates in its CTA
// until the stop rule of the control kernel (same rule, same FP64 history, one SSD partial per pair)
// ends it, so the level needs no launch per iteration.  Iterations k >= 1; iteration 0 (which reads
// u_0) runs as a plain launch first.  A CTA whose pair stops takes the next item of the active list
// from an atomic counter, so pairs with many iterations do not hold up a fixed share of the list.
struct LoopArgs {
    float2 *s0, *s1;        // s_k for even / odd k
    double *hist;           // [B][hist_stride]
    int32_t *iters;         // [B][levels]
    int32_t *status;        // [B]
    int *work;              // the next item of the active list to take (zero at launch)
    int hist_stride, cap, window, level, levels;
    float tol;
};

// x pass of the run of RUN outputs starting at column c0 of a row with halo (data column c at
// index c + HO = c + r + 1): an aligned window of RUN + 2r + 2 elements from column c0 - r - 1,
// used from its second element.  Same sums as run_x.
template <int RAD>
__device__ __forceinline__ void run_x_halo(const float2 *row, int c0, float2 *out, const float2 (&t)[2 * RAD + 1])
{
    constexpr int NW = RUN + 2 * RAD + 2;   // 16 elements: columns c0 - 4 .. c0 + 11
    float2 win[NW];
    const float4 *in4 = reinterpret_cast<const float4 *>(row + c0);   // index c0 = column c0 - 4
#pragma unroll
    for (int j = 0; j < NW / 2; ++j) {
        const float4 v = in4[j];
        win[2 * j] = make_float2(v.x, v.y);
        win[2 * j + 1] = make_float2(v.z, v.w);
    }
    float2 acc[RUN];
#pragma unroll
    for (int o = 0; o < RUN; ++o) acc[o] = __fmul2_rn(t[0], win[o + 1]);
#pragma unroll
    for (int k = 1; k <= 2 * RAD; ++k)
#pragma unroll
        for (int o = 0; o < RUN; ++o) acc[o] = ffma2(t[k], win[o + 1 + k], acc[o]);
    float4 *out4 = reinterpret_cast<float4 *>(out);
#pragma unroll
    for (int o = 0; o < RUN; o += 2) out4[o / 2] = make_float4(acc[o].x, acc[o].y, acc[o + 1].x, acc[o + 1].y);
}

template <int RAD, int NT, bool IN_S, bool LOOP, bool TEX>
__global__ void __launch_bounds__(NT, 512 / NT) demons_strip_kernel(IterArgs a, LoopArgs c)
{
    static_assert(!LOOP || IN_S, "the loop form runs the iterations k >= 1, which read s_k");
    using G = Geo<RAD, NT>;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sS0 = reinterpret_cast<float2 *>(smraw + G::S_OFF);
    float *sF0 = reinterpret_cast<float *>(smraw + G::F_OFF);
    float2 *sD0 = reinterpret_cast<float2 *>(smraw + G::D_OFF);
    float2 *sRX = reinterpret_cast<float2 *>(smraw + G::X_OFF);
    float2 *sDX = reinterpret_cast<float2 *>(smraw + G::Y_OFF);
    __shared__ float red[NT / 32];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_next;   // LOOP: the pair's next iteration, or -1 once the stop rule ended it
    __shared__ int s_item;   // LOOP: the item taken from the counter

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int NWARP = NT / 32;
    // the Gaussian taps are symmetric (t[j] = t[2r - j]): half of them in registers
    float2 tfh[RAD + 1], tuh[RAD + 1];
#pragma unroll
    for (int k = 0; k <= RAD; ++k) {
        tfh[k] = make_float2(a.taps.f[k], a.taps.f[k]);
        tuh[k] = make_float2(a.taps.up[k], a.taps.up[k]);
    }
    float2 tf[2 * RAD + 1], tu[2 * RAD + 1];
#pragma unroll
    for (int k = 0; k <= 2 * RAD; ++k) {
        tf[k] = tfh[k <= RAD ? k : 2 * RAD - k];
        tu[k] = tuh[k <= RAD ? k : 2 * RAD - k];
    }
    const int n_active = *a.n_active;
    if (!LOOP && blockIdx.x == 0 && t == 0) {
        *a.n_next_reset = 0;
        if (a.px_count) atomicAdd(a.px_count, (unsigned long long)n_active * a.h * a.w);
    }
    if (t == 0) {
        hr_tma::mbar_init(&bar[0], 1);
        hr_tma::mbar_init(&bar[1], 1);
        hr_tma::fence_mbar_init();
    }
    __syncthreads();
    const int h = a.h;
    const size_t plane = (size_t)h * NT;
    const int nsteps = (h + 2 * RAD + R - 1) / R;   // >= 2 for h >= 8
    // a step whose u / du rows R k - r .. R k + r all lie in 1 .. h - 2 and whose s rows start below
    // row 0: no window fill, no edge row, no row outside the image (and likewise for its outputs)
    auto interior_step = [&](int k) { return k >= 1 && R * k + RAD <= h - 2; };
    // one-sided difference (scale 1) in the first and last column; clamped neighbour columns
    const float sx = (t == 0 || t == NT - 1) ? 1.0f : 0.5f;
    const int tl = max(t - 1, 0), tr = min(t + 1, NT - 1);
    const float tf_ = (float)t, mx2 = (float)(NT - 2), my2 = (float)(h - 2);
    const float al2 = a.alpha2;
    // this lane's x-pass run: row xi, run xs of the warp's 4 (columns [xc0, xc0 + RUN)).  The 28 runs
    // of R rows x 4 fill lanes 0..6 of each group of 8 (lane 7 idle), chosen so that the 16-byte
    // slots (5 xi + 4 xs + j) mod 8 that the 8 lanes of a shared-memory phase touch are distinct
    // (row strides of 5 mod 8 slots): rows 0-2 x runs {0,1} and {2,3} with row 3 run 0 / 1 in the
    // first two groups, row 3 run 2 / 3 with rows 4-6 x runs {0,1} and {2,3} in the last two.
    const int xp = lane >> 3, xq = lane & 7;
    const bool xlane = xq != 7;
    const int xi = xp < 2 ? (xq < 6 ? xq >> 1 : 3) : (xq == 0 ? 3 : 4 + ((xq - 1) >> 1));
    const int xs = xp < 2 ? (xq < 6 ? (xq & 1) + 2 * xp : xp) : (xq == 0 ? xp : ((xq - 1) & 1) + 2 * (xp - 2));
    const int xc0 = (4 * warp + xs) * RUN;
    // the r halo columns on each side of R halo rows take the row's edge value (lanes 0 .. R - 1 of
    // the first and the last warp, one row each), visible to the warp after the __syncwarp
    auto fill_halo = [&](float2 *rows) {
        if ((warp == 0 || warp == NWARP - 1) && lane < R) {
            float2 *row = rows + lane * G::HST;
            const int c = warp == 0 ? 0 : NT - 1, o = warp == 0 ? -RAD : 1;
            const float2 v = row[G::HO + c];
#pragma unroll
            for (int j = 0; j < RAD; ++j) row[G::HO + c + o + j] = v;
        }
        __syncwarp();
    };

    // the planes that iteration kk of a pair reads (s_kk, or u_0 when !IN_S) and writes (s_kk+1)
    auto src_of = [&](int pair, int kk) -> const float2 * {
        return (LOOP ? ((kk & 1) ? c.s1 : c.s0) : a.in) + (size_t)pair * plane;
    };
    auto dst_of = [&](int pair, int kk) -> float2 * {
        return (LOOP ? (((kk + 1) & 1) ? c.s1 : c.s0) : a.out) + (size_t)pair * plane;
    };
    auto fsrc_of = [&](int pair) { return a.Ftest + (size_t)pair * plane; };
    constexpr int K_FIRST = LOOP ? 1 : 0;   // the iteration of an item's first sweep (LOOP: after k = 0)

    int item = blockIdx.x;
    if (LOOP) {
        if (t == 0) s_item = atomicAdd(c.work, 1);
        __syncthreads();
        item = s_item;
    }
    uint32_t g = 0;   // steps of this CTA so far: step g uses buffer g & 1, phase parity (g >> 1) & 1
    if (warp == 0 && item < n_active) {
        const int p0 = a.active[item];
        issue_step<RAD, NT>(IN_S, src_of(p0, K_FIRST), fsrc_of(p0), h, 0, sS0, sF0, &bar[0], lane);
        issue_step<RAD, NT>(IN_S, src_of(p0, K_FIRST), fsrc_of(p0), h, 1, sS0 + R * G::HST, sF0 + G::FR_ * G::FST,
                            &bar[1], lane);
    }
    while (item < n_active) {
        const int pair = a.active[item];
        const int next_pair = !LOOP && item + (int)gridDim.x < n_active ? a.active[item + gridDim.x] : -1;
        int next_item = item + (int)gridDim.x;
        const int ref = __ldg(a.ref_idx + pair);
        const float *M = a.Mref + (size_t)ref * plane;
        // TEX: texture row of the cell's upper row y0 is ref h + y0, and the gather of the texels
        // (x0, y0) .. (x0 + 1, y0 + 1) is taken at the coordinate (x0 + 1, ref h + y0 + 1)
        const float yt = (float)(ref * h) + 1.0f;
        const float2 *u0 = a.in + (size_t)pair * plane;   // the level's initial field when !IN_S
        const float *fp = fsrc_of(pair);
      for (int kit = K_FIRST;; ++kit) {   // LOOP: the pair's iterations; otherwise the one sweep
        const float2 *sp = src_of(pair, kit);
        float2 *dst = dst_of(pair, kit);
        float2 rxw[R], dxw[R], ucur[R], uprev[RAD], last_dx = make_float2(0.0f, 0.0f);
        float ssd = 0.0f;
        for (int k = 0; k <= nsteps; ++k) {
            // ---- outputs of step k - 1: y pass of G_u over the DX window, s = u + G_u * du
            // (DX rows of the warp's own columns, written by this warp before its __syncwarp).
            // Interior steps (every row inside, none at an edge) run without the edge handling.
            if (k > 0) {
                const int kp = k - 1;
                float2 *dk = dst + (ptrdiff_t)(R * kp - 2 * RAD) * NT + t;   // row yo for i = 0
                auto outputs = [&](auto interior) {
                    constexpr bool IN = decltype(interior)::value;
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        const int yu = R * kp + i - RAD, yo = yu - RAD;   // du row entering, output row
                        if (IN || yu >= 0) {
                            const float2 v = (IN || yu < h) ? sDX[i * G::XST + t] : last_dx;
                            if (!IN && yu < h) last_dx = v;
                            dxw[(i + R - RAD) % R] = v;   // row yu in slot yu mod R
                            if (!IN && yu == 0) {
#pragma unroll
                                for (int j = 0; j < R; ++j) dxw[j] = v;
                            }
                        }
                        if (IN || (yo >= 0 && yo < h)) {
                            // rows yo - r + j = yu - 2r + j sit in slots (i - 3r + j) mod R
                            float2 acc = __fmul2_rn(tu[0], dxw[(i + 2 * R - 3 * RAD) % R]);
#pragma unroll
                            for (int j = 1; j < R; ++j) acc = ffma2(tu[j], dxw[(i + 2 * R - 3 * RAD + j) % R], acc);
                            const float2 uo = i >= RAD ? ucur[i - RAD] : uprev[i];
                            dk[i * NT] = __fadd2_rn(uo, acc);   // row yo
                        }
                    }
                };
                if (interior_step(kp)) outputs(std::true_type());
                else outputs(std::false_type());
#pragma unroll
                for (int i = 0; i < RAD; ++i) uprev[i] = ucur[R - RAD + i];
            }
            if (k == nsteps) {
                // LOOP: the next iteration's bulk copies read these rows of s_{k+1} (async proxy)
                if (LOOP) asm volatile("fence.proxy.async.global;" ::: "memory");
                break;
            }
            const int b = g & 1;
            float2 *sS = sS0 + b * R * G::HST;
            float *sF = sF0 + b * G::FR_ * G::FST;
            float2 *sD = sD0 + b * R * G::HST;
            // step k's rows: every thread waits for the bulk copies (bounded; a wait that gives up
            // is reported at the barrier below, which every thread reaches)
            bool ok = hr_tma::mbar_wait(&bar[b], (g >> 1) & 1u);
            // ---- x pass of G_f on the s rows -> RX (the warp's own columns; the edge warps first
            // fill the halo columns of the rows with the edge values)
            if (IN_S) {
                fill_halo(sS);
                if (xlane) run_x_halo<RAD>(sS + xi * G::HST, xc0, sRX + xi * G::XST + xc0, tf);
                __syncwarp();
            }
            // ---- y pass of G_f: u for rows yu = R k + i - r; the moving image at x - u (every row's
            // four gathers first); the force of Eq. 1
            const float yk = (float)(R * k - RAD);
            auto force_rows = [&](auto interior) {
                constexpr bool IN = decltype(interior)::value;
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int y = R * k + i, yu = y - RAD;
                    float2 u;
                    if (IN_S) {
                        const float2 v = sRX[i * G::XST + t];
                        rxw[i] = v;   // row y in slot y mod R = i
                        if (!IN && y == 0) {
#pragma unroll
                            for (int j = 0; j < R; ++j) rxw[j] = v;
                        }
                        // rows y - 2r + j sit in slots (i - 2r + j) mod R
                        u = __fmul2_rn(tf[0], rxw[(i + R - 2 * RAD) % R]);
#pragma unroll
                        for (int j = 1; j < R; ++j) u = ffma2(tf[j], rxw[(i + R - 2 * RAD + j) % R], u);
                    } else {
                        u = (IN || (yu >= 0 && yu < h)) ? u0[(size_t)yu * NT + t] : make_float2(0.0f, 0.0f);
                    }
                    ucur[i] = u;
                }
                float mA[R], mB[R], mC[R], mD[R], fxv[R], fyv[R];
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int yu = R * k + i - RAD;
                    // row coordinate as a float (exact integers); rows outside: any valid cell
                    const float yc = IN ? yk + (float)i : (float)min(max(yu, 0), h - 1);
                    if constexpr (TEX) {
                        // one gather returns (x0, y0 + 1), (x0 + 1, y0 + 1), (x0 + 1, y0), (x0, y0)
                        float xc, ycl;
                        warp_cell_ff(tf_, ucur[i].x, mx2, xc, fxv[i]);
                        warp_cell_ff(yc, ucur[i].y, my2, ycl, fyv[i]);
                        const float4 q = tex2Dgather<float4>(a.mtex, xc + 1.0f, ycl + yt, 0);
                        mA[i] = q.w;
                        mB[i] = q.z;
                        mC[i] = q.x;
                        mD[i] = q.y;
                    } else {
                        int x0, y0;
                        warp_cell_f(tf_, ucur[i].x, mx2, x0, fxv[i]);
                        warp_cell_f(yc, ucur[i].y, my2, y0, fyv[i]);
                        const float *p = M + y0 * NT + x0;
                        mA[i] = __ldg(p);
                        mB[i] = __ldg(p + 1);
                        mC[i] = __ldg(p + NT);
                        mD[i] = __ldg(p + NT + 1);
                    }
                }
                // the force of one row (scalar) ...
                auto force1 = [&](int i, int yu) {
                    // test image rows yu - 1 .. yu + 1 are staged rows i .. i + 2
                    const float *fr_ = sF + i * G::FST;
                    const float fc = fr_[G::FST + t], fup = fr_[t], fdn = fr_[2 * G::FST + t];
                    const float fl = fr_[G::FST + tl], frt = fr_[G::FST + tr];
                    const float sy = (!IN && (yu == 0 || yu == h - 1)) ? 1.0f : 0.5f;
                    const float fx = fxv[i], fy = fyv[i];
                    const float omx = fmaf(fx, -1.0f, 1.0f), omy = fmaf(fy, -1.0f, 1.0f);
                    const float top = fmaf(fx, mB[i], omx * mA[i]), bot = fmaf(fx, mD[i], omx * mC[i]);
                    const float mw = fmaf(fy, bot, omy * top);
                    const float gx = sx * fmaf(fl, -1.0f, frt), gy = sy * fmaf(fup, -1.0f, fdn);
                    const float d = fmaf(fc, -1.0f, mw);
                    const float den = fmaf(gx, gx, fmaf(gy, gy, (al2 * d) * d));
                    const float tt = den > 1e-9f ? __fdividef(d, den) : 0.0f;
                    sD[i * G::HST + G::HO + t] = make_float2(tt * gx, tt * gy);
                    ssd = fmaf(d, d, ssd);
                };
                // ... and of rows i, i + 1 of an interior step in packed FP32x2 arithmetic (every
                // rounding step that of force1: a - b as fma(b, -1, a), products and fmas in order)
                auto force2 = [&](int i) {
                    const float *fr_ = sF + i * G::FST;
                    const float f0 = fr_[t], f1 = fr_[G::FST + t], f2 = fr_[2 * G::FST + t], f3 = fr_[3 * G::FST + t];
                    const float2 fl = make_float2(fr_[G::FST + tl], fr_[2 * G::FST + tl]);
                    const float2 frt = make_float2(fr_[G::FST + tr], fr_[2 * G::FST + tr]);
                    const float2 n1 = make_float2(-1.0f, -1.0f), one = make_float2(1.0f, 1.0f);
                    const float2 fx = make_float2(fxv[i], fxv[i + 1]), fy = make_float2(fyv[i], fyv[i + 1]);
                    const float2 omx = __ffma2_rn(fx, n1, one), omy = __ffma2_rn(fy, n1, one);
                    const float2 top = __ffma2_rn(fx, make_float2(mB[i], mB[i + 1]),
                                                  __fmul2_rn(omx, make_float2(mA[i], mA[i + 1])));
                    const float2 bot = __ffma2_rn(fx, make_float2(mD[i], mD[i + 1]),
                                                  __fmul2_rn(omx, make_float2(mC[i], mC[i + 1])));
                    const float2 mw = __ffma2_rn(fy, bot, __fmul2_rn(omy, top));
                    const float2 gx = __fmul2_rn(make_float2(sx, sx), __ffma2_rn(fl, n1, frt));
                    const float2 gy = __fmul2_rn(make_float2(0.5f, 0.5f), __ffma2_rn(make_float2(f0, f1), n1, make_float2(f2, f3)));
                    const float2 d = __ffma2_rn(make_float2(f1, f2), n1, mw);
                    const float2 a2 = make_float2(al2, al2);
                    const float2 den = __ffma2_rn(gx, gx, __ffma2_rn(gy, gy, __fmul2_rn(__fmul2_rn(a2, d), d)));
                    const float t0 = den.x > 1e-9f ? __fdividef(d.x, den.x) : 0.0f;
                    const float t1 = den.y > 1e-9f ? __fdividef(d.y, den.y) : 0.0f;
                    sD[i * G::HST + G::HO + t] = make_float2(t0 * gx.x, t0 * gy.x);
                    sD[(i + 1) * G::HST + G::HO + t] = make_float2(t1 * gx.y, t1 * gy.y);
                    ssd = fmaf(d.x, d.x, ssd);
                    ssd = fmaf(d.y, d.y, ssd);
                };
                if (IN) {
#pragma unroll
                    for (int i = 0; i + 1 < R; i += 2) force2(i);
                    force1(R - 1, R * k - RAD + R - 1);
                } else {
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        const int yu = R * k + i - RAD;
                        if (yu >= 0 && yu < h) force1(i, yu);
                    }
                }
            };
            if (interior_step(k)) force_rows(std::true_type());
            else force_rows(std::false_type());
            // du rows complete; step k's s and test rows consumed by every warp
            if (!__syncthreads_and(ok)) {   // a copy did not arrive: report, let this CTA's copies land, stop
                if (t == 0) {
                    atomicExch(a.err, 1);
                    hr_tma::mbar_wait(&bar[b], (g >> 1) & 1u);
                    if (k + 1 < nsteps || (!LOOP && next_pair >= 0))
                        hr_tma::mbar_wait(&bar[b ^ 1], ((g + 1) >> 1) & 1u);
                }
                return;
            }
            if (warp == 0) {   // step k + 2 into the buffer just consumed
                if (k + 2 < nsteps)
                    issue_step<RAD, NT>(IN_S, sp, fp, h, k + 2, sS, sF, &bar[b], lane);
                else if (!LOOP && next_pair >= 0)
                    issue_step<RAD, NT>(IN_S, src_of(next_pair, K_FIRST), fsrc_of(next_pair), h, k + 2 - nsteps, sS,
                                        sF, &bar[b], lane);
            }
            // ---- x pass of G_u on the du rows that exist -> DX (the warp's own columns; the edge
            // warps first fill the halo columns with the edge values)
            fill_halo(sD);
            if (xlane) {
                const int yu = R * k + xi - RAD;
                if (yu >= 0 && yu < h) run_x_halo<RAD>(sD + xi * G::HST, xc0, sDX + xi * G::XST + xc0, tu);
            }
            __syncwarp();
            ++g;
        }
        // SSD of the pair (one partial: the level runs with tiles = 1)
        for (int o = 16; o > 0; o >>= 1) ssd += __shfl_xor_sync(0xffffffffu, ssd, o);
        if (lane == 0) red[warp] = ssd;
        __syncthreads();
        if (!LOOP) {
            if (t == 0) {
                float s = 0.0f;
                for (int j = 0; j < NWARP; ++j) s += red[j];
                a.part[(size_t)pair * a.tiles] = s;
            }
            break;
        }
        if (t == 0) {   // the control kernel's stop rule after iteration kit, on the same FP64 history
            float s = 0.0f;
            for (int j = 0; j < NWARP; ++j) s += red[j];
            const double E = 0.0 + (double)s;
            double *hh = c.hist + (size_t)pair * c.hist_stride;
            hh[kit] = E;
            int32_t *itp = c.iters + (size_t)pair * c.levels + c.level;
            int nk = -1;
            if (!isfinite(E)) {
                *itp = kit;
                c.status[pair] |= HREBSD_PAIR_NONFINITE;
            } else if (c.window > 0 && kit >= c.window && (hh[kit - c.window] - E) < (double)c.tol * hh[kit - c.window]) {
                *itp = kit;
            } else if (kit + 1 >= c.cap) {
                *itp = c.cap;
                c.status[pair] |= HREBSD_PAIR_CAPPED;
            } else {
                nk = kit + 1;
            }
            if (a.px_count) atomicAdd(a.px_count, (unsigned long long)h * NT);
            if (nk < 0) s_item = atomicAdd(c.work, 1);
            s_next = nk;
        }
        __syncthreads();
        const int nk = s_next;
        if (nk < 0) {   // the pair is done: the next item's first two steps
            next_item = s_item;
            if (warp == 0 && next_item < n_active) {
                const int np = a.active[next_item];
                issue_step<RAD, NT>(true, src_of(np, K_FIRST), fsrc_of(np), h, 0, sS0 + (g & 1) * R * G::HST,
                                    sF0 + (g & 1) * G::FR_ * G::FST, &bar[g & 1], lane);
                issue_step<RAD, NT>(true, src_of(np, K_FIRST), fsrc_of(np), h, 1, sS0 + ((g + 1) & 1) * R * G::HST,
                                    sF0 + ((g + 1) & 1) * G::FR_ * G::FST, &bar[(g + 1) & 1], lane);
            }
            break;
        }
        if (warp == 0) {   // the pair's next iteration: its first two steps
            issue_step<RAD, NT>(true, src_of(pair, nk), fp, h, 0, sS0 + (g & 1) * R * G::HST,
                                sF0 + (g & 1) * G::FR_ * G::FST, &bar[g & 1], lane);
            issue_step<RAD, NT>(true, src_of(pair, nk), fp, h, 1, sS0 + ((g + 1) & 1) * R * G::HST,
                                sF0 + ((g + 1) & 1) * G::FR_ * G::FST, &bar[(g + 1) & 1], lane);
        }
      }
        item = next_item;
    }
}

}  // namespace strip
