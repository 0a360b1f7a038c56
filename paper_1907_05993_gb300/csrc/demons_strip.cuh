// Demons iteration as a vertical sweep over whole pattern rows (included by
// demons.cu; same arithmetic per pixel as the tile kernels).
//
// One CTA of NT = w threads owns one active pair of a level w pixels wide and
// walks down its rows in steps of R = 7 rows; thread t owns column t.  Per step:
//   x pass of G_f on the step's s rows (runs of 8 outputs from a staged copy
//     of the rows with replicated edge columns)                    -> RX rows;
//   per column, in registers: the y pass of G_f over a rolling window of the
//     last 2r + 1 RX rows gives u (lagging the input by r rows), the warp of
//     the moving image at x - u and the force of Eq. 1 (test-image rows
//     staged in shared memory with replicated edges)               -> du rows;
//   x pass of G_u on the du rows                                   -> DX rows;
//   per column: the y pass of G_u over a rolling window of DX rows, plus u,
//     gives s_{k+1} (lagging by 2r rows), stored to HBM.
// The separable passes thus read each input once per output in the vertical
// direction (register windows) and have no halo rows at all; only the x passes
// read a halo of r columns, replicated at the image edges.  Rows outside the
// image repeat the edge row: the first row pushed into a window fills all of
// it, and after the last row the last du row is pushed again.  The window
// length 2r + 1 = 7 equals R, so the register windows rotate back to their
// starting positions every step.  The next step's s and test-image rows are
// copied by cp.async while the current step is computed.
namespace strip {

constexpr int R = 7;

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <int RAD, int NT>
struct Geo {
    static_assert(2 * RAD + 1 == R, "the register windows rotate with the step only for 2r + 1 = R");
    static constexpr int SW = NT + 2 * RAD;             // staged s / du row: columns [-r, NT + r)
    static constexpr int SST = (SW / 2) % 2 ? SW : SW + 2;   // row stride (float2): odd number of 16-byte slots
    static constexpr int FR_ = R + 2;                   // test-image rows of a step
    static constexpr int FST = NT + 2 + ((NT + 2) % 4 == 1 ? 0 : 1);  // row stride (float): columns [-1, NT]
    static constexpr int XST = NT + 2;                  // RX / DX row stride (float2)
    static constexpr size_t S_OFF = 0;                                    // [2][R][SST] float2
    static constexpr size_t F_OFF = S_OFF + (size_t)2 * R * SST * 8;      // [2][FR_][FST] float
    static constexpr size_t X_OFF = F_OFF + (((size_t)2 * FR_ * FST * 4 + 15) / 16) * 16;   // [R][XST] float2
    static constexpr size_t D_OFF = X_OFF + (size_t)R * XST * 8;         // [R][SST] float2
    static constexpr size_t BYTES = D_OFF + (size_t)R * SST * 8;
};

// The cp.async copies of step k of a pair: s rows clamp(7k + i) (i < R) with columns [-r, NT + r)
// clamped, and test-image rows clamp(7k - r - 1 + i) (i < R + 2) with columns [-1, NT] clamped.
template <int RAD, int NT, bool IN_S>
__device__ __forceinline__ void stage_copies(const IterArgs &a, int pair, int k, float2 *sS, float *sF)
{
    using G = Geo<RAD, NT>;
    const int h = a.h;
    const size_t plane = (size_t)h * NT;
    if (IN_S) {
        const float2 *src = a.in + (size_t)pair * plane;
        for (int idx = threadIdx.x; idx < R * G::SW; idx += NT) {
            const int i = idx / G::SW, c = idx - i * G::SW;
            const int gy = min(7 * k + i, h - 1), gx = min(max(c - RAD, 0), NT - 1);
            cp_async8(sS + i * G::SST + c, src + (size_t)gy * NT + gx);
        }
    }
    const float *fsrc = a.Ftest + (size_t)pair * plane;
    for (int idx = threadIdx.x; idx < G::FR_ * (NT + 2); idx += NT) {
        const int i = idx / (NT + 2), c = idx - i * (NT + 2);
        const int gy = min(max(7 * k - RAD - 1 + i, 0), h - 1), gx = min(max(c - 1, 0), NT - 1);
        cp_async4(sF + i * G::FST + c, fsrc + (size_t)gy * NT + gx);
    }
    cp_async_commit();
}

template <int RAD, int NT, bool IN_S>
__global__ void __launch_bounds__(NT, 512 / NT) demons_strip_kernel(IterArgs a)
{
    using G = Geo<RAD, NT>;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sS0 = reinterpret_cast<float2 *>(smraw + G::S_OFF);
    float *sF0 = reinterpret_cast<float *>(smraw + G::F_OFF);
    float2 *sX = reinterpret_cast<float2 *>(smraw + G::X_OFF);
    float2 *sD = reinterpret_cast<float2 *>(smraw + G::D_OFF);
    __shared__ float red[NT / 32];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float2 tf[2 * RAD + 1], tu[2 * RAD + 1];
#pragma unroll
    for (int k = 0; k <= 2 * RAD; ++k) {
        tf[k] = make_float2(a.taps.f[k], a.taps.f[k]);
        tu[k] = make_float2(a.taps.up[k], a.taps.up[k]);
    }
    const int n_active = *a.n_active;
    if (blockIdx.x == 0 && t == 0) {
        *a.n_next_reset = 0;
        if (a.px_count) atomicAdd(a.px_count, (unsigned long long)n_active * a.h * a.w);
    }
    const int h = a.h;
    const size_t plane = (size_t)h * NT;
    const int nsteps = (h + 2 * RAD + R - 1) / R;
    // one-sided difference (scale 1) in the first and last column
    const float sx = (t == 0 || t == NT - 1) ? 1.0f : 0.5f;
    const float al2 = a.alpha2;

    for (int item = blockIdx.x; item < n_active; item += gridDim.x) {
        const int pair = a.active[item];
        const float *M = a.Mref + (size_t)__ldg(a.ref_idx + pair) * plane;
        const float2 *u0 = a.in + (size_t)pair * plane;   // the level's initial field when !IN_S
        float2 *dst = a.out + (size_t)pair * plane;
        float2 rxw[R], dxw[R], ucur[R], uprev[R], last_dx = make_float2(0.0f, 0.0f);
        float ssd = 0.0f;
        stage_copies<RAD, NT, IN_S>(a, pair, 0, sS0, sF0);
        for (int k = 0; k < nsteps; ++k) {
            float2 *sS = sS0 + (k & 1) * R * G::SST;
            float *sF = sF0 + (k & 1) * G::FR_ * G::FST;
            cp_async_wait_all();
            __syncthreads();   // step k's rows staged; the previous step's DX rows consumed
            if (k + 1 < nsteps)
                stage_copies<RAD, NT, IN_S>(a, pair, k + 1, sS0 + ((k + 1) & 1) * R * G::SST,
                                            sF0 + ((k + 1) & 1) * G::FR_ * G::FST);
            // ---- x pass of G_f on the step's s rows: RX [R][NT]
            if (IN_S) {
                constexpr int NSEG = NT / RUN;
                for (int it = t; it < R * NSEG; it += NT) {
                    const int i = it % R, seg = it / R;
                    run_x<RAD>(sS + i * G::SST + seg * RUN, sX + i * G::XST + seg * RUN, tf);
                }
                __syncthreads();
            }
            // ---- per column: y pass of G_f, warp, force, du rows
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int y = R * k + i, yu = y - RAD;   // input row, u row
                float2 u;
                if (IN_S) {
                    const float2 v = sX[i * G::XST + t];
                    if (y == 0) {
#pragma unroll
                        for (int j = 0; j < R; ++j) rxw[j] = v;
                    } else {
#pragma unroll
                        for (int j = 0; j < R - 1; ++j) rxw[j] = rxw[j + 1];
                        rxw[R - 1] = v;
                    }
                    u = __fmul2_rn(tf[0], rxw[0]);
#pragma unroll
                    for (int j = 1; j < R; ++j) u = ffma2(tf[j], rxw[j], u);
                } else {
                    u = yu >= 0 && yu < h ? u0[(size_t)yu * NT + t] : make_float2(0.0f, 0.0f);
                }
                ucur[i] = u;
                if (yu >= 0 && yu < h) {
                    // test image rows yu - 1 .. yu + 1 are staged rows i .. i + 2
                    const float *fr_ = sF + i * G::FST + t + 1;
                    const float fc = fr_[G::FST], fup = fr_[0], fdn = fr_[2 * G::FST];
                    const float fl = fr_[G::FST - 1], frt = fr_[G::FST + 1];
                    const float sy = (yu == 0 || yu == h - 1) ? 1.0f : 0.5f;
                    int x0, y0;
                    float fx, fy;
                    warp_cell(t, u.x, NT, x0, fx);
                    warp_cell(yu, u.y, h, y0, fy);
                    const float *p = M + y0 * NT + x0;
                    const float A = __ldg(p), Bv = __ldg(p + 1), C = __ldg(p + NT), D = __ldg(p + NT + 1);
                    const float omx = fmaf(fx, -1.0f, 1.0f), omy = fmaf(fy, -1.0f, 1.0f);
                    const float top = fmaf(fx, Bv, omx * A), bot = fmaf(fx, D, omx * C);
                    const float mw = fmaf(fy, bot, omy * top);
                    const float gx = sx * fmaf(fl, -1.0f, frt), gy = sy * fmaf(fup, -1.0f, fdn);
                    const float d = fmaf(fc, -1.0f, mw);
                    const float den = fmaf(gx, gx, fmaf(gy, gy, (al2 * d) * d));
                    const float tt = den > 1e-9f ? __fdividef(d, den) : 0.0f;
                    const float2 du = make_float2(tt * gx, tt * gy);
                    float2 *drow = sD + i * G::SST;
                    drow[RAD + t] = du;
                    if (t == 0) {
#pragma unroll
                        for (int j = 0; j < RAD; ++j) drow[j] = du;
                    }
                    if (t == NT - 1) {
#pragma unroll
                        for (int j = 0; j < RAD; ++j) drow[RAD + NT + j] = du;
                    }
                    ssd = fmaf(d, d, ssd);
                }
            }
            __syncthreads();   // du rows complete
            // ---- x pass of G_u on the du rows that exist: DX [R][NT]
            {
                constexpr int NSEG = NT / RUN;
                for (int it = t; it < R * NSEG; it += NT) {
                    const int i = it % R, seg = it / R, yu = R * k + i - RAD;
                    if (yu >= 0 && yu < h) run_x<RAD>(sD + i * G::SST + seg * RUN, sX + i * G::XST + seg * RUN, tu);
                }
            }
            __syncthreads();   // DX rows complete
            // ---- per column: y pass of G_u, s_{k+1} = u + G_u * du, stored
#pragma unroll
            for (int i = 0; i < R; ++i) {
                const int y = R * k + i, yu = y - RAD, yo = yu - RAD;   // input, u/du, output rows
                if (yu >= 0) {
                    const float2 v = yu < h ? sX[i * G::XST + t] : last_dx;
                    if (yu < h) last_dx = v;
                    if (yu == 0) {
#pragma unroll
                        for (int j = 0; j < R; ++j) dxw[j] = v;
                    } else {
#pragma unroll
                        for (int j = 0; j < R - 1; ++j) dxw[j] = dxw[j + 1];
                        dxw[R - 1] = v;
                    }
                }
                if (yo >= 0 && yo < h) {
                    float2 acc = __fmul2_rn(tu[0], dxw[0]);
#pragma unroll
                    for (int j = 1; j < R; ++j) acc = ffma2(tu[j], dxw[j], acc);
                    const float2 uo = i >= RAD ? ucur[i - RAD] : uprev[i - RAD + R];
                    dst[(size_t)yo * NT + t] = __fadd2_rn(uo, acc);
                }
            }
#pragma unroll
            for (int i = 0; i < R; ++i) uprev[i] = ucur[i];
        }
        // SSD of the pair (one partial: the level runs with tiles = 1)
        for (int o = 16; o > 0; o >>= 1) ssd += __shfl_xor_sync(0xffffffffu, ssd, o);
        if (lane == 0) red[warp] = ssd;
        __syncthreads();
        if (t == 0) {
            float s = 0.0f;
            for (int j = 0; j < NT / 32; ++j) s += red[j];
            a.part[(size_t)pair * a.tiles] = s;
        }
    }
}

}  // namespace strip
