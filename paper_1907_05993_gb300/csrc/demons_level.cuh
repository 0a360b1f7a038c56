// Demons level resident in shared memory (included by demons.cu): for
// levels of at most 64 x 64 pixels one CTA owns a pair for the whole level,
// iterates Eq. 1 with the fields in shared memory, applies the stop rule of
// the control kernel itself and writes the level's final field, so the level
// costs one launch instead of two per iteration and the field never leaves
// the SM.  Each output pixel gets the same operations in the same order as in
// the tile kernels (x pass then y pass of each Gaussian with replicated
// borders, the force of Eq. 1 with the same warp cell and rounding steps), so
// the field is bit-identical to theirs; only the SSD is summed in another
// grouping (one partial per pair).
//
// Per pair: F (test image) and u_0 are loaded; iteration k computes
// u_k = G_f * s_k (k >= 1; u_0 as given), the force du and the SSD E_k, then
// the stop rule on E_k; a pair that continues (or reaches the cap) gets
// s_{k+1} = u_k + G_u * du.  The final field is u_n: u_k itself when the rule
// stops the pair at k, G_f * s_cap at the cap.  Pairs are taken from an
// atomic counter, so a pair with many iterations holds up no fixed share of
// the batch.
namespace lvl {

constexpr int NT = 512;
constexpr int MAXD = 64, MAXPX = MAXD * MAXD;
// A, B (float2, XOR-swizzled rows of 64), C (float2, rows of 64), F (float, rows of 64)
constexpr size_t BYTES = (size_t)3 * MAXPX * 8 + (size_t)MAXPX * 4;

struct LevelArgs {
    const float *Ftest;          // [B][h][w] test images of the level
    const float *Mref;           // [R][h][w] reference images of the level
    const int *ref_idx;          // [B]
    const float2 *u0;            // [B][h][w] the level's initial field
    float *uout;                 // final field: planar [B][2][h][w] (planar) or [B][h][w] float2
    double *hist;                // [B][hist_stride]
    int32_t *iters;              // [B][levels]
    int32_t *status;             // [B]
    int *work;                   // next pair to take (zero at launch)
    unsigned long long *px_count;   // tracing: pixel-iterations (NULL = off)
    int B, h, w, hist_stride, cap, window, level, levels, planar;
    float tol, alpha2;
    Taps taps;
};

// Index of (y, x) in a swizzled buffer: rows of 64, column x ^ (y mod 16), so that 16 lanes on 16
// consecutive rows of one column (x pass) and 16 lanes on consecutive columns of one row (y pass) hit
// distinct banks.
__device__ __forceinline__ int swz(int y, int x) { return (y << 6) + (x ^ (y & 15)); }

// x pass (RUN outputs along a row per work item, rows fastest) of the swizzled `in` into swizzled `out`.
template <int RAD>
__device__ __forceinline__ void xpass(const float2 *in, float2 *out, int h, int w, const float *t)
{
    const int nseg = (w + RUN - 1) / RUN;
    for (int j = threadIdx.x; j < h * nseg; j += NT) {
        const int seg = j / h, y = j - seg * h, x0 = seg * RUN;
        float2 win[RUN + 2 * RAD];
#pragma unroll
        for (int q = 0; q < RUN + 2 * RAD; ++q) win[q] = in[swz(y, clampi(x0 - RAD + q, 0, w - 1))];
        float2 acc[RUN];
#pragma unroll
        for (int o = 0; o < RUN; ++o) acc[o] = __fmul2_rn(make_float2(t[0], t[0]), win[o]);
#pragma unroll
        for (int k = 1; k <= 2 * RAD; ++k)
#pragma unroll
            for (int o = 0; o < RUN; ++o) acc[o] = ffma2(make_float2(t[k], t[k]), win[o + k], acc[o]);
#pragma unroll
        for (int o = 0; o < RUN; ++o)
            if (x0 + o < w) out[swz(y, x0 + o)] = acc[o];
    }
}

// y pass (RUN outputs down a column per work item, columns fastest) of the swizzled `in` into the plain
// `out` (rows of 64); with ADD, out = add + pass (the s update u + G_u * du), out swizzled.
template <int RAD, bool ADD>
__device__ __forceinline__ void ypass(const float2 *in, float2 *out, const float2 *add, int h, int w, const float *t)
{
    const int nseg = (h + RUN - 1) / RUN;
    for (int j = threadIdx.x; j < w * nseg; j += NT) {
        const int seg = j / w, x = j - seg * w, y0 = seg * RUN;
        float2 win[RUN + 2 * RAD];
#pragma unroll
        for (int q = 0; q < RUN + 2 * RAD; ++q) win[q] = in[swz(clampi(y0 - RAD + q, 0, h - 1), x)];
        float2 acc[RUN];
#pragma unroll
        for (int o = 0; o < RUN; ++o) acc[o] = __fmul2_rn(make_float2(t[0], t[0]), win[o]);
#pragma unroll
        for (int k = 1; k <= 2 * RAD; ++k)
#pragma unroll
            for (int o = 0; o < RUN; ++o) acc[o] = ffma2(make_float2(t[k], t[k]), win[o + k], acc[o]);
#pragma unroll
        for (int o = 0; o < RUN; ++o) {
            const int y = y0 + o;
            if (y < h) {
                if (ADD) out[swz(y, x)] = __fadd2_rn(add[(y << 6) + x], acc[o]);
                else out[(y << 6) + x] = acc[o];
            }
        }
    }
}

template <int RAD>
__global__ void __launch_bounds__(NT, 2) demons_level_kernel(LevelArgs a)
{
    extern __shared__ __align__(16) unsigned char lvl_smem[];
    float2 *A = reinterpret_cast<float2 *>(lvl_smem);   // s_k, then du (swizzled)
    float2 *Bx = A + MAXPX;                              // x-pass results (swizzled)
    float2 *C = Bx + MAXPX;                              // u_k (rows of 64)
    float *F = reinterpret_cast<float *>(C + MAXPX);     // test image (rows of 64)
    __shared__ float red[NT / 32];
    __shared__ int s_pair, s_next;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int h = a.h, w = a.w, n = h * w;
    const float al2 = a.alpha2;
    enum { CONTINUE = 0, STOP = 1, CAPPED = 2 };
    for (;;) {
        if (t == 0) s_pair = atomicAdd(a.work, 1);
        __syncthreads();
        const int pair = s_pair;
        if (pair >= a.B) break;
        const float *Fg = a.Ftest + (size_t)pair * n;
        const float2 *ug = a.u0 + (size_t)pair * n;
        const float *M = a.Mref + (size_t)__ldg(a.ref_idx + pair) * n;
        for (int p = t; p < n; p += NT) {
            const int y = p / w, x = p - y * w;
            F[(y << 6) + x] = Fg[p];
            C[(y << 6) + x] = ug[p];   // u_0
        }
        __syncthreads();
        for (int k = 0;; ++k) {
            if (k > 0) {   // u_k = G_f * s_k
                xpass<RAD>(A, Bx, h, w, a.taps.f);
                __syncthreads();
                ypass<RAD, false>(Bx, C, nullptr, h, w, a.taps.f);
                __syncthreads();
            }
            // the force of Eq. 1 at every pixel (rows outside clamp; one-sided differences at the
            // edges), du into A, and this thread's share of E_k
            float ssd = 0.0f;
            constexpr int GB = 4;   // pixels whose moving-image gathers are in flight together
            for (int p0 = t; p0 < n; p0 += GB * NT) {
                float mA[GB], mB[GB], mC[GB], mD[GB], fxv[GB], fyv[GB];
#pragma unroll
                for (int i = 0; i < GB; ++i) {
                    const int p = min(p0 + i * NT, n - 1);   // past the end: any pixel, result unused
                    const int y = p / w, x = p - y * w;
                    const float2 u = C[(y << 6) + x];
                    int x0, y0;
                    warp_cell(x, u.x, w, x0, fxv[i]);
                    warp_cell(y, u.y, h, y0, fyv[i]);
                    const float *q = M + y0 * w + x0;
                    mA[i] = __ldg(q);
                    mB[i] = __ldg(q + 1);
                    mC[i] = __ldg(q + w);
                    mD[i] = __ldg(q + w + 1);
                }
#pragma unroll
                for (int i = 0; i < GB; ++i) {
                    const int p = p0 + i * NT;
                    if (p >= n) break;
                    const int y = p / w, x = p - y * w;
                    const float *fr_ = F + (y << 6);
                    const float fc = fr_[x], fl = fr_[max(x - 1, 0)], frt = fr_[min(x + 1, w - 1)];
                    const float fup = F[(max(y - 1, 0) << 6) + x], fdn = F[(min(y + 1, h - 1) << 6) + x];
                    const float sx = (x == 0 || x == w - 1) ? 1.0f : 0.5f, sy = (y == 0 || y == h - 1) ? 1.0f : 0.5f;
                    const float fx = fxv[i], fy = fyv[i];
                    const float omx = fmaf(fx, -1.0f, 1.0f), omy = fmaf(fy, -1.0f, 1.0f);
                    const float top = fmaf(fx, mB[i], omx * mA[i]), bot = fmaf(fx, mD[i], omx * mC[i]);
                    const float mw = fmaf(fy, bot, omy * top);
                    const float gx = sx * fmaf(fl, -1.0f, frt), gy = sy * fmaf(fup, -1.0f, fdn);
                    const float d = fmaf(fc, -1.0f, mw);
                    const float den = fmaf(gx, gx, fmaf(gy, gy, (al2 * d) * d));
                    const float tt = den > 1e-9f ? __fdividef(d, den) : 0.0f;
                    A[swz(y, x)] = make_float2(tt * gx, tt * gy);
                    ssd = fmaf(d, d, ssd);
                }
            }
            for (int o = 16; o > 0; o >>= 1) ssd += __shfl_xor_sync(0xffffffffu, ssd, o);
            if (lane == 0) red[warp] = ssd;
            __syncthreads();
            if (t == 0) {   // the control kernel's stop rule after iteration k, on E_k in FP64
                float s = 0.0f;
                for (int j = 0; j < NT / 32; ++j) s += red[j];
                const double E = 0.0 + (double)s;
                double *hh = a.hist + (size_t)pair * a.hist_stride;
                hh[k] = E;
                int32_t *itp = a.iters + (size_t)pair * a.levels + a.level;
                int next = CONTINUE;
                if (!isfinite(E)) {
                    *itp = k;
                    a.status[pair] |= HREBSD_PAIR_NONFINITE;
                    next = STOP;
                } else if (a.window > 0 && k >= a.window && (hh[k - a.window] - E) < (double)a.tol * hh[k - a.window]) {
                    *itp = k;
                    next = STOP;
                } else if (k + 1 >= a.cap) {
                    *itp = a.cap;
                    a.status[pair] |= HREBSD_PAIR_CAPPED;
                    next = CAPPED;
                }
                if (a.px_count) atomicAdd(a.px_count, (unsigned long long)n);
                s_next = next;
            }
            __syncthreads();
            const int next = s_next;
            if (next == STOP) break;   // the final field is u_k, in C
            // s_{k+1} = u_k + G_u * du
            xpass<RAD>(A, Bx, h, w, a.taps.up);
            __syncthreads();
            ypass<RAD, true>(Bx, A, C, h, w, a.taps.up);
            __syncthreads();
            if (next == CAPPED) {   // the final field is u_cap = G_f * s_cap
                xpass<RAD>(A, Bx, h, w, a.taps.f);
                __syncthreads();
                ypass<RAD, false>(Bx, C, nullptr, h, w, a.taps.f);
                __syncthreads();
                break;
            }
        }
        for (int p = t; p < n; p += NT) {
            const int y = p / w, x = p - y * w;
            const float2 v = C[(y << 6) + x];
            if (a.planar) {
                a.uout[(size_t)pair * 2 * n + p] = v.x;
                a.uout[(size_t)pair * 2 * n + n + p] = v.y;
            } else {
                reinterpret_cast<float2 *>(a.uout)[(size_t)pair * n + p] = v;
            }
        }
        __syncthreads();   // C and F are read before the next pair overwrites them
    }
}

}  // namespace lvl
