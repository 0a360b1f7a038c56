// a2-a4, a9: batched multi-resolution demons registration (Section 1, Eq. 1).
//
// Data layout (HBM): every buffer is pair-major, [B][h][w] for images and
// [B][2][h][w] for fields (x plane, then y plane), so that a tile of one pair
// is a set of contiguous row segments.  The reference pyramid ([R][h][w],
// R <= a few grains) is small and stays in L2; the per-pair test pyramid and
// the field buffers stream from HBM.
//
// One demons iteration u_{k+1} = G_f * (u_k + G_u * du(u_k)) is ONE fused
// kernel launch over every (active pair, tile).  The launch stores the
// unsmoothed field s_{k+1} = u_k + G_u * du(u_k) instead of u_{k+1}; the next
// launch recomputes u_{k+1} = G_f * s_{k+1} on the fly from a tile with a
// 2r halo (r the Gaussian radius).  This keeps the expensive part (warp +
// force) on a halo of r instead of 2r and costs one smoothing pass that would
// otherwise be a separate read+write of the field.  Per pixel-iteration the
// kernel reads the test image (4 B) and s (8 B) and writes s (8 B); the
// bilinear gathers of the moving image hit the L2-resident reference pyramid.
//
// Border handling: every Gaussian pass has replicated borders.  Tiles load s
// with clamped addresses (so out-of-image halo values are the replicated
// ones) and evaluate the force at the clamped position of every halo point;
// with that, every value the passes read at an in-image position is exact, and
// out-of-image values are never consumed.
//
// Uneven work (a9): pairs stop independently (stop rule on the SSD history).
// A small control kernel after each iteration compacts the list of active
// pairs; the iteration kernel is persistent (grid = SMs x resident CTAs) and
// walks the (active pair, tile) work list, so stopped pairs cost nothing.
#include <math.h>
#include <string.h>

#include "internal.cuh"

int hr_launch_reduce2(hrebsd_ctx *ctx, const float *in, float *out, int n, int H, int W, cudaStream_t st);

namespace {

constexpr int TX = 32;
constexpr int TY = 32;
constexpr int kIterThreads = 256;
constexpr int kMaxRad = 6;

struct Taps {
    float up[2 * kMaxRad + 1];   // G_u (update smoothing), centred at index RAD
    float f[2 * kMaxRad + 1];    // G_f (field smoothing)
};

struct IterArgs {
    const float *Ftest;      // test level images [B][h][w]
    const float *Mref;       // reference level images [R][h][w]
    const int *ref_idx;      // [B]
    const float *in;         // k == 0: u_0 [B][2][h][w]; k > 0: s_k
    float *out;              // s_{k+1}
    float *part;             // SSD partials [B][tiles]
    const int *active;       // active pair list
    const int *n_active;     // its length
    int *n_next_reset;       // counter of the next list, zeroed by this launch
    unsigned long long *px_count;   // tracing: pixel-iterations (NULL = off)
    int h, w, tiles_x, tiles;
    int in_is_s;
    float alpha2;
    Taps taps;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Bilinear sample of M at index coordinates (x, y), clamped to the image.
__device__ __forceinline__ float bilinear_clamped(const float *__restrict__ M, int h, int w, float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    int x0 = min((int)floorf(x), w - 2);
    int y0 = min((int)floorf(y), h - 2);
    float fx = x - (float)x0, fy = y - (float)y0;
    const float *p = M + (size_t)y0 * w + x0;
    float a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + w), d = __ldg(p + w + 1);
    // (1 - f) a + f b: exact at both nodes (f = 0 and f = 1)
    float top = fmaf(fx, b, (1.0f - fx) * a);
    float bot = fmaf(fx, d, (1.0f - fx) * c);
    return fmaf(fy, bot, (1.0f - fy) * top);
}

template <int RAD>
struct IterSmem {
    static constexpr int AW = TX + 4 * RAD, AH = TY + 4 * RAD;   // s tile (T + 2r halo)
    static constexpr int BW = TX + 2 * RAD, BH = TY + 2 * RAD;   // u, du (T + r halo)
    static constexpr int FW = BW + 2, FH = BH + 2;               // test image (T + r + 1)
    static constexpr int A_ELEMS = 2 * (AW * AH > BW * BH ? AW * AH : BW * BH);
    static constexpr int X_ELEMS = 2 * (AH * BW > BH * TX ? AH * BW : BH * TX);
    static constexpr int U_ELEMS = 2 * BW * BH;
    static constexpr int F_ELEMS = FW * FH;
    static constexpr int TOTAL = A_ELEMS + X_ELEMS + U_ELEMS + F_ELEMS;
};

template <int RAD>
__global__ void __launch_bounds__(kIterThreads) demons_iter_kernel(IterArgs a)
{
    using L = IterSmem<RAD>;
    extern __shared__ float sm[];
    float *bufA = sm;                        // s tile, later du
    float *bufX = bufA + L::A_ELEMS;         // x-pass results
    float *bufU = bufX + L::X_ELEMS;         // u on T + r
    float *bufF = bufU + L::U_ELEMS;         // test image on T + r + 1
    __shared__ float red[kIterThreads / 32];

    const int tid = threadIdx.x;
    const int n_active = *a.n_active;
    if (blockIdx.x == 0 && tid == 0) {
        *a.n_next_reset = 0;
        if (a.px_count) atomicAdd(a.px_count, (unsigned long long)n_active * a.h * a.w);
    }
    const long long work = (long long)n_active * a.tiles;
    const int h = a.h, w = a.w;
    const size_t plane = (size_t)h * w;

    for (long long item = blockIdx.x; item < work; item += gridDim.x) {
        const int pair = a.active[item / a.tiles];
        const int tile = (int)(item % a.tiles);
        const int x0 = (tile % a.tiles_x) * TX, y0 = (tile / a.tiles_x) * TY;
        const float *Fimg = a.Ftest + (size_t)pair * plane;
        const float *M = a.Mref + (size_t)__ldg(a.ref_idx + pair) * plane;
        const float *src = a.in + (size_t)pair * 2 * plane;

        // ---- test image on T + r + 1 (clamped addresses)
        for (int idx = tid; idx < L::FW * L::FH; idx += kIterThreads) {
            int ly = idx / L::FW, lx = idx - ly * L::FW;
            int gy = clampi(y0 - RAD - 1 + ly, 0, h - 1), gx = clampi(x0 - RAD - 1 + lx, 0, w - 1);
            bufF[idx] = __ldg(Fimg + (size_t)gy * w + gx);
        }
        if (a.in_is_s && RAD > 0) {
            // ---- s on T + 2r, then u = G_f * s on T + r (x pass, y pass)
            for (int idx = tid; idx < L::AW * L::AH; idx += kIterThreads) {
                int ly = idx / L::AW, lx = idx - ly * L::AW;
                int gy = clampi(y0 - 2 * RAD + ly, 0, h - 1), gx = clampi(x0 - 2 * RAD + lx, 0, w - 1);
                size_t g = (size_t)gy * w + gx;
                bufA[idx] = __ldg(src + g);
                bufA[L::AW * L::AH + idx] = __ldg(src + plane + g);
            }
            __syncthreads();
            for (int idx = tid; idx < L::AH * L::BW; idx += kIterThreads) {
                int ly = idx / L::BW, lx = idx - ly * L::BW;
                const float *r0 = bufA + ly * L::AW + lx;
                const float *r1 = r0 + L::AW * L::AH;
                float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                for (int k = 0; k <= 2 * RAD; ++k) {
                    s0 = fmaf(a.taps.f[k], r0[k], s0);
                    s1 = fmaf(a.taps.f[k], r1[k], s1);
                }
                bufX[idx] = s0;
                bufX[L::AH * L::BW + idx] = s1;
            }
            __syncthreads();
            for (int idx = tid; idx < L::BH * L::BW; idx += kIterThreads) {
                int ly = idx / L::BW, lx = idx - ly * L::BW;
                const float *c0 = bufX + ly * L::BW + lx;
                const float *c1 = c0 + L::AH * L::BW;
                float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
                for (int k = 0; k <= 2 * RAD; ++k) {
                    s0 = fmaf(a.taps.f[k], c0[k * L::BW], s0);
                    s1 = fmaf(a.taps.f[k], c1[k * L::BW], s1);
                }
                bufU[idx] = s0;
                bufU[L::BW * L::BH + idx] = s1;
            }
        } else {
            // ---- u itself on T + r (first iteration of a level, or no field smoothing)
            for (int idx = tid; idx < L::BW * L::BH; idx += kIterThreads) {
                int ly = idx / L::BW, lx = idx - ly * L::BW;
                int gy = clampi(y0 - RAD + ly, 0, h - 1), gx = clampi(x0 - RAD + lx, 0, w - 1);
                size_t g = (size_t)gy * w + gx;
                bufU[idx] = __ldg(src + g);
                bufU[L::BW * L::BH + idx] = __ldg(src + plane + g);
            }
        }
        __syncthreads();

        // ---- warp + force at the clamped position of every point of T + r
        float ssd = 0.0f;
        float *du0 = bufA, *du1 = bufA + L::BW * L::BH;
        for (int idx = tid; idx < L::BW * L::BH; idx += kIterThreads) {
            int ly = idx / L::BW, lx = idx - ly * L::BW;
            int vy = y0 - RAD + ly, vx = x0 - RAD + lx;
            int qy = clampi(vy, 0, h - 1), qx = clampi(vx, 0, w - 1);
            int qly = qy - (y0 - RAD), qlx = qx - (x0 - RAD);   // local (B) coordinates of q
            float ux = bufU[qly * L::BW + qlx], uy = bufU[L::BW * L::BH + qly * L::BW + qlx];
            const float *fc = bufF + (qly + 1) * L::FW + (qlx + 1);
            int xl = max(qx - 1, 0) - qx, xr = min(qx + 1, w - 1) - qx;
            int yl = max(qy - 1, 0) - qy, yr = min(qy + 1, h - 1) - qy;
            float gx = (fc[xr] - fc[xl]) * ((xr - xl) == 2 ? 0.5f : 1.0f);
            float gy = (fc[yr * L::FW] - fc[yl * L::FW]) * ((yr - yl) == 2 ? 0.5f : 1.0f);
            float mw = bilinear_clamped(M, h, w, (float)qx - ux, (float)qy - uy);
            float d = mw - fc[0];
            float den = fmaf(gx, gx, fmaf(gy, gy, a.alpha2 * d * d));
            float dx = 0.0f, dy = 0.0f;
            if (den > 1e-9f) {
                float t = d / den;
                dx = t * gx;
                dy = t * gy;
            }
            du0[idx] = dx;
            du1[idx] = dy;
            if (vy == qy && vx == qx && ly >= RAD && ly < RAD + TY && lx >= RAD && lx < RAD + TX)
                ssd = fmaf(d, d, ssd);
        }
        __syncthreads();
        // ---- G_u * du: x pass on rows of T + r, columns of T
        for (int idx = tid; idx < L::BH * TX; idx += kIterThreads) {
            int ly = idx / TX, lx = idx - ly * TX;
            const float *r0 = du0 + ly * L::BW + lx;
            const float *r1 = du1 + ly * L::BW + lx;
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int k = 0; k <= 2 * RAD; ++k) {
                s0 = fmaf(a.taps.up[k], r0[k], s0);
                s1 = fmaf(a.taps.up[k], r1[k], s1);
            }
            bufX[idx] = s0;
            bufX[L::BH * TX + idx] = s1;
        }
        __syncthreads();
        // ---- y pass, s_{k+1} = u_k + G_u * du on T
        float *dst = a.out + (size_t)pair * 2 * plane;
        for (int idx = tid; idx < TY * TX; idx += kIterThreads) {
            int ly = idx / TX, lx = idx - ly * TX;
            int gy = y0 + ly, gx = x0 + lx;
            if (gy >= h || gx >= w) continue;
            const float *c0 = bufX + ly * TX + lx;
            const float *c1 = c0 + L::BH * TX;
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int k = 0; k <= 2 * RAD; ++k) {
                s0 = fmaf(a.taps.up[k], c0[k * TX], s0);
                s1 = fmaf(a.taps.up[k], c1[k * TX], s1);
            }
            int u_idx = (ly + RAD) * L::BW + lx + RAD;
            size_t g = (size_t)gy * w + gx;
            dst[g] = bufU[u_idx] + s0;
            dst[plane + g] = bufU[L::BW * L::BH + u_idx] + s1;
        }
        // ---- SSD partial of this tile
        for (int o = 16; o > 0; o >>= 1) ssd += __shfl_xor_sync(0xffffffffu, ssd, o);
        if ((tid & 31) == 0) red[tid >> 5] = ssd;
        __syncthreads();
        if (tid == 0) {
            float t = 0.0f;
            for (int i = 0; i < kIterThreads / 32; ++i) t += red[i];
            a.part[(size_t)pair * a.tiles + tile] = t;
        }
        __syncthreads();
    }
}

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
template <int RAD>
__global__ void __launch_bounds__(256) demons_finalize_kernel(const float *u0, const float *s0, const float *s1,
                                                              const int32_t *iters, int levels, int level,
                                                              float *uout, int B, int h, int w, int tiles_x,
                                                              int tiles, Taps taps)
{
    constexpr int AW = TX + 2 * RAD, AH = TY + 2 * RAD;
    __shared__ float sa[2 * AW * AH];
    __shared__ float sx[2 * AH * TX];
    const size_t plane = (size_t)h * w;
    for (long long item = blockIdx.x; item < (long long)B * tiles; item += gridDim.x) {
        const int pair = (int)(item / tiles), tile = (int)(item % tiles);
        const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;
        const int n = iters[(size_t)pair * levels + level];
        const float *src = (n == 0 ? u0 : ((n & 1) ? s1 : s0)) + (size_t)pair * 2 * plane;
        float *dst = uout + (size_t)pair * 2 * plane;
        if (n == 0 || RAD == 0) {
            for (int idx = threadIdx.x; idx < TX * TY; idx += blockDim.x) {
                int gy = y0 + idx / TX, gx = x0 + idx % TX;
                if (gy < h && gx < w) {
                    size_t g = (size_t)gy * w + gx;
                    dst[g] = src[g];
                    dst[plane + g] = src[plane + g];
                }
            }
            continue;
        }
        for (int idx = threadIdx.x; idx < AW * AH; idx += blockDim.x) {
            int ly = idx / AW, lx = idx - ly * AW;
            int gy = clampi(y0 - RAD + ly, 0, h - 1), gx = clampi(x0 - RAD + lx, 0, w - 1);
            size_t g = (size_t)gy * w + gx;
            sa[idx] = src[g];
            sa[AW * AH + idx] = src[plane + g];
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < AH * TX; idx += blockDim.x) {
            int ly = idx / TX, lx = idx - ly * TX;
            float a0 = 0.0f, a1 = 0.0f;
            for (int k = 0; k <= 2 * RAD; ++k) {
                a0 = fmaf(taps.f[k], sa[ly * AW + lx + k], a0);
                a1 = fmaf(taps.f[k], sa[AW * AH + ly * AW + lx + k], a1);
            }
            sx[idx] = a0;
            sx[AH * TX + idx] = a1;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < TX * TY; idx += blockDim.x) {
            int ly = idx / TX, lx = idx - ly * TX;
            int gy = y0 + ly, gx = x0 + lx;
            if (gy >= h || gx >= w) continue;
            float a0 = 0.0f, a1 = 0.0f;
            for (int k = 0; k <= 2 * RAD; ++k) {
                a0 = fmaf(taps.f[k], sx[(ly + k) * TX + lx], a0);
                a1 = fmaf(taps.f[k], sx[AH * TX + (ly + k) * TX + lx], a1);
            }
            size_t g = (size_t)gy * w + gx;
            dst[g] = a0;
            dst[plane + g] = a1;
        }
        __syncthreads();
    }
}

// Prolongation (Section 1): fine(x_f) = 2 * bilinear(coarse, (x_f + 0.5)/2 - 0.5).
__global__ void prolong_kernel(const float *__restrict__ uc, float *__restrict__ uf, int B, int h, int w)
{
    const int H = 2 * h, W = 2 * w;
    const size_t total = (size_t)B * 2 * H * W;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        size_t pl = idx / ((size_t)H * W);   // pair * 2 + component
        int rem = (int)(idx - pl * H * W);
        int i = rem / W, j = rem - i * W;
        const float *c = uc + pl * h * w;
        float x = ((float)j + 0.5f) * 0.5f - 0.5f, y = ((float)i + 0.5f) * 0.5f - 0.5f;
        uf[idx] = 2.0f * bilinear_clamped(c, h, w, x, y);
    }
}

__global__ void iota_kernel(int *a, int n, int *count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = n;
}

template <int RAD>
int launch_iter(hrebsd_ctx *ctx, const IterArgs &a, int max_items, cudaStream_t st)
{
    constexpr size_t smem = IterSmem<RAD>::TOTAL * sizeof(float);
    static int configured_dev = -1;
    static int occ = 0;
    if (configured_dev != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(demons_iter_kernel<RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        HR_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, demons_iter_kernel<RAD>, kIterThreads, smem));
        if (occ < 1) occ = 1;
        configured_dev = ctx->device;
    }
    int grid = ctx->num_sms * occ;
    if (grid > max_items) grid = max_items;
    if (grid < 1) grid = 1;
    hr_prof_begin(ctx, st);
    demons_iter_kernel<RAD><<<grid, kIterThreads, smem, st>>>(a);
    hr_prof_end(ctx, PROF_ITER, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
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

int dispatch_finalize(hrebsd_ctx *ctx, int rad, const float *u0, const float *s0, const float *s1,
                      const int32_t *iters, int levels, int level, float *uout, int B, int h, int w, int tiles_x,
                      int tiles, const Taps &taps, cudaStream_t st)
{
    long long items = (long long)B * tiles;
    int grid = (int)(items < ctx->num_sms * 8LL ? items : ctx->num_sms * 8LL);
    hr_prof_begin(ctx, st);
#define HR_FIN(R) demons_finalize_kernel<R><<<grid, 256, 0, st>>>(u0, s0, s1, iters, levels, level, uout, B, h, w, tiles_x, tiles, taps)
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

enum { WS_TPYR = 0, WS_RPYR, WS_U0, WS_S0, WS_S1, WS_UOUT, WS_PART, WS_HIST, WS_LIST };

// Register B pairs (all buffers already offset to this chunk).
int register_chunk(hrebsd_ctx *ctx, const float *ref, const float *test, const int32_t *ref_idx, int R, int B,
                   int H, int W, const hrebsd_demons_params *p, const float *init_field, float *field,
                   int32_t *iters, int32_t *status, cudaStream_t st)
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
    if ((e = hr_ws(ctx, WS_TPYR, pyr_px * 4 + 16, &tpyr))) return e;
    if ((e = hr_ws(ctx, WS_RPYR, rpyr_px * 4 + 16, &rpyr))) return e;
    if ((e = hr_ws(ctx, WS_U0, field_elems * 4, &u0))) return e;
    if ((e = hr_ws(ctx, WS_S0, field_elems * 4, &s0))) return e;
    if ((e = hr_ws(ctx, WS_S1, field_elems * 4, &s1))) return e;
    if ((e = hr_ws(ctx, WS_UOUT, (L > 1 ? field_elems / 4 : 1) * 4, &uout))) return e;
    if ((e = hr_ws(ctx, WS_PART, (size_t)B * tiles0 * 4, &part))) return e;
    if ((e = hr_ws(ctx, WS_HIST, (size_t)B * (cap_max + 1) * 8, &hist))) return e;
    if ((e = hr_ws(ctx, WS_LIST, ((size_t)2 * B + 64) * 4, &lists))) return e;
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
        size_t n0 = (size_t)B * 2 * (H >> start) * (W >> start) * 4;
        if (init_field) HR_CHECK(cudaMemcpyAsync(u0, init_field, n0, cudaMemcpyDeviceToDevice, st));
        else HR_CHECK(cudaMemsetAsync(u0, 0, n0, st));
    }

    for (int l = start; l >= 0; --l) {
        const int h = H >> l, w = W >> l;
        const int tiles_x = (w + TX - 1) / TX, tiles = tiles_x * ((h + TY - 1) / TY);
        const int cap = p->max_iters[l];
        hr_prof_begin(ctx, st);
        iota_kernel<<<(B + 255) / 256, 256, 0, st>>>(list0, B, cnt);
        hr_prof_end(ctx, PROF_DEMONS_AUX, st);
        HR_LAUNCHED(ctx);
        for (int k = 0; k < cap; ++k) {
            int *cur = (k & 1) ? list1 : list0, *nxt = (k & 1) ? list0 : list1;
            IterArgs a;
            a.Ftest = tl[l];
            a.Mref = rl[l];
            a.ref_idx = ref_idx;
            a.in = k == 0 ? (const float *)u0 : ((k & 1) ? (const float *)s1 : (const float *)s0);
            a.out = ((k + 1) & 1) ? (float *)s1 : (float *)s0;
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
            if ((e = dispatch_iter(ctx, rad, a, B * tiles, st))) return e;
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
        float *dst = l == 0 ? field : (float *)uout;
        if ((e = dispatch_finalize(ctx, rad, (const float *)u0, (const float *)s0, (const float *)s1, iters, L, l,
                                   dst, B, h, w, tiles_x, tiles, taps, st)))
            return e;
        if (l > 0) {
            size_t total = (size_t)B * 2 * (2 * h) * (2 * w);
            int grid = (int)((total + 255) / 256);
            if (grid > ctx->num_sms * 16) grid = ctx->num_sms * 16;
            hr_prof_begin(ctx, st);
            prolong_kernel<<<grid, 256, 0, st>>>((const float *)uout, (float *)u0, B, h, w);
            hr_prof_end(ctx, PROF_DEMONS_AUX, st);
            HR_LAUNCHED(ctx);
        }
    }
    return HREBSD_OK;
}

}  // namespace

extern "C" int hrebsd_demons_register_batch(hrebsd_ctx *ctx, const float *ref, const float *test,
                                            const int32_t *ref_idx, int R, int B, int H, int W,
                                            const hrebsd_demons_params *p, const float *init_field, float *field,
                                            int32_t *iters, int32_t *pair_status, void *stream)
{
    if (!ctx || !p || B < 0 || R < 1) return HREBSD_EINVAL;
    if (p->levels < 1 || p->levels > 8) return HREBSD_EINVAL;
    const int L = p->levels;
    if (H % (1 << (L - 1)) || W % (1 << (L - 1))) return HREBSD_EINVAL;
    if ((H >> (L - 1)) < 8 || (W >> (L - 1)) < 8) return HREBSD_EINVAL;
    for (int l = 0; l < L; ++l)
        if (p->max_iters[l] < 0 || p->max_iters[l] > 4096) return HREBSD_EINVAL;
    if (!(p->alpha >= 0.0f) || p->stop_window < 0) return HREBSD_EINVAL;
    if (hr_gauss_radius(p->sigma_update) > kMaxRad || hr_gauss_radius(p->sigma_field) > kMaxRad) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!ref || !test || !ref_idx || !field || !iters || !pair_status) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
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
