// a7: second-pass ROI cross-correlation (Section 2).
//
// One CTA owns one (pair, ROI).  The two real ROIs (test t, remapped
// reference r) are zero-meaned, Hann-windowed and packed into one complex
// array z = t + i r in shared memory, so that a single complex 2-D FFT gives
// both spectra: T(k) = (Z(k) + conj Z(-k))/2, R(k) = (Z(k) - conj Z(-k))/2i.
// The cross-power T conj(R) is Hermitian; its inverse FFT is the real
// correlation c(s) = sum_x t(x+s) r(x).  The FFTs are radix-2 decimation in
// time over the shared-memory array (a 2-D bit-reversal, then row stages,
// then column stages), with a twiddle table per CTA.  The peak search is a
// CTA reduction of (value, first index) pairs by warp shuffles that also
// keeps the runner-up for the near-tie flag.
#include <math.h>

#include "internal.cuh"

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

template <int S>
__device__ __forceinline__ int bitrev(int v)
{
    constexpr int LOG = S == 16 ? 4 : S == 32 ? 5 : S == 64 ? 6 : 7;
    return (int)(__brev((unsigned)v) >> (32 - LOG));
}

// In-place 2-D FFT of z [S][S] (row-major, row stride S).  sign = -1 forward,
// +1 inverse (unscaled).  tw[j] = exp(-2 pi i j / S), j < S/2.
template <int S, int NT>
__device__ void fft2d(float2 *z, const float2 *tw, int sign)
{
    // 2-D bit-reversal permutation
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const int y = idx / S, x = idx % S;
        const int j = bitrev<S>(y) * S + bitrev<S>(x);
        if (idx < j) {
            float2 t = z[idx];
            z[idx] = z[j];
            z[j] = t;
        }
    }
    __syncthreads();
    // rows, then columns
    for (int dim = 0; dim < 2; ++dim) {
        const int es = dim == 0 ? 1 : S;        // element stride within one transform
        const int ls = dim == 0 ? S : 1;        // stride between transforms
        for (int half = 1; half < S; half <<= 1) {
            const int tstep = S / (2 * half);
            for (int b = threadIdx.x; b < S * S / 2; b += NT) {
                const int line = b / (S / 2), bf = b % (S / 2);
                const int grp = bf / half, j = bf % half;
                const int i0 = grp * 2 * half + j, i1 = i0 + half;
                float2 w = tw[j * tstep];
                if (sign > 0) w.y = -w.y;
                float2 *p0 = z + line * ls + i0 * es;
                float2 *p1 = z + line * ls + i1 * es;
                const float2 v = cmul(*p1, w), u = *p0;
                *p0 = make_float2(u.x + v.x, u.y + v.y);
                *p1 = make_float2(u.x - v.x, u.y - v.y);
            }
            __syncthreads();
        }
    }
}

template <int NT>
__device__ float block_sum(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    for (int i = 0; i < NT / 32; ++i) t += red[i];
    __syncthreads();
    return t;
}

// (value, index) ordering: larger value first, then smaller index.
__device__ __forceinline__ bool better(float v, int i, float bv, int bi) { return v > bv || (v == bv && i < bi); }

template <int S, int NT>
__global__ void __launch_bounds__(NT) xcf_kernel(const float *__restrict__ rem, const float *__restrict__ test, int B,
                                                 int H, int W, const int32_t *__restrict__ roi, int N, int window,
                                                 float *q, int32_t *peak, float *ph, int32_t *near_tie)
{
    extern __shared__ float2 z[];                 // [S][S]
    __shared__ float2 tw[S / 2];
    __shared__ float win[S];
    __shared__ float red[NT / 32];
    __shared__ float rv[NT / 32], rv2[NT / 32];
    __shared__ int ri[NT / 32];

    const int b = blockIdx.x / N, r = blockIdx.x % N;
    const int cx = roi[2 * r], cy = roi[2 * r + 1];
    const int x0 = cx - S / 2, y0 = cy - S / 2;
    const size_t o = (size_t)blockIdx.x;
    if (x0 < 0 || y0 < 0 || x0 + S > W || y0 + S > H) {   // ROI outside the image
        if (threadIdx.x == 0) {
            q[2 * o] = q[2 * o + 1] = __int_as_float(0x7fc00000);
            peak[2 * o] = peak[2 * o + 1] = 0;
            ph[o] = 0.0f;
            if (near_tie) near_tie[o] = 0;
        }
        return;
    }
    for (int j = threadIdx.x; j < S / 2; j += NT) {
        float s, c;
        sincospif(-2.0f * (float)j / (float)S, &s, &c);
        tw[j] = make_float2(c, s);
    }
    for (int n = threadIdx.x; n < S; n += NT)
        win[n] = window ? 0.5f * (1.0f - cospif(2.0f * (float)n / (float)(S - 1))) : 1.0f;

    const float *T = test + (size_t)b * H * W + (size_t)y0 * W + x0;
    const float *Rr = rem + (size_t)b * H * W + (size_t)y0 * W + x0;
    float st = 0.0f, sr = 0.0f;
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const int y = idx / S, x = idx % S;
        const float tv = __ldg(T + (size_t)y * W + x), rv_ = __ldg(Rr + (size_t)y * W + x);
        z[idx] = make_float2(tv, rv_);
        st += tv;
        sr += rv_;
    }
    const float mt = block_sum<NT>(st, red) * (1.0f / (S * S));
    const float mr = block_sum<NT>(sr, red) * (1.0f / (S * S));
    float nt = 0.0f, nr = 0.0f;
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const int y = idx / S, x = idx % S;
        const float wgt = win[y] * win[x];
        float2 v = z[idx];
        v.x = (v.x - mt) * wgt;
        v.y = (v.y - mr) * wgt;
        z[idx] = v;
        nt = fmaf(v.x, v.x, nt);
        nr = fmaf(v.y, v.y, nr);
    }
    nt = sqrtf(block_sum<NT>(nt, red));
    nr = sqrtf(block_sum<NT>(nr, red));   // (block_sum ends with a barrier: z is complete)

    fft2d<S, NT>(z, tw, -1);

    // cross-power P(k) = T(k) conj(R(k)), P(-k) = conj(P(k)); pairs (k, -k) in place
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const int ky = idx / S, kx = idx % S;
        const int m = ((S - ky) & (S - 1)) * S + ((S - kx) & (S - 1));
        if (idx > m) continue;
        const float2 zk = z[idx], zm = z[m];
        const float2 Tk = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 Rk = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        const float2 P = make_float2(Tk.x * Rk.x + Tk.y * Rk.y, Tk.y * Rk.x - Tk.x * Rk.y);
        z[idx] = P;
        if (m != idx) z[m] = make_float2(P.x, -P.y);
    }
    __syncthreads();
    fft2d<S, NT>(z, tw, +1);

    // argmax of c = Re(z) / S^2 (first maximum in row-major order) and runner-up
    const float scale = 1.0f / (float)(S * S);
    float bv = -INFINITY, bv2 = -INFINITY;
    int bi = 0x7fffffff;
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const float v = z[idx].x * scale;
        if (better(v, idx, bv, bi)) {
            bv2 = bv;
            bv = v;
            bi = idx;
        } else if (v > bv2) {
            bv2 = v;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const float ov2 = __shfl_xor_sync(0xffffffffu, bv2, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (better(ov, oi, bv, bi)) {
            bv2 = fmaxf(bv, ov2);
            bv = ov;
            bi = oi;
        } else {
            bv2 = fmaxf(bv2, ov);
        }
    }
    if ((threadIdx.x & 31) == 0) {
        rv[threadIdx.x >> 5] = bv;
        rv2[threadIdx.x >> 5] = bv2;
        ri[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = rv[0], v2 = rv2[0];
        int i = ri[0];
        for (int k = 1; k < NT / 32; ++k) {
            if (better(rv[k], ri[k], v, i)) {
                v2 = fmaxf(v, rv2[k]);
                v = rv[k];
                i = ri[k];
            } else {
                v2 = fmaxf(v2, rv[k]);
            }
        }
        const int py = i / S, px = i % S;
        const float c0 = v;
        const float cxm = z[py * S + ((px + S - 1) & (S - 1))].x * scale;
        const float cxp = z[py * S + ((px + 1) & (S - 1))].x * scale;
        const float cym = z[((py + S - 1) & (S - 1)) * S + px].x * scale;
        const float cyp = z[((py + 1) & (S - 1)) * S + px].x * scale;
        float dx = 0.0f, dy = 0.0f, den;
        den = cxm - 2.0f * c0 + cxp;
        if (den != 0.0f) dx = (cxm - cxp) / (2.0f * den);
        den = cym - 2.0f * c0 + cyp;
        if (den != 0.0f) dy = (cym - cyp) / (2.0f * den);
        const int wx = px >= S / 2 ? px - S : px, wy = py >= S / 2 ? py - S : py;
        peak[2 * o] = wx;
        peak[2 * o + 1] = wy;
        q[2 * o] = (float)wx + dx;
        q[2 * o + 1] = (float)wy + dy;
        ph[o] = (nr > 0.0f && nt > 0.0f) ? c0 / (nr * nt) : 0.0f;
        if (near_tie) near_tie[o] = (c0 - v2) < 1e-6f * fabsf(c0);
    }
}

// ---------------------------------------------------------------------------
// S = 64 (the batched-scan ROIs): radix-8 transforms in registers.  A 64-point
// line transform is 8 x 8 (Cooley-Tukey): eight 8-point DFTs over the stride-8
// subsequences, a twiddle W64^(n2 k1), eight 8-point DFTs over n2, natural-
// order output.  512 threads = 64 lines x 8; thread (line = tid % 64,
// t = tid / 64) so that a warp touches 32 consecutive rows or columns and the
// twiddles are warp-uniform.  Rows are padded to 65 elements (conflict-free
// column access).  4 shared-memory passes per 2-D transform instead of 12
// radix-2 stages.
namespace r8 {

constexpr int S = 64, ZS = 65, NT = 512;

// multiply by s*i (s = -1: forward twiddle sign)
template <int SG>
__device__ __forceinline__ float2 mul_si(float2 z) { return SG < 0 ? make_float2(z.y, -z.x) : make_float2(-z.y, z.x); }

__device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// 4-point DFT with sign SG, in place on (a0, a1, a2, a3)
template <int SG>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = add(a0, a2), t1 = sub(a0, a2), t2 = add(a1, a3), t3 = mul_si<SG>(sub(a1, a3));
    a0 = add(t0, t2);
    a2 = sub(t0, t2);
    a1 = add(t1, t3);
    a3 = sub(t1, t3);
}

// 8-point DFT with sign SG: X[k] = sum_n x[n] exp(SG 2 pi i n k / 8)
template <int SG>
__device__ __forceinline__ void dft8(float2 (&x)[8])
{
    float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4<SG>(e0, e1, e2, e3);
    dft4<SG>(o0, o1, o2, o3);
    const float c = 0.70710678118654752f;
    const float2 w1o1 = make_float2(c * (o1.x - SG * o1.y), c * (o1.y + SG * o1.x));   // (c, SG c) * o1
    const float2 w2o2 = mul_si<SG>(o2);
    const float2 w3o3 = make_float2(c * (-o3.x - SG * o3.y), c * (-o3.y + SG * o3.x));  // (-c, SG c) * o3
    x[0] = add(e0, o0);
    x[4] = sub(e0, o0);
    x[1] = add(e1, w1o1);
    x[5] = sub(e1, w1o1);
    x[2] = add(e2, w2o2);
    x[6] = sub(e2, w2o2);
    x[3] = add(e3, w3o3);
    x[7] = sub(e3, w3o3);
}

// One 64-point pass over all 64 lines.  ROWS: line = row, element stride 1;
// else line = column, element stride ZS.  tw[j] = exp(-2 pi i j / 64).
template <int SG, bool ROWS>
__device__ __forceinline__ void pass64(float2 *z, const float2 *tw)
{
    const int line = threadIdx.x & 63, t = threadIdx.x >> 6;
    const int ls = ROWS ? ZS : 1, es = ROWS ? 1 : ZS;
    float2 *zl = z + line * ls;
    float2 v[8];
    // stage 1: DFT over n1 of x[8 n1 + t], twiddle W64^(t k1)
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) v[n1] = zl[(8 * n1 + t) * es];
    dft8<SG>(v);
#pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) {
        float2 w = tw[t * k1];
        if (SG > 0) w.y = -w.y;
        v[k1] = make_float2(v[k1].x * w.x - v[k1].y * w.y, v[k1].x * w.y + v[k1].y * w.x);
    }
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) zl[(8 * t + k1) * es] = v[k1];
    __syncthreads();
    // stage 2: DFT over n2 of Y'[n2][k1 = t] -> X[t + 8 k2]
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) v[n2] = zl[(8 * n2 + t) * es];
    dft8<SG>(v);
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) zl[(t + 8 * k2) * es] = v[k2];
    __syncthreads();
}

__global__ void __launch_bounds__(NT) xcf64_kernel(const float *__restrict__ rem, const float *__restrict__ test, int B,
                                                   int H, int W, const int32_t *__restrict__ roi, int N, int window,
                                                   float *q, int32_t *peak, float *ph, int32_t *near_tie)
{
    __shared__ float2 z[S * ZS];
    __shared__ float2 tw[S];
    __shared__ float win[S];
    __shared__ float red[NT / 32];
    __shared__ float rv[NT / 32], rv2[NT / 32];
    __shared__ int ri[NT / 32];

    const int b = blockIdx.x / N, r = blockIdx.x % N;
    const int cx = roi[2 * r], cy = roi[2 * r + 1];
    const int x0 = cx - S / 2, y0 = cy - S / 2;
    const size_t o = (size_t)blockIdx.x;
    if (x0 < 0 || y0 < 0 || x0 + S > W || y0 + S > H) {   // ROI outside the image
        if (threadIdx.x == 0) {
            q[2 * o] = q[2 * o + 1] = __int_as_float(0x7fc00000);
            peak[2 * o] = peak[2 * o + 1] = 0;
            ph[o] = 0.0f;
            if (near_tie) near_tie[o] = 0;
        }
        return;
    }
    if (threadIdx.x < S) {
        float sn, cs;
        sincospif(-2.0f * (float)threadIdx.x / (float)S, &sn, &cs);
        tw[threadIdx.x] = make_float2(cs, sn);
        win[threadIdx.x] = window ? 0.5f * (1.0f - cospif(2.0f * (float)threadIdx.x / (float)(S - 1))) : 1.0f;
    }
    const float *T = test + (size_t)b * H * W + (size_t)y0 * W + x0;
    const float *Rr = rem + (size_t)b * H * W + (size_t)y0 * W + x0;
    float st = 0.0f, sr = 0.0f;
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const int y = idx / S, x = idx % S;
        const float tv = __ldg(T + (size_t)y * W + x), rv_ = __ldg(Rr + (size_t)y * W + x);
        z[y * ZS + x] = make_float2(tv, rv_);
        st += tv;
        sr += rv_;
    }
    const float mt = block_sum<NT>(st, red) * (1.0f / (S * S));
    const float mr = block_sum<NT>(sr, red) * (1.0f / (S * S));
    float nt = 0.0f, nr = 0.0f;
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const int y = idx / S, x = idx % S;
        const float wgt = win[y] * win[x];
        float2 v = z[y * ZS + x];
        v.x = (v.x - mt) * wgt;
        v.y = (v.y - mr) * wgt;
        z[y * ZS + x] = v;
        nt = fmaf(v.x, v.x, nt);
        nr = fmaf(v.y, v.y, nr);
    }
    nt = sqrtf(block_sum<NT>(nt, red));
    nr = sqrtf(block_sum<NT>(nr, red));   // ends with a barrier: z complete

    pass64<-1, true>(z, tw);
    pass64<-1, false>(z, tw);

    // cross-power P(k) = T(k) conj(R(k)), P(-k) = conj(P(k)); pairs (k, -k) in place
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const int ky = idx / S, kx = idx % S;
        const int my = (S - ky) & (S - 1), mx = (S - kx) & (S - 1);
        const int m = my * S + mx;
        if (idx > m) continue;
        const float2 zk = z[ky * ZS + kx], zm = z[my * ZS + mx];
        const float2 Tk = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 Rk = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        const float2 P = make_float2(Tk.x * Rk.x + Tk.y * Rk.y, Tk.y * Rk.x - Tk.x * Rk.y);
        z[ky * ZS + kx] = P;
        if (m != idx) z[my * ZS + mx] = make_float2(P.x, -P.y);
    }
    __syncthreads();
    pass64<1, true>(z, tw);
    pass64<1, false>(z, tw);

    // argmax of c = Re(z) / S^2 (first maximum in row-major order) and runner-up
    const float scale = 1.0f / (float)(S * S);
    float bv = -INFINITY, bv2 = -INFINITY;
    int bi = 0x7fffffff;
    for (int idx = threadIdx.x; idx < S * S; idx += NT) {
        const float v = z[(idx / S) * ZS + idx % S].x * scale;
        if (better(v, idx, bv, bi)) {
            bv2 = bv;
            bv = v;
            bi = idx;
        } else if (v > bv2) {
            bv2 = v;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const float ov2 = __shfl_xor_sync(0xffffffffu, bv2, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (better(ov, oi, bv, bi)) {
            bv2 = fmaxf(bv, ov2);
            bv = ov;
            bi = oi;
        } else {
            bv2 = fmaxf(bv2, ov);
        }
    }
    if ((threadIdx.x & 31) == 0) {
        rv[threadIdx.x >> 5] = bv;
        rv2[threadIdx.x >> 5] = bv2;
        ri[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = rv[0], v2 = rv2[0];
        int i = ri[0];
        for (int k = 1; k < NT / 32; ++k) {
            if (better(rv[k], ri[k], v, i)) {
                v2 = fmaxf(v, rv2[k]);
                v = rv[k];
                i = ri[k];
            } else {
                v2 = fmaxf(v2, rv[k]);
            }
        }
        const int py = i / S, px = i % S;
        const float c0 = v;
        const float cxm = z[py * ZS + ((px + S - 1) & (S - 1))].x * scale;
        const float cxp = z[py * ZS + ((px + 1) & (S - 1))].x * scale;
        const float cym = z[((py + S - 1) & (S - 1)) * ZS + px].x * scale;
        const float cyp = z[((py + 1) & (S - 1)) * ZS + px].x * scale;
        float dx = 0.0f, dy = 0.0f, den;
        den = cxm - 2.0f * c0 + cxp;
        if (den != 0.0f) dx = (cxm - cxp) / (2.0f * den);
        den = cym - 2.0f * c0 + cyp;
        if (den != 0.0f) dy = (cym - cyp) / (2.0f * den);
        const int wx = px >= S / 2 ? px - S : px, wy = py >= S / 2 ? py - S : py;
        peak[2 * o] = wx;
        peak[2 * o + 1] = wy;
        q[2 * o] = (float)wx + dx;
        q[2 * o + 1] = (float)wy + dy;
        ph[o] = (nr > 0.0f && nt > 0.0f) ? c0 / (nr * nt) : 0.0f;
        if (near_tie) near_tie[o] = (c0 - v2) < 1e-6f * fabsf(c0);
    }
}

}  // namespace r8

// ---------------------------------------------------------------------------
// S = 256 (the paper's ROIs of 256 x 256 on 1244 x 1024 patterns): the 2-D
// array (512 KB of complex values) does not fit in shared memory, so the
// transform goes through a global scratch array Z [roi][256][256] in three
// launches, each staging lines in shared memory:
//   rows:  per ROI, means and window norms, then 32-row chunks: zero mean,
//          Hann window, pack z = t + i r, forward row FFTs, store;
//   cols:  per ROI and group of 16 columns k with their mirrors -k: forward
//          column FFTs, the cross power P(k) = T(k) conj R(k) with
//          T = (Z(k) + conj Z(-k))/2, R = (Z(k) - conj Z(-k))/2i (and
//          P(-k) = conj P(k)), inverse column FFTs, store;
//   peak:  per ROI, 32-row chunks: inverse row FFTs, the real correlation
//          c = Re / S^2 written over the scratch, first maximum in row-major
//          order and runner-up, then the parabolic sub-pixel fit from the
//          stored surface.
// The arithmetic per element is that of the shared-memory kernel (radix-2
// transforms, FP32).
namespace x256 {

constexpr int S = 256, NT = 256, LS = S + 1;   // line stride (odd: conflict-free column access)

__device__ __forceinline__ int brev8(int v) { return (int)(__brev((unsigned)v) >> 24); }

// In-place 256-point transforms of nl lines z[line * LS + i]; sign -1 forward, +1 inverse (unscaled).
__device__ void fft_lines(float2 *z, int nl, const float2 *tw, int sign)
{
    for (int idx = threadIdx.x; idx < nl * S; idx += NT) {
        const int line = idx >> 8, x = idx & (S - 1), j = brev8(x);
        if (x < j) {
            float2 *p = z + line * LS;
            const float2 t = p[x];
            p[x] = p[j];
            p[j] = t;
        }
    }
    __syncthreads();
    for (int half = 1; half < S; half <<= 1) {
        const int tstep = S / (2 * half);
        for (int b = threadIdx.x; b < nl * (S / 2); b += NT) {
            const int line = b >> 7, bf = b & (S / 2 - 1);
            const int grp = bf / half, j = bf % half;
            const int i0 = grp * 2 * half + j, i1 = i0 + half;
            float2 w = tw[j * tstep];
            if (sign > 0) w.y = -w.y;
            float2 *p = z + line * LS;
            const float2 v = cmul(p[i1], w), u = p[i0];
            p[i0] = make_float2(u.x + v.x, u.y + v.y);
            p[i1] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

__device__ void twiddles(float2 *tw)
{
    for (int j = threadIdx.x; j < S / 2; j += NT) {
        float s, c;
        sincospif(-2.0f * (float)j / (float)S, &s, &c);
        tw[j] = make_float2(c, s);
    }
}

// Block sum of a double per thread (result broadcast).
__device__ double block_sum_d(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < NT / 32; ++i) t += red[i];
    __syncthreads();
    return t;
}

constexpr int RCH = 32;   // rows (or columns) staged at a time

// One CTA per (pair, ROI) of the chunk.  norms[2 * roi] = |t_w|, |r_w| (negative: ROI outside the image).
__global__ void __launch_bounds__(NT) rows_kernel(const float *__restrict__ rem, const float *__restrict__ test, int b0,
                                                  int H, int W, const int32_t *__restrict__ roi, int N, int window,
                                                  float2 *Z, float *norms)
{
    extern __shared__ float2 zs[];   // [RCH][LS]
    __shared__ float2 tw[S / 2];
    __shared__ float win[S];
    __shared__ double red[NT / 32];
    const int lr = blockIdx.x, b = b0 + lr / N, r = lr % N;
    const int x0 = roi[2 * r] - S / 2, y0 = roi[2 * r + 1] - S / 2;
    if (x0 < 0 || y0 < 0 || x0 + S > W || y0 + S > H) {
        if (threadIdx.x == 0) norms[2 * lr] = norms[2 * lr + 1] = -1.0f;
        return;
    }
    twiddles(tw);
    for (int n = threadIdx.x; n < S; n += NT)
        win[n] = window ? 0.5f * (1.0f - cospif(2.0f * (float)n / (float)(S - 1))) : 1.0f;
    const float *T = test + (size_t)b * H * W + (size_t)y0 * W + x0;
    const float *R = rem + (size_t)b * H * W + (size_t)y0 * W + x0;
    // means (FP32 partial sums of one row per thread, combined in FP64)
    double st = 0.0, sr = 0.0;
    for (int y = threadIdx.x; y < S; y += NT) {
        float a = 0.0f, c = 0.0f;
        for (int x = 0; x < S; ++x) {
            a += __ldg(T + (size_t)y * W + x);
            c += __ldg(R + (size_t)y * W + x);
        }
        st += a;
        sr += c;
    }
    const float mt = (float)(block_sum_d(st, red) / (S * S)), mr = (float)(block_sum_d(sr, red) / (S * S));
    float2 *Zr = Z + (size_t)lr * S * S;
    double nt = 0.0, nr = 0.0;
    for (int c0 = 0; c0 < S; c0 += RCH) {
        float at = 0.0f, ar = 0.0f;
        for (int idx = threadIdx.x; idx < RCH * S; idx += NT) {
            const int y = c0 + (idx >> 8), x = idx & (S - 1);
            const float wgt = win[y] * win[x];
            const float tv = (__ldg(T + (size_t)y * W + x) - mt) * wgt, rv = (__ldg(R + (size_t)y * W + x) - mr) * wgt;
            zs[(idx >> 8) * LS + x] = make_float2(tv, rv);
            at = fmaf(tv, tv, at);
            ar = fmaf(rv, rv, ar);
        }
        nt += at;
        nr += ar;
        __syncthreads();
        fft_lines(zs, RCH, tw, -1);
        for (int idx = threadIdx.x; idx < RCH * S; idx += NT)
            Zr[(size_t)(c0 + (idx >> 8)) * S + (idx & (S - 1))] = zs[(idx >> 8) * LS + (idx & (S - 1))];
        __syncthreads();
    }
    nt = block_sum_d(nt, red);
    nr = block_sum_d(nr, red);
    if (threadIdx.x == 0) {
        norms[2 * lr] = (float)sqrt(nt);
        norms[2 * lr + 1] = (float)sqrt(nr);
    }
}

// One CTA per (pair, ROI, column group g): g < 8: columns 16 g .. 16 g + 15 and their mirrors; g = 8: column 128.
__global__ void __launch_bounds__(NT) cols_kernel(float2 *Z, const float *__restrict__ norms)
{
    extern __shared__ float2 zs[];   // [32][LS]: slot k < 16 column C_k, slot 16 + k column -C_k
    __shared__ float2 tw[S / 2];
    const int lr = blockIdx.x / 9, g = blockIdx.x % 9;
    if (norms[2 * lr] < 0.0f) return;
    const int nc = g < 8 ? 16 : 1;
    twiddles(tw);
    float2 *Zr = Z + (size_t)lr * S * S;
    auto col = [&](int slot) {
        const int k = slot & 15, c = g < 8 ? 16 * g + k : 128;
        return slot < 16 ? c : (S - c) & (S - 1);
    };
    const int nl = 2 * nc;
    for (int idx = threadIdx.x; idx < S * nl; idx += NT) {
        const int y = idx / nl, sl = idx - y * nl, slot = sl < nc ? sl : 16 + (sl - nc);
        zs[slot * LS + y] = Zr[(size_t)y * S + col(slot)];
    }
    __syncthreads();
    // forward column transforms of the loaded lines (slots 0..nc-1 and 16..16+nc-1)
    fft_lines(zs, 16 + nc, tw, -1);
    // cross power: element (ky, C_k) with its partner (-ky, -C_k)
    for (int idx = threadIdx.x; idx < nc * S; idx += NT) {
        const int k = idx / S, ky = idx - k * S, my = (S - ky) & (S - 1);
        const int c = col(k);
        const bool self = c == ((S - c) & (S - 1));   // columns 0 and 128 pair with themselves
        float2 *pk = zs + k * LS + ky;
        float2 *pm = self ? zs + k * LS + my : zs + (16 + k) * LS + my;
        if (self && ky > my) continue;
        const float2 zk = *pk, zm = *pm;
        const float2 Tk = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        const float2 Rk = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        const float2 P = make_float2(Tk.x * Rk.x + Tk.y * Rk.y, Tk.y * Rk.x - Tk.x * Rk.y);
        *pk = P;
        if (pm != pk) *pm = make_float2(P.x, -P.y);
    }
    __syncthreads();
    fft_lines(zs, 16 + nc, tw, +1);
    for (int idx = threadIdx.x; idx < S * nl; idx += NT) {
        const int y = idx / nl, sl = idx - y * nl, slot = sl < nc ? sl : 16 + (sl - nc);
        const int c = col(slot);
        if (slot >= 16 && c == col(slot - 16)) continue;   // self-paired column: stored once
        Zr[(size_t)y * S + c] = zs[slot * LS + y];
    }
}

__global__ void __launch_bounds__(NT) peak_kernel(float2 *Z, const float *__restrict__ norms, int b0, int N, float *q,
                                                  int32_t *peak, float *ph, int32_t *near_tie)
{
    extern __shared__ float2 zs[];   // [RCH][LS]
    __shared__ float2 tw[S / 2];
    __shared__ float rv[NT / 32], rv2[NT / 32];
    __shared__ int ri[NT / 32];
    const int lr = blockIdx.x;
    const size_t o = (size_t)b0 * N + lr;
    const float nt = norms[2 * lr], nr = norms[2 * lr + 1];
    if (nt < 0.0f) {
        if (threadIdx.x == 0) {
            q[2 * o] = q[2 * o + 1] = __int_as_float(0x7fc00000);
            peak[2 * o] = peak[2 * o + 1] = 0;
            ph[o] = 0.0f;
            if (near_tie) near_tie[o] = 0;
        }
        return;
    }
    twiddles(tw);
    float2 *Zr = Z + (size_t)lr * S * S;
    float *Cr = reinterpret_cast<float *>(Zr);   // the real surface overwrites the rows already read
    const float scale = 1.0f / (float)(S * S);
    float bv = -INFINITY, bv2 = -INFINITY;
    int bi = 0x7fffffff;
    for (int c0 = 0; c0 < S; c0 += RCH) {
        for (int idx = threadIdx.x; idx < RCH * S; idx += NT)
            zs[(idx >> 8) * LS + (idx & (S - 1))] = Zr[(size_t)(c0 + (idx >> 8)) * S + (idx & (S - 1))];
        __syncthreads();
        fft_lines(zs, RCH, tw, +1);
        for (int idx = threadIdx.x; idx < RCH * S; idx += NT) {
            const int i = c0 * S + idx;
            const float v = zs[(idx >> 8) * LS + (idx & (S - 1))].x * scale;
            Cr[i] = v;
            if (better(v, i, bv, bi)) {
                bv2 = bv;
                bv = v;
                bi = i;
            } else if (v > bv2) {
                bv2 = v;
            }
        }
        __syncthreads();
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
        const float ov2 = __shfl_xor_sync(0xffffffffu, bv2, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (better(ov, oi, bv, bi)) {
            bv2 = fmaxf(bv, ov2);
            bv = ov;
            bi = oi;
        } else {
            bv2 = fmaxf(bv2, ov);
        }
    }
    if ((threadIdx.x & 31) == 0) {
        rv[threadIdx.x >> 5] = bv;
        rv2[threadIdx.x >> 5] = bv2;
        ri[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = rv[0], v2 = rv2[0];
        int i = ri[0];
        for (int k = 1; k < NT / 32; ++k) {
            if (better(rv[k], ri[k], v, i)) {
                v2 = fmaxf(v, rv2[k]);
                v = rv[k];
                i = ri[k];
            } else {
                v2 = fmaxf(v2, rv[k]);
            }
        }
        const int py = i / S, px = i % S;
        const float c0 = v;
        const float cxm = Cr[py * S + ((px + S - 1) & (S - 1))], cxp = Cr[py * S + ((px + 1) & (S - 1))];
        const float cym = Cr[((py + S - 1) & (S - 1)) * S + px], cyp = Cr[((py + 1) & (S - 1)) * S + px];
        float dx = 0.0f, dy = 0.0f, den;
        den = cxm - 2.0f * c0 + cxp;
        if (den != 0.0f) dx = (cxm - cxp) / (2.0f * den);
        den = cym - 2.0f * c0 + cyp;
        if (den != 0.0f) dy = (cym - cyp) / (2.0f * den);
        const int wx = px >= S / 2 ? px - S : px, wy = py >= S / 2 ? py - S : py;
        peak[2 * o] = wx;
        peak[2 * o + 1] = wy;
        q[2 * o] = (float)wx + dx;
        q[2 * o + 1] = (float)wy + dy;
        ph[o] = (nr > 0.0f && nt > 0.0f) ? c0 / (nr * nt) : 0.0f;
        if (near_tie) near_tie[o] = (c0 - v2) < 1e-6f * fabsf(c0);
    }
}

constexpr int WS_Z = 19, WS_NORMS = 20;
constexpr size_t kMaxScratch = (size_t)2 << 30;   // bound of the scratch array (pairs are processed in chunks)

int launch(hrebsd_ctx *ctx, const float *rem, const float *test, int B, int H, int W, const int32_t *roi, int N,
           int window, float *q, int32_t *peak, float *ph, int32_t *near_tie, cudaStream_t st)
{
    const size_t per_pair = (size_t)N * S * S * sizeof(float2);
    int chunk = (int)(kMaxScratch / per_pair);
    if (chunk < 1) chunk = 1;
    if (chunk > B) chunk = B;
    void *zb, *nb;
    int e;
    if ((e = hr_ws(ctx, WS_Z, per_pair * chunk, &zb))) return e;
    if ((e = hr_ws(ctx, WS_NORMS, (size_t)chunk * N * 2 * sizeof(float), &nb))) return e;
    float2 *Z = (float2 *)zb;
    float *norms = (float *)nb;
    const int smem_lines = 32 * LS * (int)sizeof(float2);
    HR_CHECK(cudaFuncSetAttribute(rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_lines));
    HR_CHECK(cudaFuncSetAttribute(cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_lines));
    HR_CHECK(cudaFuncSetAttribute(peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_lines));
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nb_ = B - b0 < chunk ? B - b0 : chunk;
        const unsigned rois = (unsigned)nb_ * (unsigned)N;
        hr_prof_begin(ctx, st);
        rows_kernel<<<rois, NT, smem_lines, st>>>(rem, test, b0, H, W, roi, N, window, Z, norms);
        hr_prof_end(ctx, PROF_XCF, st);
        HR_LAUNCHED(ctx);
        hr_prof_begin(ctx, st);
        cols_kernel<<<rois * 9u, NT, smem_lines, st>>>(Z, norms);
        hr_prof_end(ctx, PROF_XCF, st);
        HR_LAUNCHED(ctx);
        hr_prof_begin(ctx, st);
        peak_kernel<<<rois, NT, smem_lines, st>>>(Z, norms, b0, N, q, peak, ph, near_tie);
        hr_prof_end(ctx, PROF_XCF, st);
        HR_LAUNCHED(ctx);
    }
    return HREBSD_OK;
}

}  // namespace x256

template <int S, int NT>
int launch_xcf(hrebsd_ctx *ctx, const float *rem, const float *test, int B, int H, int W, const int32_t *roi, int N,
               int window, float *q, int32_t *peak, float *ph, int32_t *near_tie, cudaStream_t st)
{
    const size_t smem = sizeof(float2) * S * S;
    if (smem > 48 * 1024) HR_CHECK(cudaFuncSetAttribute(xcf_kernel<S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    hr_prof_begin(ctx, st);
    xcf_kernel<S, NT><<<B * N, NT, smem, st>>>(rem, test, B, H, W, roi, N, window, q, peak, ph, near_tie);
    hr_prof_end(ctx, PROF_XCF, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

}  // namespace

extern "C" int hrebsd_xcf_roi_batch(hrebsd_ctx *ctx, const float *remapped, const float *test, int B, int H, int W,
                                    const int32_t *roi_xy, int N, int S, int window, float *q, int32_t *peak,
                                    float *peak_height, int32_t *near_tie, void *stream)
{
    if (!ctx || B < 0 || N < 0 || H < 2 || W < 2) return HREBSD_EINVAL;
    if (S != 16 && S != 32 && S != 64 && S != 128 && S != 256) return HREBSD_EINVAL;
    if ((long long)B * N > 0x7fffffffLL) return HREBSD_EINVAL;
    if (B == 0 || N == 0) return HREBSD_OK;
    if (!remapped || !test || !roi_xy || !q || !peak || !peak_height) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    cudaStream_t st = hr_stream(stream);
    switch (S) {
    case 16: return launch_xcf<16, 128>(ctx, remapped, test, B, H, W, roi_xy, N, window, q, peak, peak_height, near_tie, st);
    case 32: return launch_xcf<32, 256>(ctx, remapped, test, B, H, W, roi_xy, N, window, q, peak, peak_height, near_tie, st);
    case 64: {
        hr_prof_begin(ctx, st);
        r8::xcf64_kernel<<<B * N, r8::NT, 0, st>>>(remapped, test, B, H, W, roi_xy, N, window, q, peak, peak_height,
                                                   near_tie);
        hr_prof_end(ctx, PROF_XCF, st);
        HR_LAUNCHED(ctx);
        return HREBSD_OK;
    }
    case 128: return launch_xcf<128, 512>(ctx, remapped, test, B, H, W, roi_xy, N, window, q, peak, peak_height, near_tie, st);
    default: return x256::launch(ctx, remapped, test, B, H, W, roi_xy, N, window, q, peak, peak_height, near_tie, st);
    }
}
