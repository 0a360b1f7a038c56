// a5, a8: FP64 deformation-gradient fits (Section 2, Eq. 2-5 and Eq. 12).
//
// Eq. 2 maps a reference point r (lifted to (x - xpc, y - ypc, Z*)) to the
// test point Z* F r / ((F r).k).  Eq. 3 fits F to N point pairs by least
// squares.  The objective is invariant under F -> lambda F, so the fit runs
// in the gauge F_33 = 1: a linear start from the cross-multiplied equations
// Z* (F r)_a - r'_a (F r)_3 = 0 (8 unknowns, normal equations), then
// Gauss-Newton on the projected residuals; last, det F = 1.  The rotation is
// the polar factor R = P Q^T of F = P D Q^T (Eq. 4-5), computed with the
// Newton iteration X <- (X + X^-T)/2, which converges to the same orthogonal
// factor as the SVD.
//
// One thread owns one pair: the work per pair is a few thousand FP64 flops,
// so the kernels are latency-, not throughput-bound, and FP64 (slow on this
// part) costs microseconds for a whole scan.
#include <math.h>

#include "internal.cuh"

namespace {

constexpr int kMaxRoi = 512;

// Solve the n x n system A x = b (row-major, destroyed) by Gaussian
// elimination with partial pivoting.  Returns false if singular.
__device__ bool gauss_solve(double *A, double *b, int n, double *x)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = fabs(A[c * n + c]);
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > best) { best = fabs(A[r * n + c]); piv = r; }
        if (!(best > 1e-300)) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
        x[r] = s / A[r * n + r];
    }
    return true;
}

__device__ double det3(const double *F)
{
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
}

// Fit F (det 1) to N point pairs: pts(i, p) fills p = {rx, ry, tx, ty}, the
// reference and test points relative to the pattern centre (recomputed on
// demand instead of stored, to keep per-thread local memory small).  Returns
// false on a singular system.
template <class Pts>
__device__ bool fit_F(Pts pts, int N, double zs, double *F)
{
    double A[64], b[8], x[8];
    // linear start, F_33 = 1: Z* (F r)_a - t_a (F r)_3 = 0
    for (int i = 0; i < 64; ++i) A[i] = 0.0;
    for (int i = 0; i < 8; ++i) b[i] = 0.0;
    for (int i = 0; i < N; ++i) {
        double pt[4];
        pts(i, pt);
        const double r[3] = {pt[0], pt[1], zs};
        const double t[2] = {pt[2], pt[3]};
        for (int a = 0; a < 2; ++a) {
            double row[8];
            for (int k = 0; k < 8; ++k) row[k] = 0.0;
            for (int c = 0; c < 3; ++c) row[a * 3 + c] = zs * r[c];
            row[6] = -t[a] * r[0];
            row[7] = -t[a] * r[1];
            const double rhs = t[a] * zs;   // moves -t_a F_33 r_3 = -t_a Z* to the right
            for (int p = 0; p < 8; ++p) {
                b[p] += row[p] * rhs;
                for (int q = 0; q < 8; ++q) A[p * 8 + q] += row[p] * row[q];
            }
        }
    }
    if (!gauss_solve(A, b, 8, x)) return false;
    for (int k = 0; k < 8; ++k) F[k] = x[k];
    F[8] = 1.0;
    // Gauss-Newton on the Eq. 3 residuals Z* (F r)_a / (F r)_3 - t_a
    for (int it = 0; it < 60; ++it) {
        for (int i = 0; i < 64; ++i) A[i] = 0.0;
        for (int i = 0; i < 8; ++i) b[i] = 0.0;
        for (int i = 0; i < N; ++i) {
            double pt[4];
            pts(i, pt);
            const double r[3] = {pt[0], pt[1], zs};
            double v[3];
            for (int a = 0; a < 3; ++a) v[a] = F[a * 3] * r[0] + F[a * 3 + 1] * r[1] + F[a * 3 + 2] * r[2];
            const double iv = 1.0 / v[2];
            const double t[2] = {pt[2], pt[3]};
            for (int a = 0; a < 2; ++a) {
                const double res = zs * v[a] * iv - t[a];
                double J[8];
                for (int k = 0; k < 8; ++k) J[k] = 0.0;
                for (int c = 0; c < 3; ++c) J[a * 3 + c] = zs * r[c] * iv;
                J[6] = -zs * v[a] * r[0] * iv * iv;
                J[7] = -zs * v[a] * r[1] * iv * iv;
                for (int p = 0; p < 8; ++p) {
                    b[p] -= J[p] * res;
                    for (int q = 0; q < 8; ++q) A[p * 8 + q] += J[p] * J[q];
                }
            }
        }
        if (!gauss_solve(A, b, 8, x)) return false;
        double sn = 0.0, fn = 0.0;
        for (int k = 0; k < 8; ++k) {
            F[k] += x[k];
            sn += x[k] * x[k];
            fn += F[k] * F[k];
        }
        if (sqrt(sn) <= 1e-15 * sqrt(fn + 1.0)) break;
    }
    const double d = det3(F);
    if (!(d > 0.0)) return false;
    const double sc = cbrt(d);
    for (int k = 0; k < 9; ++k) F[k] /= sc;
    return true;
}

// Polar factor by Newton's iteration X <- (X + X^-T)/2 (Higham), FP64.
__device__ void polar_newton(const double *F, double *R)
{
    double X[9];
    for (int k = 0; k < 9; ++k) X[k] = F[k];
    for (int it = 0; it < 100; ++it) {
        // X^-T = cof(X) / det(X)
        double C[9];
        C[0] = X[4] * X[8] - X[5] * X[7];
        C[1] = X[5] * X[6] - X[3] * X[8];
        C[2] = X[3] * X[7] - X[4] * X[6];
        C[3] = X[2] * X[7] - X[1] * X[8];
        C[4] = X[0] * X[8] - X[2] * X[6];
        C[5] = X[1] * X[6] - X[0] * X[7];
        C[6] = X[1] * X[5] - X[2] * X[4];
        C[7] = X[2] * X[3] - X[0] * X[5];
        C[8] = X[0] * X[4] - X[1] * X[3];
        const double d = X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
        double diff = 0.0, nrm = 0.0;
        for (int k = 0; k < 9; ++k) {
            double nx = 0.5 * (X[k] + C[k] / d);
            diff += (nx - X[k]) * (nx - X[k]);
            nrm += nx * nx;
            X[k] = nx;
        }
        if (diff <= 1e-32 * nrm) break;
    }
    for (int k = 0; k < 9; ++k) R[k] = X[k];
}

__device__ float bilinear_clamped(const float *M, int h, int w, float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(w - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(h - 1));
    int x0 = min((int)floorf(x), w - 2);
    int y0 = min((int)floorf(y), h - 2);
    float fx = x - (float)x0, fy = y - (float)y0;
    const float *p = M + (size_t)y0 * w + x0;
    float top = fmaf(fx, p[1], (1.0f - fx) * p[0]);
    float bot = fmaf(fx, p[w + 1], (1.0f - fx) * p[w]);
    return fmaf(fy, bot, (1.0f - fy) * top);
}

__device__ void set_identity(double *M)
{
    for (int k = 0; k < 9; ++k) M[k] = (k % 4 == 0) ? 1.0 : 0.0;
}

__global__ void fit_rotation_kernel(const float *__restrict__ field, int B, int H, int W,
                                    const int32_t *__restrict__ roi, int N, double xpc, double ypc, double zs,
                                    double *F_first, double *R_finite, int32_t *status)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float *fx = field + (size_t)b * 2 * H * W;
    const float *fy = fx + (size_t)H * W;
    // r_i = c_i - u(c_i), r'_i = c_i; the field is sampled at the ROI centre
    // (index coordinates c - 0.5)
    auto pts = [&](int i, double *pt) {
        const double cx = roi[2 * i], cy = roi[2 * i + 1];
        const float ux = bilinear_clamped(fx, H, W, (float)(cx - 0.5), (float)(cy - 0.5));
        const float uy = bilinear_clamped(fy, H, W, (float)(cx - 0.5), (float)(cy - 0.5));
        pt[0] = cx - (double)ux - xpc;
        pt[1] = cy - (double)uy - ypc;
        pt[2] = cx - xpc;
        pt[3] = cy - ypc;
    };
    bool finite = true;
    for (int i = 0; i < N; ++i) {
        double pt[4];
        pts(i, pt);
        finite = finite && isfinite(pt[0]) && isfinite(pt[1]);
    }
    double F[9], R[9];
    if (!finite || !fit_F(pts, N, zs, F)) {
        set_identity(F);
        set_identity(R);
        if (status) atomicOr(status + b, finite ? HREBSD_PAIR_FIT_FAILED : (HREBSD_PAIR_FIT_FAILED | HREBSD_PAIR_NONFINITE));
    } else {
        polar_newton(F, R);
    }
    for (int k = 0; k < 9; ++k) {
        F_first[(size_t)b * 9 + k] = F[k];
        R_finite[(size_t)b * 9 + k] = R[k];
    }
}

__global__ void solve_F_kernel(const float *__restrict__ q, const int32_t *__restrict__ roi, int N, int B,
                               double xpc, double ypc, double zs, const double *R_finite, double *Fout,
                               int32_t *status)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    // r_i = c_i, r'_i = c_i + q_i
    auto pts = [&](int i, double *pt) {
        const double cx = roi[2 * i], cy = roi[2 * i + 1];
        const float qx = q[((size_t)b * N + i) * 2], qy = q[((size_t)b * N + i) * 2 + 1];
        pt[0] = cx - xpc;
        pt[1] = cy - ypc;
        pt[2] = cx + (double)qx - xpc;
        pt[3] = cy + (double)qy - ypc;
    };
    bool finite = true;
    for (int i = 0; i < N; ++i) {
        double pt[4];
        pts(i, pt);
        finite = finite && isfinite(pt[2]) && isfinite(pt[3]);
    }
    double Fi[9], F[9];
    if (!finite || !fit_F(pts, N, zs, Fi)) {
        set_identity(Fi);
        if (status) atomicOr(status + b, finite ? HREBSD_PAIR_FIT_FAILED : (HREBSD_PAIR_FIT_FAILED | HREBSD_PAIR_NONFINITE));
    }
    if (R_finite) {
        const double *Rf = R_finite + (size_t)b * 9;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                F[i * 3 + j] = Fi[i * 3] * Rf[j] + Fi[i * 3 + 1] * Rf[3 + j] + Fi[i * 3 + 2] * Rf[6 + j];
    } else {
        for (int k = 0; k < 9; ++k) F[k] = Fi[k];
    }
    for (int k = 0; k < 9; ++k) Fout[(size_t)b * 9 + k] = F[k];
}

// Rotation part of arbitrary F (Eq. 4-5), one thread per pair.
__global__ void polar_kernel(const double *__restrict__ F, int B, double *R)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double Fb[9], Rb[9];
    for (int k = 0; k < 9; ++k) Fb[k] = F[(size_t)b * 9 + k];
    polar_newton(Fb, Rb);
    for (int k = 0; k < 9; ++k) R[(size_t)b * 9 + k] = Rb[k];
}

// Quality of an Eq. 3 fit (Section 3.1, Fig. 3).  Point pairs: from the XCF
// shifts (r = c, r' = c + q) or from the demons field (r = c - u(c), r' = c).
// Model F_m = F R^T when R is given (the second pass, Eq. 12), else F.
// MAE = mean over ROIs of the angle between the measured test direction
// (r' - PC, Z*) and F_m (r - PC, Z*); PH = mean of the peak heights.
__global__ void fit_quality_kernel(const double *__restrict__ F, const double *__restrict__ R,
                                   const float *__restrict__ q, const float *__restrict__ field,
                                   const float *__restrict__ ph, int B, int H, int W, const int32_t *__restrict__ roi,
                                   int N, double xpc, double ypc, double zs, double *mae, double *ph_mean)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double Fm[9];
    const double *Fb = F + (size_t)b * 9;
    if (R) {
        const double *Rb = R + (size_t)b * 9;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Fm[i * 3 + j] = Fb[i * 3] * Rb[j * 3] + Fb[i * 3 + 1] * Rb[j * 3 + 1] + Fb[i * 3 + 2] * Rb[j * 3 + 2];
    } else {
        for (int k = 0; k < 9; ++k) Fm[k] = Fb[k];
    }
    const float *fx = field ? field + (size_t)b * 2 * H * W : nullptr;
    double sum = 0.0, phs = 0.0;
    for (int i = 0; i < N; ++i) {
        const double cx = roi[2 * i], cy = roi[2 * i + 1];
        double r[2], rp[2];
        if (q) {
            r[0] = cx;
            r[1] = cy;
            rp[0] = cx + (double)q[((size_t)b * N + i) * 2];
            rp[1] = cy + (double)q[((size_t)b * N + i) * 2 + 1];
        } else {
            const float ux = bilinear_clamped(fx, H, W, (float)(cx - 0.5), (float)(cy - 0.5));
            const float uy = bilinear_clamped(fx + (size_t)H * W, H, W, (float)(cx - 0.5), (float)(cy - 0.5));
            r[0] = cx - (double)ux;
            r[1] = cy - (double)uy;
            rp[0] = cx;
            rp[1] = cy;
        }
        const double v[3] = {r[0] - xpc, r[1] - ypc, zs};
        double p[3];
        for (int a = 0; a < 3; ++a) p[a] = Fm[a * 3] * v[0] + Fm[a * 3 + 1] * v[1] + Fm[a * 3 + 2] * v[2];
        const double m[3] = {rp[0] - xpc, rp[1] - ypc, zs};
        const double cr[3] = {p[1] * m[2] - p[2] * m[1], p[2] * m[0] - p[0] * m[2], p[0] * m[1] - p[1] * m[0]};
        sum += atan2(sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]), p[0] * m[0] + p[1] * m[1] + p[2] * m[2]);
        if (ph) phs += (double)ph[(size_t)b * N + i];
    }
    mae[b] = sum / N;
    if (ph_mean) ph_mean[b] = ph ? phs / N : 0.0;
}

}  // namespace

extern "C" int hrebsd_fit_rotation(hrebsd_ctx *ctx, const float *field, int B, int H, int W, const int32_t *roi_xy,
                                   int N, const hrebsd_geometry *g, double *F_first, double *R_finite,
                                   int32_t *pair_status, void *stream)
{
    if (!ctx || !g || B < 0 || H < 2 || W < 2 || N < 4 || N > kMaxRoi) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!field || !roi_xy || !F_first || !R_finite) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    hr_prof_begin(ctx, hr_stream(stream));
    fit_rotation_kernel<<<(B + 63) / 64, 64, 0, hr_stream(stream)>>>(field, B, H, W, roi_xy, N, g->xstar * W,
                                                                     g->ystar * H, g->zstar * W, F_first,
                                                                     R_finite, pair_status);
    hr_prof_end(ctx, PROF_FIT, hr_stream(stream));
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

extern "C" int hrebsd_solve_F(hrebsd_ctx *ctx, const float *q, const int32_t *roi_xy, int N, int B, int H, int W,
                              const hrebsd_geometry *g, const double *R_finite, int normalization,
                              const hrebsd_elastic *elastic, double *F, int32_t *pair_status, void *stream)
{
    if (!ctx || !g || B < 0 || H < 2 || W < 2 || N < 4 || N > kMaxRoi) return HREBSD_EINVAL;
    if (normalization != HREBSD_NORM_DET1 && normalization != HREBSD_NORM_TRACTION_FREE) return HREBSD_EINVAL;
    if (normalization == HREBSD_NORM_TRACTION_FREE && (!elastic || !elastic->g || elastic->R < 1))
        return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!q || !roi_xy || !F) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    cudaStream_t st = hr_stream(stream);
    hr_prof_begin(ctx, st);
    solve_F_kernel<<<(B + 63) / 64, 64, 0, st>>>(q, roi_xy, N, B, g->xstar * W, g->ystar * H, g->zstar * W, R_finite,
                                                 F, pair_status);
    hr_prof_end(ctx, PROF_SOLVE, st);
    HR_LAUNCHED(ctx);
    if (normalization == HREBSD_NORM_TRACTION_FREE) return hr_launch_traction_scale(ctx, F, elastic, B, pair_status, st);
    return HREBSD_OK;
}

extern "C" int hrebsd_polar_batch(hrebsd_ctx *ctx, const double *F, int B, double *R, void *stream)
{
    if (!ctx || B < 0) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!F || !R) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    hr_prof_begin(ctx, hr_stream(stream));
    polar_kernel<<<(B + 63) / 64, 64, 0, hr_stream(stream)>>>(F, B, R);
    hr_prof_end(ctx, PROF_FIT, hr_stream(stream));
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

extern "C" int hrebsd_fit_quality(hrebsd_ctx *ctx, const double *F, const double *R, const float *q, const float *field,
                                  const float *ph, int B, int H, int W, const int32_t *roi_xy, int N,
                                  const hrebsd_geometry *g, double *mae, double *ph_mean, void *stream)
{
    if (!ctx || !g || B < 0 || H < 2 || W < 2 || N < 1 || N > kMaxRoi) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!F || !roi_xy || !mae || (!q) == (!field)) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    hr_prof_begin(ctx, hr_stream(stream));
    fit_quality_kernel<<<(B + 63) / 64, 64, 0, hr_stream(stream)>>>(F, R, q, field, ph, B, H, W, roi_xy, N,
                                                                    g->xstar * W, g->ystar * H, g->zstar * W, mae,
                                                                    ph_mean);
    hr_prof_end(ctx, PROF_SOLVE, hr_stream(stream));
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}
