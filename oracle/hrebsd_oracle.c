/*
 * hrebsd_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of the HR-EBSD
 * demons-remapping method of Zhu, Kaufmann & Vecchio, "Novel Remapping
 * Approach for HR-EBSD based on Demons Registration" (arXiv 1907.05993).
 * It is what the CUDA library is checked against: only the tests, the smoke check and
 * the benchmark's CPU-baseline leg load it.  It shares no code, header,
 * table or constant with the CUDA path, and the product never calls it.
 *
 * Every step follows the paper's order; where the paper is silent the
 * reading used is stated at the function.  Conventions:
 *   - images are row-major [H][W]; index coordinates (x = column, y = row)
 *     put pixel centres on integers; continuous detector coordinates put
 *     them at (column + 0.5, row + 0.5), rows downward;
 *   - a displacement field is two planes [2][H][W]: u_x then u_y, in pixels
 *     of the grid it lives on;
 *   - geometry: pattern centre (xstar*W, ystar*H), detector distance
 *     Z* = zstar*W, all in pixels; k = (0,0,1) is the screen normal (Eq. 2).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_RADIUS 32

/* ------------------------------------------------------------------ a1 */
/* Intensity normalisation (Section 2: patterns are first normalised to zero
 * mean).  Reading: zero mean and unit (population) standard deviation; the
 * demons force of Eq. 1 is invariant to the scale, so the unit variance only
 * fixes the meaning of alpha and of the denominator guard.  An image whose
 * standard deviation is at most 1e-6 |mean| (or zero) counts as constant and
 * normalises to all zeros. */
void oracle_normalize(const double *in, long n, double *out)
{
    double s = 0.0, ss = 0.0;
    for (long i = 0; i < n; ++i) s += in[i];
    double mean = s / (double)n;
    for (long i = 0; i < n; ++i) ss += (in[i] - mean) * (in[i] - mean);
    double sd = sqrt(ss / (double)n);
    double inv = (sd > 0.0 && sd > 1e-6 * fabs(mean)) ? 1.0 / sd : 0.0;
    for (long i = 0; i < n; ++i) out[i] = (in[i] - mean) * inv;
}

static int chol_solve(const double *A, const double *b, int n, double *x);

/* Static background correction (Section 3.3 applies background correction
 * before registration; reading for a smooth detector background): fit the
 * quadric c0 + c1 x + c2 y + c3 x^2 + c4 xy + c5 y^2 by least squares over
 * the pattern (x, y in [-1, 1] at pixel centres, normal equations), divide
 * the pattern by it, then normalise (zero mean, unit variance).  flat = 0
 * only normalises.  Where the fitted surface is not positive at every pixel
 * the division is skipped. */
void oracle_preprocess(const double *in, int H, int W, int flat, double *out)
{
    long n = (long)H * W;
    if (!flat) { oracle_normalize(in, n, out); return; }
    double G[36] = {0}, b[6] = {0}, c[6];
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double x = (j + 0.5) / W * 2.0 - 1.0, y = (i + 0.5) / H * 2.0 - 1.0;
            double phi[6] = {1.0, x, y, x * x, x * y, y * y};
            for (int k = 0; k < 6; ++k) {
                b[k] += phi[k] * in[(long)i * W + j];
                for (int l = 0; l < 6; ++l) G[k * 6 + l] += phi[k] * phi[l];
            }
        }
    double *tmp = (double *)malloc(sizeof(double) * n);
    int ok = chol_solve(G, b, 6, c) == 0;
    for (int i = 0; i < H && ok; ++i)
        for (int j = 0; j < W; ++j) {
            double x = (j + 0.5) / W * 2.0 - 1.0, y = (i + 0.5) / H * 2.0 - 1.0;
            double fit = c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y;
            if (!(fit > 0.0)) { ok = 0; break; }
            tmp[(long)i * W + j] = in[(long)i * W + j] / fit;
        }
    oracle_normalize(ok ? tmp : in, n, out);
    free(tmp);
}

/* Multi-resolution pyramid (Section 1, multi-resolution demons): one level
 * down is the 2x2 box mean.  Reading for sizes that do not halve (the paper's
 * 1244 x 1024 patterns with 7 levels): the coarser level is floor(H/2) x
 * floor(W/2), so an odd last row or column takes no part in the mean. */
void oracle_reduce2(const double *in, int H, int W, double *out)
{
    int h = H / 2, w = W / 2;
    for (int i = 0; i < h; ++i)
        for (int j = 0; j < w; ++j)
            out[i * w + j] = 0.25 * (in[(2 * i) * W + 2 * j] + in[(2 * i) * W + 2 * j + 1] +
                                     in[(2 * i + 1) * W + 2 * j] + in[(2 * i + 1) * W + 2 * j + 1]);
}

/* Gaussian taps for the field regularisation: radius ceil(3 sigma),
 * weights exp(-k^2 / (2 sigma^2)) normalised to sum to one.  sigma <= 0 is
 * the identity (the paper's own runs use no smoothing, Section 3.1). */
int oracle_gauss_taps(double sigma, double *taps)
{
    if (!(sigma > 0.0)) { taps[0] = 1.0; return 0; }
    int r = (int)ceil(3.0 * sigma);
    if (r > OR_MAX_RADIUS) r = OR_MAX_RADIUS;
    double s = 0.0;
    for (int k = -r; k <= r; ++k) { taps[k + r] = exp(-(double)(k * k) / (2.0 * sigma * sigma)); s += taps[k + r]; }
    for (int k = 0; k <= 2 * r; ++k) taps[k] /= s;
    return r;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Separable Gaussian, x pass then y pass, replicated borders. */
void oracle_smooth(const double *in, int H, int W, double sigma, double *out)
{
    double taps[2 * OR_MAX_RADIUS + 1];
    int r = oracle_gauss_taps(sigma, taps);
    double *tmp = (double *)malloc(sizeof(double) * (size_t)H * W);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double a = 0.0;
            for (int k = -r; k <= r; ++k) a += taps[k + r] * in[i * W + clampi(j + k, 0, W - 1)];
            tmp[i * W + j] = a;
        }
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double a = 0.0;
            for (int k = -r; k <= r; ++k) a += taps[k + r] * tmp[clampi(i + k, 0, H - 1) * W + j];
            out[i * W + j] = a;
        }
    free(tmp);
}

/* Image gradient: central differences inside, one-sided at the borders. */
void oracle_gradient(const double *f, int H, int W, double *gx, double *gy)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double dx, dy;
            if (j == 0) dx = f[i * W + 1] - f[i * W];
            else if (j == W - 1) dx = f[i * W + j] - f[i * W + j - 1];
            else dx = 0.5 * (f[i * W + j + 1] - f[i * W + j - 1]);
            if (i == 0) dy = f[W + j] - f[j];
            else if (i == H - 1) dy = f[i * W + j] - f[(i - 1) * W + j];
            else dy = 0.5 * (f[(i + 1) * W + j] - f[(i - 1) * W + j]);
            gx[i * W + j] = dx;
            gy[i * W + j] = dy;
        }
}

/* Bilinear sample at index coordinates (x, y), clamped to the image. */
double oracle_bilinear(const double *img, int H, int W, double x, double y)
{
    if (x < 0.0) x = 0.0;
    if (x > W - 1) x = W - 1;
    if (y < 0.0) y = 0.0;
    if (y > H - 1) y = H - 1;
    int x0 = (int)floor(x), y0 = (int)floor(y);
    if (x0 > W - 2) x0 = W - 2;
    if (y0 > H - 2) y0 = H - 2;
    double fx = x - x0, fy = y - y0;
    const double *p = img + (size_t)y0 * W + x0;
    return (1.0 - fy) * ((1.0 - fx) * p[0] + fx * p[1]) + fy * ((1.0 - fx) * p[W] + fx * p[W + 1]);
}

/* Warp of the moving (reference) image: Mw(x) = M(x - u(x)). */
void oracle_warp(const double *M, const double *u, int H, int W, double *out)
{
    const double *ux = u, *uy = u + (size_t)H * W;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j)
            out[i * W + j] = oracle_bilinear(M, H, W, j - ux[i * W + j], i - uy[i * W + j]);
}

/* ------------------------------------------------------------------ a2 */
/* One demons force evaluation (Eq. 1 with the alpha weighting of the
 * diffusion-demons form): d = Mw - F, du = d grad F / (|grad F|^2 + alpha^2 d^2),
 * du = 0 where the denominator is <= 1e-9.  Returns the SSD sum d^2. */
double oracle_demons_force(const double *Fimg, const double *gx, const double *gy, const double *M,
                           const double *u, int H, int W, double alpha, double *du)
{
    long n = (long)H * W;
    double *mw = (double *)malloc(sizeof(double) * n);
    oracle_warp(M, u, H, W, mw);
    double ssd = 0.0;
    for (long p = 0; p < n; ++p) {
        double d = mw[p] - Fimg[p];
        ssd += d * d;
        double den = gx[p] * gx[p] + gy[p] * gy[p] + alpha * alpha * d * d;
        if (den > 1e-9) { du[p] = d * gx[p] / den; du[n + p] = d * gy[p] / den; }
        else { du[p] = 0.0; du[n + p] = 0.0; }
    }
    free(mw);
    return ssd;
}

/* One pyramid level of demons (Section 1; Eq. 1 iterated).  Iteration k at
 * field u_k: force and SSD E_k; stop test (reading of the unstated
 * convergence rule: stop when w > 0, k >= w and E_{k-w} - E_k < tol E_{k-w});
 * else du <- G_su * du, u <- u + du, u <- G_sf * u.  At most `cap` updates.
 * replay >= 0 applies exactly that many updates and ignores the stop rule.
 * ssd_trace (nullable, length cap) receives E_0..E_{k}.  Returns the number
 * of updates applied. */
int oracle_demons_level(const double *Fimg, const double *M, int H, int W, double *u, double alpha,
                        double sigma_up, double sigma_f, int cap, int window, double tol, int replay,
                        double *ssd_trace)
{
    long n = (long)H * W;
    double *gx = (double *)malloc(sizeof(double) * n), *gy = (double *)malloc(sizeof(double) * n);
    double *du = (double *)malloc(sizeof(double) * 2 * n), *tmp = (double *)malloc(sizeof(double) * n);
    double *E = (double *)malloc(sizeof(double) * (cap + 1));
    oracle_gradient(Fimg, H, W, gx, gy);
    int limit = replay >= 0 ? replay : cap;
    int k = 0;
    for (;;) {
        if (k >= limit) break;
        E[k] = oracle_demons_force(Fimg, gx, gy, M, u, H, W, alpha, du);
        if (ssd_trace) ssd_trace[k] = E[k];
        if (replay < 0 && window > 0 && k >= window && (E[k - window] - E[k]) < tol * E[k - window]) break;
        for (int c = 0; c < 2; ++c) {
            oracle_smooth(du + c * n, H, W, sigma_up, tmp);
            for (long p = 0; p < n; ++p) u[c * n + p] += tmp[p];
            oracle_smooth(u + c * n, H, W, sigma_f, tmp);
            memcpy(u + c * n, tmp, sizeof(double) * n);
        }
        ++k;
    }
    free(gx); free(gy); free(du); free(tmp); free(E);
    return k;
}

/* ------------------------------------------------------------------ a4 */
/* Field prolongation to the next finer level (Section 1: the coarse field
 * is the input of the finer level): bilinear at x_c = (x_f + 0.5)/2 - 0.5,
 * replicated edges, values doubled.  The finer level is the stored size H x W
 * of that level, 2h x 2w or one more where the size did not halve (the
 * extra last row or column samples past the coarse edge, i.e. the clamped
 * edge value). */
void oracle_prolong_to(const double *uc, int h, int w, int H, int W, double *uf)
{
    for (int c = 0; c < 2; ++c)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j)
                uf[(size_t)c * H * W + i * W + j] =
                    2.0 * oracle_bilinear(uc + (size_t)c * h * w, h, w, (j + 0.5) * 0.5 - 0.5, (i + 0.5) * 0.5 - 0.5);
}

void oracle_prolong(const double *uc, int h, int w, double *uf) { oracle_prolong_to(uc, h, w, 2 * h, 2 * w, uf); }

/* Multi-resolution demons registration of one pair (a2-a4) on preprocessed
 * patterns (oracle_preprocess).  ref = moving image M, test = fixed image F
 * (reading: the field moves the reference toward the test, Section 2).  Level 0 is the finest; `levels` levels;
 * start_level < 0 means the coarsest.  init (nullable) is the field at the
 * start level [2][H>>s][W>>s].  caps[l], replay[l] (nullable) per level.
 * field_out [2][H][W]; iters_out[l] = updates applied at level l (0 for
 * skipped levels). */
int oracle_demons_register(const double *ref, const double *test, int H, int W, int levels,
                           const int *caps, double alpha, double sigma_up, double sigma_f, int window,
                           double tol, int start_level, const double *init, const int *replay,
                           double *field_out, int *iters_out)
{
    if (levels < 1 || levels > 8) return -1;
    if (start_level < 0 || start_level >= levels) start_level = levels - 1;
    double *Fp[8], *Mp[8];
    long n0 = (long)H * W;
    Fp[0] = (double *)malloc(sizeof(double) * n0);
    Mp[0] = (double *)malloc(sizeof(double) * n0);
    memcpy(Fp[0], test, sizeof(double) * n0);
    memcpy(Mp[0], ref, sizeof(double) * n0);
    for (int l = 1; l < levels; ++l) {
        int h = H >> l, w = W >> l;
        Fp[l] = (double *)malloc(sizeof(double) * h * w);
        Mp[l] = (double *)malloc(sizeof(double) * h * w);
        oracle_reduce2(Fp[l - 1], H >> (l - 1), W >> (l - 1), Fp[l]);
        oracle_reduce2(Mp[l - 1], H >> (l - 1), W >> (l - 1), Mp[l]);
    }
    for (int l = 0; l < levels; ++l) iters_out[l] = 0;
    int hs = H >> start_level, ws = W >> start_level;
    double *u = (double *)calloc(2 * (size_t)hs * ws, sizeof(double));
    if (init) memcpy(u, init, sizeof(double) * 2 * hs * ws);
    for (int l = start_level; l >= 0; --l) {
        int h = H >> l, w = W >> l;
        iters_out[l] = oracle_demons_level(Fp[l], Mp[l], h, w, u, alpha, sigma_up, sigma_f, caps[l], window,
                                           tol, replay ? replay[l] : -1, NULL);
        if (l > 0) {
            int Hf = H >> (l - 1), Wf = W >> (l - 1);
            double *uf = (double *)malloc(sizeof(double) * 2 * (size_t)Hf * Wf);
            oracle_prolong_to(u, h, w, Hf, Wf, uf);
            free(u);
            u = uf;
        }
    }
    memcpy(field_out, u, sizeof(double) * 2 * n0);
    free(u);
    for (int l = 0; l < levels; ++l) { free(Fp[l]); free(Mp[l]); }
    return 0;
}

/* ------------------------------------------------------------ linear algebra */
/* Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix A (row-major,
 * destroyed).  Eigenvalues to w, eigenvectors to the columns of V. */
static void jacobi_eig(double *A, int n, double *w, double *V)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) { tot += A[i * n + j] * A[i * n + j]; if (i != j) off += A[i * n + j] * A[i * n + j]; }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {   /* A <- A J (columns p, q) */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {   /* A <- J^T A (rows p, q) */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

/* Cholesky solve of the SPD system A x = b (n <= 9). Returns 0 on success. */
static int chol_solve(const double *A, const double *b, int n, double *x)
{
    double L[81];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) { if (!(s > 0.0)) return -1; L[i * n + i] = sqrt(s); }
            else L[i * n + j] = s / L[j * n + j];
        }
    double y[9];
    for (int i = 0; i < n; ++i) { double s = b[i]; for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k]; y[i] = s / L[i * n + i]; }
    for (int i = n - 1; i >= 0; --i) { double s = y[i]; for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k]; x[i] = s / L[i * n + i]; }
    return 0;
}

static double det3(const double *F)
{
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) + F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* ------------------------------------------------------------- a5, a8 */
/* Deformation gradient from point pairs (Eq. 2 and Eq. 3).  ref_xy[i] is a
 * reference-pattern point r_i, test_xy[i] its image r'_i = r_i + q_i, both
 * in continuous detector pixels.  Lifted to 3-D as (x - xpc, y - ypc, Z*).
 * Start: the homogeneous linear system Z*(F r)_a - r'_a (F r)_3 = 0
 * (a = 1, 2), solved as the eigenvector of A^T A with the smallest eigenvalue
 * (cyclic Jacobi).  Then Gauss-Newton on the Eq. 3 objective
 * sum 1/2 |Z* F r / ((F r).k) - r'|^2 with the scale gauge F_33 = 1 (the
 * objective is invariant under F -> lambda F, so only 8 parameters are
 * determined), until the step is below 1e-14 or 100 iterations.  Last, the
 * scale is fixed by det F = 1 (reading of the scale indeterminacy; the
 * traction-free gauge needs the elastic constants).  Returns 0, or -1 when
 * fewer than 4 points or the normal matrix is singular. */
int oracle_fit_F(const double *ref_xy, const double *test_xy, int N, double xpc, double ypc, double zs, double *F)
{
    if (N < 4) return -1;
    double AtA[81];
    memset(AtA, 0, sizeof(AtA));
    for (int i = 0; i < N; ++i) {
        double r[3] = {ref_xy[2 * i] - xpc, ref_xy[2 * i + 1] - ypc, zs};
        double rp[2] = {test_xy[2 * i] - xpc, test_xy[2 * i + 1] - ypc};
        for (int a = 0; a < 2; ++a) {
            double row[9] = {0};
            for (int c = 0; c < 3; ++c) { row[a * 3 + c] = zs * r[c]; row[6 + c] = -rp[a] * r[c]; }
            for (int p = 0; p < 9; ++p)
                for (int q = 0; q < 9; ++q) AtA[p * 9 + q] += row[p] * row[q];
        }
    }
    double w[9], V[81];
    jacobi_eig(AtA, 9, w, V);
    int m = 0;
    for (int i = 1; i < 9; ++i) if (w[i] < w[m]) m = i;
    for (int p = 0; p < 9; ++p) F[p] = V[p * 9 + m];
    if (fabs(F[8]) < 1e-300) return -1;
    double s33 = F[8];
    for (int p = 0; p < 9; ++p) F[p] /= s33;
    /* Gauss-Newton over the 8 entries other than F_33. */
    for (int it = 0; it < 100; ++it) {
        double JtJ[64], Jtr[8];
        memset(JtJ, 0, sizeof(JtJ)); memset(Jtr, 0, sizeof(Jtr));
        for (int i = 0; i < N; ++i) {
            double r[3] = {ref_xy[2 * i] - xpc, ref_xy[2 * i + 1] - ypc, zs};
            double v[3];
            for (int a = 0; a < 3; ++a) v[a] = F[a * 3] * r[0] + F[a * 3 + 1] * r[1] + F[a * 3 + 2] * r[2];
            double rp[2] = {test_xy[2 * i] - xpc, test_xy[2 * i + 1] - ypc};
            for (int a = 0; a < 2; ++a) {
                double pred = zs * v[a] / v[2];
                double res = pred - rp[a];
                double J9[9] = {0};
                for (int c = 0; c < 3; ++c) { J9[a * 3 + c] = zs * r[c] / v[2]; J9[6 + c] = -zs * v[a] * r[c] / (v[2] * v[2]); }
                double J[8];
                for (int p = 0; p < 8; ++p) J[p] = J9[p];
                for (int p = 0; p < 8; ++p) { Jtr[p] += J[p] * res; for (int q = 0; q < 8; ++q) JtJ[p * 8 + q] += J[p] * J[q]; }
            }
        }
        double step[8], nb[8];
        for (int p = 0; p < 8; ++p) nb[p] = -Jtr[p];
        if (chol_solve(JtJ, nb, 8, step)) return -1;
        double sn = 0.0, fn = 0.0;
        for (int p = 0; p < 8; ++p) { F[p] += step[p]; sn += step[p] * step[p]; fn += F[p] * F[p]; }
        if (sqrt(sn) <= 1e-14 * sqrt(fn + 1.0)) break;
    }
    double d = det3(F);
    if (d == 0.0) return -1;
    double sc = cbrt(d);
    for (int p = 0; p < 9; ++p) F[p] /= sc;
    return 0;
}

/* Rotation part of F (Eq. 4-5): F = P D Q^T, R = P Q^T.  The SVD is the
 * one-sided (Hestenes) Jacobi method: rotate column pairs of A = F until
 * orthogonal, A = F Q = P D. */
void oracle_polar(const double *F, double *R)
{
    double A[9], Q[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(A, F, sizeof(A));
    for (int sweep = 0; sweep < 60; ++sweep) {
        double offmax = 0.0;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double al = 0, be = 0, ga = 0;
                for (int k = 0; k < 3; ++k) { al += A[k * 3 + p] * A[k * 3 + p]; be += A[k * 3 + q] * A[k * 3 + q]; ga += A[k * 3 + p] * A[k * 3 + q]; }
                double rel = fabs(ga) / sqrt(al * be);
                if (rel > offmax) offmax = rel;
                if (ga == 0.0) continue;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int k = 0; k < 3; ++k) {
                    double x = A[k * 3 + p], y = A[k * 3 + q];
                    A[k * 3 + p] = c * x - s * y; A[k * 3 + q] = s * x + c * y;
                    x = Q[k * 3 + p]; y = Q[k * 3 + q];
                    Q[k * 3 + p] = c * x - s * y; Q[k * 3 + q] = s * x + c * y;
                }
            }
        if (offmax < 1e-15) break;
    }
    /* P = A D^-1 (columns normalised). */
    double P[9];
    for (int c = 0; c < 3; ++c) {
        double nrm = sqrt(A[c] * A[c] + A[3 + c] * A[3 + c] + A[6 + c] * A[6 + c]);
        for (int k = 0; k < 3; ++k) P[k * 3 + c] = A[k * 3 + c] / nrm;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i * 3 + j] = P[i * 3] * Q[j * 3] + P[i * 3 + 1] * Q[j * 3 + 1] + P[i * 3 + 2] * Q[j * 3 + 2];
}

/* a5: sample the finest-level field at the ROI centres (Section 2, the ROI
 * centres of the cross-correlation give the demons shifts; centre c in
 * continuous pixels is index coordinate c - 0.5), form r_i = c_i - u(c_i),
 * r'_i = c_i, fit F_first (Eq. 3) and R_finite = polar(F_first) (Eq. 4-5). */
int oracle_fit_rotation(const double *field, int H, int W, const double *roi_xy, int N, double xstar,
                        double ystar, double zstar, double *F_first, double *R_finite)
{
    double *rx = (double *)malloc(sizeof(double) * 2 * N), *tx = (double *)malloc(sizeof(double) * 2 * N);
    for (int i = 0; i < N; ++i) {
        double cx = roi_xy[2 * i], cy = roi_xy[2 * i + 1];
        double ux = oracle_bilinear(field, H, W, cx - 0.5, cy - 0.5);
        double uy = oracle_bilinear(field + (size_t)H * W, H, W, cx - 0.5, cy - 0.5);
        rx[2 * i] = cx - ux; rx[2 * i + 1] = cy - uy;
        tx[2 * i] = cx; tx[2 * i + 1] = cy;
    }
    int st = oracle_fit_F(rx, tx, N, xstar * W, ystar * H, zstar * W, F_first);
    free(rx); free(tx);
    if (st) return st;
    oracle_polar(F_first, R_finite);
    return 0;
}

/* ------------------------------------------------------------------ a6 */
/* Keys (1981) cubic convolution kernel, a = -0.5. */
static double keys(double s)
{
    const double a = -0.5;
    s = fabs(s);
    if (s <= 1.0) return (a + 2.0) * s * s * s - (a + 3.0) * s * s + 1.0;
    if (s < 2.0) return a * s * s * s - 5.0 * a * s * s + 8.0 * a * s - 4.0 * a;
    return 0.0;
}

/* Remap of the reference by R_finite (Section 2, remapping with a cubic
 * interpolation scheme; Eq. 12): output pixel x' looks up the reference at
 * the gnomonic projection of R^T r', r' = (x' - xpc, y' - ypc, Z*).
 * Bicubic Keys interpolation with replicated borders. */
void oracle_remap(const double *ref, int H, int W, const double *R, double xstar, double ystar, double zstar,
                  double *out)
{
    double xpc = xstar * W, ypc = ystar * H, zs = zstar * W;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double rp[3] = {j + 0.5 - xpc, i + 0.5 - ypc, zs};
            double v[3];
            for (int a = 0; a < 3; ++a) v[a] = R[0 * 3 + a] * rp[0] + R[1 * 3 + a] * rp[1] + R[2 * 3 + a] * rp[2];
            double x = xpc + zs * v[0] / v[2] - 0.5, y = ypc + zs * v[1] / v[2] - 0.5;
            int x0 = (int)floor(x), y0 = (int)floor(y);
            double fx = x - x0, fy = y - y0, acc = 0.0;
            for (int m = -1; m <= 2; ++m) {
                double wy = keys(fy - m), row = 0.0;
                int yy = clampi(y0 + m, 0, H - 1);
                for (int k = -1; k <= 2; ++k) row += keys(fx - k) * ref[yy * W + clampi(x0 + k, 0, W - 1)];
                acc += wy * row;
            }
            out[i * W + j] = acc;
        }
}

/* ------------------------------------------------------------------ a7 */
/* Textbook iterative radix-2 Cooley-Tukey FFT (n a power of two),
 * X_k = sum_j x_j exp(-+2 pi i jk/n); the inverse includes 1/n. */
void oracle_fft(double *re, double *im, int n, int inverse)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { double t = re[i]; re[i] = re[j]; re[j] = t; t = im[i]; im[i] = im[j]; im[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        double ang = 2.0 * M_PI / len * (inverse ? 1.0 : -1.0);
        for (int i = 0; i < n; i += len)
            for (int k = 0; k < len / 2; ++k) {
                double wr = cos(ang * k), wi = sin(ang * k);
                double ur = re[i + k], ui = im[i + k];
                double vr = re[i + k + len / 2] * wr - im[i + k + len / 2] * wi;
                double vi = re[i + k + len / 2] * wi + im[i + k + len / 2] * wr;
                re[i + k] = ur + vr; im[i + k] = ui + vi;
                re[i + k + len / 2] = ur - vr; im[i + k + len / 2] = ui - vi;
            }
    }
    if (inverse)
        for (int i = 0; i < n; ++i) { re[i] /= n; im[i] /= n; }
}

/* 2-D FFT of an S x S complex array: rows then columns. */
void oracle_fft2(double *re, double *im, int S, int inverse)
{
    double *cr = (double *)malloc(sizeof(double) * S), *ci = (double *)malloc(sizeof(double) * S);
    for (int i = 0; i < S; ++i) oracle_fft(re + (size_t)i * S, im + (size_t)i * S, S, inverse);
    for (int j = 0; j < S; ++j) {
        for (int i = 0; i < S; ++i) { cr[i] = re[i * S + j]; ci[i] = im[i * S + j]; }
        oracle_fft(cr, ci, S, inverse);
        for (int i = 0; i < S; ++i) { re[i * S + j] = cr[i]; im[i * S + j] = ci[i]; }
    }
    free(cr); free(ci);
}

/* Windowed ROI: zero mean over the ROI, then (window != 0) the symmetric
 * Hann window 0.5 (1 - cos(2 pi n/(S-1))) in both directions (Section 2).
 * Returns the norm of the windowed ROI. */
static double prep_roi(const double *img, int W, int x0, int y0, int S, int window, double *out)
{
    double s = 0.0;
    for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j) s += img[(size_t)(y0 + i) * W + x0 + j];
    double mean = s / ((double)S * S), nrm = 0.0;
    for (int i = 0; i < S; ++i) {
        double wy = window ? 0.5 * (1.0 - cos(2.0 * M_PI * i / (S - 1))) : 1.0;
        for (int j = 0; j < S; ++j) {
            double wx = window ? 0.5 * (1.0 - cos(2.0 * M_PI * j / (S - 1))) : 1.0;
            double v = (img[(size_t)(y0 + i) * W + x0 + j] - mean) * wy * wx;
            out[i * S + j] = v;
            nrm += v * v;
        }
    }
    return sqrt(nrm);
}

/* Cross-correlation surface of one ROI (Section 2): the inverse FFT of
 * FFT(test) times the conjugate of FFT(ref), i.e. c(s) = sum_x test(x + s)
 * ref(x) over the windowed ROIs, circular in s.  The ROI has top-left pixel
 * (x0, y0) and size S (a power of two).  c [S][S]; norms of the windowed
 * ROIs to nr, nt. */
void oracle_xcf_surface(const double *refimg, const double *testimg, int W, int x0, int y0, int S, int window,
                        double *c, double *nr, double *nt)
{
    size_t n = (size_t)S * S;
    double *ai = (double *)calloc(n, sizeof(double));
    double *br = (double *)malloc(sizeof(double) * n), *bi = (double *)calloc(n, sizeof(double));
    *nr = prep_roi(refimg, W, x0, y0, S, window, br);
    *nt = prep_roi(testimg, W, x0, y0, S, window, c);
    oracle_fft2(c, ai, S, 0);
    oracle_fft2(br, bi, S, 0);
    for (size_t p = 0; p < n; ++p) {   /* test * conj(ref) */
        double xr = c[p] * br[p] + ai[p] * bi[p];
        double xi = ai[p] * br[p] - c[p] * bi[p];
        c[p] = xr; ai[p] = xi;
    }
    oracle_fft2(c, ai, S, 1);
    free(ai); free(br); free(bi);
}

/* ROI shifts (Section 2).  Peak: first maximum of the correlation surface
 * in row-major order; the index is wrapped to [-S/2, S/2).  Sub-pixel
 * ("interpolating the XCF peak"; reading): 3-point parabola per axis on
 * circular neighbours, delta = (c- - c+)/(2(c- - 2c0 + c+)).  q = peak +
 * delta as (x, y).  Peak height c0 / (|ref_w| |test_w|).  near_tie flags ROIs
 * whose two largest values differ by less than 1e-6 |c0|.  roi_xy are integer
 * ROI centres; the ROI covers rows/columns [c - S/2, c + S/2). */
void oracle_xcf_roi(const double *refimg, const double *testimg, int H, int W, const int *roi_xy, int N, int S,
                    int window, double *q, int *peak, double *ph, int *near_tie)
{
    (void)H;
    size_t n = (size_t)S * S;
    double *ar = (double *)malloc(sizeof(double) * n);
    for (int r = 0; r < N; ++r) {
        int x0 = roi_xy[2 * r] - S / 2, y0 = roi_xy[2 * r + 1] - S / 2;
        double nr, nt;
        oracle_xcf_surface(refimg, testimg, W, x0, y0, S, window, ar, &nr, &nt);
        size_t best = 0;
        for (size_t p = 1; p < n; ++p) if (ar[p] > ar[best]) best = p;
        double c0 = ar[best], second = -INFINITY;
        for (size_t p = 0; p < n; ++p) if (p != best && ar[p] > second) second = ar[p];
        int py = (int)(best / S), px = (int)(best % S);
        double cxm = ar[py * S + (px + S - 1) % S], cxp = ar[py * S + (px + 1) % S];
        double cym = ar[((py + S - 1) % S) * S + px], cyp = ar[((py + 1) % S) * S + px];
        double dx = 0.0, dy = 0.0, den;
        den = cxm - 2.0 * c0 + cxp; if (den != 0.0) dx = (cxm - cxp) / (2.0 * den);
        den = cym - 2.0 * c0 + cyp; if (den != 0.0) dy = (cym - cyp) / (2.0 * den);
        int wx = px >= S / 2 ? px - S : px, wy = py >= S / 2 ? py - S : py;
        peak[2 * r] = wx; peak[2 * r + 1] = wy;
        q[2 * r] = wx + dx; q[2 * r + 1] = wy + dy;
        ph[r] = (nr > 0 && nt > 0) ? c0 / (nr * nt) : 0.0;
        near_tie[r] = (c0 - second) < 1e-6 * fabs(c0);
    }
    free(ar);
}

/* a8: second-pass deformation gradient (Section 2, Eq. 3 on the XCF shifts
 * between the remapped reference and the test; Eq. 12 F = F_inf R_finite).
 * r_i = c_i, r'_i = c_i + q_i.  R_finite nullable (then F = F_inf). */
int oracle_solve_F(const double *q, const double *roi_xy, int N, int H, int W, double xstar, double ystar,
                   double zstar, const double *R_finite, double *F)
{
    double *rx = (double *)malloc(sizeof(double) * 2 * N), *tx = (double *)malloc(sizeof(double) * 2 * N);
    for (int i = 0; i < N; ++i) {
        rx[2 * i] = roi_xy[2 * i]; rx[2 * i + 1] = roi_xy[2 * i + 1];
        tx[2 * i] = roi_xy[2 * i] + q[2 * i]; tx[2 * i + 1] = roi_xy[2 * i + 1] + q[2 * i + 1];
    }
    double Fi[9];
    int st = oracle_fit_F(rx, tx, N, xstar * W, ystar * H, zstar * W, Fi);
    free(rx); free(tx);
    if (st) return st;
    if (!R_finite) { memcpy(F, Fi, sizeof(Fi)); return 0; }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i * 3 + j] = Fi[i * 3] * R_finite[j] + Fi[i * 3 + 1] * R_finite[3 + j] + Fi[i * 3 + 2] * R_finite[6 + j];
    return 0;
}

/* ----------------------------------------------------------------- a12 */
/* Axis-angle of a rotation R (Section 2, text after Eq. 5): the angle is
 * acos((tr R - 1)/2) and the axis the eigenvector of eigenvalue one, taken
 * here from the antisymmetric part (R - R^T)/2 = sin(theta) [m]x (valid for
 * 0 < theta < pi; axis (0,0,0) when theta = 0).  Lattice rotation tensor of
 * Eq. 6-7: theta_k = m_k theta, omega = [[0,-t3,t2],[t3,0,-t1],[-t2,t1,0]]. */
void oracle_axis_angle(const double *R, double *m, double *theta, double *omega)
{
    double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    double th = acos(c), s = sin(th);
    double v[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]};
    for (int k = 0; k < 3; ++k) m[k] = s > 0.0 ? v[k] / (2.0 * s) : 0.0;
    *theta = th;
    double t1 = m[0] * th, t2 = m[1] * th, t3 = m[2] * th;
    double w[9] = {0.0, -t3, t2, t3, 0.0, -t1, -t2, t1, 0.0};
    memcpy(omega, w, sizeof(w));
}
