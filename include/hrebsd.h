/*
 * hrebsd.h -- C ABI of the GB300 (sm_103a) HR-EBSD demons-remapping library.
 *
 * The method is Zhu, Kaufmann & Vecchio, "Novel Remapping Approach for
 * HR-EBSD based on Demons Registration" (arXiv 1907.05993).  For every scan
 * point the test Kikuchi pattern is registered against its reference by
 * multi-resolution demons (Section 1, Eq. 1), the lattice rotation is fitted
 * to the displacement field at the ROI centres (Section 2, Eq. 2-5), the
 * reference is remapped by that rotation (Eq. 12), and a second-pass ROI
 * cross-correlation (Section 2) gives the shifts for the final deformation
 * gradient F = F_inf R_finite (Eq. 3, Eq. 12).
 *
 * Conventions shared by every call
 *   - All array arguments are DEVICE pointers (cudaMalloc / torch CUDA
 *     tensors) owned by the caller, unless a call says otherwise.  The
 *     library only allocates its own workspace inside the context.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  The caller synchronises before reading outputs.
 *   - Images are FP32 row-major [n][H][W].  Index coordinates put pixel
 *     centres on integers (x = column, y = row, rows downward); continuous
 *     detector coordinates put them at (column + 0.5, row + 0.5).
 *   - A displacement field is FP32 [B][2][H][W]: the x plane then the y
 *     plane, in pixels.  The reference pattern is the moving image M, the
 *     test pattern the fixed image; M warped by u is M(x - u(x)).
 *   - Geometry: pattern centre at (xstar*W, ystar*H) continuous pixels,
 *     detector distance Z* = zstar*W pixels, screen normal k = (0,0,1)
 *     (Eq. 2).  Points are lifted to r = (x - xpc, y - ypc, Z*).
 *   - 3x3 matrices are FP64 row-major [B][9].
 *   - ROI centres roi_xy are int32 [N][2] (x, y) in continuous pixels; a
 *     ROI of size S covers rows/columns [c - S/2, c + S/2).
 *   - Return value: HREBSD_OK or a negative HREBSD_E* code (argument checks
 *     happen before any launch; on a CUDA error the context stays usable
 *     unless the error is sticky).  Problems of single pairs never fail a
 *     call: they are reported as bits of pair_status[B].
 */
#ifndef HREBSD_H
#define HREBSD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HREBSD_OK 0
#define HREBSD_EINVAL -1   /* bad argument (null pointer, size, unsupported parameter) */
#define HREBSD_ECUDA -2    /* a CUDA runtime call or launch failed */
#define HREBSD_ENOMEM -3   /* workspace allocation failed */
#define HREBSD_ETIMEOUT -4 /* a bounded device-side wait expired */
#define HREBSD_ESCRATCH -5 /* request larger than the static scratch of hrebsd_demons_register_batch_noalloc */
#define HREBSD_EIO -6      /* a file could not be opened, read or written */
#define HREBSD_EFORMAT -7  /* a model file is not one this library wrote for this network */

/* pair_status bits */
#define HREBSD_PAIR_CAPPED 1      /* some pyramid level stopped at its iteration cap */
#define HREBSD_PAIR_NONFINITE 2   /* the field or an input contained NaN/Inf */
#define HREBSD_PAIR_FIT_FAILED 4  /* Eq. 3 fit degenerate (singular normal matrix) */

typedef struct hrebsd_ctx hrebsd_ctx;

/* Create a context on CUDA device `device` (made current for the calls of
 * this context).  *ctx receives the handle.  Errors: EINVAL (null ctx or
 * bad device), ECUDA. */
int hrebsd_create(hrebsd_ctx **ctx, int device);

/* Free the context and its workspace (synchronises the device first). */
int hrebsd_destroy(hrebsd_ctx *ctx);

/* Human-readable text of a status code (static storage, never NULL). */
const char *hrebsd_status_string(int status);

/* Kernel launches of this context since creation (for accounting). */
long long hrebsd_launch_count(const hrebsd_ctx *ctx);

/* Synchronise the device; HREBSD_ETIMEOUT if a kernel of this library gave
 * up a bounded wait on an asynchronous copy since the last call (the flag is
 * then cleared and the affected outputs are invalid), else HREBSD_OK. */
int hrebsd_device_error(hrebsd_ctx *ctx);

/* Context options.  HREBSD_OPT_NO_TMA (value 0/1): run the demons iteration
 * without tensor-memory-accelerator tile loads (same results; used to test
 * both paths; the environment variable HREBSD_NO_TMA sets it at creation). */
#define HREBSD_OPT_NO_TMA 1
/* HREBSD_OPT_GRAPHS (value 0/1, default 1; the environment variable
 * HREBSD_NO_GRAPHS clears it at creation): each pyramid level of a
 * registration (its list reset, cap x (iteration, stop control), finalize and
 * prolongation launches) is captured once into a CUDA graph on a private
 * stream and replayed on the caller's stream; the cache (32 graphs, least
 * recently used replaced) is keyed by every pointer, size and parameter of the
 * launches.  Not used while tracing is on, inside the allocation-free entry
 * point, or when the caller's stream is itself capturing (the launches then go
 * into the caller's graph).  Same results either way. */
#define HREBSD_OPT_GRAPHS 2
/* HREBSD_OPT_CNN_TC (value 0/1, default 1): run the 3x3 convolutions of the
 * learned initialiser on the fifth-generation tensor cores (input halo tiles
 * by TMA, tcgen05 MMAs into tensor memory): the forward pass, the weight
 * gradients, and the input gradients of every layer whose channel counts the
 * tcgen05 kernel takes (the others run the mma.sync kernel); 0 selects the
 * mma.sync kernels for all of them.
 * Same operands and FP32 accumulation; the sums are grouped differently, so
 * results agree to FP32 rounding before the BF16 store. */
#define HREBSD_OPT_CNN_TC 3
/* HREBSD_OPT_TEX_GATHER (value 0/1, default 1): the row-sweep demons
 * iteration (tile shapes 5 and 6) reads the four moving-image pixels of each
 * bilinear sample with one texture gather from a copy of the level's
 * reference images in a CUDA array held by the context (one array per level
 * width, grown when a call needs more rows; growing it synchronises the device
 * and drops the cached graphs); 0 selects plain global loads.  The same four
 * values enter the same arithmetic, so the results are identical.  Levels whose
 * R x h rows exceed the device's texture-gather height, and the
 * allocation-free entry point, use the plain loads. */
#define HREBSD_OPT_TEX_GATHER 4
int hrebsd_set_option(hrebsd_ctx *ctx, int option, int value);

/* Tracing: per kernel class, CUDA-event time of every launch (events are
 * recorded on the launch stream around each kernel while enabled).  Classes:
 * 0 demons iteration, 1 demons stop control, 2 demons pyramid/finalize/
 * prolongation, 3 preprocess, 4 rotation fit, 5 remap, 6 ROI XCF,
 * 7 deformation-gradient solve, 8 learned initialiser.  pixel_iters counts demons pixel-iterations
 * (active pairs x level pixels, summed over iteration launches). */
#define HREBSD_PROF_CLASSES 9
typedef struct {
    double ms[HREBSD_PROF_CLASSES];
    long long launches[HREBSD_PROF_CLASSES];
    long long pixel_iters;
} hrebsd_profile;

/* Enable (1) or disable (0) tracing; either call resets the counters. */
int hrebsd_profile_enable(hrebsd_ctx *ctx, int enable);

/* Synchronise the device and return the counters gathered since the last
 * reset.  Errors: EINVAL (null pointers), ECUDA. */
int hrebsd_profile_read(hrebsd_ctx *ctx, hrebsd_profile *out);

typedef struct {
    double xstar, ystar, zstar;
} hrebsd_geometry;

/* Demons parameters.  levels: pyramid levels (1..8; level 0 is the full
 * size, level l is (H >> l) x (W >> l), i.e. each level floor(h/2) x
 * floor(w/2) of the one above (an odd last row or column takes no part in
 * the 2x2 box mean, and the prolongation fills the finer level's stored
 * size); the coarsest must stay >= 8 x 8).  max_iters[l]: iteration cap of level l
 * (0..4096).  alpha: force weight of Eq. 1 (du = d grad F / (|grad F|^2 +
 * alpha^2 d^2)).  sigma_update, sigma_field: Gaussian smoothing of the update
 * and of the field (radius ceil(3 sigma) <= 6; 0 = none).  stop_window w and
 * stop_tol: a level stops at iteration k >= w when E_{k-w} - E_k <
 * stop_tol * E_{k-w} (E = SSD); w = 0 runs every level to its cap.
 * start_level: first (coarsest) level to run, -1 = levels - 1. */
typedef struct {
    int levels;
    int max_iters[8];
    float alpha;
    float sigma_update;
    float sigma_field;
    float stop_tol;
    int stop_window;
    int start_level;
} hrebsd_demons_params;

/* The Gaussian of the field regularisation (Section 1; the workloads smooth
 * the update and the field with it): radius r = ceil(3 sigma) (at most 6),
 * taps[0 .. 2r] = exp(-k^2 / 2 sigma^2) normalised, k = -r .. r, in FP32.  The
 * FP32 taps are chosen so that their exact sum is one (the rounded weights
 * alone would leave it a few 1e-8 short, a systematic shrink of the field by
 * that much at every smoothing pass); the smallest outer tap may differ from
 * its rounded weight by a few units in the last place.  Host only, no GPU.
 * Returns r (taps[0 .. 2r] written) or HREBSD_EINVAL (null taps, r > 6). */
int hrebsd_gauss_taps(float sigma, float *taps);

/* a1 -- intensity normalisation (Section 2) with static background
 * correction (Section 3.3): for each of the n patterns in [n][H][W], if
 * `flat` the least-squares quadric c0 + c1 x + c2 y + c3 x^2 + c4 xy + c5 y^2
 * (x, y in [-1, 1] at pixel centres) is divided out, then the pattern is
 * brought to zero mean and unit standard deviation (a constant pattern
 * becomes all zeros).  The quadric and the quotient are evaluated in
 * double-FP32 precision (hi + lo), so the FP32 output is within a few units
 * in the last place of the exact result.  in and out may alias.  Errors:
 * EINVAL (n < 0, H or W < 2, H or W > 1536 with `flat`, null pointers with
 * n > 0). */
int hrebsd_preprocess_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, int flat, float *out,
                            void *stream);

/* Box mean of f x f blocks, [n][H][W] -> [n][H/f][W/f] FP32 (equal to the
 * pyramid level log2(f) of the registration up to rounding order; used for the
 * inputs and targets of the learned initialiser).  H, W divisible by f. */
int hrebsd_downsample_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, int f, float *out, void *stream);

/* Displacement field between pyramid resolutions (learned initialiser):
 * planar [B][2][h][w] FP32 -> [B][2][h2][w2], values converted to the new pixel
 * unit.  h2 = h / f (box mean of f x f blocks, divided by f) or h2 = h * f
 * (bilinear sample at x_c = (x_f + 0.5) / f - 0.5, clamped, times f; for f = 2
 * the prolongation between registration levels, Section 1), f a power of two,
 * the same for both axes.  EINVAL for other ratios or null pointers. */
int hrebsd_field_resample(hrebsd_ctx *ctx, const float *in, int B, int h, int w, float *out, int h2, int w2,
                          void *stream);

/* a2-a4, a9 -- multi-resolution demons registration of B pairs (Section 1,
 * Eq. 1).  ref [R][H][W] and test [B][H][W] must be preprocessed
 * (hrebsd_preprocess_batch).  Pair b registers ref[ref_idx[b]] (moving) onto
 * test[b] (fixed).  Per level, from params->start_level down to 0: the
 * pyramid images are 2x2 box means; the field starts at zero on the first
 * level (or at init_field [B][2][H>>s][W>>s], s the start level, if not
 * NULL) and at twice the bilinear prolongation of the coarser result
 * otherwise; each iteration warps M by u (bilinear, clamped), forms the
 * force from the gradient of the test image (central differences, one-sided
 * at borders; du = 0 where the denominator <= 1e-9), smooths du, adds it,
 * smooths u (separable Gaussians, x pass then y pass, replicated borders).
 * Pairs stop independently (stop rule above); the batch runs until every
 * pair has stopped.  Outputs: field [B][2][H][W] (finest level), iters
 * [B][levels] (updates applied per level, 0 for skipped levels),
 * pair_status [B] (CAPPED, NONFINITE bits set; other bits cleared).
 * Errors: EINVAL, ENOMEM, ECUDA. */
int hrebsd_demons_register_batch(hrebsd_ctx *ctx, const float *ref, const float *test, const int32_t *ref_idx,
                                 int R, int B, int H, int W, const hrebsd_demons_params *params,
                                 const float *init_field, float *field, int32_t *iters, int32_t *pair_status,
                                 void *stream);

/* Allocation-free variant of hrebsd_demons_register_batch (the paper has no
 * counterpart).  It exists for callers that cannot allocate device memory:
 * hosts that fix the device-memory budget before they start, plugins whose
 * host application owns the allocator, and latency-bound services that may not
 * allocate (a cudaMalloc can synchronise the device) while serving a request.
 * Same arguments, outputs and results as hrebsd_demons_register_batch, but
 * the workspace is a static device array of HREBSD_NOALLOC_SCRATCH_BYTES
 * (16 MiB) inside this library, held by every process that loads it on each
 * device it uses, until exit; the call never calls cudaMalloc/cudaFree or any
 * allocating routine.  The first call on a device looks the array's device
 * address up (cudaGetSymbolAddress) with that device current: make that first
 * call before any stream capture.  The whole batch must fit: about
 * 8 B x 3 x H x W + 8 B x H x W / 4 + 4 B x H x W / 3 per pair plus small
 * per-pair lists (about 9 pairs of 256 x 256 with 4 levels, or 37 pairs of
 * 128 x 128 with 3 levels);
 * larger requests return HREBSD_ESCRATCH before any launch.  All calls share
 * the array and it keeps the last call's contents (every slot is written
 * before it is read), so calls that overlap on the GPU race: serialise them.
 * Tracing (hrebsd_profile_*) does not record this call. */
#define HREBSD_NOALLOC_SCRATCH_BYTES (16u << 20)
int hrebsd_demons_register_batch_noalloc(hrebsd_ctx *ctx, const float *ref, const float *test,
                                         const int32_t *ref_idx, int R, int B, int H, int W,
                                         const hrebsd_demons_params *params, const float *init_field, float *field,
                                         int32_t *iters, int32_t *pair_status, void *stream);

/* Tile shapes of the demons iteration (batching; the paper has no
 * counterpart): 0 = 64x32 outputs, 256 threads (2 CTAs per SM), 1 = 32x32
 * (3 per SM), 2 = 64x16 (3 per SM), 3 = 64x32 with 512 threads (2 per SM),
 * 4 = 64x64 with 768 threads (1 per SM; of 512, 768, 896 and 1024 threads
 * the fastest on GB300), all fed by tensor-memory-accelerator tile copies;
 * 5 = the row sweep: one CTA of w threads per pair walks down whole rows of
 * the level with the separable y passes in per-column register windows (no
 * halo rows; levels 64, 128 or 256 pixels wide; other levels fall back to
 * shape 4); 6 = the row sweep with every iteration after the first of a
 * level in one launch, each pair iterating in its CTA until the stop rule
 * (applied in the CTA, the same rule on the same history) ends it, so a level
 * costs 5 launches instead of two per iteration (levels with a cap of one
 * iteration run as shape 5); shape 5 itself takes this form when the batch has
 * no more pairs than the level has resident CTAs (one pair per CTA: nobody
 * waits), and per-iteration launches otherwise (they re-balance the uneven
 * iteration counts of the pairs after every iteration).  A level without a
 * set or tuned shape runs shape 5 where it applies and shape 0 elsewhere.
 * 7 = the whole level in shared memory (levels of at most 64 x 64 pixels):
 * one CTA of 512 threads per pair holds the field, iterates, applies the stop
 * rule and writes the level's final field, one launch per level (other
 * levels run shape 5).  Shapes 1-6 exist for the Gaussian radius 3
 * (sigma = 1); other radii always use shape 0.  Every shape computes each
 * output pixel with the same operations in the same order, so the field is
 * the same; only the grouping of the per-tile SSD partials changes (shapes 5
 * and 6 share theirs: same counts, same field). */
#define HREBSD_TILE_VARIANTS 8

/* Autotuner: for each pyramid level of an H x W registration with `params`,
 * time every tile shape on synthetic striped patterns displaced by a small
 * rotation field (min(B, 2048) pairs; 2 warm-up iterations, then the best of
 * 3 timed batches of 4, CUDA events on `stream`; shapes 6 and 7: one warm-up
 * launch, then the best of 3 launches of 7 (shape 6) or 8 (shape 7)
 * iterations; shape 6 is reported but never chosen,
 * since the synthetic pairs all run the same number of iterations) and keep, for later
 * registrations of that level size in this context, the shape with the least
 * time x (1 + 0.01 log2(4096 / tile area)): smaller tiles carry a 1 % handicap
 * per halving of the area, because the synthetic timing showed a tie where
 * the 64x64 shape was 4 % faster on scan data; shapes 0-6 count 0.005 ms more
 * per iteration for the stop-control launch that follows each of their
 * iterations (shape 7 applies the stop rule in its CTAs), which the timing
 * leaves out.  Synchronises `stream`; uses context
 * workspace.  ms_out (host, nullable): [levels][HREBSD_TILE_VARIANTS]
 * milliseconds per iteration, NaN where a shape is unavailable.  Returns
 * HREBSD_EINVAL for invalid parameters (as hrebsd_demons_register_batch). */
int hrebsd_autotune(hrebsd_ctx *ctx, int B, int H, int W, const hrebsd_demons_params *params, float *ms_out,
                    void *stream);
/* Set (variant 0..HREBSD_TILE_VARIANTS-1) or clear (-1) the tile shape used
 * for levels of size h x w; get returns the current choice (0 if none was set
 * or tuned: the level then runs the default above). */
int hrebsd_set_tile_variant(hrebsd_ctx *ctx, int h, int w, int variant);
int hrebsd_get_tile_variant(const hrebsd_ctx *ctx, int h, int w);

/* a5 -- rotation fit (Section 2, Eq. 2-5).  The field [B][2][H][W] is
 * sampled bilinearly at the N ROI centres c (index coordinates c - 0.5);
 * with reference points r_i = c_i - u(c_i) and test points r'_i = c_i the
 * Eq. 3 least-squares problem is solved in FP64 (linear start with
 * F_33 = 1, Gauss-Newton, then det F = 1), and R_finite is the polar factor
 * of F (Eq. 4-5, Newton polar iteration).  Outputs F_first, R_finite
 * [B][9]; pair_status |= FIT_FAILED on a singular fit (then F_first =
 * R_finite = I).  N >= 4.  pair_status may be NULL. */
int hrebsd_fit_rotation(hrebsd_ctx *ctx, const float *field, int B, int H, int W, const int32_t *roi_xy, int N,
                        const hrebsd_geometry *geom, double *F_first, double *R_finite, int32_t *pair_status,
                        void *stream);

/* a6 -- remap of the reference by R_finite (Section 2, Eq. 12 with cubic
 * interpolation): remapped[b](x') = ref[ref_idx[b]] at the gnomonic
 * projection of R_finite[b]^T r', Keys cubic convolution (a = -0.5),
 * replicated borders.  remapped [B][H][W]. */
int hrebsd_remap(hrebsd_ctx *ctx, const float *ref, const int32_t *ref_idx, const double *R_finite, int B, int H,
                 int W, const hrebsd_geometry *geom, float *remapped, void *stream);

/* a7 -- second-pass ROI cross-correlation (Section 2).  For each pair and
 * ROI: zero mean over the ROI, symmetric Hann window if `window`
 * (0.5 (1 - cos(2 pi n/(S-1)))), c = IFFT(FFT(test) conj(FFT(ref))), i.e.
 * c(s) = sum_x test(x+s) ref(x); integer peak = first maximum in row-major
 * order, wrapped to [-S/2, S/2); sub-pixel 3-point parabola per axis.
 * S in {16, 32, 64, 128}; ROIs must lie inside the image.  Outputs
 * q [B][N][2] (x, y shift: test(x + q) ~ ref(x)), peak [B][N][2],
 * peak_height [B][N] (c0 / (|ref_w| |test_w|)), near_tie [B][N] (top two
 * correlation values within 1e-6 |c0|; may be NULL). */
int hrebsd_xcf_roi_batch(hrebsd_ctx *ctx, const float *remapped, const float *test, int B, int H, int W,
                         const int32_t *roi_xy, int N, int S, int window, float *q, int32_t *peak,
                         float *peak_height, int32_t *near_tie, void *stream);

/* a8 -- second-pass deformation gradient (Eq. 3 on the XCF shifts, Eq. 12):
 * r_i = c_i, r'_i = c_i + q_i, F_inf by the same FP64 fit as
 * hrebsd_fit_rotation, F = F_inf R_finite (R_finite may be NULL: F = F_inf).
 * Eq. 3 fixes F only up to a scale (F and lambda F project every point to the
 * same place); `normalization` picks it:
 *   HREBSD_NORM_DET1: det F = 1 (elastic is ignored and may be NULL);
 *   HREBSD_NORM_TRACTION_FREE: the traction-free condition of Section 2
 *     (Eq. 16 with sigma_33 = 0 at the free surface): F = lambda F_det1 with
 *     lambda > 0 such that the stress C_S : 1/2 (F_S F_S^T - I) of
 *     F_S = T F T^T (the tilt of Eq. 13-14) has a zero 33 component, C_S the
 *     cubic stiffness (elastic->c11, c12, c44) rotated to the sample frame by
 *     elastic->g[ref_idx[b]] as in hrebsd_strain_stress.  A pair whose
 *     condition has no positive solution, or whose ref_idx is outside [0, R),
 *     gets F = NaN and FIT_FAILED.
 * F [B][9]; pair_status |= FIT_FAILED on a singular fit (may be NULL).
 * Errors: EINVAL (sizes, null pointers, unknown normalization, missing elastic
 * data for TRACTION_FREE). */
#define HREBSD_NORM_DET1 0
#define HREBSD_NORM_TRACTION_FREE 1
typedef struct {
    double tilt_rad;          /* sample tilt theta of Eq. 13 */
    double c11, c12, c44;     /* cubic stiffness in crystal axes, Pa (nickel: 276e9, 159e9, 132e9) */
    const double *g;          /* device [R][9]: passive orientation matrix (sample -> crystal) per reference */
    const int32_t *ref_idx;   /* device [B], nullable: every pair uses g[0] */
    int R;
} hrebsd_elastic;
int hrebsd_solve_F(hrebsd_ctx *ctx, const float *q, const int32_t *roi_xy, int N, int B, int H, int W,
                   const hrebsd_geometry *geom, const double *R_finite, int normalization,
                   const hrebsd_elastic *elastic, double *F, int32_t *pair_status, void *stream);

/* f2 -- pattern preprocessing for real scans (Section 3.2-3.3).  The paper
 * names the steps without kernels; the readings (FP32, replicated borders):
 * Gaussian filters of radius ceil(3 sigma) (at most 96, i.e. sigma <= 32) with
 * weights exp(-k^2 / 2 sigma^2) normalised to one, x pass then y pass.
 * Arrays [n][H][W] FP32 on the device; in and out may alias except for
 * hrebsd_shift_zoom_batch.  EINVAL for bad sizes, sigmas or pointers.
 *
 * hrebsd_bandpass_batch: out = LP(in) - G_hp * in, LP(in) = G_lp * in
 * (sigma_lp = 0: LP = identity; sigma_hp = 0: no high-pass term), the
 * low-pass / high-pass pair applied before the demons registration.
 * hrebsd_mean_pattern: out [H][W] = mean of the n patterns (the static
 * background of a scan).
 * hrebsd_background_batch: static correction out = in / static_bg (nullable,
 * [H][W]) then dynamic correction out = out / (G_dyn * out) (sigma_dyn = 0:
 * none); a divisor below 1e-12 in magnitude gives 0.
 * hrebsd_shift_zoom_batch: out(x) = in(pc + (x - pc - t) / s) in index
 * coordinates, pc = (xstar W - 0.5, ystar H - 0.5), t = shift[b] (pixels,
 * nullable: 0), s = zoom[b] (nullable: 1), Keys cubic (a = -0.5): the pattern
 * shift correction (beam-position shift moved to the detector frame) and the
 * zoom/shrink by the ratio of detector distances. */
int hrebsd_bandpass_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, float sigma_lp, float sigma_hp,
                          float *out, void *stream);
int hrebsd_mean_pattern(hrebsd_ctx *ctx, const float *in, int n, int H, int W, float *out, void *stream);
int hrebsd_background_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, const float *static_bg,
                            float sigma_dyn, float *out, void *stream);
int hrebsd_shift_zoom_batch(hrebsd_ctx *ctx, const float *in, int n, int H, int W, const float *shift,
                            const float *zoom, const hrebsd_geometry *g, float *out, void *stream);

/* f3 -- comparison methods and quality measures (Section 3.1, Fig. 2-3).
 * The four rotation measurements of Fig. 2 compose the calls above:
 * (a) hrebsd_xcf_roi_batch on the un-remapped reference + hrebsd_solve_F with
 * R_finite = NULL; (b) F_first of hrebsd_fit_rotation; (c) (a), then
 * hrebsd_polar_batch, hrebsd_remap by that rotation, hrebsd_xcf_roi_batch,
 * hrebsd_solve_F; (d) the method of the paper (a1-a8).
 *
 * hrebsd_polar_batch: R [B][9] = rotation part of each F [B][9] (Eq. 4-5).
 *
 * hrebsd_fit_quality: per pair, MAE = the mean over the N ROIs of the angle
 * (rad) between the measured test direction (r' - PC, Z*) and the direction
 * F_m (r - PC, Z*) predicted by the fitted model, F_m = F R^T when R is given
 * (a second-pass F of Eq. 12 with its R_finite), else F.  Point pairs from XCF
 * shifts q [B][N][2] (r = c, r' = c + q) or from a demons field [B][2][H][W]
 * (r = c - u(c), r' = c); exactly one of q and field is non-null.  ph [B][N]
 * (nullable) gives ph_mean [B] = mean peak height (PH of Fig. 3).  Outputs
 * mae [B], ph_mean [B] (nullable) FP64.  EINVAL for bad arguments. */
int hrebsd_polar_batch(hrebsd_ctx *ctx, const double *F, int B, double *R, void *stream);
int hrebsd_fit_quality(hrebsd_ctx *ctx, const double *F, const double *R, const float *q, const float *field,
                       const float *ph, int B, int H, int W, const int32_t *roi_xy, int N, const hrebsd_geometry *g,
                       double *mae, double *ph_mean, void *stream);

/* SSIM of Fig. 3 (the quality measure of the demons-only method): mean SSIM
 * between the warped reference M(x - u(x)) (ref[ref_idx[b]], clamped bilinear as
 * in the registration; field NULL = no warp) and test[b], 11 x 11 Gaussian
 * window of sigma 1.5, C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = max - min of the
 * test pattern, over the window centres whose window lies inside the image.
 * ref [R][H][W], test [B][H][W], field [B][2][H][W]; ref_idx may be NULL
 * (all pairs use ref[0]).  Output ssim [B] FP64.  H, W >= 11. */
int hrebsd_ssim_warped(hrebsd_ctx *ctx, const float *ref, const int32_t *ref_idx, const float *test,
                       const float *field, int B, int H, int W, double *ssim, void *stream);

/* Check of the fifth-generation tensor-core building blocks the library uses
 * (no counterpart in the paper; a test hook): D[128][N] = A[128][16 KS] x
 * B[N][16 KS]^T with BF16 A, B (row-major, device) and FP32 D, computed by
 * tcgen05 MMAs from shared-memory descriptors into tensor memory.  N in
 * {16, 32, 64}, KS in 1..4.  One CTA on `stream`; a bounded wait that gives up
 * sets the flag read by hrebsd_device_error (D is then not written). */
int hrebsd_tc_selftest(hrebsd_ctx *ctx, const uint16_t *A, const uint16_t *B, int N, int KS, float *D, void *stream);

/* Failure-path self-test (no counterpart in the paper): one CTA on `stream`
 * waits on an mbarrier that nothing completes, with the try-wait loop of the
 * library's kernels limited to `max_polls` polls (1 .. 2^22); when the limit
 * runs out it sets the flag that hrebsd_device_error reports as
 * HREBSD_ETIMEOUT, and returns.  The context stays usable.  EINVAL for a
 * limit outside the range. */
int hrebsd_wait_selftest(hrebsd_ctx *ctx, unsigned max_polls, void *stream);

/* Measurement helper (no counterpart in the paper): launch an FP32 FMA
 * throughput probe on `stream` (SMs x 8 CTAs of 256 threads, each thread 8
 * independent chains of packed FP32x2 FMAs, `iters` steps); *flops receives the
 * floating-point operations of the launch, to be divided by its event time.
 * The denominator of the ALU roofline of the ROI cross-correlation. */
int hrebsd_probe_fp32_fma(hrebsd_ctx *ctx, int iters, double *flops, void *stream);

/* f1 -- strain and stress of each pair (Eq. 13-16; Supplementary Part 2).
 * F [B][9]: detector-frame deformation gradients (e.g. from hrebsd_solve_F).
 * F_S = T F T^T with the tilt rotation T = [[c, s, 0], [-s, c, 0], [0, 0, 1]]
 * of Eq. 13 (c, s of tilt_rad), Eq. 14.  With traction_free the scale of F_S
 * (undetermined by Eq. 3) is set so that sigma_33 = 0.  Strain
 * eps = 1/2 (F_S F_S^T - I) (Eq. 15, exact for the finite rotation of the
 * remapping); stress sigma = C_S : eps (Eq. 16), C_S the cubic stiffness
 * (c11, c12, c44 in Pa; nickel 276e9, 159e9, 132e9) rotated to the sample frame
 * by the passive orientation matrix g[ref_idx[b]] (sample -> crystal, [R][9]).
 * ref_idx may be NULL (all pairs use g[0]); an index outside [0, R) gives NaN
 * outputs.  Outputs [B][9]: F_S (may be NULL), eps, sigma (Pa). */
int hrebsd_strain_stress(hrebsd_ctx *ctx, const double *F, const int32_t *ref_idx, const double *g, int R, int B,
                         double tilt_rad, double c11, double c12, double c44, int traction_free, double *F_S,
                         double *eps, double *sigma, void *stream);

/* a10 -- learned initialiser of the coarse field (project addition; the paper
 * has none: its future-work remark is to optimise the multi-resolution
 * demons).  A 4-level U-Net (3x3 convolutions 16-32-64-128, 2x2 max-pool,
 * nearest x2 up-sampling, skip concatenations, 1x1 head, ReLU after every 3x3
 * convolution) maps the 64x64 (reference, test) pair to the field at the 64x64
 * pyramid level (x plane, y plane, 64x64-level pixels), to be passed as
 * init_field of hrebsd_demons_register_batch with start_level = log2(H/64).
 * BF16 tensor-core convolutions, FP32 accumulation and FP32 master weights.
 * Parameter vector (host FP32, hrebsd_cnn_num_params entries): per 3x3 layer
 * in the order e1a e1b e2a e2b e3a e3b ba bb d3a d3b d2a d2b d1a d1b the
 * weights [cout][ky*3+kx][cin padded to 16] then the bias [cout]; then the head
 * weights [2][16] and bias [2].  The network lives in the context (allocated
 * on first use). */
long long hrebsd_cnn_num_params(hrebsd_ctx *ctx);
/* Set the parameters (params_host may be NULL: keep) and reset Adam. */
int hrebsd_cnn_init(hrebsd_ctx *ctx, const float *params_host, long long n_params);
/* Copy parameters and the gradients of the last training step to the host (either may be NULL). */
int hrebsd_cnn_get_params(hrebsd_ctx *ctx, float *params_host, float *grads_host);
/* Training checkpoint: the Adam moments (host FP32, hrebsd_cnn_num_params
 * entries each; get: either may be NULL) and the step count that sets the
 * bias corrections.  set after hrebsd_cnn_init(params) resumes training
 * exactly where get left it.  Both synchronise the device.  EINVAL: no
 * network (get), a NULL moment or a negative step (set). */
int hrebsd_cnn_get_state(hrebsd_ctx *ctx, float *m_host, float *v_host, int *step);
int hrebsd_cnn_set_state(hrebsd_ctx *ctx, const float *m_host, const float *v_host, int step);
/* Model file (weights, Adam moments and step; the paper has no learned part,
 * so the format is this library's own: magic "HRCNN001", int64 parameter
 * count, int64 step, FP32 parameters, first and second moments, and an FNV-1a
 * hash of all preceding bytes; little-endian).  hrebsd_cnn_save synchronises
 * the device and writes the network of the context (EINVAL if it has none) to
 * `path` through a temporary file renamed into place (an interrupted save
 * leaves an earlier file intact).  hrebsd_cnn_load replaces the context's
 * network state by the file's, so that training continues exactly where the
 * saved context stood.  Errors: EIO (open/read/write/rename failed), EFORMAT
 * (wrong magic, parameter count, size or hash: nothing is loaded). */
int hrebsd_cnn_save(hrebsd_ctx *ctx, const char *path);
int hrebsd_cnn_load(hrebsd_ctx *ctx, const char *path);
/* Inference on x [B][2][64][64] BF16 (channel 0 reference, 1 test) -> field64 [B][2][64][64] FP32. */
int hrebsd_cnn_infer(hrebsd_ctx *ctx, const uint16_t *x_bf16, int B, float *field64, void *stream);
/* Inference from preprocessed patterns (as for the registration): the input is
 * the (H/64 x W/64)-block mean of ref[ref_idx[b]] and test[b]; H = W, a multiple of 64. */
int hrebsd_cnn_infer_patterns(hrebsd_ctx *ctx, const float *ref, const float *test, const int32_t *ref_idx, int B,
                              int H, int W, float *field64, void *stream);
/* One training step: forward, MSE loss against target [B][2][64][64] FP32 (its
 * value to *loss_out, a device float, may be NULL), backward, and one Adam
 * update (beta 0.9 / 0.999, eps 1e-8) with step size lr (lr = 0: gradients only). */
int hrebsd_cnn_train_step(hrebsd_ctx *ctx, const uint16_t *x_bf16, const float *target, int B, float lr,
                          float *loss_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HREBSD_H */
