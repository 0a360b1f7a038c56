// Context, workspace and status handling of the HR-EBSD library.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "internal.cuh"

int hr_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    if (getenv("HREBSD_VERBOSE"))
        fprintf(stderr, "hrebsd: %s failed at %s:%d: %s\n", what, file, line, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HREBSD_ENOMEM : HREBSD_ECUDA;
}

int hr_set_device(hrebsd_ctx *ctx)
{
    int cur = -1;
    HR_CHECK(cudaGetDevice(&cur));
    if (cur != ctx->device) HR_CHECK(cudaSetDevice(ctx->device));
    return HREBSD_OK;
}

int hr_ws(hrebsd_ctx *ctx, int slot, size_t bytes, void **out)
{
    if (slot < 0 || slot >= (int)(sizeof(ctx->ws) / sizeof(ctx->ws[0]))) return HREBSD_EINVAL;
    hr_buf &b = ctx->ws[slot];
    if (b.bytes < bytes) {
        if (b.ptr) {
            HR_CHECK(cudaDeviceSynchronize());
            HR_CHECK(cudaFree(b.ptr));
            b.ptr = nullptr;
            b.bytes = 0;
        }
        size_t want = bytes + bytes / 8;   // headroom against repeated small growth
        cudaError_t e = cudaMalloc(&b.ptr, want);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            b.ptr = nullptr;
            return HREBSD_ENOMEM;
        }
        b.bytes = want;
    }
    *out = b.ptr;
    return HREBSD_OK;
}

int hr_gauss_radius(float sigma)
{
    if (!(sigma > 0.0f)) return 0;
    int r = (int)ceil(3.0 * (double)sigma);
    return r;
}

// FP32 taps whose exact sum is one.  Rounding each normalised weight to FP32
// on its own leaves the sum off by a few 1e-8 (1 - 2.8e-8 at sigma = 1); the
// field smoothing applies the taps twice per iteration, so a registration of
// a few hundred iterations would scale the whole field by ~1e-5 (a systematic
// shrink).  Instead the outer taps are rounded to multiples of one quantum q
// (the unit in the last place of the largest outer tap, or half that of the
// centre tap if coarser: every such multiple is an FP32 value), so that the
// centre tap 1 - 2 sum_{k>0} t_k is exactly representable and the taps sum
// to one exactly.  The outer taps stay within half a quantum (at most half a
// unit in the last place of the centre tap) of their normalised weights; the
// centre tap takes up the sum of their rounding errors.
int hr_gauss_taps(float sigma, int rad, float *taps)
{
    int r = hr_gauss_radius(sigma);
    if (r > 6 || r > rad) return -1;
    for (int k = 0; k <= 2 * rad; ++k) taps[k] = 0.0f;
    if (r == 0) {
        taps[rad] = 1.0f;
        return 0;
    }
    double w[7], s = 0.0;
    for (int k = -r; k <= r; ++k) s += exp(-(double)(k * k) / (2.0 * (double)sigma * (double)sigma));
    for (int k = 0; k <= r; ++k) w[k] = exp(-(double)(k * k) / (2.0 * (double)sigma * (double)sigma)) / s;
    auto ulp = [](double v) {
        const float f = (float)v;
        return (double)nextafterf(f, 2.0f * f + 1.0f) - (double)f;
    };
    double q = fmax(ulp(w[1]), 0.5 * ulp(w[0]));
    float t[7];
    for (int attempt = 0; attempt < 8; ++attempt, q *= 2.0) {
        double S = 0.0;   // exact: every term is a multiple of q below 1
        for (int k = 1; k <= r; ++k) {
            t[k] = (float)(q * nearbyint(w[k] / q));
            S += (double)t[k];
        }
        const double c = 1.0 - 2.0 * S;
        t[0] = (float)c;
        if ((double)t[0] == c) break;
    }
    for (int k = -r; k <= r; ++k) taps[rad + k] = t[k < 0 ? -k : k];
    return r;
}

extern "C" int hrebsd_gauss_taps(float sigma, float *taps)
{
    if (!taps) return HREBSD_EINVAL;
    const int r = hr_gauss_radius(sigma);
    if (r > 6) return HREBSD_EINVAL;
    return hr_gauss_taps(sigma, r, taps) < 0 ? HREBSD_EINVAL : r;
}

// Set by kernels whose bounded wait on an asynchronous copy gave up.
__device__ int hr_device_error_flag;

static cudaEvent_t pool_get(hrebsd_ctx *ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void hr_prof_begin(hrebsd_ctx *ctx, cudaStream_t st)
{
    if (!ctx->prof_on || ctx->no_events) return;
    ctx->cur_a = pool_get(ctx);
    if (ctx->cur_a) cudaEventRecord(ctx->cur_a, st);
}

void hr_prof_end(hrebsd_ctx *ctx, int cls, cudaStream_t st)
{
    if (!ctx->prof_on || ctx->no_events || !ctx->cur_a) return;
    cudaEvent_t b = pool_get(ctx);
    if (!b) return;
    cudaEventRecord(b, st);
    ctx->pending.push_back({cls, ctx->cur_a, b});
    ctx->cur_a = nullptr;
    // fold completed pairs now and then so that the pending list stays short
    if (ctx->pending.size() > 4096) {
        std::vector<hr_pending> keep;
        for (auto &p : ctx->pending) {
            float ms = 0.0f;
            if (cudaEventQuery(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
                ctx->prof_ms[p.cls] += ms;
                ctx->prof_launches[p.cls]++;
                ctx->pool.push_back(p.a);
                ctx->pool.push_back(p.b);
            } else {
                keep.push_back(p);
            }
        }
        (void)cudaGetLastError();
        ctx->pending.swap(keep);
    }
}

extern "C" {

int hrebsd_profile_enable(hrebsd_ctx *ctx, int enable)
{
    if (!ctx) return HREBSD_EINVAL;
    int st = hr_set_device(ctx);
    if (st) return st;
    HR_CHECK(cudaDeviceSynchronize());
    for (auto &p : ctx->pending) {
        ctx->pool.push_back(p.a);
        ctx->pool.push_back(p.b);
    }
    ctx->pending.clear();
    for (int i = 0; i < HREBSD_PROF_CLASSES; ++i) {
        ctx->prof_ms[i] = 0.0;
        ctx->prof_launches[i] = 0;
    }
    if (!ctx->d_pixiters) HR_CHECK(cudaMalloc(&ctx->d_pixiters, sizeof(unsigned long long)));
    HR_CHECK(cudaMemset(ctx->d_pixiters, 0, sizeof(unsigned long long)));
    ctx->prof_on = enable ? 1 : 0;
    return HREBSD_OK;
}

int hrebsd_profile_read(hrebsd_ctx *ctx, hrebsd_profile *out)
{
    if (!ctx || !out) return HREBSD_EINVAL;
    int st = hr_set_device(ctx);
    if (st) return st;
    HR_CHECK(cudaDeviceSynchronize());
    for (auto &p : ctx->pending) {
        float ms = 0.0f;
        HR_CHECK(cudaEventElapsedTime(&ms, p.a, p.b));
        ctx->prof_ms[p.cls] += ms;
        ctx->prof_launches[p.cls]++;
        ctx->pool.push_back(p.a);
        ctx->pool.push_back(p.b);
    }
    ctx->pending.clear();
    for (int i = 0; i < HREBSD_PROF_CLASSES; ++i) {
        out->ms[i] = ctx->prof_ms[i];
        out->launches[i] = ctx->prof_launches[i];
    }
    unsigned long long px = 0;
    if (ctx->d_pixiters) HR_CHECK(cudaMemcpy(&px, ctx->d_pixiters, sizeof(px), cudaMemcpyDeviceToHost));
    out->pixel_iters = (long long)px;
    return HREBSD_OK;
}

int hrebsd_create(hrebsd_ctx **ctx, int device)
{
    if (!ctx) return HREBSD_EINVAL;
    *ctx = nullptr;
    int n = 0;
    HR_CHECK(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return HREBSD_EINVAL;
    HR_CHECK(cudaSetDevice(device));
    hrebsd_ctx *c = new hrebsd_ctx();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&c->d_err, hr_device_error_flag);
    if (e != cudaSuccess) {
        delete c;
        return hr_cuda_error(e, "hrebsd_create", __FILE__, __LINE__);
    }
    if (getenv("HREBSD_NO_TMA")) c->no_tma = 1;
    if (getenv("HREBSD_NO_GRAPHS")) c->graphs = 0;
    *ctx = c;
    return HREBSD_OK;
}

int hrebsd_destroy(hrebsd_ctx *ctx)
{
    if (!ctx) return HREBSD_EINVAL;
    int st = hr_set_device(ctx);
    cudaDeviceSynchronize();
    for (auto &b : ctx->ws)
        if (b.ptr) cudaFree(b.ptr);
    hr_cnn_destroy(ctx);
    for (auto &g : ctx->graph_cache) cudaGraphExecDestroy(g.exec);
    for (auto &m : ctx->mtex) {
        cudaDestroyTextureObject(m.tex);
        cudaFreeArray(m.arr);
    }
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (auto &p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    if (ctx->d_pixiters) cudaFree(ctx->d_pixiters);
    delete ctx;
    return st;
}

const char *hrebsd_status_string(int status)
{
    switch (status) {
    case HREBSD_OK: return "ok";
    case HREBSD_EINVAL: return "invalid argument";
    case HREBSD_ECUDA: return "CUDA error";
    case HREBSD_ENOMEM: return "out of device memory";
    case HREBSD_ETIMEOUT: return "bounded device wait expired";
    case HREBSD_ESCRATCH: return "request exceeds the static scratch array of the allocation-free entry point";
    case HREBSD_EIO: return "file could not be opened, read or written";
    case HREBSD_EFORMAT: return "not a model file of this network (wrong header, size or checksum)";
    default: return "unknown status";
    }
}

long long hrebsd_launch_count(const hrebsd_ctx *ctx) { return ctx ? ctx->launches : -1; }

int hrebsd_device_error(hrebsd_ctx *ctx)
{
    if (!ctx) return HREBSD_EINVAL;
    int st = hr_set_device(ctx);
    if (st) return st;
    HR_CHECK(cudaDeviceSynchronize());
    int flag = 0, zero = 0;
    HR_CHECK(cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) HR_CHECK(cudaMemcpy(ctx->d_err, &zero, sizeof(int), cudaMemcpyHostToDevice));
    return flag ? HREBSD_ETIMEOUT : HREBSD_OK;
}

int hrebsd_set_option(hrebsd_ctx *ctx, int option, int value)
{
    if (!ctx) return HREBSD_EINVAL;
    switch (option) {
    case HREBSD_OPT_NO_TMA: ctx->no_tma = value ? 1 : 0; return HREBSD_OK;
    case HREBSD_OPT_GRAPHS: ctx->graphs = value ? 1 : 0; return HREBSD_OK;
    case HREBSD_OPT_CNN_TC: ctx->cnn_tc = value ? 1 : 0; return HREBSD_OK;
    case HREBSD_OPT_TEX_GATHER: ctx->tex_gather = value ? 1 : 0; return HREBSD_OK;
    default: return HREBSD_EINVAL;
    }
}

}  // extern "C"

// ---------------------------------------------------------------- tensor maps
#include "tma.cuh"

typedef CUresult (*hr_encode_tiled_fn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                       const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                       CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                       CUtensorMapFloatOOBfill);

static hr_encode_tiled_fn encode_fn()
{
    static hr_encode_tiled_fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<hr_encode_tiled_fn>(p);
        else
            (void)cudaGetLastError();
    }
    return fn;
}

int hr_encode_tmap_3d(CUtensorMap *tm, const void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1,
                      uint64_t s2, uint32_t b0, uint32_t b1, uint32_t b2)
{
    hr_encode_tiled_fn fn = encode_fn();
    if (!fn) return -1;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (s1 & 15) || (s2 & 15) || ((b0 * 4) & 15)) return -1;
    if (b0 > 256 || b1 > 256 || b2 > 256 || b0 == 0 || b1 == 0 || b2 == 0) return -1;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {s1, s2};
    cuuint32_t box[3] = {b0, b1, b2};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int hr_encode_tmap_bf16_4d(CUtensorMap *tm, const void *base, const uint64_t dims[4], const uint64_t strides[3],
                           const uint32_t box[4], int swizzle_bytes)
{
    hr_encode_tiled_fn fn = encode_fn();
    if (!fn) return -1;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || ((box[0] * 2) & 15)) return -1;
    CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_NONE;
    if (swizzle_bytes) {
        if ((int)box[0] * 2 != swizzle_bytes) return -1;
        sw = swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
             : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
             : swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                    : CU_TENSOR_MAP_SWIZZLE_NONE;
        if (sw == CU_TENSOR_MAP_SWIZZLE_NONE) return -1;
    }
    for (int i = 0; i < 3; ++i)
        if (strides[i] & 15) return -1;
    for (int i = 0; i < 4; ++i)
        if (box[i] == 0 || box[i] > 256 || dims[i] == 0) return -1;
    cuuint64_t d[4] = {dims[0], dims[1], dims[2], dims[3]};
    cuuint64_t st[3] = {strides[0], strides[1], strides[2]};
    cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), d, st, bx, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}
