// Internal declarations of the HR-EBSD CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "hrebsd.h"

#define HR_CHECK(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return hr_cuda_error(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define HR_LAUNCHED(ctx)                                                       \
    do {                                                                       \
        cudaError_t e_ = cudaGetLastError();                                   \
        if (e_ != cudaSuccess) return hr_cuda_error(e_, "kernel launch", __FILE__, __LINE__); \
        (ctx)->launches++;                                                     \
    } while (0)

int hr_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// One growable device allocation owned by the context.
struct hr_buf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

enum { PROF_ITER = 0, PROF_CTRL, PROF_DEMONS_AUX, PROF_PRE, PROF_FIT, PROF_REMAP, PROF_XCF, PROF_SOLVE, PROF_CNN };

struct hr_cnn_net;
void hr_cnn_destroy(hrebsd_ctx *ctx);

struct hr_pending {
    int cls;
    cudaEvent_t a, b;
};

// Cached CUDA graph of one pyramid level of a registration (demons.cu).
struct hr_graph_key {
    const void *p[16];
    int i[16];
    float f[32];
};
struct hr_graph_entry {
    hr_graph_key key;
    cudaGraphExec_t exec;
    long long nodes;          // kernel launches in the graph
    unsigned long long last;  // LRU clock
};
// Tile shape chosen for a level size (autotuner or caller).
struct hr_tune_entry {
    int h, w, var;
};
// Copy of a level's reference images in a CUDA array (rows R x h stacked, one array per level width)
// behind a texture object, for the four-texel gathers of the row sweep (demons.cu).
struct hr_mtex {
    int w, rows;
    cudaArray_t arr;
    unsigned long long tex;
};

struct hrebsd_ctx {
    int device = 0;
    int num_sms = 0;
    long long launches = 0;
    hr_buf ws[24];   // named workspace slots (demons.cu 0-13, metrics.cu 14, probe.cu 15, filters.cu 16-18)
    // tracing
    int prof_on = 0;
    int no_events = 0;   // set while a call must not create CUDA events
    int no_tma = 0;      // force the non-TMA demons iteration (testing, unsupported shapes)
    int graphs = 1;      // replay each registration level from a cached CUDA graph
    int cnn_tc = 1;      // learned initialiser: 3x3 convolutions on tcgen05 (else mma.sync kernels)
    int tex_gather = 1;  // row sweep: moving image by texture gathers from a CUDA array copy (else plain loads)
    int tex_max_rows = 0;         // texture-gather array height limit of the device (0 = not queried)
    std::vector<hr_mtex> mtex;    // reference arrays per level width
    cudaStream_t cap_stream = nullptr;   // private stream the graphs are captured on
    std::vector<hr_graph_entry> graph_cache;
    unsigned long long graph_clock = 0;
    std::vector<hr_tune_entry> tune;
    int *d_err = nullptr;   // device flag: a bounded wait gave up (static device symbol)
    hr_cnn_net *cnn = nullptr;   // learned initialiser (allocated on first use)
    double prof_ms[HREBSD_PROF_CLASSES] = {};
    long long prof_launches[HREBSD_PROF_CLASSES] = {};
    unsigned long long *d_pixiters = nullptr;
    std::vector<hr_pending> pending;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t cur_a = nullptr;
};

// Bracket a launch with events when tracing is on.
void hr_prof_begin(hrebsd_ctx *ctx, cudaStream_t st);
void hr_prof_end(hrebsd_ctx *ctx, int cls, cudaStream_t st);
// Device counter of demons pixel-iterations (NULL when tracing is off, and
// inside a call that is kept out of the trace).
static inline unsigned long long *hr_prof_pixiters(hrebsd_ctx *ctx)
{
    return ctx->prof_on && !ctx->no_events ? ctx->d_pixiters : nullptr;
}

// Make sure workspace slot `slot` holds at least `bytes`; returns the pointer
// through *out.  Allocation is synchronous (cudaMalloc) and happens only on
// growth.
int hr_ws(hrebsd_ctx *ctx, int slot, size_t bytes, void **out);
int hr_set_device(hrebsd_ctx *ctx);

static inline cudaStream_t hr_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Gaussian taps as used by the demons field regularisation (radius
// ceil(3 sigma), weights exp(-k^2/(2 sigma^2)) normalised to one), padded with
// zeros to radius `rad`.  Returns the natural radius, or -1 if > 6.
int hr_gauss_taps(float sigma, int rad, float *taps);
int hr_gauss_radius(float sigma);

// Traction-free rescaling of second-pass deformation gradients in place
// (strain.cu; used by hrebsd_solve_F with HREBSD_NORM_TRACTION_FREE).
int hr_launch_traction_scale(hrebsd_ctx *ctx, double *F, const hrebsd_elastic *el, int B, int32_t *status,
                             cudaStream_t st);
