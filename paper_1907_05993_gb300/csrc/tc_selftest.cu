// Self-tests: the bounded-wait failure path, and the tcgen05 building blocks
// (descriptors, MMA, commit, TMEM loads)
// on one GEMM tile: D[128][N] = A[128][K] B[N][K]^T, BF16 operands, FP32
// accumulation in tensor memory.  The operand area of shared memory is padded
// well beyond the operands and the whole TMEM range an N field can name is
// allocated, so that every address a descriptor can reach stays inside the
// CTA's allocations.
#include "internal.cuh"
#include "tc.cuh"

namespace {

constexpr int kM = 128;
constexpr uint32_t kOffB = 48 * 1024, kSmem = 96 * 1024, kTmemCols = 256;

__global__ void __launch_bounds__(128) tc_selftest_kernel(const uint16_t *__restrict__ A, const uint16_t *__restrict__ B,
                                                          int N, int KS, float *__restrict__ D, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int K = 16 * KS;
    const uint32_t planeA = kM * 16, planeB = (uint32_t)N * 16;
    // operands into the core-matrix layout: row r, K-group g at plane * g + 16 r
    for (int i = tid; i < kM * K / 8; i += blockDim.x) {
        const int r = i / (K / 8), g = i - r * (K / 8);
        *reinterpret_cast<uint4 *>(sm + g * planeA + r * 16) = *reinterpret_cast<const uint4 *>(A + (size_t)r * K + g * 8);
    }
    for (int i = tid; i < N * K / 8; i += blockDim.x) {
        const int r = i / (K / 8), g = i - r * (K / 8);
        *reinterpret_cast<uint4 *>(sm + kOffB + g * planeB + r * 16) =
            *reinterpret_cast<const uint4 *>(B + (size_t)r * K + g * 8);
    }
    if (tid == 0) {
        hr_tma::mbar_init(&bar, 1);
        hr_tma::fence_mbar_init();
    }
    if (warp == 0) hr_tc::tmem_alloc(&tmem_base, kTmemCols);
    hr_tma::fence_proxy_async();   // generic-proxy stores -> visible to the tensor cores
    hr_tc::fence_before_sync();
    __syncthreads();
    hr_tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    if (tid == 0) {
        const uint32_t a0 = hr_tma::smem_u32(sm), b0 = hr_tma::smem_u32(sm + kOffB);
        const uint32_t id = hr_tc::idesc_bf16(kM, N);
        for (int j = 0; j < KS; ++j)
            hr_tc::mma_bf16(tb, hr_tc::smem_desc(a0 + 2 * j * planeA, planeA, 128),
                            hr_tc::smem_desc(b0 + 2 * j * planeB, planeB, 128), id, j > 0);
        hr_tc::commit(&bar);
    }
    const bool ok = __syncthreads_and(hr_tma::mbar_wait(&bar, 0));
    if (!ok && tid == 0) atomicExch(err, 1);
    hr_tc::fence_after_sync();
    if (ok) {
        const int row = warp * 32 + (tid & 31);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            hr_tc::ld16(tb + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            for (int i = 0; i < 16; ++i) D[(size_t)row * N + c0 + i] = v[i];
        }
    }
    hr_tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) hr_tc::tmem_dealloc(tb, kTmemCols);
}

// Failure-path check of the bounded waits: an mbarrier that nothing arrives at,
// waited on with the same try-wait loop as the library's kernels but with a
// caller-given poll limit; when it runs out the kernel raises the context's
// error flag and returns.
__global__ void wait_selftest_kernel(uint32_t max_polls, int *err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        hr_tma::mbar_init(&bar, 1);
        hr_tma::fence_mbar_init();
    }
    __syncthreads();
    bool done = false;
    for (uint32_t i = 0; i < max_polls && !done; ++i) done = hr_tma::mbar_try_wait(&bar, 0);
    if (!__syncthreads_or(done) && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace

extern "C" int hrebsd_wait_selftest(hrebsd_ctx *ctx, unsigned max_polls, void *stream)
{
    if (!ctx || max_polls < 1 || max_polls > (1u << 22)) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    wait_selftest_kernel<<<1, 32, 0, hr_stream(stream)>>>(max_polls, ctx->d_err);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

extern "C" int hrebsd_tc_selftest(hrebsd_ctx *ctx, const uint16_t *A, const uint16_t *B, int N, int KS, float *D,
                                  void *stream)
{
    if (!ctx || !A || !B || !D || KS < 1 || KS > 4 || (N != 16 && N != 32 && N != 64)) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    static int configured = -1;
    if (configured != ctx->device) {
        HR_CHECK(cudaFuncSetAttribute(tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
        configured = ctx->device;
    }
    tc_selftest_kernel<<<1, 128, kSmem, hr_stream(stream)>>>(A, B, N, KS, D, ctx->d_err);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}
