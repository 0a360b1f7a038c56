// 3x3 convolution on the fifth-generation tensor cores (tcgen05): the
// implicit GEMM of conv3x3_kernel (128 output pixels x BN output channels per
// CTA, K = 9 taps x cin walked in k-steps of 16 channels of one tap, STAGES
// cp.async stages of KS k-steps) with the MMAs issued by one thread from
// shared-memory descriptors into an FP32 accumulator in tensor memory.
//
// Shared layout of a k-step: the A rows (shifted input pixels) and B rows
// (weights) in the K-major core-matrix layout: row r, 8-channel group g at
// base + g * plane + 16 r (plane = rows x 16 bytes).  A stage is reused only
// after the MMAs that read it have completed (one mbarrier per stage, armed by
// tcgen05.commit).  Every wait is bounded; a wait that gives up sets the error
// flag and the CTA skips its epilogue.
#pragma once

#include "cnn_kernels.cuh"
#include "tc.cuh"

namespace hr_cnn {

template <int BN, int KS, int STAGES>
struct TcConv {
    static constexpr int BM = 128;
    static constexpr uint32_t A_PLANE = BM * 16, B_PLANE = BN * 16;
    static constexpr uint32_t STEP = 2 * A_PLANE + 2 * B_PLANE;   // one k-step: 16 channels of A and B
    static constexpr uint32_t STAGE = KS * STEP;
    static constexpr uint32_t SMEM = STAGES * STAGE;
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;      // power of two >= 32
};

template <int BN, int KS, int STAGES>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(ConvArgs a, int *err)
{
    using G = TcConv<BN, KS, STAGES>;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar[STAGES];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int P = a.N * a.H * a.W;
    const int p0 = blockIdx.x * G::BM, o0 = blockIdx.y * BN;
    // loader: A row tid (one output pixel), both 8-channel halves; B rows tid / 2 (half tid % 2) for tid < 2 BN
    const int lp = p0 + tid;
    int pn = 0, py = 0, px = 0;
    if (lp < P) {
        pn = lp / (a.H * a.W);
        const int rem = lp - pn * a.H * a.W;
        py = rem / a.W;
        px = rem - py * a.W;
    }
    const int lo = o0 + (tid >> 1), bhalf = tid & 1;
    const int ncb = a.cin / 16, KT = 9 * ncb, nstage = (KT + KS - 1) / KS;
    auto load_stage = [&](int s) {
        unsigned char *base = tc_smem + (s % STAGES) * G::STAGE;
#pragma unroll
        for (int j = 0; j < KS; ++j) {
            const int kt = s * KS + j;
            const int tap = kt / ncb, cb = kt - tap * ncb;
            const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
            const bool oka = kt < KT && lp < P && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            unsigned char *st = base + j * G::STEP;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const bf16 *src = oka ? a.x + ((size_t)(pn * a.H + yy) * a.W + xx) * a.xs + a.xo + cb * 16 + hh * 8 : a.x;
                cp_async16(st + hh * G::A_PLANE + tid * 16, src, oka ? 16 : 0);
            }
            if (tid < 2 * BN) {
                const bool okb = kt < KT && lo < a.cout;
                const bf16 *src = okb ? a.w + ((size_t)lo * 9 + tap) * a.cin + cb * 16 + bhalf * 8 : a.w;
                cp_async16(st + 2 * G::A_PLANE + bhalf * G::B_PLANE + (tid >> 1) * 16, src, okb ? 16 : 0);
            }
        }
    };
    if (tid == 0) {
        for (int i = 0; i < STAGES; ++i) hr_tma::mbar_init(&bar[i], 1);
        hr_tma::fence_mbar_init();
    }
    if (warp == 0) hr_tc::tmem_alloc(&tmem_base, G::TMEM_COLS);
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nstage) load_stage(s);
        cp_async_commit();
    }
    hr_tc::fence_before_sync();
    __syncthreads();
    hr_tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    constexpr uint32_t idesc = hr_tc::idesc_bf16(128, BN);
    bool ok = true;
    for (int s = 0; s < nstage; ++s) {
        cp_async_wait<STAGES - 2>();
        hr_tma::fence_proxy_async();   // this thread's cp.async data -> visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            hr_tc::fence_after_sync();
            const uint32_t sb = hr_tma::smem_u32(tc_smem + (s % STAGES) * G::STAGE);
#pragma unroll
            for (int j = 0; j < KS; ++j) {
                const uint32_t st = sb + j * G::STEP;
                hr_tc::mma_bf16(tb, hr_tc::smem_desc(st, G::A_PLANE, 128),
                                hr_tc::smem_desc(st + 2 * G::A_PLANE, G::B_PLANE, 128), idesc, (s | j) != 0);
            }
            hr_tc::commit(&bar[s % STAGES]);
        }
        // the buffer of stage s + STAGES - 1 was read by the MMAs of stage s - 1
        const int nx = s + STAGES - 1;
        if (nx < nstage) {
            if (s >= 1) ok = hr_tma::mbar_wait(&bar[(s - 1) % STAGES], ((s - 1) / STAGES) & 1) && ok;
            load_stage(nx);
        }
        cp_async_commit();
    }
    // the last commit covers every MMA of this CTA
    ok = hr_tma::mbar_wait(&bar[(nstage - 1) % STAGES], ((nstage - 1) / STAGES) & 1) && ok;
    ok = __syncthreads_and(ok);
    cp_async_wait<0>();
    hr_tc::fence_after_sync();
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        const int p = p0 + warp * 32 + (tid & 31);   // TMEM lane = A row = output pixel
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            hr_tc::ld16(tb + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (p < P) {
#pragma unroll
                for (int i = 0; i < 16; i += 2) {
                    const int o = o0 + c0 + i;
                    if (o >= a.cout) continue;
                    float v0 = v[i], v1 = v[i + 1];
                    if (a.bias) {
                        v0 += a.bias[o];
                        v1 += a.bias[o + 1];
                    }
                    if (a.relu) {
                        v0 = fmaxf(v0, 0.0f);
                        v1 = fmaxf(v1, 0.0f);
                    }
                    const size_t off = (size_t)p * a.ys + a.yo + o;
                    if (a.y_fp32) {
                        *reinterpret_cast<float2 *>(reinterpret_cast<float *>(a.y) + off) = make_float2(v0, v1);
                    } else {
                        *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(a.y) + off) =
                            __floats2bfloat162_rn(v0, v1);
                    }
                }
            }
        }
    }
    hr_tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) hr_tc::tmem_dealloc(tb, G::TMEM_COLS);
}

}  // namespace hr_cnn
