// f1: strain and stress of each scan point (Eq. 13-16, Supplementary Part 2).
//
// The detector-frame deformation gradient goes to the sample frame with the
// tilt rotation of Eq. 13 (F_S = R F R^T, Eq. 14); the strain is
// 1/2 (F_S F_S^T - I) (Eq. 15, which removes the finite rotation of the
// remapping exactly); the stress is sigma = C_S : epsilon (Eq. 16) with the
// cubic stiffness rotated to the sample frame in Voigt form, C_S = M C M^T,
// M the 6x6 stress-transformation (Bond) matrix of the rotation g^T (the
// supplement's R_sigma C R_eps^-1).  With the traction-free option the
// unknown scale of F is fixed by sigma_33 = 0, which is linear in the square
// of the scale.  FP64, one thread per pair.
#include <math.h>

#include "internal.cuh"

namespace {

__device__ void mat3_mul(const double *A, const double *B, double *C)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i * 3 + j] = A[i * 3] * B[j] + A[i * 3 + 1] * B[3 + j] + A[i * 3 + 2] * B[6 + j];
}

// Voigt pairs (11, 22, 33, 23, 13, 12)
__device__ __forceinline__ void vpair(int k, int &i, int &j)
{
    const int I[6] = {0, 1, 2, 1, 0, 0}, J[6] = {0, 1, 2, 2, 2, 1};
    i = I[k];
    j = J[k];
}

// C_S = M C M^T (Voigt, 6x6): the cubic stiffness rotated from crystal to
// sample axes, M the Bond matrix of a = g^T (crystal -> sample), gr = g of the
// pair's reference (sample -> crystal).
__device__ void stiffness_sample(const double *gr, double c11, double c12, double c44, double *CS)
{
    double a[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a[i * 3 + j] = gr[j * 3 + i];
    double M[36], C[36], MC[36];
    for (int I = 0; I < 6; ++I) {
        int i, j;
        vpair(I, i, j);
        for (int P = 0; P < 6; ++P) {
            int p, q;
            vpair(P, p, q);
            M[I * 6 + P] = p == q ? a[i * 3 + p] * a[j * 3 + p]
                                  : a[i * 3 + p] * a[j * 3 + q] + a[i * 3 + q] * a[j * 3 + p];
            C[I * 6 + P] = (I < 3 && P < 3) ? (I == P ? c11 : c12) : (I == P ? c44 : 0.0);
        }
    }
    for (int I = 0; I < 6; ++I)
        for (int P = 0; P < 6; ++P) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += M[I * 6 + k] * C[k * 6 + P];
            MC[I * 6 + P] = s;
        }
    for (int I = 0; I < 6; ++I)
        for (int P = 0; P < 6; ++P) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += MC[I * 6 + k] * M[P * 6 + k];
            CS[I * 6 + P] = s;
        }
}

// Eq. 13-14: F_S = T F T^T
__device__ void tilt_to_sample(const double *F, double ct, double st, double *Fs)
{
    const double T[9] = {ct, st, 0.0, -st, ct, 0.0, 0.0, 0.0, 1.0};
    const double Tt[9] = {ct, -st, 0.0, st, ct, 0.0, 0.0, 0.0, 1.0};
    double tmp[9];
    mat3_mul(T, F, tmp);
    mat3_mul(tmp, Tt, Fs);
}

// A = 1/2 F_S F_S^T
__device__ void half_ffT(const double *Fs, double *A)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            A[i * 3 + j] = 0.5 * (Fs[i * 3] * Fs[j * 3] + Fs[i * 3 + 1] * Fs[j * 3 + 1] + Fs[i * 3 + 2] * Fs[j * 3 + 2]);
}

// Traction-free scale (Eq. 16, sigma_33 = 0): lambda^2 with
// sigma_33(lambda^2 A - I/2) = 0, A = 1/2 F_S F_S^T.
__device__ double traction_lam2(const double *A, const double *CS)
{
    double sa = 0.0;
    for (int k = 0; k < 6; ++k) {
        int i, j;
        vpair(k, i, j);
        sa += CS[2 * 6 + k] * (k < 3 ? A[i * 3 + j] : 2.0 * A[i * 3 + j]);
    }
    const double sb = 0.5 * (CS[12] + CS[13] + CS[14]);
    return sb / sa;
}

__global__ void strain_stress_kernel(const double *__restrict__ F, const int32_t *__restrict__ ref_idx,
                                     const double *__restrict__ g, int R, int B, double ct, double st, double c11,
                                     double c12, double c44, int traction_free, double *F_S, double *eps,
                                     double *sigma)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int r = ref_idx ? ref_idx[b] : 0;
    double Fs[9], E[9], S[9];
    if (r < 0 || r >= R) {
        for (int k = 0; k < 9; ++k) Fs[k] = E[k] = S[k] = nan("");
    } else {
        tilt_to_sample(F + (size_t)b * 9, ct, st, Fs);
        double CS[36];
        stiffness_sample(g + (size_t)r * 9, c11, c12, c44, CS);
        // engineering Voigt strain of 1/2 F_S F_S^T
        double A[9];
        half_ffT(Fs, A);
        if (traction_free) {
            const double lam2 = traction_lam2(A, CS);
            const double lam = sqrt(lam2);
            for (int k = 0; k < 9; ++k) {
                Fs[k] *= lam;
                A[k] *= lam2;
            }
        }
        for (int k = 0; k < 9; ++k) E[k] = A[k] - (k % 4 == 0 ? 0.5 : 0.0);
        double ev[6], sv[6];
        for (int k = 0; k < 6; ++k) {
            int i, j;
            vpair(k, i, j);
            ev[k] = k < 3 ? E[i * 3 + j] : 2.0 * E[i * 3 + j];
        }
        for (int I = 0; I < 6; ++I) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += CS[I * 6 + k] * ev[k];
            sv[I] = s;
        }
        for (int k = 0; k < 6; ++k) {
            int i, j;
            vpair(k, i, j);
            S[i * 3 + j] = S[j * 3 + i] = sv[k];
        }
    }
    for (int k = 0; k < 9; ++k) {
        if (F_S) F_S[(size_t)b * 9 + k] = Fs[k];
        eps[(size_t)b * 9 + k] = E[k];
        sigma[(size_t)b * 9 + k] = S[k];
    }
}

// Traction-free scale of the second-pass F (hrebsd_solve_F): F <- lambda F in
// place (the scale commutes with the tilt, so lambda of F_S scales F itself).
__global__ void traction_scale_kernel(double *__restrict__ F, const int32_t *__restrict__ ref_idx,
                                      const double *__restrict__ g, int R, int B, double ct, double st, double c11,
                                      double c12, double c44, int32_t *status)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double *Fb = F + (size_t)b * 9;
    const int r = ref_idx ? ref_idx[b] : 0;
    double lam = nan("");
    if (r >= 0 && r < R) {
        double Fs[9], A[9], CS[36];
        tilt_to_sample(Fb, ct, st, Fs);
        stiffness_sample(g + (size_t)r * 9, c11, c12, c44, CS);
        half_ffT(Fs, A);
        const double lam2 = traction_lam2(A, CS);
        if (lam2 > 0.0 && isfinite(lam2)) lam = sqrt(lam2);
    }
    if (!(lam > 0.0)) {
        if (status) status[b] |= HREBSD_PAIR_FIT_FAILED;
        for (int k = 0; k < 9; ++k) Fb[k] = nan("");
        return;
    }
    for (int k = 0; k < 9; ++k) Fb[k] *= lam;
}

}  // namespace

extern "C" int hrebsd_strain_stress(hrebsd_ctx *ctx, const double *F, const int32_t *ref_idx, const double *g, int R,
                                    int B, double tilt_rad, double c11, double c12, double c44, int traction_free,
                                    double *F_S, double *eps, double *sigma, void *stream)
{
    if (!ctx || B < 0 || R < 1) return HREBSD_EINVAL;
    if (B == 0) return HREBSD_OK;
    if (!F || !g || !eps || !sigma) return HREBSD_EINVAL;
    int e = hr_set_device(ctx);
    if (e) return e;
    hr_prof_begin(ctx, hr_stream(stream));
    strain_stress_kernel<<<(B + 127) / 128, 128, 0, hr_stream(stream)>>>(F, ref_idx, g, R, B, cos(tilt_rad),
                                                                        sin(tilt_rad), c11, c12, c44, traction_free,
                                                                        F_S, eps, sigma);
    hr_prof_end(ctx, PROF_SOLVE, hr_stream(stream));
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}

int hr_launch_traction_scale(hrebsd_ctx *ctx, double *F, const hrebsd_elastic *el, int B, int32_t *status,
                             cudaStream_t st)
{
    hr_prof_begin(ctx, st);
    traction_scale_kernel<<<(B + 127) / 128, 128, 0, st>>>(F, el->ref_idx, el->g, el->R, B, cos(el->tilt_rad),
                                                           sin(el->tilt_rad), el->c11, el->c12, el->c44, status);
    hr_prof_end(ctx, PROF_SOLVE, st);
    HR_LAUNCHED(ctx);
    return HREBSD_OK;
}
