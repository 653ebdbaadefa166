// Precomputation of the mollified truncated Green's function (Section 4.3), FP64:
//  1. B^R(k) (eq. BhatR; stokeslet, stresslet) or H^R(k) (eq. HhatR; rotlet) on
//     the oversampled Mg^3 grid, k = 2 pi kbar / (Mg h), R = sqrt(3) Ltilde;
//     only the half spectrum kx in [0, Mg/2] is formed (the data are real and even);
//  2. inverse FFT (complex-to-real), normalised by 1/Mg^3;
//  3. keep the 2 Mt values per dimension centred at zero (j in [-Mt, Mt-1]),
//     stored wrap-ordered on the (2 Mt)^3 grid;
//  4. forward FFT (real-to-complex); the result is real and even, so the
//     (Mt+1)^3 octant of its real part is all the scaling step needs.
#include <vector>

#include "se_internal.cuh"

namespace se {

namespace {

// Truncated biharmonic transform, with its Taylor series for R k < 1 where the
// closed form cancels (4 pi sum_n (-1)^n k^{2n} R^{2n+4} / ((2n+1)! (2n+4))).
__device__ double bhat_trunc(double k, double R) {
    double x = R * k;
    if (x < 1.0) {
        double s = 0.0, term = R * R * R * R;  // n = 0: R^4 / (1! * 4)
        double fact = 1.0;                      // (2n+1)!
        double pk = 1.0;                        // (kR)^{2n}
        for (int n = 0; n < 12; n++) {
            if (n > 0) {
                fact *= (2.0 * n) * (2.0 * n + 1.0);
                pk *= -x * x;
            }
            s += pk * term / (fact * (2.0 * n + 4.0));
        }
        return 4.0 * M_PI * s;
    }
    double k4 = k * k * k * k;
    return 4.0 * M_PI * ((2.0 - x * x) * cos(x) + 2.0 * x * sin(x) - 2.0) / k4;
}

__device__ double hhat_trunc(double k, double R) {
    if (k == 0.0) return 2.0 * M_PI * R * R;
    double s = sin(R * k / 2.0) / k;
    return 8.0 * M_PI * s * s;
}

__global__ void k_eval_truncated(int Mg, double dk, double R, int harmonic, cufftDoubleComplex *out) {
    const int nxh = Mg / 2 + 1;
    size_t nk = (size_t)Mg * Mg * nxh;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nk) return;
    int kx = idx % nxh;
    int ky = (idx / nxh) % Mg;
    int kz = idx / ((size_t)nxh * Mg);
    int by = (ky < Mg / 2) ? ky : ky - Mg;
    int bz = (kz < Mg / 2) ? kz : kz - Mg;
    double kk = dk * sqrt((double)kx * kx + (double)by * by + (double)bz * bz);
    double v = harmonic ? hhat_trunc(kk, R) : bhat_trunc(kk, R);
    out[idx] = make_cuDoubleComplex(v, 0.0);
}

// Gt[j mod Mf] = G[j mod Mg] / Mg^3 for j in [-Mt, Mt-1]^3
__global__ void k_truncate(int Mg, int Mt, double scale, const double *G, double *Gt) {
    const int Mf = 2 * Mt;
    size_t n = (size_t)Mf * Mf * Mf;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int ix = idx % Mf, iy = (idx / Mf) % Mf, iz = idx / ((size_t)Mf * Mf);
    // destination index i holds j = i (i < Mt) or i - Mf (i >= Mt)
    int jx = ix < Mt ? ix : ix - Mf;
    int jy = iy < Mt ? iy : iy - Mf;
    int jz = iz < Mt ? iz : iz - Mf;
    int sx = (jx + Mg) % Mg, sy = (jy + Mg) % Mg, sz = (jz + Mg) % Mg;
    Gt[idx] = G[((size_t)sz * Mg + sy) * Mg + sx] * scale;
}

__global__ void k_octant(int Mt, const cufftDoubleComplex *spec, double *oct64, float *oct32) {
    const int Mf = 2 * Mt, nxh = Mt + 1, O = Mt + 1;
    size_t n = (size_t)O * O * O;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int ax = idx % O, ay = (idx / O) % O, az = idx / ((size_t)O * O);
    double v = spec[((size_t)az * Mf + ay) * nxh + ax].x;
    oct64[idx] = v;
    if (oct32) oct32[idx] = (float)v;
}

}  // namespace

se_status_t precompute(se_plan_s *p) {
    const int Mg = p->Mg, Mt = p->Mt, Mf = p->Mf;
    const size_t nkg = (size_t)Mg * Mg * (Mg / 2 + 1);
    const size_t ng = (size_t)Mg * Mg * Mg;
    const size_t nf = (size_t)Mf * Mf * Mf;
    const size_t nkf = (size_t)Mf * Mf * (Mf / 2 + 1);
    cufftDoubleComplex *spec = nullptr;
    double *G = nullptr;
    cufftHandle plan = 0;
    se_status_t st = SE_OK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, 0);
    auto cleanup = [&]() {
        if (plan) cufftDestroy(plan);
        cudaFree(spec);
        cudaFree(G);
    };
    size_t big = nkg > nkf ? nkg : nkf;
    if (cudaMalloc(&spec, big * sizeof(cufftDoubleComplex)) != cudaSuccess ||
        cudaMalloc(&G, (ng > nf ? ng : nf) * sizeof(double)) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(SE_ERR_OOM, "precompute: device allocation failed");
    }
    double dk = 2.0 * M_PI / (Mg * p->h);
    int harmonic = (p->kernel == SE_ROTLET);
    k_eval_truncated<<<(unsigned)((nkg + 255) / 256), 256>>>(Mg, dk, p->R, harmonic, spec);
    if (cufftPlan3d(&plan, Mg, Mg, Mg, CUFFT_Z2D) != CUFFT_SUCCESS) {
        cleanup();
        return fail(SE_ERR_CUFFT, "precompute: Z2D plan failed");
    }
    if (cufftExecZ2D(plan, spec, G) != CUFFT_SUCCESS) {
        cleanup();
        return fail(SE_ERR_CUFFT, "precompute: Z2D failed");
    }
    cufftDestroy(plan);
    plan = 0;
    double *Gt = (double *)spec;  // reuse: Mf^3 doubles fit in the spectrum buffer? use a fresh area
    double *Gt_buf = nullptr;
    if (cudaMalloc(&Gt_buf, nf * sizeof(double)) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(SE_ERR_OOM, "precompute: device allocation failed");
    }
    Gt = Gt_buf;
    k_truncate<<<(unsigned)((nf + 255) / 256), 256>>>(Mg, Mt, 1.0 / (double)ng, G, Gt);
    if (cufftPlan3d(&plan, Mf, Mf, Mf, CUFFT_D2Z) != CUFFT_SUCCESS) {
        cudaFree(Gt_buf);
        cleanup();
        return fail(SE_ERR_CUFFT, "precompute: D2Z plan failed");
    }
    if (cufftExecD2Z(plan, Gt, spec) != CUFFT_SUCCESS) {
        cudaFree(Gt_buf);
        cleanup();
        return fail(SE_ERR_CUFFT, "precompute: D2Z failed");
    }
    size_t no = (size_t)(Mt + 1) * (Mt + 1) * (Mt + 1);
    k_octant<<<(unsigned)((no + 255) / 256), 256>>>(Mt, spec, p->ghat64,
                                                    p->prec == SE_FP32 ? (float *)p->ghat : nullptr);
    cudaError_t ce = cudaDeviceSynchronize();
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    p->precompute_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(Gt_buf);
    cleanup();
    if (ce != cudaSuccess) st = fail(SE_ERR_CUDA, std::string("precompute: ") + cudaGetErrorString(ce));
    if (p->prec == SE_FP64 && st == SE_OK)
        p->ghat = p->ghat64;
    return st;
}

}  // namespace se
