// Triply periodic plans (the periodic problem of Section 1.1, with the
// screening of Section 3): the Fourier part is the free-space pipeline on the
// unpadded periodic grid.  Points are spread onto the extended grid of
// mt = M + n_ext points per dimension (grid point e at x0 + (e - n_ext/2) h),
// whose halo is folded onto the periodic M^3 grid (point i collects every e
// with e - n_ext/2 = i mod M); after the transforms the periodic grid is
// unfolded back onto the extended layout that the gather reads.  The scaling
// uses the exact transforms of the harmonic and biharmonic kernels, 4 pi/k^2
// and -8 pi/k^4 (eq. def_harm_biharm), at k = 2 pi j / L; the k = 0 term is
// zero (the mean force is balanced by a mean pressure gradient, Hasimoto's
// convention).
#include "se_internal.cuh"

namespace se {

namespace {

// per[c][i] = sum of ext[c][e] over e = i + he + a M in [0, mt), a in {-1, 0, 1}
template <typename T>
__global__ void k_fold(const T *__restrict__ ext, T *__restrict__ per, int nc, int M, int mt, int he) {
    const size_t n = (size_t)M * M * M;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nc) return;
    const int c = (int)(idx / n);
    const size_t r = idx - (size_t)c * n;
    const int i = (int)(r % M), j = (int)((r / M) % M), k = (int)(r / ((size_t)M * M));
    const T *src = ext + (size_t)c * mt * mt * mt;
    T s = T(0);
    for (int az = -1; az <= 1; az++) {
        const int ez = k + he + az * M;
        if (ez < 0 || ez >= mt) continue;
        for (int ay = -1; ay <= 1; ay++) {
            const int ey = j + he + ay * M;
            if (ey < 0 || ey >= mt) continue;
            for (int ax = -1; ax <= 1; ax++) {
                const int ex = i + he + ax * M;
                if (ex < 0 || ex >= mt) continue;
                s += src[((size_t)ez * mt + ey) * mt + ex];
            }
        }
    }
    per[idx] = s;
}

// ext[c][e] = per[c][(e - he) mod M]
template <typename T>
__global__ void k_unfold(const T *__restrict__ per, T *__restrict__ ext, int nc, int M, int mt, int he) {
    const size_t n = (size_t)mt * mt * mt;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nc) return;
    const int c = (int)(idx / n);
    const size_t r = idx - (size_t)c * n;
    const int ex = (int)(r % mt), ey = (int)((r / mt) % mt), ez = (int)(r / ((size_t)mt * mt));
    const int i = (ex - he + 2 * M) % M, j = (ey - he + 2 * M) % M, k = (ez - he + 2 * M) % M;
    ext[idx] = per[(size_t)c * M * M * M + ((size_t)k * M + j) * M + i];
}

// octant (a_x, a_y, a_z) in [0, M/2]^3 of the exact transform at |k| = dk |a|
__global__ void k_periodic_octant(int O, double dk, int harmonic, double *oct64, float *oct32) {
    const size_t n = (size_t)O * O * O;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int ax = (int)(idx % O), ay = (int)((idx / O) % O), az = (int)(idx / ((size_t)O * O));
    const double k2 = dk * dk * ((double)ax * ax + (double)ay * ay + (double)az * az);
    const double v = (k2 == 0.0) ? 0.0 : (harmonic ? 4.0 * M_PI / k2 : -8.0 * M_PI / (k2 * k2));
    oct64[idx] = v;
    if (oct32) oct32[idx] = (float)v;
}

}  // namespace

template <typename T>
cudaError_t launch_fold(se_plan_s *p, cudaStream_t st, const void *ext, void *per, int nc) {
    const int M = p->mp, mt = p->mt[0], he = p->n_ext / 2;
    const size_t n = (size_t)nc * M * M * M;
    k_fold<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const T *)ext, (T *)per, nc, M, mt, he);
    p->launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unfold(se_plan_s *p, cudaStream_t st, const void *per, void *ext, int nc) {
    const int M = p->mp, mt = p->mt[0], he = p->n_ext / 2;
    const size_t n = (size_t)nc * mt * mt * mt;
    k_unfold<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const T *)per, (T *)ext, nc, M, mt, he);
    p->launches++;
    return cudaGetLastError();
}

template cudaError_t launch_fold<float>(se_plan_s *, cudaStream_t, const void *, void *, int);
template cudaError_t launch_fold<double>(se_plan_s *, cudaStream_t, const void *, void *, int);
template cudaError_t launch_unfold<float>(se_plan_s *, cudaStream_t, const void *, void *, int);
template cudaError_t launch_unfold<double>(se_plan_s *, cudaStream_t, const void *, void *, int);

se_status_t periodic_octant(se_plan_s *p) {
    const int O = p->mp / 2 + 1;
    const size_t n = (size_t)O * O * O;
    const double dk = 2.0 * M_PI / (p->mp * p->h);
    k_periodic_octant<<<(unsigned)((n + 255) / 256), 256>>>(O, dk, p->kernel == SE_ROTLET ? 1 : 0, p->ghat64,
                                                            p->prec == SE_FP32 ? (float *)p->ghat : nullptr);
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(SE_ERR_CUDA, std::string("periodic octant: ") + cudaGetErrorString(e));
    if (p->prec == SE_FP64) p->ghat = p->ghat64;
    p->precompute_ms = 0;
    p->precompute_cached = false;
    return SE_OK;
}

}  // namespace se
