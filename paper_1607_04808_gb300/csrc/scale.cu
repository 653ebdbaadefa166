// Step 3 of Section 5.2 (scaling, eq. gridfcnsc) as a pass over the spectrum
// (the multipliers are in multiplier.cuh).  Memory-bound: reads nc complex
// values and writes 3 per k-point, in place.
#include "multiplier.cuh"

namespace se {

namespace {

// Half-spectrum point idx of the [kz][ky][kx] R2C layout: its wave vector and
// the index of |k| in the stored octant of the precomputed kernel.
template <typename T>
__device__ __forceinline__ size_t kpoint(const ScaleConst &sc, size_t idx, T kv[3]) {
    const int kx = idx % sc.nxh;
    const int ky = (idx / sc.nxh) % sc.mf[1];
    const int kz = idx / ((size_t)sc.nxh * sc.mf[1]);
    return kpoint3<T>(sc, kx, ky, kz, kv);
}

__host__ __device__ inline size_t half_spectrum(const ScaleConst &sc) {
    return (size_t)sc.mf[2] * sc.mf[1] * sc.nxh;
}

// The multiplier at half-spectrum point idx applied to ngroups groups of
// source components (each group nc consecutive spectra of nk points).
template <typename T, int KERNEL>
__device__ __forceinline__ void scale_point(const ScaleConst &sc, const T *__restrict__ ghat,
                                            cplx<T> *__restrict__ spec, size_t idx, int ngroups,
                                            size_t scs = 0, size_t szs = 0) {
    // scs, szs: the spectra's component and z-plane strides (0: one whole
    // spectrum after the other, idx its own offset)
    using C = cplx<T>;
    const size_t plane = (size_t)sc.mf[1] * sc.nxh;
    const size_t nk = scs ? scs : half_spectrum(sc);
    size_t off = idx;
    if (szs) {
        const size_t kz = idx / plane;
        off = kz * szs + (idx - kz * plane);
    }
    T kv[3];
    const T G = ghat[kpoint<T>(sc, idx, kv)];
    constexpr int NCG = (KERNEL == SE_STRESSLET) ? 6 : 3;
    for (int grp = 0; grp < ngroups; grp++) {
        C *w0 = spec + (size_t)grp * NCG * nk + off;
        C g[NCG], o[3];
        for (int c = 0; c < NCG; c++) g[c] = w0[c * nk];
        apply_multiplier<T, KERNEL>(sc, kv, G, g, o);
        for (int j = 0; j < 3; j++) w0[j * nk] = o[j];
    }
}

template <typename T, int KERNEL>
__global__ void k_scale(ScaleConst sc, const T *__restrict__ ghat, cplx<T> *__restrict__ spec) {
    const size_t nk = half_spectrum(sc);
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nk) return;
    scale_point<T, KERNEL>(sc, ghat, spec, idx, 1);
}

// Adjoint of the stresslet (backward pass): from the spread upstream gradient
// g^ (3 spectra) to the symmetric tensor field V_lk(y) = sum_m T_jlk(x_m - y) g_mj
// (6 spectra: xx, yy, zz, xy, xz, yz).  T is odd, so its adjoint symbol is
// minus the forward one contracted on its first index:
//   V^_lk = i F [k^2 (k_k g^_l + k_l g^_k + (k.g^) d_lk) - 2 (k.g^) k_l k_k],
// with F the forward stresslet factor (1 + k^2/4xi^2) G~^ and the Gaussians.
template <typename T>
__global__ void k_scale_adj_stresslet(ScaleConst sc, const T *__restrict__ ghat, cplx<T> *__restrict__ spec) {
    using C = cplx<T>;
    const size_t nk = half_spectrum(sc);
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nk) return;
    T kv[3];
    const T G = ghat[kpoint<T>(sc, idx, kv)];
    const T k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
    const T F = (T)sc.norm * G * mexp((T)sc.ecoef * k2) * (T(1) + k2 * (T)sc.inv4xi2);
    C *w0 = spec + idx;
    C g[3];
    for (int c = 0; c < 3; c++) g[c] = w0[c * nk];
    C kg;
    kg.x = kv[0] * g[0].x + kv[1] * g[1].x + kv[2] * g[2].x;
    kg.y = kv[0] * g[0].y + kv[1] * g[1].y + kv[2] * g[2].y;
    const int L_[6] = {0, 1, 2, 0, 0, 1}, K_[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; c++) {
        const int l = L_[c], k = K_[c];
        C v;
        v.x = k2 * (kv[k] * g[l].x + kv[l] * g[k].x + (l == k ? kg.x : T(0))) - T(2) * kg.x * kv[l] * kv[k];
        v.y = k2 * (kv[k] * g[l].y + kv[l] * g[k].y + (l == k ? kg.y : T(0))) - T(2) * kg.y * kv[l] * kv[k];
        // multiply by i F: (a + ib) i = -b + ia
        C o;
        o.x = -F * v.y;
        o.y = F * v.x;
        w0[c * nk] = o;
    }
}

// Batched: block b belongs to the system s with blk_base[s] <= b < blk_base[s+1];
// each thread scales one k-point of that system for all n_rhs right-hand sides,
// reading the precomputed kernel once.
template <typename T, int KERNEL>
__global__ void k_bscale(const BSys<T> *__restrict__ sys, const int *__restrict__ blk_base, int S, int n_rhs) {
    const int s = find_range(blk_base, S, (int)blockIdx.x);
    const BSys<T> &B = sys[s];
    const ScaleConst sc = B.sc;
    const size_t nk = half_spectrum(sc);
    const size_t idx = (size_t)(blockIdx.x - blk_base[s]) * blockDim.x + threadIdx.x;
    if (idx >= nk) return;
    scale_point<T, KERNEL>(sc, B.ghat, B.spec, idx, n_rhs, B.scs, B.szs);
}

}  // namespace

ScaleConst make_scale_const(const se_plan_s *p) {
    ScaleConst sc;
    for (int d = 0; d < 3; d++) {
        sc.mt[d] = p->mt[d];
        sc.mf[d] = p->mf[d];
        sc.dk[d] = 2.0 * M_PI / (p->mf[d] * p->h);
    }
    sc.nxh = p->mf[0] / 2 + 1;
    sc.inv4xi2 = 1.0 / (4.0 * p->xi * p->xi);
    sc.ecoef = -(1.0 - p->eta) / (4.0 * p->xi * p->xi);
    double pre = pow(2.0 * p->xi * p->xi / (M_PI * p->eta), 1.5);
    sc.norm = p->h * p->h * p->h / ((double)p->mf[0] * p->mf[1] * p->mf[2]) * pre * pre;
    if (p->periodic) {
        // the unpadded periodic grid M^3: k = 2 pi j / (M h), octant of M/2 + 1
        for (int d = 0; d < 3; d++) {
            sc.mt[d] = p->mp / 2;
            sc.mf[d] = p->mp;
            sc.dk[d] = 2.0 * M_PI / (p->mp * p->h);
        }
        sc.nxh = p->mp / 2 + 1;
        sc.norm = p->h * p->h * p->h / ((double)p->mp * p->mp * p->mp) * pre * pre;
    }
    return sc;
}

template <typename T>
cudaError_t launch_scale(se_plan_s *p, cudaStream_t st, void *spec, int transpose) {
    (void)transpose;  // the stokeslet and rotlet multipliers equal their transposes
    const ScaleConst sc = make_scale_const(p);
    size_t nk = half_spectrum(sc);
    int bs = SCALE_BS;
    unsigned gs = (unsigned)((nk + bs - 1) / bs);
    const T *gh = (const T *)p->ghat;
    cplx<T> *sp = (cplx<T> *)spec;
    if (p->kernel == SE_STOKESLET)
        k_scale<T, SE_STOKESLET><<<gs, bs, 0, st>>>(sc, gh, sp);
    else if (p->kernel == SE_STRESSLET)
        k_scale<T, SE_STRESSLET><<<gs, bs, 0, st>>>(sc, gh, sp);
    else
        k_scale<T, SE_ROTLET><<<gs, bs, 0, st>>>(sc, gh, sp);
    p->launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale_adj_stresslet(se_plan_s *p, cudaStream_t st, void *spec) {
    const ScaleConst sc = make_scale_const(p);
    const size_t nk = half_spectrum(sc);
    k_scale_adj_stresslet<T><<<(unsigned)((nk + SCALE_BS - 1) / SCALE_BS), SCALE_BS, 0, st>>>(
        sc, (const T *)p->ghat, (cplx<T> *)spec);
    p->launches++;
    return cudaGetLastError();
}

template cudaError_t launch_scale_adj_stresslet<float>(se_plan_s *, cudaStream_t, void *);
template cudaError_t launch_scale_adj_stresslet<double>(se_plan_s *, cudaStream_t, void *);

template <typename T>
cudaError_t launch_bscale(int kernel, const BSys<T> *sys, const int *blk_base, int S, int nblk, int n_rhs,
                          cudaStream_t st) {
    if (kernel == SE_STOKESLET)
        k_bscale<T, SE_STOKESLET><<<nblk, SCALE_BS, 0, st>>>(sys, blk_base, S, n_rhs);
    else if (kernel == SE_ROTLET)
        k_bscale<T, SE_ROTLET><<<nblk, SCALE_BS, 0, st>>>(sys, blk_base, S, n_rhs);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template cudaError_t launch_bscale<float>(int, const BSys<float> *, const int *, int, int, int, cudaStream_t);
template cudaError_t launch_bscale<double>(int, const BSys<double> *, const int *, int, int, int, cudaStream_t);
template cudaError_t launch_scale<float>(se_plan_s *, cudaStream_t, void *, int);
template cudaError_t launch_scale<double>(se_plan_s *, cudaStream_t, void *, int);

}  // namespace se
