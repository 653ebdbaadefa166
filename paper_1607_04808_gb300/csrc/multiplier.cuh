// The Fourier-space multipliers of step 3 (Section 5.2, eq. gridfcnsc) at one
// wave vector, shared by the scaling pass (scale.cu) and the fused z-direction
// transform and scaling (zfft.cu):
//   w^_j(k) = e^{-(1-eta) k^2 / 4 xi^2} A_j..(k) g^_..(k)
// with the multipliers of eqs. AS, AT, AR where the truncated harmonic /
// biharmonic transform is replaced by the precomputed mollified kernel G~^(k)
// (Section 4.3, stored as the (Mt+1)^3 octant of a real, even array).
//   stokeslet  A_jl  = -(k^2 d_jl - k_j k_l)(1 + k^2/4xi^2) G~^
//   stresslet  A_jlm = -i[(k_m d_jl + k_j d_lm + k_l d_mj) k^2 - 2 k_j k_l k_m](1 + k^2/4xi^2) G~^
//   rotlet     A_jl  = -i eps_jlm k_m G~^
// The odd symbols are the transform of the kernel under f^(k) = int f e^{-ik.x}
// (d/dx_m -> +i k_m), and the rotlet is the definition eps_jlm r_m / r^3.
// The constant `norm` folds in the inverse-FFT normalisation 1/Mf^3, the
// quadrature weight h^3 (Section 5.2 step 5) and the two Gaussian prefactors
// (2 xi^2/(pi eta))^{3/2} of eqs. Hx and u_integr.
#pragma once

#include "se_internal.cuh"

namespace se {

__device__ __forceinline__ float mexp(float v) { return expf(v); }
__device__ __forceinline__ double mexp(double v) { return exp(v); }

// The wave vector of half-spectrum point (kx, ky, kz) of the [kz][ky][kx] R2C
// layout and the index of |k| in the stored octant of the precomputed kernel.
template <typename T>
__device__ __forceinline__ size_t kpoint3(const ScaleConst &sc, int kx, int ky, int kz, T kv[3]) {
    const int bx = (kx == sc.mt[0]) ? -sc.mt[0] : kx;
    const int by = (ky < sc.mt[1]) ? ky : ky - sc.mf[1];
    const int bz = (kz < sc.mt[2]) ? kz : kz - sc.mf[2];
    kv[0] = (T)sc.dk[0] * bx;
    kv[1] = (T)sc.dk[1] * by;
    kv[2] = (T)sc.dk[2] * bz;
    return ((size_t)abs(bz) * (sc.mt[1] + 1) + abs(by)) * (sc.mt[0] + 1) + abs(bx);
}

// The multiplier applied to the source components g (3, or the stresslet's 6
// symmetric ones xx, yy, zz, xy, xz, yz) at wave vector kv with the kernel
// value G: the three components o of w^.
template <typename T, int KERNEL>
__device__ __forceinline__ void apply_multiplier(const ScaleConst &sc, const T kv[3], T G, const cplx<T> *g,
                                                 cplx<T> o[3]) {
    using C = cplx<T>;
    const T k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
    T F = (T)sc.norm * G * mexp((T)sc.ecoef * k2);
    if (KERNEL != SE_ROTLET) F *= (T(1) + k2 * (T)sc.inv4xi2);
    if (KERNEL == SE_STOKESLET) {
        C kg;
        kg.x = kv[0] * g[0].x + kv[1] * g[1].x + kv[2] * g[2].x;
        kg.y = kv[0] * g[0].y + kv[1] * g[1].y + kv[2] * g[2].y;
        for (int j = 0; j < 3; j++) {
            o[j].x = -F * (k2 * g[j].x - kv[j] * kg.x);
            o[j].y = -F * (k2 * g[j].y - kv[j] * kg.y);
        }
    } else if (KERNEL == SE_ROTLET) {
        // (g x k)_j = eps_jlm g_l k_m ; multiply by -i F: (a + ib)(-i) = b - ia
        C cr[3];
        cr[0].x = g[1].x * kv[2] - g[2].x * kv[1];
        cr[0].y = g[1].y * kv[2] - g[2].y * kv[1];
        cr[1].x = g[2].x * kv[0] - g[0].x * kv[2];
        cr[1].y = g[2].y * kv[0] - g[0].y * kv[2];
        cr[2].x = g[0].x * kv[1] - g[1].x * kv[0];
        cr[2].y = g[0].y * kv[1] - g[1].y * kv[0];
        for (int j = 0; j < 3; j++) {
            o[j].x = F * cr[j].y;
            o[j].y = -F * cr[j].x;
        }
    } else {
        // symmetric source s: xx, yy, zz, xy, xz, yz
        const C *s = g;
        C sk[3], tr, ksk;
        sk[0].x = s[0].x * kv[0] + s[3].x * kv[1] + s[4].x * kv[2];
        sk[0].y = s[0].y * kv[0] + s[3].y * kv[1] + s[4].y * kv[2];
        sk[1].x = s[3].x * kv[0] + s[1].x * kv[1] + s[5].x * kv[2];
        sk[1].y = s[3].y * kv[0] + s[1].y * kv[1] + s[5].y * kv[2];
        sk[2].x = s[4].x * kv[0] + s[5].x * kv[1] + s[2].x * kv[2];
        sk[2].y = s[4].y * kv[0] + s[5].y * kv[1] + s[2].y * kv[2];
        tr.x = s[0].x + s[1].x + s[2].x;
        tr.y = s[0].y + s[1].y + s[2].y;
        ksk.x = kv[0] * sk[0].x + kv[1] * sk[1].x + kv[2] * sk[2].x;
        ksk.y = kv[0] * sk[0].y + kv[1] * sk[1].y + kv[2] * sk[2].y;
        for (int j = 0; j < 3; j++) {
            // b = k^2 (2 (s k)_j + k_j tr s) - 2 k_j (k.s.k); out = -i F b
            const T bx_ = k2 * (T(2) * sk[j].x + kv[j] * tr.x) - T(2) * kv[j] * ksk.x;
            const T by_ = k2 * (T(2) * sk[j].y + kv[j] * tr.y) - T(2) * kv[j] * ksk.y;
            o[j].x = F * by_;
            o[j].y = -F * bx_;
        }
    }
}

}  // namespace se
