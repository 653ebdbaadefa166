// Step 5 of Section 5.2 (quadrature, eq. u_integr):
//   u^F(x_m) = h^3 sum_{i in P^3 support} w(y_i) (2 xi^2/(pi eta))^{3/2} exp(-2 xi^2 |x_m - y_i|^2/eta)
// (h^3 and the prefactor are folded into the scaling step), followed by the
// self-interaction correction of eq. Slimit, -4 xi/sqrt(pi) f_m (stokeslet),
// added in FP64.  One warp per target; lanes cover the (x, y) columns of the
// support and loop over z.  Also the position-gradient quadrature used by
// the backward pass.
#include "se_internal.cuh"

namespace se {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WPB = 8;  // warps per block

__device__ __forceinline__ float gexp(float v) { return expf(v); }
__device__ __forceinline__ double gexp(double v) { return exp(v); }

// Writes the 1-D weights (and the window start, and t - i0) of one point into
// the warp's shared arrays: sw[d*32 + k] = exp(-a h^2 (t_d - i0_d - k)^2).
template <typename T>
__device__ __forceinline__ void warp_weights(const vec4<T> &xv, const Geom &g, int lane, int i0[3], T *sw,
                                             T fr0[3]) {
    T ah2 = (T)(g.a * g.h * g.h);
    double rel[3] = {clamp_rel((double)xv.x - g.x0[0], g.L), clamp_rel((double)xv.y - g.x0[1], g.L),
                     clamp_rel((double)xv.z - g.x0[2], g.L)};
    for (int d = 0; d < 3; d++) {
        double t;
        int s = window_start(rel[d], g, t);
        s = min(max(s, 0), g.Mt - g.P);
        i0[d] = s;
        fr0[d] = (T)(t - (double)s);
        T fr = fr0[d] - (T)lane;
        if (lane < g.P) sw[d * 32 + lane] = gexp(-ah2 * fr * fr);
    }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(WPB * 32) k_gather(Geom g, int N, const vec4<T> *__restrict__ xs,
                                                     const int *__restrict__ perm, const T *__restrict__ w,
                                                     const T *__restrict__ f_orig, double self_coef,
                                                     T *__restrict__ u) {
    __shared__ T sw_all[WPB][96];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.x * WPB + wib;
    if (n >= N) return;
    T *sw = sw_all[wib];
    const int P = g.P, P2 = P * P;
    int i0[3];
    T fr0[3];
    warp_weights<T>(xs[n], g, lane, i0, sw, fr0);
    const size_t Mf = g.Mf, Mf2 = Mf * Mf, Mf3 = Mf2 * Mf;
    T acc0 = 0, acc1 = 0, acc2 = 0;
    for (int idx = lane; idx < P2; idx += 32) {
        int ky = idx / P, kx = idx - ky * P;
        T wxy = sw[kx] * sw[32 + ky];
        const T *col = w + ((size_t)i0[2] * Mf + (i0[1] + ky)) * Mf + (i0[0] + kx);
        T a0 = 0, a1 = 0, a2 = 0;
        for (int kz = 0; kz < P; kz++) {
            T wz = sw[64 + kz];
            const T *pz = col + kz * Mf2;
            a0 += __ldg(pz) * wz;
            a1 += __ldg(pz + Mf3) * wz;
            a2 += __ldg(pz + 2 * Mf3) * wz;
        }
        acc0 += a0 * wxy;
        acc1 += a1 * wxy;
        acc2 += a2 * wxy;
    }
    acc0 = warp_sum(acc0);
    acc1 = warp_sum(acc1);
    acc2 = warp_sum(acc2);
    if (lane == 0) {
        int m = perm[n];
        double o0 = (double)acc0, o1 = (double)acc1, o2 = (double)acc2;
        if (self_coef != 0.0) {
            o0 += self_coef * (double)f_orig[3 * m];
            o1 += self_coef * (double)f_orig[3 * m + 1];
            o2 += self_coef * (double)f_orig[3 * m + 2];
        }
        u[3 * m] = (T)o0;
        u[3 * m + 1] = (T)o1;
        u[3 * m + 2] = (T)o2;
    }
}

// Position gradient of the Fourier part of L = sum_m g_m . u_m:
//   gx_p = h^3 sum_i [g_p . w_i + f_p . w'_i] grad Gauss(x_p - y_i),
// grad Gauss(r) = -(4 xi^2/eta) r Gauss(r) = -2 a r Gauss(r); w (forward grid
// from f) and w' (adjoint grid from g) already carry h^3 and the prefactors.
template <typename T>
__global__ void __launch_bounds__(WPB * 32) k_gather_grad(Geom g, int N, const vec4<T> *__restrict__ xs,
                                                          const int *__restrict__ perm,
                                                          const T *__restrict__ wf, const T *__restrict__ wa,
                                                          const T *__restrict__ f_orig,
                                                          const T *__restrict__ g_orig, T *__restrict__ gx) {
    __shared__ T sw_all[WPB][96];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.x * WPB + wib;
    if (n >= N) return;
    T *sw = sw_all[wib];
    const int P = g.P, P2 = P * P;
    int i0[3];
    T fr0[3];
    warp_weights<T>(xs[n], g, lane, i0, sw, fr0);
    const int m = perm[n];
    const T gm[3] = {g_orig[3 * m], g_orig[3 * m + 1], g_orig[3 * m + 2]};
    const T fm[3] = {f_orig[3 * m], f_orig[3 * m + 1], f_orig[3 * m + 2]};
    const size_t Mf = g.Mf, Mf2 = Mf * Mf, Mf3 = Mf2 * Mf;
    // distance (grid units) from the target to support point k along d: fr0[d] - k
    // d/dx_d Gauss = -2 a h (fr0 - k) Gauss  (x - y = (t - i) h)
    T acc[3] = {0, 0, 0};
    for (int idx = lane; idx < P2; idx += 32) {
        int ky = idx / P, kx = idx - ky * P;
        T wx = sw[kx], wy = sw[32 + ky];
        T dx = fr0[0] - (T)kx, dy = fr0[1] - (T)ky;
        const size_t off = ((size_t)i0[2] * Mf + (i0[1] + ky)) * Mf + (i0[0] + kx);
        T s0 = 0, sz = 0;  // sum_kz s wz, sum_kz s wz dz
        for (int kz = 0; kz < P; kz++) {
            T wz = sw[64 + kz];
            size_t o = off + kz * Mf2;
            T s = gm[0] * __ldg(wf + o) + gm[1] * __ldg(wf + o + Mf3) + gm[2] * __ldg(wf + o + 2 * Mf3) +
                  fm[0] * __ldg(wa + o) + fm[1] * __ldg(wa + o + Mf3) + fm[2] * __ldg(wa + o + 2 * Mf3);
            s0 += s * wz;
            sz += s * wz * (fr0[2] - (T)kz);
        }
        T wxy = wx * wy;
        acc[0] += s0 * wxy * dx;
        acc[1] += s0 * wxy * dy;
        acc[2] += sz * wxy;
    }
    T c = (T)(-2.0 * g.a * g.h);
    for (int d = 0; d < 3; d++) acc[d] = warp_sum(acc[d]);
    if (lane == 0) {
        gx[3 * m] = c * acc[0];
        gx[3 * m + 1] = c * acc[1];
        gx[3 * m + 2] = c * acc[2];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_gather(se_plan_s *p, cudaStream_t st, const void *wgrid, const T *f_orig, T *u) {
    int N = (int)p->N;
    double self_coef = (p->kernel == SE_STOKESLET) ? -4.0 * p->xi / sqrt(M_PI) : 0.0;
    k_gather<T><<<(N + WPB - 1) / WPB, WPB * 32, 0, st>>>(p->geom, N, (const vec4<T> *)p->b.xs_t, p->b.perm_t,
                                                          (const T *)wgrid, f_orig, self_coef, u);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_grad(se_plan_s *p, cudaStream_t st, const void *w_fwd, const void *w_adj,
                               const T *f_orig, const T *g_orig, T *gx) {
    int N = (int)p->N;
    k_gather_grad<T><<<(N + WPB - 1) / WPB, WPB * 32, 0, st>>>(p->geom, N, (const vec4<T> *)p->b.xs_t,
                                                               p->b.perm_t, (const T *)w_fwd, (const T *)w_adj,
                                                               f_orig, g_orig, gx);
    return cudaGetLastError();
}

template cudaError_t launch_gather<float>(se_plan_s *, cudaStream_t, const void *, const float *, float *);
template cudaError_t launch_gather<double>(se_plan_s *, cudaStream_t, const void *, const double *, double *);
template cudaError_t launch_gather_grad<float>(se_plan_s *, cudaStream_t, const void *, const void *,
                                               const float *, const float *, float *);
template cudaError_t launch_gather_grad<double>(se_plan_s *, cudaStream_t, const void *, const void *,
                                                const double *, const double *, double *);

}  // namespace se
