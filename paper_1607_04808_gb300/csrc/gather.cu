// Step 5 of Section 5.2 (quadrature, eq. u_integr):
//   u^F(x_m) = h^3 sum_{i in P^3 support} w(y_i) (2 xi^2/(pi eta))^{3/2} exp(-2 xi^2 |x_m - y_i|^2/eta)
// (h^3 and the prefactor are folded into the scaling step), followed by the
// self-interaction correction of eq. Slimit, -4 xi/sqrt(pi) f_m (stokeslet),
// added in FP64.  One warp per target; lanes cover the (x, y) columns of the
// support and loop over z, so each load instruction reads a few contiguous
// rows of the grid.  Also the position-gradient quadrature of the backward pass.
#include "se_internal.cuh"

namespace se {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WPB = 8;  // warps per block

__device__ __forceinline__ float gexp(float v) { return __expf(v); }
__device__ __forceinline__ double gexp(double v) { return exp(v); }

// 1-D weights of the P support points of the target along each dimension into
// the warp's shared arrays sw[d][k]; fr[d] = t_d - i0_d (grid units).
template <typename T>
__device__ __forceinline__ void warp_weights(const vec4<T> &xv, const GP<T> &g, int lane, int i0[3],
                                             T (*sw)[32], T fr[3]) {
    unpack3(get_tag(xv), i0[0], i0[1], i0[2]);
    const T rel[3] = {xv.x - g.x0[0], xv.y - g.x0[1], xv.z - g.x0[2]};
    for (int d = 0; d < 3; d++) {
        fr[d] = (rel[d] * g.inv_h + g.half_ext) - (T)i0[d];
        T t = fr[d] - (T)lane;
        if (lane < g.P) sw[d][lane] = gexp(-g.ah2 * t * t);
    }
    __syncwarp();
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// One target (sorted position n, original index m): lanes cover the (x, y)
// columns of the support (NIT static slots, P <= 16, or a strided loop) and
// loop over z; the weights are computed once and applied to the n_rhs groups
// of three grids (group r at w + 3 r mf_x mf_y mf_z).  u and f_orig hold n_rhs
// three-vectors per point.
template <typename T, int NIT>
__device__ __forceinline__ void gather_point(const GP<T> &g, const vec4<T> &xv, int m, const T *__restrict__ w,
                                             int n_rhs, const T *__restrict__ f_orig, double self_coef,
                                             T *__restrict__ u, int lane, T (*sw)[32]) {
    const int P = g.P, P2 = P * P;
    int i0[3];
    T fr[3];
    warp_weights<T>(xv, g, lane, i0, sw, fr);
    const size_t Mf = g.mf[0], Mfy = g.mf[1], Mf2 = Mf * Mfy, Mf3 = vol(g);
    for (int r = 0; r < n_rhs; r++) {
        const T *base = w + (size_t)r * 3 * Mf3 + ((size_t)i0[2] * Mfy + i0[1]) * Mf + i0[0];
        T acc0 = 0, acc1 = 0, acc2 = 0;
        auto column = [&](int kx, int ky) {
            const T wxy = sw[0][kx] * sw[1][ky];
            const T *col = base + (size_t)ky * Mf + kx;
            T a0 = 0, a1 = 0, a2 = 0;
            for (int kz = 0; kz < P; kz++) {
                const T wz = sw[2][kz];
                const T *pz = col + kz * Mf2;
                a0 += __ldg(pz) * wz;
                a1 += __ldg(pz + Mf3) * wz;
                a2 += __ldg(pz + 2 * Mf3) * wz;
            }
            acc0 += a0 * wxy;
            acc1 += a1 * wxy;
            acc2 += a2 * wxy;
        };
        if (NIT > 0) {
#pragma unroll
            for (int it = 0; it < (NIT > 0 ? NIT : 1); it++) {
                int idx = it * 32 + lane;
                if (idx < P2) {
                    int ky = idx / P;
                    column(idx - ky * P, ky);
                }
            }
        } else {
            for (int idx = lane; idx < P2; idx += 32) {
                int ky = idx / P;
                column(idx - ky * P, ky);
            }
        }
        acc0 = warp_sum(acc0);
        acc1 = warp_sum(acc1);
        acc2 = warp_sum(acc2);
        if (lane < 3) {
            // lanes 0..2 each finish one component (FP64 self-interaction correction)
            const size_t o3 = ((size_t)m * n_rhs + r) * 3 + lane;
            const T a = lane == 0 ? acc0 : (lane == 1 ? acc1 : acc2);
            double o = (double)a;
            if (self_coef != 0.0) o += self_coef * (double)f_orig[o3];
            u[o3] = (T)o;
        }
    }
}

template <typename T, int NIT>
__global__ void __launch_bounds__(WPB * 32) k_gather(GP<T> g, int N, const vec4<T> *__restrict__ xs,
                                                     const int *__restrict__ perm, const T *__restrict__ w,
                                                     const T *__restrict__ f_orig, double self_coef,
                                                     T *__restrict__ u) {
    __shared__ T sw_all[WPB][3][32];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.x * WPB + wib;
    if (n >= N) return;
    gather_point<T, NIT>(g, xs[n], perm[n], w, 1, f_orig, self_coef, u, lane, sw_all[wib]);
}

// Batched: one warp per sorted point of the concatenated systems; the point's
// system is the range of `off` that holds its sorted position.
template <typename T, int NIT>
__global__ void __launch_bounds__(WPB * 32) k_bgather(const BSys<T> *__restrict__ sys, const int *__restrict__ off,
                                                      int S, int Ntot, int n_rhs, const vec4<T> *__restrict__ xs,
                                                      const int *__restrict__ perm, const T *__restrict__ f_orig,
                                                      T *__restrict__ u) {
    __shared__ T sw_all[WPB][3][32];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.x * WPB + wib;
    if (n >= Ntot) return;
    const BSys<T> &B = sys[find_range(off, S, n)];
    const GP<T> g = B.g;
    gather_point<T, NIT>(g, xs[n], perm[n], B.wgrid, n_rhs, f_orig, B.self_coef, u, lane, sw_all[wib]);
}

// Stresslet backward, strengths: the adjoint tensor field V_lk (6 grids: xx, yy,
// zz, xy, xz, yz) gathered at each point and contracted,
//   gf_p,l = V_lk(x_p) q_p,k,   gq_p,k = V_lk(x_p) f_p,l  (V symmetric).
// Outputs are overwritten (either may be NULL).
template <typename T>
__global__ void __launch_bounds__(WPB * 32) k_gather_adjT(GP<T> g, int N, const vec4<T> *__restrict__ xs,
                                                          const int *__restrict__ perm, const T *__restrict__ V,
                                                          const T *__restrict__ f_orig,
                                                          const T *__restrict__ q_orig, T *__restrict__ gf,
                                                          T *__restrict__ gq) {
    __shared__ T sw_all[WPB][3][32];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.x * WPB + wib;
    if (n >= N) return;
    T(*sw)[32] = sw_all[wib];
    const int P = g.P, P2 = P * P;
    int i0[3];
    T fr[3];
    warp_weights<T>(xs[n], g, lane, i0, sw, fr);
    const size_t Mf = g.mf[0], Mfy = g.mf[1], Mf2 = Mf * Mfy, Mf3 = vol(g);
    const T *base = V + ((size_t)i0[2] * Mfy + i0[1]) * Mf + i0[0];
    T acc[6] = {0, 0, 0, 0, 0, 0};
    for (int idx = lane; idx < P2; idx += 32) {
        const int ky = idx / P, kx = idx - ky * P;
        const T wxy = sw[0][kx] * sw[1][ky];
        const T *col = base + (size_t)ky * Mf + kx;
        T a[6] = {0, 0, 0, 0, 0, 0};
        for (int kz = 0; kz < P; kz++) {
            const T wz = sw[2][kz];
            const T *pz = col + kz * Mf2;
#pragma unroll
            for (int c = 0; c < 6; c++) a[c] += __ldg(pz + c * Mf3) * wz;
        }
#pragma unroll
        for (int c = 0; c < 6; c++) acc[c] += a[c] * wxy;
    }
#pragma unroll
    for (int c = 0; c < 6; c++) acc[c] = warp_sum(acc[c]);
    if (lane < 3) {
        const int m = perm[n];
        // row `lane` of the symmetric V: (xx, xy, xz), (xy, yy, yz), (xz, yz, zz)
        const T row[3] = {lane == 0 ? acc[0] : (lane == 1 ? acc[3] : acc[4]),
                          lane == 0 ? acc[3] : (lane == 1 ? acc[1] : acc[5]),
                          lane == 0 ? acc[4] : (lane == 1 ? acc[5] : acc[2])};
        if (gf) gf[3 * m + lane] = row[0] * q_orig[3 * m] + row[1] * q_orig[3 * m + 1] + row[2] * q_orig[3 * m + 2];
        if (gq) gq[3 * m + lane] = row[0] * f_orig[3 * m] + row[1] * f_orig[3 * m + 1] + row[2] * f_orig[3 * m + 2];
    }
}

// Position gradient of the Fourier part of L = sum_m g_m . u_m:
//   gx_p = h^3 sum_i [g_p . w_i + f_p . w'_i] grad Gauss(x_p - y_i),
// grad Gauss(r) = -(4 xi^2/eta) r Gauss(r); w (forward grid from f) and w'
// (adjoint grid from g) already carry h^3 and the prefactors.  In grid units
// x - y = (t - i) h, so d/dx_d Gauss = -2 a h (fr_d - k) Gauss.
// Stresslet (NA = 6): w' is the adjoint tensor field V (xx, yy, zz, xy, xz,
// yz) and f_p . w' becomes sum_lk f_p,l q_p,k V_lk.
template <typename T, int NA>
__global__ void __launch_bounds__(WPB * 32) k_gather_grad(GP<T> g, T c_grad, int N, const vec4<T> *__restrict__ xs,
                                                          const int *__restrict__ perm,
                                                          const T *__restrict__ wf, const T *__restrict__ wa,
                                                          const T *__restrict__ f_orig,
                                                          const T *__restrict__ q_orig,
                                                          const T *__restrict__ g_orig, T *__restrict__ gx) {
    __shared__ T sw_all[WPB][3][32];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.x * WPB + wib;
    if (n >= N) return;
    T(*sw)[32] = sw_all[wib];
    const int P = g.P, P2 = P * P;
    int i0[3];
    T fr[3];
    warp_weights<T>(xs[n], g, lane, i0, sw, fr);
    const int m = perm[n];
    const T gm[3] = {g_orig[3 * m], g_orig[3 * m + 1], g_orig[3 * m + 2]};
    const T fm[3] = {f_orig[3 * m], f_orig[3 * m + 1], f_orig[3 * m + 2]};
    T cm[NA];
    if (NA == 3) {
        for (int c = 0; c < NA; c++) cm[c] = fm[c % 3];
    } else {
        const T qm[3] = {q_orig[3 * m], q_orig[3 * m + 1], q_orig[3 * m + 2]};
        const int L_[6] = {0, 1, 2, 0, 0, 1}, K_[6] = {0, 1, 2, 1, 2, 2};
        for (int c = 0; c < NA; c++)
            cm[c] = (c < 3) ? fm[c] * qm[c] : fm[L_[c]] * qm[K_[c]] + fm[K_[c]] * qm[L_[c]];
    }
    const size_t Mf = g.mf[0], Mfy = g.mf[1], Mf2 = Mf * Mfy, Mf3 = vol(g);
    T acc[3] = {0, 0, 0};
    for (int idx = lane; idx < P2; idx += 32) {
        int ky = idx / P, kx = idx - ky * P;
        T wx = sw[0][kx], wy = sw[1][ky];
        T dx = fr[0] - (T)kx, dy = fr[1] - (T)ky;
        const size_t off = ((size_t)i0[2] * Mfy + (i0[1] + ky)) * Mf + (i0[0] + kx);
        T s0 = 0, sz = 0;  // sum_kz s wz, sum_kz s wz dz
        for (int kz = 0; kz < P; kz++) {
            T wz = sw[2][kz];
            size_t o = off + kz * Mf2;
            T s = gm[0] * __ldg(wf + o) + gm[1] * __ldg(wf + o + Mf3) + gm[2] * __ldg(wf + o + 2 * Mf3);
#pragma unroll
            for (int c = 0; c < NA; c++) s += cm[c] * __ldg(wa + o + c * Mf3);
            s0 += s * wz;
            sz += s * wz * (fr[2] - (T)kz);
        }
        T wxy = wx * wy;
        acc[0] += s0 * wxy * dx;
        acc[1] += s0 * wxy * dy;
        acc[2] += sz * wxy;
    }
    for (int d = 0; d < 3; d++) acc[d] = warp_sum(acc[d]);
    if (lane == 0) {
        gx[3 * m] = c_grad * acc[0];
        gx[3 * m + 1] = c_grad * acc[1];
        gx[3 * m + 2] = c_grad * acc[2];
    }
}

}  // namespace

template <typename T>
cudaError_t launch_gather(se_plan_s *p, cudaStream_t st, const void *wgrid, const T *f_orig, T *u) {
    if (sizeof(T) == 4 && p->colk)
        return launch_gather_col(p, st, wgrid, (const float *)f_orig, (float *)u);
    int N = (int)p->N;
    double self_coef = (p->kernel == SE_STOKESLET) ? -4.0 * p->xi / sqrt(M_PI) : 0.0;
    dim3 gs((N + WPB - 1) / WPB), bs(WPB * 32);
    const vec4<T> *xs = (const vec4<T> *)p->b.xs_t;
    const T *w = (const T *)wgrid;
    const GP<T> &g = gp<T>(p);
    switch ((p->P * p->P + 31) / 32) {
        case 1: k_gather<T, 1><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
        case 2: k_gather<T, 2><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
        case 3: k_gather<T, 3><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
        case 4: k_gather<T, 4><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
        case 5: k_gather<T, 5><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
        case 6: k_gather<T, 6><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
        case 7: k_gather<T, 7><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
        case 8: k_gather<T, 8><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
        default: k_gather<T, 0><<<gs, bs, 0, st>>>(g, N, xs, p->b.perm_t, w, f_orig, self_coef, u); break;
    }
    p->launches++;
    return cudaGetLastError();
}

#ifndef SE_GRAD_COL
#define SE_GRAD_COL 1
#endif

template <typename T>
cudaError_t launch_gather_grad(se_plan_s *p, cudaStream_t st, const void *w_fwd, const void *w_adj,
                               const T *f_orig, const T *q_orig, const T *g_orig, T *gx) {
    // FP32 column plans, stokeslet and rotlet (the stresslet's three passes at
    // P = 14 cost more than its single pass over the global grids)
    if (sizeof(T) == 4 && p->colk && SE_GRAD_COL && p->kernel != SE_STRESSLET)
        return launch_gather_grad_col(p, st, (const float *)w_fwd, (const float *)w_adj, (const float *)f_orig,
                                      (const float *)q_orig, (const float *)g_orig, (float *)gx);
    int N = (int)p->N;
    T c_grad = (T)(-2.0 * p->geom.a * p->h);
    const unsigned gs = (N + WPB - 1) / WPB;
    if (p->kernel == SE_STRESSLET)
        k_gather_grad<T, 6><<<gs, WPB * 32, 0, st>>>(gp<T>(p), c_grad, N, (const vec4<T> *)p->b.xs_t, p->b.perm_t,
                                                     (const T *)w_fwd, (const T *)w_adj, f_orig, q_orig, g_orig,
                                                     gx);
    else
        k_gather_grad<T, 3><<<gs, WPB * 32, 0, st>>>(gp<T>(p), c_grad, N, (const vec4<T> *)p->b.xs_t, p->b.perm_t,
                                                     (const T *)w_fwd, (const T *)w_adj, f_orig, q_orig, g_orig,
                                                     gx);
    p->launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bgather(const BSys<T> *sys, const int *off, int S, int Ntot, int P, int n_rhs, const Buffers &b,
                           const T *f, T *u, cudaStream_t st) {
    dim3 gs((Ntot + WPB - 1) / WPB), bs(WPB * 32);
    const vec4<T> *xs = (const vec4<T> *)b.xs_t;
    switch ((P * P + 31) / 32) {
        case 1: k_bgather<T, 1><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
        case 2: k_bgather<T, 2><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
        case 3: k_bgather<T, 3><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
        case 4: k_bgather<T, 4><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
        case 5: k_bgather<T, 5><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
        case 6: k_bgather<T, 6><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
        case 7: k_bgather<T, 7><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
        case 8: k_bgather<T, 8><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
        default: k_bgather<T, 0><<<gs, bs, 0, st>>>(sys, off, S, Ntot, n_rhs, xs, b.perm_t, f, u); break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_bgather<float>(const BSys<float> *, const int *, int, int, int, int, const Buffers &,
                                           const float *, float *, cudaStream_t);
template cudaError_t launch_bgather<double>(const BSys<double> *, const int *, int, int, int, int, const Buffers &,
                                            const double *, double *, cudaStream_t);
// SE_ADJ_COL: the FP32 stresslet adjoint gather on the shared-memory tiles
#ifndef SE_ADJ_COL
#define SE_ADJ_COL 1
#endif
template <typename T>
cudaError_t launch_gather_adjT(se_plan_s *p, cudaStream_t st, const void *V, const T *f_orig, const T *q_orig,
                               T *gf, T *gq) {
    if (sizeof(T) == 4 && p->colk && SE_ADJ_COL)
        return launch_gather_adj_col(p, st, (const float *)V, (const float *)f_orig, (const float *)q_orig,
                                     (float *)gf, (float *)gq);
    const int N = (int)p->N;
    k_gather_adjT<T><<<(N + WPB - 1) / WPB, WPB * 32, 0, st>>>(gp<T>(p), N, (const vec4<T> *)p->b.xs_t, p->b.perm_t,
                                                              (const T *)V, f_orig, q_orig, gf, gq);
    p->launches++;
    return cudaGetLastError();
}

template cudaError_t launch_gather_adjT<float>(se_plan_s *, cudaStream_t, const void *, const float *,
                                               const float *, float *, float *);
template cudaError_t launch_gather_adjT<double>(se_plan_s *, cudaStream_t, const void *, const double *,
                                                const double *, double *, double *);
// Gather at separate targets (binned into bt): the Fourier part only, no self term.
template <typename T>
cudaError_t launch_gather_targets(se_plan_s *p, cudaStream_t st, const Buffers &bt, int Nt, const void *wgrid,
                                  T *ut) {
    if (sizeof(T) == 4 && p->colk) return launch_gather_col_set(p, st, bt, wgrid, nullptr, 0.0, (float *)ut, Nt);
    dim3 gs((Nt + WPB - 1) / WPB), bs(WPB * 32);
    const vec4<T> *xs = (const vec4<T> *)bt.xs_t;
    const T *w = (const T *)wgrid;
    const GP<T> &g = gp<T>(p);
    switch ((p->P * p->P + 31) / 32) {
        case 1: k_gather<T, 1><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
        case 2: k_gather<T, 2><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
        case 3: k_gather<T, 3><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
        case 4: k_gather<T, 4><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
        case 5: k_gather<T, 5><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
        case 6: k_gather<T, 6><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
        case 7: k_gather<T, 7><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
        case 8: k_gather<T, 8><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
        default: k_gather<T, 0><<<gs, bs, 0, st>>>(g, Nt, xs, bt.perm_t, w, nullptr, 0.0, ut); break;
    }
    p->launches++;
    return cudaGetLastError();
}

template cudaError_t launch_gather_targets<float>(se_plan_s *, cudaStream_t, const Buffers &, int, const void *,
                                                  float *);
template cudaError_t launch_gather_targets<double>(se_plan_s *, cudaStream_t, const Buffers &, int, const void *,
                                                   double *);
template cudaError_t launch_gather<float>(se_plan_s *, cudaStream_t, const void *, const float *, float *);
template cudaError_t launch_gather<double>(se_plan_s *, cudaStream_t, const void *, const double *, double *);
template cudaError_t launch_gather_grad<float>(se_plan_s *, cudaStream_t, const void *, const void *,
                                               const float *, const float *, const float *, float *);
template cudaError_t launch_gather_grad<double>(se_plan_s *, cudaStream_t, const void *, const void *,
                                                const double *, const double *, const double *, double *);

}  // namespace se
