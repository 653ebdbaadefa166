// Real-space part (Section 6): u^R(x_m) = sum_{0 < |x_m - x_n| <= rc} K^R(x_m - x_n) . f_n
// with the screened kernels of Section 3.2:
//   S^R     = (erfc(xi r)/r - c e) delta + (erfc(xi r)/r + c e) r^ r^            (eq. SR_Op)
//   T^R     = A1 r^ r^ r^ + A2 (delta r^ + ...),  A1 = -(2/r)[3 erfc/r + c(3 + 2 xi^2 r^2) e],
//             A2 = (4 xi^3 r / sqrt(pi)) e                                        (eq. TR_Op; A2 with
//             the factor r that the third derivative of r - Phi^H gives)
//   Omega^R = eps_jlm r^_m (erfc/r^2 + c e / r)                                   (eq. RR_Op / 2)
// c = 2 xi / sqrt(pi), e = exp(-xi^2 r^2).
//
// Cell list: points are sorted by cell (cells of width >= rc/2, x fastest), so
// one row of cells along x is a contiguous range.  One warp per target: lanes
// first compute, for each (y, z) row of cells within reach, the x-range of cells
// that can hold points within rc of this target (trimmed by the target's own
// distance to the row), then stream those candidates 32 at a time.  Candidates
// inside the cutoff are compacted (ballot + popc) into a per-warp queue, and each
// full queue of 32 pairs is evaluated with every lane busy.  FP32 partial sums are
// folded into Kahan-compensated totals after each row of cells; the final
// cross-lane sum and the update of u (which already holds u^F + u^self) are FP64.
#include "se_internal.cuh"

namespace se {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WPB = 8;
constexpr int QCAP = 64;
constexpr int MAXROWS = 49;  // reach <= 3 cells

__device__ __forceinline__ float s_erfc(float v) { return erfcf(v); }
__device__ __forceinline__ double s_erfc(double v) { return erfc(v); }
__device__ __forceinline__ float s_exp(float v) { return expf(v); }
__device__ __forceinline__ double s_exp(double v) { return exp(v); }
__device__ __forceinline__ float s_rsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double s_rsqrt(double v) { return rsqrt(v); }

struct RealConst {
    double xi, xi2, c, c3;  // xi, xi^2, 2 xi/sqrt(pi), 4 xi^3/sqrt(pi)
    double rc2;
    int reach;
};

// K^R(d) . source, added to acc (d = x_target - x_source, r2 = |d|^2 > 0)
template <typename T, int KERNEL>
__device__ __forceinline__ void pair(const RealConst &rk, T dx, T dy, T dz, T r2, const vec4<T> &f,
                                     const vec4<T> &q, T acc[3]) {
    T rinv = s_rsqrt(r2);
    T r = r2 * rinv;
    T e = s_exp(-(T)rk.xi2 * r2);
    T ec = s_erfc((T)rk.xi * r);
    T ce = (T)rk.c * e;
    T ecr = ec * rinv;
    if (KERNEL == SE_STOKESLET) {
        T A = ecr - ce;
        T B = (ecr + ce) * rinv * rinv;
        T rf = dx * f.x + dy * f.y + dz * f.z;
        T Brf = B * rf;
        acc[0] += A * f.x + Brf * dx;
        acc[1] += A * f.y + Brf * dy;
        acc[2] += A * f.z + Brf * dz;
    } else if (KERNEL == SE_ROTLET) {
        T B = (ecr + ce) * rinv * rinv;
        acc[0] += B * (f.y * dz - f.z * dy);
        acc[1] += B * (f.z * dx - f.x * dz);
        acc[2] += B * (f.x * dy - f.y * dx);
    } else {
        T hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
        T A1 = -T(2) * rinv * (T(3) * ecr + (T)rk.c * (T(3) + T(2) * (T)rk.xi2 * r2) * e);
        T A2 = (T)rk.c3 * r * e;
        T hf = hx * f.x + hy * f.y + hz * f.z;
        T hq = hx * q.x + hy * q.y + hz * q.z;
        T fq = f.x * q.x + f.y * q.y + f.z * q.z;
        T a1 = A1 * hf * hq;
        acc[0] += a1 * hx + A2 * (hx * fq + f.x * hq + q.x * hf);
        acc[1] += a1 * hy + A2 * (hy * fq + f.y * hq + q.y * hf);
        acc[2] += a1 * hz + A2 * (hz * fq + f.z * hq + q.z * hf);
    }
}

template <typename T>
__device__ __forceinline__ void kahan_add(T &s, T &comp, T x) {
    T y = x - comp;
    T t = s + y;
    comp = (t - s) - y;
    s = t;
}

template <typename T, int KERNEL>
__global__ void __launch_bounds__(WPB * 32) k_real(Geom g, RealConst rk, int N, const vec4<T> *__restrict__ xs,
                                                   const vec4<T> *__restrict__ fs,
                                                   const vec4<T> *__restrict__ qs,
                                                   const int *__restrict__ cell_start,
                                                   const int *__restrict__ perm, T *__restrict__ u,
                                                   int *__restrict__ status) {
    __shared__ vec4<T> qd_all[WPB][QCAP];
    __shared__ int qn_all[WPB][QCAP];
    __shared__ int2 seg_all[WPB][MAXROWS];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * WPB + wib;
    if (t >= N) return;
    vec4<T> *qd = qd_all[wib];
    int *qn = qn_all[wib];
    int2 *seg = seg_all[wib];
    const vec4<T> xt = xs[t];
    const double rel[3] = {(double)xt.x - g.x0[0], (double)xt.y - g.x0[1], (double)xt.z - g.x0[2]};
    int cc[3];
    for (int d = 0; d < 3; d++) cc[d] = min(max((int)(rel[d] * g.inv_cw), 0), g.ncd - 1);
    const int R = rk.reach, W = 2 * R + 1, nrows = W * W;
    // candidate range of each (y, z) row of cells
    for (int r = lane; r < nrows; r += 32) {
        int iy = cc[1] + (r % W) - R, iz = cc[2] + (r / W) - R;
        int2 sg = make_int2(0, 0);
        if (iy >= 0 && iy < g.ncd && iz >= 0 && iz < g.ncd) {
            double ylo = iy * g.cw, zlo = iz * g.cw;
            double dy = fmax(0.0, fmax(ylo - rel[1], rel[1] - (ylo + g.cw)));
            double dz = fmax(0.0, fmax(zlo - rel[2], rel[2] - (zlo + g.cw)));
            double d2 = dy * dy + dz * dz;
            if (d2 <= rk.rc2) {
                double del = sqrt(rk.rc2 - d2);
                int ixl = max(0, (int)floor((rel[0] - del) * g.inv_cw));
                int ixh = min(g.ncd - 1, (int)floor((rel[0] + del) * g.inv_cw));
                if (ixl <= ixh) {
                    int base = (iz * g.ncd + iy) * g.ncd;
                    sg = make_int2(cell_start[base + ixl], cell_start[base + ixh + 1]);
                }
            }
        }
        seg[r] = sg;
    }
    __syncwarp();
    const T rc2 = (T)rk.rc2;
    T acc[3] = {0, 0, 0}, ks[3] = {0, 0, 0}, kc[3] = {0, 0, 0};
    int cnt = 0;
    bool coinc = false;
    const unsigned lt = (1u << lane) - 1u;
    vec4<T> zero4;
    zero4.x = zero4.y = zero4.z = zero4.w = 0;
    for (int r = 0; r < nrows; r++) {
        const int2 sg = seg[r];
        for (int base = sg.x; base < sg.y; base += 32) {
            int n = base + lane;
            bool in = false;
            T dx = 0, dy = 0, dz = 0, r2 = 0;
            if (n < sg.y) {
                vec4<T> xv = xs[n];
                dx = xt.x - xv.x;
                dy = xt.y - xv.y;
                dz = xt.z - xv.z;
                r2 = dx * dx + dy * dy + dz * dz;
                in = (r2 <= rc2) && (n != t);
                if (in && r2 == T(0)) {
                    in = false;
                    coinc = true;
                }
            }
            unsigned mask = __ballot_sync(FULL, in);
            if (in) {
                int pos = cnt + __popc(mask & lt);
                vec4<T> v;
                v.x = dx; v.y = dy; v.z = dz; v.w = r2;
                qd[pos] = v;
                qn[pos] = n;
            }
            cnt += __popc(mask);
            __syncwarp();
            if (cnt >= 32) {
                vec4<T> v = qd[lane];
                int m = qn[lane];
                vec4<T> qv = (KERNEL == SE_STRESSLET) ? qs[m] : zero4;
                pair<T, KERNEL>(rk, v.x, v.y, v.z, v.w, fs[m], qv, acc);
                __syncwarp();
                if (lane < cnt - 32) {
                    qd[lane] = qd[32 + lane];
                    qn[lane] = qn[32 + lane];
                }
                cnt -= 32;
                __syncwarp();
            }
        }
        for (int d = 0; d < 3; d++) {
            kahan_add(ks[d], kc[d], acc[d]);
            acc[d] = 0;
        }
    }
    if (lane < cnt) {
        vec4<T> v = qd[lane];
        int m = qn[lane];
        vec4<T> qv = (KERNEL == SE_STRESSLET) ? qs[m] : zero4;
        pair<T, KERNEL>(rk, v.x, v.y, v.z, v.w, fs[m], qv, acc);
    }
    double tot[3];
    for (int d = 0; d < 3; d++) {
        kahan_add(ks[d], kc[d], acc[d]);
        double v = (double)ks[d] - (double)kc[d];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        tot[d] = v;
    }
    if (__any_sync(FULL, coinc) && lane == 0) atomicOr(status, FLAG_COINCIDENT);
    if (lane == 0) {
        int m = perm[t];
        for (int d = 0; d < 3; d++) u[3 * m + d] = (T)((double)u[3 * m + d] + tot[d]);
    }
}


// Position gradient of the real-space part of L = sum_m g_m . u_m (stokeslet,
// rotlet), r = x_p - x_n, over 0 < |r| <= rc:
//  stokeslet: S^R = a delta + b r r^T,
//    gx_p += r^ [a' (g_p.f_n + g_n.f_p) + b' ((g_p.r)(r.f_n) + (g_n.r)(r.f_p))]
//            + b [g_p (r.f_n) + f_n (g_p.r) + g_n (r.f_p) + f_p (g_n.r)]
//  rotlet: Omega^R_jl = eps_jlm r_m b,  c = g_p x f_n - g_n x f_p,
//    gx_p += b c + b' r^ (r.c)
// a = erfc/r - c1 e, b = (erfc/r + c1 e)/r^2, c1 = 2 xi/sqrt(pi), e = exp(-xi^2 r^2),
// a' = -c1 e/r - erfc/r^2 + 2 c1 xi^2 r e,  b' = -3 c1 e/r^3 - 3 erfc/r^4 - 2 c1 xi^2 e/r.
// Same cell traversal and compaction as the forward kernel; g of a source is
// read through the permutation.
template <typename T, int KERNEL>
__global__ void __launch_bounds__(WPB * 32) k_real_grad(Geom g, RealConst rk, int N, const vec4<T> *__restrict__ xs,
                                                        const vec4<T> *__restrict__ fs,
                                                        const int *__restrict__ cell_start,
                                                        const int *__restrict__ perm, const T *__restrict__ g_orig,
                                                        T *__restrict__ gx) {
    __shared__ vec4<T> qd_all[WPB][QCAP];
    __shared__ int qn_all[WPB][QCAP];
    __shared__ int2 seg_all[WPB][MAXROWS];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * WPB + wib;
    if (t >= N) return;
    vec4<T> *qd = qd_all[wib];
    int *qn = qn_all[wib];
    int2 *seg = seg_all[wib];
    const vec4<T> xt = xs[t];
    const vec4<T> fp = fs[t];
    const int mp = perm[t];
    const T gp[3] = {g_orig[3 * mp], g_orig[3 * mp + 1], g_orig[3 * mp + 2]};
    const double rel[3] = {(double)xt.x - g.x0[0], (double)xt.y - g.x0[1], (double)xt.z - g.x0[2]};
    int cc[3];
    for (int d = 0; d < 3; d++) cc[d] = min(max((int)(rel[d] * g.inv_cw), 0), g.ncd - 1);
    const int R = rk.reach, W = 2 * R + 1, nrows = W * W;
    for (int r = lane; r < nrows; r += 32) {
        int iy = cc[1] + (r % W) - R, iz = cc[2] + (r / W) - R;
        int2 sg = make_int2(0, 0);
        if (iy >= 0 && iy < g.ncd && iz >= 0 && iz < g.ncd) {
            double ylo = iy * g.cw, zlo = iz * g.cw;
            double dy = fmax(0.0, fmax(ylo - rel[1], rel[1] - (ylo + g.cw)));
            double dz = fmax(0.0, fmax(zlo - rel[2], rel[2] - (zlo + g.cw)));
            double d2 = dy * dy + dz * dz;
            if (d2 <= rk.rc2) {
                double del = sqrt(rk.rc2 - d2);
                int ixl = max(0, (int)floor((rel[0] - del) * g.inv_cw));
                int ixh = min(g.ncd - 1, (int)floor((rel[0] + del) * g.inv_cw));
                if (ixl <= ixh) {
                    int base = (iz * g.ncd + iy) * g.ncd;
                    sg = make_int2(cell_start[base + ixl], cell_start[base + ixh + 1]);
                }
            }
        }
        seg[r] = sg;
    }
    __syncwarp();
    const T rc2 = (T)rk.rc2;
    T acc[3] = {0, 0, 0};
    int cnt = 0;
    const unsigned lt = (1u << lane) - 1u;
    auto eval = [&](int slot) {
        vec4<T> v = qd[slot];
        int n = qn[slot];
        vec4<T> fn = fs[n];
        int mn = perm[n];
        T gn[3] = {g_orig[3 * mn], g_orig[3 * mn + 1], g_orig[3 * mn + 2]};
        T dx = v.x, dy = v.y, dz = v.z, r2 = v.w;
        T rinv = s_rsqrt(r2);
        T r = r2 * rinv;
        T e = s_exp(-(T)rk.xi2 * r2);
        T ec = s_erfc((T)rk.xi * r);
        T c1 = (T)rk.c;
        T ecr = ec * rinv;
        T rinv2 = rinv * rinv;
        T b = (ecr + c1 * e) * rinv2;
        T bp = -T(3) * c1 * e * rinv2 * rinv - T(3) * ec * rinv2 * rinv2 - T(2) * c1 * (T)rk.xi2 * e * rinv;
        T d[3] = {dx, dy, dz};
        if (KERNEL == SE_STOKESLET) {
            T ap = -c1 * e * rinv - ec * rinv2 + T(2) * c1 * (T)rk.xi2 * r * e;
            T f_n[3] = {fn.x, fn.y, fn.z}, f_p[3] = {fp.x, fp.y, fp.z};
            T gpf = gp[0] * f_n[0] + gp[1] * f_n[1] + gp[2] * f_n[2];
            T gnf = gn[0] * f_p[0] + gn[1] * f_p[1] + gn[2] * f_p[2];
            T gpr = gp[0] * dx + gp[1] * dy + gp[2] * dz;
            T gnr = gn[0] * dx + gn[1] * dy + gn[2] * dz;
            T rfn = dx * f_n[0] + dy * f_n[1] + dz * f_n[2];
            T rfp = dx * f_p[0] + dy * f_p[1] + dz * f_p[2];
            T rad = (ap * (gpf + gnf) + bp * (gpr * rfn + gnr * rfp)) * rinv;
            for (int a = 0; a < 3; a++)
                acc[a] += rad * d[a] + b * (gp[a] * rfn + f_n[a] * gpr + gn[a] * rfp + f_p[a] * gnr);
        } else {
            T c[3];
            c[0] = (gp[1] * fn.z - gp[2] * fn.y) - (gn[1] * fp.z - gn[2] * fp.y);
            c[1] = (gp[2] * fn.x - gp[0] * fn.z) - (gn[2] * fp.x - gn[0] * fp.z);
            c[2] = (gp[0] * fn.y - gp[1] * fn.x) - (gn[0] * fp.y - gn[1] * fp.x);
            T rcd = (dx * c[0] + dy * c[1] + dz * c[2]) * bp * rinv;
            for (int a = 0; a < 3; a++) acc[a] += b * c[a] + rcd * d[a];
        }
    };
    for (int r = 0; r < nrows; r++) {
        const int2 sg = seg[r];
        for (int base = sg.x; base < sg.y; base += 32) {
            int n = base + lane;
            bool in = false;
            T dx = 0, dy = 0, dz = 0, r2 = 0;
            if (n < sg.y) {
                vec4<T> xv = xs[n];
                dx = xt.x - xv.x;
                dy = xt.y - xv.y;
                dz = xt.z - xv.z;
                r2 = dx * dx + dy * dy + dz * dz;
                in = (r2 <= rc2) && (n != t) && (r2 > T(0));
            }
            unsigned mask = __ballot_sync(FULL, in);
            if (in) {
                int pos = cnt + __popc(mask & lt);
                vec4<T> v;
                v.x = dx; v.y = dy; v.z = dz; v.w = r2;
                qd[pos] = v;
                qn[pos] = n;
            }
            cnt += __popc(mask);
            __syncwarp();
            if (cnt >= 32) {
                eval(lane);
                __syncwarp();
                if (lane < cnt - 32) {
                    qd[lane] = qd[32 + lane];
                    qn[lane] = qn[32 + lane];
                }
                cnt -= 32;
                __syncwarp();
            }
        }
    }
    if (lane < cnt) eval(lane);
    double tot[3];
    for (int d = 0; d < 3; d++) {
        double v = (double)acc[d];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        tot[d] = v;
    }
    if (lane == 0)
        for (int d = 0; d < 3; d++) gx[3 * mp + d] = (T)((double)gx[3 * mp + d] + tot[d]);
}

}  // namespace

RealConst make_real_const(const se_plan_s *p) {
    RealConst rk;
    rk.xi = p->xi;
    rk.xi2 = p->xi * p->xi;
    rk.c = 2.0 * p->xi / sqrt(M_PI);
    rk.c3 = 4.0 * p->xi * p->xi * p->xi / sqrt(M_PI);
    rk.rc2 = p->rc * p->rc;
    rk.reach = (int)ceil(p->rc * p->geom.inv_cw - 1e-12);
    return rk;
}

template <typename T>
cudaError_t launch_real(se_plan_s *p, cudaStream_t st, T *u) {
    int N = (int)p->N;
    RealConst rk = make_real_const(p);
    if (rk.reach > 3) return cudaErrorInvalidValue;
    unsigned gs = (N + WPB - 1) / WPB;
    const vec4<T> *xs = (const vec4<T> *)p->b.xs_r, *fs = (const vec4<T> *)p->b.fs_r,
                  *qs = (const vec4<T> *)p->b.qs_r;
    if (p->kernel == SE_STOKESLET)
        k_real<T, SE_STOKESLET><<<gs, WPB * 32, 0, st>>>(p->geom, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, u,
                                                       p->b.status);
    else if (p->kernel == SE_STRESSLET)
        k_real<T, SE_STRESSLET><<<gs, WPB * 32, 0, st>>>(p->geom, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, u,
                                                       p->b.status);
    else
        k_real<T, SE_ROTLET><<<gs, WPB * 32, 0, st>>>(p->geom, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, u,
                                                    p->b.status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_real_grad(se_plan_s *p, cudaStream_t st, const T *g_orig, T *gx) {
    int N = (int)p->N;
    RealConst rk = make_real_const(p);
    if (rk.reach > 3) return cudaErrorInvalidValue;
    unsigned gs = (N + WPB - 1) / WPB;
    const vec4<T> *xs = (const vec4<T> *)p->b.xs_r, *fs = (const vec4<T> *)p->b.fs_r;
    if (p->kernel == SE_STOKESLET)
        k_real_grad<T, SE_STOKESLET><<<gs, WPB * 32, 0, st>>>(p->geom, rk, N, xs, fs, p->b.cnt_r, p->b.perm_r,
                                                            g_orig, gx);
    else if (p->kernel == SE_ROTLET)
        k_real_grad<T, SE_ROTLET><<<gs, WPB * 32, 0, st>>>(p->geom, rk, N, xs, fs, p->b.cnt_r, p->b.perm_r,
                                                         g_orig, gx);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template cudaError_t launch_real_grad<float>(se_plan_s *, cudaStream_t, const float *, float *);
template cudaError_t launch_real_grad<double>(se_plan_s *, cudaStream_t, const double *, double *);
template cudaError_t launch_real<float>(se_plan_s *, cudaStream_t, float *);
template cudaError_t launch_real<double>(se_plan_s *, cudaStream_t, double *);

}  // namespace se
