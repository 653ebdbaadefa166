// Real-space part (Section 6): u^R(x_m) = sum_{0 < |x_m - x_n| <= rc} K^R(x_m - x_n) . f_n
// with the screened kernels of Section 3.2:
//   S^R     = (erfc(xi r)/r - c e) delta + (erfc(xi r)/r + c e) r^ r^            (eq. SR_Op)
//   T^R     = A1 r^ r^ r^ + A2 (delta r^ + ...),  A1 = -(2/r)[3 erfc/r + c(3 + 2 xi^2 r^2) e],
//             A2 = (4 xi^3 r / sqrt(pi)) e                                        (eq. TR_Op; A2 with
//             the factor r that the third derivative of r - Phi^H gives)
//   Omega^R = eps_jlm r^_m (erfc/r^2 + c e / r)                                   (eq. RR_Op / 2)
// c = 2 xi / sqrt(pi), e = exp(-xi^2 r^2).  In FP32, erfc(x) = e Q(2/(2+x)) with
// the fitted polynomial Q ~ erfcx of erfc_poly.cuh, so one exponential serves
// both terms; FP64 uses the library erfc.
//
// Cell list: points are sorted by cell (cells of width >= rc/3, x fastest), so
// one row of cells along x is a contiguous range.  One warp per target: lanes
// first compute, for each (y, z) row of cells within reach, the x-range of cells
// that can hold points within rc of this target (trimmed by the target's own
// distance to the row), then stream those candidates 32 at a time.  Candidates
// inside the cutoff are compacted (ballot + popc) into a per-warp queue, and each
// full queue of 32 pairs is evaluated with every lane busy.  FP32 partial sums are
// folded into Kahan-compensated totals after each row of cells; the final
// cross-lane sum and the update of u (which already holds u^F + u^self) are FP64.
#include "erfc_poly.cuh"
#include "se_internal.cuh"

namespace se {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WPB = 8;
constexpr int QCAP = 64;
constexpr int MAXROWS = 49;  // reach <= 3 cells

template <typename T>
struct RC {
    T xi, xi2, c, c3, rc2;  // xi, xi^2, 2 xi/sqrt(pi), 4 xi^3/sqrt(pi), rc^2
    int reach;
};

// rsqrt, exp(-xi^2 r^2) and erfc(xi r) of one pair
__device__ __forceinline__ void radial(const RC<float> &rk, float r2, float &rinv, float &r, float &e, float &ec) {
    rinv = rsqrtf(r2);
    r = r2 * rinv;
    e = __expf(-rk.xi2 * r2);
    const float x = rk.xi * r;
    const float t = __fdividef(2.0f, 2.0f + x);
    float q = ERFC_Q[SE_ERFC_DEG];
#pragma unroll
    for (int k = SE_ERFC_DEG - 1; k >= 0; k--) q = fmaf(q, t, ERFC_Q[k]);
    ec = e * q;
}
__device__ __forceinline__ void radial(const RC<double> &rk, double r2, double &rinv, double &r, double &e,
                                       double &ec) {
    rinv = rsqrt(r2);
    r = r2 * rinv;
    e = exp(-rk.xi2 * r2);
    ec = erfc(rk.xi * r);
}

// K^R(d) . source, added to acc (d = x_target - x_source, r2 = |d|^2 > 0)
template <typename T, int KERNEL>
__device__ __forceinline__ void pair(const RC<T> &rk, T dx, T dy, T dz, T r2, const vec4<T> &f,
                                     const vec4<T> &q, T acc[3]) {
    T rinv, r, e, ec;
    radial(rk, r2, rinv, r, e, ec);
    const T ce = rk.c * e;
    const T ecr = ec * rinv;
    if (KERNEL == SE_STOKESLET) {
        const T A = ecr - ce;
        const T B = (ecr + ce) * rinv * rinv;
        const T Brf = B * (dx * f.x + dy * f.y + dz * f.z);
        acc[0] += A * f.x + Brf * dx;
        acc[1] += A * f.y + Brf * dy;
        acc[2] += A * f.z + Brf * dz;
    } else if (KERNEL == SE_ROTLET) {
        const T B = (ecr + ce) * rinv * rinv;
        acc[0] += B * (f.y * dz - f.z * dy);
        acc[1] += B * (f.z * dx - f.x * dz);
        acc[2] += B * (f.x * dy - f.y * dx);
    } else {
        const T hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
        const T A1 = -T(2) * rinv * (T(3) * ecr + rk.c * (T(3) + T(2) * rk.xi2 * r2) * e);
        const T A2 = rk.c3 * r * e;
        const T hf = hx * f.x + hy * f.y + hz * f.z;
        const T hq = hx * q.x + hy * q.y + hz * q.z;
        const T fq = f.x * q.x + f.y * q.y + f.z * q.z;
        const T a1 = A1 * hf * hq;
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

// For each (y, z) row of cells around the target: the contiguous range of
// sorted points in the cells whose x-extent meets [x - del, x + del], del the
// half-chord of the cutoff sphere at the row's distance.  A small relative
// margin keeps rounding from dropping a cell; the exact test comes later.
template <typename T>
__device__ __forceinline__ void row_segments(const GP<T> &g, const RC<T> &rk, const vec4<T> &xt,
                                             const int *__restrict__ cell_start, int lane, int2 *seg) {
    int cc[3];
    unpack3(get_tag(xt), cc[0], cc[1], cc[2]);
    const T rel[3] = {xt.x - g.x0[0], xt.y - g.x0[1], xt.z - g.x0[2]};
    const T rc2m = rk.rc2 * T(1.0001);
    const int R = rk.reach, W = 2 * R + 1, nrows = W * W;
    for (int r = lane; r < nrows; r += 32) {
        int iy = cc[1] + (r % W) - R, iz = cc[2] + (r / W) - R;
        int2 sg = make_int2(0, 0);
        if (iy >= 0 && iy < g.ncd && iz >= 0 && iz < g.ncd) {
            const T ylo = iy * g.cw, zlo = iz * g.cw;
            const T dy = max(T(0), max(ylo - rel[1], rel[1] - (ylo + g.cw)));
            const T dz = max(T(0), max(zlo - rel[2], rel[2] - (zlo + g.cw)));
            const T d2 = dy * dy + dz * dz;
            if (d2 <= rc2m) {
                const T del = sqrt(rc2m - d2) + T(1e-4) * g.cw;
                const int ixl = max(0, (int)floor((rel[0] - del) * g.inv_cw));
                const int ixh = min(g.ncd - 1, (int)floor((rel[0] + del) * g.inv_cw));
                if (ixl <= ixh) {
                    const int base = (iz * g.ncd + iy) * g.ncd;
                    sg = make_int2(cell_start[base + ixl], cell_start[base + ixh + 1]);
                }
            }
        }
        seg[r] = sg;
    }
    __syncwarp();
}

template <typename T, int KERNEL>
__global__ void __launch_bounds__(WPB * 32) k_real(GP<T> g, RC<T> rk, int N, const vec4<T> *__restrict__ xs,
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
    row_segments(g, rk, xt, cell_start, lane, seg);
    const int W = 2 * rk.reach + 1, nrows = W * W;
    T acc[3] = {0, 0, 0}, ks[3] = {0, 0, 0}, kc[3] = {0, 0, 0};
    int cnt = 0;
    bool coinc = false;
    const unsigned lt = (1u << lane) - 1u;
    vec4<T> zero4;
    zero4.x = zero4.y = zero4.z = zero4.w = 0;
    for (int r = 0; r < nrows; r++) {
        const int2 sg = seg[r];
        for (int base = sg.x; base < sg.y; base += 32) {
            const int n = base + lane;
            bool in = false;
            T dx = 0, dy = 0, dz = 0, r2 = 0;
            if (n < sg.y) {
                const vec4<T> xv = xs[n];
                dx = xt.x - xv.x;
                dy = xt.y - xv.y;
                dz = xt.z - xv.z;
                r2 = dx * dx + dy * dy + dz * dz;
                in = (r2 <= rk.rc2) && (n != t);
                if (in && r2 == T(0)) {
                    in = false;
                    coinc = true;
                }
            }
            const unsigned mask = __ballot_sync(FULL, in);
            if (in) {
                const int pos = cnt + __popc(mask & lt);
                vec4<T> v;
                v.x = dx; v.y = dy; v.z = dz; v.w = r2;
                qd[pos] = v;
                qn[pos] = n;
            }
            cnt += __popc(mask);
            __syncwarp();
            if (cnt >= 32) {
                const vec4<T> v = qd[lane];
                const int m = qn[lane];
                const vec4<T> qv = (KERNEL == SE_STRESSLET) ? qs[m] : zero4;
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
        const vec4<T> v = qd[lane];
        const int m = qn[lane];
        const vec4<T> qv = (KERNEL == SE_STRESSLET) ? qs[m] : zero4;
        pair<T, KERNEL>(rk, v.x, v.y, v.z, v.w, fs[m], qv, acc);
    }
    T tot[3];
    for (int d = 0; d < 3; d++) {
        kahan_add(ks[d], kc[d], acc[d]);
        // tree sum of the compensated lane totals
        T s = ks[d], c = kc[d];
        for (int o = 16; o > 0; o >>= 1) {
            const T so = __shfl_xor_sync(FULL, s, o), co = __shfl_xor_sync(FULL, c, o);
            kahan_add(s, c, so);  // s - c now holds s_self + s_partner - c_self
            c += co;              // minus the partner's compensation
        }
        tot[d] = s - c;
    }
    if (__any_sync(FULL, coinc) && lane == 0) atomicOr(status, FLAG_COINCIDENT);
    if (lane < 3) {
        // lanes 0..2 each finish one component in FP64
        const int m = perm[t];
        const T v = lane == 0 ? tot[0] : (lane == 1 ? tot[1] : tot[2]);
        u[3 * m + lane] = (T)((double)u[3 * m + lane] + (double)v);
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
__global__ void __launch_bounds__(WPB * 32) k_real_grad(GP<T> g, RC<T> rk, int N, const vec4<T> *__restrict__ xs,
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
    const T gp_[3] = {g_orig[3 * mp], g_orig[3 * mp + 1], g_orig[3 * mp + 2]};
    row_segments(g, rk, xt, cell_start, lane, seg);
    const int W = 2 * rk.reach + 1, nrows = W * W;
    T acc[3] = {0, 0, 0};
    int cnt = 0;
    const unsigned lt = (1u << lane) - 1u;
    auto eval = [&](int slot) {
        const vec4<T> v = qd[slot];
        const int n = qn[slot];
        const vec4<T> fn = fs[n];
        const int mn = perm[n];
        const T gn[3] = {g_orig[3 * mn], g_orig[3 * mn + 1], g_orig[3 * mn + 2]};
        const T d[3] = {v.x, v.y, v.z};
        T rinv, r, e, ec;
        radial(rk, v.w, rinv, r, e, ec);
        const T c1 = rk.c;
        const T ecr = ec * rinv;
        const T rinv2 = rinv * rinv;
        const T b = (ecr + c1 * e) * rinv2;
        const T bp = -T(3) * c1 * e * rinv2 * rinv - T(3) * ec * rinv2 * rinv2 - T(2) * c1 * rk.xi2 * e * rinv;
        if (KERNEL == SE_STOKESLET) {
            const T ap = -c1 * e * rinv - ec * rinv2 + T(2) * c1 * rk.xi2 * r * e;
            const T f_n[3] = {fn.x, fn.y, fn.z}, f_p[3] = {fp.x, fp.y, fp.z};
            const T gpf = gp_[0] * f_n[0] + gp_[1] * f_n[1] + gp_[2] * f_n[2];
            const T gnf = gn[0] * f_p[0] + gn[1] * f_p[1] + gn[2] * f_p[2];
            const T gpr = gp_[0] * d[0] + gp_[1] * d[1] + gp_[2] * d[2];
            const T gnr = gn[0] * d[0] + gn[1] * d[1] + gn[2] * d[2];
            const T rfn = d[0] * f_n[0] + d[1] * f_n[1] + d[2] * f_n[2];
            const T rfp = d[0] * f_p[0] + d[1] * f_p[1] + d[2] * f_p[2];
            const T rad = (ap * (gpf + gnf) + bp * (gpr * rfn + gnr * rfp)) * rinv;
            for (int a = 0; a < 3; a++)
                acc[a] += rad * d[a] + b * (gp_[a] * rfn + f_n[a] * gpr + gn[a] * rfp + f_p[a] * gnr);
        } else {
            T c[3];
            c[0] = (gp_[1] * fn.z - gp_[2] * fn.y) - (gn[1] * fp.z - gn[2] * fp.y);
            c[1] = (gp_[2] * fn.x - gp_[0] * fn.z) - (gn[2] * fp.x - gn[0] * fp.z);
            c[2] = (gp_[0] * fn.y - gp_[1] * fn.x) - (gn[0] * fp.y - gn[1] * fp.x);
            const T rcd = (d[0] * c[0] + d[1] * c[1] + d[2] * c[2]) * bp * rinv;
            for (int a = 0; a < 3; a++) acc[a] += b * c[a] + rcd * d[a];
        }
    };
    for (int r = 0; r < nrows; r++) {
        const int2 sg = seg[r];
        for (int base = sg.x; base < sg.y; base += 32) {
            const int n = base + lane;
            bool in = false;
            T dx = 0, dy = 0, dz = 0, r2 = 0;
            if (n < sg.y) {
                const vec4<T> xv = xs[n];
                dx = xt.x - xv.x;
                dy = xt.y - xv.y;
                dz = xt.z - xv.z;
                r2 = dx * dx + dy * dy + dz * dz;
                in = (r2 <= rk.rc2) && (n != t) && (r2 > T(0));
            }
            const unsigned mask = __ballot_sync(FULL, in);
            if (in) {
                const int pos = cnt + __popc(mask & lt);
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

template <typename T>
RC<T> make_rc(const se_plan_s *p) {
    RC<T> rk;
    rk.xi = (T)p->xi;
    rk.xi2 = (T)(p->xi * p->xi);
    rk.c = (T)(2.0 * p->xi / sqrt(M_PI));
    rk.c3 = (T)(4.0 * p->xi * p->xi * p->xi / sqrt(M_PI));
    rk.rc2 = (T)(p->rc * p->rc);
    rk.reach = (int)ceil(p->rc * p->geom.inv_cw - 1e-9);
    return rk;
}

}  // namespace

template <typename T>
cudaError_t launch_real(se_plan_s *p, cudaStream_t st, T *u) {
    int N = (int)p->N;
    RC<T> rk = make_rc<T>(p);
    if (rk.reach > 3) return cudaErrorInvalidValue;
    unsigned gs = (N + WPB - 1) / WPB;
    const vec4<T> *xs = (const vec4<T> *)p->b.xs_r, *fs = (const vec4<T> *)p->b.fs_r,
                  *qs = (const vec4<T> *)p->b.qs_r;
    const GP<T> &g = gp<T>(p);
    if (p->kernel == SE_STOKESLET)
        k_real<T, SE_STOKESLET><<<gs, WPB * 32, 0, st>>>(g, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, u,
                                                       p->b.status);
    else if (p->kernel == SE_STRESSLET)
        k_real<T, SE_STRESSLET><<<gs, WPB * 32, 0, st>>>(g, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, u,
                                                       p->b.status);
    else
        k_real<T, SE_ROTLET><<<gs, WPB * 32, 0, st>>>(g, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, u,
                                                    p->b.status);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_real_grad(se_plan_s *p, cudaStream_t st, const T *g_orig, T *gx) {
    int N = (int)p->N;
    RC<T> rk = make_rc<T>(p);
    if (rk.reach > 3) return cudaErrorInvalidValue;
    unsigned gs = (N + WPB - 1) / WPB;
    const vec4<T> *xs = (const vec4<T> *)p->b.xs_r, *fs = (const vec4<T> *)p->b.fs_r;
    const GP<T> &g = gp<T>(p);
    if (p->kernel == SE_STOKESLET)
        k_real_grad<T, SE_STOKESLET><<<gs, WPB * 32, 0, st>>>(g, rk, N, xs, fs, p->b.cnt_r, p->b.perm_r, g_orig,
                                                            gx);
    else if (p->kernel == SE_ROTLET)
        k_real_grad<T, SE_ROTLET><<<gs, WPB * 32, 0, st>>>(g, rk, N, xs, fs, p->b.cnt_r, p->b.perm_r, g_orig, gx);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template cudaError_t launch_real<float>(se_plan_s *, cudaStream_t, float *);
template cudaError_t launch_real<double>(se_plan_s *, cudaStream_t, double *);
template cudaError_t launch_real_grad<float>(se_plan_s *, cudaStream_t, const float *, float *);
template cudaError_t launch_real_grad<double>(se_plan_s *, cudaStream_t, const double *, double *);

}  // namespace se
