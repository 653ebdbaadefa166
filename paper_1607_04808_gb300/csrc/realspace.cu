// Real-space part (Section 6): u^R(x_m) = sum_{0 < |x_m - x_n| <= rc} K^R(x_m - x_n) . f_n
// with the screened kernels of Section 3.2 (x = xi r, e = exp(-x^2), c = 2 xi/sqrt(pi)):
//   S^R     = A delta + B r r^T,  A r = erfc(x) - (2/sqrt(pi)) x e,  B r^3 = erfc(x) + (2/sqrt(pi)) x e
//             (eq. SR_Op)
//   T^R     = A1 r^ r^ r^ + A2 (delta r^ + ...),  A1 r^2 = -2 [3 erfc(x) + (2/sqrt(pi)) x (3 + 2 x^2) e],
//             A2 = xi^2 (4/sqrt(pi)) x e   (eq. TR_Op; A2 with the factor r that the third
//             derivative of r - Phi^H gives)
//   Omega^R = eps_jlm r_m B                                                (eq. RR_Op / 2)
// Each kernel needs two radial multipliers (a, b below), functions of r.  FP32
// evaluates erfc(x) = e Q(1/(2+x)) with a fitted erfcx polynomial Q
// (erfc_poly.cuh), sharing the exponential e; FP64 uses exp and a degree-18
// fit of erfcx in the same variable (the library erfc beyond x = 8).
//
// Cell list: points are sorted by cell (cells of width >= rc/5 across rows in
// FP32, rc/3 in FP64, and >= rc/16 along x, x fastest), so each (y, z) row of
// cells is a contiguous range of sorted points.  FP32 forward sum: every row is
// cut into clusters of 16 consecutive targets (a cluster never crosses a row,
// so it spans a few cells along x and one across); one warp per cluster, lane
// = (target, candidate stream).  The candidates of every row of cells within
// reach, trimmed along x to the cutoff sphere around the cluster's cells, form
// one flat stream, staged 32 at a time in shared memory; each of the 2 streams
// takes every other one, so every lane tests and evaluates its own (target,
// candidate) pairs with no compaction.  Partial sums are folded into
// Kahan-compensated totals after each staged chunk; the streams are combined
// with a compensated shuffle sum and u (which already holds u^F + u^self) is
// updated in FP64.  The FP64 forward sum and the backward kernels keep one warp
// per target with ballot compaction of the candidates.
#include <math.h>

#include <algorithm>
#include <vector>

#include "erfc_poly.cuh"
#include "se_internal.cuh"

namespace se {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int QCAP = 64;
// SE_RS_PAIR: paired FP32 arithmetic (sm_100+) in the FP32 pair sums
#ifndef SE_RS_PAIR
#define SE_RS_PAIR 1
#endif
// SE_GRAD_SYM: the FP32 real-space position gradient (stokeslet, rotlet) by the
// symmetric cluster kernel, each pair once
#ifndef SE_GRAD_SYM
#define SE_GRAD_SYM 1
#endif
// SE_GRAD_SYM_STR: the same for the stresslet's position gradient
#ifndef SE_GRAD_SYM_STR
#define SE_GRAD_SYM_STR 1
#endif
// SE_RS_PAIR_STR: the same for the stresslet's symmetric pair sum
#ifndef SE_RS_PAIR_STR
#define SE_RS_PAIR_STR 1
#endif
// SE_RS_BRANCH: the paired sums skip the radial functions of a target pair
// none of whose two pairs is within the cutoff (0: always evaluate, masked)
#ifndef SE_RS_BRANCH
#define SE_RS_BRANCH 1
#endif
constexpr int MAXROWS = 121;  // (2 reach_y + 1)(2 reach_z + 1) rows of cells at most

__device__ __forceinline__ float ex2_approx(float v) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// SE_RS_RAWMUFU: the reciprocal square root and reciprocal of the paired pair
// sums as the plain PTX approximations (one special-function instruction
// each, flush-to-zero).  Their arguments are normal numbers by construction
// (r^2 of distinct FP32 points, 2 + xi r), so the special-value handling of
// rsqrtf and __fdividef is never needed; 0 restores those.
#ifndef SE_RS_RAWMUFU
#define SE_RS_RAWMUFU 1
#endif
__device__ __forceinline__ float rsqrt_fast(float v) {
#if SE_RS_RAWMUFU
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
#else
    return rsqrtf(v);
#endif
}
__device__ __forceinline__ float rcp_fast(float v) {
#if SE_RS_RAWMUFU
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
#else
    return __fdividef(1.0f, v);
#endif
}

// erfcx(x) ~ Q(t), t = 1/(2 + x), from the fits of erfc_poly.cuh: PV = 1 for
// x <= 5 (degree 8), PV = 0 for x <= 8 (degree 10).
template <int PV>
__device__ __forceinline__ float erfcx_poly(float t) {
    if (PV == 1) {
        float q = ERFC_Q5[SE_ERFC_DEG5];
#pragma unroll
        for (int k = SE_ERFC_DEG5 - 1; k >= 0; k--) q = fmaf(q, t, ERFC_Q5[k]);
        return q;
    }
    float q = ERFC_Q8[SE_ERFC_DEG8];
#pragma unroll
    for (int k = SE_ERFC_DEG8 - 1; k >= 0; k--) q = fmaf(q, t, ERFC_Q8[k]);
    return q;
}

// Two values at once with the paired FP32 instructions of sm_100 and later
// (per component the same rounding as the scalar operations).
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

template <int PV>
__device__ __forceinline__ float2 erfcx_poly2(float2 t) {
    if (PV == 1) {
        float2 q = f2(ERFC_Q5[SE_ERFC_DEG5]);
#pragma unroll
        for (int k = SE_ERFC_DEG5 - 1; k >= 0; k--) q = __ffma2_rn(q, t, f2(ERFC_Q5[k]));
        return q;
    }
    float2 q = f2(ERFC_Q8[SE_ERFC_DEG8]);
#pragma unroll
    for (int k = SE_ERFC_DEG8 - 1; k >= 0; k--) q = __ffma2_rn(q, t, f2(ERFC_Q8[k]));
    return q;
}

// radial_ab (stokeslet, rotlet) for two distances at once.  A slot whose mask
// is off gets 1/r = 0 and so a = b = 0 (r2 finite in every slot: the paired
// path keeps empty slots at a far but finite position); q -+ c r and 2 + xi r
// are fused multiply-adds.
template <int PV>
__device__ __forceinline__ void radial_ab2(const RC<float> &rk, float2 r2, bool ua, bool ub, float2 &a,
                                           float2 &b) {
    const float2 rinv = make_float2(ua ? rsqrt_fast(r2.x) : 0.f, ub ? rsqrt_fast(r2.y) : 0.f);
    const float2 r = __fmul2_rn(r2, rinv);
    const float2 ce = __fmul2_rn(f2(rk.ce), r2);
    const float2 e = make_float2(ex2_approx(ce.x), ex2_approx(ce.y));
    const float2 y = __ffma2_rn(f2(rk.xi), r, f2(2.0f));
    const float2 q = erfcx_poly2<PV>(make_float2(rcp_fast(y.x), rcp_fast(y.y)));
    const float2 er = __fmul2_rn(e, rinv);
    a = __fmul2_rn(er, __ffma2_rn(f2(-rk.c), r, q));
    b = __fmul2_rn(__fmul2_rn(er, __fmul2_rn(rinv, rinv)), __ffma2_rn(f2(rk.c), r, q));
}

// Stresslet multipliers of two pairs at once, scaled for the displacement d
// itself instead of the unit vector d/r:  A = A1 / r^3 and B = A2 / r, so that
//   T(d) . (f, q) = A (d.f)(d.q) d + B [(f.q) d + (d.q) f + (d.f) q]
// (Eq. for T^R in Section 6).  A masked slot gets 1/r = 0, hence A = B = 0.
template <int PV>
__device__ __forceinline__ void radial_ab2_str(const RC<float> &rk, float2 r2, bool ua, bool ub, float2 &A,
                                               float2 &B) {
    const float2 rinv = make_float2(ua ? rsqrt_fast(r2.x) : 0.f, ub ? rsqrt_fast(r2.y) : 0.f);
    const float2 r = __fmul2_rn(r2, rinv);
    const float2 ce = __fmul2_rn(f2(rk.ce), r2);
    const float2 e = make_float2(ex2_approx(ce.x), ex2_approx(ce.y));
    const float2 y = __ffma2_rn(f2(rk.xi), r, f2(2.0f));
    const float2 q = erfcx_poly2<PV>(make_float2(rcp_fast(y.x), rcp_fast(y.y)));
    // A1 = -2 e [c r (2 x^2 + 3) + 3 Q] / r^2,  A2 = 2 xi^2 c r e,  x = xi r (from r,
    // not r2: a masked slot far away has r = 0, and 0 * (2 xi^2 r2) could be 0 * inf)
    const float2 cr = __fmul2_rn(f2(rk.c), r);
    const float2 x = __fmul2_rn(f2(rk.xi), r);
    const float2 poly = __ffma2_rn(cr, __ffma2_rn(__fmul2_rn(f2(2.0f), x), x, f2(3.0f)), __fmul2_rn(f2(3.0f), q));
    const float2 ri2 = __fmul2_rn(rinv, rinv);
    const float2 ri5 = __fmul2_rn(__fmul2_rn(ri2, ri2), rinv);
    A = __fmul2_rn(__fmul2_rn(f2(-2.0f), e), __fmul2_rn(poly, ri5));
    B = __fmul2_rn(__fmul2_rn(f2(2.0f * rk.xi2 * rk.c), e), __fmul2_rn(r, rinv));
}

// The two radial multipliers of a pair at distance r (r2 = r^2 > 0):
//   stokeslet, rotlet: a = (erfc(x) - (2/sqrt(pi)) x e) / r,  b = (erfc(x) + (2/sqrt(pi)) x e) / r^3
//   stresslet:         a = A1 = -2 [3 erfc(x) + (2/sqrt(pi)) x (3 + 2 x^2) e] / r^2,  b = A2 = 2 xi^2 (2/sqrt(pi)) x e
// FP32: erfc(x) = e Q(1/(2+x)) shares e = exp(-xi^2 r^2) with the Gaussian
// terms, so a = (e / r)(Q - c r) and b = (e / r^3)(Q + c r), c = 2 xi/sqrt(pi).
template <int KERNEL, int PV>
__device__ __forceinline__ void radial_ab(const RC<float> &rk, float r2, float &rinv, float &a, float &b) {
    rinv = rsqrt_fast(r2);
    const float r = r2 * rinv;
    const float x = rk.xi * r;
    const float e = ex2_approx(rk.ce * r2);
    const float q = erfcx_poly<PV>(rcp_fast(2.0f + x));
    const float cr = rk.c * r;  // (2/sqrt(pi)) x
    if (KERNEL == SE_STRESSLET) {
        a = -2.0f * e * fmaf(cr, fmaf(2.0f * x, x, 3.0f), 3.0f * q) * (rinv * rinv);
        b = 2.0f * rk.xi2 * cr * e;
    } else {
        const float er = e * rinv;
        a = er * (q - cr);
        b = er * (rinv * rinv) * (q + cr);
    }
}

// Gradient with respect to x_t of the pair term of L = sum g . u (stokeslet,
// rotlet; FP32), d = x_t - x_j, r = |d|, c1 = 2 xi/sqrt(pi), e = exp(-xi^2 r^2):
//   b = (erfc/r + c1 e)/r^2,  b' = -3 c1 e/r^3 - 3 erfc/r^4 - 2 c1 xi^2 e/r,
//   stokeslet: a' = -c1 e/r - erfc/r^2 + 2 c1 xi^2 r e,
//     G = d/r [a' (g_t.f_j + g_j.f_t) + b' ((g_t.d)(d.f_j) + (g_j.d)(d.f_t))]
//         + b [g_t (d.f_j) + f_j (g_t.d) + g_j (d.f_t) + f_t (g_j.d)]
//   rotlet: c = g_t x f_j - g_j x f_t,  G = b c + (b'/r)(d.c) d
template <int KERNEL, int PV>
__device__ __forceinline__ void grad_pair(const RC<float> &rk, float dx, float dy, float dz, float r2,
                                          const float4 &ft, const float4 &gt, const float4 &fj, const float4 &gj,
                                          float G[3]) {
    const float rinv = rsqrt_fast(r2), r = r2 * rinv, rinv2 = rinv * rinv;
    const float e = ex2_approx(rk.ce * r2);
    const float ec = e * erfcx_poly<PV>(rcp_fast(2.0f + rk.xi * r));
    const float c1 = rk.c;
    const float b = fmaf(ec, rinv, c1 * e) * rinv2;
    const float bp = -3.0f * c1 * e * rinv2 * rinv - 3.0f * ec * rinv2 * rinv2 - 2.0f * c1 * rk.xi2 * e * rinv;
    if (KERNEL == SE_STOKESLET) {
        const float ap = -c1 * e * rinv - ec * rinv2 + 2.0f * c1 * rk.xi2 * r * e;
        const float gpf = gt.x * fj.x + gt.y * fj.y + gt.z * fj.z;
        const float gnf = gj.x * ft.x + gj.y * ft.y + gj.z * ft.z;
        const float gpr = gt.x * dx + gt.y * dy + gt.z * dz;
        const float gnr = gj.x * dx + gj.y * dy + gj.z * dz;
        const float rfn = dx * fj.x + dy * fj.y + dz * fj.z;
        const float rfp = dx * ft.x + dy * ft.y + dz * ft.z;
        const float rad = (ap * (gpf + gnf) + bp * (gpr * rfn + gnr * rfp)) * rinv;
        G[0] = rad * dx + b * (gt.x * rfn + fj.x * gpr + gj.x * rfp + ft.x * gnr);
        G[1] = rad * dy + b * (gt.y * rfn + fj.y * gpr + gj.y * rfp + ft.y * gnr);
        G[2] = rad * dz + b * (gt.z * rfn + fj.z * gpr + gj.z * rfp + ft.z * gnr);
    } else {
        const float c0 = (gt.y * fj.z - gt.z * fj.y) - (gj.y * ft.z - gj.z * ft.y);
        const float cy = (gt.z * fj.x - gt.x * fj.z) - (gj.z * ft.x - gj.x * ft.z);
        const float cz = (gt.x * fj.y - gt.y * fj.x) - (gj.x * ft.y - gj.y * ft.x);
        const float rcd = (dx * c0 + dy * cy + dz * cz) * bp * rinv;
        G[0] = b * c0 + rcd * dx;
        G[1] = b * cy + rcd * dy;
        G[2] = b * cz + rcd * dz;
    }
}

// The stresslet's pair term of L = sum g . u as a trilinear form of d = x_t -
// x_j (Section 6, T^R rescaled for d itself: A = A1/r^3, B = A2/r):
//   Phi(d; a, b, c) = A (d.a)(d.b)(d.c) + B [(a.b)(d.c) + (b.c)(d.a) + (c.a)(d.b)],
//   A = -2 N / r^5, N = 3 erfc(x) + c r (3 + 2 x^2) e,  B = 2 xi^2 c e
// (x = xi r, c = 2 xi/sqrt(pi), e = exp(-x^2)), with the radial derivatives
//   A'/r = 8 c xi^4 e / r^2 + 10 N / r^7,  B'/r = -4 xi^4 c e.
// The pair contributes Phi(d; g_t, f_j, q_j) - Phi(d; g_j, f_t, q_t) (T is odd),
// so G = grad_d of that goes to x_t and -G to x_j:
//   grad Phi = [(A'/r)(d.a)(d.b)(d.c) + (B'/r)((a.b)(d.c) + (b.c)(d.a) + (c.a)(d.b))] d
//              + A [(d.b)(d.c) a + (d.a)(d.c) b + (d.a)(d.b) c] + B [(a.b) c + (b.c) a + (c.a) b].
__device__ __forceinline__ void grad_phi_str(float dx, float dy, float dz, float Ar, float A, float Br, float B,
                                             const float4 &a, const float4 &b, const float4 &c, float sgn,
                                             float G[3]) {
    const float da = dx * a.x + dy * a.y + dz * a.z, db = dx * b.x + dy * b.y + dz * b.z,
                dc = dx * c.x + dy * c.y + dz * c.z;
    const float ab = a.x * b.x + a.y * b.y + a.z * b.z, bc = b.x * c.x + b.y * c.y + b.z * c.z,
                ca = c.x * a.x + c.y * a.y + c.z * a.z;
    const float S = sgn * (Ar * da * db * dc + Br * (ab * dc + bc * da + ca * db));
    const float pa = sgn * (A * db * dc + B * bc), pb = sgn * (A * da * dc + B * ca),
                pc = sgn * (A * da * db + B * ab);
    G[0] += S * dx + pa * a.x + pb * b.x + pc * c.x;
    G[1] += S * dy + pa * a.y + pb * b.y + pc * c.y;
    G[2] += S * dz + pa * a.z + pb * b.z + pc * c.z;
}

template <int PV>
__device__ __forceinline__ void grad_pair_str(const RC<float> &rk, float dx, float dy, float dz, float r2,
                                              const float4 &ft, const float4 &qt, const float4 &gt, const float4 &fj,
                                              const float4 &qj, const float4 &gj, float G[3]) {
    const float rinv = rsqrt_fast(r2), r = r2 * rinv, rinv2 = rinv * rinv;
    const float x = rk.xi * r;
    const float e = ex2_approx(rk.ce * r2);
    const float Q = erfcx_poly<PV>(rcp_fast(2.0f + x));
    const float N = e * fmaf(rk.c * r, fmaf(2.0f * x, x, 3.0f), 3.0f * Q);
    const float rinv5 = rinv2 * rinv2 * rinv, x4c = rk.xi2 * rk.xi2 * rk.c;
    const float A = -2.0f * N * rinv5;
    const float Ar = 8.0f * x4c * e * rinv2 + 10.0f * N * rinv5 * rinv2;
    const float B = 2.0f * rk.xi2 * rk.c * e;
    const float Br = -4.0f * x4c * e;
    G[0] = G[1] = G[2] = 0.0f;
    grad_phi_str(dx, dy, dz, Ar, A, Br, B, gt, fj, qj, 1.0f, G);
    grad_phi_str(dx, dy, dz, Ar, A, Br, B, gj, ft, qt, -1.0f, G);
}

// FP64 erfc(x) = e Q64(s), e = exp(-x^2), s = SA t + SB, t = 1/(2 + x): the
// degree-18 fit of erfcx (relative error 8e-15 on [0, 8]); the library's erfc
// beyond (erfc(8) < 1e-28).
#ifndef SE_ERFC_FIT64
#define SE_ERFC_FIT64 1
#endif
__device__ __forceinline__ double erfc_fit64(double x, double e) {
    if (SE_ERFC_FIT64 && x <= SE_ERFC_XMAX64) {
        const double s = fma(SE_ERFC_SA64, 1.0 / (2.0 + x), SE_ERFC_SB64);
        double q = ERFC_QD[SE_ERFC_DEG64];
#pragma unroll
        for (int k = SE_ERFC_DEG64 - 1; k >= 0; k--) q = fma(q, s, ERFC_QD[k]);
        return e * q;
    }
    return erfc(x);
}

// FP64 table of erfc(x) and g(x) = (2/sqrt(pi)) x exp(-x^2) on [0, ERFT_XMAX]:
// ERFT_N intervals of width h, on each the degree-ERFT_D polynomials in t =
// 2 (x - x0) / h - 1 that interpolate both functions at the Chebyshev points
// (coefficients from the discrete Chebyshev transform of the values there,
// turned into powers of t), stored as (erfc, g) pairs, constant term first.
// Both functions are analytic in x; the interpolation error is below 2e-15
// absolute on the whole range and 5e-14 relative on [0, 5] (x = xi r <= xi
// rc, about 4.7 on FP64 plans at 1e-10).  One 16-byte load and two FMAs per
// degree replace exp, a division and the degree-18 erfcx fit.
constexpr int ERFT_N = 256, ERFT_D = 7;
constexpr double ERFT_XMAX = 8.0;
__device__ double2 g_erft[ERFT_N * (ERFT_D + 1)];

__device__ __forceinline__ void erfc_g_tab(double x, double &ec, double &g) {
    const double s = x * (ERFT_N / ERFT_XMAX);
    const int i = min((int)s, ERFT_N - 1);
    const double t = 2.0 * (s - (double)i) - 1.0;
    const double2 *c = g_erft + i * (ERFT_D + 1);
    double2 v = __ldg(c + ERFT_D);
#pragma unroll
    for (int k = ERFT_D - 1; k >= 0; k--) {
        const double2 ck = __ldg(c + k);
        v.x = fma(v.x, t, ck.x);
        v.y = fma(v.y, t, ck.y);
    }
    ec = v.x;
    g = v.y;
}

// FP64: the same multipliers from erfc and the Gaussian term (the table, or
// exp and the erfcx fit)
template <int KERNEL, int PV>
__device__ __forceinline__ void radial_ab(const RC<double> &rk, double r2, double &rinv, double &a, double &b) {
    rinv = rsqrt(r2);
    const double r = r2 * rinv;
    const double x = rk.xi * r;
    double ec, g;
    if (rk.tab && x < ERFT_XMAX) {
        erfc_g_tab(x, ec, g);
    } else {
        const double e = exp(-x * x);
        ec = erfc_fit64(x, e);
        g = 1.1283791670955126 * x * e;  // (2/sqrt(pi)) x e
    }
    if (KERNEL == SE_STRESSLET) {
        a = -2.0 * (3.0 * ec + g * (3.0 + 2.0 * x * x)) * (rinv * rinv);
        b = 2.0 * rk.xi2 * g;
    } else {
        a = (ec - g) * rinv;
        b = (ec + g) * (rinv * rinv * rinv);
    }
}

// K^R(d) . source, added to acc (d = x_target - x_source, r2 = |d|^2 > 0)
template <typename T, int KERNEL, int PV = 0>
__device__ __forceinline__ void pair(const RC<T> &rk, T dx, T dy, T dz, T r2, const vec4<T> &f, const vec4<T> &q,
                                     T acc[3]) {
    T rinv, a, b;
    radial_ab<KERNEL, PV>(rk, r2, rinv, a, b);
    if (KERNEL == SE_STOKESLET) {
        const T Brf = b * (dx * f.x + dy * f.y + dz * f.z);
        acc[0] += a * f.x + Brf * dx;
        acc[1] += a * f.y + Brf * dy;
        acc[2] += a * f.z + Brf * dz;
    } else if (KERNEL == SE_ROTLET) {
        acc[0] += b * (f.y * dz - f.z * dy);
        acc[1] += b * (f.z * dx - f.x * dz);
        acc[2] += b * (f.x * dy - f.y * dx);
    } else {
        const T hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
        const T hf = hx * f.x + hy * f.y + hz * f.z;
        const T hq = hx * q.x + hy * q.y + hz * q.z;
        const T fq = f.x * q.x + f.y * q.y + f.z * q.z;
        const T a1 = a * hf * hq;
        acc[0] += a1 * hx + b * (hx * fq + f.x * hq + q.x * hf);
        acc[1] += a1 * hy + b * (hy * fq + f.y * hq + q.y * hf);
        acc[2] += a1 * hz + b * (hz * fq + f.z * hq + q.z * hf);
    }
}

// The stresslet pair applied to two strength pairs (a, b) and (a, c) with one
// evaluation of the radial multipliers: acc += T^R(d)(a, b), acc2 += T^R(d)(a, c).
template <typename T>
__device__ __forceinline__ void pair_str2(const RC<T> &rk, T dx, T dy, T dz, T r2, const vec4<T> &a,
                                          const vec4<T> &b, const vec4<T> &c, T acc[3], T acc2[3]) {
    T rinv, A1, A2;
    radial_ab<SE_STRESSLET, 0>(rk, r2, rinv, A1, A2);
    const T hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
    const T ha = hx * a.x + hy * a.y + hz * a.z;
    {
        const T hb = hx * b.x + hy * b.y + hz * b.z;
        const T ab = a.x * b.x + a.y * b.y + a.z * b.z;
        const T a1 = A1 * ha * hb;
        acc[0] += a1 * hx + A2 * (hx * ab + a.x * hb + b.x * ha);
        acc[1] += a1 * hy + A2 * (hy * ab + a.y * hb + b.y * ha);
        acc[2] += a1 * hz + A2 * (hz * ab + a.z * hb + b.z * ha);
    }
    {
        const T hc = hx * c.x + hy * c.y + hz * c.z;
        const T ac = a.x * c.x + a.y * c.y + a.z * c.z;
        const T a1 = A1 * ha * hc;
        acc2[0] += a1 * hx + A2 * (hx * ac + a.x * hc + c.x * ha);
        acc2[1] += a1 * hy + A2 * (hy * ac + a.y * hc + c.y * ha);
        acc2[2] += a1 * hz + A2 * (hz * ac + a.z * hc + c.z * ha);
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
__device__ __forceinline__ int row_segments(const GP<T> &g, const RC<T> &rk, const vec4<T> &xt,
                                            const int *__restrict__ cell_start, int lane, int2 *seg) {
    int cc[3];
    unpack3(get_tag(xt), cc[0], cc[1], cc[2]);
    const T rel[3] = {xt.x - g.x0[0], xt.y - g.x0[1], xt.z - g.x0[2]};
    const T rc2m = rk.rc2 * T(1.0001);
    const int Ry = rk.reach[0], Rz = rk.reach[1], Wy = 2 * Ry + 1, nrows = Wy * (2 * Rz + 1);
    for (int r = lane; r < nrows; r += 32) {
        int iy = cc[1] + (r % Wy) - Ry, iz = cc[2] + (r / Wy) - Rz;
        int2 sg = make_int2(0, 0);
        if (iy >= 0 && iy < g.ncel[1] && iz >= 0 && iz < g.ncel[2]) {
            const T ylo = iy * g.cw[1], zlo = iz * g.cw[2];
            const T dy = max(T(0), max(ylo - rel[1], rel[1] - (ylo + g.cw[1])));
            const T dz = max(T(0), max(zlo - rel[2], rel[2] - (zlo + g.cw[2])));
            const T d2 = dy * dy + dz * dz;
            if (d2 <= rc2m) {
                const T del = sqrt(rc2m - d2) + T(1e-4) * g.cw[0];
                const int ixl = max(0, (int)floor((rel[0] - del) * g.icw[0]));
                const int ixh = min(g.ncel[0] - 1, (int)floor((rel[0] + del) * g.icw[0]));
                if (ixl <= ixh) {
                    const int base = (iz * g.ncel[1] + iy) * g.ncel[0];
                    sg = make_int2(cell_start[base + ixl], cell_start[base + ixh + 1]);
                }
            }
        }
        seg[r] = sg;
    }
    __syncwarp();
    return nrows;
}

// Clusters: each (y, z) row of cells is a contiguous range of sorted points;
// it is cut into clusters of at most TPW consecutive points (never crossing a
// row), so a cluster is compact (at most a few cells along x, one cell across).
// Periodic plans (rc < L/2): the rows of cells within reach wrap around the
// box in y and z, each row at most once (all rows once when the reach spans the
// box, and then without pruning by the row's distance, which the unwrapped
// index could overestimate); each row's x-range wraps into at most two
// segments (the whole row once when it spans the box).  Two entries of seg per
// row; the pair test takes the nearest image.
template <typename T>
__device__ __forceinline__ int row_segments_per(const GP<T> &g, const RC<T> &rk, const vec4<T> &xt,
                                                const int *__restrict__ cell_start, int lane, int2 *seg) {
    int cc[3];
    unpack3(get_tag(xt), cc[0], cc[1], cc[2]);
    const T rel[3] = {xt.x - g.x0[0], xt.y - g.x0[1], xt.z - g.x0[2]};
    const T rc2m = rk.rc2 * T(1.0001);
    const int ny = g.ncel[1], nz = g.ncel[2], nx = g.ncel[0];
    const int Wy = min(2 * rk.reach[0] + 1, ny), Wz = min(2 * rk.reach[1] + 1, nz);
    const int oy = (Wy - 1) / 2, oz = (Wz - 1) / 2, nrows = Wy * Wz;
    for (int r = lane; r < nrows; r += 32) {
        const int iyu = cc[1] + (r % Wy) - oy, izu = cc[2] + (r / Wy) - oz;  // unwrapped
        const int iy = (iyu + ny) % ny, iz = (izu + nz) % nz;
        int2 s0 = make_int2(0, 0), s1 = make_int2(0, 0);
        const T ylo = iyu * g.cw[1], zlo = izu * g.cw[2];
        const T dy = (Wy == ny) ? T(0) : max(T(0), max(ylo - rel[1], rel[1] - (ylo + g.cw[1])));
        const T dz = (Wz == nz) ? T(0) : max(T(0), max(zlo - rel[2], rel[2] - (zlo + g.cw[2])));
        const T d2 = dy * dy + dz * dz;
        if (d2 <= rc2m) {
            const T del = sqrt(rc2m - d2) + T(1e-4) * g.cw[0];
            const int ixl = (int)floor((rel[0] - del) * g.icw[0]);
            const int ixh = (int)floor((rel[0] + del) * g.icw[0]);
            const int base = (iz * ny + iy) * nx;
            if (ixh - ixl + 1 >= nx) {
                s0 = make_int2(cell_start[base], cell_start[base + nx]);
            } else {
                const int a = ((ixl % nx) + nx) % nx, b = ((ixh % nx) + nx) % nx;
                if (a <= b) {
                    s0 = make_int2(cell_start[base + a], cell_start[base + b + 1]);
                } else {
                    s0 = make_int2(cell_start[base + a], cell_start[base + nx]);
                    s1 = make_int2(cell_start[base], cell_start[base + b + 1]);
                }
            }
        }
        seg[2 * r] = s0;
        seg[2 * r + 1] = s1;
    }
    __syncwarp();
    return 2 * nrows;
}

__global__ void k_cluster_count(int nrows, int ncdx, int tpw, const int *__restrict__ cell_start, int *ncl) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    int len = cell_start[(r + 1) * ncdx] - cell_start[r * ncdx];
    ncl[r] = (len + tpw - 1) / tpw;
}

__global__ void k_cluster_fill(int nrows, int ncdx, int tpw, const int *__restrict__ cell_start,
                               const int *__restrict__ ncl_start, int2 *__restrict__ cl) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int a = cell_start[r * ncdx], b = cell_start[(r + 1) * ncdx];
    int o = ncl_start[r];
    for (int s = a; s < b; s += tpw) cl[o++] = make_int2(s, min(tpw, b - s));
}

// K^R(d) applied to NR sources at once (the radial multipliers are evaluated
// once per pair): acc[r] += K^R(d) . f[r] (stokeslet, rotlet).
template <typename T, int KERNEL, int NR, int PV>
__device__ __forceinline__ void pair_multi(const RC<T> &rk, T dx, T dy, T dz, T r2, const vec4<T> *f,
                                           const vec4<T> &q, T (*acc)[3], int nq) {
    if (NR == 1) {
        pair<T, KERNEL, PV>(rk, dx, dy, dz, r2, f[0], q, acc[0]);
        return;
    }
    T rinv, a, b;
    radial_ab<KERNEL, PV>(rk, r2, rinv, a, b);
    if (KERNEL == SE_STOKESLET) {
#pragma unroll
        for (int r = 0; r < NR; r++) {
            if (r >= nq) break;
            const vec4<T> fv = f[r];
            const T Brf = b * (dx * fv.x + dy * fv.y + dz * fv.z);
            acc[r][0] += a * fv.x + Brf * dx;
            acc[r][1] += a * fv.y + Brf * dy;
            acc[r][2] += a * fv.z + Brf * dz;
        }
    } else {
#pragma unroll
        for (int r = 0; r < NR; r++) {
            if (r >= nq) break;
            const vec4<T> fv = f[r];
            acc[r][0] += b * (fv.y * dz - fv.z * dy);
            acc[r][1] += b * (fv.z * dx - fv.x * dz);
            acc[r][2] += b * (fv.x * dy - fv.y * dx);
        }
    }
}

// pair_multi for 8 right-hand sides in pairs (r, r + 4) with the paired FP32
// instructions: fp holds the candidate's sources as [3 p + d] = (f_p.d, f_{p+4}.d).
template <int KERNEL, int PV>
__device__ __forceinline__ void pair_multi8p(const RC<float> &rk, float dx, float dy, float dz, float r2,
                                             const float2 *fp, float2 (*acc)[3]) {
    float rinv, a, b;
    radial_ab<KERNEL, PV>(rk, r2, rinv, a, b);
    const float2 A = f2(a), Bm = f2(b), DX = f2(dx), DY = f2(dy), DZ = f2(dz);
#pragma unroll
    for (int p = 0; p < 4; p++) {
        const float2 fx = fp[3 * p], fy = fp[3 * p + 1], fz = fp[3 * p + 2];
        if (KERNEL == SE_STOKESLET) {
            const float2 brf = __fmul2_rn(Bm, __ffma2_rn(DZ, fz, __ffma2_rn(DY, fy, __fmul2_rn(DX, fx))));
            acc[p][0] = __ffma2_rn(A, fx, __ffma2_rn(brf, DX, acc[p][0]));
            acc[p][1] = __ffma2_rn(A, fy, __ffma2_rn(brf, DY, acc[p][1]));
            acc[p][2] = __ffma2_rn(A, fz, __ffma2_rn(brf, DZ, acc[p][2]));
        } else {
            // rotlet: b (f x d)
            const float2 NX = f2(-dx), NY = f2(-dy), NZ = f2(-dz);
            acc[p][0] = __ffma2_rn(Bm, __ffma2_rn(fy, DZ, __fmul2_rn(fz, NY)), acc[p][0]);
            acc[p][1] = __ffma2_rn(Bm, __ffma2_rn(fz, DX, __fmul2_rn(fx, NZ)), acc[p][1]);
            acc[p][2] = __ffma2_rn(Bm, __ffma2_rn(fx, DY, __fmul2_rn(fy, NX)), acc[p][2]);
        }
    }
}

// Kahan addition of x into (s, c) for two values at once (t - s and y - c as
// fused multiply-adds with -1, exact like the subtractions they replace)
__device__ __forceinline__ void kahan_add2(float2 &s, float2 &c, float2 x) {
    const float2 m1 = f2(-1.f);
    const float2 y = __ffma2_rn(m1, c, x);
    const float2 t = __fadd2_rn(s, y);
    c = __ffma2_rn(m1, y, __ffma2_rn(m1, s, t));
    s = t;
}

// One warp per cluster: lane = (target k = lane % TPW, candidate stream
// s = lane / TPW).  Candidates of every row within reach are loaded 32 at a
// time into shared memory and stream s takes every NS-th of them, so each lane
// tests and evaluates (target k, candidate) pairs without any compaction.
// Sources: right-hand sides q0 .. q0 + nq - 1 (nq <= NR) of the fstride
// 4-vectors stored per sorted point in fs; u holds fstride three-vectors per
// original point.  BATCH: the cluster's system
// (cl_sys) supplies the geometry, the screening constants and the offset of
// its cells; otherwise g0, rk0 and cell_start0 are the one system's.
// PV selects the FP32 erfcx fit (1: x = xi r <= 5, 0: x <= 8).  TGT: the
// targets are separate points (sorted by cell in xtg, permutation tperm, the
// clusters built over their rows): no pair is excluded, and any candidate at
// distance zero is reported as coincident.
template <typename T, int KERNEL, int TPW, int NR, bool BATCH, int PV, bool TGT = false>
__global__ void __launch_bounds__(256) k_real_cl(GP<T> g0, RC<T> rk0, const BSys<T> *__restrict__ sys,
                                                 const int *__restrict__ cl_sys, const vec4<T> *__restrict__ xs,
                                                 const vec4<T> *__restrict__ fs, const vec4<T> *__restrict__ qs,
                                                 const int *__restrict__ cell_start0,
                                                 const int2 *__restrict__ clusters, const int *__restrict__ ncl_total,
                                                 const int *__restrict__ perm, T *__restrict__ u,
                                                 int *__restrict__ status, int fstride, int q0, int nq,
                                                 const vec4<T> *__restrict__ xtg = nullptr,
                                                 const int *__restrict__ tperm = nullptr) {
    constexpr int WPB = 8, NS = 32 / TPW;
    // 8 right-hand sides of the stokeslet or rotlet in FP32: pairs (r, r + 4)
    constexpr bool PAIRRHS = sizeof(T) == 4 && NR == 8 && KERNEL != SE_STRESSLET && SE_RS_PAIR;
    __shared__ vec4<T> sx_all[WPB][32];
    __shared__ vec4<T> sf_all[WPB][32 * NR];
    __shared__ vec4<T> sq_all[KERNEL == SE_STRESSLET ? WPB : 1][32];
    __shared__ int2 seg_all[WPB][MAXROWS];
    __shared__ int pre_all[WPB][MAXROWS + 1];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // one cluster per warp; consecutive clusters (neighbours in space) share a
    // block, so their candidate loads share the L1 cache
    const int c = blockIdx.x * WPB + wib;
    if (c >= *ncl_total) return;
    vec4<T> *sx = sx_all[wib];
    vec4<T> *sf = sf_all[wib];
    vec4<T> *sq = sq_all[KERNEL == SE_STRESSLET ? wib : 0];
    int2 *seg = seg_all[wib];
    GP<T> g;
    RC<T> rk;
    const int *cell_start;
    if constexpr (BATCH) {
        const BSys<T> &B = sys[cl_sys[c]];
        g = B.g;
        rk = B.rk;
        cell_start = cell_start0 + B.cell_base;
    } else {
        g = g0;
        rk = rk0;
        cell_start = cell_start0;
    }
    const int2 cl = clusters[c];
    const int k = lane % TPW, s = lane / TPW;
    const bool has = k < cl.y;
    const int t = cl.x + min(k, cl.y - 1);
    const vec4<T> *xT = TGT ? xtg : xs;
    const vec4<T> xt = xT[t];
    // rows of cells within reach of the cluster's cells
    int c0[3], c1[3];
    unpack3(get_tag(xT[cl.x]), c0[0], c0[1], c0[2]);
    unpack3(get_tag(xT[cl.x + cl.y - 1]), c1[0], c1[1], c1[2]);
    const int Ry = rk.reach[0], Rz = rk.reach[1], Wy = 2 * Ry + 1, nrows = Wy * (2 * Rz + 1);
    const T rc2m = rk.rc2 * T(1.0001);
    for (int r = lane; r < nrows; r += 32) {
        const int dyc = (r % Wy) - Ry, dzc = (r / Wy) - Rz;
        const int iy = c0[1] + dyc, iz = c0[2] + dzc;
        int2 sg = make_int2(0, 0);
        if (iy >= 0 && iy < g.ncel[1] && iz >= 0 && iz < g.ncel[2]) {
            const T dy = T(max(abs(dyc) - 1, 0)) * g.cw[1], dz = T(max(abs(dzc) - 1, 0)) * g.cw[2];
            const T d2 = dy * dy + dz * dz;
            if (d2 <= rc2m) {
                const T del = sqrt(rc2m - d2) + T(1e-4) * g.cw[0];
                const int ixl = max(0, (int)floor((T(c0[0]) * g.cw[0] - del) * g.icw[0]));
                const int ixh = min(g.ncel[0] - 1, (int)floor((T(c1[0] + 1) * g.cw[0] + del) * g.icw[0]));
                if (ixl <= ixh) {
                    const int base = (iz * g.ncel[1] + iy) * g.ncel[0];
                    sg = make_int2(cell_start[base + ixl], cell_start[base + ixh + 1]);
                }
            }
        }
        seg[r] = sg;
    }
    __syncwarp();
    // flat candidate stream over all row segments: exclusive prefix of the
    // segment lengths (warp scan), then each lane finds its segment by bisection
    int *pre = pre_all[wib];
    int run = 0;
    for (int r0 = 0; r0 < nrows; r0 += 32) {
        const int r = r0 + lane;
        int len = (r < nrows) ? seg[r].y - seg[r].x : 0;
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (r < nrows) pre[r] = run + incl - len;
        run += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) pre[nrows] = run;
    __syncwarp();
    const int total = run;
    T acc[NR][3], ks[NR][3], kc[NR][3];
#pragma unroll
    for (int q = 0; q < NR; q++)
        for (int d = 0; d < 3; d++) acc[q][d] = ks[q][d] = kc[q][d] = T(0);
    float2 acc2[4][3], ks2[4][3], kc2[4][3];  // PAIRRHS: right-hand sides (p, p + 4)
#pragma unroll
    for (int q = 0; q < 4; q++)
        for (int d = 0; d < 3; d++) acc2[q][d] = ks2[q][d] = kc2[q][d] = f2(0.f);
    // PAIRRHS staging of the candidates' sources: 12 float2 per candidate
    float2 *sp = reinterpret_cast<float2 *>(sf);
    int zeros = 0;  // candidates at distance 0 seen by this lane (its own target included once)
    vec4<T> zero4;
    zero4.x = zero4.y = zero4.z = zero4.w = 0;
    int lo = 0;  // the lane's segment: pre[lo] <= v < pre[lo + 1] (positions only grow)
    for (int cb = 0; cb < total; cb += 32) {
        const int v = cb + lane;
        if (v < total) {
            while (pre[lo + 1] <= v) lo++;
            const int m = seg[lo].x + (v - pre[lo]);
            vec4<T> xv = xs[m];
            xv.w = T(0);
            sx[lane] = xv;
            if constexpr (PAIRRHS) {
                const vec4<T> *fm = fs + (size_t)m * fstride + q0;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const float4 lo = (q < nq) ? fm[q] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 hi = (q + 4 < nq) ? fm[q + 4] : make_float4(0.f, 0.f, 0.f, 0.f);
                    sp[lane * 12 + 3 * q] = make_float2(lo.x, hi.x);
                    sp[lane * 12 + 3 * q + 1] = make_float2(lo.y, hi.y);
                    sp[lane * 12 + 3 * q + 2] = make_float2(lo.z, hi.z);
                }
            } else {
#pragma unroll
                for (int q = 0; q < NR; q++)
                    if (q < nq) sf[lane * NR + q] = fs[(size_t)m * fstride + q0 + q];
            }
            if (KERNEL == SE_STRESSLET) sq[lane] = qs[m];
        }
        __syncwarp();
        const int nch = min(32, total - cb);
        auto step = [&](int j) {
            const vec4<T> xv = sx[j];
            const T dx = xt.x - xv.x, dy = xt.y - xv.y, dz = xt.z - xv.z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (has && r2 <= rk.rc2) {
                if (r2 > T(0)) {
                    if constexpr (PAIRRHS) {
                        pair_multi8p<KERNEL, PV>(rk, dx, dy, dz, r2, sp + j * 12, acc2);
                    } else {
                        const vec4<T> qv = (KERNEL == SE_STRESSLET) ? sq[j] : zero4;
                        pair_multi<T, KERNEL, NR, PV>(rk, dx, dy, dz, r2, sf + j * NR, qv, acc, nq);
                    }
                } else {
                    zeros++;  // the target itself, or a coincident point
                }
            }
        };
        if (nch == 32) {
#pragma unroll
            for (int i = 0; i < 32 / NS; i++) step(s + i * NS);
        } else {
            for (int j = s; j < nch; j += NS) step(j);
        }
        __syncwarp();
        if constexpr (PAIRRHS) {
#pragma unroll
            for (int q = 0; q < 4; q++)
                for (int d = 0; d < 3; d++) {
                    kahan_add2(ks2[q][d], kc2[q][d], acc2[q][d]);
                    acc2[q][d] = f2(0.f);
                }
        } else {
#pragma unroll
            for (int q = 0; q < NR; q++)
                for (int d = 0; d < 3; d++) {
                    kahan_add(ks[q][d], kc[q][d], acc[q][d]);
                    acc[q][d] = 0;
                }
        }
    }
    if constexpr (PAIRRHS) {
#pragma unroll
        for (int q = 0; q < 4; q++)
            for (int d = 0; d < 3; d++) {
                ks[q][d] = ks2[q][d].x;
                ks[q + 4][d] = ks2[q][d].y;
                kc[q][d] = kc2[q][d].x;
                kc[q + 4][d] = kc2[q][d].y;
            }
    }
    // combine the NS streams of each target (lanes k, k + TPW, ...)
    T tot[NR][3];
#pragma unroll
    for (int q = 0; q < NR; q++)
        for (int d = 0; d < 3; d++) {
            T sm_ = ks[q][d], cm_ = kc[q][d];
            for (int o = TPW; o < 32; o <<= 1) {
                const T so = __shfl_xor_sync(FULL, sm_, o), co = __shfl_xor_sync(FULL, cm_, o);
                kahan_add(sm_, cm_, so);  // sm_ - cm_ now holds the own and the partner's sums
                cm_ += co;                // minus the partner's compensation
            }
            tot[q][d] = sm_ - cm_;
        }
    for (int o = TPW; o < 32; o <<= 1) zeros += __shfl_xor_sync(FULL, zeros, o);
    if (__any_sync(FULL, zeros > (TGT ? 0 : 1)) && lane == 0) atomicOr(status, FLAG_COINCIDENT);
    if (s == 0 && has) {
        const size_t mi = (TGT ? tperm : perm)[t];
#pragma unroll
        for (int q = 0; q < NR; q++) {
            if (q >= nq) break;
            for (int d = 0; d < 3; d++) {
                T *ud = u + (mi * fstride + q0 + q) * 3 + d;
                *ud = (T)((double)*ud + (double)tot[q][d]);
            }
        }
    }
}

// FP32, one system, one right-hand side: every pair within the cutoff is
// evaluated once.  The cluster's candidate stream keeps only points that come
// later in the sorted order (rows after the cluster's row, and the cluster's
// own row from its first point on), and a pair (target t, candidate m) counts
// only when m > t, so each unordered pair belongs to exactly one cluster.  The
// radial multipliers are evaluated once and applied both ways:
//   u_t += K^R(x_t - x_m) . s_m  (register accumulator, Kahan per chunk), and
//   u_m += K^R(x_m - x_t) . s_t = sign K^R(x_t - x_m) . s_t (sign -1 for the odd
//   stresslet and rotlet), accumulated per staged candidate in registers
//   (16 candidates per lane), then summed over the 16 targets by a warp
//   reduce-scatter so that each lane ends with one candidate's total, added to
//   uj (sorted order, float4) with one vector atomic.
// uj is added to u by k_add_uj after the kernel.
#ifndef SE_RS_SYM_MINB
#define SE_RS_SYM_MINB 4
#endif
// uj holds 4 values of T per sorted point (x, y, z, unused).  FP64 keeps two
// blocks per SM (its accumulators need twice the registers).
template <typename T, int KERNEL, int PV, int TPW>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? SE_RS_SYM_MINB : 2)
    k_real_sym(GP<T> g, RC<T> rk, const vec4<T> *__restrict__ xs, const vec4<T> *__restrict__ fs,
               const vec4<T> *__restrict__ qs, const int *__restrict__ cell_start, const int2 *__restrict__ clusters,
               const int *__restrict__ ncl_total, const int *__restrict__ perm, T *__restrict__ u,
               T *__restrict__ uj, int *__restrict__ status) {
    // lane = (target k = lane % TPW, stream s = lane / TPW); each staged chunk of
    // 32 candidates gives every stream NC = TPW of them
    constexpr int WPB = 8, NS = 32 / TPW, NC = TPW;
    __shared__ vec4<T> sx_all[WPB][32];
    __shared__ vec4<T> sf_all[WPB][32];
    __shared__ vec4<T> sq_all[KERNEL == SE_STRESSLET ? WPB : 1][32];
    __shared__ int sm_all[WPB][32];
    __shared__ int2 seg_all[WPB][MAXROWS];
    __shared__ int pre_all[WPB][MAXROWS + 1];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * WPB + wib;
    if (c >= *ncl_total) return;
    vec4<T> *sx = sx_all[wib];
    vec4<T> *sf = sf_all[wib];
    vec4<T> *sq = sq_all[KERNEL == SE_STRESSLET ? wib : 0];
    int *smi = sm_all[wib];
    int2 *seg = seg_all[wib];
    const int2 cl = clusters[c];
    const int k = lane % TPW, s = lane / TPW;
    const bool has = k < cl.y;
    const int t = cl.x + min(k, cl.y - 1);
    vec4<T> xt = xs[t];
    if (!has) xt.x = T(INFINITY);  // no candidate passes the cutoff test
    const vec4<T> ft = fs[t];
    vec4<T> qt;
    qt.x = qt.y = qt.z = qt.w = T(0);
    if (KERNEL == SE_STRESSLET) qt = qs[t];
    int c0[3], c1[3];
    unpack3(get_tag(xs[cl.x]), c0[0], c0[1], c0[2]);
    unpack3(get_tag(xs[cl.x + cl.y - 1]), c1[0], c1[1], c1[2]);
    const int Ry = rk.reach[0], Rz = rk.reach[1], Wy = 2 * Ry + 1, nrows = Wy * (2 * Rz + 1);
    const T rc2m = rk.rc2 * T(1.0001);
    const int own_row = c0[2] * g.ncel[1] + c0[1];
    // rows at or after the cluster's row in the sorted order; the own row from
    // the cluster's first point on, so that it leads the stream and stream
    // position v < cl.y is the cluster's own point cl.x + v
    for (int r = lane; r < nrows; r += 32) {
        const int dyc = (r % Wy) - Ry, dzc = (r / Wy) - Rz;
        const int iy = c0[1] + dyc, iz = c0[2] + dzc;
        int2 sg = make_int2(0, 0);
        const int row = iz * g.ncel[1] + iy;
        if (iy >= 0 && iy < g.ncel[1] && iz >= 0 && iz < g.ncel[2] && row >= own_row) {
            const T dy = T(max(abs(dyc) - 1, 0)) * g.cw[1], dz = T(max(abs(dzc) - 1, 0)) * g.cw[2];
            const T d2 = dy * dy + dz * dz;
            if (d2 <= rc2m) {
                const T del = sqrt(rc2m - d2) + T(1e-4) * g.cw[0];
                const int ixl = max(0, (int)floor((T(c0[0]) * g.cw[0] - del) * g.icw[0]));
                const int ixh = min(g.ncel[0] - 1, (int)floor((T(c1[0] + 1) * g.cw[0] + del) * g.icw[0]));
                if (ixl <= ixh) {
                    const int base = row * g.ncel[0];
                    sg = make_int2(cell_start[base + ixl], cell_start[base + ixh + 1]);
                    if (row == own_row) sg.x = cl.x;
                }
            }
        }
        seg[r] = sg;
    }
    __syncwarp();
    int *pre = pre_all[wib];
    int run = 0;
    for (int r0 = 0; r0 < nrows; r0 += 32) {
        const int r = r0 + lane;
        int len = (r < nrows) ? seg[r].y - seg[r].x : 0;
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (r < nrows) pre[r] = run + incl - len;
        run += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) pre[nrows] = run;
    __syncwarp();
    const int total = run;
    T acc[3] = {0, 0, 0}, ks[3] = {0, 0, 0}, kc[3] = {0, 0, 0};
    bool coinc = false;
    int lo = 0;  // the lane's segment: pre[lo] <= v < pre[lo + 1] (positions only grow)
    for (int cb = 0; cb < total; cb += 32) {
        const int v = cb + lane;
        if (v < total) {
            while (pre[lo + 1] <= v) lo++;
            const int m = seg[lo].x + (v - pre[lo]);
            sx[lane] = xs[m];
            sf[lane] = fs[m];
            if (KERNEL == SE_STRESSLET) sq[lane] = qs[m];
            smi[lane] = m;
        }
        __syncwarp();
        const int nch = min(32, total - cb);
        T aj[NC][3];
#pragma unroll
        for (int i = 0; i < NC; i++) aj[i][0] = aj[i][1] = aj[i][2] = T(0);
        // one (target, candidate) pair: candidate slot j, stream position cb + j;
        // it counts when the candidate comes after the target (position > k)
        auto step = [&](int i, int j) {
            const vec4<T> xv = sx[j];
            const T dx = xt.x - xv.x, dy = xt.y - xv.y, dz = xt.z - xv.z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 <= rk.rc2 && cb + j > k) {
                if (r2 > T(0)) {
                    T rinv, a, b;
                    radial_ab<KERNEL, PV>(rk, r2, rinv, a, b);
                    const vec4<T> fv = sf[j];
                    if (KERNEL == SE_STOKESLET) {
                        const T bj = b * (dx * fv.x + dy * fv.y + dz * fv.z);
                        acc[0] += a * fv.x + bj * dx;
                        acc[1] += a * fv.y + bj * dy;
                        acc[2] += a * fv.z + bj * dz;
                        const T bt = b * (dx * ft.x + dy * ft.y + dz * ft.z);
                        aj[i][0] += a * ft.x + bt * dx;
                        aj[i][1] += a * ft.y + bt * dy;
                        aj[i][2] += a * ft.z + bt * dz;
                    } else if (KERNEL == SE_ROTLET) {
                        acc[0] += b * (fv.y * dz - fv.z * dy);
                        acc[1] += b * (fv.z * dx - fv.x * dz);
                        acc[2] += b * (fv.x * dy - fv.y * dx);
                        aj[i][0] -= b * (ft.y * dz - ft.z * dy);
                        aj[i][1] -= b * (ft.z * dx - ft.x * dz);
                        aj[i][2] -= b * (ft.x * dy - ft.y * dx);
                    } else {
                        const vec4<T> qv = sq[j];
                        const T hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
                        {
                            const T hf = hx * fv.x + hy * fv.y + hz * fv.z;
                            const T hq = hx * qv.x + hy * qv.y + hz * qv.z;
                            const T fq = fv.x * qv.x + fv.y * qv.y + fv.z * qv.z;
                            const T a1 = a * hf * hq;
                            acc[0] += a1 * hx + b * (hx * fq + fv.x * hq + qv.x * hf);
                            acc[1] += a1 * hy + b * (hy * fq + fv.y * hq + qv.y * hf);
                            acc[2] += a1 * hz + b * (hz * fq + fv.z * hq + qv.z * hf);
                        }
                        {
                            const T hf = hx * ft.x + hy * ft.y + hz * ft.z;
                            const T hq = hx * qt.x + hy * qt.y + hz * qt.z;
                            const T fq = ft.x * qt.x + ft.y * qt.y + ft.z * qt.z;
                            const T a1 = a * hf * hq;
                            aj[i][0] -= a1 * hx + b * (hx * fq + ft.x * hq + qt.x * hf);
                            aj[i][1] -= a1 * hy + b * (hy * fq + ft.y * hq + qt.y * hf);
                            aj[i][2] -= a1 * hz + b * (hz * fq + ft.z * hq + qt.z * hf);
                        }
                    }
                } else {
                    coinc = true;  // a distinct point at the same position
                }
            }
        };
        if (nch == 32) {
#pragma unroll
            for (int i = 0; i < NC; i++) step(i, s + NS * i);
        } else {
#pragma unroll
            for (int i = 0; i < NC; i++)
                if (s + NS * i < nch) step(i, s + NS * i);
        }
        for (int d = 0; d < 3; d++) {
            kahan_add(ks[d], kc[d], acc[d]);
            acc[d] = T(0);
        }
        // reduce-scatter over the TPW lanes of the stream: afterwards aj[0] of
        // lane k holds the total of candidate i = k (slot s + NS k)
#pragma unroll
        for (int h = NC / 2; h >= 1; h >>= 1) {
            const bool up = (k & h) != 0;
#pragma unroll
            for (int q = 0; q < h; q++)
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const T send = up ? aj[q][d] : aj[q + h][d];
                    const T keep = up ? aj[q + h][d] : aj[q][d];
                    aj[q][d] = keep + __shfl_xor_sync(FULL, send, h);
                }
        }
        const int jm = s + NS * k;
        if (jm < nch && (aj[0][0] != T(0) || aj[0][1] != T(0) || aj[0][2] != T(0))) {
            T *dst = uj + 4 * (size_t)smi[jm];
            if constexpr (sizeof(T) == 4) {
                atomicAdd(reinterpret_cast<float4 *>(dst), make_float4(aj[0][0], aj[0][1], aj[0][2], 0.f));
            } else {
                atomicAdd(dst, aj[0][0]);
                atomicAdd(dst + 1, aj[0][1]);
                atomicAdd(dst + 2, aj[0][2]);
            }
        }
        __syncwarp();
    }
    // combine the NS streams of each target
    T tot[3];
    for (int d = 0; d < 3; d++) {
        T sm_ = ks[d], cm_ = kc[d];
        for (int o = TPW; o < 32; o <<= 1) {
            const T so = __shfl_xor_sync(FULL, sm_, o), co = __shfl_xor_sync(FULL, cm_, o);
            kahan_add(sm_, cm_, so);
            cm_ += co;
        }
        tot[d] = sm_ - cm_;
    }
    if (__any_sync(FULL, coinc) && lane == 0) atomicOr(status, FLAG_COINCIDENT);
    if (s == 0 && has) {
        const int mi = perm[t];
        for (int d = 0; d < 3; d++) u[3 * mi + d] = (T)((double)u[3 * mi + d] + (double)tot[d]);
    }
}

// FP32, one system, one right-hand side, each pair within the cutoff once,
// with the lanes transposed relative to k_real_sym: a warp owns a cluster of up
// to TC = 8 consecutive targets, held in shared memory and read as broadcasts,
// and each lane evaluates one candidate against all TC targets in turn.  The
// candidate stream is the one of k_real_sym (rows at or after the cluster's row,
// the own row from the cluster's first point on).  Each streamed candidate is
// first tested against the bounding box of the cluster's targets (farther than
// rc from the box means farther than rc from every target; the box test rounds
// the same way as the pair test, so it never drops a pair), and the survivors
// are queued in shared memory with their stream position.  Each queue of 32 is
// evaluated one candidate per lane:
//   u_t += K^R(x_t - x_m) . s_m   in TC x 3 register accumulators per lane,
//                                  summed over the lanes once per cluster, and
//   u_m += sign K^R(x_t - x_m) . s_t  in 3 registers, added to uj with one
//                                  vector atomic per candidate (sign -1 for the
//                                  odd stresslet and rotlet).
// A pair counts when the candidate's stream position exceeds the target's slot
// (positions below the cluster's size are the cluster's own points).
#ifndef SE_RS_SYMC_MINB
#define SE_RS_SYMC_MINB 4
#endif
// the stresslet's paired pair sum needs more registers: 2 blocks of 256 (128 each)
#ifndef SE_RS_SYMC_MINB_STR
#define SE_RS_SYMC_MINB_STR 2
#endif
// PER (periodic plans, stokeslet and rotlet): the rows of cells wrap around
// the box, each at most once, the own row rotated to the front of the stream;
// each row's x-range wraps into at most two segments (in the own row only the
// positions from the cluster's first point on).  Every candidate is moved to
// its image nearest the centre of the targets' box, which is every target's
// nearest image when the box's half-width plus rc stays below L/2; a wider
// cluster takes nearest images pair by pair instead.
// GRAD: the position gradient of the real-space part of L = sum_m g_m . u_m
// instead of u (stokeslet, rotlet; qs holds g in cell order): the pair term
// Phi = g_t . K(d) f_j + g_j . K(-d) f_t, d = x_t - x_j, adds grad Phi to the
// target and -grad Phi to the candidate.
template <int KERNEL, int PV, bool PER = false, bool GRAD = false>
__global__ void __launch_bounds__(256, (KERNEL == SE_STRESSLET || GRAD) ? SE_RS_SYMC_MINB_STR : SE_RS_SYMC_MINB)
    k_real_symc(GP<float> g, RC<float> rk, const float4 *__restrict__ xs, const float4 *__restrict__ fs,
                const float4 *__restrict__ qs, const int *__restrict__ cell_start, const int2 *__restrict__ clusters,
                const int *__restrict__ ncl_total, const int *__restrict__ perm, float *__restrict__ u,
                float *__restrict__ uj, int *__restrict__ status, float *__restrict__ rt,
                const float4 *__restrict__ gs = nullptr) {
    constexpr int WPB = 8, TC = 8, QN = 64;
    constexpr bool STR = (KERNEL == SE_STRESSLET);
    static_assert(!(PER && STR), "periodic plans sum the stresslet with k_real_cmp");
    static_assert(!(GRAD && PER), "the gradient mode is for free-space plans");
    constexpr bool HQ = STR || GRAD;   // a third vector per point: q, or g
    constexpr bool HG = STR && GRAD;   // and a fourth: the stresslet's gradient needs q and g
    constexpr int NSEG = PER ? 2 * MAXROWS : MAXROWS;  // entries of the segment list
    // PAIR: neighbouring targets 2p and 2p + 1 side by side (their cutoff
    // tests mostly agree); the components are x, f and, for the stresslet, q
    // and f.q
    constexpr bool PAIR = SE_RS_PAIR && (!STR || SE_RS_PAIR_STR) && !GRAD;
    constexpr int NTP = STR ? 10 : 6;
    // one warp's shared memory in one record, so that one base address serves
    // every access
    struct __align__(16) WarpSmem {
        float4 tx[TC], tf[TC], tq[HQ ? TC : 1], tg[HG ? TC : 1];
        // the candidate queue (the stresslet's gradient reads q and g of a
        // candidate through its index instead, to stay within 48 KB per block)
        float4 qx[QN], qf[QN], qq[HQ && !HG ? QN : 1];
        float tp[PAIR ? TC / 2 : 1][NTP][2];      // [pair p][component][slot]: 16-byte loads of two components
        int qm[QN];
        int2 seg[NSEG];
        int pre[NSEG + 1];
        float box[6];
    };
    __shared__ WarpSmem ws_all[WPB];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * WPB + wib;
    if (c >= *ncl_total) return;
    WarpSmem &W = ws_all[wib];
    float4 *tx = W.tx, *tf = W.tf, *tq = W.tq;
    float (*tp)[NTP][2] = W.tp;
    float *box = W.box;
    float4 *qx = W.qx, *qf = W.qf, *qq = W.qq;
    int *qm = W.qm;
    int2 *seg = W.seg;
    int *pre = W.pre;
    const int2 cl = clusters[c];
    const float INF = __int_as_float(0x7f800000);
    // the cluster's targets (slots beyond its size at infinity: no pair) and
    // their bounding box
    float blo[3] = {INF, INF, INF}, bhi[3] = {-INF, -INF, -INF};
    if (lane < TC) {
        float4 xo = make_float4(INF, INF, INF, 0.f), fo = make_float4(0.f, 0.f, 0.f, 0.f), qo = fo, go = fo;
        if (lane < cl.y) {
            xo = xs[cl.x + lane];
            fo = fs[cl.x + lane];
            if (HQ) qo = qs[cl.x + lane];
            if (HG) go = gs[cl.x + lane];
            blo[0] = bhi[0] = xo.x;
            blo[1] = bhi[1] = xo.y;
            blo[2] = bhi[2] = xo.z;
        }
        tx[lane] = xo;
        tf[lane] = fo;
        if (HQ) tq[lane] = qo;
        if (HG) W.tg[lane] = go;
        if (PAIR) {
            // empty slots far away but finite: a masked slot's products stay 0
            const int pp = lane >> 1, o = lane & 1;  // pair p = t / 2, slot t mod 2
            const bool real = lane < cl.y;
            tp[pp][0][o] = real ? xo.x : 1e18f;
            tp[pp][1][o] = real ? xo.y : 1e18f;
            tp[pp][2][o] = real ? xo.z : 1e18f;
            tp[pp][3][o] = fo.x;
            tp[pp][4][o] = fo.y;
            tp[pp][5][o] = fo.z;
            if (STR) {
                tp[pp][6][o] = qo.x;
                tp[pp][7][o] = qo.y;
                tp[pp][8][o] = qo.z;
                tp[pp][9][o] = fo.x * qo.x + fo.y * qo.y + fo.z * qo.z;
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            blo[d] = fminf(blo[d], __shfl_xor_sync(FULL, blo[d], o));
            bhi[d] = fmaxf(bhi[d], __shfl_xor_sync(FULL, bhi[d], o));
        }
        if (lane == 0) {
            box[d] = blo[d];
            box[3 + d] = bhi[d];
        }
    }
    int c0[3], c1[3];
    unpack3(get_tag(xs[cl.x]), c0[0], c0[1], c0[2]);
    unpack3(get_tag(xs[cl.x + cl.y - 1]), c1[0], c1[1], c1[2]);
    const float rc2m = rk.rc2 * 1.0001f;
    const int own_row = c0[2] * g.ncel[1] + c0[1];
    // PER: the centre of the targets' box and whether one image shift per
    // candidate serves every target
    float ctr[3] = {0.f, 0.f, 0.f};
    bool wide = false;
    if constexpr (PER) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            ctr[d] = 0.5f * (blo[d] + bhi[d]);
            wide |= 0.5f * (bhi[d] - blo[d]) + sqrtf(rk.rc2) >= 0.49f * g.len[d];
        }
    }
    int nseg;
    if constexpr (PER) {
        const int ny = g.ncel[1], nz = g.ncel[2], nx = g.ncel[0];
        const int Wy = min(2 * rk.reach[0] + 1, ny), Wz = min(2 * rk.reach[1] + 1, nz);
        const int oy = (Wy - 1) / 2, oz = (Wz - 1) / 2, nrows = Wy * Wz, centre = oz * Wy + oy;
        for (int r = lane; r < nrows; r += 32) {
            const int rr = (r + centre) % nrows;  // r = 0: the own row
            const int dyc = (rr % Wy) - oy, dzc = (rr / Wy) - oz;
            const int iy = (c0[1] + dyc + ny) % ny, iz = (c0[2] + dzc + nz) % nz;
            const int row = iz * ny + iy;
            int2 s0 = make_int2(0, 0), s1 = make_int2(0, 0);
            if (row >= own_row) {
                const float dy = (Wy == ny) ? 0.f : float(max(abs(dyc) - 1, 0)) * g.cw[1];
                const float dz = (Wz == nz) ? 0.f : float(max(abs(dzc) - 1, 0)) * g.cw[2];
                const float d2 = dy * dy + dz * dz;
                if (d2 <= rc2m) {
                    const float del = sqrtf(rc2m - d2) + 1e-4f * g.cw[0];
                    const int ixl = (int)floorf((float(c0[0]) * g.cw[0] - del) * g.icw[0]);
                    const int ixh = (int)floorf((float(c1[0] + 1) * g.cw[0] + del) * g.icw[0]);
                    const int base = row * nx;
                    const bool own = (row == own_row);
                    if (ixh - ixl + 1 >= nx) {
                        s0 = make_int2(own ? cl.x : cell_start[base], cell_start[base + nx]);
                    } else {
                        // the unwrapped core (it holds the cluster in the own row)
                        const int a = max(ixl, 0), b = min(ixh, nx - 1);
                        s0 = make_int2(own ? cl.x : cell_start[base + a], cell_start[base + b + 1]);
                        if (ixl < 0)  // cells at the end of the row (later positions)
                            s1 = make_int2(cell_start[base + nx + ixl], cell_start[base + nx]);
                        else if (ixh >= nx && !own)  // cells at its start (earlier positions)
                            s1 = make_int2(cell_start[base], cell_start[base + ixh - nx + 1]);
                    }
                }
            }
            seg[2 * r] = s0;
            seg[2 * r + 1] = s1;
        }
        nseg = 2 * nrows;
    } else {
    const int Ry = rk.reach[0], Rz = rk.reach[1], Wy = 2 * Ry + 1, nrows = Wy * (2 * Rz + 1);
    nseg = nrows;
    for (int r = lane; r < nrows; r += 32) {
        const int dyc = (r % Wy) - Ry, dzc = (r / Wy) - Rz;
        const int iy = c0[1] + dyc, iz = c0[2] + dzc;
        int2 sg = make_int2(0, 0);
        const int row = iz * g.ncel[1] + iy;
        if (iy >= 0 && iy < g.ncel[1] && iz >= 0 && iz < g.ncel[2] && row >= own_row) {
            const float dy = float(max(abs(dyc) - 1, 0)) * g.cw[1], dz = float(max(abs(dzc) - 1, 0)) * g.cw[2];
            const float d2 = dy * dy + dz * dz;
            if (d2 <= rc2m) {
                const float del = sqrtf(rc2m - d2) + 1e-4f * g.cw[0];
                const int ixl = max(0, (int)floorf((float(c0[0]) * g.cw[0] - del) * g.icw[0]));
                const int ixh = min(g.ncel[0] - 1, (int)floorf((float(c1[0] + 1) * g.cw[0] + del) * g.icw[0]));
                if (ixl <= ixh) {
                    const int base = row * g.ncel[0];
                    sg = make_int2(cell_start[base + ixl], cell_start[base + ixh + 1]);
                    if (row == own_row) sg.x = cl.x;
                }
            }
        }
        seg[r] = sg;
    }
    }
    __syncwarp();
    int run = 0;
    for (int r0 = 0; r0 < nseg; r0 += 32) {
        const int r = r0 + lane;
        const int len = (r < nseg) ? seg[r].y - seg[r].x : 0;
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (r < nseg) pre[r] = run + incl - len;
        run += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) pre[nseg] = run;
    __syncwarp();
    const int total = run;
    float acc[TC][3];
#pragma unroll
    for (int t = 0; t < TC; t++) acc[t][0] = acc[t][1] = acc[t][2] = 0.f;
    float2 accp[TC / 2][3];  // PAIR: targets (2p, 2p + 1)
#pragma unroll
    for (int p2 = 0; p2 < TC / 2; p2++) accp[p2][0] = accp[p2][1] = accp[p2][2] = f2(0.f);
    bool coinc = false;
    int lo = 0, fill = 0, cb = 0;
    while (true) {
        // queue candidates until 32 wait or the stream ends
        while (fill < 32 && cb < total) {
            const int v = cb + lane;
            bool keep = false;
            int m = 0;
            float4 xm = make_float4(0.f, 0.f, 0.f, 0.f);
            if (v < total) {
                while (pre[lo + 1] <= v) lo++;
                m = seg[lo].x + (v - pre[lo]);
                xm = xs[m];
                if (PER && !wide) {
                    // the image nearest the centre of the targets' box
                    xm.x += g.len[0] * rintf((ctr[0] - xm.x) * g.ilen[0]);
                    xm.y += g.len[1] * rintf((ctr[1] - xm.y) * g.ilen[1]);
                    xm.z += g.len[2] * rintf((ctr[2] - xm.z) * g.ilen[2]);
                }
                const float ex = fmaxf(fmaxf(box[0] - xm.x, xm.x - box[3]), 0.f);
                const float ey = fmaxf(fmaxf(box[1] - xm.y, xm.y - box[4]), 0.f);
                const float ez = fmaxf(fmaxf(box[2] - xm.z, xm.z - box[5]), 0.f);
                keep = (PER && wide) || ex * ex + ey * ey + ez * ez <= rc2m;
            }
            const unsigned bal = __ballot_sync(FULL, keep);
            if (keep) {
                const int pos = fill + __popc(bal & ((1u << lane) - 1u));
                xm.w = __int_as_float(min(v, TC));  // the stream position, capped
                qx[pos] = xm;
                qf[pos] = fs[m];
                if (HQ && !HG) qq[pos] = qs[m];
                qm[pos] = m;
            }
            fill += __popc(bal);
            cb += 32;
        }
        if (fill == 0) break;
        __syncwarp();
        const int nq = min(fill, 32);
        {
            const bool valid = lane < nq;
            // an idle lane's candidate: at infinity, or far but finite on the paired
            // path, on the other side from the empty target slots (+1e18), so that
            // the two never meet at distance zero
            const float far = PAIR ? -1e18f : INF;
            float4 xj = make_float4(far, far, far, 0.f);
            float4 fj = make_float4(0.f, 0.f, 0.f, 0.f), qj = fj, gj = fj;
            int vs = 0, mj = 0;
            if (valid) {
                xj = qx[lane];
                fj = qf[lane];
                if (HQ && !HG) qj = qq[lane];
                if (HG) {
                    qj = qs[qm[lane]];
                    gj = gs[qm[lane]];
                }
                vs = __float_as_int(xj.w);
                mj = qm[lane];
            }
            float cj[3] = {0.f, 0.f, 0.f};
            if constexpr (PAIR) {
                const float2 nx = f2(-xj.x), ny = f2(-xj.y), nz = f2(-xj.z);
                const float2 fx = f2(fj.x), fy = f2(fj.y), fz = f2(fj.z);
                const float2 qx = f2(qj.x), qy = f2(qj.y), qz = f2(qj.z);
                const float2 fqj = f2(fj.x * qj.x + fj.y * qj.y + fj.z * qj.z);
                float2 c2[3] = {f2(0.f), f2(0.f), f2(0.f)};
#pragma unroll
                for (int p2 = 0; p2 < TC / 2; p2++) {
                    const float4 *t4 = reinterpret_cast<const float4 *>(tp[p2]);
                    const float4 v0 = t4[0], v1 = t4[1], v2 = t4[2];
                    float2 dx = __fadd2_rn(make_float2(v0.x, v0.y), nx);
                    float2 dy = __fadd2_rn(make_float2(v0.z, v0.w), ny);
                    float2 dz = __fadd2_rn(make_float2(v1.x, v1.y), nz);
                    if (PER && wide) {
                        // nearest images pair by pair
                        dx.x -= g.len[0] * rintf(dx.x * g.ilen[0]);
                        dx.y -= g.len[0] * rintf(dx.y * g.ilen[0]);
                        dy.x -= g.len[1] * rintf(dy.x * g.ilen[1]);
                        dy.y -= g.len[1] * rintf(dy.y * g.ilen[1]);
                        dz.x -= g.len[2] * rintf(dz.x * g.ilen[2]);
                        dz.y -= g.len[2] * rintf(dz.y * g.ilen[2]);
                    }
                    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                    bool ia = r2.x <= rk.rc2 && 2 * p2 < vs, ib = r2.y <= rk.rc2 && 2 * p2 + 1 < vs;
                    if (PER && wide) {
                        // the empty slots' far position folds back under nearest images
                        ia = ia && 2 * p2 < cl.y;
                        ib = ib && 2 * p2 + 1 < cl.y;
                    }
                    if (!SE_RS_BRANCH || ia || ib) {
                        // zero distance: a distinct point at the same position, skipped
                        const bool ua = ia && r2.x > 0.f, ub = ib && r2.y > 0.f;
                        coinc |= (ia && !ua) || (ib && !ub);
                        float2 a, b;
                        if constexpr (!STR) radial_ab2<PV>(rk, r2, ua, ub, a, b);
                        const float2 gx = make_float2(v1.z, v1.w), gy = make_float2(v2.x, v2.y),
                                     gz = make_float2(v2.z, v2.w);
                        if constexpr (STR) {
                            // u_t += T(d).(f_j, q_j),  u_j -= T(d).(f_t, q_t)
                            float2 A, B;
                            radial_ab2_str<PV>(rk, r2, ua, ub, A, B);
                            const float2 df = __ffma2_rn(dz, fz, __ffma2_rn(dy, fy, __fmul2_rn(dx, fx)));
                            const float2 dq = __ffma2_rn(dz, qz, __ffma2_rn(dy, qy, __fmul2_rn(dx, qx)));
                            const float2 s = __fmul2_rn(__fmul2_rn(A, df), dq);
                            const float2 w0 = __ffma2_rn(df, qx, __ffma2_rn(dq, fx, __fmul2_rn(fqj, dx)));
                            const float2 w1 = __ffma2_rn(df, qy, __ffma2_rn(dq, fy, __fmul2_rn(fqj, dy)));
                            const float2 w2 = __ffma2_rn(df, qz, __ffma2_rn(dq, fz, __fmul2_rn(fqj, dz)));
                            accp[p2][0] = __ffma2_rn(s, dx, __ffma2_rn(B, w0, accp[p2][0]));
                            accp[p2][1] = __ffma2_rn(s, dy, __ffma2_rn(B, w1, accp[p2][1]));
                            accp[p2][2] = __ffma2_rn(s, dz, __ffma2_rn(B, w2, accp[p2][2]));
                            const float4 v3 = t4[3], v4 = t4[4];
                            const float2 hx = make_float2(v3.x, v3.y), hy = make_float2(v3.z, v3.w);
                            const float2 hz = make_float2(v4.x, v4.y), fqt = make_float2(v4.z, v4.w);
                            const float2 dg = __ffma2_rn(dz, gz, __ffma2_rn(dy, gy, __fmul2_rn(dx, gx)));
                            const float2 dh = __ffma2_rn(dz, hz, __ffma2_rn(dy, hy, __fmul2_rn(dx, hx)));
                            const float2 nB = __fmul2_rn(f2(-1.f), B);
                            const float2 ns = __fmul2_rn(__fmul2_rn(__fmul2_rn(f2(-1.f), A), dg), dh);
                            const float2 v0 = __ffma2_rn(dg, hx, __ffma2_rn(dh, gx, __fmul2_rn(fqt, dx)));
                            const float2 v1 = __ffma2_rn(dg, hy, __ffma2_rn(dh, gy, __fmul2_rn(fqt, dy)));
                            const float2 v2 = __ffma2_rn(dg, hz, __ffma2_rn(dh, gz, __fmul2_rn(fqt, dz)));
                            c2[0] = __ffma2_rn(ns, dx, __ffma2_rn(nB, v0, c2[0]));
                            c2[1] = __ffma2_rn(ns, dy, __ffma2_rn(nB, v1, c2[1]));
                            c2[2] = __ffma2_rn(ns, dz, __ffma2_rn(nB, v2, c2[2]));
                        } else if (KERNEL == SE_STOKESLET) {
                            const float2 bj = __fmul2_rn(b, __ffma2_rn(dz, fz, __ffma2_rn(dy, fy, __fmul2_rn(dx, fx))));
                            accp[p2][0] = __ffma2_rn(a, fx, __ffma2_rn(bj, dx, accp[p2][0]));
                            accp[p2][1] = __ffma2_rn(a, fy, __ffma2_rn(bj, dy, accp[p2][1]));
                            accp[p2][2] = __ffma2_rn(a, fz, __ffma2_rn(bj, dz, accp[p2][2]));
                            const float2 bt = __fmul2_rn(b, __ffma2_rn(dz, gz, __ffma2_rn(dy, gy, __fmul2_rn(dx, gx))));
                            c2[0] = __ffma2_rn(a, gx, __ffma2_rn(bt, dx, c2[0]));
                            c2[1] = __ffma2_rn(a, gy, __ffma2_rn(bt, dy, c2[1]));
                            c2[2] = __ffma2_rn(a, gz, __ffma2_rn(bt, dz, c2[2]));
                        } else {
                            // rotlet: u_t += b (f_j x d), u_j -= b (f_t x d)
                            const float2 nb = __fmul2_rn(f2(-1.f), b);
                            accp[p2][0] = __ffma2_rn(b, __ffma2_rn(fy, dz, __fmul2_rn(f2(-fj.z), dy)), accp[p2][0]);
                            accp[p2][1] = __ffma2_rn(b, __ffma2_rn(fz, dx, __fmul2_rn(f2(-fj.x), dz)), accp[p2][1]);
                            accp[p2][2] = __ffma2_rn(b, __ffma2_rn(fx, dy, __fmul2_rn(f2(-fj.y), dx)), accp[p2][2]);
                            c2[0] = __ffma2_rn(nb, __ffma2_rn(gy, dz, __fmul2_rn(__fmul2_rn(f2(-1.f), gz), dy)), c2[0]);
                            c2[1] = __ffma2_rn(nb, __ffma2_rn(gz, dx, __fmul2_rn(__fmul2_rn(f2(-1.f), gx), dz)), c2[1]);
                            c2[2] = __ffma2_rn(nb, __ffma2_rn(gx, dy, __fmul2_rn(__fmul2_rn(f2(-1.f), gy), dx)), c2[2]);
                        }
                    }
                }
#pragma unroll
                for (int d = 0; d < 3; d++) cj[d] = c2[d].x + c2[d].y;
            } else
#pragma unroll
            for (int t = 0; t < TC; t++) {
                const float4 xt = tx[t];
                const float dx = xt.x - xj.x, dy = xt.y - xj.y, dz = xt.z - xj.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (r2 <= rk.rc2 && t < vs) {
                    if (GRAD && r2 > 0.f) {
                        float G[3];
                        if constexpr (HG)
                            grad_pair_str<PV>(rk, dx, dy, dz, r2, tf[t], tq[t], W.tg[t], fj, qj, gj, G);
                        else
                            grad_pair<KERNEL, PV>(rk, dx, dy, dz, r2, tf[t], tq[t], fj, qj, G);
                        acc[t][0] += G[0];
                        acc[t][1] += G[1];
                        acc[t][2] += G[2];
                        cj[0] -= G[0];
                        cj[1] -= G[1];
                        cj[2] -= G[2];
                    } else if (r2 > 0.f) {
                        float rinv, a, b;
                        radial_ab<KERNEL, PV>(rk, r2, rinv, a, b);
                        const float4 ft = tf[t];
                        if (KERNEL == SE_STOKESLET) {
                            const float bj = b * (dx * fj.x + dy * fj.y + dz * fj.z);
                            acc[t][0] += a * fj.x + bj * dx;
                            acc[t][1] += a * fj.y + bj * dy;
                            acc[t][2] += a * fj.z + bj * dz;
                            const float bt = b * (dx * ft.x + dy * ft.y + dz * ft.z);
                            cj[0] += a * ft.x + bt * dx;
                            cj[1] += a * ft.y + bt * dy;
                            cj[2] += a * ft.z + bt * dz;
                        } else if (KERNEL == SE_ROTLET) {
                            acc[t][0] += b * (fj.y * dz - fj.z * dy);
                            acc[t][1] += b * (fj.z * dx - fj.x * dz);
                            acc[t][2] += b * (fj.x * dy - fj.y * dx);
                            cj[0] -= b * (ft.y * dz - ft.z * dy);
                            cj[1] -= b * (ft.z * dx - ft.x * dz);
                            cj[2] -= b * (ft.x * dy - ft.y * dx);
                        } else {
                            const float4 qt = tq[t];
                            const float hx = dx * rinv, hy = dy * rinv, hz = dz * rinv;
                            {
                                const float hf = hx * fj.x + hy * fj.y + hz * fj.z;
                                const float hq = hx * qj.x + hy * qj.y + hz * qj.z;
                                const float fq = fj.x * qj.x + fj.y * qj.y + fj.z * qj.z;
                                const float a1 = a * hf * hq;
                                acc[t][0] += a1 * hx + b * (hx * fq + fj.x * hq + qj.x * hf);
                                acc[t][1] += a1 * hy + b * (hy * fq + fj.y * hq + qj.y * hf);
                                acc[t][2] += a1 * hz + b * (hz * fq + fj.z * hq + qj.z * hf);
                            }
                            {
                                const float hf = hx * ft.x + hy * ft.y + hz * ft.z;
                                const float hq = hx * qt.x + hy * qt.y + hz * qt.z;
                                const float fq = ft.x * qt.x + ft.y * qt.y + ft.z * qt.z;
                                const float a1 = a * hf * hq;
                                cj[0] -= a1 * hx + b * (hx * fq + ft.x * hq + qt.x * hf);
                                cj[1] -= a1 * hy + b * (hy * fq + ft.y * hq + qt.y * hf);
                                cj[2] -= a1 * hz + b * (hz * fq + ft.z * hq + qt.z * hf);
                            }
                        }
                    } else {
                        coinc = true;  // a distinct point at the same position
                    }
                }
            }
            if (valid && (cj[0] != 0.f || cj[1] != 0.f || cj[2] != 0.f))
                atomicAdd(reinterpret_cast<float4 *>(uj + 4 * (size_t)mj), make_float4(cj[0], cj[1], cj[2], 0.f));
        }
        __syncwarp();
        // keep the queue's tail
        if (lane < fill - nq) {
            qx[lane] = qx[nq + lane];
            qf[lane] = qf[nq + lane];
            if (HQ && !HG) qq[lane] = qq[nq + lane];
            qm[lane] = qm[nq + lane];
        }
        fill -= nq;
        __syncwarp();
    }
    if constexpr (PAIR) {
#pragma unroll
        for (int p2 = 0; p2 < TC / 2; p2++)
#pragma unroll
            for (int d = 0; d < 3; d++) {
                acc[2 * p2][d] = accp[p2][d].x;
                acc[2 * p2 + 1][d] = accp[p2][d].y;
            }
    }
    // sum the accumulators over the lanes: a reduce-scatter over lane bits 4,
    // 3, 2 leaves lane l with the 3 components of target ((l >> 2) & 7) summed
    // over 8 lanes, then butterflies over bits 1, 0 finish the sums
    float* a = &acc[0][0];
#pragma unroll
    for (int h = 16, len = 3 * TC; h >= 4; h >>= 1, len >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < len / 2; i++) {
            const float send = up ? a[i] : a[i + len / 2];
            const float keep = up ? a[i + len / 2] : a[i];
            a[i] = keep + __shfl_xor_sync(FULL, send, h);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; d++) {
        a[d] += __shfl_xor_sync(FULL, a[d], 2);
        a[d] += __shfl_xor_sync(FULL, a[d], 1);
    }
    if (__any_sync(FULL, coinc) && lane == 0) atomicOr(status, FLAG_COINCIDENT);
    const int tt = (((lane >> 4) & 1) << 2) | (((lane >> 3) & 1) << 1) | ((lane >> 2) & 1);
    if ((lane & 3) == 0 && tt < cl.y) {
        if (rt) {
            // overlapped evaluation: u is being written by the gather meanwhile
            *reinterpret_cast<float4 *>(rt + 4 * (size_t)(cl.x + tt)) = make_float4(a[0], a[1], a[2], 0.f);
        } else {
            const int mi = perm[cl.x + tt];
            for (int d = 0; d < 3; d++) u[3 * mi + d] = (float)((double)u[3 * mi + d] + (double)a[d]);
        }
    }
}

// u[perm[n]] += uj[n] (the contributions scattered to the candidates)
template <typename T>
__global__ void k_add_uj(int N, const T *__restrict__ uj, const int *__restrict__ perm, T *__restrict__ u,
                         const T *__restrict__ rt = nullptr) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int m = perm[n];
    if (rt) {
        // u[perm[n]] += rt[n] + uj[n] (the target and the candidate sums)
        for (int d = 0; d < 3; d++)
            u[3 * m + d] = (T)((double)u[3 * m + d] + (double)rt[4 * (size_t)n + d] + (double)uj[4 * (size_t)n + d]);
        return;
    }
    for (int d = 0; d < 3; d++) u[3 * m + d] = (T)((double)u[3 * m + d] + (double)uj[4 * (size_t)n + d]);
}

// Batched cluster lists: row `row` of all systems' cell rows belongs to the
// system s with row_base[s] <= row < row_base[s+1].
template <typename T>
__global__ void k_bcluster_count(int nrows_tot, const BSys<T> *__restrict__ sys, const int *__restrict__ row_base,
                                 int S, int tpw, const int *__restrict__ cell_start, int *ncl) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows_tot) return;
    const int s = find_range(row_base, S, row);
    const BSys<T> &B = sys[s];
    const int ncdx = B.g.ncel[0], lr = row - row_base[s];
    const int *cs = cell_start + B.cell_base;
    const int len = cs[(lr + 1) * ncdx] - cs[lr * ncdx];
    ncl[row] = (len + tpw - 1) / tpw;
}

template <typename T>
__global__ void k_bcluster_fill(int nrows_tot, const BSys<T> *__restrict__ sys, const int *__restrict__ row_base,
                                int S, int tpw, const int *__restrict__ cell_start,
                                const int *__restrict__ ncl_start, int2 *__restrict__ cl, int *__restrict__ cl_sys) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows_tot) return;
    const int s = find_range(row_base, S, row);
    const BSys<T> &B = sys[s];
    const int ncdx = B.g.ncel[0], lr = row - row_base[s];
    const int *cs = cell_start + B.cell_base;
    const int a = cs[lr * ncdx], b = cs[(lr + 1) * ncdx];
    int o = ncl_start[row];
    for (int q = a; q < b; q += tpw) {
        cl[o] = make_int2(q, min(tpw, b - q));
        cl_sys[o] = s;
        o++;
    }
}

// One warp per target with ballot compaction of the candidates (the FP64 path,
// where evaluating a pair costs far more than testing one): lanes stream the
// candidates of the target's rows 32 at a time, those inside the cutoff are
// appended to a per-warp queue, and every full queue of 32 pairs is evaluated
// with all lanes busy.
// ADJ (stresslet backward, fs holding the upstream gradient g in cell order):
// the strength gradients of the real-space part, for target p
//   u[p]  += gf_p = -sum_m T^R(x_p - x_m)(g_m, q_p),
//   gq[p] += gq_p = -sum_m T^R(x_p - x_m)(g_m, f_p)
// (T^R(x_m - x_p) = -T^R(x_p - x_m); T^R(r)(a, b)_j = T^R_jlk a_l b_k).
// PER: periodic plan, nearest images (rc < L/2).
template <typename T, int KERNEL, bool ADJ = false, bool PER = false>
__global__ void __launch_bounds__(256) k_real_cmp(GP<T> g, RC<T> rk, int N, const vec4<T> *__restrict__ xs,
                                                  const vec4<T> *__restrict__ fs, const vec4<T> *__restrict__ qs,
                                                  const int *__restrict__ cell_start, const int *__restrict__ perm,
                                                  T *__restrict__ u, int *__restrict__ status,
                                                  const T *__restrict__ f_orig = nullptr,
                                                  const T *__restrict__ q_orig = nullptr, T *__restrict__ gq = nullptr) {
    constexpr int WPB = 8;
    __shared__ vec4<T> qd_all[WPB][QCAP];
    __shared__ int qn_all[WPB][QCAP];
    __shared__ int2 seg_all[WPB][PER ? 2 * MAXROWS : MAXROWS];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * WPB + wib;
    if (t >= N) return;
    vec4<T> *qd = qd_all[wib];
    int *qn = qn_all[wib];
    int2 *seg = seg_all[wib];
    const vec4<T> xt = xs[t];
    int nrows;
    if constexpr (PER)
        nrows = row_segments_per(g, rk, xt, cell_start, lane, seg);
    else
        nrows = row_segments(g, rk, xt, cell_start, lane, seg);
    T acc[3] = {0, 0, 0}, acc2[3] = {0, 0, 0};
    int cnt = 0;
    bool coinc = false;
    const unsigned lt = (1u << lane) - 1u;
    vec4<T> zero4;
    zero4.x = zero4.y = zero4.z = zero4.w = 0;
    vec4<T> fp4 = zero4, qp4 = zero4;
    if (ADJ) {
        const int mp = perm[t];
        fp4.x = f_orig[3 * mp]; fp4.y = f_orig[3 * mp + 1]; fp4.z = f_orig[3 * mp + 2];
        qp4.x = q_orig[3 * mp]; qp4.y = q_orig[3 * mp + 1]; qp4.z = q_orig[3 * mp + 2];
    }
    auto eval = [&](int slot) {
        const vec4<T> v = qd[slot];
        const int m = qn[slot];
        if (ADJ) {
            pair_str2<T>(rk, v.x, v.y, v.z, v.w, fs[m], qp4, fp4, acc, acc2);
            return;
        }
        const vec4<T> qv = (KERNEL == SE_STRESSLET) ? qs[m] : zero4;
        pair<T, KERNEL>(rk, v.x, v.y, v.z, v.w, fs[m], qv, acc);
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
                if constexpr (PER) {
                    dx -= g.len[0] * rint(dx * g.ilen[0]);
                    dy -= g.len[1] * rint(dy * g.ilen[1]);
                    dz -= g.len[2] * rint(dz * g.ilen[2]);
                }
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
    double tot[3], tot2[3];
    for (int d = 0; d < 3; d++) {
        double v = (double)acc[d], w = (double)acc2[d];
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(FULL, v, o);
            if (ADJ) w += __shfl_xor_sync(FULL, w, o);
        }
        tot[d] = v;
        tot2[d] = w;
    }
    if (__any_sync(FULL, coinc) && lane == 0) atomicOr(status, FLAG_COINCIDENT);
    if (lane < 3) {
        const int m = perm[t];
        const double v = lane == 0 ? tot[0] : (lane == 1 ? tot[1] : tot[2]);
        if (ADJ) {
            const double w = lane == 0 ? tot2[0] : (lane == 1 ? tot2[1] : tot2[2]);
            if (u) u[3 * m + lane] = (T)((double)u[3 * m + lane] - v);
            if (gq) gq[3 * m + lane] = (T)((double)gq[3 * m + lane] - w);
        } else {
            u[3 * m + lane] = (T)((double)u[3 * m + lane] + v);
        }
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
// e = exp(-xi^2 r^2) and erfc(xi r): FP32 from one exp2 and the erfcx fit
// (erfc = e Q(1/(2 + x)), x = xi r <= 8 on FP32 plans), FP64 from exp and the
// FP64 fit.
__device__ __forceinline__ void s_exp_erfc(const RC<float> &rk, float r2, float r, float &e, float &ec) {
    e = ex2_approx(rk.ce * r2);
    ec = e * erfcx_poly<0>(__fdividef(1.0f, 2.0f + rk.xi * r));
}
__device__ __forceinline__ void s_exp_erfc(const RC<double> &rk, double r2, double r, double &e, double &ec) {
    e = exp(-rk.xi2 * r2);
    ec = erfc_fit64(rk.xi * r, e);
}
__device__ __forceinline__ float s_rsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double s_rsqrt(double v) { return rsqrt(v); }

// The upstream gradient g in the cell order of the real-space sum (as a source).
template <typename T>
__global__ void k_sort_g(int N, const int *__restrict__ perm, const T *__restrict__ g, vec4<T> *__restrict__ gs) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int m = perm[n];
    vec4<T> v;
    v.x = g[3 * m];
    v.y = g[3 * m + 1];
    v.z = g[3 * m + 2];
    v.w = T(0);
    gs[n] = v;
}

template <typename T, int KERNEL>
__global__ void __launch_bounds__(256) k_real_grad(GP<T> g, RC<T> rk, int N, const vec4<T> *__restrict__ xs,
                                                   const vec4<T> *__restrict__ fs, const vec4<T> *__restrict__ qs,
                                                   const int *__restrict__ cell_start,
                                                   const int *__restrict__ perm, const vec4<T> *__restrict__ gs,
                                                   T *__restrict__ gx) {
    constexpr int WPB = 8;
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
    vec4<T> qp;
    if (KERNEL == SE_STRESSLET) qp = qs[t];
    const int mp = perm[t];
    const vec4<T> gpv = gs[t];
    const T gp_[3] = {gpv.x, gpv.y, gpv.z};
    const int nrows = row_segments(g, rk, xt, cell_start, lane, seg);
    T acc[3] = {0, 0, 0};
    int cnt = 0;
    const unsigned lt = (1u << lane) - 1u;
    auto eval = [&](int slot) {
        const vec4<T> v = qd[slot];
        const int n = qn[slot];
        const vec4<T> fn = fs[n];
        const vec4<T> gnv = gs[n];
        const T gn[3] = {gnv.x, gnv.y, gnv.z};
        const T d[3] = {v.x, v.y, v.z};
        const T rinv = s_rsqrt(v.w);
        const T r = v.w * rinv;
        T e, ec;
        s_exp_erfc(rk, v.w, r, e, ec);
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
        } else if (KERNEL == SE_STRESSLET) {
            // Phi(r; g, f, q) = T^R_jlk g_j f_l q_k = a (g.r)(f.r)(q.r) + b [(g.f)(q.r) + (f.q)(g.r) + (q.g)(f.r)],
            // a = t1 / rho^5, b = xi^2 t2 / rho with t1, t2 the stresslet radial functions of x = xi rho,
            // dt1/drho = 8 c1 x^4 e, dt2/drho = 2 c1 (1 - 2 x^2) e; gx_p += grad Phi(r; g_p, f_n, q_n)
            // - grad Phi(r; g_n, f_p, q_p)
            const vec4<T> qn4 = qs[n];
            const T xx = rk.xi * r, x2 = xx * xx;
            const T G2 = c1 * r * e;
            const T t1 = -T(2) * (T(3) * ec + G2 * (T(3) + T(2) * x2));
            const T t2 = T(2) * G2;
            const T dt1 = T(8) * c1 * x2 * x2 * e;
            const T dt2 = T(2) * c1 * (T(1) - T(2) * x2) * e;
            const T r5 = rinv2 * rinv2 * rinv;
            const T aT = t1 * r5;
            const T apT = (dt1 - T(5) * t1 * rinv) * r5 * rinv;
            const T bT = rk.xi2 * t2 * rinv;
            const T bpT = rk.xi2 * (dt2 - t2 * rinv) * rinv2;
            auto gphi = [&](const T gv[3], const T fv[3], const T qv[3], T sgn) {
                const T gd = gv[0] * d[0] + gv[1] * d[1] + gv[2] * d[2];
                const T fd = fv[0] * d[0] + fv[1] * d[1] + fv[2] * d[2];
                const T qd = qv[0] * d[0] + qv[1] * d[1] + qv[2] * d[2];
                const T gf = gv[0] * fv[0] + gv[1] * fv[1] + gv[2] * fv[2];
                const T fq = fv[0] * qv[0] + fv[1] * qv[1] + fv[2] * qv[2];
                const T qg = qv[0] * gv[0] + qv[1] * gv[1] + qv[2] * gv[2];
                const T cr = apT * gd * fd * qd + bpT * (gf * qd + fq * gd + qg * fd);
                for (int a = 0; a < 3; a++)
                    acc[a] += sgn * (cr * d[a] + aT * (fd * qd * gv[a] + gd * qd * fv[a] + gd * fd * qv[a]) +
                                     bT * (gf * qv[a] + fq * gv[a] + qg * fv[a]));
            };
            const T f_n[3] = {fn.x, fn.y, fn.z}, q_n[3] = {qn4.x, qn4.y, qn4.z};
            const T f_p[3] = {fp.x, fp.y, fp.z}, q_p[3] = {qp.x, qp.y, qp.z};
            gphi(gp_, f_n, q_n, T(1));
            gphi(gn, f_p, q_p, T(-1));
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

// The FP32 erfcx fit that covers x = xi r up to xi rc: degree 8 up to 5, else
// degree 10 up to 8 (beyond 8, erfc(x) < 1e-28 and the pair terms vanish in FP32).
inline int real_pv(double xi_rc) { return xi_rc <= 5.0 ? 1 : 0; }

// FP32 single-system real-space sum with each pair evaluated once (1) or the
// full candidate lists (0)
#ifndef SE_RS_SYM
#define SE_RS_SYM 1
#endif
#ifndef SE_RS_SYMC
#define SE_RS_SYMC 1
#endif
#ifndef SE_RS_SYM_TPW
#define SE_RS_SYM_TPW 8
#endif
#ifndef SE_RS_SYM_TPW64
#define SE_RS_SYM_TPW64 8
#endif

#ifndef SE_RS_TPW
#define SE_RS_TPW 16
#endif

template <typename T, int KERNEL>
cudaError_t launch_real_k(se_plan_s *p, cudaStream_t st, const RC<T> &rk, T *u, bool defer) {
    const int N = (int)p->N;
    const vec4<T> *xs = (const vec4<T> *)p->b.xs_r, *fs = (const vec4<T> *)p->b.fs_r,
                  *qs = (const vec4<T> *)p->b.qs_r;
    const GP<T> &g = gp<T>(p);
    // periodic plans: the symmetric kernel for the FP32 stokeslet and rotlet,
    // otherwise one warp per target over the wrapped rows
    constexpr bool per_sym = sizeof(T) == 4 && KERNEL != SE_STRESSLET && SE_RS_SYM && SE_RS_SYMC;
    if (p->periodic && !per_sym) {
        if (p->timing && p->ev_real) cudaEventRecord(p->ev_real, st);
        k_real_cmp<T, KERNEL, false, true><<<(N + 7) / 8, 256, 0, st>>>(g, rk, N, xs, fs, qs, p->b.cnt_r,
                                                                      p->b.perm_r, u, p->b.status);
        p->launches++;
        return cudaGetLastError();
    }
    if (sizeof(T) == 8 && !(p->b.uj && SE_RS_SYM)) {
        if (p->timing && p->ev_real) cudaEventRecord(p->ev_real, st);
        k_real_cmp<T, KERNEL><<<(N + 7) / 8, 256, 0, st>>>(g, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, u,
                                                           p->b.status);
        p->launches++;
        return cudaGetLastError();
    }
    // (deterministic plans: the full lists, whose sums need no atomics)
    const bool sym = p->b.uj && SE_RS_SYM && !p->deterministic;
    // targets per cluster: the symmetric kernel's or the full-list kernel's
    // (FP32 runs the transposed symmetric kernel, clusters of 8 targets)
    constexpr bool symc = sizeof(T) == 4 && SE_RS_SYMC;
    constexpr int TPW = SE_RS_TPW, TPWS = symc ? 8 : sizeof(T) == 4 ? SE_RS_SYM_TPW : SE_RS_SYM_TPW64;
    const int tpw = sym ? TPWS : TPW;
    const int nrows = p->geom.ncel[1] * p->geom.ncel[2];
    k_cluster_count<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, p->geom.ncel[0], tpw, p->b.cnt_r, p->b.ncl);
    launch_scan(p->b.ncl, nrows, st);
    k_cluster_fill<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, p->geom.ncel[0], tpw, p->b.cnt_r, p->b.ncl,
                                                         p->b.clusters);
    const long max_cl = N / tpw + nrows + 1;
    const unsigned nblk = (unsigned)((max_cl + 7) / 8);
    if (sym) {
        // each pair once, the candidate's share through uj
        cudaError_t e = cudaMemsetAsync(p->b.uj, 0, 4 * sizeof(T) * (size_t)N, st);
        if (e) return e;
        if (p->timing && p->ev_real) cudaEventRecord(p->ev_real, st);
        T *ujt = (T *)p->b.uj;
        if constexpr (symc) {
            const float4 *xf = (const float4 *)xs, *ff = (const float4 *)fs, *qf = (const float4 *)qs;
            float *rtf = defer ? (float *)p->b.rt : nullptr;
            if constexpr (KERNEL != SE_STRESSLET) {
                if (p->periodic) {
                    if (real_pv(p->xi * p->rc) == 1)
                        k_real_symc<KERNEL, 1, true><<<nblk, 256, 0, st>>>(
                            p->gpf, rk, xf, ff, qf, p->b.cnt_r, p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                            (float *)u, (float *)ujt, p->b.status, nullptr);
                    else
                        k_real_symc<KERNEL, 0, true><<<nblk, 256, 0, st>>>(
                            p->gpf, rk, xf, ff, qf, p->b.cnt_r, p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                            (float *)u, (float *)ujt, p->b.status, nullptr);
                    k_add_uj<T><<<(N + 255) / 256, 256, 0, st>>>(N, ujt, p->b.perm_r, u);
                    p->launches += 4 + scan_launch_count(nrows);
                    return cudaGetLastError();
                }
            }
            if (real_pv(p->xi * p->rc) == 1)
                k_real_symc<KERNEL, 1><<<nblk, 256, 0, st>>>(p->gpf, rk, xf, ff, qf, p->b.cnt_r, p->b.clusters,
                                                             p->b.ncl + nrows, p->b.perm_r, (float *)u,
                                                             (float *)ujt, p->b.status, rtf);
            else
                k_real_symc<KERNEL, 0><<<nblk, 256, 0, st>>>(p->gpf, rk, xf, ff, qf, p->b.cnt_r, p->b.clusters,
                                                             p->b.ncl + nrows, p->b.perm_r, (float *)u,
                                                             (float *)ujt, p->b.status, rtf);
            if (defer) {
                p->launches += 3 + scan_launch_count(nrows);
                return cudaGetLastError();
            }
        } else if (real_pv(p->xi * p->rc) == 1)
            k_real_sym<T, KERNEL, 1, TPWS><<<nblk, 256, 0, st>>>(g, rk, xs, fs, qs, p->b.cnt_r, p->b.clusters,
                                                                p->b.ncl + nrows, p->b.perm_r, u, ujt, p->b.status);
        else
            k_real_sym<T, KERNEL, 0, TPWS><<<nblk, 256, 0, st>>>(g, rk, xs, fs, qs, p->b.cnt_r, p->b.clusters,
                                                                p->b.ncl + nrows, p->b.perm_r, u, ujt, p->b.status);
        k_add_uj<T><<<(N + 255) / 256, 256, 0, st>>>(N, ujt, p->b.perm_r, u);
        p->launches += 4 + scan_launch_count(nrows);
        return cudaGetLastError();
    }
    if (p->timing && p->ev_real) cudaEventRecord(p->ev_real, st);
    if (real_pv(p->xi * p->rc) == 1)
        k_real_cl<T, KERNEL, TPW, 1, false, 1><<<nblk, 256, 0, st>>>(g, rk, nullptr, nullptr, xs, fs, qs, p->b.cnt_r,
                                                                     p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                                                                     u, p->b.status, 1, 0, 1);
    else
        k_real_cl<T, KERNEL, TPW, 1, false, 0><<<nblk, 256, 0, st>>>(g, rk, nullptr, nullptr, xs, fs, qs, p->b.cnt_r,
                                                                     p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                                                                     u, p->b.status, 1, 0, 1);
    p->launches += 3 + scan_launch_count(nrows);
    return cudaGetLastError();
}

// Batched real-space sum: cluster lists of all systems, then one pass of the
// clustered kernel per group of up to NRMAX right-hand sides (8 in FP32, 2 in
// FP64, so that the staged candidates fit in the 48 KB of static shared memory).

template <typename T, int KERNEL>
cudaError_t launch_breal_k(const BSys<T> *sys, const int *row_base, int S, int nrows_tot, int Ntot, int n_rhs,
                           const Buffers &b, int *cl_sys, T *u, cudaStream_t st, int64_t *launches) {
    constexpr int TPW = SE_RS_TPW;
    const unsigned rb = (unsigned)((nrows_tot + 255) / 256);
    k_bcluster_count<T><<<rb, 256, 0, st>>>(nrows_tot, sys, row_base, S, TPW, b.cnt_r, b.ncl);
    cudaError_t e = launch_scan(b.ncl, nrows_tot, st);
    if (e) return e;
    k_bcluster_fill<T><<<rb, 256, 0, st>>>(nrows_tot, sys, row_base, S, TPW, b.cnt_r, b.ncl, b.clusters, cl_sys);
    *launches += 2 + scan_launch_count(nrows_tot);
    const long max_cl = Ntot / TPW + nrows_tot + 1;
    const unsigned nblk = (unsigned)((max_cl + 7) / 8);
    constexpr int NRMAX = sizeof(T) == 4 ? 8 : 2;
    for (int q0 = 0; q0 < n_rhs; q0 += NRMAX) {
        const int nq = std::min(NRMAX, n_rhs - q0);
        // the general erfcx fit: systems of a batch may have any xi rc
        k_real_cl<T, KERNEL, TPW, NRMAX, true, 0><<<nblk, 256, 0, st>>>(
            GP<T>{}, RC<T>{}, sys, cl_sys, (const vec4<T> *)b.xs_r, (const vec4<T> *)b.fs_r, nullptr, b.cnt_r,
            b.clusters, b.ncl + nrows_tot, b.perm_r, u, b.status, n_rhs, q0, nq);
        *launches += 1;
    }
    return cudaGetLastError();
}

}  // namespace

// The table's coefficients, computed once on the host in FP64 from the C
// library's erfc and exp, and whether each device holds them.
static int g_erft_ready[64];

static void erfc_table_host(std::vector<double> &tab) {
    tab.assign(2 * ERFT_N * (ERFT_D + 1), 0.0);
    constexpr int K = ERFT_D + 1;
    // powers of t in T_0 .. T_D (T_{k+1} = 2 t T_k - T_{k-1})
    double tp[K][K] = {};
    tp[0][0] = 1.0;
    if (K > 1) tp[1][1] = 1.0;
    for (int k = 1; k + 1 < K; k++)
        for (int m = 0; m < K; m++) tp[k + 1][m] = (m > 0 ? 2.0 * tp[k][m - 1] : 0.0) - tp[k - 1][m];
    const double h = ERFT_XMAX / ERFT_N;
    for (int i = 0; i < ERFT_N; i++) {
        double fv[2][K], tj[K];
        for (int j = 0; j < K; j++) {
            tj[j] = cos(M_PI * (j + 0.5) / K);
            const double x = i * h + 0.5 * (tj[j] + 1.0) * h;
            fv[0][j] = erfc(x);
            fv[1][j] = 2.0 / sqrt(M_PI) * x * exp(-x * x);
        }
        for (int f = 0; f < 2; f++) {
            double cheb[K];
            for (int k = 0; k < K; k++) {
                double sum = 0.0;
                for (int j = 0; j < K; j++) sum += fv[f][j] * cos(M_PI * k * (j + 0.5) / K);
                cheb[k] = (k == 0 ? 1.0 : 2.0) * sum / K;
            }
            for (int m = 0; m < K; m++) {
                double a = 0.0;
                for (int k = 0; k < K; k++) a += cheb[k] * tp[k][m];
                tab[2 * (i * K + m) + f] = a;
            }
        }
    }
}

static int erfc_table_ready() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    return g_erft_ready[dev];
}

// Copied at every FP64 plan or batch creation (32 KB), so that a context
// reset (cudaDeviceReset) followed by new plans finds the table again.
cudaError_t erfc_table_init() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= 64) return cudaSuccess;
    static std::vector<double> tab;
    if (tab.empty()) erfc_table_host(tab);
    if ((e = cudaMemcpyToSymbol(g_erft, tab.data(), tab.size() * sizeof(double)))) return e;
    g_erft_ready[dev] = 1;
    return cudaSuccess;
}

template <typename T>
RC<T> make_rc(const se_plan_s *p) {
    RC<T> rk;
    rk.xi = (T)p->xi;
    rk.xi2 = (T)(p->xi * p->xi);
    rk.c = (T)(2.0 * p->xi / sqrt(M_PI));
    rk.c3 = (T)(4.0 * p->xi * p->xi * p->xi / sqrt(M_PI));
    rk.rc2 = (T)(p->rc * p->rc);
    rk.ce = (T)(-p->xi * p->xi / log(2.0));  // exp(-xi^2 r^2) = 2^(ce r^2)
    // rows farther than the last cell of a side hold nothing: cap the reach
    rk.reach[0] = std::min((int)ceil(p->rc * p->geom.icw[1] - 1e-9), p->geom.ncel[1] - 1);
    rk.reach[1] = std::min((int)ceil(p->rc * p->geom.icw[2] - 1e-9), p->geom.ncel[2] - 1);
    rk.tab = (sizeof(T) == 8 && !p->erfc_table_off) ? erfc_table_ready() : 0;
    return rk;
}

// The row lists of the real-space kernels hold at most MAXROWS rows of cells.
template <typename T>
static bool reach_ok(const RC<T> &rk) {
    return (2 * rk.reach[0] + 1) * (2 * rk.reach[1] + 1) <= MAXROWS;
}

template RC<float> make_rc<float>(const se_plan_s *);
template RC<double> make_rc<double>(const se_plan_s *);

template <typename T>
cudaError_t launch_breal(int kernel, const BSys<T> *sys, const int *row_base, int S, int nrows_tot, int Ntot,
                         int n_rhs, const Buffers &b, int *cl_sys, T *u, cudaStream_t st, int64_t *launches) {
    if (kernel == SE_STOKESLET)
        return launch_breal_k<T, SE_STOKESLET>(sys, row_base, S, nrows_tot, Ntot, n_rhs, b, cl_sys, u, st, launches);
    if (kernel == SE_ROTLET)
        return launch_breal_k<T, SE_ROTLET>(sys, row_base, S, nrows_tot, Ntot, n_rhs, b, cl_sys, u, st, launches);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_breal<float>(int, const BSys<float> *, const int *, int, int, int, int, const Buffers &,
                                         int *, float *, cudaStream_t, int64_t *);
template cudaError_t launch_breal<double>(int, const BSys<double> *, const int *, int, int, int, int,
                                          const Buffers &, int *, double *, cudaStream_t, int64_t *);

template <typename T>
cudaError_t launch_real(se_plan_s *p, cudaStream_t st, T *u, bool defer) {
    RC<T> rk = make_rc<T>(p);
    if (!reach_ok(rk)) return cudaErrorInvalidValue;
    if (defer && !real_can_defer(p)) return cudaErrorInvalidValue;
    if (p->kernel == SE_STOKESLET) return launch_real_k<T, SE_STOKESLET>(p, st, rk, u, defer);
    if (p->kernel == SE_STRESSLET) return launch_real_k<T, SE_STRESSLET>(p, st, rk, u, defer);
    return launch_real_k<T, SE_ROTLET>(p, st, rk, u, defer);
}

// The FP32 symmetric kernel can leave u alone (its sums in b.rt and b.uj).
bool real_can_defer(const se_plan_s *p) {
    return p->prec == SE_FP32 && !p->periodic && SE_RS_SYM && SE_RS_SYMC && p->b.uj && p->b.rt &&
           !p->deterministic;
}

template <typename T>
cudaError_t launch_add_uj(se_plan_s *p, cudaStream_t st, T *u) {
    const int N = (int)p->N;
    k_add_uj<T><<<(N + 255) / 256, 256, 0, st>>>(N, (const T *)p->b.uj, p->b.perm_r, u, (const T *)p->b.rt);
    p->launches++;
    return cudaGetLastError();
}

template cudaError_t launch_add_uj<float>(se_plan_s *, cudaStream_t, float *);
template cudaError_t launch_add_uj<double>(se_plan_s *, cudaStream_t, double *);

// Real-space sum at separate targets (binned into bt, Nt points): clusters of
// the targets' cell rows, candidates from the plan's sources; adds to ut.
template <typename T, int KERNEL>
cudaError_t launch_real_targets_k(se_plan_s *p, cudaStream_t st, Buffers &bt, int Nt, T *ut) {
    constexpr int TPW = SE_RS_TPW;
    const int nrows = p->geom.ncel[1] * p->geom.ncel[2];
    k_cluster_count<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, p->geom.ncel[0], TPW, bt.cnt_r, bt.ncl);
    cudaError_t e = launch_scan(bt.ncl, nrows, st);
    if (e) return e;
    k_cluster_fill<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, p->geom.ncel[0], TPW, bt.cnt_r, bt.ncl, bt.clusters);
    const long max_cl = Nt / TPW + nrows + 1;
    const unsigned nblk = (unsigned)((max_cl + 7) / 8);
    const RC<T> rk = make_rc<T>(p);
    const vec4<T> *xs = (const vec4<T> *)p->b.xs_r, *fs = (const vec4<T> *)p->b.fs_r,
                  *qs = (const vec4<T> *)p->b.qs_r, *xt = (const vec4<T> *)bt.xs_r;
    const GP<T> &g = gp<T>(p);
    if (real_pv(p->xi * p->rc) == 1)
        k_real_cl<T, KERNEL, TPW, 1, false, 1, true><<<nblk, 256, 0, st>>>(
            g, rk, nullptr, nullptr, xs, fs, qs, p->b.cnt_r, bt.clusters, bt.ncl + nrows, p->b.perm_r, ut, p->b.status,
            1, 0, 1, xt, bt.perm_r);
    else
        k_real_cl<T, KERNEL, TPW, 1, false, 0, true><<<nblk, 256, 0, st>>>(
            g, rk, nullptr, nullptr, xs, fs, qs, p->b.cnt_r, bt.clusters, bt.ncl + nrows, p->b.perm_r, ut, p->b.status,
            1, 0, 1, xt, bt.perm_r);
    p->launches += 3 + scan_launch_count(nrows);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_real_targets(se_plan_s *p, cudaStream_t st, Buffers &bt, int Nt, T *ut) {
    if (!reach_ok(make_rc<T>(p))) return cudaErrorInvalidValue;
    if (p->kernel == SE_STOKESLET) return launch_real_targets_k<T, SE_STOKESLET>(p, st, bt, Nt, ut);
    if (p->kernel == SE_STRESSLET) return launch_real_targets_k<T, SE_STRESSLET>(p, st, bt, Nt, ut);
    return launch_real_targets_k<T, SE_ROTLET>(p, st, bt, Nt, ut);
}

template cudaError_t launch_real_targets<float>(se_plan_s *, cudaStream_t, Buffers &, int, float *);
template cudaError_t launch_real_targets<double>(se_plan_s *, cudaStream_t, Buffers &, int, double *);

template <typename T>
cudaError_t launch_real_grad(se_plan_s *p, cudaStream_t st, const T *g_orig, T *gx) {
    int N = (int)p->N;
    RC<T> rk = make_rc<T>(p);
    if (!reach_ok(rk)) return cudaErrorInvalidValue;
    if (!p->gsort) return cudaErrorInvalidValue;
    vec4<T> *gsort = (vec4<T> *)p->gsort;
    k_sort_g<T><<<(N + 255) / 256, 256, 0, st>>>(N, p->b.perm_r, g_orig, gsort);
    p->launches++;
    if constexpr (sizeof(T) == 4) {
        if (SE_RS_SYMC && SE_GRAD_SYM && (p->kernel != SE_STRESSLET || SE_GRAD_SYM_STR) && !p->periodic &&
            p->b.uj) {
            // each pair once over the clusters of 8 targets, the candidate's share through uj
            const int nrows = p->geom.ncel[1] * p->geom.ncel[2];
            k_cluster_count<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, p->geom.ncel[0], 8, p->b.cnt_r, p->b.ncl);
            launch_scan(p->b.ncl, nrows, st);
            k_cluster_fill<<<(nrows + 255) / 256, 256, 0, st>>>(nrows, p->geom.ncel[0], 8, p->b.cnt_r, p->b.ncl,
                                                                 p->b.clusters);
            const long max_cl = N / 8 + nrows + 1;
            const unsigned nblk = (unsigned)((max_cl + 7) / 8);
            cudaError_t e = cudaMemsetAsync(p->b.uj, 0, 4 * sizeof(float) * (size_t)N, st);
            if (e) return e;
            const float4 *xf = (const float4 *)p->b.xs_r, *ff = (const float4 *)p->b.fs_r,
                         *gf4 = (const float4 *)gsort;
            float *ujf = (float *)p->b.uj;
            const bool pv1 = real_pv(p->xi * p->rc) == 1;
            if (p->kernel == SE_STRESSLET) {
                // the targets and candidates carry f (fs), q (qs) and g (gs)
                const float4 *qf4 = (const float4 *)p->b.qs_r;
                if (pv1)
                    k_real_symc<SE_STRESSLET, 1, false, true><<<nblk, 256, 0, st>>>(
                        p->gpf, rk, xf, ff, qf4, p->b.cnt_r, p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                        (float *)gx, ujf, p->b.status, nullptr, gf4);
                else
                    k_real_symc<SE_STRESSLET, 0, false, true><<<nblk, 256, 0, st>>>(
                        p->gpf, rk, xf, ff, qf4, p->b.cnt_r, p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                        (float *)gx, ujf, p->b.status, nullptr, gf4);
            } else if (p->kernel == SE_STOKESLET) {
                if (pv1)
                    k_real_symc<SE_STOKESLET, 1, false, true><<<nblk, 256, 0, st>>>(
                        p->gpf, rk, xf, ff, gf4, p->b.cnt_r, p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                        (float *)gx, ujf, p->b.status, nullptr);
                else
                    k_real_symc<SE_STOKESLET, 0, false, true><<<nblk, 256, 0, st>>>(
                        p->gpf, rk, xf, ff, gf4, p->b.cnt_r, p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                        (float *)gx, ujf, p->b.status, nullptr);
            } else {
                if (pv1)
                    k_real_symc<SE_ROTLET, 1, false, true><<<nblk, 256, 0, st>>>(
                        p->gpf, rk, xf, ff, gf4, p->b.cnt_r, p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                        (float *)gx, ujf, p->b.status, nullptr);
                else
                    k_real_symc<SE_ROTLET, 0, false, true><<<nblk, 256, 0, st>>>(
                        p->gpf, rk, xf, ff, gf4, p->b.cnt_r, p->b.clusters, p->b.ncl + nrows, p->b.perm_r,
                        (float *)gx, ujf, p->b.status, nullptr);
            }
            k_add_uj<float><<<(N + 255) / 256, 256, 0, st>>>(N, ujf, p->b.perm_r, (float *)gx);
            p->launches += 4 + scan_launch_count(nrows);
            return cudaGetLastError();
        }
    }
    unsigned gs = (N + 7) / 8;
    const vec4<T> *xs = (const vec4<T> *)p->b.xs_r, *fs = (const vec4<T> *)p->b.fs_r;
    const GP<T> &g = gp<T>(p);
    const vec4<T> *qs = (const vec4<T> *)p->b.qs_r;
    if (p->kernel == SE_STOKESLET)
        k_real_grad<T, SE_STOKESLET><<<gs, 256, 0, st>>>(g, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, gsort, gx);
    else if (p->kernel == SE_ROTLET)
        k_real_grad<T, SE_ROTLET><<<gs, 256, 0, st>>>(g, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, gsort, gx);
    else
        k_real_grad<T, SE_STRESSLET><<<gs, 256, 0, st>>>(g, rk, N, xs, fs, qs, p->b.cnt_r, p->b.perm_r, gsort,
                                                          gx);
    p->launches++;
    return cudaGetLastError();
}

template cudaError_t launch_real<float>(se_plan_s *, cudaStream_t, float *, bool);
template cudaError_t launch_real<double>(se_plan_s *, cudaStream_t, double *, bool);
template <typename T>
cudaError_t launch_real_adjT(se_plan_s *p, cudaStream_t st, const T *f_orig, const T *q_orig, T *gf, T *gq) {
    const int N = (int)p->N;
    const RC<T> rk = make_rc<T>(p);
    if (!reach_ok(rk)) return cudaErrorInvalidValue;
    k_real_cmp<T, SE_STRESSLET, true><<<(N + 7) / 8, 256, 0, st>>>(
        gp<T>(p), rk, N, (const vec4<T> *)p->b.xs_r, (const vec4<T> *)p->b.fs_r, nullptr, p->b.cnt_r,
        p->b.perm_r, gf, p->b.status, f_orig, q_orig, gq);
    p->launches++;
    return cudaGetLastError();
}

template cudaError_t launch_real_adjT<float>(se_plan_s *, cudaStream_t, const float *, const float *, float *,
                                             float *);
template cudaError_t launch_real_adjT<double>(se_plan_s *, cudaStream_t, const double *, const double *, double *,
                                              double *);
template cudaError_t launch_real_grad<float>(se_plan_s *, cudaStream_t, const float *, float *);
template cudaError_t launch_real_grad<double>(se_plan_s *, cudaStream_t, const double *, double *);

}  // namespace se
