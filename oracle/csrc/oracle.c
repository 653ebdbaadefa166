/*
 * Oracle (test infrastructure only): plain FP64 CPU loops for the free-space
 * Spectral Ewald method for Stokes potentials (af Klinteberg, Shamshirgar,
 * Tornberg, "Fast Ewald summation for free-space Stokes potentials").
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load this library.  It shares no code with the CUDA path.
 *
 * Every loop is the literal definition it cites: no blocking, no
 * factorisation of the Gaussians, no cell lists.  OpenMP parallelises loops
 * over independent targets only; spreading is serial (each point adds into a
 * shared grid).
 *
 * Kernel ids: 0 = stokeslet S, 1 = stresslet T (source f_l q_m), 2 = rotlet.
 * The rotlet is the definition Omega_jl = eps_jlm r_m / r^3 (Section 2,
 * eq. def_rotlet); the paper's operator form carries a factor 2 on top.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define K_STOKESLET 0
#define K_STRESSLET 1
#define K_ROTLET 2

static const double SQRT_PI = 1.77245385090551602729816748334;

static int eps3(int j, int l, int m) {
    /* Levi-Civita symbol */
    if (j == l || l == m || j == m) return 0;
    if ((j == 0 && l == 1 && m == 2) || (j == 1 && l == 2 && m == 0) ||
        (j == 2 && l == 0 && m == 1))
        return 1;
    return -1;
}

/* ------------------------------------------------------------------------
 * Free-space kernels, Section 2 eqs def_stokeslet, def_stresslet, def_rotlet.
 * G[j][l][m]: for S and Omega only m = 0 is used (G[j][l][0]).
 * ---------------------------------------------------------------------- */
static void kernel_full(int kernel, const double r[3], double G[3][3][3]) {
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rn = sqrt(r2);
    for (int j = 0; j < 3; j++)
        for (int l = 0; l < 3; l++)
            for (int m = 0; m < 3; m++) G[j][l][m] = 0.0;
    if (kernel == K_STOKESLET) {
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++)
                G[j][l][0] = (j == l ? 1.0 / rn : 0.0) + r[j] * r[l] / (r2 * rn);
    } else if (kernel == K_STRESSLET) {
        double r5 = r2 * r2 * rn;
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++)
                for (int m = 0; m < 3; m++) G[j][l][m] = -6.0 * r[j] * r[l] * r[m] / r5;
    } else {
        double r3 = r2 * rn;
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++)
                for (int m = 0; m < 3; m++) G[j][l][0] += eps3(j, l, m) * r[m] / r3;
    }
}

/* Gradient dG[a][j][l][m] = d/dr_a G_jlm(r) of the kernels above. */
static void kernel_full_grad(int kernel, const double r[3], double dG[3][3][3][3]) {
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rn = sqrt(r2);
    double r3 = r2 * rn, r5 = r3 * r2, r7 = r5 * r2;
    for (int a = 0; a < 3; a++)
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++)
                for (int m = 0; m < 3; m++) {
                    double v = 0.0;
                    if (kernel == K_STOKESLET) {
                        if (m != 0) { dG[a][j][l][m] = 0.0; continue; }
                        v = -(j == l ? r[a] / r3 : 0.0) +
                            ((a == j ? r[l] : 0.0) + (a == l ? r[j] : 0.0)) / r3 -
                            3.0 * r[j] * r[l] * r[a] / r5;
                    } else if (kernel == K_STRESSLET) {
                        v = -6.0 * (((a == j) ? r[l] * r[m] : 0.0) +
                                    ((a == l) ? r[j] * r[m] : 0.0) +
                                    ((a == m) ? r[j] * r[l] : 0.0)) / r5 +
                            30.0 * r[j] * r[l] * r[m] * r[a] / r7;
                    } else {
                        if (m != 0) { dG[a][j][l][m] = 0.0; continue; }
                        v = eps3(j, l, a) / r3;
                        for (int mm = 0; mm < 3; mm++) v -= 3.0 * eps3(j, l, mm) * r[mm] * r[a] / r5;
                    }
                    dG[a][j][l][m] = v;
                }
}

/* Real-space (screened) kernels, Section 3.2:
 *  S^R: eq. SR_Op.
 *  T^R: eq. TR_Op with the delta-term coefficient (4 xi^3 r / sqrt(pi)) e^{-xi^2 r^2};
 *       the third radial derivative of r - Phi^H (Table 1, Hasimoto row) gives
 *       this factor r, which the printed equation drops.
 *  Omega^R: eq. RR_Op divided by 2 (definition normalisation, see header). */
static void kernel_real(int kernel, const double r[3], double xi, double G[3][3][3]) {
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rn = sqrt(r2);
    double rh[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    double ec = erfc(xi * rn);
    double ex = exp(-xi * xi * r2);
    for (int j = 0; j < 3; j++)
        for (int l = 0; l < 3; l++)
            for (int m = 0; m < 3; m++) G[j][l][m] = 0.0;
    if (kernel == K_STOKESLET) {
        double c = 2.0 * (xi * ex / SQRT_PI + ec / (2.0 * rn));
        double s = 4.0 * xi / SQRT_PI * ex;
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++)
                G[j][l][0] = c * ((j == l ? 1.0 : 0.0) + rh[j] * rh[l]) - (j == l ? s : 0.0);
    } else if (kernel == K_STRESSLET) {
        double A1 = -2.0 / rn * (3.0 * ec / rn + 2.0 * xi / SQRT_PI * (3.0 + 2.0 * xi * xi * r2) * ex);
        double A2 = 4.0 * xi * xi * xi * rn / SQRT_PI * ex;
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++)
                for (int m = 0; m < 3; m++)
                    G[j][l][m] = A1 * rh[j] * rh[l] * rh[m] +
                                 A2 * ((j == l ? rh[m] : 0.0) + (l == m ? rh[j] : 0.0) +
                                       (m == j ? rh[l] : 0.0));
    } else {
        double c = ec / r2 + 2.0 * xi / SQRT_PI * ex / rn;
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++)
                for (int m = 0; m < 3; m++) G[j][l][0] += eps3(j, l, m) * rh[m] * c;
    }
}

/* Gradient of the real-space kernels for S and Omega (the stresslet gradient
 * is not provided).  Written from the radial forms
 *   S^R_jl = a(r) delta_jl + b(r) r_j r_l,   a = erfc/r - c e,  b = (erfc/r + c e)/r^2
 *   Omega^R_jl = eps_jlm r_m b(r)
 * with c = 2 xi / sqrt(pi), e = exp(-xi^2 r^2). */
static int kernel_real_grad(int kernel, const double r[3], double xi, double dG[3][3][3]) {
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rn = sqrt(r2);
    double ec = erfc(xi * rn);
    double ex = exp(-xi * xi * r2);
    double c = 2.0 * xi / SQRT_PI;
    double a = ec / rn - c * ex;
    double b = (ec / rn + c * ex) / r2;
    double da = -c * ex / rn - ec / r2 + 2.0 * c * xi * xi * rn * ex;
    double db = -3.0 * c * ex / (r2 * rn) - 3.0 * ec / (r2 * r2) - 2.0 * c * xi * xi * ex / rn;
    for (int q = 0; q < 3; q++)
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++) {
                double v;
                if (kernel == K_STOKESLET) {
                    v = da * r[q] / rn * (j == l ? 1.0 : 0.0) + db * r[q] / rn * r[j] * r[l] +
                        b * ((q == j ? r[l] : 0.0) + (q == l ? r[j] : 0.0));
                } else if (kernel == K_ROTLET) {
                    v = eps3(j, l, q) * b;
                    for (int m = 0; m < 3; m++) v += eps3(j, l, m) * r[m] * db * r[q] / rn;
                } else {
                    return -1;
                }
                dG[q][j][l] = v;
            }
    (void)a;
    return 0;
}

/* apply G to the source of point n: out_j = G_jl f_l (S, Omega) or G_jlm f_l q_m (T) */
static void apply(int kernel, double G[3][3][3], const double *f, const double *q, double out[3]) {
    for (int j = 0; j < 3; j++) {
        double s = 0.0;
        if (kernel == K_STRESSLET) {
            for (int l = 0; l < 3; l++)
                for (int m = 0; m < 3; m++) s += G[j][l][m] * f[l] * q[m];
        } else {
            for (int l = 0; l < 3; l++) s += G[j][l][0] * f[l];
        }
        out[j] = s;
    }
}

/* ------------------------------------------------------------------------
 * O1: direct sum, Section 1 eq. usumfree / Section 2 eq. usum.
 * Targets: if tidx != NULL the t-th target is source tidx[t] and the n == m
 * term is skipped; otherwise targets are the points xt[t] and nothing is
 * skipped.  Pairs at distance exactly zero are skipped and counted.
 * Returns the number of skipped coincident pairs.
 * ---------------------------------------------------------------------- */
int64_t o1_direct(int kernel, int64_t N, const double *x, const double *f, const double *q,
                  int64_t nt, const int64_t *tidx, const double *xt, double *u) {
    int64_t ncoinc = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : ncoinc)
    for (int64_t t = 0; t < nt; t++) {
        const double *xm = tidx ? x + 3 * tidx[t] : xt + 3 * t;
        int64_t self = tidx ? tidx[t] : -1;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t n = 0; n < N; n++) {
            if (n == self) continue;
            double r[3] = {xm[0] - x[3 * n], xm[1] - x[3 * n + 1], xm[2] - x[3 * n + 2]};
            if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) { ncoinc++; continue; }
            double G[3][3][3], v[3];
            kernel_full(kernel, r, G);
            apply(kernel, G, f + 3 * n, q ? q + 3 * n : 0, v);
            acc[0] += v[0]; acc[1] += v[1]; acc[2] += v[2];
        }
        u[3 * t] = acc[0]; u[3 * t + 1] = acc[1]; u[3 * t + 2] = acc[2];
    }
    return ncoinc;
}

/* Gradient of L = sum_m g_m . u_m (targets = all sources) with respect to the
 * positions: gx_p = sum_{n != p} [ g_p . dG(x_p - x_n) s_n  -  g_n . dG(x_n - x_p) s_p ]
 * where s = f (S, Omega) or f q^T (T) and dG is the gradient in the first
 * argument.  Only the targets tidx[t] are computed. */
void o1_grad_x(int kernel, int64_t N, const double *x, const double *f, const double *q,
               const double *g, int64_t nt, const int64_t *tidx, double *gx) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t p = tidx[t];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t n = 0; n < N; n++) {
            if (n == p) continue;
            double r[3] = {x[3 * p] - x[3 * n], x[3 * p + 1] - x[3 * n + 1], x[3 * p + 2] - x[3 * n + 2]};
            if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) continue;
            double mr[3] = {-r[0], -r[1], -r[2]};
            double dA[3][3][3][3], dB[3][3][3][3];
            kernel_full_grad(kernel, r, dA);
            kernel_full_grad(kernel, mr, dB);
            for (int a = 0; a < 3; a++) {
                double s = 0.0;
                for (int j = 0; j < 3; j++)
                    for (int l = 0; l < 3; l++) {
                        if (kernel == K_STRESSLET) {
                            for (int m = 0; m < 3; m++) {
                                s += g[3 * p + j] * dA[a][j][l][m] * f[3 * n + l] * q[3 * n + m];
                                s -= g[3 * n + j] * dB[a][j][l][m] * f[3 * p + l] * q[3 * p + m];
                            }
                        } else {
                            s += g[3 * p + j] * dA[a][j][l][0] * f[3 * n + l];
                            s -= g[3 * n + j] * dB[a][j][l][0] * f[3 * p + l];
                        }
                    }
                acc[a] += s;
            }
        }
        gx[3 * t] = acc[0]; gx[3 * t + 1] = acc[1]; gx[3 * t + 2] = acc[2];
    }
}

/* Gradient of L = sum_m g_m . u_m with respect to the strengths f (S, Omega):
 * gf_n = sum_{m != n} G(x_m - x_n)^T g_m. */
void o1_grad_f(int kernel, int64_t N, const double *x, const double *g, int64_t nt,
               const int64_t *tidx, double *gf) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t n = tidx[t];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t m = 0; m < N; m++) {
            if (m == n) continue;
            double r[3] = {x[3 * m] - x[3 * n], x[3 * m + 1] - x[3 * n + 1], x[3 * m + 2] - x[3 * n + 2]};
            if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) continue;
            double G[3][3][3];
            kernel_full(kernel, r, G);
            for (int l = 0; l < 3; l++)
                for (int j = 0; j < 3; j++) acc[l] += G[j][l][0] * g[3 * m + j];
        }
        gf[3 * t] = acc[0]; gf[3 * t + 1] = acc[1]; gf[3 * t + 2] = acc[2];
    }
}

/* Gradients of L = sum_m g_m . u_m with respect to the stresslet strengths f
 * and q (u_j(x_m) = sum_n T_jlk(x_m - x_n) f_nl q_nk):
 *   gf_nl = sum_{m != n} g_mj T_jlk(x_m - x_n) q_nk,
 *   gq_nk = sum_{m != n} g_mj T_jlk(x_m - x_n) f_nl. */
void o1_grad_fq(int64_t N, const double *x, const double *f, const double *q, const double *g, int64_t nt,
                const int64_t *tidx, double *gf, double *gq) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t n = tidx[t];
        double V[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  /* V_lk = sum_m g_mj T_jlk(x_m - x_n) */
        for (int64_t m = 0; m < N; m++) {
            if (m == n) continue;
            double r[3] = {x[3 * m] - x[3 * n], x[3 * m + 1] - x[3 * n + 1], x[3 * m + 2] - x[3 * n + 2]};
            if (r[0] == 0.0 && r[1] == 0.0 && r[2] == 0.0) continue;
            double G[3][3][3];
            kernel_full(K_STRESSLET, r, G);
            for (int l = 0; l < 3; l++)
                for (int k = 0; k < 3; k++)
                    for (int j = 0; j < 3; j++) V[l][k] += g[3 * m + j] * G[j][l][k];
        }
        for (int l = 0; l < 3; l++) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 3; k++) {
                a += V[l][k] * q[3 * n + k];
                b += V[k][l] * f[3 * n + k];
            }
            gf[3 * t + l] = a;
            gq[3 * t + l] = b;
        }
    }
}

/* Single-kernel evaluation helpers (vectorised over r) for tests. */
void o_kernel_full(int kernel, int64_t n, const double *r, double *G27) {
    for (int64_t i = 0; i < n; i++) {
        double G[3][3][3];
        kernel_full(kernel, r + 3 * i, G);
        for (int a = 0; a < 27; a++) G27[27 * i + a] = ((double *)G)[a];
    }
}
void o_kernel_real(int kernel, int64_t n, const double *r, double xi, double *G27) {
    for (int64_t i = 0; i < n; i++) {
        double G[3][3][3];
        kernel_real(kernel, r + 3 * i, xi, G);
        for (int a = 0; a < 27; a++) G27[27 * i + a] = ((double *)G)[a];
    }
}
int o_kernel_real_grad(int kernel, int64_t n, const double *r, double xi, double *dG27) {
    for (int64_t i = 0; i < n; i++) {
        double G[3][3][3];
        if (kernel_real_grad(kernel, r + 3 * i, xi, G)) return -1;
        for (int a = 0; a < 27; a++) dG27[27 * i + a] = ((double *)G)[a];
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * O2 real-space part, Section 6: sum over 0 < |x_m - x_n| <= rc of the
 * screened kernel, by checking the distance of every pair (no cell list).
 * ---------------------------------------------------------------------- */
int64_t o2_real(int kernel, int64_t N, const double *x, const double *f, const double *q,
                int64_t nt, const int64_t *tidx, const double *xt, double xi, double rc,
                double *u) {
    int64_t npairs = 0;
    double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : npairs)
    for (int64_t t = 0; t < nt; t++) {
        const double *xm = tidx ? x + 3 * tidx[t] : xt + 3 * t;
        int64_t self = tidx ? tidx[t] : -1;
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t n = 0; n < N; n++) {
            if (n == self) continue;
            double r[3] = {xm[0] - x[3 * n], xm[1] - x[3 * n + 1], xm[2] - x[3 * n + 2]};
            double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            if (r2 == 0.0 || r2 > rc2) continue;
            double G[3][3][3], v[3];
            kernel_real(kernel, r, xi, G);
            apply(kernel, G, f + 3 * n, q ? q + 3 * n : 0, v);
            acc[0] += v[0]; acc[1] += v[1]; acc[2] += v[2];
            npairs++;
        }
        u[3 * t] = acc[0]; u[3 * t + 1] = acc[1]; u[3 * t + 2] = acc[2];
    }
    return npairs;
}

/* Position gradient of the real-space part of L = sum g.u (S and Omega):
 * gx_p = sum_{0<|r|<=rc} [ g_p . dG^R(x_p - x_n) f_n - g_n . dG^R(x_n - x_p) f_p ]. */
int o2_real_grad_x(int kernel, int64_t N, const double *x, const double *f, const double *g,
                   int64_t nt, const int64_t *tidx, double xi, double rc, double *gx) {
    if (kernel == K_STRESSLET) return -1;
    double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t p = tidx[t];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t n = 0; n < N; n++) {
            if (n == p) continue;
            double r[3] = {x[3 * p] - x[3 * n], x[3 * p + 1] - x[3 * n + 1], x[3 * p + 2] - x[3 * n + 2]};
            double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            if (r2 == 0.0 || r2 > rc2) continue;
            double mr[3] = {-r[0], -r[1], -r[2]};
            double dA[3][3][3], dB[3][3][3];
            kernel_real_grad(kernel, r, xi, dA);
            kernel_real_grad(kernel, mr, xi, dB);
            for (int a = 0; a < 3; a++)
                for (int j = 0; j < 3; j++)
                    for (int l = 0; l < 3; l++)
                        acc[a] += g[3 * p + j] * dA[a][j][l] * f[3 * n + l] -
                                  g[3 * n + j] * dB[a][j][l] * f[3 * p + l];
        }
        gx[3 * t] = acc[0]; gx[3 * t + 1] = acc[1]; gx[3 * t + 2] = acc[2];
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * O2 grid steps, Section 5.2.  The grid covers the extended box with Mt^3
 * points y_i = y0 + i h, stored grid[c][iz][iy][ix] (x fastest).  Each point
 * touches the P^3 block of grid points starting at i0 in each dimension:
 *   P even: i0 = floor((x - y0)/h) - P/2 + 1   (P/2 points on each side)
 *   P odd : i0 = round((x - y0)/h) - (P-1)/2
 * The Gaussian is eq. Hx's  (2 xi^2/(pi eta))^{3/2} exp(-2 xi^2 |y - x|^2 / eta).
 * ---------------------------------------------------------------------- */
static int64_t window_start(double x, double y0, double h, int P) {
    double t = (x - y0) / h;
    if (P % 2 == 0) return (int64_t)floor(t) - P / 2 + 1;
    return (int64_t)floor(t + 0.5) - (P - 1) / 2;
}

/* Spreading (step 1, eq. Hx): grid[c][i] += src[n][c] * Gauss(y_i - x_n).
 * Returns -1 if some window leaves the grid (nothing is written past it). */
int o2_spread(int64_t N, const double *x, int nc, const double *src, int Mt, int P, double h,
              const double *y0, double xi, double eta, double *grid) {
    double pre = pow(2.0 * xi * xi / (M_PI * eta), 1.5);
    double a = 2.0 * xi * xi / eta;
    int64_t Mt3 = (int64_t)Mt * Mt * Mt;
    for (int64_t n = 0; n < N; n++) {
        int64_t i0[3];
        for (int d = 0; d < 3; d++) {
            i0[d] = window_start(x[3 * n + d], y0[d], h, P);
            if (i0[d] < 0 || i0[d] + P > Mt) return -1;
        }
        for (int kz = 0; kz < P; kz++)
            for (int ky = 0; ky < P; ky++)
                for (int kx = 0; kx < P; kx++) {
                    int64_t ix = i0[0] + kx, iy = i0[1] + ky, iz = i0[2] + kz;
                    double dx = y0[0] + ix * h - x[3 * n];
                    double dy = y0[1] + iy * h - x[3 * n + 1];
                    double dz = y0[2] + iz * h - x[3 * n + 2];
                    double w = pre * exp(-a * (dx * dx + dy * dy + dz * dz));
                    int64_t gi = (iz * Mt + iy) * Mt + ix;
                    for (int c = 0; c < nc; c++) grid[c * Mt3 + gi] += src[n * nc + c] * w;
                }
    }
    return 0;
}

/* Quadrature sum (step 5, eq. u_integr without the h^3 weight):
 * out[t][c] = sum_{i in window} grid[c][i] * Gauss(x_t - y_i). */
int o2_gather(int64_t nt, const double *xt, int nc, const double *grid, int Mt, int P, double h,
              const double *y0, double xi, double eta, double *out) {
    double pre = pow(2.0 * xi * xi / (M_PI * eta), 1.5);
    double a = 2.0 * xi * xi / eta;
    int64_t Mt3 = (int64_t)Mt * Mt * Mt;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i0[3];
        int ok = 1;
        for (int d = 0; d < 3; d++) {
            i0[d] = window_start(xt[3 * t + d], y0[d], h, P);
            if (i0[d] < 0 || i0[d] + P > Mt) ok = 0;
        }
        for (int c = 0; c < nc; c++) out[t * nc + c] = 0.0;
        if (!ok) { bad = 1; continue; }
        for (int kz = 0; kz < P; kz++)
            for (int ky = 0; ky < P; ky++)
                for (int kx = 0; kx < P; kx++) {
                    int64_t ix = i0[0] + kx, iy = i0[1] + ky, iz = i0[2] + kz;
                    double dx = xt[3 * t] - (y0[0] + ix * h);
                    double dy = xt[3 * t + 1] - (y0[1] + iy * h);
                    double dz = xt[3 * t + 2] - (y0[2] + iz * h);
                    double w = pre * exp(-a * (dx * dx + dy * dy + dz * dz));
                    int64_t gi = (iz * Mt + iy) * Mt + ix;
                    for (int c = 0; c < nc; c++) out[t * nc + c] += grid[c * Mt3 + gi] * w;
                }
    }
    return bad ? -1 : 0;
}

/* Gradient quadrature: out[t][a] = sum_i s_t(i) * d/dx_a Gauss(x_t - y_i) with
 * s_t(i) = sum_c coefA[t][c] gridA[c][i] + coefB[t][c] gridB[c][i]
 * (d/dx_a Gauss(r) = -(4 xi^2/eta) r_a Gauss(r)). */
int o2_gather_grad(int64_t nt, const double *xt, int nc, const double *coefA, const double *gridA,
                   const double *coefB, const double *gridB, int Mt, int P, double h,
                   const double *y0, double xi, double eta, double *out) {
    double pre = pow(2.0 * xi * xi / (M_PI * eta), 1.5);
    double a = 2.0 * xi * xi / eta;
    int64_t Mt3 = (int64_t)Mt * Mt * Mt;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i0[3];
        int ok = 1;
        for (int d = 0; d < 3; d++) {
            i0[d] = window_start(xt[3 * t + d], y0[d], h, P);
            if (i0[d] < 0 || i0[d] + P > Mt) ok = 0;
        }
        out[3 * t] = out[3 * t + 1] = out[3 * t + 2] = 0.0;
        if (!ok) { bad = 1; continue; }
        for (int kz = 0; kz < P; kz++)
            for (int ky = 0; ky < P; ky++)
                for (int kx = 0; kx < P; kx++) {
                    int64_t ix = i0[0] + kx, iy = i0[1] + ky, iz = i0[2] + kz;
                    double r[3] = {xt[3 * t] - (y0[0] + ix * h), xt[3 * t + 1] - (y0[1] + iy * h),
                                   xt[3 * t + 2] - (y0[2] + iz * h)};
                    double w = pre * exp(-a * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]));
                    int64_t gi = (iz * Mt + iy) * Mt + ix;
                    double s = 0.0;
                    for (int c = 0; c < nc; c++)
                        s += coefA[t * nc + c] * gridA[c * Mt3 + gi] + coefB[t * nc + c] * gridB[c * Mt3 + gi];
                    for (int d = 0; d < 3; d++) out[3 * t + d] += s * (-2.0 * a) * r[d] * w;
                }
    }
    return bad ? -1 : 0;
}

/* Transposed real-space sum (S and Omega): out_l(x_t) = sum_{0<|r|<=rc} G^R_jl(x_n - x_t) src_nj
 * over sources n != t, i.e. the real-space part of the transposed operator. */
void o2_real_T(int kernel, int64_t N, const double *x, const double *src, int64_t nt,
               const int64_t *tidx, double xi, double rc, double *out) {
    double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t p = tidx[t];
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t n = 0; n < N; n++) {
            if (n == p) continue;
            double r[3] = {x[3 * n] - x[3 * p], x[3 * n + 1] - x[3 * p + 1], x[3 * n + 2] - x[3 * p + 2]};
            double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            if (r2 == 0.0 || r2 > rc2) continue;
            double G[3][3][3];
            kernel_real(kernel, r, xi, G);
            for (int l = 0; l < 3; l++)
                for (int j = 0; j < 3; j++) acc[l] += G[j][l][0] * src[3 * n + j];
        }
        out[3 * t] = acc[0]; out[3 * t + 1] = acc[1]; out[3 * t + 2] = acc[2];
    }
}
