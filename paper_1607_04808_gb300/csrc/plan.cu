// Plan creation: parameter selection (Section 8.2 with the truncation-error
// estimates of Tables 2 and 3), grid sizing (Sections 4.2, 5.2, 5.3, 9),
// workspace allocation, cuFFT plans and the FP64 precomputation (Section 4.3).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <type_traits>
#include <vector>

#include "se_internal.cuh"

namespace se {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
se_status_t fail(se_status_t st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

// ---------------------------------------------------------------- parameter selection
namespace {

// Fourier truncation error, Table 2 (absolute RMS), Q = sum |f|^2.
double est_fourier(int kernel, double Q, double xi, double L, int M, int P) {
    double kinf = M_PI * M / L;
    double Lt = L * (M + P) / (double)M;  // Ltilde with delta_L = d
    double R = sqrt(3.0) * Lt;
    double ex = exp(-kinf * kinf / (4.0 * xi * xi));
    if (kernel == SE_STOKESLET) return sqrt(Q) * R * kinf * kinf * kinf / (xi * xi * M_PI * L) * ex;
    if (kernel == SE_STRESSLET)
        return sqrt(7.0 * Q / 6.0) * R * kinf * kinf * kinf * kinf / (xi * xi * M_PI * L) * ex;
    return sqrt(8.0 * xi * xi * Q / (3.0 * M_PI * L * L * L * kinf)) * ex;
}

// Real-space truncation error, Table 3 (absolute RMS).
double est_real(int kernel, double Q, double xi, double L, double rc) {
    double ex = exp(-xi * xi * rc * rc);
    double L3 = L * L * L;
    if (kernel == SE_STOKESLET) return sqrt(4.0 * Q * rc / L3) * ex;
    if (kernel == SE_STRESSLET) return sqrt(112.0 * Q * xi * xi * xi * xi * rc * rc * rc / (9.0 * L3)) * ex;
    return sqrt(8.0 * Q / (3.0 * L3 * rc)) * ex;
}

// Smallest M meeting the Fourier budget (the estimate decreases with M).
int min_M(int kernel, double Q, double xi, double L, int P, double budget) {
    for (int M = 2; M < 4096; M++)
        if (est_fourier(kernel, Q, xi, L, M, P) <= budget) return M;
    return 4096;
}

double min_rc(int kernel, double Q, double xi, double L, double budget) {
    double lo = 1e-6 * L, hi = 2.0 * L;
    if (est_real(kernel, Q, xi, L, hi) > budget) return hi;
    for (int it = 0; it < 100; it++) {
        double mid = 0.5 * (lo + hi);
        if (est_real(kernel, Q, xi, L, mid) <= budget) hi = mid; else lo = mid;
    }
    return hi;
}

// FFT lengths cuFFT handles fast and accurately: only prime factors 2, 3, 5, 7.
// In FP32 the powers of two from 32 on are excluded: cuFFT's single-precision
// real-to-complex and complex-to-real transforms at 128^3 and 256^3 left the
// Fourier part an order of magnitude less accurate (2.8e-6 and 5.2e-6
// relative, N = 46030 and 1e6 uniform points at 2e-6) than the neighbouring
// lengths 96 to 200 and 252 (3e-7 to 9e-7); the complex-to-complex transforms
// of the same lengths were accurate, and so were 96 and 192.
bool pow2_fp32_bad(int n, int prec) { return prec == SE_FP32 && n >= 32 && (n & (n - 1)) == 0; }

bool good_fft(int n, int prec) {
    if (n < 2) return false;
    if (pow2_fp32_bad(n, prec)) return false;
    int m = n;
    for (int f : {2, 3, 5, 7})
        while (m % f == 0) m /= f;
    return m == 1;
}

// Work model of an evaluation, relative to one ordered real-space pair: the
// pairs within rc (times the points' neighbour factor), the spreading and
// gather updates (N P^3, twice) and the FFT work (Mf^3 log2 Mf, six
// transforms, the scaling folded in).  FP64 weights measured on GB300 at N =
// 1e6 (200 ps per pair, 7.2 ps per update, 21 ps per FFT unit).  FP32 keeps
// weights that favour smaller xi: a larger xi moves more of the sum into the
// FP32 Fourier part, whose rounding error grows with it.  Several right-hand
// sides: the grid and FFT work repeats per side, a pair's radial functions
// are shared (batches evaluate full candidate lists: 1.5 x a pair, +1/3 per
// extra side).
}  // namespace

#ifndef SE_MODEL_CGRID32
#define SE_MODEL_CGRID32 0.12
#endif
#ifndef SE_MODEL_CFFT32
#define SE_MODEL_CFFT32 0.6
#endif
double model_cost(int prec, int64_t N, double L, int P, int M, double rc, const PairFactor *pf, int n_rhs) {
    const double cpair = 1.0, cgrid = (prec == SE_FP32) ? SE_MODEL_CGRID32 : 0.036,
                 cfft = (prec == SE_FP32) ? SE_MODEL_CFFT32 : 0.11;
    const double Mf = 2.0 * (M + P);
    double pairs = (double)N * (double)N * 4.18879 * rc * rc * rc / (L * L * L);
    if (pf) pairs *= pf->at(rc);
    const double wpair = (n_rhs > 1) ? 1.5 * (1.0 + (n_rhs - 1) / 3.0) : 1.0;
    return cpair * wpair * pairs +
           n_rhs * (cgrid * (double)N * P * P * P * 2.0 + cfft * Mf * Mf * Mf * log2(Mf) * 6.0);
}

// FFT lengths measured fast with cuFFT on GB300: 2^a 3^b, times at most one 5,
// and a multiple of 4 (350, 400, 420 and 448 took 1.2 to 1.5 times the time
// per point of 320, 360, 384 and 432).
bool fast_fft_len(int n, int prec) {
    if (n < 8 || (n & 3)) return false;
    if (pow2_fp32_bad(n, prec)) return false;
    int m = n, fives = 0;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    while (m % 5 == 0) m /= 5, fives++;
    return m == 1 && fives <= 1;
}

// Parameter selection.  Relative tolerances are turned into absolute RMS
// budgets with the RMS of u for uniformly distributed points and unit-variance
// sources, |u|_rms^2 ~ 6 <1/r^2> N ~ 33.6 N / L^2 (stokeslet; the same scale is
// used, conservatively, for the stresslet and rotlet whose RMS is larger).  P is
// the smallest even support whose approximation error 10^{-(P+1)/2} stays below
// tol/4 (Section 8.2: P = 16 ~ 8 digits, 24 ~ 12 digits).  With a bound on the
// FFT size, xi is the largest value whose Fourier estimate at the largest
// admissible M meets the budget; otherwise xi minimises a work model.
double PairFactor::at(double r) const {
    if (n <= 0 || !f) return 1.0;
    const double u = r / dr - 1.0;  // f[i] at r = (i + 1) dr
    if (u <= 0.0) return f[0];
    if (u >= n - 1) return f[n - 1];
    const int i = (int)u;
    return f[i] + (u - i) * (f[i + 1] - f[i]);
}

se_status_t choose_params(int kernel, int prec, int64_t N, double L, double tol, const se_params_t *in,
                          double xi_arg, se_params_t *out, int n_rhs, const PairFactor *pf) {
    se_params_t p;
    memset(&p, 0, sizeof(p));
    if (in) p = *in;
    if (tol <= 0) tol = (prec == SE_FP32) ? 2e-6 : 1e-10;
    double Q = 3.0 * (double)N;
    double deg = (kernel == SE_STOKESLET) ? 1.0 : 2.0;
    double uabs = sqrt(33.6 * (double)N) / pow(L, deg);
    double budget = 0.5 * tol * uabs;  // each of the three error sources within tol/2
    if (p.P <= 0) {
        // the stresslet's window error is larger (its multiplier grows one power
        // of k faster than the stokeslet's; measured at N = 4e4 and 1e5, P = 12
        // leaves 2.6e-6 and 4.8e-6 where P = 14 leaves 4e-8 and 7e-8): a
        // quarter of the stokeslet's budget
        const double ptol = (kernel == SE_STRESSLET) ? tol / 16.0 : tol / 4.0;
        int P = 4;
        while (P < 32 && pow(10.0, -0.5 * P - 0.5) > ptol) P += 2;
        p.P = P;
    }
    double xi = (p.xi > 0) ? p.xi : xi_arg;
    if (!(xi > 0)) {
        if (p.max_fft > 0 && p.M <= 0) {
            int Mmax = p.max_fft / 2 - p.P;
            if (Mmax < 2) return fail(SE_ERR_INVALID_ARG, "max_fft too small for the support P");
            double lo = 0.1 / L, hi = 10.0 * Mmax / L;
            for (int it = 0; it < 100; it++) {
                double mid = 0.5 * (lo + hi);
                if (est_fourier(kernel, Q, mid, L, Mmax, p.P) <= budget) lo = mid; else hi = mid;
            }
            xi = lo;
        } else if (p.M > 0) {
            double lo = 0.1 / L, hi = 10.0 * p.M / L;
            for (int it = 0; it < 100; it++) {
                double mid = 0.5 * (lo + hi);
                if (est_fourier(kernel, Q, mid, L, p.M, p.P) <= budget) lo = mid; else hi = mid;
            }
            xi = lo;
        } else {
            // the xi of least modelled work (model_cost)
            double best = 1e300, bxi = 1.0 / L;
            for (double x = 0.5 / L; x < 4000.0 / L; x *= 1.03) {
                int M = min_M(kernel, Q, x, L, p.P, budget);
                double rc = min_rc(kernel, Q, x, L, budget);
                if (rc > L) continue;
                const double cost = model_cost(prec, N, L, p.P, M, rc, pf, n_rhs);
                if (cost < best) { best = cost; bxi = x; }
            }
            xi = bxi;
        }
    }
    p.xi = xi;
    const bool fixed_M = (in && in->M > 0);
    if (p.M <= 0) p.M = min_M(kernel, Q, xi, L, p.P, budget);
    if (!fixed_M && p.deltaL_policy == 0) {
        // FFT length 2 (M + P): move M to a fast, accurate length (up, or down
        // under a cap), then re-derive xi for that M when xi was chosen here
        int M = p.M;
        if (p.max_fft > 0 && 2 * (M + p.P) > p.max_fft) M = p.max_fft / 2 - p.P;
        if (p.max_fft > 0) {
            while (M > 2 && !good_fft(2 * (M + p.P), prec)) M--;
        } else {
            while (!good_fft(2 * (M + p.P), prec)) M++;
        }
        p.M = M;
        if (!(in && in->xi > 0) && !(xi_arg > 0)) {
            double lo = 0.1 / L, hi = 10.0 * p.M / L;
            for (int it = 0; it < 100; it++) {
                double mid = 0.5 * (lo + hi);
                if (est_fourier(kernel, Q, mid, L, p.M, p.P) <= budget) lo = mid; else hi = mid;
            }
            p.xi = lo;
        }
    } else if (p.max_fft > 0 && 2 * (p.M + p.P) > p.max_fft) {
        p.M = p.max_fft / 2 - p.P;
    }
    if (p.rc <= 0) p.rc = min_rc(kernel, Q, p.xi, L, budget);
    *out = p;
    return SE_OK;
}

}  // namespace se

using namespace se;

void free_plan(se_plan_s *p) {
    if (!p) return;
    if (p->have_fwd) cufftDestroy(p->fwd);
    if (p->have_inv) cufftDestroy(p->inv);
    if (p->have_fwd3) cufftDestroy(p->fwd3);
    if (p->f2d) cufftDestroy(p->f2d);
    if (p->i2d) cufftDestroy(p->i2d);
    if (p->zc) cufftDestroy(p->zc);
    void *ptrs[] = {p->b.uj, p->b.ncl, p->b.clusters, p->ghat64, (p->ghat != p->ghat64) ? p->ghat : nullptr, p->grid, p->spec, p->wgrid, p->wgrid2,
                    p->spec2, p->tmp3, p->b.xs_t, p->b.fs_t, p->b.qs_t, p->b.perm_t, p->b.cnt_t, p->b.slot_t,
                    p->b.key_t, p->b.xs_r, p->b.fs_r, p->b.qs_r, p->b.perm_r, p->b.cnt_r, p->b.slot_r,
                    p->b.key_r, p->b.tag_t, p->b.tag_r, p->b.status, p->dx, p->df, p->dq, p->du, p->pgrid, p->b.rt,
                    p->gsort, p->zw, p->tilebuf, p->rs_scratch};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    void *tptrs[] = {p->bt.xs_t, p->bt.perm_t, p->bt.slot_t, p->bt.key_t, p->bt.tag_t, p->bt.cnt_t, p->bt.xs_r,
                     p->bt.perm_r, p->bt.slot_r, p->bt.key_r, p->bt.tag_r, p->bt.cnt_r, p->bt.ncl, p->bt.clusters};
    for (void *q : tptrs)
        if (q) cudaFree(q);
    for (int i = 0; i < 9; i++)
        if (p->ev[i]) cudaEventDestroy(p->ev[i]);
    if (p->ev_real) cudaEventDestroy(p->ev_real);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->s_four) cudaStreamDestroy(p->s_four);
    delete p;
}

template <typename P_>
static cudaError_t dmalloc(P_ **ptr, size_t bytes) {
    return cudaMalloc((void **)ptr, bytes ? bytes : 16);
}

// Parameters, grid sizes and geometry of a plan (no device work).
se_status_t se::setup_plan(se_plan_s *p, int kernel, int prec, int64_t N, const double box[6],
                           const se_params_t &pr, bool periodic) {
    p->kernel = kernel;
    p->prec = prec;
    p->N = N;
    double lmax = 0;
    for (int d = 0; d < 3; d++) {
        p->x0[d] = box[d];
        p->len[d] = box[3 + d];
        lmax = std::max(lmax, p->len[d]);
    }
    p->xi = pr.xi;
    p->rc = pr.rc;
    p->P = pr.P;
    p->deltaL_policy = pr.deltaL_policy;
    p->max_fft = pr.max_fft;
    p->cell_width = pr.cell_width;
    // Sections 5.2-5.3: h = L/M (M points along the longest side), d = hP,
    // m = C sqrt(pi P), eta = (xi d / m)^2
    p->h = lmax / pr.M;
    double d = p->h * p->P;
    p->m = 0.976 * sqrt(M_PI * p->P);
    p->eta = (p->xi * d / p->m) * (p->xi * d / p->m);
    double need = d;
    if (p->deltaL_policy == 1 && p->eta < 1.0)
        need = std::max(d, sqrt(2.0 * (1.0 - p->eta) * p->m * p->m / (p->xi * p->xi)));
    p->n_ext = (int)ceil(need / p->h - 1e-9);
    p->periodic = periodic;
    if (periodic) {
        // a halo of P points (rounded up to even, so that the extended grid
        // points fall on the periodic ones) holds every point's support; the
        // fold wraps it once, so it may not exceed the grid
        p->n_ext = p->P + (p->P & 1);
        p->mp = pr.M;
        if (p->n_ext > 2 * p->mp) return fail(SE_ERR_INVALID_ARG, "periodic plan: P above 2 M");
    }
    p->deltaL = p->n_ext * p->h;
    double r2 = 0;
    for (int dd = 0; dd < 3; dd++) {
        // the shorter sides: the smallest M covering the side whose FFT length
        // 2 (M + n_ext) has prime factors 2, 3, 5, 7 (the grid may extend past
        // the box; the points only need to lie inside it)
        int M = (p->len[dd] == lmax) ? pr.M : (int)ceil(p->len[dd] / p->h - 1e-9);
        if (p->len[dd] != lmax)
            while (!good_fft(2 * (M + p->n_ext), prec)) M++;
        if (periodic) M = pr.M;
        p->mm[dd] = M;
        p->mt[dd] = M + p->n_ext;
        // the periodic plan's spreading grid is the extended grid itself
        p->mf[dd] = periodic ? p->mt[dd] : 2 * p->mt[dd];
        r2 += (p->mt[dd] * p->h) * (p->mt[dd] * p->h);
    }
    // truncation radius: the diagonal of the extended box (Section 4.1;
    // sqrt(3) Ltilde for a cube)
    p->R = sqrt(r2);
    // precompute grid per dimension: the smallest even size above
    // (1 + R / Ltilde_d) mt_d, the oversampling of Section 4.2 ((1 + sqrt 3) mt
    // for a cube, Section 9), rounded up to a length with prime factors 2, 3, 5,
    // 7 (a larger oversampling factor is still valid and avoids cuFFT's slow path)
    for (int dd = 0; dd < 3 && !periodic; dd++) {
        const double sf = 1.0 + p->R / (p->mt[dd] * p->h);
        int Mg = 2 * (int)floor(sf * p->mt[dd] / 2.0) + 2;
        while (!good_fft(Mg, SE_FP64) || (Mg & 1)) Mg++;
        p->mg[dd] = Mg;
    }
    if (periodic) p->R = 0;
    p->nc = (kernel == SE_STRESSLET) ? 6 : 3;
    for (int dd = 0; dd < 3; dd++) {
        if (p->max_fft > 0 && (periodic ? p->mp : p->mf[dd]) > p->max_fft)
            return fail(SE_ERR_INVALID_ARG, "FFT size exceeds max_fft");
        if (p->mt[dd] > 1023) return fail(SE_ERR_INVALID_ARG, "extended grid above 1023 points per dimension");
    }
    // geometry
    Geom &g = p->geom;
    for (int dd = 0; dd < 3; dd++) {
        g.x0[dd] = p->x0[dd];
        g.len[dd] = p->len[dd];
        g.mt[dd] = p->mt[dd];
        g.mf[dd] = p->mf[dd];
    }
    g.h = p->h;
    g.inv_h = 1.0 / p->h;
    g.half_ext = 0.5 * p->n_ext;
    g.P = p->P;
    g.a = 2.0 * p->xi * p->xi / p->eta;
    g.xi = p->xi;
    g.rc = p->rc;
    size_t esz = (prec == SE_FP32) ? 4 : 8;
    // spreading tiles: the largest edge whose padded tile (all components) fits
    // in 110 KB of shared memory; otherwise the atomic spreading path is used and
    // tiles of 8 only order the points
    int T = 0;
    for (int cand : {8, 6, 4, 2}) {
        size_t PT = cand + p->P - 1;
        if ((size_t)p->nc * PT * PT * PT * esz <= 110 * 1024) { T = cand; break; }
    }
    p->tiled = (T > 0);
    g.T = (T > 0) ? T : 8;
#ifndef SE_USE_COL
#define SE_USE_COL 1
#endif
    if (SE_USE_COL && col_supported(prec, p->P)) {
        // register-column kernels: their own tile edge, no shared-memory limit
        p->colk = true;
        p->tiled = true;
        g.T = COL_TE;
    }
    p->ntiles = 1;
    for (int dd = 0; dd < 3; dd++) {
        g.nt[dd] = (p->mt[dd] - p->P + 1 + g.T - 1) / g.T;
        p->ntiles *= g.nt[dd];
    }
    // real-space cells: width >= rc/5 (FP32) or rc/3 (FP64) across rows (y, z;
    // at most 200) and >= rc/16 along the rows (x; at most 1000), so that
    // trimming each row to the cutoff sphere wastes little
#ifndef SE_RS_YZDIV32
#define SE_RS_YZDIV32 5.0
#endif
#ifndef SE_RS_XDIV
#define SE_RS_XDIV 16.0
#endif
#ifndef SE_RS_YZDIV64
#define SE_RS_YZDIV64 3.0
#endif
#ifndef SE_RS_YZ_ADAPT
#define SE_RS_YZ_ADAPT 1
#endif
    double yzdiv = (prec == SE_FP32) ? SE_RS_YZDIV32 : SE_RS_YZDIV64;
    if (SE_RS_YZ_ADAPT && prec == SE_FP32 && N > 0) {
        // FP32 clusters of 8 consecutive points of a row: with a cutoff below
        // 3.4 times w = 1.1 (8/density)^(1/3), cells of width w across, so that
        // a cluster spans about as much along the row as across it (its
        // bounding box, which filters the candidates, then adds least volume
        // around the cutoff sphere); at least rc/1.5.  Measured at N = 1e6
        // uniform, rc = 2.8 w: real-space sum 2.63 -> 2.26 ms (rotlet, N = 2e5,
        // rc = 2.8 w: 0.52 -> 0.43 ms); above that the rc/5 cells measured as
        // fast or faster (N = 1e6 at rc = 4.2 w, clustered points, whose mean
        // density understates the density around most pairs)
        const double vol = p->len[0] * p->len[1] * p->len[2];
        const double w = 1.1 * cbrt(8.0 * vol / (double)N);
        if (p->rc < 3.4 * w) yzdiv = std::max(1.5, p->rc / w);
        if (p->cell_width > 0) yzdiv = std::min(SE_RS_YZDIV32, std::max(1.5, p->rc / p->cell_width));
    }
    for (int dd = 1; dd < 3; dd++) g.ncel[dd] = std::max(1, std::min((int)floor(yzdiv * p->len[dd] / p->rc), 200));
    g.ncel[0] = std::max(1, std::min((int)floor(SE_RS_XDIV * p->len[0] / p->rc), 1000));
    const long rows = (long)g.ncel[1] * g.ncel[2];
    if (rows * g.ncel[0] > (1L << 26)) g.ncel[0] = (int)std::max(1L, (1L << 26) / rows);
    for (int dd = 0; dd < 3; dd++) {
        g.cw[dd] = p->len[dd] / g.ncel[dd];
        g.icw[dd] = g.ncel[dd] / p->len[dd];
    }
    p->ncells = g.ncel[0] * g.ncel[1] * g.ncel[2];
    // the same geometry in each arithmetic precision
    auto fill = [&](auto &G) {
        using TT = std::remove_reference_t<decltype(G.inv_h)>;
        for (int dd = 0; dd < 3; dd++) {
            G.x0[dd] = (TT)p->x0[dd];
            G.len[dd] = (TT)p->len[dd];
            G.icw[dd] = (TT)g.icw[dd];
            G.ilen[dd] = (TT)(1.0 / p->len[dd]);
            G.cw[dd] = (TT)g.cw[dd];
            G.mt[dd] = g.mt[dd];
            G.mf[dd] = g.mf[dd];
            G.nt[dd] = g.nt[dd];
            G.ncel[dd] = g.ncel[dd];
        }
        G.inv_h = (TT)(1.0 / p->h);
        G.half_ext = (TT)(0.5 * p->n_ext);
        G.ah2 = (TT)(g.a * p->h * p->h);
        G.P = p->P;
        G.T_ = g.T;
    };
    fill(p->gpf);
    fill(p->gpd);
    return SE_OK;
}

// Parameters for a box with sides (Lx, Ly, Lz): the selection for the cube of
// the longest side at the same point density (the error estimates depend on
// the density, xi and h), so M counts grid intervals along the longest side.
se_status_t se::choose_box_params(int kernel, int prec, int64_t N, const double box[6], double tol,
                                  const se_params_t *params, double xi, se_params_t *out, int n_rhs,
                                  const PairFactor *pf) {
    const double lmax = std::max(box[3], std::max(box[4], box[5]));
    const double vol = box[3] * box[4] * box[5];
    const double neff = std::max(1.0, (double)N * lmax * lmax * lmax / vol);
    return choose_params(kernel, prec, (int64_t)llround(neff), lmax, tol, params, xi, out, n_rhs, pf);
}

// Probability that two independent uniform points of the box a x b x c lie
// within r of each other (r <= the shortest side): the volume of the
// difference set's ball, [4 pi r^3 abc / 3 - pi r^4 (ab + bc + ca) / 2 +
// 8 r^5 (a + b + c) / 15 - r^6 / 6] / (abc)^2.
static double pair_prob_box(double r, double a, double b, double c) {
    const double V = a * b * c, r3 = r * r * r;
    return (4.18879020478639 * r3 * V - 1.5707963267948966 * r3 * r * (a * b + b * c + c * a) +
            8.0 / 15.0 * r3 * r * r * (a + b + c) - r3 * r3 / 6.0) /
           (V * V);
}

// Neighbour counts within r_i = (i + 1) r_max / NR of up to 4096 sampled points
// (every (N / S)-th), from a cell list of side >= r_max, over the counts that
// uniform points would give.
static std::vector<double> pair_factor_table(const double *x, int64_t N, const double box[6], double r_max,
                                             int NR) {
    int nc[3];
    double cs[3];
    for (int d = 0; d < 3; d++) {
        nc[d] = (int)std::max(1.0, std::min(256.0, floor(box[3 + d] / r_max)));
        cs[d] = box[3 + d] / nc[d];
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    auto cell_of = [&](const double *p, int c[3]) {
        for (int d = 0; d < 3; d++) c[d] = std::min(nc[d] - 1, std::max(0, (int)((p[d] - box[d]) / cs[d])));
    };
    std::vector<int64_t> start(ncell + 1, 0), order(N);
    std::vector<int64_t> key(N);
    for (int64_t i = 0; i < N; i++) {
        int c[3];
        cell_of(x + 3 * i, c);
        key[i] = ((int64_t)c[2] * nc[1] + c[1]) * nc[0] + c[0];
        start[key[i] + 1]++;
    }
    for (int64_t k = 0; k < ncell; k++) start[k + 1] += start[k];
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t i = 0; i < N; i++) order[fill[key[i]]++] = i;
    }
    const int64_t S = std::min<int64_t>(N, 4096);
    std::vector<double> hist(NR, 0.0);
    const double r2max = r_max * r_max, inv_dr = NR / r_max;
    for (int64_t k = 0; k < S; k++) {
        const int64_t s = k * N / S;
        const double *ps = x + 3 * s;
        int c[3];
        cell_of(ps, c);
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int ix = c[0] + dx, iy = c[1] + dy, iz = c[2] + dz;
                    if (ix < 0 || iy < 0 || iz < 0 || ix >= nc[0] || iy >= nc[1] || iz >= nc[2]) continue;
                    const int64_t cell = ((int64_t)iz * nc[1] + iy) * nc[0] + ix;
                    for (int64_t q = start[cell]; q < start[cell + 1]; q++) {
                        const int64_t j = order[q];
                        if (j == s) continue;
                        const double ex = x[3 * j] - ps[0], ey = x[3 * j + 1] - ps[1], ez = x[3 * j + 2] - ps[2];
                        const double d2 = ex * ex + ey * ey + ez * ez;
                        if (d2 <= r2max) hist[std::min(NR - 1, (int)(sqrt(d2) * inv_dr))] += 1.0;
                    }
                }
    }
    std::vector<double> f(NR);
    double cum = 0.0;
    for (int i = 0; i < NR; i++) {
        cum += hist[i];
        const double r = (i + 1) * r_max / NR;
        const double expect = (double)(N - 1) * pair_prob_box(r, box[3], box[4], box[5]);
        f[i] = (expect > 0.0 && cum > 0.0) ? (cum / S) / expect : 1.0;
    }
    return f;
}

extern "C" se_status_t se_choose_params_points(se_kernel_t kernel, se_prec_t prec, int64_t N, const double box[6],
                                               const void *x_host, double tol, const se_params_t *in,
                                               se_params_t *out) {
    if (!out || !box || !x_host) return fail(SE_ERR_INVALID_ARG, "NULL argument");
    if (kernel < SE_STOKESLET || kernel > SE_ROTLET) return fail(SE_ERR_INVALID_ARG, "unknown kernel");
    if (N < 1) return fail(SE_ERR_INVALID_ARG, "N must be positive");
    for (int d = 0; d < 3; d++)
        if (!(box[3 + d] > 0)) return fail(SE_ERR_INVALID_ARG, "box sides must be positive");
    // the choice for uniform points first: clustering adds pairs at every
    // radius, so the work model's optimum moves to a smaller cutoff
    se_params_t uni;
    se_status_t s = choose_box_params(kernel, prec, N, box, tol, in, 0.0, &uni);
    if (s != SE_OK) return s;
    const bool model = !(in && (in->xi > 0 || in->M > 0 || in->max_fft > 0 || in->rc > 0));
    const double smin = std::min(box[3], std::min(box[4], box[5]));
    if (!model || N < 2 || !(uni.rc < smin)) {
        *out = uni;
        return SE_OK;
    }
    std::vector<double> xd;
    const double *x = (const double *)x_host;
    if (prec == SE_FP32) {
        xd.resize(3 * (size_t)N);
        const float *xf = (const float *)x_host;
        for (size_t i = 0; i < xd.size(); i++) xd[i] = xf[i];
        x = xd.data();
    }
    const int NR = 64;
    const std::vector<double> f = pair_factor_table(x, N, box, uni.rc, NR);
    PairFactor pf;
    pf.n = NR;
    pf.dr = uni.rc / NR;
    pf.f = f.data();
    se_params_t pm;
    s = choose_box_params(kernel, prec, N, box, tol, in, 0.0, &pm, 1, &pf);
    if (s != SE_OK) return s;
    // FFT length: of the fast lengths (fast_fft_len) around 2 (M + P), the one
    // of least modelled work
    auto fast = [prec](int n) { return fast_fft_len(n, prec); };
    const int Mf0 = 2 * (pm.M + pm.P);
    int lo = Mf0, hi = Mf0;
    while (lo > 2 * (pm.P + 2) && !fast(lo)) lo -= 2;
    while (!fast(hi)) hi += 2;
    const double lmax = std::max(box[3], std::max(box[4], box[5]));
    const int64_t neff = (int64_t)llround(std::max(1.0, (double)N * lmax * lmax * lmax / (box[3] * box[4] * box[5])));
    double best = 1e300;
    *out = pm;
    for (int Mf : {lo, hi}) {
        if (!fast(Mf)) continue;
        se_params_t fin;
        memset(&fin, 0, sizeof(fin));
        if (in) fin = *in;
        fin.M = Mf / 2 - pm.P;
        fin.P = pm.P;
        if (fin.M < 2) continue;
        se_params_t c;
        if (choose_box_params(kernel, prec, N, box, tol, &fin, 0.0, &c, 1, &pf) != SE_OK) continue;
        const double cost = model_cost(prec, neff, lmax, c.P, c.M, c.rc, &pf, 1);
        if (cost < best) {
            best = cost;
            *out = c;
        }
    }
    // FP32 real-space cells from the density around the pairs (the mean
    // density times the neighbour factor at the cutoff): clusters of 8 points
    // about as long as wide there
    if (prec == SE_FP32 && !(in && in->cell_width > 0)) {
        const double vol = box[3] * box[4] * box[5];
        out->cell_width = 1.1 * cbrt(8.0 * vol / ((double)N * std::max(1.0, pf.at(out->rc))));
    }
    return SE_OK;
}

extern "C" se_status_t se_plan_create(se_kernel_t kernel, int64_t N, double xi, const double box[4], double tol,
                                      se_prec_t prec, const se_params_t *params, se_plan_t *plan_out) {
    if (!box) return fail(SE_ERR_INVALID_ARG, "box is NULL");
    const double b6[6] = {box[0], box[1], box[2], box[3], box[3], box[3]};
    return se_plan_create_box(kernel, N, xi, b6, tol, prec, params, plan_out);
}

// Parameters of a triply periodic plan in the cube of side L: the selection of
// the free-space plan (the estimates of Tables 2 and 3 hold for the periodic
// sums they were derived for), then M rounded up to an even FFT-friendly size
// and, when the cutoff is not below L/2 (minimum images), xi raised until it is.
static se_status_t choose_periodic_params(int kernel, int prec, int64_t N, double L, double tol,
                                          const se_params_t *params, double xi, se_params_t *out) {
    se_status_t s = choose_params(kernel, prec, N, L, tol, params, xi, out);
    if (s != SE_OK) return s;
    const bool fixed_rc = params && params->rc > 0;
    for (int it = 0; it < 8 && !(out->rc < 0.5 * L); it++) {
        if (fixed_rc) break;
        se_params_t in;
        memset(&in, 0, sizeof(in));
        if (params) in = *params;
        in.xi = 0;
        in.M = 0;
        s = choose_params(kernel, prec, N, L, tol, &in, out->xi * out->rc / (0.45 * L), out);
        if (s != SE_OK) return s;
    }
    if (!(out->rc < 0.5 * L)) return fail(SE_ERR_INVALID_ARG, "periodic plan: rc must be below L/2");
    int M = out->M;
    if (params && params->M > 0) {
        if (M & 1) return fail(SE_ERR_INVALID_ARG, "periodic plan: M must be even");
    } else {
        while ((M & 1) || !good_fft(M, prec)) M++;
    }
    out->M = M;
    return SE_OK;
}

// Plan creation shared by the free-space and the periodic entry points.
static se_status_t create_plan(se_kernel_t kernel, int64_t N, double xi, const double box[6], double tol,
                               se_prec_t prec, const se_params_t *params, bool periodic, se_plan_t *plan_out) {
    if (!plan_out) return fail(SE_ERR_INVALID_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (kernel < SE_STOKESLET || kernel > SE_ROTLET) return fail(SE_ERR_INVALID_ARG, "unknown kernel");
    if (prec != SE_FP32 && prec != SE_FP64) return fail(SE_ERR_INVALID_ARG, "unknown precision");
    if (N < 1 || N > (int64_t)INT32_MAX / 4) return fail(SE_ERR_INVALID_ARG, "N out of range");
    if (!box || !(box[3] > 0) || !(box[4] > 0) || !(box[5] > 0))
        return fail(SE_ERR_INVALID_ARG, "box sides must be positive");
    se_params_t pr;
    se_status_t s = periodic ? choose_periodic_params(kernel, prec, N, box[3], tol, params, xi, &pr)
                             : choose_box_params(kernel, prec, N, box, tol, params, xi, &pr);
    if (s != SE_OK) return s;
    if (pr.P < 1 || pr.P > 32) return fail(SE_ERR_INVALID_ARG, "P must be in [1, 32]");
    if (pr.M < 1 || !(pr.xi > 0) || !(pr.rc > 0)) return fail(SE_ERR_INVALID_ARG, "invalid M, xi or rc");

    se_plan_s *p = new se_plan_s();
    s = setup_plan(p, kernel, prec, N, box, pr, periodic);
    if (s != SE_OK) {
        free_plan(p);
        return s;
    }
    size_t esz = (prec == SE_FP32) ? 4 : 8;
    // allocations
    cudaError_t e = cudaSuccess;
    const size_t Nn = (size_t)N;
    const size_t Mf3 = (size_t)p->mf[0] * p->mf[1] * p->mf[2];
    // FFT sizes (z, y, x): the zero-padded 2 Mtilde, or the periodic M
    const int fn[3] = {periodic ? p->mp : p->mf[2], periodic ? p->mp : p->mf[1], periodic ? p->mp : p->mf[0]};
    const size_t nfft = (size_t)fn[0] * fn[1] * fn[2];
    const size_t nk = (size_t)fn[0] * fn[1] * (fn[2] / 2 + 1);
    const size_t O3 = periodic ? (size_t)(p->mp / 2 + 1) * (p->mp / 2 + 1) * (p->mp / 2 + 1)
                               : (size_t)(p->mt[0] + 1) * (p->mt[1] + 1) * (p->mt[2] + 1);
    const size_t v4 = 4 * esz;
    int tile_keys = p->ntiles;
    do {
        if ((e = dmalloc(&p->ghat64, O3 * sizeof(double)))) break;
        if (prec == SE_FP32 && (e = dmalloc(&p->ghat, O3 * sizeof(float)))) break;
        if ((e = dmalloc(&p->grid, (size_t)p->nc * Mf3 * esz))) break;
        if ((e = dmalloc(&p->spec, (size_t)p->nc * nk * 2 * esz))) break;
        if ((e = dmalloc(&p->wgrid, 3 * Mf3 * esz))) break;
        if ((e = dmalloc(&p->b.xs_t, Nn * v4))) break;
        if ((e = dmalloc(&p->b.fs_t, Nn * v4))) break;
        if ((e = dmalloc(&p->b.qs_t, (kernel == SE_STRESSLET ? Nn : 1) * v4))) break;
        if ((e = dmalloc(&p->b.perm_t, Nn * 4))) break;
        if ((e = dmalloc(&p->b.slot_t, Nn * 4))) break;
        if ((e = dmalloc(&p->b.key_t, Nn * 4))) break;
        // counting-sort arrays carry room for the scan's tile sums (see launch_scan)
        auto scan_len = [](size_t n) { return n + 2 + (n + 4095) / 4096 + 1; };
        if ((e = dmalloc(&p->b.cnt_t, scan_len(tile_keys) * 4))) break;
        if ((e = dmalloc(&p->b.xs_r, Nn * v4))) break;
        if ((e = dmalloc(&p->b.fs_r, Nn * v4))) break;
        if ((e = dmalloc(&p->b.qs_r, (kernel == SE_STRESSLET ? Nn : 1) * v4))) break;
        if ((e = dmalloc(&p->b.perm_r, Nn * 4))) break;
        if ((e = dmalloc(&p->b.slot_r, Nn * 4))) break;
        if ((e = dmalloc(&p->b.key_r, Nn * 4))) break;
        if ((e = dmalloc(&p->b.tag_t, Nn * 4))) break;
        if ((e = dmalloc(&p->b.tag_r, Nn * 4))) break;
        {
            const size_t nrows = (size_t)p->geom.ncel[1] * p->geom.ncel[2];
            if ((e = dmalloc(&p->b.ncl, scan_len(nrows) * 4))) break;
            if ((e = dmalloc(&p->b.clusters, (Nn / 4 + nrows + 1) * sizeof(int2)))) break;
        }
        if ((e = dmalloc(&p->b.cnt_r, scan_len(p->ncells) * 4))) break;
        if ((e = dmalloc(&p->b.uj, Nn * 4 * esz))) break;
        if ((e = dmalloc(&p->b.status, 16))) break;
        if ((e = cudaMemset(p->grid, 0, (size_t)p->nc * Mf3 * esz))) break;
        if ((e = cudaMemset(p->b.status, 0, 16))) break;
        if (periodic && (e = dmalloc(&p->pgrid, (size_t)p->nc * nfft * esz))) break;
        if (prec == SE_FP32 && !periodic) {
            // overlapped evaluation: real-space target sums, internal stream
            if ((e = dmalloc(&p->b.rt, Nn * 4 * esz))) break;
            int least = 0, greatest = 0;
            if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest))) break;
            if ((e = cudaStreamCreateWithPriority(&p->s_four, cudaStreamNonBlocking, greatest))) break;
            if ((e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming))) break;
            if ((e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming))) break;
            p->overlap = true;
        }
    } while (0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return fail(e == cudaErrorMemoryAllocation ? SE_ERR_OOM : SE_ERR_CUDA,
                    std::string("plan allocation: ") + cudaGetErrorString(e));
    }
    // cuFFT plans: forward R2C batched over nc components, inverse C2R over 3
    {
        int n[3] = {fn[0], fn[1], fn[2]};
        cufftType tf = (prec == SE_FP32) ? CUFFT_R2C : CUFFT_D2Z;
        cufftType ti = (prec == SE_FP32) ? CUFFT_C2R : CUFFT_Z2D;
        int idist = (int)nfft, odist = (int)nk;
        if (cufftPlanMany(&p->fwd, 3, n, nullptr, 1, idist, nullptr, 1, odist, tf, p->nc) != CUFFT_SUCCESS) {
            free_plan(p);
            return fail(SE_ERR_CUFFT, "cufftPlanMany (forward) failed");
        }
        p->have_fwd = true;
        if (cufftPlanMany(&p->inv, 3, n, nullptr, 1, odist, nullptr, 1, idist, ti, 3) != CUFFT_SUCCESS) {
            free_plan(p);
            return fail(SE_ERR_CUFFT, "cufftPlanMany (inverse) failed");
        }
        p->have_inv = true;
        if (p->nc != 3) {
            if (cufftPlanMany(&p->fwd3, 3, n, nullptr, 1, idist, nullptr, 1, odist, tf, 3) != CUFFT_SUCCESS) {
                free_plan(p);
                return fail(SE_ERR_CUFFT, "cufftPlanMany (forward, 3) failed");
            }
            p->have_fwd3 = true;
        }
#ifndef SE_PRUNED_FFT
#define SE_PRUNED_FFT 1
#endif
#ifndef SE_ZFUSE
#define SE_ZFUSE 1
#endif
        if (SE_PRUNED_FFT && !periodic) {
            // the spread grid is zero outside z, y, x < Mtilde and the gather reads
            // only that corner: the 2D (y, x) transforms run on the Mtilde planes
            // z < Mtilde, the transform along z on every (ky, kx) column
            int n2[2] = {p->mf[1], p->mf[0]};
            int re2[2] = {p->mf[1], p->mf[0]}, ce2[2] = {p->mf[1], p->mf[0] / 2 + 1};
            const int plane_r = p->mf[1] * p->mf[0], plane_c = p->mf[1] * (p->mf[0] / 2 + 1);
            int nz[1] = {p->mf[2]};
            cufftType tz = (prec == SE_FP32) ? CUFFT_C2C : CUFFT_Z2Z;
            if (cufftPlanMany(&p->f2d, 2, n2, re2, 1, plane_r, ce2, 1, plane_c, tf, p->mt[2]) != CUFFT_SUCCESS ||
                cufftPlanMany(&p->i2d, 2, n2, ce2, 1, plane_c, re2, 1, plane_r, ti, p->mt[2]) != CUFFT_SUCCESS ||
                cufftPlanMany(&p->zc, 1, nz, nz, plane_c, 1, nz, plane_c, 1, tz, plane_c) != CUFFT_SUCCESS) {
                free_plan(p);
                return fail(SE_ERR_CUFFT, "cufftPlanMany (zero-padding-aware transforms) failed");
            }
            p->pruned = true;
            // FP32: the z-transforms and the scaling fused into one kernel
            if (SE_ZFUSE && prec == SE_FP32 && zfuse_supported(p->mf[2], p->nc) &&
                zfuse_twiddles(p->mf[2], &p->zw) != cudaSuccess) {
                free_plan(p);
                return fail(SE_ERR_OOM, "twiddle table of the fused z-transforms");
            }
        }
    }
    if (prec == SE_FP64 && erfc_table_init() != cudaSuccess) {
        free_plan(p);
        return fail(SE_ERR_CUDA, "the FP64 erfc table could not be copied to the device");
    }
    for (int i = 0; i < 9; i++) cudaEventCreate(&p->ev[i]);
    cudaEventCreate(&p->ev_real);
    s = periodic ? periodic_octant(p) : precompute(p);
    if (s != SE_OK) {
        free_plan(p);
        return s;
    }
    *plan_out = p;
    return SE_OK;
}

extern "C" se_status_t se_plan_create_box(se_kernel_t kernel, int64_t N, double xi, const double box[6],
                                          double tol, se_prec_t prec, const se_params_t *params,
                                          se_plan_t *plan_out) {
    return create_plan(kernel, N, xi, box, tol, prec, params, false, plan_out);
}

extern "C" se_status_t se_plan_create_periodic(se_kernel_t kernel, int64_t N, double xi, const double box[4],
                                               double tol, se_prec_t prec, const se_params_t *params,
                                               se_plan_t *plan_out) {
    if (!box) return fail(SE_ERR_INVALID_ARG, "box is NULL");
    const double b6[6] = {box[0], box[1], box[2], box[3], box[3], box[3]};
    return create_plan(kernel, N, xi, b6, tol, prec, params, true, plan_out);
}

extern "C" se_status_t se_choose_params(se_kernel_t kernel, se_prec_t prec, int64_t N, double L, double tol,
                                        double xi, const se_params_t *in, se_params_t *out) {
    if (!out) return fail(SE_ERR_INVALID_ARG, "out is NULL");
    if (kernel < SE_STOKESLET || kernel > SE_ROTLET) return fail(SE_ERR_INVALID_ARG, "unknown kernel");
    if (N < 1 || !(L > 0)) return fail(SE_ERR_INVALID_ARG, "N and L must be positive");
    return choose_params(kernel, prec, N, L, tol, in, xi, out);
}

extern "C" se_status_t se_plan_destroy(se_plan_t plan) {
    if (!plan) return SE_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return SE_OK;
}

extern "C" se_status_t se_plan_get_params(se_plan_t p, se_params_t *out) {
    if (!p || !out) return fail(SE_ERR_INVALID_ARG, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->xi = p->xi;
    out->rc = p->rc;
    // the longest dimension's sizes (all equal for a cube; se_plan_get_grid has each)
    out->M = std::max(p->mm[0], std::max(p->mm[1], p->mm[2]));
    out->P = p->P;
    out->deltaL_policy = p->deltaL_policy;
    out->max_fft = p->max_fft;
    out->cell_width = p->cell_width;
    out->Mtilde = std::max(p->mt[0], std::max(p->mt[1], p->mt[2]));
    out->Mg = std::max(p->mg[0], std::max(p->mg[1], p->mg[2]));
    out->eta = p->eta;
    out->h = p->h;
    return SE_OK;
}

extern "C" se_status_t se_plan_get_grid(se_plan_t p, int M[3], int Mtilde[3], int Mf[3], int Mg[3]) {
    if (!p) return fail(SE_ERR_INVALID_ARG, "NULL plan");
    for (int d = 0; d < 3; d++) {
        if (M) M[d] = p->mm[d];
        if (Mtilde) Mtilde[d] = p->mt[d];
        if (Mf) Mf[d] = p->periodic ? p->mp : p->mf[d];  // the FFT size
        if (Mg) Mg[d] = p->mg[d];
    }
    return SE_OK;
}

extern "C" se_status_t se_plan_check(se_plan_t p) {
    if (!p) return fail(SE_ERR_INVALID_ARG, "NULL plan");
    cudaError_t e = p->last_stream ? cudaStreamSynchronize(p->last_stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(SE_ERR_CUDA, std::string("se_plan_check: ") + cudaGetErrorString(e));
    int flags = 0;
    if ((e = cudaMemcpy(&flags, p->b.status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(SE_ERR_CUDA, std::string("se_plan_check: ") + cudaGetErrorString(e));
    cudaMemset(p->b.status, 0, sizeof(int));
    if (flags & FLAG_TIMEOUT) return fail(SE_ERR_TIMEOUT, "a bounded device wait ran out (tensor copy)");
    if (flags & FLAG_OOB) return fail(SE_ERR_OUT_OF_BOX, "a point lies outside the plan's box");
    if (flags & FLAG_COINCIDENT) return fail(SE_ERR_COINCIDENT, "coincident points were skipped");
    return SE_OK;
}

extern "C" se_status_t se_plan_set_timing(se_plan_t p, int on) {
    if (!p) return fail(SE_ERR_INVALID_ARG, "NULL plan");
    p->timing = on != 0;
    return SE_OK;
}

extern "C" se_status_t se_plan_set_test_flags(se_plan_t p, int flags) {
    if (!p) return fail(SE_ERR_INVALID_ARG, "NULL plan");
    if (flags & ~SE_TEST_SKIP_TILE_COPY) return fail(SE_ERR_INVALID_ARG, "unknown test flag");
    p->test_flags = flags;
    return SE_OK;
}

extern "C" se_status_t se_plan_set_overlap(se_plan_t p, int on) {
    if (!p) return fail(SE_ERR_INVALID_ARG, "NULL plan");
    if (on && !p->s_four) return fail(SE_ERR_NOT_SUPPORTED, "overlapped evaluation needs an FP32 free-space plan");
    p->overlap = on != 0;
    return SE_OK;
}

extern "C" se_status_t se_plan_set_keep_grid(se_plan_t p, int on) {
    if (!p) return fail(SE_ERR_INVALID_ARG, "NULL plan");
    p->keep_grid = on != 0;
    return SE_OK;
}

extern "C" int se_plan_stage_times(se_plan_t p, float *ms, int max_n) {
    if (!p || !ms) return 0;
    int n = std::min(max_n, p->n_stage);
    for (int i = 0; i < n; i++) ms[i] = p->stage_ms[i];
    return n;
}

extern "C" int64_t se_plan_launch_count(se_plan_t p) { return p ? p->launches : -1; }

extern "C" const char *se_last_error(void) { return g_last_error.c_str(); }
extern "C" const char *se_version(void) { return "se-gb300 0.1 (sm_103a)"; }
