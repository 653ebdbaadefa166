/*
 * se.h -- C ABI of the GB300 free-space Spectral Ewald library (libse.so).
 *
 * Computes, for N points x_n in a cube and their sources,
 *
 *     u(x_m) = sum_{n != m} K(x_m - x_n) . f_n            (Section 1, eq. usumfree;
 *                                                           Section 2, eq. usum)
 *
 * for the stokeslet  u_j = S_jl f_l,       S_jl = delta_jl/r + r_j r_l/r^3   (eq. def_stokeslet)
 *     stresslet      u_j = T_jlm f_l q_m,  T_jlm = -6 r_j r_l r_m / r^5     (eq. def_stresslet)
 *     rotlet         u_j = Omega_jl f_l,   Omega_jl = eps_jlm r_m / r^3      (eq. def_rotlet)
 *
 * with the free-space Ewald split of Section 3.2 (Hasimoto screening for S and
 * T, Ewald screening for Omega): u = u^R + u^F + u^self (Section 8).  u^F uses
 * the Spectral Ewald steps of Section 5.2 (spreading, zero-padded FFT, scaling
 * by the precomputed truncated Green's function of Section 4.3, inverse FFT,
 * quadrature) and u^R the screened real-space sum over |r| <= rc (Section 6).
 * No 1/(8 pi mu) prefactor is applied.  The rotlet is the definition above;
 * the operator form of eq. rotlet_op is twice as large.
 *
 * Conventions for every call below:
 *  - Arrays are row-major, contiguous, in the plan's precision (float for
 *    SE_FP32, double for SE_FP64): x, f, q, u, grad_* are N x 3.
 *  - Device pointers are owned by the caller; the library never frees them.
 *    Host pointers are accepted only where a name ends in _host.
 *  - Points must lie in the half-open cube [x0, x0+L)^3 of the plan.
 *  - Calls taking a stream are asynchronous on that stream (0 = legacy
 *    default stream).  A plan is used by one stream at a time and is not
 *    thread-safe.
 *  - Every call returns an se_status_t.  Errors found on the device (a point
 *    outside the box, coincident points) are recorded in the plan and
 *    reported by se_plan_check, which synchronises the plan's last stream.
 *  - se_last_error() returns a message for the last failing call on the
 *    calling thread.
 */
#ifndef SE_H
#define SE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { SE_STOKESLET = 0, SE_STRESSLET = 1, SE_ROTLET = 2 } se_kernel_t;
typedef enum { SE_FP32 = 0, SE_FP64 = 1 } se_prec_t;

typedef enum {
    SE_OK = 0,
    SE_ERR_INVALID_ARG = 1,   /* bad size, pointer, parameter or kernel/precision combination */
    SE_ERR_OUT_OF_BOX = 2,    /* a point lies outside [x0, x0+L)^3 (results undefined)        */
    SE_ERR_COINCIDENT = 3,    /* two distinct points coincide; the pair was skipped (warning)  */
    SE_ERR_OOM = 4,           /* device or host allocation failed                             */
    SE_ERR_CUDA = 5,          /* a CUDA runtime call failed                                   */
    SE_ERR_CUFFT = 6,         /* a cuFFT call failed                                          */
    SE_ERR_TIMEOUT = 7,       /* a bounded device wait ran out                                */
    SE_ERR_NOT_SUPPORTED = 8  /* valid request that the library does not implement            */
} se_status_t;

typedef struct se_plan_s *se_plan_t;

/* Method parameters (Section 8.2).  A zero/negative field is chosen by the
 * library's parameter selection (Tables 2 and 3, Section 8.2); set fields are
 * taken as given.  After se_plan_create, se_plan_get_params fills every field. */
typedef struct {
    double xi;          /* Ewald parameter xi                                          */
    double rc;          /* real-space cutoff radius r_c                                */
    int M;              /* grid points across the box side L (h = L/M)                 */
    int P;              /* Gaussian support: P^3 grid points per source (Section 5.2)  */
    int deltaL_policy;  /* 0: delta_L = d = hP;  1: eq. deltaL_cond (Section 5.3)      */
    int max_fft;        /* upper bound on the FFT size 2*Mtilde per dimension (0: none) */
    double cell_width;  /* FP32 real-space cells across their rows (0: from the mean point
                           density; se_choose_params_points sets it from the density
                           around the points' pairs)                                   */
    /* derived, filled by se_plan_get_params (ignored on input) */
    int Mtilde;         /* extended grid points per dimension, M + delta_L/h           */
    int Mg;             /* precompute grid size: smallest even > (1+sqrt 3) Mtilde      */
    double eta;         /* Gaussian shape parameter eta = (xi d / m)^2, m = 0.976 sqrt(pi P) */
    double h;           /* grid spacing L/M                                            */
} se_params_t;

/* Create a plan for N points in the cube box = {x0, y0, z0, L}.
 *   kernel  SE_STOKESLET, SE_STRESSLET or SE_ROTLET
 *   N       number of points (sources = targets), N >= 1
 *   xi      Ewald parameter; <= 0 lets the library choose (overridden by params->xi > 0)
 *   tol     target relative RMS error used when parameters are chosen (e.g. 2e-6)
 *   prec    SE_FP32 or SE_FP64 arithmetic for spreading, FFTs, gather and real space;
 *           the truncated Green's function is always precomputed in FP64
 *   params  optional overrides (NULL: choose everything)
 * Allocates all device workspaces, builds the cuFFT plans and runs the FP64
 * precomputation of Section 4.3 on the current device (synchronously).
 * The plan owns its memory until se_plan_destroy. */
se_status_t se_plan_create(se_kernel_t kernel, int64_t N, double xi, const double box[4], double tol,
                           se_prec_t prec, const se_params_t *params, se_plan_t *plan_out);

/* As se_plan_create for a rectangular box: box = (x0, y0, z0, Lx, Ly, Lz).
 * One grid spacing h in all dimensions (M of se_params_t counts the intervals
 * along the longest side; the others take the smallest M covering their side
 * with an FFT-friendly length), the truncation radius R is the diagonal of the
 * extended box and the precompute grid is oversampled by 1 + R/Ltilde_d per
 * dimension (Section 4.2).  Parameters are selected as for the cube of the
 * longest side at the same point density. */
se_status_t se_plan_create_box(se_kernel_t kernel, int64_t N, double xi, const double box[6], double tol,
                               se_prec_t prec, const se_params_t *params, se_plan_t *plan_out);

/* A plan for the triply periodic sums in the cube box = (x0, y0, z0, L): u(x_m)
 * = sum over n and over all periodic images of K(x_m - x_n + p L) . f_n (the
 * n = m term of the unshifted image excluded), split as the free-space sum
 * (Section 3, Table 1) with the Fourier part summed over k = 2 pi j / L, j !=
 * 0 (the periodic problem of Section 1.1; the k = 0 term is left out, i.e. the
 * mean force is balanced by a mean pressure gradient, Hasimoto's convention).
 * The Fourier part runs on the unpadded periodic M^3 grid with the exact
 * transforms 4 pi/k^2 and -8 pi/k^4 in place of the precomputed truncated
 * ones (no precomputation); the real-space part takes nearest images.
 * Arguments as for se_plan_create.  Parameters are selected as for the
 * free-space cube, then M is rounded up to an even FFT-friendly size and xi is
 * raised until rc < L/2 (an explicit params->rc must satisfy rc < L/2 and an
 * explicit params->M must be even: SE_ERR_INVALID_ARG otherwise).  Points must
 * lie in the half-open box (SE_ERR_OUT_OF_BOX from se_plan_check otherwise).
 * Supported calls on such a plan: se_eval, se_eval_host, se_eval_real_space,
 * the status, timing and parameter queries; se_eval_targets and the backward
 * calls return SE_ERR_NOT_SUPPORTED. */
se_status_t se_plan_create_periodic(se_kernel_t kernel, int64_t N, double xi, const double box[4], double tol,
                                    se_prec_t prec, const se_params_t *params, se_plan_t *plan_out);

/* u = sum_{n != m} K(x_m - x_n) . f_n at every point (Section 8).
 *   x  N x 3 device positions; f N x 3 device strengths (forces, dipoles or torques)
 *   q  N x 3 device second source vector for the stresslet (u_j = T_jlm f_l q_m), else NULL
 *   u  N x 3 device output (overwritten)
 * Asynchronous on `stream`. */
se_status_t se_eval(se_plan_t plan, const void *x, const void *f, const void *q, void *u, void *stream);

/* u at separate targets: ut(y_i) = sum_n K(y_i - x_n) . f_n for Nt target
 * points y (the paper evaluates the sums at the sources or at any other points,
 * Section 2 below eq. usumfree): the Fourier part gathered at the targets plus
 * the real-space sum over the sources within rc of each target, with no self
 * term and no excluded pair.  x, f (, q): the plan's N sources as in se_eval;
 * xt: Nt x 3 targets in the plan's box, ut: Nt x 3 output (overwritten); device
 * arrays in the plan's precision.  A source at distance zero from a target is
 * skipped and reported by se_plan_check as SE_ERR_COINCIDENT.  The first call
 * with a larger Nt than before allocates the plan's target buffers (and
 * synchronises the device).  Asynchronous on `stream` otherwise. */
se_status_t se_eval_targets(se_plan_t plan, const void *x, const void *f, const void *q, int64_t Nt, const void *xt,
                            void *ut, void *stream);

/* Same as se_eval with HOST arrays: copies x, f (, q) to the device, evaluates,
 * copies u back and synchronises `stream` before returning. */
se_status_t se_eval_host(se_plan_t plan, const void *x_host, const void *f_host, const void *q_host,
                         void *u_host, void *stream);

/* Gradients of L = sum_m grad_u_m . u_m (no counterpart in the paper; derived
 * from the Fourier representation of Section 5.2, eqs. Hx and u_integr, and the
 * real-space kernels of Section 3.2):
 *   stokeslet, rotlet: grad_f_n = sum_m K(x_m - x_n)^T grad_u_m (the same SE
 *              operator applied to grad_u, since both operators are symmetric)
 *   stresslet: grad_f_n,l = V_lk(x_n) q_n,k, grad_q_n,k = V_lk(x_n) f_n,l with the
 *              adjoint field V_lk(y) = sum_m T_jlk(x_m - y) grad_u_m,j (the
 *              negated stresslet symbol on 3 -> 6 grids)
 *   grad_x_p = d L / d x_p: Gaussian-derivative quadrature on the forward grid
 *              and on the adjoint grid, plus the derivative of the real-space
 *              kernel (the self term does not depend on x).
 * Same arrays as se_eval (q: the stresslet's q, else NULL); grad_u, grad_f,
 * grad_q, grad_x are N x 3 device arrays in the plan's precision, overwritten.
 * Any output may be NULL.  The forward grid (needed by grad_x) is recomputed
 * from x, f (, q), unless keep-grid is on (se_plan_set_keep_grid) and the
 * plan's last se_eval or se_eval_targets was given the same x, f and q arrays.
 * se_eval_backward is se_eval_backward_q without grad_q.  grad_q must be NULL
 * for the stokeslet and the rotlet (SE_ERR_INVALID_ARG). */
se_status_t se_eval_backward_q(se_plan_t plan, const void *x, const void *f, const void *q, const void *grad_u,
                               void *grad_f, void *grad_q, void *grad_x, void *stream);
se_status_t se_eval_backward(se_plan_t plan, const void *x, const void *f, const void *q,
                             const void *grad_u, void *grad_f, void *grad_x, void *stream);

/* The screened real-space part alone (Section 6): u^R(x_m) = sum over
 * 0 < |x_m - x_n| <= rc of K^R(x_m - x_n) . f_n with the split kernels of
 * Section 3.2 and the plan's xi and rc (no Fourier part, no self term).
 * Same argument conventions as se_eval; u is overwritten.  Uses the plan's
 * cell-list workspaces.  Asynchronous on `stream`. */
se_status_t se_eval_real_space(se_plan_t plan, const void *x, const void *f, const void *q, void *u, void *stream);

/* The real-space sum of se_eval_real_space for callers that cannot allocate
 * device memory (their host program's arena owns all of it, or they run in a
 * loop that must never call the allocator).  No plan: the method parameters
 * xi and rc and the box are passed directly; x, f (, q for the stresslet) and u
 * are N x 3 device arrays of the precision `prec`, u is overwritten.  All
 * temporaries live in one fixed-size __device__ array inside the library
 * (about 9 MB, held on every GPU that loads the library until the process
 * exits); nothing is allocated.  Limits: N <= 32768 and L / rc <= 25 (the cell
 * list's size); larger requests return SE_ERR_INVALID_ARG.  The first call on a
 * device looks up the array's address (make it before any stream capture);
 * later calls outside a capture look it up again, so a context destroyed and
 * created again (cudaDeviceReset) is followed.
 * Calls whose GPU work overlaps race on the shared array.  Device-side flags
 * (points outside the box, coincident points) are not reported.  The paper has
 * no counterpart to this entry point.  Asynchronous on `stream`. */
se_status_t se_real_space_noalloc(se_kernel_t kernel, se_prec_t prec, int64_t N, const double box[4], double xi,
                                  double rc, const void *x, const void *f, const void *q, void *u, void *stream);

/* ---------------------------------------------------------------- batches
 * Many independent systems, each with several right-hand sides, in one call.
 * The paper evaluates one system at a time; it notes that the FFT of the
 * truncated Green's function is done once for several right-hand sides
 * (Section 4.3) and that the precomputation is amortised over many calls
 * (Section 9).  A batch applies Section 8 to every system: the precomputed
 * kernel of each system is made once, at creation, and every stage runs as one
 * launch over all systems (the FFTs as one batched transform per FFT size).
 * Stokeslet and rotlet only.
 *
 * Layout: system s owns points [off_s, off_s + N_s) of the concatenated arrays
 * (off_s = N_0 + ... + N_{s-1}).  x: sumN x 3, f and u: sumN x n_rhs x 3
 * (right-hand side r of point i at ((i * n_rhs + r) * 3)), row-major, device
 * memory, in the batch's precision; u is overwritten.  box_s: S x 4 (x0, y0,
 * z0, L) on the host.  Each system's points must lie in its half-open box. */
typedef struct se_batch_s *se_batch_t;

/* Create a batch of S systems with N_s[s] points and box box_s[4 s ..] each,
 * n_rhs in [1, 64] right-hand sides, target relative error tol.  Each system
 * gets M, xi and rc from the single-plan parameter selection (params: NULL or
 * overrides common to all systems, e.g. max_fft); the support P is the largest
 * chosen and is common to the batch (P <= 16, so tol >= about 1e-8).  Allocates
 * all device memory and runs every system's FP64 precomputation.
 * SE_ERR_NOT_SUPPORTED for the stresslet or P > 16. */
se_status_t se_batch_create(se_kernel_t kernel, int S, const int64_t *N_s, const double *box_s, int n_rhs,
                            double tol, se_prec_t prec, const se_params_t *params, se_batch_t *out);

/* Evaluate all systems and right-hand sides: u = u^R + u^F + u^self per system.
 * With graph mode on (the default) the first call for a given (x, f, u)
 * captures the whole sequence into a CUDA graph (on an internal stream) and
 * every call launches that graph on `stream`; new pointers re-capture.
 * Asynchronous on `stream`. */
se_status_t se_batch_eval(se_batch_t batch, const void *x, const void *f, void *u, void *stream);

/* Graph mode on (1, default) or off (0: every call launches the kernels). */
se_status_t se_batch_set_graph(se_batch_t batch, int on);

/* Stage timing on (1) or off (0, default).  While on, se_batch_eval launches
 * the kernels without the graph and records events between the stages;
 * se_batch_stage_times then gives the device times (milliseconds) of the last
 * timed call in the order bin, spread (octant zeroing included), fft, scale,
 * ifft, gather, real (the cluster lists and the pair sums): returns the
 * number written (7, or 0 before the first timed call or for NULL arguments).
 * No counterpart in the paper (measurement only). */
se_status_t se_batch_set_timing(se_batch_t batch, int on);
int se_batch_stage_times(se_batch_t batch, float *ms, int max_n);

/* Parameters chosen for system s (as se_plan_get_params). */
se_status_t se_batch_get_params(se_batch_t batch, int s, se_params_t *out);

/* Synchronise the stream of the last call; return (and clear) the device-side
 * status: SE_OK, SE_ERR_OUT_OF_BOX or SE_ERR_COINCIDENT. */
se_status_t se_batch_check(se_batch_t batch);

/* Number of this library's kernels in one evaluation of the batch (cuFFT's
 * transforms and memsets not counted); -1 for NULL. */
int64_t se_batch_launch_count(se_batch_t batch);

/* Free everything the batch holds (synchronises the device). */
se_status_t se_batch_destroy(se_batch_t batch);

/* Parameter selection without a device (host only; the same rules as
 * se_plan_create, Section 8.2 with Tables 2 and 3): fills M, P, xi and rc of
 * *out from the overrides in *in (may be NULL), the box side L, N, tol and
 * the precision.  Derived fields are not filled. */
se_status_t se_choose_params(se_kernel_t kernel, se_prec_t prec, int64_t N, double L, double tol, double xi,
                             const se_params_t *in, se_params_t *out);

/* Fill *out with the plan's parameters (chosen or given, plus derived values). */
/* Parameter selection that looks at the points: x_host holds the N points
 * (host memory, N x 3 row-major, float for SE_FP32 and double for SE_FP64) in
 * the box (x0, y0, z0, Lx, Ly, Lz).  The mean number of neighbours of up to
 * 4096 sampled points (every (N/4096)-th) is measured at 64 radii up to the
 * cutoff chosen for uniform points and divided by its value for uniform points
 * in the box; the work model that balances the real-space pairs against the
 * grid and FFT work (used when xi, M, rc and max_fft are left to the library)
 * then counts pairs with that factor, so clustered points get a larger xi and
 * a smaller cutoff.  With any of xi, M, rc or max_fft fixed in `in`, the
 * result is that of se_choose_params.  Host only; the points are not kept.
 * Errors: SE_ERR_INVALID_ARG for NULL pointers, N < 1 or a side <= 0. */
se_status_t se_choose_params_points(se_kernel_t kernel, se_prec_t prec, int64_t N, const double box[6],
                                    const void *x_host, double tol, const se_params_t *in, se_params_t *out);

se_status_t se_plan_get_params(se_plan_t plan, se_params_t *out);

/* Grid sizes per dimension (x, y, z): M (box), Mtilde (extended grid), the FFT
 * size (2 Mtilde; M for a periodic plan) and the precompute grid (0 for a
 * periodic plan); any pointer may be NULL. */
se_status_t se_plan_get_grid(se_plan_t plan, int M[3], int Mtilde[3], int Mf[3], int Mg[3]);

/* Synchronise the stream of the plan's last call and return (and clear) the
 * device-side status: SE_OK, SE_ERR_TIMEOUT (a bounded device wait ran out;
 * the outputs of that call are undefined and must be discarded, the plan stays
 * usable), SE_ERR_OUT_OF_BOX or SE_ERR_COINCIDENT. */
se_status_t se_plan_check(se_plan_t plan);

/* Test flags of a plan (0 restores normal operation).  SE_TEST_SKIP_TILE_COPY:
 * the FP32 gather does not issue its tiles' tensor copies, so each tile's
 * bounded wait (one second) runs out; the evaluation then leaves u undefined
 * and se_plan_check returns SE_ERR_TIMEOUT, with the context still usable.
 * For tests of the failure path only.  SE_ERR_INVALID_ARG for unknown flags. */
#define SE_TEST_SKIP_TILE_COPY 1
se_status_t se_plan_set_test_flags(se_plan_t plan, int flags);

/* Per-stage device times of the plan's last se_eval or se_eval_backward, in
 * milliseconds, when stage timing was enabled with se_plan_set_timing(plan, 1).
 * se_eval order: bin, spread, fft, scale, ifft, gather, real_setup (the
 * real-space cluster list; 0 in FP64), real (the real-space pair-sum kernel
 * alone).  se_eval_backward order: adj_bin (g sorted as the source), adj_fourier
 * (spread of g, transforms and scaling), adj_gather, adj_real (du/df, du/dq),
 * bin, fourier (the forward grid, recomputed), grad_gather, grad_real (du/dx);
 * a step the call skips takes 0.  Returns the number written (8, or 0 before
 * the first timed call). */
int se_plan_stage_times(se_plan_t plan, float *ms, int max_n);
se_status_t se_plan_set_timing(se_plan_t plan, int on);

/* Overlapped evaluation (FP32 free-space plans; on by default there): se_eval
 * runs the Fourier part (spreading to gather) on an internal high-priority
 * stream, forked from and joined back to the caller's stream, while the
 * real-space sum runs on the caller's stream; the real-space sums are added
 * to u after the join.  The call stays asynchronous on the caller's stream
 * and may be captured into a CUDA graph.  With stage timing on, or with
 * overlap off, the stages run one after another on the caller's stream.
 * Returns SE_ERR_NOT_SUPPORTED when turning it on for a plan without it
 * (FP64 and periodic plans). */
se_status_t se_plan_set_overlap(se_plan_t plan, int on);

/* Keep-grid mode (off by default).  Every se_eval and se_eval_targets leaves
 * the forward grid (the field on the grid after scaling and the inverse
 * transforms, 3 or 9 components) in a plan buffer; with keep-grid on,
 * se_eval_backward / se_eval_backward_q reuse it for grad_x instead of
 * spreading and transforming again, when the x, f and q pointers equal those
 * of the plan's last se_eval or se_eval_targets.  Only the pointers are
 * compared: the caller promises that the arrays' contents did not change
 * in between and that the backward is ordered after that evaluation (same
 * stream, or an event); a failed evaluation, or a backward that recomputed the
 * grid for other inputs, leaves the kept grid to those inputs.  The grid buffer
 * exists in every plan, so the mode costs no memory.  Errors: SE_ERR_INVALID_ARG
 * for a NULL plan. */
se_status_t se_plan_set_keep_grid(se_plan_t plan, int on);

/* Deterministic mode (off by default): se_eval, se_eval_host and
 * se_eval_targets give bit-identical results for identical inputs, call after
 * call.  The method itself (Sections 5 and 6) fixes no summation order; in the
 * default mode three sums take theirs from the order in which threads run:
 * the points inside each spreading tile and real-space cell (slots from
 * atomic counters), and the real-space sum's scattered candidate terms.  With
 * the mode on, the binning ranks the points of each bin by index (a stable
 * radix sort of the bin keys), the spreading stores each tile's padded block
 * and a second pass adds the tiles into the grid in a fixed order (no
 * atomics), and the real-space sum takes the full candidate
 * lists (each pair evaluated from both ends, no scatter), with the Fourier and
 * real-space parts in sequence.  Costs, at N = 1e6 uniform points: about twice
 * the real-space time.  The backward pass is not covered.  Turning it on
 * allocates the radix sort's scratch (about 16 N bytes, grown by
 * se_eval_targets for more targets) and the spreading's tile buffer, and
 * synchronises the device.  Errors: SE_ERR_INVALID_ARG for a NULL plan;
 * SE_ERR_NOT_SUPPORTED when turning it on for an FP64 or a periodic plan;
 * SE_ERR_OOM. */
se_status_t se_plan_set_deterministic(se_plan_t plan, int on);

/* Number of this library's kernels launched by the plan's last se_eval,
 * se_eval_host, se_eval_real_space or se_eval_backward call (cuFFT's kernels
 * and memsets are not counted; the count is taken on the host at launch).
 * Returns -1 for a NULL plan. */
int64_t se_plan_launch_count(se_plan_t plan);

/* The precomputed kernel (Section 4.3) depends only on the Green's function,
 * the grid sizes and h, not on xi, P or the points, so plans with equal grids
 * share it: a host-side cache (on by default, `memory` = 1; 0 turns it off and
 * empties it) and, when `dir` is not NULL, one file per grid in that directory
 * (read before computing, written after).  Process-wide; thread-safe. */
se_status_t se_set_precompute_cache(int memory, const char *dir);

/* Time the plan's precomputation took (ms; for a cache hit, the time of the
 * lookup and upload) and whether it came from the cache (1) or was computed. */
se_status_t se_plan_precompute_info(se_plan_t plan, double *ms, int *cached);

/* Destroy the plan and free its device memory (synchronises the device). */
se_status_t se_plan_destroy(se_plan_t plan);

/* Message of the last failing call on this thread ("" if none). */
const char *se_last_error(void);

/* Library version string. */
const char *se_version(void);

/* Arithmetic rates of the current device, measured (no counterpart in the
 * paper, which reports CPU times only): the denominators of the roofline
 * fractions of the kernels bound by arithmetic rather than memory.  Each rate
 * is the best of three launches, timed with CUDA events, of a register-only
 * kernel in which every thread of 8 blocks of 256 per SM runs 8 independent
 * chains of fused multiply-adds; the iteration count is calibrated so that
 * one launch takes about 20 ms.  Flops count 2 per FMA (4 per paired FMA).
 *   fp32_fma_tflops    scalar FP32 fmaf
 *   fp32_ffma2_tflops  paired FP32 (__ffma2_rn: two FMAs per instruction)
 *   fp64_fma_tflops    FP64 fma
 *   sm_count           multiprocessors of the device
 * Synchronous on the legacy default stream; allocates and frees a small
 * device buffer; about a quarter of a second.  SE_ERR_INVALID_ARG for a NULL
 * out, SE_ERR_CUDA if a launch fails. */
typedef struct {
    double fp32_fma_tflops;
    double fp32_ffma2_tflops;
    double fp64_fma_tflops;
    int sm_count;
} se_peaks_t;
se_status_t se_measure_peaks(se_peaks_t *out);

#ifdef __cplusplus
}
#endif

#endif /* SE_H */
