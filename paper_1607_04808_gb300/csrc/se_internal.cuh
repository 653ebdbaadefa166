// Internal declarations of the GB300 free-space Spectral Ewald library.
// Plan layout, precision traits and the launchers of each stage.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <string>

#include "../../include/se.h"

namespace se {

// ---------------------------------------------------------------- status
enum : int { FLAG_OOB = 1, FLAG_COINCIDENT = 2, FLAG_TIMEOUT = 4 };

void set_error(const std::string &msg);
se_status_t fail(se_status_t st, const std::string &msg);

#define SE_CUDA_TRY(expr)                                                                  \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess)                                                             \
            return ::se::fail(SE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

#define SE_CUFFT_TRY(expr)                                                               \
    do {                                                                                 \
        cufftResult _r = (expr);                                                         \
        if (_r != CUFFT_SUCCESS)                                                         \
            return ::se::fail(SE_ERR_CUFFT, std::string(#expr) + " failed, code " +      \
                                                std::to_string((int)_r));               \
    } while (0)

// ---------------------------------------------------------------- precision traits
template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4_32a; };
template <typename T> using vec4 = typename V4<T>::type;

template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using cplx = typename Cplx<T>::type;

// ---------------------------------------------------------------- geometry shared by kernels
// Everything a kernel needs to place a point on the grids and in the cells.
// Per-dimension arrays are indexed x, y, z; grids are stored z-major with x
// fastest.  The box is a rectangular cuboid with one grid spacing h.
struct Geom {
    double x0[3];      // box corner
    double len[3];     // box sides
    double h, inv_h;   // grid spacing and its inverse
    double half_ext;   // n_ext / 2 (grid units): t = (x - x0)/h + n_ext/2 is (x - y0)/h
    int P;             // Gaussian support (grid points per dimension)
    int mt[3];         // extended grid points per dimension
    int mf[3];         // FFT size per dimension (2 mt)
    int T;             // spreading tile edge (window starts per tile per dimension)
    int nt[3];         // tiles per dimension
    double a;          // Gaussian exponent 2 xi^2 / eta (per unit length^2)
    // real-space cells: rows of cells run along x (split finer along x)
    int ncel[3];       // cells per dimension
    double cw[3], icw[3];  // cell widths and their inverses
    double rc;         // cutoff
    double xi;
};

// Geometry in the arithmetic precision T of the path, so that the FP32 kernels
// never touch the (slow on this part) FP64 pipe for bookkeeping.
template <typename T>
struct GP {
    T x0[3], len[3];   // box corner and sides
    T inv_h, half_ext; // t = (x - x0) / h + n_ext / 2 = (x - y0) / h (grid units)
    T ah2;             // a h^2 = 2 xi^2 h^2 / eta: Gaussian exponent per grid unit^2
    T icw[3], cw[3];   // real-space cell widths (x: along the rows) and inverses
    T ilen[3];         // inverse box sides (minimum images of periodic plans)
    int P, T_;
    int mt[3], mf[3], nt[3], ncel[3];
};

// Screened real-space constants of one system (x = xi r).
template <typename T>
struct RC {
    T xi, xi2, c, c3, rc2;  // xi, xi^2, 2 xi/sqrt(pi), 4 xi^3/sqrt(pi), rc^2
    T ce;                   // -xi^2 / ln 2: exp(-xi^2 r^2) = 2^(ce r^2)
    int reach[2];           // rows of cells within reach on each side in y and in z
    int tab;                // FP64: erfc and the Gaussian term from the device table (erfc_table_init)
};

// Constants of the k-space scaling of one system.
struct ScaleConst {
    double dk[3];     // 2 pi / (mf h) per dimension
    double inv4xi2;   // 1 / (4 xi^2)
    double ecoef;     // -(1 - eta) / (4 xi^2)
    double norm;      // h^3 / (mf_x mf_y mf_z) * pre^2
    int mt[3], mf[3], nxh;  // nxh = mf_x/2 + 1
};

// One system of a batch as the batched kernels see it: its geometry and
// method constants, where its grids live and where its points, tiles, cells
// and cell rows start in the concatenated (and sorted) arrays.
template <typename T>
struct BSys {
    GP<T> g;
    RC<T> rk;
    ScaleConst sc;
    const T *ghat;     // (mt+1) octant of the precomputed kernel
    T *grid;           // spread grids: 3 n_rhs grids of mf_x mf_y mf_z (zero padded)
    cplx<T> *spec;     // their spectra: 3 n_rhs x mf_z x mf_y x (mf_x/2+1)
    T *wgrid;          // inverse transforms: 3 n_rhs grids
    // strides (elements): real grids (grid, wgrid) between z-planes and between
    // the system's 3 n_rhs components, and the same for the spectra.  FP64
    // batches store each grid whole (z stride mf_x mf_y, component stride
    // mf_x mf_y mf_z); FP32 batches interleave the grids of an FFT size class
    // plane by plane, [z][grid][y][x], keeping only the z < mt_z planes of the
    // real grids (z stride: the class's grids times a plane, component stride:
    // a plane)
    size_t gzs, gcs, szs, scs;
    double self_coef;  // -4 xi / sqrt(pi) (stokeslet), 0 otherwise
    int off, n;        // points [off, off + n) of the concatenated and of the sorted order
    int tile_base, cell_base, row_base;
    int blk_base;      // first block of this system in the scaling launch
    int zblk_base;     // first block of this system in the octant-zeroing launch
    int tma;           // the batched gather stages tiles by tensor copy (map s of the batch)
};

// Index s of the range holding v, for ascending bases b[0..S) with b[0] = 0.
__host__ __device__ inline int find_range(const int *b, int S, int v) {
    int lo = 0, hi = S;  // b[lo] <= v < b[hi] (b[S] taken as infinity)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (b[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

// Coordinate relative to the box corner, clamped into [0, L) for points outside
// the box (they are flagged by the binning kernel; clamping keeps every kernel's
// indexing in bounds).
template <typename T>
__host__ __device__ inline T clamp_rel(T rel, T L) {  // L: the box side in this dimension
    if (!(rel >= T(0) && rel < L)) rel = (rel >= L) ? L * T(1.0 - 1e-6) : T(0);
    return rel;
}

// Window start of a point in one dimension (Section 5.2 with the P^3 block):
//   P even: floor(t) - P/2 + 1, P odd: floor(t + 1/2) - (P-1)/2, t = (x - y0)/h,
// clamped to [0, Mt - P].  Computed once, in the binning kernel, and stored
// with the sorted point so that every later kernel uses the same support.
template <typename T>
__host__ __device__ inline int window_start(T rel, const GP<T> &g, int d) {
    T t = rel * g.inv_h + g.half_ext;
    int i0 = ((g.P & 1) == 0) ? (int)floor(t) - g.P / 2 + 1 : (int)floor(t + T(0.5)) - (g.P - 1) / 2;
    return min(max(i0, 0), g.mt[d] - g.P);
}

// Grid sizes as 64-bit products
template <typename G>
__host__ __device__ inline size_t vol(const G &g) { return (size_t)g.mf[0] * g.mf[1] * g.mf[2]; }

// Three indices < 1024 packed into the spare 4th component of a sorted point.
__host__ __device__ inline int pack3(int a, int b, int c) { return a | (b << 10) | (c << 20); }
__host__ __device__ inline void unpack3(int v, int &a, int &b, int &c) {
    a = v & 1023;
    b = (v >> 10) & 1023;
    c = (v >> 20) & 1023;
}
__device__ inline void set_tag(float4 &v, int t) { v.w = __int_as_float(t); }
__device__ inline void set_tag(double4_32a &v, int t) { v.w = __longlong_as_double((long long)t); }
__device__ inline int get_tag(const float4 &v) { return __float_as_int(v.w); }
__device__ inline int get_tag(const double4_32a &v) { return (int)__double_as_longlong(v.w); }

// ---------------------------------------------------------------- the plan
struct Buffers {
    // points sorted by spreading tile
    void *xs_t = nullptr;   // N vec4<T>: x, y, z, (unused)
    void *fs_t = nullptr;   // N vec4<T>: f
    void *qs_t = nullptr;   // N vec4<T>: q (stresslet)
    int *perm_t = nullptr;  // sorted -> original
    int *cnt_t = nullptr;   // ntiles (+1) histogram, then exclusive scan (starts)
    int *slot_t = nullptr;  // N rank within tile
    int *key_t = nullptr;   // N tile id
    // points sorted by real-space cell
    void *xs_r = nullptr;
    void *fs_r = nullptr;
    void *qs_r = nullptr;
    int *perm_r = nullptr;
    void *rt = nullptr;     // N x 4 T: real-space sums at the targets (overlapped evaluation)
    int *cnt_r = nullptr;
    int *slot_r = nullptr;
    int *key_r = nullptr;
    int *tag_t = nullptr;   // N packed window starts (original order)
    int *tag_r = nullptr;   // N packed cell coordinates (original order)
    int *ncl = nullptr;     // clusters per row of cells, then their exclusive scan (+ total)
    int2 *clusters = nullptr;  // (first sorted index, count) of each real-space cluster
    void *uj = nullptr;        // real-space contributions scattered to candidates (4 values per sorted point)
    int *status = nullptr;  // device flags
};

}  // namespace se

struct se_plan_s {
    int kernel = 0;
    int prec = 0;
    int64_t N = 0;
    double x0[3] = {0, 0, 0};
    double len[3] = {1, 1, 1};  // box sides
    // method parameters
    double xi = 0, rc = 0, h = 0, eta = 0, m = 0, deltaL = 0, R = 0;
    int mm[3] = {0, 0, 0};  // M per dimension (grid points on the box)
    int mt[3] = {0, 0, 0};  // extended grid M + n_ext
    int mf[3] = {0, 0, 0};  // FFT sizes 2 mt
    int mg[3] = {0, 0, 0};  // precompute grid
    int P = 0, n_ext = 0, deltaL_policy = 0, max_fft = 0;
    // triply periodic plan: the sources are spread onto the extended grid
    // (mt = M + n_ext points, no zero padding), folded onto the periodic M^3
    // grid `pgrid` for the FFTs, and the inverse transform is unfolded back
    bool periodic = false;
    int mp = 0;               // periodic grid size M (even)
    void *pgrid = nullptr;    // nc x M^3 real (FFT input, then the C2R output)
    int nc = 3;  // spread components (3; stresslet 6)
    se::Geom geom{};
    se::GP<float> gpf{};
    se::GP<double> gpd{};
    int ntiles = 0, ncells = 0;
    bool tiled = true;  // tiled shared-memory spreading (else global atomics)
    bool colk = false;  // FP32 register-column spreading and gather (columns.cu)
    // device memory
    double *ghat64 = nullptr;  // (Mt+1)^3 octant of the precomputed kernel, FP64
    void *ghat = nullptr;      // same in the plan precision
    void *grid = nullptr;      // nc x Mf^3 real, zero padded (R2C input)
    void *spec = nullptr;      // nc x Mf x Mf x (Mf/2+1) complex
    void *wgrid = nullptr;     // 3 x Mf^3 real (C2R output)
    void *wgrid2 = nullptr;    // 3 x Mf^3 real (backward: adjoint grid)
    void *gsort = nullptr;     // N x 4 (backward: the upstream gradient in cell order)
    double cell_width = 0.0;   // se_params_t.cell_width (0: from the mean density)
    int test_flags = 0;        // se_plan_set_test_flags
    void *spec2 = nullptr;     // backward spectrum
    void *tmp3 = nullptr;      // N x 3 scratch in plan precision (backward)
    se::Buffers b;
    se::Buffers bt;          // evaluation targets (positions only), allocated on first use
    int64_t nt_cap = 0;      // targets bt holds room for
    cufftHandle fwd = 0, inv = 0, fwd3 = 0;
    // zero-padding-aware transforms (free-space plans): 2D transforms of the
    // Mtilde planes that hold data or are read, and a 1D transform along z
    bool pruned = false;
    cufftHandle f2d = 0, i2d = 0, zc = 0;
    void *zw = nullptr;  // FP32 pruned plans: twiddles of the fused z-transforms and scaling (zfft.cu)
    float *tilebuf = nullptr;  // deterministic plans: the tiles' padded blocks (atomic-free spreading)
    // se_plan_set_deterministic: stable bin order, the atomic-free spreading,
    // the full-list real-space kernel, no overlap
    bool deterministic = false;
    int *rs_scratch = nullptr;  // stable_scratch_ints(rs_cap) ints
    int64_t rs_cap = 0;
    // FP64 radial functions from exp and the erfcx fit instead of the device
    // table (the allocation-free entry point, which keeps nothing that a
    // context reset would lose)
    bool erfc_table_off = false;
    bool have_fwd = false, have_inv = false, have_fwd3 = false;
    cudaStream_t last_stream = nullptr;
    // overlapped evaluation (FP32): the Fourier part on a high-priority internal
    // stream while the real-space sum runs on the caller's stream
    bool overlap = false;
    cudaStream_t s_four = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool timing = false;
    cudaEvent_t ev[9] = {};
    cudaEvent_t ev_real = nullptr;  // recorded before the main real-space kernel when timing
    float stage_ms[8] = {};
    int n_stage = 0;
    int64_t launches = 0;  // kernels of this library launched by the last evaluation call
    // se_plan_set_keep_grid: the backward pass reuses the forward grid in wgrid
    // when its sources are the arrays (device pointers) that produced it
    bool keep_grid = false;
    bool grid_valid = false;
    const void *grid_src[3] = {nullptr, nullptr, nullptr};
    double precompute_ms = 0;
    bool precompute_cached = false;  // the precomputed kernel came from the cache
    // host staging for se_eval_host
    void *dx = nullptr, *df = nullptr, *dq = nullptr, *du = nullptr;
};

// Free a plan's device memory, cuFFT plans and events, then the plan.
void free_plan(se_plan_s *p);

namespace se {

// Parameters, grid sizes and geometry of a plan from chosen parameters (host only).
// box: x0, y0, z0, Lx, Ly, Lz
se_status_t setup_plan(se_plan_s *p, int kernel, int prec, int64_t N, const double box[6], const se_params_t &pr,
                       bool periodic = false);
// Periodic plans: fold the extended spreading grid onto the periodic grid,
// unfold the periodic grid onto the extended layout the gather reads, and
// fill the octant of the exact transforms (4 pi / k^2 or -8 pi / k^4, zero at k = 0).
template <typename T>
cudaError_t launch_fold(se_plan_s *p, cudaStream_t st, const void *ext, void *per, int nc);
template <typename T>
cudaError_t launch_unfold(se_plan_s *p, cudaStream_t st, const void *per, void *ext, int nc);
se_status_t periodic_octant(se_plan_s *p);

// launchers (defined in the .cu files); all asynchronous on `st`
template <typename T>
cudaError_t launch_bin(se_plan_s *p, const T *x, const T *f, const T *q, cudaStream_t st);
template <typename T>
cudaError_t launch_bin_set(se_plan_s *p, Buffers &b, int N, const T *x, const T *f, const T *q, cudaStream_t st);
// evaluation at separate targets: gather (no self term) and real-space sum
// with the targets binned into bt (Nt points) and the sources in the plan's set
template <typename T>
cudaError_t launch_gather_targets(se_plan_s *p, cudaStream_t st, const Buffers &bt, int Nt, const void *wgrid,
                                  T *ut);
template <typename T>
cudaError_t launch_real_targets(se_plan_s *p, cudaStream_t st, Buffers &bt, int Nt, T *ut);
template <typename T>
cudaError_t launch_spread(se_plan_s *p, cudaStream_t st, const void *xs, const void *fs, const void *qs,
                          void *grid, int nc_mode);
template <typename T>
cudaError_t launch_scale(se_plan_s *p, cudaStream_t st, void *spec, int transpose);
template <typename T>
cudaError_t launch_gather(se_plan_s *p, cudaStream_t st, const void *wgrid, const T *f_orig, T *u);
// defer: the target sums go to b.rt and nothing is added to u; launch_add_uj
// adds them (and the candidate sums b.uj) later.  Only where real_can_defer.
template <typename T>
cudaError_t launch_real(se_plan_s *p, cudaStream_t st, T *u, bool defer = false);
template <typename T>
cudaError_t launch_add_uj(se_plan_s *p, cudaStream_t st, T *u);
bool real_can_defer(const se_plan_s *p);
template <typename T>
cudaError_t launch_zero_octant(se_plan_s *p, cudaStream_t st, void *grid, int nc);
template <typename T>
cudaError_t launch_gather_grad(se_plan_s *p, cudaStream_t st, const void *w_fwd, const void *w_adj,
                               const T *f_orig, const T *q_orig, const T *g_orig, T *gx);
template <typename T>
cudaError_t launch_real_grad(se_plan_s *p, cudaStream_t st, const T *g_orig, T *gx);
// stresslet backward: adjoint scaling (3 -> 6 spectra), adjoint gather and the
// adjoint real-space sum for the strength gradients
template <typename T>
cudaError_t launch_scale_adj_stresslet(se_plan_s *p, cudaStream_t st, void *spec);
template <typename T>
cudaError_t launch_gather_adjT(se_plan_s *p, cudaStream_t st, const void *V, const T *f_orig, const T *q_orig,
                               T *gf, T *gq);
template <typename T>
cudaError_t launch_real_adjT(se_plan_s *p, cudaStream_t st, const T *f_orig, const T *q_orig, T *gf, T *gq);

// FP32 register-column spreading and gather (columns.cu): tiles of COL_TE^3
// window starts, even P in [4, 16]
constexpr int COL_TE = 8;
bool col_supported(int prec, int P);
cudaError_t launch_spread_col(se_plan_s *p, cudaStream_t st, const void *xs, const void *fs, const void *qs,
                              void *grid, int nc);
cudaError_t launch_gather_col(se_plan_s *p, cudaStream_t st, const void *wgrid, const float *f_orig, float *u);
cudaError_t launch_gather_col_set(se_plan_s *p, cudaStream_t st, const Buffers &b, const void *wgrid,
                                  const float *f_orig, double self_coef, float *u, int64_t n_pts);
// the stresslet's adjoint strength gradients from the tensor field V on the
// shared-memory tiles (FP32 column plans)
cudaError_t launch_gather_adj_col(se_plan_s *p, cudaStream_t st, const float *V, const float *f, const float *q,
                                  float *gf, float *gq);
// du/dx of the Fourier part on the shared-memory tiles (FP32 column plans)
cudaError_t launch_gather_grad_col(se_plan_s *p, cudaStream_t st, const float *w_fwd, const float *w_adj,
                                   const float *f_orig, const float *q_orig, const float *g_orig, float *gx);
// FP32 z-direction transforms fused with the scaling (zfft.cu): the fused
// kernel handles FFT lengths n whose factors are 2, 3, 5, 7 with nc source
// components; zfuse_twiddles allocates the table e^{-2 pi i t / n}
constexpr int ZF_MAXPASS = 16;
bool zfuse_supported(int n, int nc);
cudaError_t zfuse_twiddles(int n, void **out);
cudaError_t launch_zscale(const se_plan_s *p, cudaStream_t st, void *spec, int nc);

// FP32 spreading on sub-tiles of 4 x 4 x 8 window starts (subtile.cu), P = 10 or 12;
// the plan's tiles and binning are those of the column kernels
bool sub_supported(int P);
cudaError_t launch_spread_sub(const GP<float> &g, int ntiles, int c0, bool stress, const int *tile_start,
                              const float4 *xs, const float4 *fs, const float4 *qs, float *grid, cudaStream_t st);
cudaError_t launch_bspread_sub(const BSys<float> *sys, const int4 *items, int nitems, int P, int n_rhs,
                               const int *tile_start, const float4 *xs, const float4 *fs, cudaStream_t st);
// Tile buffer of the atomic-free spreading (deterministic plans): the three
// components of a tile's padded block, (8 + P - 1)^3 grid points, z-major
// planes of x rows padded to whole float4; tiles of COL_TE window starts.
template <int P>
struct TileBufCfg {
    static constexpr int PE = COL_TE + P - 1;    // grid points per edge
    static constexpr int XB = (PE + 3) / 4 * 4;  // row length
    static constexpr int NQ = XB / 4;            // float4 per row
    static constexpr size_t FLOATS = (size_t)3 * PE * PE * XB;
};

size_t tilebuf_floats(int P, int ntiles);
// Atomic-free spreading: the tile kernels store each tile's padded block in
// the tile buffer tb (k_spread_c2 with a tile buffer; on sub-tiles, P = 10 or
// 12, the four sub-tiles of a tile as one cluster of CTAs add their blocks in a
// fixed order), then launch_merge_tiles writes the corner [0, Mt)^3 of
// components c0 .. c0 + 2 of `grid` from it, adding the tiles in a fixed order
// (no zeroing needed before)
cudaError_t launch_spread_sub_tb(const GP<float> &g, int ntiles, int c0, bool stress, const int *tile_start,
                                 const float4 *xs, const float4 *fs, const float4 *qs, float *tb, cudaStream_t st);
cudaError_t launch_merge_tiles(const GP<float> &g, const int *tile_start, const float *tb, float *grid, int c0,
                               cudaStream_t st);
// FP64 real-space sums: the piecewise-polynomial table of erfc(x) and
// (2/sqrt(pi)) x exp(-x^2) on the current device (realspace.cu); call before
// the first evaluation of an FP64 plan (not during stream capture), then
// make_rc<double> selects it
cudaError_t erfc_table_init();
// Stable slots (stable.cu): slot[i] = the rank of point i among the points
// with its key and smaller indices, from the keys (< nkeys) and the bins'
// starts; scratch holds stable_scratch_ints(N) ints
size_t stable_scratch_ints(int64_t n);
cudaError_t launch_stable_slots(int N, const int *keys, int nkeys, const int *start, int *slot, int *scratch,
                                cudaStream_t st, int64_t *launches);
// true when a plan's FP32 spreading runs on the sub-tiles (columns.cu)
bool spread_uses_sub(const se_plan_s *p);
cudaError_t launch_gather_sub(const GP<float> &g, int ntiles, const int *tile_start, const float4 *xs,
                              const int *perm, const float *w, const float *f_orig, double self_coef, float *u,
                              cudaStream_t st);
cudaError_t launch_bspread_col(const BSys<float> *sys, const int4 *items, int nitems, int P, int n_rhs,
                               const Buffers &b, cudaStream_t st);
cudaError_t launch_bgather_col(const BSys<float> *sys, const int4 *items, int nitems, int P, int n_rhs,
                               const Buffers &b, const float *f, float *u, const void *maps, cudaStream_t st);
// one system's tensor map (128 bytes at `map`, 64-byte aligned) for the batched
// gather's tile copies; false when the grids do not allow one
constexpr size_t TENSOR_MAP_BYTES = 128;
bool encode_bgather_map(void *map, const GP<float> &g, const float *wgrid, size_t gzs, size_t gcs, int n_rhs, int P);

// batched launchers (one launch over all systems of a batch)
constexpr int SCALE_BS = 256;  // threads per block of the scaling kernels
ScaleConst make_scale_const(const se_plan_s *p);
template <typename T>
RC<T> make_rc(const se_plan_s *p);
template <typename T>
cudaError_t launch_bscale(int kernel, const BSys<T> *sys, const int *blk_base, int S, int nblk, int n_rhs,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_bzero(const BSys<T> *sys, const int *zblk_base, int S, int nblk, int n_rhs, cudaStream_t st);
template <typename T>
cudaError_t launch_bbin(const BSys<T> *sys, const int *off, int S, int Ntot, int n_rhs, int ntiles_tot,
                        int ncells_tot, const T *x, const T *f, Buffers &b, cudaStream_t st, int64_t *launches);
template <typename T>
cudaError_t launch_bspread(const BSys<T> *sys, const int4 *items, int nitems, int P, int T_, int n_rhs,
                           const Buffers &b, cudaStream_t st);
template <typename T>
cudaError_t launch_bgather(const BSys<T> *sys, const int *off, int S, int Ntot, int P, int n_rhs, const Buffers &b,
                           const T *f, T *u, cudaStream_t st);
template <typename T>
cudaError_t launch_breal(int kernel, const BSys<T> *sys, const int *row_base, int S, int nrows_tot, int Ntot,
                         int n_rhs, const Buffers &b, int *cl_sys, T *u, cudaStream_t st, int64_t *launches);

se_status_t precompute(se_plan_s *p);
cudaError_t launch_scan(int *cnt, int n, cudaStream_t st);
// number of kernels launch_scan issues for an array of n counts
inline int scan_launch_count(int n) { return n <= 64 * 1024 ? 1 : 3; }
template <typename T> const GP<T> &gp(const se_plan_s *p);
template <> inline const GP<float> &gp<float>(const se_plan_s *p) { return p->gpf; }
template <> inline const GP<double> &gp<double>(const se_plan_s *p) { return p->gpd; }
// Neighbour statistics of actual points for the work model: f[i] is the mean
// number of neighbours within r_i = (i + 1) dr divided by its value for
// uniformly distributed points in the same box (1 for uniform points).
struct PairFactor {
    int n = 0;
    double dr = 0.0;
    const double *f = nullptr;
    double at(double r) const;
};
se_status_t choose_params(int kernel, int prec, int64_t N, double L, double tol, const se_params_t *in,
                          double xi_arg, se_params_t *out, int n_rhs = 1, const PairFactor *pf = nullptr);
se_status_t choose_box_params(int kernel, int prec, int64_t N, const double box[6], double tol,
                              const se_params_t *params, double xi, se_params_t *out, int n_rhs = 1,
                              const PairFactor *pf = nullptr);
// the work model of the parameter selection (relative to one real-space pair)
double model_cost(int prec, int64_t N, double L, int P, int M, double rc, const PairFactor *pf, int n_rhs);
// FFT lengths measured fast with cuFFT on GB300 (and, in FP32, accurate)
bool fast_fft_len(int n, int prec);

}  // namespace se
