// Step 1 of Section 5.2 (spreading, eq. Hx): every source adds
//   s_n * exp(-2 xi^2 |y_i - x_n|^2 / eta)
// to the P^3 grid points of its support (the Gaussian's normalisation is
// applied later, in the scaling step).  The Gaussian is separable, so each
// point needs 3P exponentials (one 1-D weight vector per dimension).
//
// Tiled kernel: one CTA per spreading tile (T^3 window starts), 8 warps.  The
// CTA accumulates the padded tile ((T+P-1)^3 points, all components) in shared
// memory.  Points are taken 32 at a time: their weights, sources and support
// offsets are staged in shared memory once per CTA, then every warp adds the
// batch into the padded z-planes it owns (z = w mod 8), so no two warps ever
// touch the same word and no shared atomics are needed.  The padded tile is
// finally added to the zero-padded FFT input; neighbouring tiles overlap in
// their halos, so that flush uses global atomics.
//
// Fallback kernel (P > 16, or a padded tile that does not fit in shared
// memory, e.g. the FP64 path at P >= 20): one warp per point adding straight
// into the grid with global atomics.
#include "se_internal.cuh"

namespace se {

namespace {

constexpr int NW = 8;   // warps per CTA in the tiled kernel
constexpr int NB = 32;  // points staged per batch

__device__ __forceinline__ float gexp(float v) { return __expf(v); }
__device__ __forceinline__ double gexp(double v) { return exp(v); }

// Source components that are spread: f (3) or the symmetric part of f q^T
// (6: xx, yy, zz, xy, xz, yz), see the stresslet scaling.
template <typename T>
__device__ __forceinline__ T source_comp(int c, const vec4<T> &f) {
    return c == 0 ? f.x : (c == 1 ? f.y : f.z);
}
template <typename T>
__device__ __forceinline__ T stress_comp(int c, const vec4<T> &f, const vec4<T> &q) {
    switch (c) {
        case 0: return f.x * q.x;
        case 1: return f.y * q.y;
        case 2: return f.z * q.z;
        case 3: return T(0.5) * (f.x * q.y + f.y * q.x);
        case 4: return T(0.5) * (f.x * q.z + f.z * q.x);
        default: return T(0.5) * (f.y * q.z + f.z * q.y);
    }
}

// 1-D weight of support point k along one dimension: exp(-a h^2 (t - i0 - k)^2)
template <typename T>
__device__ __forceinline__ T weight(T rel, int i0, int k, const GP<T> &g) {
    T fr = (rel * g.inv_h + g.half_ext) - (T)(i0 + k);
    return gexp(-g.ah2 * fr * fr);
}

// The CTA's work on one spreading tile: sorted points [beg, end) (sources
// fs[n * fstride + foff]) into the padded tile, then into grid.
template <typename T, int NIT>
__device__ __forceinline__ void spread_tile_body(const GP<T> &g, int tile, int beg, int end, int nc,
                                                 const vec4<T> *__restrict__ xs, const vec4<T> *__restrict__ fs,
                                                 int fstride, int foff, const vec4<T> *__restrict__ qs,
                                                 T *__restrict__ grid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T sw[NB][3][32];
    __shared__ T ssrc[NB][6];
    __shared__ int soff[NB];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int P = g.P, PT = g.T_ + P - 1, PT2 = PT * PT, PT3 = PT2 * PT;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int gx0 = tx * g.T_, gy0 = ty * g.T_, gz0 = tz * g.T_;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this lane's (kx, ky) positions of the P x P support plane
    int kxs[NIT], kys[NIT], offs[NIT];
    bool val[NIT];
#pragma unroll
    for (int it = 0; it < NIT; it++) {
        int idx = it * 32 + lane;
        val[it] = idx < P * P;
        kys[it] = val[it] ? idx / P : 0;
        kxs[it] = val[it] ? idx - kys[it] * P : 0;
        offs[it] = kys[it] * PT + kxs[it];
    }
    for (int e = threadIdx.x; e < nc * PT3; e += blockDim.x) sm[e] = T(0);
    for (int b0 = beg; b0 < end; b0 += NB) {
        const int nb = min(NB, end - b0);
        __syncthreads();  // previous batch consumed (and the zeroing finished)
        // stage the batch: warp w prepares points w, w + 8, ...
        for (int j = warp; j < nb; j += NW) {
            const int n = b0 + j;
            const vec4<T> xv = xs[n];
            int i0[3];
            unpack3(get_tag(xv), i0[0], i0[1], i0[2]);
            if (lane < P) {
                sw[j][0][lane] = weight(xv.x - g.x0[0], i0[0], lane, g);
                sw[j][1][lane] = weight(xv.y - g.x0[1], i0[1], lane, g);
                sw[j][2][lane] = weight(xv.z - g.x0[2], i0[2], lane, g);
            }
            if (lane < nc) {
                const vec4<T> fv = fs[(size_t)n * fstride + foff];
                ssrc[j][lane] = (nc == 6) ? stress_comp<T>(lane, fv, qs[n]) : source_comp<T>(lane, fv);
            }
            if (lane == 0) {
                int ox = min(max(i0[0] - gx0, 0), g.T_ - 1), oy = min(max(i0[1] - gy0, 0), g.T_ - 1),
                    oz = min(max(i0[2] - gz0, 0), g.T_ - 1);
                soff[j] = pack3(ox, oy, oz);
            }
        }
        __syncthreads();
        for (int j = 0; j < nb; j++) {
            int ox, oy, oz;
            unpack3(soff[j], ox, oy, oz);
            T wxy[NIT];
#pragma unroll
            for (int it = 0; it < NIT; it++) wxy[it] = sw[j][0][kxs[it]] * sw[j][1][kys[it]];
            T s[6];
#pragma unroll
            for (int c = 0; c < 6; c++) s[c] = (c < nc) ? ssrc[j][c] : T(0);
            int z = oz + (((warp - oz) % NW) + NW) % NW;
            for (; z < oz + P; z += NW) {
                const T wz = sw[j][2][z - oz];
                T *plane = sm + z * PT2 + oy * PT + ox;
#pragma unroll
                for (int it = 0; it < NIT; it++) {
                    if (val[it]) {
                        const T wt = wxy[it] * wz;
                        T *pp = plane + offs[it];
                        pp[0] += s[0] * wt;
                        pp[PT3] += s[1] * wt;
                        pp[2 * PT3] += s[2] * wt;
                        if (nc == 6) {
                            pp[3 * PT3] += s[3] * wt;
                            pp[4 * PT3] += s[4] * wt;
                            pp[5 * PT3] += s[5] * wt;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    const size_t Mf3 = vol(g);
    for (int e = threadIdx.x; e < PT3; e += blockDim.x) {
        int px = e % PT, py = (e / PT) % PT, pz = e / PT2;
        int gx = gx0 + px, gy = gy0 + py, gz = gz0 + pz;
        if (gx >= g.mt[0] || gy >= g.mt[1] || gz >= g.mt[2]) continue;
        size_t gi = ((size_t)gz * g.mf[1] + gy) * g.mf[0] + gx;
        for (int c = 0; c < nc; c++) {
            T v = sm[c * PT3 + e];
            if (v != T(0)) atomicAdd(grid + c * Mf3 + gi, v);
        }
    }
}

template <typename T, int NIT>
__global__ void __launch_bounds__(NW * 32) k_spread_tile(GP<T> g, int nc, const int *__restrict__ tile_start,
                                                         const vec4<T> *__restrict__ xs,
                                                         const vec4<T> *__restrict__ fs,
                                                         const vec4<T> *__restrict__ qs, T *__restrict__ grid) {
    const int tile = blockIdx.x;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    spread_tile_body<T, NIT>(g, tile, beg, end, nc, xs, fs, 1, 0, qs, grid);
}

// Batched: one CTA per item (system, tile of that system, right-hand side);
// the tile's points are the system's, their sources the item's right-hand
// side, and the grid that right-hand side's three components.
template <typename T, int NIT>
__global__ void __launch_bounds__(NW * 32) k_bspread_tile(const BSys<T> *__restrict__ sys,
                                                          const int4 *__restrict__ items,
                                                          const int *__restrict__ tile_start, int n_rhs,
                                                          const vec4<T> *__restrict__ xs,
                                                          const vec4<T> *__restrict__ fs) {
    const int4 it = items[blockIdx.x];  // (system, local tile, right-hand side, -)
    const BSys<T> &B = sys[it.x];
    const int key = B.tile_base + it.y;
    const int beg = tile_start[key], end = tile_start[key + 1];
    if (beg == end) return;
    const GP<T> g = B.g;
    const size_t Mf3 = vol(g);
    spread_tile_body<T, NIT>(g, it.y, beg, end, 3, xs, fs, n_rhs, it.z, nullptr, B.grid + (size_t)it.z * 3 * Mf3);
}

template <typename T>
__global__ void k_spread_atomic(GP<T> g, int nc, int N, const vec4<T> *__restrict__ xs,
                                const vec4<T> *__restrict__ fs, const vec4<T> *__restrict__ qs,
                                T *__restrict__ grid) {
    __shared__ T sw_all[8][3][32];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = blockIdx.x * 8 + wib;
    if (n >= N) return;
    T(*sw)[32] = sw_all[wib];
    const int P = g.P, P2 = P * P;
    const vec4<T> xv = xs[n];
    int i0[3];
    unpack3(get_tag(xv), i0[0], i0[1], i0[2]);
    if (lane < P) {
        sw[0][lane] = weight(xv.x - g.x0[0], i0[0], lane, g);
        sw[1][lane] = weight(xv.y - g.x0[1], i0[1], lane, g);
        sw[2][lane] = weight(xv.z - g.x0[2], i0[2], lane, g);
    }
    __syncwarp();
    const vec4<T> fv = fs[n];
    T s[6];
    for (int c = 0; c < nc; c++) s[c] = (nc == 6) ? stress_comp<T>(c, fv, qs[n]) : source_comp<T>(c, fv);
    const size_t Mfx = g.mf[0], Mf2 = Mfx * g.mf[1], Mf3 = vol(g);
    for (int idx = lane; idx < P2; idx += 32) {
        int ky = idx / P, kx = idx - ky * P;
        const T wxy = sw[0][kx] * sw[1][ky];
        const size_t base = ((size_t)i0[2] * g.mf[1] + (i0[1] + ky)) * Mfx + (i0[0] + kx);
        for (int kz = 0; kz < P; kz++) {
            const T wt = wxy * sw[2][kz];
            for (int c = 0; c < nc; c++) atomicAdd(grid + c * Mf3 + base + kz * Mf2, s[c] * wt);
        }
    }
}

// Zero the mt_x x mt_y x mt_z corner of nc grids (one warp-row per (c, z, y)
// row of mt_x values); the rest of the padded grids stays zero.
template <typename T>
__device__ __forceinline__ void zero_rows(T *__restrict__ grid, const int mt[3], const int mf[3], size_t row) {
    const int y = row % mt[1], z = (row / mt[1]) % mt[2];
    const size_t c = row / ((size_t)mt[1] * mt[2]);
    T *p = grid + c * mf[0] * mf[1] * mf[2] + ((size_t)z * mf[1] + y) * mf[0];
    for (int x = threadIdx.x; x < mt[0]; x += blockDim.x) p[x] = T(0);
}

template <typename T>
__global__ void k_zero_octant(T *__restrict__ grid, GP<T> g, int nc) {
    size_t row = (size_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (row >= (size_t)nc * g.mt[1] * g.mt[2]) return;
    zero_rows(grid, g.mt, g.mf, row);
}

// Batched: zero the octant of every grid of every system (rows of Mt values;
// block b belongs to the system s with zblk_base[s] <= b < zblk_base[s+1]).
template <typename T>
__global__ void k_bzero_octant(const BSys<T> *__restrict__ sys, const int *__restrict__ zblk_base, int S,
                               int n_rhs) {
    const int s = find_range(zblk_base, S, (int)blockIdx.x);
    const BSys<T> &B = sys[s];
    const size_t row = (size_t)(blockIdx.x - zblk_base[s]) * blockDim.y + threadIdx.y;
    if (row >= (size_t)3 * n_rhs * B.g.mt[1] * B.g.mt[2]) return;
    const int y = row % B.g.mt[1], z = (row / B.g.mt[1]) % B.g.mt[2];
    const size_t c = row / ((size_t)B.g.mt[1] * B.g.mt[2]);
    T *p = B.grid + c * B.gcs + z * B.gzs + (size_t)y * B.g.mf[0];
    for (int x = threadIdx.x; x < B.g.mt[0]; x += blockDim.x) p[x] = T(0);
}

template <typename T, int NIT>
cudaError_t launch_tile(se_plan_s *p, cudaStream_t st, size_t smem, int nc, const void *xs, const void *fs,
                        const void *qs, void *grid) {
    cudaError_t e = cudaFuncSetAttribute(k_spread_tile<T, NIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    k_spread_tile<T, NIT><<<p->ntiles, NW * 32, smem, st>>>(gp<T>(p), nc, p->b.cnt_t, (const vec4<T> *)xs,
                                                            (const vec4<T> *)fs, (const vec4<T> *)qs, (T *)grid);
    p->launches++;
    return cudaGetLastError();
}

}  // namespace

size_t spread_smem_bytes(const se_plan_s *p, int nc, size_t elem) {
    size_t PT = p->geom.T + p->P - 1;
    return (size_t)nc * PT * PT * PT * elem;
}

template <typename T>
cudaError_t launch_zero_octant(se_plan_s *p, cudaStream_t st, void *grid, int nc) {
    dim3 bs(32, 8);
    size_t nrows = (size_t)nc * p->mt[1] * p->mt[2];
    dim3 gs((unsigned)((nrows + bs.y - 1) / bs.y));
    k_zero_octant<T><<<gs, bs, 0, st>>>((T *)grid, gp<T>(p), nc);
    p->launches++;
    return cudaGetLastError();
}

// nc: number of spread components (3, or 6 for the stresslet source f q^T)
template <typename T>
cudaError_t launch_spread(se_plan_s *p, cudaStream_t st, const void *xs, const void *fs, const void *qs,
                          void *grid, int nc) {
    cudaError_t e;
    if (sizeof(T) == 4 && p->colk && p->deterministic && p->tilebuf)  // writes the whole corner
        return launch_spread_col(p, st, xs, fs, qs, grid, nc);
    if ((e = launch_zero_octant<T>(p, st, grid, nc))) return e;
    if (sizeof(T) == 4 && p->colk) return launch_spread_col(p, st, xs, fs, qs, grid, nc);
    size_t smem = spread_smem_bytes(p, nc, sizeof(T));
    const int nit = (p->P * p->P + 31) / 32;
    if (p->tiled && p->P <= 16 && smem <= 190 * 1024) {
        switch (nit) {
            case 1: return launch_tile<T, 1>(p, st, smem, nc, xs, fs, qs, grid);
            case 2: return launch_tile<T, 2>(p, st, smem, nc, xs, fs, qs, grid);
            case 3: return launch_tile<T, 3>(p, st, smem, nc, xs, fs, qs, grid);
            case 4: return launch_tile<T, 4>(p, st, smem, nc, xs, fs, qs, grid);
            case 5: return launch_tile<T, 5>(p, st, smem, nc, xs, fs, qs, grid);
            case 6: return launch_tile<T, 6>(p, st, smem, nc, xs, fs, qs, grid);
            case 7: return launch_tile<T, 7>(p, st, smem, nc, xs, fs, qs, grid);
            default: return launch_tile<T, 8>(p, st, smem, nc, xs, fs, qs, grid);
        }
    }
    int N = (int)p->N;
    k_spread_atomic<T><<<(N + 7) / 8, 256, 0, st>>>(gp<T>(p), nc, N, (const vec4<T> *)xs, (const vec4<T> *)fs,
                                                   (const vec4<T> *)qs, (T *)grid);
    p->launches++;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bzero(const BSys<T> *sys, const int *zblk_base, int S, int nblk, int n_rhs, cudaStream_t st) {
    k_bzero_octant<T><<<nblk, dim3(32, 8), 0, st>>>(sys, zblk_base, S, n_rhs);
    return cudaGetLastError();
}

template <typename T, int NIT>
static cudaError_t bspread_nit(const BSys<T> *sys, const int4 *items, int nitems, size_t smem, int n_rhs,
                               const Buffers &b, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_bspread_tile<T, NIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e) return e;
    k_bspread_tile<T, NIT><<<nitems, NW * 32, smem, st>>>(sys, items, b.cnt_t, n_rhs, (const vec4<T> *)b.xs_t,
                                                          (const vec4<T> *)b.fs_t);
    return cudaGetLastError();
}

// Batched spreading: P and the tile edge T_ are common to all systems.
template <typename T>
cudaError_t launch_bspread(const BSys<T> *sys, const int4 *items, int nitems, int P, int T_, int n_rhs,
                           const Buffers &b, cudaStream_t st) {
    const size_t PT = T_ + P - 1;
    const size_t smem = 3 * PT * PT * PT * sizeof(T);
    if (P > 16 || smem > 190 * 1024) return cudaErrorInvalidValue;
    switch ((P * P + 31) / 32) {
        case 1: return bspread_nit<T, 1>(sys, items, nitems, smem, n_rhs, b, st);
        case 2: return bspread_nit<T, 2>(sys, items, nitems, smem, n_rhs, b, st);
        case 3: return bspread_nit<T, 3>(sys, items, nitems, smem, n_rhs, b, st);
        case 4: return bspread_nit<T, 4>(sys, items, nitems, smem, n_rhs, b, st);
        case 5: return bspread_nit<T, 5>(sys, items, nitems, smem, n_rhs, b, st);
        case 6: return bspread_nit<T, 6>(sys, items, nitems, smem, n_rhs, b, st);
        case 7: return bspread_nit<T, 7>(sys, items, nitems, smem, n_rhs, b, st);
        default: return bspread_nit<T, 8>(sys, items, nitems, smem, n_rhs, b, st);
    }
}

template cudaError_t launch_bzero<float>(const BSys<float> *, const int *, int, int, int, cudaStream_t);
template cudaError_t launch_bzero<double>(const BSys<double> *, const int *, int, int, int, cudaStream_t);
template cudaError_t launch_bspread<float>(const BSys<float> *, const int4 *, int, int, int, int, const Buffers &,
                                           cudaStream_t);
template cudaError_t launch_bspread<double>(const BSys<double> *, const int4 *, int, int, int, int, const Buffers &,
                                            cudaStream_t);
template cudaError_t launch_spread<float>(se_plan_s *, cudaStream_t, const void *, const void *, const void *,
                                          void *, int);
template cudaError_t launch_spread<double>(se_plan_s *, cudaStream_t, const void *, const void *, const void *,
                                           void *, int);
template cudaError_t launch_zero_octant<float>(se_plan_s *, cudaStream_t, void *, int);
template cudaError_t launch_zero_octant<double>(se_plan_s *, cudaStream_t, void *, int);

}  // namespace se
