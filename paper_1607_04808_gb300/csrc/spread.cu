// Step 1 of Section 5.2 (spreading, eq. Hx): every source adds
//   s_n * exp(-2 xi^2 |y_i - x_n|^2 / eta)
// to the P^3 grid points of its support (the Gaussian's normalisation is
// applied later, in the scaling step).
//
// Tiled kernel: one CTA per spreading tile (T^3 window starts).  The CTA
// accumulates the padded tile ((T+P-1)^3 points, all components) in shared
// memory.  Warp w owns the padded z-planes z = w (mod 8), so warps never touch
// the same word: no shared atomics and no barriers inside the point loop.  The
// padded tile is then added to the zero-padded FFT input; neighbouring tiles
// overlap in their halos, so that flush uses global atomics.
//
// Fallback kernel (large P in FP64, where a padded tile does not fit in shared
// memory): one warp per point adding straight into the grid with atomics.
#include "se_internal.cuh"

namespace se {

namespace {

constexpr int NW = 8;  // warps per CTA in the tiled kernel
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float gexp(float v) { return expf(v); }
__device__ __forceinline__ double gexp(double v) { return exp(v); }

// Source components that are spread: f (3) or the symmetric part of f q^T
// (6: xx, yy, zz, xy, xz, yz), see the stresslet scaling.
template <typename T>
__device__ __forceinline__ void source_comps(int nc, const vec4<T> &f, const vec4<T> *qs, int n, T s[6]) {
    if (nc == 3) {
        s[0] = f.x; s[1] = f.y; s[2] = f.z;
    } else {
        vec4<T> q = qs[n];
        s[0] = f.x * q.x;
        s[1] = f.y * q.y;
        s[2] = f.z * q.z;
        s[3] = T(0.5) * (f.x * q.y + f.y * q.x);
        s[4] = T(0.5) * (f.x * q.z + f.z * q.x);
        s[5] = T(0.5) * (f.y * q.z + f.z * q.y);
    }
}

// 1-D Gaussian weights of the P points of the support along each dimension:
// lane k < P holds w_d(k) = exp(-a h^2 (t_d - i0_d - k)^2).
template <typename T>
__device__ __forceinline__ void lane_weights(const vec4<T> &xv, const Geom &g, int lane, int i0[3], T w[3]) {
    T ah2 = (T)(g.a * g.h * g.h);
    double rel[3] = {clamp_rel((double)xv.x - g.x0[0], g.L), clamp_rel((double)xv.y - g.x0[1], g.L),
                     clamp_rel((double)xv.z - g.x0[2], g.L)};
    for (int d = 0; d < 3; d++) {
        double t;
        int s = window_start(rel[d], g, t);
        s = min(max(s, 0), g.Mt - g.P);
        i0[d] = s;
        T fr = (T)(t - (double)s) - (T)lane;
        w[d] = (lane < g.P) ? gexp(-ah2 * fr * fr) : T(0);
    }
}

template <typename T>
__global__ void __launch_bounds__(NW * 32) k_spread_tile(Geom g, int nc, const int *__restrict__ tile_start,
                                                         const vec4<T> *__restrict__ xs,
                                                         const vec4<T> *__restrict__ fs,
                                                         const vec4<T> *__restrict__ qs, T *__restrict__ grid) {
    extern __shared__ unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    const int tile = blockIdx.x;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    const int P = g.P, PT = g.T + g.P - 1, PT2 = PT * PT, PT3 = PT2 * PT;
    const int tx = tile % g.ntd, ty = (tile / g.ntd) % g.ntd, tz = tile / (g.ntd * g.ntd);
    const int gx0 = tx * g.T, gy0 = ty * g.T, gz0 = tz * g.T;
    for (int e = threadIdx.x; e < nc * PT3; e += blockDim.x) sm[e] = T(0);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P2 = P * P;
    for (int n = beg; n < end; n++) {
        vec4<T> xv = xs[n];
        int i0[3];
        T w[3];
        lane_weights<T>(xv, g, lane, i0, w);
        T s[6];
        source_comps<T>(nc, fs[n], qs, n, s);
        // offsets of the support inside the padded tile (in [0, T) by construction of the bins)
        const int ox = min(max(i0[0] - gx0, 0), g.T - 1), oy = min(max(i0[1] - gy0, 0), g.T - 1),
                  oz = min(max(i0[2] - gz0, 0), g.T - 1);
        int z = oz + (((warp - oz) % NW) + NW) % NW;
        for (; z < oz + P; z += NW) {
            T wz = __shfl_sync(FULL, w[2], z - oz);
            T *plane = sm + z * PT2 + oy * PT + ox;
            for (int base = 0; base < P2; base += 32) {
                int idx = base + lane;
                int ky = idx / P, kx = idx - ky * P;
                T wx = __shfl_sync(FULL, w[0], kx);
                T wy = __shfl_sync(FULL, w[1], min(ky, P - 1));
                if (idx < P2) {
                    T wt = wx * wy * wz;
                    T *pp = plane + ky * PT + kx;
                    for (int c = 0; c < nc; c++) pp[c * PT3] += s[c] * wt;
                }
            }
        }
    }
    __syncthreads();
    const size_t Mf3 = (size_t)g.Mf * g.Mf * g.Mf;
    for (int e = threadIdx.x; e < PT3; e += blockDim.x) {
        int px = e % PT, py = (e / PT) % PT, pz = e / PT2;
        int gx = gx0 + px, gy = gy0 + py, gz = gz0 + pz;
        if (gx >= g.Mt || gy >= g.Mt || gz >= g.Mt) continue;
        size_t gi = ((size_t)gz * g.Mf + gy) * g.Mf + gx;
        for (int c = 0; c < nc; c++) {
            T v = sm[c * PT3 + e];
            if (v != T(0)) atomicAdd(grid + c * Mf3 + gi, v);
        }
    }
}

template <typename T>
__global__ void k_spread_atomic(Geom g, int nc, int N, const vec4<T> *__restrict__ xs,
                                const vec4<T> *__restrict__ fs, const vec4<T> *__restrict__ qs,
                                T *__restrict__ grid) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int n = warp, P = g.P, P2 = P * P;
    vec4<T> xv = xs[n];
    int i0[3];
    T w[3];
    lane_weights<T>(xv, g, lane, i0, w);
    T s[6];
    source_comps<T>(nc, fs[n], qs, n, s);
    const size_t Mf3 = (size_t)g.Mf * g.Mf * g.Mf;
    for (int base = 0; base < P2; base += 32) {
        int idx = base + lane;
        int ky = idx / P, kx = idx - ky * P;
        T wx = __shfl_sync(FULL, w[0], kx);
        T wy = __shfl_sync(FULL, w[1], min(ky, P - 1));
        for (int kz = 0; kz < P; kz++) {
            T wz = __shfl_sync(FULL, w[2], kz);
            if (idx < P2) {
                T wt = wx * wy * wz;
                size_t gi = ((size_t)(i0[2] + kz) * g.Mf + (i0[1] + ky)) * g.Mf + (i0[0] + kx);
                for (int c = 0; c < nc; c++) atomicAdd(grid + c * Mf3 + gi, s[c] * wt);
            }
        }
    }
}

template <typename T>
__global__ void k_zero_octant(T *__restrict__ grid, int Mt, int Mf, int nc) {
    // one thread per (c, z, y) row of Mt values
    size_t row = (size_t)blockIdx.x * blockDim.y + threadIdx.y;
    size_t nrows = (size_t)nc * Mt * Mt;
    if (row >= nrows) return;
    int y = row % Mt, z = (row / Mt) % Mt, c = row / ((size_t)Mt * Mt);
    T *p = grid + (size_t)c * Mf * Mf * Mf + ((size_t)z * Mf + y) * Mf;
    for (int x = threadIdx.x; x < Mt; x += blockDim.x) p[x] = T(0);
}

}  // namespace

size_t spread_smem_bytes(const se_plan_s *p, int nc, size_t elem) {
    size_t PT = p->geom.T + p->P - 1;
    return (size_t)nc * PT * PT * PT * elem;
}

template <typename T>
cudaError_t launch_zero_octant(se_plan_s *p, cudaStream_t st, void *grid, int nc) {
    dim3 bs(32, 8);
    size_t nrows = (size_t)nc * p->Mt * p->Mt;
    dim3 gs((unsigned)((nrows + bs.y - 1) / bs.y));
    k_zero_octant<T><<<gs, bs, 0, st>>>((T *)grid, p->Mt, p->Mf, nc);
    return cudaGetLastError();
}

// nc_mode: number of spread components (3, or 6 for the stresslet source f q^T)
template <typename T>
cudaError_t launch_spread(se_plan_s *p, cudaStream_t st, const void *xs, const void *fs, const void *qs,
                          void *grid, int nc) {
    cudaError_t e;
    if ((e = launch_zero_octant<T>(p, st, grid, nc))) return e;
    size_t smem = spread_smem_bytes(p, nc, sizeof(T));
    if (p->tiled && smem <= 200 * 1024) {
        if ((e = cudaFuncSetAttribute(k_spread_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        k_spread_tile<T><<<p->ntiles, NW * 32, smem, st>>>(p->geom, nc, p->b.cnt_t, (const vec4<T> *)xs,
                                                          (const vec4<T> *)fs, (const vec4<T> *)qs, (T *)grid);
    } else {
        int N = (int)p->N;
        int wpb = 8;
        k_spread_atomic<T><<<(N + wpb - 1) / wpb, wpb * 32, 0, st>>>(p->geom, nc, N, (const vec4<T> *)xs,
                                                                    (const vec4<T> *)fs, (const vec4<T> *)qs,
                                                                    (T *)grid);
    }
    return cudaGetLastError();
}

template cudaError_t launch_spread<float>(se_plan_s *, cudaStream_t, const void *, const void *, const void *,
                                          void *, int);
template cudaError_t launch_spread<double>(se_plan_s *, cudaStream_t, const void *, const void *, const void *,
                                           void *, int);
template cudaError_t launch_zero_octant<float>(se_plan_s *, cudaStream_t, void *, int);
template cudaError_t launch_zero_octant<double>(se_plan_s *, cudaStream_t, void *, int);

}  // namespace se
