// Point binning (counting sort) for the spreading tiles and the real-space
// cells.  Section 6 (cell list) and Section 5.2 (points grouped by the grid
// block their Gaussian support starts in).  The window start of every point
// and its cell are computed here once and stored with the sorted copies.
#include "se_internal.cuh"

namespace se {

namespace {

// Window starts and real-space cell of a point; true when it lies outside the
// half-open box (it is then clamped inside so that all indexing stays in
// bounds; NaN fails both tests).
template <typename T>
__device__ __forceinline__ bool place_point(const GP<T> &g, const T *xp, int i0[3], int cc[3]) {
    bool oob = false;
    for (int d = 0; d < 3; d++) {
        T rel = xp[d] - g.x0[d];
        if (!(rel >= T(0) && rel < g.len[d])) oob = true;
        rel = clamp_rel(rel, g.len[d]);
        i0[d] = window_start(rel, g, d);
        cc[d] = min(max((int)(rel * g.icw[d]), 0), g.ncel[d] - 1);
    }
    return oob;
}

// Spreading tile of a window start (tiles of T_^3 window starts, x fastest)
template <typename T>
__device__ __forceinline__ int tile_key(const GP<T> &g, const int i0[3]) {
    const int t0 = min(i0[0] / g.T_, g.nt[0] - 1), t1 = min(i0[1] / g.T_, g.nt[1] - 1),
              t2 = min(i0[2] / g.T_, g.nt[2] - 1);
    return (t2 * g.nt[1] + t1) * g.nt[0] + t0;
}

template <typename T>
__global__ void k_bin_count(int N, const T *__restrict__ x, GP<T> g, int *__restrict__ cnt_t,
                            int *__restrict__ slot_t, int *__restrict__ key_t, int *__restrict__ cnt_r,
                            int *__restrict__ slot_r, int *__restrict__ key_r, int *__restrict__ tag_t,
                            int *__restrict__ tag_r, int *__restrict__ status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int i0[3], cc[3];
    if (place_point(g, x + 3 * (size_t)i, i0, cc)) atomicOr(status, FLAG_OOB);
    int kt = tile_key(g, i0);
    int kr = (cc[2] * g.ncel[1] + cc[1]) * g.ncel[0] + cc[0];
    key_t[i] = kt;
    key_r[i] = kr;
    tag_t[i] = pack3(i0[0], i0[1], i0[2]);
    tag_r[i] = pack3(cc[0], cc[1], cc[2]);
    slot_t[i] = atomicAdd(&cnt_t[kt], 1);
    slot_r[i] = atomicAdd(&cnt_r[kr], 1);
}

// Exclusive scan of cnt[0..n) in place, cnt[n] = total.  One block of 1024
// threads; each thread scans a contiguous chunk.
__global__ void k_scan_exclusive(int *cnt, int n) {
    __shared__ int part[1024];
    int tid = threadIdx.x;
    int chunk = (n + blockDim.x - 1) / blockDim.x;
    int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
    int s = 0;
    for (int i = lo; i < hi; i++) s += cnt[i];
    part[tid] = s;
    __syncthreads();
    // Hillis-Steele inclusive scan of the per-thread sums
    for (int off = 1; off < blockDim.x; off <<= 1) {
        int v = (tid >= off) ? part[tid - off] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = part[tid] - s;  // exclusive prefix of this chunk
    for (int i = lo; i < hi; i++) {
        int c = cnt[i];
        cnt[i] = run;
        run += c;
    }
    if (tid == blockDim.x - 1) cnt[n] = part[tid];
}

template <typename T>
__global__ void k_bin_scatter(int N, const T *__restrict__ x, const T *__restrict__ f, const T *__restrict__ q,
                              const int *__restrict__ start_t, const int *__restrict__ slot_t,
                              const int *__restrict__ key_t, const int *__restrict__ start_r,
                              const int *__restrict__ slot_r, const int *__restrict__ key_r,
                              const int *__restrict__ tag_t, const int *__restrict__ tag_r,
                              vec4<T> *__restrict__ xs_t, vec4<T> *__restrict__ fs_t, vec4<T> *__restrict__ qs_t,
                              int *__restrict__ perm_t, vec4<T> *__restrict__ xs_r, vec4<T> *__restrict__ fs_r,
                              vec4<T> *__restrict__ qs_r, int *__restrict__ perm_r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    vec4<T> xv, fv, qv;
    xv.x = x[3 * i]; xv.y = x[3 * i + 1]; xv.z = x[3 * i + 2];
    if (f) { fv.x = f[3 * i]; fv.y = f[3 * i + 1]; fv.z = f[3 * i + 2]; fv.w = 0; }
    if (q) { qv.x = q[3 * i]; qv.y = q[3 * i + 1]; qv.z = q[3 * i + 2]; qv.w = 0; }
    int pt = start_t[key_t[i]] + slot_t[i];
    int pr = start_r[key_r[i]] + slot_r[i];
    vec4<T> xr = xv;
    set_tag(xv, tag_t[i]);
    set_tag(xr, tag_r[i]);
    xs_t[pt] = xv; perm_t[pt] = i;
    xs_r[pr] = xr; perm_r[pr] = i;
    if (f) { fs_t[pt] = fv; fs_r[pr] = fv; }
    if (q) { qs_t[pt] = qv; qs_r[pr] = qv; }
}

// Batched: the point's system is the range of `off` holding its index; its
// keys are offset by the system's first tile and first cell, so one counting
// sort orders the points by system, then by tile (or cell).
template <typename T>
__global__ void k_bbin_count(int Ntot, const BSys<T> *__restrict__ sys, const int *__restrict__ off, int S,
                             const T *__restrict__ x, int *__restrict__ cnt_t, int *__restrict__ slot_t,
                             int *__restrict__ key_t, int *__restrict__ cnt_r, int *__restrict__ slot_r,
                             int *__restrict__ key_r, int *__restrict__ tag_t, int *__restrict__ tag_r,
                             int *__restrict__ status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ntot) return;
    const BSys<T> &B = sys[find_range(off, S, i)];
    const GP<T> g = B.g;
    int i0[3], cc[3];
    if (place_point(g, x + 3 * (size_t)i, i0, cc)) atomicOr(status, FLAG_OOB);
    int kt = B.tile_base + tile_key(g, i0);
    int kr = B.cell_base + (cc[2] * g.ncel[1] + cc[1]) * g.ncel[0] + cc[0];
    key_t[i] = kt;
    key_r[i] = kr;
    tag_t[i] = pack3(i0[0], i0[1], i0[2]);
    tag_r[i] = pack3(cc[0], cc[1], cc[2]);
    slot_t[i] = atomicAdd(&cnt_t[kt], 1);
    slot_r[i] = atomicAdd(&cnt_r[kr], 1);
}

// Batched scatter: n_rhs source three-vectors per point, stored as n_rhs
// consecutive 4-vectors of the sorted point.
template <typename T>
__global__ void k_bbin_scatter(int Ntot, int n_rhs, const T *__restrict__ x, const T *__restrict__ f,
                               const int *__restrict__ start_t, const int *__restrict__ slot_t,
                               const int *__restrict__ key_t, const int *__restrict__ start_r,
                               const int *__restrict__ slot_r, const int *__restrict__ key_r,
                               const int *__restrict__ tag_t, const int *__restrict__ tag_r,
                               vec4<T> *__restrict__ xs_t, vec4<T> *__restrict__ fs_t, int *__restrict__ perm_t,
                               vec4<T> *__restrict__ xs_r, vec4<T> *__restrict__ fs_r, int *__restrict__ perm_r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Ntot) return;
    vec4<T> xv;
    xv.x = x[3 * (size_t)i]; xv.y = x[3 * (size_t)i + 1]; xv.z = x[3 * (size_t)i + 2];
    const int pt = start_t[key_t[i]] + slot_t[i];
    const int pr = start_r[key_r[i]] + slot_r[i];
    vec4<T> xr = xv;
    set_tag(xv, tag_t[i]);
    set_tag(xr, tag_r[i]);
    xs_t[pt] = xv; perm_t[pt] = i;
    xs_r[pr] = xr; perm_r[pr] = i;
    for (int r = 0; r < n_rhs; r++) {
        const T *fr = f + ((size_t)i * n_rhs + r) * 3;
        vec4<T> fv;
        fv.x = fr[0]; fv.y = fr[1]; fv.z = fr[2]; fv.w = 0;
        fs_t[(size_t)pt * n_rhs + r] = fv;
        fs_r[(size_t)pr * n_rhs + r] = fv;
    }
}

}  // namespace

template <typename T>
cudaError_t launch_bbin(const BSys<T> *sys, const int *off, int S, int Ntot, int n_rhs, int ntiles_tot,
                        int ncells_tot, const T *x, const T *f, Buffers &b, cudaStream_t st, int64_t *launches) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.cnt_t, 0, sizeof(int) * (ntiles_tot + 1), st))) return e;
    if ((e = cudaMemsetAsync(b.cnt_r, 0, sizeof(int) * (ncells_tot + 1), st))) return e;
    const int bs = 256, gs = (Ntot + bs - 1) / bs;
    k_bbin_count<T><<<gs, bs, 0, st>>>(Ntot, sys, off, S, x, b.cnt_t, b.slot_t, b.key_t, b.cnt_r, b.slot_r, b.key_r,
                                       b.tag_t, b.tag_r, b.status);
    if ((e = launch_scan(b.cnt_t, ntiles_tot, st))) return e;
    if ((e = launch_scan(b.cnt_r, ncells_tot, st))) return e;
    k_bbin_scatter<T><<<gs, bs, 0, st>>>(Ntot, n_rhs, x, f, b.cnt_t, b.slot_t, b.key_t, b.cnt_r, b.slot_r, b.key_r,
                                         b.tag_t, b.tag_r, (vec4<T> *)b.xs_t, (vec4<T> *)b.fs_t, b.perm_t,
                                         (vec4<T> *)b.xs_r, (vec4<T> *)b.fs_r, b.perm_r);
    *launches += 2 + scan_launch_count(ntiles_tot) + scan_launch_count(ncells_tot);
    return cudaGetLastError();
}

template cudaError_t launch_bbin<float>(const BSys<float> *, const int *, int, int, int, int, int, const float *,
                                        const float *, Buffers &, cudaStream_t, int64_t *);
template cudaError_t launch_bbin<double>(const BSys<double> *, const int *, int, int, int, int, int, const double *,
                                         const double *, Buffers &, cudaStream_t, int64_t *);

template <typename T>
cudaError_t launch_bin(se_plan_s *p, const T *x, const T *f, const T *q, cudaStream_t st) {
    return launch_bin_set<T>(p, p->b, (int)p->N, x, f, q, st);
}

// Bin N points into the buffer set b with the plan's tiles and cells (f and q
// may be NULL: positions only, e.g. evaluation targets).
template <typename T>
cudaError_t launch_bin_set(se_plan_s *p, Buffers &b, int N, const T *x, const T *f, const T *q, cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.cnt_t, 0, sizeof(int) * (p->ntiles + 1), st))) return e;
    if ((e = cudaMemsetAsync(b.cnt_r, 0, sizeof(int) * (p->ncells + 1), st))) return e;
    int bs = 256, gs = (N + bs - 1) / bs;
    k_bin_count<T><<<gs, bs, 0, st>>>(N, x, gp<T>(p), b.cnt_t, b.slot_t, b.key_t, b.cnt_r, b.slot_r, b.key_r,
                                      b.tag_t, b.tag_r, b.status);
    if ((e = launch_scan(b.cnt_t, (int)p->ntiles, st))) return e;
    if ((e = launch_scan(b.cnt_r, (int)p->ncells, st))) return e;
    p->launches += 2 + scan_launch_count((int)p->ntiles) + scan_launch_count((int)p->ncells);
    if (p->deterministic) {
        // slots by index within each bin instead of the atomic counters' order
        if (N > p->rs_cap || !p->rs_scratch) return cudaErrorInvalidValue;
        if ((e = launch_stable_slots(N, b.key_t, (int)p->ntiles, b.cnt_t, b.slot_t, p->rs_scratch, st,
                                     &p->launches)))
            return e;
        if ((e = launch_stable_slots(N, b.key_r, (int)p->ncells, b.cnt_r, b.slot_r, p->rs_scratch, st,
                                     &p->launches)))
            return e;
    }
    k_bin_scatter<T><<<gs, bs, 0, st>>>(N, x, f, q, b.cnt_t, b.slot_t, b.key_t, b.cnt_r, b.slot_r, b.key_r, b.tag_t,
                                        b.tag_r, (vec4<T> *)b.xs_t, (vec4<T> *)b.fs_t, (vec4<T> *)b.qs_t, b.perm_t,
                                        (vec4<T> *)b.xs_r, (vec4<T> *)b.fs_r, (vec4<T> *)b.qs_r, b.perm_r);
    return cudaGetLastError();
}

// Three-pass exclusive scan for long arrays: per-block sums of contiguous
// tiles, a scan of the block sums, then each block scans its tile from its
// offset (block-wide scan in shared memory, coalesced loads and stores).
constexpr int SCAN_TILE = 4096;

__global__ void k_scan_tile_sums(const int *__restrict__ cnt, int n, int *__restrict__ sums) {
    __shared__ int red[32];
    const int b = blockIdx.x, lo = b * SCAN_TILE, hi = min(n, lo + SCAN_TILE);
    int s = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) s += cnt[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sums[b] = v;
    }
}

__global__ void k_scan_tiles(int *cnt, int n, const int *__restrict__ offs) {
    __shared__ int wsum[32];
    const int b = blockIdx.x, lo = b * SCAN_TILE;
    const int per = SCAN_TILE / blockDim.x;  // contiguous elements per thread
    const int i0 = lo + threadIdx.x * per;
    int v[SCAN_TILE / 1024 > 0 ? SCAN_TILE / 1024 : 1];
    int s = 0;
    for (int k = 0; k < per; k++) {
        const int i = i0 + k;
        v[k] = (i < n) ? cnt[i] : 0;
        s += v[k];
    }
    // block-wide exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = (lane < (blockDim.x >> 5)) ? wsum[lane] : 0;
        int xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        wsum[lane] = xi - x;
    }
    __syncthreads();
    int run = offs[b] + wsum[w] + incl - s;
    for (int k = 0; k < per; k++) {
        const int i = i0 + k;
        if (i < n) cnt[i] = run;
        run += v[k];
    }
    if (i0 <= n - 1 && n - 1 < i0 + per) cnt[n] = run;  // the owner of the last element writes the total
}

cudaError_t launch_scan(int *cnt, int n, cudaStream_t st) {
    if (n <= 64 * 1024) {
        k_scan_exclusive<<<1, 1024, 0, st>>>(cnt, n);
        return cudaGetLastError();
    }
    // the tile sums live past the end of the array's total slot: callers
    // allocate n + 1 + ceil(n / SCAN_TILE) + 1 ints
    const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int *sums = cnt + n + 1;
    k_scan_tile_sums<<<nb, 1024, 0, st>>>(cnt, n, sums);
    k_scan_exclusive<<<1, 1024, 0, st>>>(sums, nb);
    k_scan_tiles<<<nb, 1024, 0, st>>>(cnt, n, sums);
    return cudaGetLastError();
}

template cudaError_t launch_bin<float>(se_plan_s *, const float *, const float *, const float *, cudaStream_t);
template cudaError_t launch_bin_set<float>(se_plan_s *, Buffers &, int, const float *, const float *, const float *,
                                           cudaStream_t);
template cudaError_t launch_bin_set<double>(se_plan_s *, Buffers &, int, const double *, const double *,
                                            const double *, cudaStream_t);
template cudaError_t launch_bin<double>(se_plan_s *, const double *, const double *, const double *,
                                        cudaStream_t);

}  // namespace se
