// FP32 spreading (step 1, eq. Hx) and gather (step 5, eq. u_integr) with the
// padded grid block of a tile held in registers.
//
// A tile is TE^3 window starts; the grid points its points touch form the
// padded block of PT = TE + P - 1 points per dimension.  Thread (cx, cy) of
// the CTA owns the column of PT grid values at (cx, cy) for the three source
// components, in registers.  Points of the tile are taken NB at a time: their
// separable Gaussian weights are computed once into shared memory (the z
// weights already shifted to the point's position in the column, zero
// elsewhere), then every thread whose column lies in a point's P x P support
// updates (spreading) or reads (gather) its whole column with register FMAs.
// Compared with a shared-memory accumulator this removes the read-modify-write
// traffic of the P^3 updates; the columns are written to the zero-padded FFT
// input once per tile (global atomics: neighbouring tiles overlap in their
// halos) or read from the inverse transform once per tile.
//
// Gather reduces each point's contributions over the CTA: a warp shuffle sum,
// then one shared-memory atomic per warp and component.
#include "se_internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

namespace se {

namespace {

constexpr unsigned FULL = 0xffffffffu;

#ifndef SE_COL_NB
#define SE_COL_NB 128
#endif

template <int P, int TE>
struct ColCfg {
    static constexpr int PT = TE + P - 1;       // padded block edge
    static constexpr int PZ = (P + 3) / 4 * 4;  // z weights padded for 16-byte loads
    static constexpr int NT = (PT * PT + 31) / 32 * 32;
    static constexpr int NB = SE_COL_NB;        // points staged per batch
};

// Shared staging of a batch of points: fractional positions relative to the
// window start (grid units), offsets of the window in the padded block, the
// three 1-D weight vectors.
template <int P, int TE>
struct ColStage {
    using C = ColCfg<P, TE>;
    float wz[C::NB][C::PZ];
    float wx[C::NB][P];
    float wy[C::NB][P];
    float4 src[C::NB];
    float fr[C::NB][3];
    int oxy[C::NB];
    int oz[C::NB];
    int m[C::NB];
    float out[C::NB][3];
};

// Stage 1 (thread j < nb): point b0 + j.
template <int P, int TE>
__device__ __forceinline__ void stage_point(ColStage<P, TE> &S, const GP<float> &g, int j, int n, int gx0, int gy0,
                                            int gz0, const float4 *__restrict__ xs) {
    const float4 xv = xs[n];
    int i0[3];
    unpack3(get_tag(xv), i0[0], i0[1], i0[2]);
    S.fr[j][0] = ((xv.x - g.x0[0]) * g.inv_h + g.half_ext) - (float)i0[0];
    S.fr[j][1] = ((xv.y - g.x0[1]) * g.inv_h + g.half_ext) - (float)i0[1];
    S.fr[j][2] = ((xv.z - g.x0[2]) * g.inv_h + g.half_ext) - (float)i0[2];
    const int ox = min(max(i0[0] - gx0, 0), TE - 1), oy = min(max(i0[1] - gy0, 0), TE - 1),
              oz = min(max(i0[2] - gz0, 0), TE - 1);
    S.oxy[j] = ox | (oy << 8);
    S.oz[j] = oz;
}

// Stage 2 (all threads): the weights of the nb staged points.
template <int P, int TE>
__device__ __forceinline__ void stage_weights(ColStage<P, TE> &S, const GP<float> &g, int nb) {
    constexpr int PER = 3 * P;
    for (int e = threadIdx.x; e < nb * PER; e += blockDim.x) {
        const int j = e / PER, k = e - j * PER, d = k / P, kk = k - d * P;
        const float t = S.fr[j][d] - (float)kk;
        const float wv = __expf(-g.ah2 * t * t);
        if (d == 0) S.wx[j][kk] = wv;
        else if (d == 1) S.wy[j][kk] = wv;
        else S.wz[j][kk] = wv;
    }
}

// a_c[OZ + kz] += s_c wz[kz] for kz < P (the point's z support at offset OZ of the column)
template <int P, int PT, int OZ>
__device__ __forceinline__ void col_add(float (&a0)[PT], float (&a1)[PT], float (&a2)[PT], float s0, float s1,
                                        float s2, const float *wz) {
    const float4 *wz4 = reinterpret_cast<const float4 *>(wz);
#pragma unroll
    for (int q = 0; q < (P + 3) / 4; q++) {
        const float4 v = wz4[q];
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int kz = 4 * q + i;
            if (kz < P) {
                a0[OZ + kz] = fmaf(s0, vv[i], a0[OZ + kz]);
                a1[OZ + kz] = fmaf(s1, vv[i], a1[OZ + kz]);
                a2[OZ + kz] = fmaf(s2, vv[i], a2[OZ + kz]);
            }
        }
    }
}

// p_c += sum_kz wz[kz] w_c[OZ + kz]
template <int P, int PT, int OZ>
__device__ __forceinline__ void col_dot(const float (&w0)[PT], const float (&w1)[PT], const float (&w2)[PT],
                                        const float *wz, float &p0, float &p1, float &p2) {
    const float4 *wz4 = reinterpret_cast<const float4 *>(wz);
#pragma unroll
    for (int q = 0; q < (P + 3) / 4; q++) {
        const float4 v = wz4[q];
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int kz = 4 * q + i;
            if (kz < P) {
                p0 = fmaf(vv[i], w0[OZ + kz], p0);
                p1 = fmaf(vv[i], w1[OZ + kz], p1);
                p2 = fmaf(vv[i], w2[OZ + kz], p2);
            }
        }
    }
}

// the z offset of a point's support in the column selects a fully unrolled
// copy (register indices must be compile-time constants)
#define SE_COL_CASES(F, ...)                  \
    switch (oz) {                             \
        case 0: F<P, PT, 0>(__VA_ARGS__); break; \
        case 1: F<P, PT, 1>(__VA_ARGS__); break; \
        case 2: F<P, PT, 2>(__VA_ARGS__); break; \
        case 3: F<P, PT, 3>(__VA_ARGS__); break; \
        case 4: F<P, PT, 4>(__VA_ARGS__); break; \
        case 5: F<P, PT, 5>(__VA_ARGS__); break; \
        case 6: F<P, PT, 6>(__VA_ARGS__); break; \
        default: F<P, PT, 7>(__VA_ARGS__); break; \
    }

template <int P, int TE>
__device__ __forceinline__ void spread_col_body(const GP<float> &g, int tile, int beg, int end, int c0, bool stress,
                                                const float4 *__restrict__ xs, const float4 *__restrict__ fs,
                                                int fstride, int foff, const float4 *__restrict__ qs,
                                                float *__restrict__ grid) {
    using C = ColCfg<P, TE>;
    constexpr int PT = C::PT, NB = C::NB;
    static_assert(TE == 8, "the unrolled z offsets cover tiles of 8");
    __shared__ __align__(16) ColStage<P, TE> S;
    const int tid = threadIdx.x;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int gx0 = tx * TE, gy0 = ty * TE, gz0 = tz * TE;
    const bool own = tid < PT * PT;
    const int cx = tid % PT, cy = tid / PT;
    float a0[PT], a1[PT], a2[PT];
#pragma unroll
    for (int z = 0; z < PT; z++) a0[z] = a1[z] = a2[z] = 0.0f;
    for (int b0 = beg; b0 < end; b0 += NB) {
        const int nb = min(NB, end - b0);
        if (tid < nb) {
            const int n = b0 + tid;
            stage_point<P, TE>(S, g, tid, n, gx0, gy0, gz0, xs);
            const float4 fv = fs[(size_t)n * fstride + foff];
            float4 sv = fv;
            if (stress) {
                // components c0 .. c0+2 of the symmetric source (xx, yy, zz, xy, xz, yz)
                const float4 qv = qs[n];
                if (c0 == 0) {
                    sv = make_float4(fv.x * qv.x, fv.y * qv.y, fv.z * qv.z, 0.0f);
                } else {
                    sv = make_float4(0.5f * (fv.x * qv.y + fv.y * qv.x), 0.5f * (fv.x * qv.z + fv.z * qv.x),
                                     0.5f * (fv.y * qv.z + fv.z * qv.y), 0.0f);
                }
            }
            S.src[tid] = sv;
        }
        __syncthreads();
        stage_weights<P, TE>(S, g, nb);
        __syncthreads();
        if (own) {
            for (int j = 0; j < nb; j++) {
                const int oxy = S.oxy[j];
                const int kx = cx - (oxy & 255), ky = cy - (oxy >> 8);
                if ((unsigned)kx < (unsigned)P && (unsigned)ky < (unsigned)P) {
                    const float w = S.wx[j][kx] * S.wy[j][ky];
                    const float4 sv = S.src[j];
                    const float s0 = sv.x * w, s1 = sv.y * w, s2 = sv.z * w;
                    const int oz = S.oz[j];
                    SE_COL_CASES(col_add, a0, a1, a2, s0, s1, s2, S.wz[j])
                }
            }
        }
        __syncthreads();
    }
    if (own) {
        const int gx = gx0 + cx, gy = gy0 + cy;
        if (gx < g.mt[0] && gy < g.mt[1]) {
            const size_t Mf = g.mf[0], Mf2 = Mf * g.mf[1], Mf3 = vol(g);
            float *base = grid + (size_t)c0 * Mf3 + ((size_t)gz0 * g.mf[1] + gy) * Mf + gx;
#pragma unroll
            for (int z = 0; z < PT; z++) {
                if (gz0 + z < g.mt[2]) {
                    float *pz = base + (size_t)z * Mf2;
                    if (a0[z] != 0.0f) atomicAdd(pz, a0[z]);
                    if (a1[z] != 0.0f) atomicAdd(pz + Mf3, a1[z]);
                    if (a2[z] != 0.0f) atomicAdd(pz + 2 * Mf3, a2[z]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- paired spreading
// FP32 spreading with the paired FP32 multiply-adds of sm_100 and later
// (__ffma2_rn: two lanes of one 64-bit register pair per instruction, the
// same rounding as two fmaf).  Thread (cx, cy) owns the column of the tile's
// padded block as ZP float2 pairs per component, z values (2q, 2q + 1) in
// pair q.  A point's P z weights are staged shifted by the parity of its z
// offset oz in the column, so that they start on a pair boundary: P/2 pairs
// when oz is even, P/2 + 1 (a zero at each end) when it is odd; the update of
// one column is then P/2 (+1) paired FMAs per component; register indices
// must be compile-time constants, so a switch on oz selects one of TE unrolled
// updates.  The staged points are put in order of oy (per chunk of 32 points,
// by warp ballots), so that each warp runs only through the contiguous run of
// points whose support meets its rows of columns.  The x and y weights are
// staged over the whole padded block (zero outside the point's support), so
// every lane of such a warp takes the update without a per-lane branch.  Each
// point is staged by three threads, one per dimension, into one record, and
// the next batch is staged while the current one is accumulated (two buffers,
// one barrier per batch).
// SE_C2_MINB: blocks per SM the paired spreading kernels are compiled for
// (2: at most 80 registers per thread; 1: up to 168)
#ifndef SE_C2_MINB
#define SE_C2_MINB 2
#endif

template <int P, int TE>
struct C2Cfg {
    static constexpr int PT = TE + P - 1;        // padded block edge
    static constexpr int PTP = (PT + 3) / 4 * 4; // x, y weight rows padded to 16 bytes
    static constexpr int ZP = (PT + 1) / 2;      // z pairs per column and component
    static constexpr int WP = P / 2 + 1;         // staged z-weight pairs (odd offsets need P/2 + 1)
    static constexpr int WP4 = (WP + 1) / 2 * 2; // rounded up to whole 16-byte rows
    static constexpr int NT = (PT * PT + 31) / 32 * 32;
    static constexpr int NB = NT / 3 / 32 * 32;  // points per batch: three staging threads each, whole warps
    static constexpr int NCH = NB / 32;          // chunks of 32 points ordered by oy
};

// One staged point: everything the column threads read, in one record so that
// a single base address serves all its loads.
template <int P, int TE>
struct __align__(16) C2Rec {
    using C = C2Cfg<P, TE>;
    float4 wz[C::WP4 / 2];           // z weights as pairs, shifted by the parity of oz
    float4 src;                      // the three source components
    float wx[C::PTP];                // x weight of every column of the block (0 off the support)
    float wy[C::PTP];
    uchar4 off;                      // ox, oy, oz: window start in the padded block
};

template <int P, int TE>
struct C2Stage {
    using C = C2Cfg<P, TE>;
    C2Rec<P, TE> rec[C::NB];
    unsigned char ord[C::NB];        // chunk c's points in order of oy: 32 c + ord[32 c + i]
    unsigned char start[C::NCH][12]; // chunk c's points with oy = b: ord[32 c + start[b] .. 32 c + start[b + 1])
};

template <int P, int TE>
constexpr size_t c2_smem_bytes() {
    return 2 * sizeof(C2Stage<P, TE>);
}

// Stage points b0 .. b0 + nb - 1 into S: thread t takes dimension d = t / NB
// of point j = t mod NB.  The y threads (whole warps) also order their 32
// points by oy.
template <int P, int TE>
__device__ __forceinline__ void c2_stage(C2Stage<P, TE> &S, const GP<float> &g, int b0, int nb, int gx0, int gy0,
                                         int gz0, int c0, bool stress, const float4 *__restrict__ xs,
                                         const float4 *__restrict__ fs, int fstride, int foff,
                                         const float4 *__restrict__ qs) {
    using C = C2Cfg<P, TE>;
    const int t = threadIdx.x;
    if (t >= 3 * C::NB) return;
    const int d = t / C::NB, j = t - d * C::NB;
    const bool valid = j < nb;
    int o = TE;  // no valid point: an oz no bucket takes
    float fr = 0.0f;
    if (valid) {
        const int n = b0 + j;
        const float4 xv = xs[n];
        int i0[3];
        unpack3(get_tag(xv), i0[0], i0[1], i0[2]);
        const float xd = d == 0 ? xv.x : (d == 1 ? xv.y : xv.z);
        const int id = d == 0 ? i0[0] : (d == 1 ? i0[1] : i0[2]);
        const float x0 = d == 0 ? g.x0[0] : (d == 1 ? g.x0[1] : g.x0[2]);
        const int o0 = d == 0 ? gx0 : (d == 1 ? gy0 : gz0);
        fr = ((xd - x0) * g.inv_h + g.half_ext) - (float)id;
        o = min(max(id - o0, 0), TE - 1);
        reinterpret_cast<unsigned char *>(&S.rec[j].off)[d] = (unsigned char)o;
        if (d == 0) {
            const float4 fv = fs[(size_t)n * fstride + foff];
            float4 sv = fv;
            if (stress) {
                // components c0 .. c0+2 of the symmetric source (xx, yy, zz, xy, xz, yz)
                const float4 qv = qs[n];
                if (c0 == 0)
                    sv = make_float4(fv.x * qv.x, fv.y * qv.y, fv.z * qv.z, 0.0f);
                else
                    sv = make_float4(0.5f * (fv.x * qv.y + fv.y * qv.x), 0.5f * (fv.x * qv.z + fv.z * qv.x),
                                     0.5f * (fv.y * qv.z + fv.z * qv.y), 0.0f);
            }
            S.rec[j].src = sv;
        }
    }
    if (d == 1) {
        // order the warp's 32 points by oy: rank within the bucket by ballots
        const int lane = j & 31, ch = j >> 5;
        const unsigned lt = (1u << lane) - 1u;
        int base = 0, pos = 0;
#pragma unroll
        for (int bkt = 0; bkt < TE; bkt++) {
            const unsigned m = __ballot_sync(0xffffffffu, o == bkt);
            if (lane == 0) S.start[ch][bkt] = (unsigned char)base;
            if (o == bkt) pos = base + __popc(m & lt);
            base += __popc(m);
        }
        if (lane == 0) S.start[ch][TE] = (unsigned char)base;
        if (valid) S.ord[32 * ch + pos] = (unsigned char)lane;
    }
    if (d == 2) {
        if (valid) {
            // the P weights at slots (oz & 1) .. (oz & 1) + P - 1, zeros elsewhere
            float *w = reinterpret_cast<float *>(S.rec[j].wz);
            const int sh = o & 1;
#pragma unroll
            for (int i = 0; i < 2 * C::WP4; i++) {
                const int kk = i - sh;
                const float tt = fr - (float)kk;
                w[i] = (kk >= 0 && kk < P) ? __expf(-g.ah2 * tt * tt) : 0.0f;
            }
        }
    } else if (valid) {
        // weights of every column of the block: zero off the point's support
        float *w = d == 0 ? S.rec[j].wx : S.rec[j].wy;
#pragma unroll
        for (int c = 0; c < C::PTP; c++) {
            const int kk = c - o;
            const float tt = fr - (float)kk;
            w[c] = (kk >= 0 && kk < P) ? __expf(-g.ah2 * tt * tt) : 0.0f;
        }
    }
}

// a_c[OZ/2 + k] += s_c wz[k] for the point's NP z pairs
template <int P, int ZP, int OZ>
__device__ __forceinline__ void col_add2(float2 (&a0)[ZP], float2 (&a1)[ZP], float2 (&a2)[ZP], float2 s0, float2 s1,
                                         float2 s2, const float4 *w4) {
    constexpr int Q0 = OZ / 2, NP = P / 2 + (OZ & 1);
    static_assert(Q0 + NP <= ZP, "the point's z support stays inside the column");
#pragma unroll
    for (int k2 = 0; k2 < (NP + 1) / 2; k2++) {
        const float4 v = w4[k2];
        const float2 lo = make_float2(v.x, v.y), hi = make_float2(v.z, v.w);
        a0[Q0 + 2 * k2] = __ffma2_rn(lo, s0, a0[Q0 + 2 * k2]);
        a1[Q0 + 2 * k2] = __ffma2_rn(lo, s1, a1[Q0 + 2 * k2]);
        a2[Q0 + 2 * k2] = __ffma2_rn(lo, s2, a2[Q0 + 2 * k2]);
        if (2 * k2 + 1 < NP) {
            a0[Q0 + 2 * k2 + 1] = __ffma2_rn(hi, s0, a0[Q0 + 2 * k2 + 1]);
            a1[Q0 + 2 * k2 + 1] = __ffma2_rn(hi, s1, a1[Q0 + 2 * k2 + 1]);
            a2[Q0 + 2 * k2 + 1] = __ffma2_rn(hi, s2, a2[Q0 + 2 * k2 + 1]);
        }
    }
}

// One staged point into the thread's column (a column off the point's
// support has zero x or y weight).
template <int P, int TE, int OZ>
__device__ __forceinline__ void c2_point(const C2Rec<P, TE> &R, int cx, int cy, float2 (&a0)[C2Cfg<P, TE>::ZP],
                                         float2 (&a1)[C2Cfg<P, TE>::ZP], float2 (&a2)[C2Cfg<P, TE>::ZP]) {
    constexpr int ZP = C2Cfg<P, TE>::ZP;
    const float w = R.wx[cx] * R.wy[cy];
    const float4 sv = R.src;
    const float2 s0 = make_float2(sv.x * w, sv.x * w), s1 = make_float2(sv.y * w, sv.y * w),
                 s2 = make_float2(sv.z * w, sv.z * w);
    col_add2<P, ZP, OZ>(a0, a1, a2, s0, s1, s2, R.wz);
}

#define SE_COL2_CASES(...)                                \
    switch (oz) {                                         \
        case 0: c2_point<P, TE, 0>(__VA_ARGS__); break;   \
        case 1: c2_point<P, TE, 1>(__VA_ARGS__); break;   \
        case 2: c2_point<P, TE, 2>(__VA_ARGS__); break;   \
        case 3: c2_point<P, TE, 3>(__VA_ARGS__); break;   \
        case 4: c2_point<P, TE, 4>(__VA_ARGS__); break;   \
        case 5: c2_point<P, TE, 5>(__VA_ARGS__); break;   \
        case 6: c2_point<P, TE, 6>(__VA_ARGS__); break;   \
        default: c2_point<P, TE, 7>(__VA_ARGS__); break;  \
    }

// Accumulate the nb staged points of S into the thread's column (threads
// beyond the block's columns read column 0's weights and keep their sums to
// themselves).
template <int P, int TE>
__device__ __forceinline__ void c2_accumulate(const C2Stage<P, TE> &S, int nb, int cx, int cy, int cyl, int cyh,
                                              float2 (&a0)[C2Cfg<P, TE>::ZP], float2 (&a1)[C2Cfg<P, TE>::ZP],
                                              float2 (&a2)[C2Cfg<P, TE>::ZP]) {
    static_assert(TE == 8, "the unrolled z offsets cover tiles of 8");
    // points in order of oy: the warp takes, per chunk, the contiguous run of
    // those whose support meets its rows, with a switch on oz per point
    const int ylo = max(0, cyl - (P - 1)), yhi = min(TE - 1, cyh);
    for (int ch = 0; ch < (nb + 31) / 32; ch++) {
        const int i1 = S.start[ch][yhi + 1];
        for (int i = S.start[ch][ylo]; i < i1; i++) {
            const C2Rec<P, TE> &R = S.rec[32 * ch + S.ord[32 * ch + i]];
            const int oz = R.off.z;
            SE_COL2_CASES(R, cx, cy, a0, a1, a2)
        }
    }
}

// Add the thread's column (grid column (gx, gy), z planes gz0 ..) to the three
// grids at grid, grid + gcs, grid + 2 gcs (z-plane stride gzs): global atomics,
// since neighbouring tiles overlap in their halos.
template <int P, int TE>
__device__ __forceinline__ void c2_flush(const GP<float> &g, int gx, int gy, int gz0,
                                         const float2 (&a0)[C2Cfg<P, TE>::ZP], const float2 (&a1)[C2Cfg<P, TE>::ZP],
                                         const float2 (&a2)[C2Cfg<P, TE>::ZP], float *__restrict__ grid, size_t gzs,
                                         size_t gcs) {
    constexpr int PT = C2Cfg<P, TE>::PT, ZP = C2Cfg<P, TE>::ZP;
    if (gx >= g.mt[0] || gy >= g.mt[1]) return;
    float *base = grid + (size_t)gz0 * gzs + (size_t)gy * g.mf[0] + gx;
#pragma unroll
    for (int q = 0; q < ZP; q++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int z = 2 * q + h;
            if (z < PT && gz0 + z < g.mt[2]) {
                float *pz = base + (size_t)z * gzs;
                const float v0 = h ? a0[q].y : a0[q].x, v1 = h ? a1[q].y : a1[q].x, v2 = h ? a2[q].y : a2[q].x;
                if (v0 != 0.0f) atomicAdd(pz, v0);
                if (v1 != 0.0f) atomicAdd(pz + gcs, v1);
                if (v2 != 0.0f) atomicAdd(pz + 2 * gcs, v2);
            }
        }
    }
}

// Deterministic plans: store the thread's column (cx, cy) of the tile's padded
// block, all PT z planes, in the tile's slot tbt of the tile buffer (no
// atomics; k_merge_tiles adds the tiles later in a fixed order); the threads
// tid < PT (XB - PT) zero the row padding.
template <int P, int TE>
__device__ __forceinline__ void c2_flush_tb(int tid, int cx, int cy, const float2 (&a0)[C2Cfg<P, TE>::ZP],
                                            const float2 (&a1)[C2Cfg<P, TE>::ZP],
                                            const float2 (&a2)[C2Cfg<P, TE>::ZP], float *__restrict__ tbt) {
    using B = TileBufCfg<P>;
    constexpr int PT = C2Cfg<P, TE>::PT, ZP = C2Cfg<P, TE>::ZP, NPAD = B::XB - PT;
    static_assert(TE == COL_TE && B::PE == PT, "the tile buffer holds the kernel's padded block");
    if (tid < PT * PT) {
#pragma unroll
        for (int q = 0; q < ZP; q++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int z = 2 * q + h;
                if (z < PT) {
                    float *pz = tbt + ((size_t)z * PT + cy) * B::XB + cx;
                    pz[0] = h ? a0[q].y : a0[q].x;
                    pz[(size_t)PT * PT * B::XB] = h ? a1[q].y : a1[q].x;
                    pz[(size_t)2 * PT * PT * B::XB] = h ? a2[q].y : a2[q].x;
                }
            }
    }
    if (NPAD > 0 && tid < PT * NPAD) {
        const int y = tid / NPAD, x = PT + tid % NPAD;
        for (int cz = 0; cz < 3 * PT; cz++) tbt[((size_t)cz * PT + y) * B::XB + x] = 0.0f;
    }
}

// The column a thread owns: (cx, cy) of the block for tid < PT^2; the others
// (the last warp's tail) take column 0 for their reads and never write.
template <int P, int TE>
__device__ __forceinline__ void c2_column(int tid, int &cx, int &cy, int &cyl, int &cyh) {
    constexpr int PT = C2Cfg<P, TE>::PT;
    const bool own = tid < PT * PT;
    cx = own ? tid % PT : 0;
    cy = own ? tid / PT : 0;
    // the rows of columns this warp owns
    const int w0 = tid & ~31;
    cyl = w0 / PT;
    cyh = min(w0 + 31, PT * PT - 1) / PT;
}

template <int P, int TE>
__device__ __forceinline__ void spread_c2_body(const GP<float> &g, int tile, int beg, int end, int c0, bool stress,
                                               const float4 *__restrict__ xs, const float4 *__restrict__ fs,
                                               int fstride, int foff, const float4 *__restrict__ qs,
                                               float *__restrict__ grid, size_t gzs, size_t gcs,
                                               C2Stage<P, TE> *S, float *__restrict__ tbt = nullptr) {
    using C = C2Cfg<P, TE>;
    constexpr int PT = C::PT, ZP = C::ZP, NB = C::NB;
    const int tid = threadIdx.x;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int gx0 = tx * TE, gy0 = ty * TE, gz0 = tz * TE;
    int cx, cy, cyl, cyh;
    c2_column<P, TE>(tid, cx, cy, cyl, cyh);
    float2 a0[ZP], a1[ZP], a2[ZP];
#pragma unroll
    for (int q = 0; q < ZP; q++) a0[q] = a1[q] = a2[q] = make_float2(0.0f, 0.0f);
    c2_stage<P, TE>(S[0], g, beg, min(NB, end - beg), gx0, gy0, gz0, c0, stress, xs, fs, fstride, foff, qs);
    __syncthreads();
    int k = 0;
    for (int b0 = beg; b0 < end; b0 += NB, k ^= 1) {
        const int nb = min(NB, end - b0);
        if (b0 + NB < end)
            c2_stage<P, TE>(S[k ^ 1], g, b0 + NB, min(NB, end - b0 - NB), gx0, gy0, gz0, c0, stress, xs, fs, fstride,
                            foff, qs);
        c2_accumulate<P, TE>(S[k], nb, cx, cy, cyl, cyh, a0, a1, a2);
        __syncthreads();
    }
    if (tbt)
        c2_flush_tb<P, TE>(tid, cx, cy, a0, a1, a2, tbt);
    else if (tid < PT * PT)
        c2_flush<P, TE>(g, gx0 + cx, gy0 + cy, gz0, a0, a1, a2, grid + (size_t)c0 * gcs, gzs, gcs);
}

// w: three grids (the group of right-hand side r); u, f_orig: n_rhs three-vectors per point.
template <int P, int TE>
__device__ __forceinline__ void gather_col_body(const GP<float> &g, int tile, int beg, int end,
                                                const float4 *__restrict__ xs, const int *__restrict__ perm,
                                                const float *__restrict__ w, int n_rhs, int r,
                                                const float *__restrict__ f_orig, double self_coef,
                                                float *__restrict__ u) {
    using C = ColCfg<P, TE>;
    constexpr int PT = C::PT, NB = C::NB;
    static_assert(TE == 8, "the unrolled z offsets cover tiles of 8");
    __shared__ __align__(16) ColStage<P, TE> S;
    const int tid = threadIdx.x, lane = tid & 31;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int gx0 = tx * TE, gy0 = ty * TE, gz0 = tz * TE;
    const bool own = tid < PT * PT;
    const int cx = tid % PT, cy = tid / PT;
    // the thread's column of the three grids (zero outside the extended grid)
    float w0[PT], w1[PT], w2[PT];
    {
        const int gx = gx0 + cx, gy = gy0 + cy;
        const bool in = own && gx < g.mt[0] && gy < g.mt[1];
        const size_t Mf = g.mf[0], Mf2 = Mf * g.mf[1], Mf3 = vol(g);
        const float *base = w + ((size_t)gz0 * g.mf[1] + gy) * Mf + gx;
#pragma unroll
        for (int z = 0; z < PT; z++) {
            const bool ok = in && (gz0 + z < g.mt[2]);
            const float *pz = base + (size_t)z * Mf2;
            w0[z] = ok ? __ldg(pz) : 0.0f;
            w1[z] = ok ? __ldg(pz + Mf3) : 0.0f;
            w2[z] = ok ? __ldg(pz + 2 * Mf3) : 0.0f;
        }
    }
    for (int b0 = beg; b0 < end; b0 += NB) {
        const int nb = min(NB, end - b0);
        if (tid < nb) {
            stage_point<P, TE>(S, g, tid, b0 + tid, gx0, gy0, gz0, xs);
            S.m[tid] = perm[b0 + tid];
        }
        if (tid < 3 * NB) S.out[tid / 3][tid % 3] = 0.0f;
        __syncthreads();
        stage_weights<P, TE>(S, g, nb);
        __syncthreads();
        for (int j = 0; j < nb; j++) {
            const int oxy = S.oxy[j];
            const int kx = cx - (oxy & 255), ky = cy - (oxy >> 8);
            const bool act = own && (unsigned)kx < (unsigned)P && (unsigned)ky < (unsigned)P;
            if (!__any_sync(FULL, act)) continue;
            float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f;
            if (act) {
                const int oz = S.oz[j];
                SE_COL_CASES(col_dot, w0, w1, w2, S.wz[j], p0, p1, p2)
                const float wxy = S.wx[j][kx] * S.wy[j][ky];
                p0 *= wxy;
                p1 *= wxy;
                p2 *= wxy;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                p0 += __shfl_xor_sync(FULL, p0, o);
                p1 += __shfl_xor_sync(FULL, p1, o);
                p2 += __shfl_xor_sync(FULL, p2, o);
            }
            if (lane == 0) {
                atomicAdd(&S.out[j][0], p0);
                atomicAdd(&S.out[j][1], p1);
                atomicAdd(&S.out[j][2], p2);
            }
        }
        __syncthreads();
        if (tid < 3 * nb) {
            const int j = tid / 3, c = tid - 3 * j;
            const size_t o3 = ((size_t)S.m[j] * n_rhs + r) * 3 + c;
            double o = (double)S.out[j][c];
            if (self_coef != 0.0) o += self_coef * (double)f_orig[o3];
            u[o3] = (float)o;
        }
        __syncthreads();
    }
}

// Gather with the tile's padded block in shared memory: the CTA stages the
// PT^3 block of the three grids once (coalesced rows), then each warp takes
// one point at a time, its lanes covering the (x, y) columns of the P x P
// support and reading the P values of each column from shared memory.  Every
// grid value is read from L2 once per tile and from shared memory once per
// point that uses it; no cross-warp reduction.
#ifndef SE_GS_WARPS
#define SE_GS_WARPS 16
#endif
constexpr int GS_WARPS = SE_GS_WARPS;

// Row pitch of the staged block and the largest number of support columns per
// lane: the lanes of a warp read column (kx, ky) at offset ky * pitch + kx, so
// each lane takes the columns whose offset is its own lane id mod 32 (one
// shared-memory bank per lane, no conflicts); the pitch >= PT minimising the
// largest such class, a multiple of 4 floats (the 16-byte rows of a tensor
// copy's box).
template <int P, int PT>
struct GsLayout {
    static constexpr int count(int pitch) {
        int worst = 0;
        for (int r = 0; r < 32; r++) {
            int n = 0;
            for (int ky = 0; ky < P; ky++)
                for (int kx = 0; kx < P; kx++)
                    if ((ky * pitch + kx) % 32 == r) n++;
            worst = n > worst ? n : worst;
        }
        return worst;
    }
    static constexpr int best_pitch() {
        const int q0 = (PT + 3) / 4 * 4;
        int bp = q0, bn = count(q0);
        for (int q = q0 + 4; q <= q0 + 8; q += 4)
            if (count(q) < bn) { bn = count(q); bp = q; }
        return bp;
    }
    static constexpr int PX = best_pitch();
    static constexpr int NIT = count(PX);
};

// Bounded wait on phase `phase` of a shared-memory mbarrier; false when
// `limit_ns` nanoseconds of the global timer passed first.
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// a tile copy takes microseconds; one second means it will not come
constexpr uint64_t GS_WAIT_NS = 1000000000ull;

// Staging of a tile's padded block of three grids in shared memory (sg,
// 128-byte aligned): TMA = true by one tensor copy, a box of PX x PT x PT x 3
// floats at (gx0, gy0, gz0, 0) of the grids seen as a 4-D tensor of extent
// (Mt_x, Mt_y, Mt_z, 3) (the copy engine fills the part outside with zeros;
// gx0 is a multiple of TE = 8, so the box starts on a 32-byte boundary);
// otherwise by plain loads.  ZC (batches, with TMA): the interleaved batch
// grids are copied as a tensor (x, y, component, z), so the staged block is
// [z][c][y][x] instead of [c][z][y][x]; the box starts at component 3 r
// (right-hand side r).  False when the copy did not land within the wait limit
// (reported in status).
// skip_copy (tests of the failure path): the copy is not issued, so the wait
// runs out and the status reports it.
template <int P, int TE, bool TMA, bool ZC>
__device__ __forceinline__ bool stage_block(float *sg, uint64_t *bar_mem, const GP<float> &g, int gx0, int gy0,
                                            int gz0, int r, const float *__restrict__ w, size_t gzs, size_t gcs,
                                            const void *tmap, int *status, bool skip_copy = false) {
    static_assert(TMA || !ZC, "the z-major block comes from a tensor copy");
    constexpr int PT = TE + P - 1, PX = GsLayout<P, PT>::PX, ROWS = 3 * PT * PT;
    if constexpr (TMA) {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(bar_mem);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (threadIdx.x == 0 && !skip_copy) {
            constexpr uint32_t bytes = (uint32_t)(3 * PT * PT * PX * sizeof(float));
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                         : "memory");
            const int k2 = ZC ? 3 * r : gz0, k3 = ZC ? gz0 : 0;
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"((uint32_t)__cvta_generic_to_shared(sg)),
                "l"(reinterpret_cast<uint64_t>(tmap)), "r"(gx0), "r"(gy0), "r"(k2), "r"(k3), "r"(bar)
                : "memory");
        }
        if (!mbar_wait(bar, 0, GS_WAIT_NS)) {
            // the copy did not land: report, give a copy in flight one more
            // bounded wait, leave.  A copy still in flight after that may land
            // in shared memory another CTA has taken over, so the results of
            // an evaluation that reports the timeout are undefined (the host
            // sees SE_ERR_TIMEOUT and discards them)
            if (threadIdx.x == 0) atomicOr(status, FLAG_TIMEOUT);
            if (!skip_copy) mbar_wait(bar, 0, GS_WAIT_NS);
            return false;
        }
    } else {
        const size_t Mf = g.mf[0];
        // flat copy of the block (x fastest), several independent loads in flight per thread
#pragma unroll 8
        for (int e = threadIdx.x; e < ROWS * PT; e += GS_WARPS * 32) {
            const int row = e / PT, x = e - row * PT, c = row / (PT * PT), zy = row - c * PT * PT, z = zy / PT,
                      y = zy - z * PT;
            const int gz = gz0 + z, gy = gy0 + y, gx = gx0 + x;
            sg[row * PX + x] = (gz < g.mt[2] && gy < g.mt[1] && gx < g.mt[0])
                                   ? __ldg(w + (size_t)c * gcs + (size_t)gz * gzs + (size_t)gy * Mf + gx)
                                   : 0.0f;
        }
        __syncthreads();
    }
    return true;
}

// This lane's support columns (kx, ky): those at offset ky * PX + kx = lane
// (mod 32), in increasing order, NIT slots.
template <int P, int PX, int NIT>
__device__ __forceinline__ void lane_columns(int lane, int (&kxs)[NIT], int (&kys)[NIT], bool (&val)[NIT]) {
#pragma unroll
    for (int it = 0; it < NIT; it++) {
        val[it] = false;
        kxs[it] = kys[it] = 0;
    }
    int it = 0;
    for (int o = lane; o < P * PX; o += 32) {
        const int ky = o / PX, kx = o - ky * PX;
        if (kx < P) {
#pragma unroll
            for (int q = 0; q < NIT; q++)
                if (q == it) {
                    kxs[q] = kx;
                    kys[q] = ky;
                    val[q] = true;
                }
            it++;
        }
    }
}

// MODE 0: u = the three gathered values (+ the self term).  MODE 1, 2: the
// stresslet's adjoint strength gradients from the symmetric tensor field V
// (xx, yy, zz, xy, xz, yz), three grids per pass: MODE 1 takes the diagonal
// grids and writes grad_f_l = V_ll q_l, grad_q_l = V_ll f_l; MODE 2 takes
// (xy, xz, yz) and adds the off-diagonal terms, grad_f_l += sum_{k != l} V_lk
// q_k, grad_q_l += sum_{k != l} V_lk f_k (u is grad_f, gq grad_q; either may
// be NULL).
template <int P, int TE, bool TMA, bool ZC = false, int MODE = 0>
__device__ __forceinline__ void gather_smem_body(const GP<float> &g, int tile, int beg, int end,
                                                 const float4 *__restrict__ xs, const int *__restrict__ perm,
                                                 const float *__restrict__ w, int n_rhs, int r,
                                                 const float *__restrict__ f_orig, double self_coef,
                                                 float *__restrict__ u, size_t gzs, size_t gcs,
                                                 const void *tmap = nullptr, int *status = nullptr,
                                                 bool skip_copy = false, const float *__restrict__ q_orig = nullptr,
                                                 float *__restrict__ gq = nullptr) {
    // gzs, gcs: the grids' z-plane and component strides
    constexpr int PT = TE + P - 1, PX = GsLayout<P, PT>::PX, NIT = GsLayout<P, PT>::NIT;
    constexpr int PLANE = PT * PX;
    // shared-memory strides of a z step and of a component step
    constexpr int ZS = ZC ? 3 * PLANE : PLANE, CS = ZC ? PLANE : PT * PLANE;
    extern __shared__ __align__(128) float sg_raw[];  // [c][z][y][x] (ZC: [z][c][y][x]), x pitch PX
    __shared__ float swt[GS_WARPS][3][P];
    __shared__ __align__(8) uint64_t bar_mem;
    // the tensor copy's destination starts on a 128-byte boundary
    float *sg = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(sg_raw) + 127) & ~uintptr_t(127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int gx0 = tx * TE, gy0 = ty * TE, gz0 = tz * TE;
    if (!stage_block<P, TE, TMA, ZC>(sg, &bar_mem, g, gx0, gy0, gz0, r, w, gzs, gcs, tmap, status, skip_copy))
        return;
    int kxs[NIT], kys[NIT];
    bool val[NIT];
    lane_columns<P, PX, NIT>(lane, kxs, kys, val);
    // the next point's position, index and self-term source are loaded one
    // iteration ahead
    float4 xnext = make_float4(0.f, 0.f, 0.f, 0.f);
    int mnext = 0;
    float fnext = 0.f;
    if (beg + warp < end) {
        xnext = xs[beg + warp];
        mnext = perm[beg + warp];
        if (lane < 3 && self_coef != 0.0) fnext = f_orig[((size_t)mnext * n_rhs + r) * 3 + lane];
    }
    for (int n = beg + warp; n < end; n += GS_WARPS) {
        const float4 xv = xnext;
        const int mcur = mnext;
        const float fcur = fnext;
        if (n + GS_WARPS < end) {
            xnext = xs[n + GS_WARPS];
            mnext = perm[n + GS_WARPS];
            if (lane < 3 && self_coef != 0.0) fnext = f_orig[((size_t)mnext * n_rhs + r) * 3 + lane];
        }
        int i0[3];
        unpack3(get_tag(xv), i0[0], i0[1], i0[2]);
        if (lane < P) {
            const float fr0 = ((xv.x - g.x0[0]) * g.inv_h + g.half_ext) - (float)i0[0] - (float)lane;
            const float fr1 = ((xv.y - g.x0[1]) * g.inv_h + g.half_ext) - (float)i0[1] - (float)lane;
            const float fr2 = ((xv.z - g.x0[2]) * g.inv_h + g.half_ext) - (float)i0[2] - (float)lane;
            swt[warp][0][lane] = __expf(-g.ah2 * fr0 * fr0);
            swt[warp][1][lane] = __expf(-g.ah2 * fr1 * fr1);
            swt[warp][2][lane] = __expf(-g.ah2 * fr2 * fr2);
        }
        __syncwarp();
        const int ox = min(max(i0[0] - gx0, 0), TE - 1), oy = min(max(i0[1] - gy0, 0), TE - 1),
                  oz = min(max(i0[2] - gz0, 0), TE - 1);
        float wz[P];
#pragma unroll
        for (int kz = 0; kz < P; kz++) wz[kz] = swt[warp][2][kz];
        float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f;
#pragma unroll
        for (int it = 0; it < NIT; it++) {
            if (val[it]) {
                const float wxy = swt[warp][0][kxs[it]] * swt[warp][1][kys[it]];
                const float *col = sg + oz * ZS + (oy + kys[it]) * PX + ox + kxs[it];
                float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int kz = 0; kz < P; kz++) {
                    a0 = fmaf(col[kz * ZS], wz[kz], a0);
                    a1 = fmaf(col[CS + kz * ZS], wz[kz], a1);
                    a2 = fmaf(col[2 * CS + kz * ZS], wz[kz], a2);
                }
                acc0 = fmaf(a0, wxy, acc0);
                acc1 = fmaf(a1, wxy, acc1);
                acc2 = fmaf(a2, wxy, acc2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc0 += __shfl_xor_sync(FULL, acc0, o);
            acc1 += __shfl_xor_sync(FULL, acc1, o);
            acc2 += __shfl_xor_sync(FULL, acc2, o);
        }
        if (MODE == 0 && lane < 3) {
            const size_t o3 = ((size_t)mcur * n_rhs + r) * 3 + lane;
            double o = (double)(lane == 0 ? acc0 : (lane == 1 ? acc1 : acc2));
            if (self_coef != 0.0) o += self_coef * (double)fcur;
            u[o3] = (float)o;
        }
        if (MODE != 0 && lane < 3) {
            const size_t b3 = 3 * (size_t)mcur;
            const float q0 = q_orig[b3], q1 = q_orig[b3 + 1], q2 = q_orig[b3 + 2];
            const float f0 = f_orig[b3], f1 = f_orig[b3 + 1], f2 = f_orig[b3 + 2];
            if (MODE == 1) {
                const float v = lane == 0 ? acc0 : (lane == 1 ? acc1 : acc2);
                if (u) u[b3 + lane] = v * (lane == 0 ? q0 : (lane == 1 ? q1 : q2));
                if (gq) gq[b3 + lane] = v * (lane == 0 ? f0 : (lane == 1 ? f1 : f2));
            } else {
                // (acc0, acc1, acc2) = (V_xy, V_xz, V_yz); row l of V without its
                // diagonal: l = 0: (xy, xz) against (y, z); 1: (xy, yz) against
                // (x, z); 2: (xz, yz) against (x, y)
                float tq, tf;
                if (lane == 0) {
                    tq = acc0 * q1 + acc1 * q2;
                    tf = acc0 * f1 + acc1 * f2;
                } else if (lane == 1) {
                    tq = acc0 * q0 + acc2 * q2;
                    tf = acc0 * f0 + acc2 * f2;
                } else {
                    tq = acc1 * q0 + acc2 * q1;
                    tf = acc1 * f0 + acc2 * f1;
                }
                if (u) u[b3 + lane] += tq;
                if (gq) gq[b3 + lane] += tf;
            }
        }
        __syncwarp();
    }
}

template <int P, int TE, bool TMA>
__global__ void __launch_bounds__(GS_WARPS * 32) k_gather_smem(GP<float> g, const int *__restrict__ tile_start,
                                                               const float4 *__restrict__ xs,
                                                               const int *__restrict__ perm,
                                                               const float *__restrict__ w,
                                                               const float *__restrict__ f_orig, double self_coef,
                                                               float *__restrict__ u,
                                                               const __grid_constant__ CUtensorMap tmap,
                                                               int *__restrict__ status, int skip_copy) {
    const int tile = blockIdx.x;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    gather_smem_body<P, TE, TMA>(g, tile, beg, end, xs, perm, w, 1, 0, f_orig, self_coef, u,
                                 (size_t)g.mf[0] * g.mf[1], vol(g), &tmap, status, skip_copy != 0);
}

// Position gradient of the Fourier part (du/dx, se_eval_backward), one group
// of three grids per launch: for the points of a tile, with the block staged as
// for the gather, gx_m (+)= c_grad sum_k grad W(x_m - x_k) (c_m . w_k) where c_m
// are the point's coefficients of the three grids (mode 0: g_m against the
// forward field; mode 1: f_m against the adjoint field; stresslet modes 2 and
// 3: the symmetric f_m q_m pairs of the adjoint tensor field, diagonal and
// off-diagonal) and grad W the Gaussian's derivative, W' = -2 a h (t) W per
// dimension (c_grad = -2 a h).  Mode 0 writes gx, the others add to it.
template <int P, int TE, bool TMA>
__device__ __forceinline__ void grad_smem_body(const GP<float> &g, int tile, int beg, int end,
                                               const float4 *__restrict__ xs, const int *__restrict__ perm,
                                               const float *__restrict__ w, int mode, const float *__restrict__ ca,
                                               const float *__restrict__ cb, float c_grad, float *__restrict__ gx,
                                               const void *tmap, int *status) {
    constexpr int PT = TE + P - 1, PX = GsLayout<P, PT>::PX, NIT = GsLayout<P, PT>::NIT;
    constexpr int PLANE = PT * PX, ZS = PLANE, CS = PT * PLANE;
    extern __shared__ __align__(128) float sg_raw[];  // [c][z][y][x], x pitch PX
    __shared__ float swt[GS_WARPS][3][P];
    __shared__ __align__(8) uint64_t bar_mem;
    float *sg = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(sg_raw) + 127) & ~uintptr_t(127));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int gx0 = tx * TE, gy0 = ty * TE, gz0 = tz * TE;
    if (!stage_block<P, TE, TMA, false>(sg, &bar_mem, g, gx0, gy0, gz0, 0, w, (size_t)g.mf[0] * g.mf[1], vol(g),
                                        tmap, status))
        return;
    int kxs[NIT], kys[NIT];
    bool val[NIT];
    lane_columns<P, PX, NIT>(lane, kxs, kys, val);
    for (int n = beg + warp; n < end; n += GS_WARPS) {
        const float4 xv = xs[n];
        const int m = perm[n];
        const float *A = ca + 3 * (size_t)m;
        float c0, c1, c2;
        if (mode <= 1) {
            c0 = A[0];
            c1 = A[1];
            c2 = A[2];
        } else {
            const float *B = cb + 3 * (size_t)m;
            if (mode == 2) {
                c0 = A[0] * B[0];
                c1 = A[1] * B[1];
                c2 = A[2] * B[2];
            } else {
                c0 = A[0] * B[1] + A[1] * B[0];
                c1 = A[0] * B[2] + A[2] * B[0];
                c2 = A[1] * B[2] + A[2] * B[1];
            }
        }
        int i0[3];
        unpack3(get_tag(xv), i0[0], i0[1], i0[2]);
        // offsets of the point from the first grid point of its support, per dimension
        const float t0 = ((xv.x - g.x0[0]) * g.inv_h + g.half_ext) - (float)i0[0];
        const float t1 = ((xv.y - g.x0[1]) * g.inv_h + g.half_ext) - (float)i0[1];
        const float t2 = ((xv.z - g.x0[2]) * g.inv_h + g.half_ext) - (float)i0[2];
        if (lane < P) {
            const float d0 = t0 - (float)lane, d1 = t1 - (float)lane, d2 = t2 - (float)lane;
            swt[warp][0][lane] = __expf(-g.ah2 * d0 * d0);
            swt[warp][1][lane] = __expf(-g.ah2 * d1 * d1);
            swt[warp][2][lane] = __expf(-g.ah2 * d2 * d2);
        }
        __syncwarp();
        const int ox = min(max(i0[0] - gx0, 0), TE - 1), oy = min(max(i0[1] - gy0, 0), TE - 1),
                  oz = min(max(i0[2] - gz0, 0), TE - 1);
        float wz[P], wzd[P];
#pragma unroll
        for (int kz = 0; kz < P; kz++) {
            wz[kz] = swt[warp][2][kz];
            wzd[kz] = wz[kz] * (t2 - (float)kz);
        }
        float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f;
#pragma unroll
        for (int it = 0; it < NIT; it++) {
            if (val[it]) {
                const int kx = kxs[it], ky = kys[it];
                const float wxy = swt[warp][0][kx] * swt[warp][1][ky];
                const float *col = sg + oz * ZS + (oy + ky) * PX + ox + kx;
                float a = 0.0f, az = 0.0f;
#pragma unroll
                for (int kz = 0; kz < P; kz++) {
                    const float sv = fmaf(c2, col[2 * CS + kz * ZS], fmaf(c1, col[CS + kz * ZS], c0 * col[kz * ZS]));
                    a = fmaf(wz[kz], sv, a);
                    az = fmaf(wzd[kz], sv, az);
                }
                const float aw = a * wxy;
                acc0 = fmaf(aw, t0 - (float)kx, acc0);
                acc1 = fmaf(aw, t1 - (float)ky, acc1);
                acc2 = fmaf(az, wxy, acc2);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc0 += __shfl_xor_sync(FULL, acc0, o);
            acc1 += __shfl_xor_sync(FULL, acc1, o);
            acc2 += __shfl_xor_sync(FULL, acc2, o);
        }
        if (lane < 3) {
            const size_t o3 = 3 * (size_t)m + lane;
            const float v = c_grad * (lane == 0 ? acc0 : (lane == 1 ? acc1 : acc2));
            gx[o3] = (mode == 0) ? v : gx[o3] + v;
        }
        __syncwarp();
    }
}

template <int P, int TE, bool TMA, int MODE>
__global__ void __launch_bounds__(GS_WARPS * 32) k_gather_adj_smem(GP<float> g, const int *__restrict__ tile_start,
                                                                   const float4 *__restrict__ xs,
                                                                   const int *__restrict__ perm,
                                                                   const float *__restrict__ w,
                                                                   const float *__restrict__ f,
                                                                   const float *__restrict__ q, float *__restrict__ gf,
                                                                   float *__restrict__ gq,
                                                                   const __grid_constant__ CUtensorMap tmap,
                                                                   int *__restrict__ status) {
    const int tile = blockIdx.x;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    const size_t Mf2 = (size_t)g.mf[0] * g.mf[1], Mf3 = Mf2 * g.mf[2];
    gather_smem_body<P, TE, TMA, false, MODE>(g, tile, beg, end, xs, perm, w, 1, 0, f, 0.0, gf, Mf2, Mf3, &tmap,
                                              status, false, q, gq);
}

template <int P, int TE, bool TMA>
__global__ void __launch_bounds__(GS_WARPS * 32) k_grad_smem(GP<float> g, const int *__restrict__ tile_start,
                                                             const float4 *__restrict__ xs,
                                                             const int *__restrict__ perm,
                                                             const float *__restrict__ w, int mode,
                                                             const float *__restrict__ ca,
                                                             const float *__restrict__ cb, float c_grad,
                                                             float *__restrict__ gx,
                                                             const __grid_constant__ CUtensorMap tmap,
                                                             int *__restrict__ status) {
    const int tile = blockIdx.x;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    grad_smem_body<P, TE, TMA>(g, tile, beg, end, xs, perm, w, mode, ca, cb, c_grad, gx, &tmap, status);
}

template <int P, int TE>
__global__ void __launch_bounds__(GS_WARPS * 32) k_bgather_smem(const BSys<float> *__restrict__ sys,
                                                                const int4 *__restrict__ items,
                                                                const int *__restrict__ tile_start, int n_rhs,
                                                                const float4 *__restrict__ xs,
                                                                const int *__restrict__ perm,
                                                                const float *__restrict__ f_orig,
                                                                float *__restrict__ u,
                                                                const CUtensorMap *__restrict__ maps,
                                                                int *__restrict__ status) {
    const int4 it = items[blockIdx.x];
    const BSys<float> &B = sys[it.x];
    const int key = B.tile_base + it.y;
    const int beg = tile_start[key], end = tile_start[key + 1];
    if (beg == end) return;
    const GP<float> g = B.g;
    if (maps && B.tma)
        gather_smem_body<P, TE, true, true>(g, it.y, beg, end, xs, perm, B.wgrid, n_rhs, it.z, f_orig, B.self_coef,
                                            u, B.gzs, B.gcs, maps + it.x, status);
    else
        gather_smem_body<P, TE, false>(g, it.y, beg, end, xs, perm, B.wgrid + (size_t)it.z * 3 * B.gcs, n_rhs,
                                       it.z, f_orig, B.self_coef, u, B.gzs, B.gcs);
}

template <int P, int TE>
constexpr size_t gather_smem_bytes() {
    // + 128: room to align the block to 128 bytes
    return (size_t)3 * (TE + P - 1) * (TE + P - 1) * GsLayout<P, TE + P - 1>::PX * sizeof(float) + 128;
}

template <int P, int TE>
__global__ void __launch_bounds__(ColCfg<P, TE>::NT) k_spread_col(GP<float> g, int c0, bool stress,
                                                                    const int *__restrict__ tile_start,
                                                                    const float4 *__restrict__ xs,
                                                                    const float4 *__restrict__ fs,
                                                                    const float4 *__restrict__ qs,
                                                                    float *__restrict__ grid) {
    const int tile = blockIdx.x;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    spread_col_body<P, TE>(g, tile, beg, end, c0, stress, xs, fs, 1, 0, qs, grid);
}

template <int P, int TE>
__global__ void __launch_bounds__(C2Cfg<P, TE>::NT, P <= 12 ? SE_C2_MINB : 1) k_spread_c2(GP<float> g, int c0, bool stress,
                                                                                const int *__restrict__ tile_start,
                                                                                const float4 *__restrict__ xs,
                                                                                const float4 *__restrict__ fs,
                                                                                const float4 *__restrict__ qs,
                                                                                float *__restrict__ grid,
                                                                                float *__restrict__ tb) {
    extern __shared__ __align__(16) unsigned char c2_smem[];
    const int tile = blockIdx.x;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    const size_t Mf = g.mf[0], Mf2 = Mf * g.mf[1];
    float *tbt = nullptr;
    if constexpr (TE == COL_TE)
        if (tb) tbt = tb + (size_t)tile * TileBufCfg<P>::FLOATS;
    spread_c2_body<P, TE>(g, tile, beg, end, c0, stress, xs, fs, 1, 0, qs, grid, Mf2, Mf2 * g.mf[2],
                          reinterpret_cast<C2Stage<P, TE> *>(c2_smem), tbt);
}

template <int P, int TE>
__global__ void __launch_bounds__(ColCfg<P, TE>::NT) k_gather_col(GP<float> g, const int *__restrict__ tile_start,
                                                                    const float4 *__restrict__ xs,
                                                                    const int *__restrict__ perm,
                                                                    const float *__restrict__ w,
                                                                    const float *__restrict__ f_orig,
                                                                    double self_coef, float *__restrict__ u) {
    const int tile = blockIdx.x;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    gather_col_body<P, TE>(g, tile, beg, end, xs, perm, w, 1, 0, f_orig, self_coef, u);
}

// Batched: one CTA per item (system, tile, right-hand side).
// Batched spreading with the right-hand sides inside the item: one CTA per
// (system, tile), the points' positions and Gaussian weights staged once when
// the tile holds at most NB points (else once per batch of NB), then per
// right-hand side only the sources are loaded, the columns accumulated and
// added to that right-hand side's grids.  items: the (system, tile, rhs)
// list with the right-hand side innermost; block b takes item b * n_rhs.
template <int P, int TE>
__global__ void __launch_bounds__(ColCfg<P, TE>::NT, 2) k_bspread_col_rhs(const BSys<float> *__restrict__ sys,
                                                                         const int4 *__restrict__ items,
                                                                         const int *__restrict__ tile_start,
                                                                         int n_rhs, const float4 *__restrict__ xs,
                                                                         const float4 *__restrict__ fs) {
    using C = ColCfg<P, TE>;
    constexpr int PT = C::PT, NB = C::NB;
    static_assert(TE == 8, "the unrolled z offsets cover tiles of 8");
    __shared__ __align__(16) ColStage<P, TE> S;
    const int4 it = items[(size_t)blockIdx.x * n_rhs];
    const BSys<float> &B = sys[it.x];
    const int key = B.tile_base + it.y;
    const int beg = tile_start[key], end = tile_start[key + 1];
    if (beg == end) return;
    const GP<float> g = B.g;
    const int tile = it.y, tid = threadIdx.x;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int gx0 = tx * TE, gy0 = ty * TE, gz0 = tz * TE;
    const bool own = tid < PT * PT;
    const int cx = tid % PT, cy = tid / PT;
    const bool once = end - beg <= NB;
    if (once) {
        if (tid < end - beg) stage_point<P, TE>(S, g, tid, beg + tid, gx0, gy0, gz0, xs);
        __syncthreads();
        stage_weights<P, TE>(S, g, end - beg);
    }
    const size_t Mf = g.mf[0], Mf2 = B.gzs, Mf3 = B.gcs;  // z-plane and component strides
    for (int r = 0; r < n_rhs; r++) {
        float a0[PT], a1[PT], a2[PT];
#pragma unroll
        for (int z = 0; z < PT; z++) a0[z] = a1[z] = a2[z] = 0.0f;
        for (int b0 = beg; b0 < end; b0 += NB) {
            const int nb = min(NB, end - b0);
            if (tid < nb) {
                if (!once) stage_point<P, TE>(S, g, tid, b0 + tid, gx0, gy0, gz0, xs);
                S.src[tid] = fs[(size_t)(b0 + tid) * n_rhs + r];
            }
            __syncthreads();
            if (!once) {
                stage_weights<P, TE>(S, g, nb);
                __syncthreads();
            }
            if (own) {
                for (int j = 0; j < nb; j++) {
                    const int oxy = S.oxy[j];
                    const int kx = cx - (oxy & 255), ky = cy - (oxy >> 8);
                    if ((unsigned)kx < (unsigned)P && (unsigned)ky < (unsigned)P) {
                        const float w = S.wx[j][kx] * S.wy[j][ky];
                        const float4 sv = S.src[j];
                        const float s0 = sv.x * w, s1 = sv.y * w, s2 = sv.z * w;
                        const int oz = S.oz[j];
                        SE_COL_CASES(col_add, a0, a1, a2, s0, s1, s2, S.wz[j])
                    }
                }
            }
            __syncthreads();
        }
        if (own) {
            const int gx = gx0 + cx, gy = gy0 + cy;
            if (gx < g.mt[0] && gy < g.mt[1]) {
                float *base = B.grid + (size_t)r * 3 * Mf3 + (size_t)gz0 * Mf2 + (size_t)gy * Mf + gx;
#pragma unroll
                for (int z = 0; z < PT; z++) {
                    if (gz0 + z < g.mt[2]) {
                        float *pz = base + (size_t)z * Mf2;
                        if (a0[z] != 0.0f) atomicAdd(pz, a0[z]);
                        if (a1[z] != 0.0f) atomicAdd(pz + Mf3, a1[z]);
                        if (a2[z] != 0.0f) atomicAdd(pz + 2 * Mf3, a2[z]);
                    }
                }
            }
        }
    }
}

// Batched paired spreading: one CTA per (system, tile) with the right-hand
// sides inside the item.  A tile of at most NB points is staged once (positions
// and weights) and only its sources are staged again per right-hand side;
// larger tiles are staged batch by batch for every right-hand side.  items:
// the (system, tile, rhs) list with the right-hand side innermost; block b
// takes item b * n_rhs.
template <int P, int TE>
__global__ void __launch_bounds__(C2Cfg<P, TE>::NT, P <= 12 ? SE_C2_MINB : 1) k_bspread_c2(const BSys<float> *__restrict__ sys,
                                                                                 const int4 *__restrict__ items,
                                                                                 const int *__restrict__ tile_start,
                                                                                 int n_rhs,
                                                                                 const float4 *__restrict__ xs,
                                                                                 const float4 *__restrict__ fs) {
    using C = C2Cfg<P, TE>;
    constexpr int PT = C::PT, ZP = C::ZP, NB = C::NB;
    extern __shared__ __align__(16) unsigned char c2_smem[];
    C2Stage<P, TE> *S = reinterpret_cast<C2Stage<P, TE> *>(c2_smem);
    const int4 it = items[(size_t)blockIdx.x * n_rhs];
    const BSys<float> &B = sys[it.x];
    const int key = B.tile_base + it.y;
    const int beg = tile_start[key], end = tile_start[key + 1];
    if (beg == end) return;
    const GP<float> g = B.g;
    const int tile = it.y, tid = threadIdx.x;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int gx0 = tx * TE, gy0 = ty * TE, gz0 = tz * TE;
    int cx, cy, cyl, cyh;
    c2_column<P, TE>(tid, cx, cy, cyl, cyh);
    const bool once = end - beg <= NB;
    for (int r = 0; r < n_rhs; r++) {
        float2 a0[ZP], a1[ZP], a2[ZP];
#pragma unroll
        for (int q = 0; q < ZP; q++) a0[q] = a1[q] = a2[q] = make_float2(0.0f, 0.0f);
        if (once) {
            if (r == 0) {
                c2_stage<P, TE>(S[0], g, beg, end - beg, gx0, gy0, gz0, 0, false, xs, fs, n_rhs, 0, nullptr);
            } else if (tid < end - beg) {
                S[0].rec[tid].src = fs[(size_t)(beg + tid) * n_rhs + r];
            }
            __syncthreads();
            c2_accumulate<P, TE>(S[0], end - beg, cx, cy, cyl, cyh, a0, a1, a2);
            __syncthreads();
        } else {
            c2_stage<P, TE>(S[0], g, beg, NB, gx0, gy0, gz0, 0, false, xs, fs, n_rhs, r, nullptr);
            __syncthreads();
            int k = 0;
            for (int b0 = beg; b0 < end; b0 += NB, k ^= 1) {
                const int nb = min(NB, end - b0);
                if (b0 + NB < end)
                    c2_stage<P, TE>(S[k ^ 1], g, b0 + NB, min(NB, end - b0 - NB), gx0, gy0, gz0, 0, false, xs, fs,
                                    n_rhs, r, nullptr);
                c2_accumulate<P, TE>(S[k], nb, cx, cy, cyl, cyh, a0, a1, a2);
                __syncthreads();
            }
        }
        if (tid < PT * PT)
            c2_flush<P, TE>(g, gx0 + cx, gy0 + cy, gz0, a0, a1, a2, B.grid + (size_t)r * 3 * B.gcs, B.gzs, B.gcs);
    }
}

// Dispatch on the (even) support P, 4 <= P <= 16.
template <template <int, int> class F, typename... A>
cudaError_t with_p(int P, A... a) {
    switch (P) {
        case 4: return F<4, COL_TE>::run(a...);
        case 6: return F<6, COL_TE>::run(a...);
        case 8: return F<8, COL_TE>::run(a...);
        case 10: return F<10, COL_TE>::run(a...);
        case 12: return F<12, COL_TE>::run(a...);
        case 14: return F<14, COL_TE>::run(a...);
        case 16: return F<16, COL_TE>::run(a...);
        default: return cudaErrorInvalidValue;
    }
}

// SE_SPREAD_SUB: plans and batches with P = 10 or 12 spread on sub-tiles of 4 x 4
// x 8 window starts (k_spread_sub, k_bspread_sub in subtile.cu); 0 keeps the
// 8^3-tile kernels
#ifndef SE_SPREAD_SUB
#define SE_SPREAD_SUB 1
#endif

// SE_SPREAD_PAIR: the paired-FMA spreading kernel (k_spread_c2); 0 keeps the
// scalar register-column kernel (k_spread_col)
#ifndef SE_SPREAD_PAIR
#define SE_SPREAD_PAIR 1
#endif

template <int P, int TE>
struct SpreadRun {
    // tb: the tile buffer of a deterministic plan (the paired kernel only), else NULL
    static cudaError_t run(const GP<float> g, int ntiles, int c0, bool stress, const int *ts, const float4 *xs,
                           const float4 *fs, const float4 *qs, float *grid, float *tb, cudaStream_t st) {
        if (SE_SPREAD_PAIR || tb) {
            constexpr size_t smem = c2_smem_bytes<P, TE>();
            cudaError_t e =
                cudaFuncSetAttribute(k_spread_c2<P, TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e) return e;
            k_spread_c2<P, TE><<<ntiles, C2Cfg<P, TE>::NT, smem, st>>>(g, c0, stress, ts, xs, fs, qs, grid, tb);
        } else {
            k_spread_col<P, TE><<<ntiles, ColCfg<P, TE>::NT, 0, st>>>(g, c0, stress, ts, xs, fs, qs, grid);
        }
        return cudaGetLastError();
    }
};

#ifndef SE_GATHER_SMEM
#define SE_GATHER_SMEM 1
#endif

// SE_GATHER_SUB: plans with P = 10 or 12 gather on sub-tiles with register
// columns (k_gather_sub, subtile.cu); 0 keeps the tensor-copy tile gather
#ifndef SE_GATHER_SUB
#define SE_GATHER_SUB 1
#endif

#ifndef SE_GATHER_TMA
#define SE_GATHER_TMA 1
#endif

// cuTensorMapEncodeTiled from the driver (through the runtime: no link to libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        }
        return (PFN_cuTensorMapEncodeTiled_v12000)f;
    }();
    return fn;
}

// The gather grids as a 4-D FP32 tensor (x, y, z, component) of extent
// (Mt_x, Mt_y, Mt_z, 3) with row, plane and component strides Mf_x, gzs, gcs
// (elements), read in boxes of PX x PT x PT x 3.  False when a tensor copy
// cannot describe it (strides or base not 16-byte aligned, a box wider than
// the grid, no encoder): the caller stages with plain loads instead.
static bool encode_gather_map(CUtensorMap *map, const GP<float> &g, const float *w, size_t gzs, size_t gcs, int PX,
                              int PT) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const size_t rs = (size_t)g.mf[0] * sizeof(float), ps = gzs * sizeof(float), cs = gcs * sizeof(float);
    if ((reinterpret_cast<uintptr_t>(w) & 15) || (rs & 15) || (ps & 15) || (cs & 15)) return false;
    if (g.mt[0] < PX || g.mt[1] < PT || g.mt[2] < PT) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.mt[0], (cuuint64_t)g.mt[1], (cuuint64_t)g.mt[2], 3};
    const cuuint64_t strides[3] = {rs, ps, cs};
    const cuuint32_t box[4] = {(cuuint32_t)PX, (cuuint32_t)PT, (cuuint32_t)PT, 3};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(w), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int P, int TE>
struct GatherRun {
    static cudaError_t run(const GP<float> g, int ntiles, const int *ts, const float4 *xs, const int *perm,
                           const float *w, const float *f, double self_coef, float *u, int *status, int skip_copy,
                           cudaStream_t st) {
        if (SE_GATHER_SMEM) {
            constexpr int PT = TE + P - 1, PX = GsLayout<P, PT>::PX;
            const size_t smem = gather_smem_bytes<P, TE>();
            alignas(64) CUtensorMap map;
            memset(&map, 0, sizeof(map));
            const bool tma = SE_GATHER_TMA && encode_gather_map(&map, g, w, (size_t)g.mf[0] * g.mf[1], vol(g), PX, PT);
            auto kern = tma ? k_gather_smem<P, TE, true> : k_gather_smem<P, TE, false>;
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e) return e;
            kern<<<ntiles, GS_WARPS * 32, smem, st>>>(g, ts, xs, perm, w, f, self_coef, u, map, status,
                                                      tma ? skip_copy : 0);
        } else {
            k_gather_col<P, TE><<<ntiles, ColCfg<P, TE>::NT, 0, st>>>(g, ts, xs, perm, w, f, self_coef, u);
        }
        return cudaGetLastError();
    }
};

template <int P, int TE>
struct GatherAdjRun {
    // the two passes over V (diagonal, then off-diagonal grids)
    static cudaError_t run(const GP<float> g, int ntiles, const int *ts, const float4 *xs, const int *perm,
                           const float *V, const float *f, const float *q, float *gf, float *gq, int *status,
                           cudaStream_t st) {
        constexpr int PT = TE + P - 1, PX = GsLayout<P, PT>::PX;
        const size_t smem = gather_smem_bytes<P, TE>();
        const size_t Mf2 = (size_t)g.mf[0] * g.mf[1], Mf3 = vol(g);
        for (int pass = 0; pass < 2; pass++) {
            const float *w = V + (size_t)pass * 3 * Mf3;
            alignas(64) CUtensorMap map;
            memset(&map, 0, sizeof(map));
            const bool tma = SE_GATHER_TMA && encode_gather_map(&map, g, w, Mf2, Mf3, PX, PT);
            auto kern = pass == 0 ? (tma ? k_gather_adj_smem<P, TE, true, 1> : k_gather_adj_smem<P, TE, false, 1>)
                                  : (tma ? k_gather_adj_smem<P, TE, true, 2> : k_gather_adj_smem<P, TE, false, 2>);
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e) return e;
            kern<<<ntiles, GS_WARPS * 32, smem, st>>>(g, ts, xs, perm, w, f, q, gf, gq, map, status);
            if ((e = cudaGetLastError())) return e;
        }
        return cudaSuccess;
    }
};

template <int P, int TE>
struct GradRun {
    static cudaError_t run(const GP<float> g, int ntiles, const int *ts, const float4 *xs, const int *perm,
                           const float *w, int mode, const float *ca, const float *cb, float c_grad, float *gx,
                           int *status, cudaStream_t st) {
        constexpr int PT = TE + P - 1, PX = GsLayout<P, PT>::PX;
        const size_t smem = gather_smem_bytes<P, TE>();
        alignas(64) CUtensorMap map;
        memset(&map, 0, sizeof(map));
        const bool tma = SE_GATHER_TMA && encode_gather_map(&map, g, w, (size_t)g.mf[0] * g.mf[1], vol(g), PX, PT);
        auto kern = tma ? k_grad_smem<P, TE, true> : k_grad_smem<P, TE, false>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e) return e;
        kern<<<ntiles, GS_WARPS * 32, smem, st>>>(g, ts, xs, perm, w, mode, ca, cb, c_grad, gx, map, status);
        return cudaGetLastError();
    }
};

template <int P, int TE>
struct BSpreadRun {
    static cudaError_t run(const BSys<float> *sys, const int4 *items, int nitems, const int *ts, int n_rhs,
                           const float4 *xs, const float4 *fs, cudaStream_t st) {
        if (SE_SPREAD_PAIR) {
            constexpr size_t smem = c2_smem_bytes<P, TE>();
            cudaError_t e =
                cudaFuncSetAttribute(k_bspread_c2<P, TE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e) return e;
            k_bspread_c2<P, TE><<<nitems / n_rhs, C2Cfg<P, TE>::NT, smem, st>>>(sys, items, ts, n_rhs, xs, fs);
        } else {
            k_bspread_col_rhs<P, TE><<<nitems / n_rhs, ColCfg<P, TE>::NT, 0, st>>>(sys, items, ts, n_rhs, xs, fs);
        }
        return cudaGetLastError();
    }
};

template <int P, int TE>
struct BGatherRun {
    // the plane-interleaved FP32 batch grids are read by the shared-memory gather
    static cudaError_t run(const BSys<float> *sys, const int4 *items, int nitems, const int *ts, int n_rhs,
                           const float4 *xs, const int *perm, const float *f, float *u, const CUtensorMap *maps,
                           int *status, cudaStream_t st) {
        const size_t smem = gather_smem_bytes<P, TE>();
        cudaError_t e = cudaFuncSetAttribute(k_bgather_smem<P, TE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e) return e;
        k_bgather_smem<P, TE><<<nitems, GS_WARPS * 32, smem, st>>>(sys, items, ts, n_rhs, xs, perm, f, u, maps,
                                                                    status);
        return cudaGetLastError();
    }
};

}  // namespace

bool col_supported(int prec, int P) { return prec == SE_FP32 && P >= 4 && P <= 16 && (P % 2) == 0; }

bool spread_uses_sub(const se_plan_s *p) {
    // sub-tiles pay off from about 100 points per 8^3 tile on (N = 1e6: 296
    // per tile at M = 114, 0.95 -> 0.59 ms; 94 at M = 168, 1.06 ms both ways)
    return SE_SPREAD_SUB && p->colk && sub_supported(p->P) && p->N >= 128 * (int64_t)p->ntiles;
}

cudaError_t launch_spread_col(se_plan_s *p, cudaStream_t st, const void *xs, const void *fs, const void *qs,
                              void *grid, int nc) {
    // nc = 3: f; nc = 6: the symmetric stresslet source in two passes of three.
    // Deterministic plans: each tile's padded block goes to the tile buffer and
    // a second kernel adds the tiles into the grid in a fixed order, no
    // atomics (the caller skips the zeroing)
    const bool sub = spread_uses_sub(p);
    const bool det = p->deterministic && p->tilebuf;
    for (int c0 = 0; c0 < nc; c0 += 3) {
        cudaError_t e;
        const int *ts = (const int *)p->b.cnt_t;
        if (sub && det) {
            e = launch_spread_sub_tb(p->gpf, p->ntiles, c0, nc == 6, ts, (const float4 *)xs, (const float4 *)fs,
                                     (const float4 *)qs, p->tilebuf, st);
        } else if (sub) {
            e = launch_spread_sub(p->gpf, p->ntiles, c0, nc == 6, ts, (const float4 *)xs, (const float4 *)fs,
                                  (const float4 *)qs, (float *)grid, st);
        } else {
            e = with_p<SpreadRun>(p->P, p->gpf, p->ntiles, c0, nc == 6, ts, (const float4 *)xs, (const float4 *)fs,
                                  (const float4 *)qs, (float *)grid, det ? p->tilebuf : nullptr, st);
        }
        if (e) return e;
        p->launches++;
        if (det) {
            if ((e = launch_merge_tiles(p->gpf, ts, p->tilebuf, (float *)grid, c0, st))) return e;
            p->launches++;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_gather_col(se_plan_s *p, cudaStream_t st, const void *wgrid, const float *f_orig, float *u) {
    const double self_coef = (p->kernel == SE_STOKESLET) ? -4.0 * p->xi / sqrt(M_PI) : 0.0;
    return launch_gather_col_set(p, st, p->b, wgrid, f_orig, self_coef, u, p->N);
}

cudaError_t launch_gather_col_set(se_plan_s *p, cudaStream_t st, const Buffers &b, const void *wgrid,
                                  const float *f_orig, double self_coef, float *u, int64_t n_pts) {
    // the sub-tile gather (P = 10, 12) from 256 points per 8^3 tile on (N =
    // 1e6: 296 per tile at M = 114, 0.835 -> 0.79 ms; 94 per tile at M = 168,
    // 1.37 ms against 0.90 ms; a cost per tile linear in its points puts the
    // crossing near 250); the tiles of the failure-path test flag are those of
    // the tensor-copy gather
    if (SE_GATHER_SUB && sub_supported(p->P) && n_pts >= 256 * (int64_t)p->ntiles &&
        !(p->test_flags & SE_TEST_SKIP_TILE_COPY)) {
        cudaError_t e = launch_gather_sub(p->gpf, p->ntiles, (const int *)b.cnt_t, (const float4 *)b.xs_t,
                                          (const int *)b.perm_t, (const float *)wgrid, f_orig, self_coef, u, st);
        if (!e) p->launches++;
        return e;
    }
    cudaError_t e = with_p<GatherRun>(p->P, p->gpf, p->ntiles, (const int *)b.cnt_t, (const float4 *)b.xs_t,
                                      (const int *)b.perm_t, (const float *)wgrid, f_orig, self_coef, u,
                                      p->b.status, p->test_flags & SE_TEST_SKIP_TILE_COPY, st);
    if (!e) p->launches++;
    return e;
}

cudaError_t launch_gather_adj_col(se_plan_s *p, cudaStream_t st, const float *V, const float *f, const float *q,
                                  float *gf, float *gq) {
    cudaError_t e = with_p<GatherAdjRun>(p->P, p->gpf, p->ntiles, (const int *)p->b.cnt_t, (const float4 *)p->b.xs_t,
                                         (const int *)p->b.perm_t, V, f, q, gf, gq, p->b.status, st);
    if (!e) p->launches += 2;
    return e;
}

cudaError_t launch_gather_grad_col(se_plan_s *p, cudaStream_t st, const float *w_fwd, const float *w_adj,
                                   const float *f_orig, const float *q_orig, const float *g_orig, float *gx) {
    const float c_grad = (float)(-2.0 * p->geom.a * p->h);
    const int *ts = (const int *)p->b.cnt_t;
    const float4 *xs = (const float4 *)p->b.xs_t;
    const size_t Mf3 = vol(p->gpf);
    // the forward field against g, then the adjoint field against f (or the
    // stresslet's f q pairs, in two groups of three)
    struct Pass {
        const float *w;
        int mode;
        const float *a, *b;
    };
    Pass passes[3] = {{w_fwd, 0, g_orig, nullptr}, {w_adj, 1, f_orig, nullptr}, {nullptr, 0, nullptr, nullptr}};
    int np = 2;
    if (p->kernel == SE_STRESSLET) {
        passes[1] = {w_adj, 2, f_orig, q_orig};
        passes[2] = {w_adj + 3 * Mf3, 3, f_orig, q_orig};
        np = 3;
    }
    for (int i = 0; i < np; i++) {
        cudaError_t e = with_p<GradRun>(p->P, p->gpf, p->ntiles, ts, xs, (const int *)p->b.perm_t, passes[i].w,
                                        passes[i].mode, passes[i].a, passes[i].b, c_grad, gx, p->b.status, st);
        if (e) return e;
        p->launches++;
    }
    return cudaSuccess;
}

cudaError_t launch_bspread_col(const BSys<float> *sys, const int4 *items, int nitems, int P, int n_rhs,
                               const Buffers &b, cudaStream_t st) {
    if (SE_SPREAD_SUB && sub_supported(P))
        return launch_bspread_sub(sys, items, nitems, P, n_rhs, (const int *)b.cnt_t, (const float4 *)b.xs_t,
                                  (const float4 *)b.fs_t, st);
    return with_p<BSpreadRun>(P, sys, items, nitems, (const int *)b.cnt_t, n_rhs, (const float4 *)b.xs_t,
                              (const float4 *)b.fs_t, st);
}

cudaError_t launch_bgather_col(const BSys<float> *sys, const int4 *items, int nitems, int P, int n_rhs,
                               const Buffers &b, const float *f, float *u, const void *maps, cudaStream_t st) {
    return with_p<BGatherRun>(P, sys, items, nitems, (const int *)b.cnt_t, n_rhs, (const float4 *)b.xs_t,
                              (const int *)b.perm_t, f, u, (const CUtensorMap *)maps, (int *)b.status, st);
}

// The tensor map of one system's interleaved batch grids (FP32): a 4-D FP32
// tensor (x, y, component, z) of extent (Mt_x, Mt_y, 3 n_rhs, Mt_z) with
// strides (1, Mf_x, gcs, gzs) elements, read in boxes of PX x PT x 3 x PT.
bool encode_bgather_map(void *map, const GP<float> &g, const float *wgrid, size_t gzs, size_t gcs, int n_rhs,
                        int P) {
    if (!SE_GATHER_TMA || !col_supported(SE_FP32, P)) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const int PT = COL_TE + P - 1;
    int PX = 0;
    switch (P) {
        case 4: PX = GsLayout<4, COL_TE + 3>::PX; break;
        case 6: PX = GsLayout<6, COL_TE + 5>::PX; break;
        case 8: PX = GsLayout<8, COL_TE + 7>::PX; break;
        case 10: PX = GsLayout<10, COL_TE + 9>::PX; break;
        case 12: PX = GsLayout<12, COL_TE + 11>::PX; break;
        case 14: PX = GsLayout<14, COL_TE + 13>::PX; break;
        case 16: PX = GsLayout<16, COL_TE + 15>::PX; break;
        default: return false;
    }
    const size_t rs = (size_t)g.mf[0] * sizeof(float), cs = gcs * sizeof(float), zs = gzs * sizeof(float);
    if ((reinterpret_cast<uintptr_t>(wgrid) & 15) || (rs & 15) || (cs & 15) || (zs & 15)) return false;
    if (g.mt[0] < PX || g.mt[1] < PT || g.mt[2] < PT) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.mt[0], (cuuint64_t)g.mt[1], (cuuint64_t)(3 * n_rhs),
                                (cuuint64_t)g.mt[2]};
    const cuuint64_t strides[3] = {rs, cs, zs};
    const cuuint32_t box[4] = {(cuuint32_t)PX, (cuuint32_t)PT, 3, (cuuint32_t)PT};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return enc((CUtensorMap *)map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(wgrid), dims, strides,
               box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace se
