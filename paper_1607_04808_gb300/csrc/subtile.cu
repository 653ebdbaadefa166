// FP32 spreading (step 1, eq. Hx) on sub-tiles of 4 x 4 x 8 window starts with
// the padded grid block in registers.
//
// A spreading tile (8^3 window starts, the binning's unit) is split into four
// sub-tiles of 4 x 4 window starts in (x, y), all 8 in z; one CTA takes one
// sub-tile and filters the tile's points down to its own.  The supports of its
// points cover a padded block of PT x PT columns, PT = 4 + P - 1 (15 at P =
// 12), each PZ = 8 + P - 1 grid points long in z.  Thread (cx, cy) keeps the
// columns (cx, cy) and (cx, cy + 1) of the three source components in
// registers as z pairs and adds every point whose support covers them with
// paired FP32 FMAs (two z values per instruction); the point's z weights and
// source, read once from shared memory, serve both columns.  A warp owns four
// rows of columns (two groups of PT lanes), so a point's P x P support meets 3
// or 4 of the 4 warps and covers P of the PT columns of each of their rows.
//
// Each batch of staged points is stored in the order of the key (oz, oy) of
// its window start in the block (ranks within warps, counts combined over the
// batch), so a warp runs, for each z offset oz in turn (a compile-time
// constant: register indices must be constants), the contiguous run of
// records whose support meets its rows: no per-point branch on oz and no
// per-point test.  The columns go to the FFT input once per CTA through shared
// memory with 16-byte vector atomics (sub-tiles overlap in their halos).
#include <cooperative_groups.h>

#include "se_internal.cuh"

namespace se {

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int SUB = 4;  // sub-tile edge in x and y (window starts)

template <int P>
struct SubCfg {
    static constexpr int TE = COL_TE;              // tile edge (window starts); the sub-tile's z extent
    static constexpr int PT = SUB + P - 1;         // columns per row and rows of the padded block
    static constexpr int PZ = TE + P - 1;          // grid points per column
    static constexpr int ZP = (PZ + 1) / 2;        // z pairs per column and component
    static constexpr int TR = 2;                   // rows of columns per thread (cy, cy + 1)
    static constexpr int LR = 32 / PT;             // groups of PT lanes per warp
    static constexpr int RW = LR * TR;             // rows of columns per warp
    static constexpr int NW = (PT + RW - 1) / RW;  // warps
    static constexpr int NT = 32 * NW;
    static constexpr int WXY = 16;                 // x and y weights per record, zero slots for idle lanes
    static constexpr int WP = P / 2 + 1;           // staged z-weight pairs (odd offsets need P/2 + 1)
    static constexpr int WP4 = (WP + 1) / 2 * 2;   // in whole 16-byte rows
    static constexpr int NB = NT;                  // points per staged batch (one staging thread each)
    static constexpr int NCH = NB / 32;            // chunks of 32 points (one warp each)
    static constexpr int NKEY = TE * SUB;          // keys oz * SUB + oy
    static constexpr int CAP = 2048;               // tile points examined per round
    static constexpr int FX = 16;                  // x extent of the flush buffer (whole float4 of grid points)
    static_assert(PT + 1 <= WXY && RW * NW <= WXY, "a weight for every column and row, idle slots included");
    static_assert(NKEY == 32, "one key per lane in the start table");
    static_assert(PT <= FX, "a row of the block in the flush buffer");
    static_assert(NB <= 255, "record indices in one byte");
};

// One staged point: everything a column thread reads, in one record.
template <int P>
struct __align__(16) SubRec {
    float4 wz[SubCfg<P>::WP4 / 2];  // z weights as pairs, from slot (oz & 1) on, zeros elsewhere
    float4 sxy;                     // (s0, s0, s1, s1): source components duplicated for the pairs
    float2 sz;                      // (s2, s2)
    int n;                          // the point's index in the sorted arrays (gather)
    int pad_;
    float wx[SubCfg<P>::WXY];       // x weight of every column of the block (0 off the support)
    float wy[SubCfg<P>::WXY];
};

template <int P>
struct SubStage {
    using C = SubCfg<P>;
    SubRec<P> rec[C::NB];
    unsigned char slot[C::NB];         // staged point j goes to rec[slot[j]]: the batch in key order
    unsigned char kst[C::NKEY + 1];    // points with key k: records kst[k] .. kst[k + 1]
    unsigned char cnt[C::NCH][C::NKEY];  // points per key in each chunk of 32
};

// Shared memory of one CTA (dynamic): two staging buffers, reused as the flush
// buffer (the block's columns, x fastest in rows of FX) once the last batch is
// done, and the round's list of the sub-tile's points.
template <int P>
struct SubSmem {
    union {
        SubStage<P> S[2];
        float F[3][SubCfg<P>::PZ][SubCfg<P>::PT][SubCfg<P>::FX];
    };
    unsigned short list[SubCfg<P>::CAP];
    int wc[SubCfg<P>::NW];
};

// Stage the points list[b0 .. b0 + nb) of the round starting at tbeg (indices
// into the sorted arrays: tbeg + list[i]) in key order: thread j finds the key
// of point j and its place in the batch's key order, then writes the point's
// record there (its x, y and z weights and its source).  Called by every
// thread of the CTA (it holds a CTA barrier).
template <int P, bool GATHER = false>
__device__ __forceinline__ void sub_stage(SubStage<P> &S, const GP<float> &g, const float4 *__restrict__ xs,
                                          const float4 *__restrict__ fs, const float4 *__restrict__ qs, int fstride,
                                          int foff, int c0, bool stress, const unsigned short *list, int tbeg,
                                          int b0, int nb, int gx0, int gy0, int gz0) {
    using C = SubCfg<P>;
    const int j = threadIdx.x, lane = j & 31, ch = j >> 5;
    const bool valid = j < nb;
    int n = 0, i0[3] = {0, 0, 0};
    float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
    int key = C::NKEY;  // past every key: an empty slot of the last batch
    int oz = 0;
    if (valid) {
        n = tbeg + list[b0 + j];
        xv = xs[n];
        unpack3(get_tag(xv), i0[0], i0[1], i0[2]);
        oz = min(max(i0[2] - gz0, 0), C::TE - 1);
        key = oz * SUB + min(max(i0[1] - gy0, 0), SUB - 1);
    }
    // the chunk's points with the same key, this point's rank among them, and
    // the chunk's count of every key
    const unsigned same = __match_any_sync(FULLM, key);
    const int within = __popc(same & ((1u << lane) - 1u));
    const int kcount = (valid && within == 0) ? __popc(same) : 0;
    S.cnt[ch][lane] = 0;
    __syncwarp();
    if (kcount) S.cnt[ch][key] = (unsigned char)kcount;
    __syncthreads();
    int tot = 0, pre = 0;
#pragma unroll
    for (int c = 0; c < C::NCH; c++) {
        const int v = S.cnt[c][lane];
        tot += v;
        pre += (c < ch) ? v : 0;
    }
    // exclusive scan of the totals over the keys: start of key `lane`
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULLM, incl, o);
        if (lane >= o) incl += v;
    }
    const int kstart = incl - tot;
    if (ch == 0) {
        S.kst[lane] = (unsigned char)kstart;
        if (lane == 31) S.kst[C::NKEY] = (unsigned char)incl;
    }
    const int slot = __shfl_sync(FULLM, kstart + pre, key & 31) + within;
    if (!valid) return;
    SubRec<P> &R = S.rec[slot];
    {
        // the P z weights at slots (oz & 1) .. (oz & 1) + P - 1, zeros elsewhere
        const float fr = ((xv.z - g.x0[2]) * g.inv_h + g.half_ext) - (float)i0[2];
        float *w = reinterpret_cast<float *>(R.wz);
        const int sh = oz & 1;
#pragma unroll
        for (int i = 0; i < 2 * C::WP4; i++) {
            const int kk = i - sh;
            const float tt = fr - (float)kk;
            w[i] = (kk >= 0 && kk < P) ? __expf(-g.ah2 * tt * tt) : 0.0f;
        }
    }
    // weights of every column and row of the block: zero off the point's support
#pragma unroll
    for (int d = 0; d < 2; d++) {
        const float xd = d == 0 ? xv.x : xv.y;
        const float x0 = d == 0 ? g.x0[0] : g.x0[1];
        const int id = d == 0 ? i0[0] : i0[1];
        const int o = min(max(id - (d == 0 ? gx0 : gy0), 0), SUB - 1);
        const float fr = ((xd - x0) * g.inv_h + g.half_ext) - (float)id;
        float *w = d == 0 ? R.wx : R.wy;
#pragma unroll
        for (int c = 0; c < C::WXY; c++) {
            const int kk = c - o;
            const float tt = fr - (float)kk;
            w[c] = (kk >= 0 && kk < P) ? __expf(-g.ah2 * tt * tt) : 0.0f;
        }
    }
    R.n = n;
    if (GATHER) return;
    const float4 fv = fs[(size_t)n * fstride + foff];
    float4 sv = fv;
    if (stress) {
        // components c0 .. c0 + 2 of the symmetric source (xx, yy, zz, xy, xz, yz)
        const float4 qv = qs[n];
        if (c0 == 0)
            sv = make_float4(fv.x * qv.x, fv.y * qv.y, fv.z * qv.z, 0.0f);
        else
            sv = make_float4(0.5f * (fv.x * qv.y + fv.y * qv.x), 0.5f * (fv.x * qv.z + fv.z * qv.x),
                             0.5f * (fv.y * qv.z + fv.z * qv.y), 0.0f);
    }
    R.sxy = make_float4(sv.x, sv.x, sv.y, sv.y);
    R.sz = make_float2(sv.z, sv.z);
}

// Accumulators of a thread: rows r = 0, 1 (columns (cx, cy + r)), components
// c, z pairs q
template <int P>
using SubAcc = float2[SubCfg<P>::TR][3][SubCfg<P>::ZP];

// a[r][c][OZ/2 + k] += w_r s_c wz[k] for the point's z pairs (P/2, or P/2 + 1
// for odd OZ), w_r = wx[cx] wy[cy + r]
template <int P, int OZ>
__device__ __forceinline__ void sub_point(const SubRec<P> &R, int cx, int cy, SubAcc<P> &a) {
    constexpr int Q0 = OZ / 2, NP = P / 2 + (OZ & 1);
    static_assert(Q0 + NP <= SubCfg<P>::ZP, "the point's z support stays inside the column");
    const float wxv = R.wx[cx];
    const float2 wyv = *reinterpret_cast<const float2 *>(&R.wy[cy]);
    const float4 sv = R.sxy;
    const float2 sz = R.sz;
    float2 s[2][3];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const float w = wxv * (r ? wyv.y : wyv.x);
        const float2 ww = make_float2(w, w);
        s[r][0] = __fmul2_rn(ww, make_float2(sv.x, sv.y));
        s[r][1] = __fmul2_rn(ww, make_float2(sv.z, sv.w));
        s[r][2] = __fmul2_rn(ww, sz);
    }
#pragma unroll
    for (int k2 = 0; k2 < (NP + 1) / 2; k2++) {
        const float4 v = R.wz[k2];
        const float2 lo = make_float2(v.x, v.y), hi = make_float2(v.z, v.w);
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                a[r][c][Q0 + 2 * k2] = __ffma2_rn(lo, s[r][c], a[r][c][Q0 + 2 * k2]);
                if (2 * k2 + 1 < NP) a[r][c][Q0 + 2 * k2 + 1] = __ffma2_rn(hi, s[r][c], a[r][c][Q0 + 2 * k2 + 1]);
            }
    }
}

// The batch's records with z offset OZ, OZ + 1, ... whose oy lies in [ylo, yhi].
template <int P, int OZ>
__device__ __forceinline__ void sub_runs(const SubStage<P> &S, int ylo, int yhi, int cx, int cy, SubAcc<P> &a) {
    if constexpr (OZ < SubCfg<P>::TE) {
        const int i0 = S.kst[OZ * SUB + ylo], i1 = S.kst[OZ * SUB + yhi + 1];
        for (int i = i0; i < i1; i++) sub_point<P, OZ>(S.rec[i], cx, cy, a);
        sub_runs<P, OZ + 1>(S, ylo, yhi, cx, cy, a);
    }
}

// The points of tile points rb .. rb + rn (window starts from the tags) that
// lie in sub-tile (sx, sy) of the tile starting at (tx0, ty0): their offsets
// from rb go to list in increasing order, their count is returned.  Each
// chunk of NT points is compacted by warp ballots and a prefix over the
// warps' counts, so the list does not depend on the order in which threads
// run.  Called by every thread of the CTA (it holds CTA barriers; the first
// also orders the previous round's reads of the list before it is rewritten).
template <int NT>
__device__ __forceinline__ int sub_filter(const int *__restrict__ tags, int rb, int rn, int tx0, int ty0, int sx,
                                          int sy, unsigned short *list, int *wc) {
    constexpr int NWF = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int base = 0;
    for (int k0 = 0; k0 < rn; k0 += NT) {
        const int k = k0 + tid;
        bool in = false;
        if (k < rn) {
            int a, b, c;
            unpack3(__ldg(tags + 4 * (size_t)(rb + k) + 3), a, b, c);
            const int lx = min(max(a - tx0, 0), COL_TE - 1), ly = min(max(b - ty0, 0), COL_TE - 1);
            in = (lx >> 2) == sx && (ly >> 2) == sy;
        }
        const unsigned m = __ballot_sync(FULLM, in);
        __syncthreads();
        if (lane == 0) wc[w] = __popc(m);
        __syncthreads();
        int off = base, tot = 0;
#pragma unroll
        for (int i = 0; i < NWF; i++) {
            const int c = wc[i];
            off += (i < w) ? c : 0;
            tot += c;
        }
        if (in) list[off + __popc(m & ((1u << lane) - 1u))] = (unsigned short)k;
        base += tot;
    }
    __syncthreads();
    return base;
}


// The four sub-tiles of a tile run as one cluster of CTAs (rank = sub-tile).
// Once all four hold their columns in shared memory (F, rows of FX with zero
// padding), CTA `sub` forms the planes pl = sub, sub + 4, ... of the tile's
// padded block by adding the four sub-tiles' values from distributed shared
// memory in a fixed order (sub-tile 0 to 3), and stores them to the tile
// buffer tb.  The second cluster barrier keeps every CTA's shared memory alive
// until the other three have read it.
template <int P>
__device__ __forceinline__ void tile_combine(SubSmem<P> &sm, float *__restrict__ tb, int sub) {
    using C = SubCfg<P>;
    using B = TileBufCfg<P>;
    static_assert(C::PZ == B::PE, "a sub-tile's columns span the tile's z extent");
    static_assert(C::FX % 4 == 0 && C::FX >= C::PT, "whole float4 rows in the flush buffer");
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const float *Fs[4];
#pragma unroll
    for (int s = 0; s < 4; s++) Fs[s] = cl.map_shared_rank(&sm.F[0][0][0][0], (unsigned)s);
    constexpr int PER = B::PE * B::NQ;  // float4 of one plane
    const int npl = (3 * B::PE - sub + 3) / 4;
    for (int i = threadIdx.x; i < npl * PER; i += C::NT) {
        const int k = i / PER, r = i - k * PER;
        const int pl = sub + 4 * k, y = r / B::NQ, x = 4 * (r - (r / B::NQ) * B::NQ);
        float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int s = 0; s < 4; s++) {
            const int yl = y - SUB * (s >> 1), xl = x - SUB * (s & 1);
            if (yl >= 0 && yl < C::PT && xl >= 0 && xl + 4 <= C::FX) {
                const float4 v =
                    *reinterpret_cast<const float4 *>(Fs[s] + ((size_t)pl * C::PT + yl) * C::FX + xl);
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
            }
        }
        *reinterpret_cast<float4 *>(tb + ((size_t)pl * B::PE + y) * B::XB + x) = acc;
    }
    __threadfence();  // the block is visible to every CTA before the tile is signalled done
    cl.sync();
}

// Spread the points [beg, end) of tile `tile` that lie in sub-tile `sub` (x
// half sub & 1, y half sub >> 1) onto the three grids at grid + c0 gcs (z-plane
// stride gzs, component stride gcs); the sources are fs[n * fstride + foff].
// TB: the CTA is one of the tile's cluster of four, and the tile's padded block
// goes to its tile buffer at `grid` instead (tile_combine).  Called by every
// thread of the CTA.
template <int P, bool TB = false>
__device__ __forceinline__ void spread_sub_body(const GP<float> &g, int tile, int sub, int beg, int end, int c0,
                                                bool stress, const float4 *__restrict__ xs,
                                                const float4 *__restrict__ fs, const float4 *__restrict__ qs,
                                                int fstride, int foff, float *__restrict__ grid, size_t gzs,
                                                size_t gcs, SubSmem<P> &sm) {
    using C = SubCfg<P>;
    constexpr int ZP = C::ZP, TE = C::TE;
    SubStage<P> *S = sm.S;
    unsigned short *list = sm.list;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int sx = sub & 1, sy = sub >> 1;
    const int gx0 = tx * TE + SUB * sx, gy0 = ty * TE + SUB * sy, gz0 = tz * TE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the thread's columns (cx, cy) and (cx, cy + 1); idle lanes read the zero
    // x weight of slot PT (a row cy + 1 = PT reads the zero y weight there)
    const int lr = lane / C::PT;
    const int cyw = warp * C::RW + lr * C::TR;
    const bool own = lr < C::LR && cyw < C::PT;
    const int cx = own ? lane - lr * C::PT : C::PT, cy = own ? cyw : 0;
    // the window-start rows oy whose support meets the warp's rows
    const int r0 = warp * C::RW, r1 = min(r0 + C::RW, C::PT) - 1;
    const int ylo = max(0, r0 - (P - 1)), yhi = min(SUB - 1, r1);
    SubAcc<P> a;
#pragma unroll
    for (int r = 0; r < C::TR; r++)
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int q = 0; q < ZP; q++) a[r][c][q] = make_float2(0.0f, 0.0f);
    const int *tags = reinterpret_cast<const int *>(xs);
    for (int rb = beg; rb < end; rb += C::CAP) {
        // the round's points of this sub-tile (tile points rb .. rb + rn)
        const int cnt = sub_filter<C::NT>(tags, rb, min(C::CAP, end - rb), tx * TE, ty * TE, sx, sy, list, sm.wc);
        if (cnt > 0) {
            sub_stage<P>(S[0], g, xs, fs, qs, fstride, foff, c0, stress, list, rb, 0, min(C::NB, cnt), gx0, gy0,
                         gz0);
            __syncthreads();
            int k = 0;
            for (int b0 = 0; b0 < cnt; b0 += C::NB, k ^= 1) {
                if (b0 + C::NB < cnt)
                    sub_stage<P>(S[k ^ 1], g, xs, fs, qs, fstride, foff, c0, stress, list, rb, b0 + C::NB,
                                 min(C::NB, cnt - b0 - C::NB), gx0, gy0, gz0);
                sub_runs<P, 0>(S[k], ylo, yhi, cx, cy, a);
                __syncthreads();
            }
        }
    }
    // flush: the columns through shared memory (x fastest), then added to the
    // grids a float4 of x at a time (16-byte vector atomics) where the rows
    // allow it; grid points beyond the grid's Mtilde are zero and skipped
    if (own) {
#pragma unroll
        for (int r = 0; r < C::TR; r++) {
            if (cy + r < C::PT) {
#pragma unroll
                for (int c = 0; c < 3; c++)
#pragma unroll
                    for (int q = 0; q < ZP; q++) {
                        sm.F[c][2 * q][cy + r][cx] = a[r][c][q].x;
                        if (2 * q + 1 < C::PZ) sm.F[c][2 * q + 1][cy + r][cx] = a[r][c][q].y;
                    }
            }
        }
    }
    // the padding columns of every row read as zero
    constexpr int NPAD = C::FX - C::PT;
    for (int i = tid; i < 3 * C::PZ * C::PT * NPAD; i += C::NT) {
        const int r = i / NPAD;
        (&sm.F[0][0][0][0])[r * C::FX + C::PT + (i - r * NPAD)] = 0.0f;
    }
    __syncthreads();
    if constexpr (TB) {
        tile_combine<P>(sm, grid, sub);
        return;
    }
    float *gbase = grid + (size_t)c0 * gcs;
    const bool vec = ((g.mf[0] | gzs | gcs) & 3) == 0 && (reinterpret_cast<size_t>(gbase) & 15) == 0;
    // thread -> (plane parity, row y, float4 xq) of the (component, z) planes,
    // two planes per pass
    constexpr int NQ = C::FX / 4, PER = C::PT * NQ, NPL = 3 * C::PZ;
    static_assert(2 * PER <= C::NT, "two planes of float4 per pass");
    if (tid < 2 * PER) {
        const int par = tid / PER, yq = tid - par * PER, y = yq / NQ, xq = yq - y * NQ;
        const int gx = gx0 + 4 * xq, gy = gy0 + y;
        if (gx < g.mt[0] && gy < g.mt[1]) {
            const bool v4 = vec && gx + 3 < g.mt[0];
            const float *src = &sm.F[0][0][y][4 * xq];
            for (int pl = par; pl < NPL; pl += 2) {
                const int c = pl / C::PZ, z = pl - c * C::PZ;
                if (gz0 + z >= g.mt[2]) continue;
                const float4 v = *reinterpret_cast<const float4 *>(src + (size_t)pl * C::PT * C::FX);
                if (v.x == 0.0f && v.y == 0.0f && v.z == 0.0f && v.w == 0.0f) continue;
                float *dst = gbase + (size_t)c * gcs + (size_t)(gz0 + z) * gzs + (size_t)gy * g.mf[0] + gx;
                if (v4) {
                    atomicAdd(reinterpret_cast<float4 *>(dst), v);
                } else {
                    if (v.x != 0.0f) atomicAdd(dst, v.x);
                    if (v.y != 0.0f && gx + 1 < g.mt[0]) atomicAdd(dst + 1, v.y);
                    if (v.z != 0.0f && gx + 2 < g.mt[0]) atomicAdd(dst + 2, v.z);
                    if (v.w != 0.0f && gx + 3 < g.mt[0]) atomicAdd(dst + 3, v.w);
                }
            }
        }
    }
}

// SE_SUB_MINB: CTAs per SM the sub-tile spreading kernels are compiled for
#ifndef SE_SUB_MINB
#define SE_SUB_MINB 3
#endif

// One CTA per (tile, sub-tile): block b takes sub-tile b mod 4 of tile b / 4.
template <int P>
__global__ void __launch_bounds__(SubCfg<P>::NT, SE_SUB_MINB)
    k_spread_sub(GP<float> g, int c0, bool stress, const int *__restrict__ tile_start,
                 const float4 *__restrict__ xs, const float4 *__restrict__ fs, const float4 *__restrict__ qs,
                 float *__restrict__ grid, size_t gzs, size_t gcs) {
    extern __shared__ __align__(16) unsigned char sub_smem_raw[];
    const int tile = blockIdx.x >> 2;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    spread_sub_body<P>(g, tile, blockIdx.x & 3, beg, end, c0, stress, xs, fs, qs, 1, 0, grid, gzs, gcs,
                       *reinterpret_cast<SubSmem<P> *>(sub_smem_raw));
}

// The float4 at grid (x4, y, z) of component c, x4 a multiple of 4: the sum,
// in a fixed order (tiles by z, then y, then x), of the tile-buffer values of
// the tiles whose padded blocks hold it; a tile without points adds nothing.
template <int P>
__device__ __forceinline__ float4 merge_point4(const GP<float> &g, const int *__restrict__ tile_start,
                                               const float *__restrict__ tb, int c, int z, int y, int x4) {
    using B = TileBufCfg<P>;
    constexpr int TE = COL_TE;
    // tiles t with t TE <= z < t TE + PE (truncating division: a negative
    // numerator gives at most 0, clamped to 0); in x the float4 lies inside
    // the tile's row: t TE <= x4 <= t TE + XB - 4
    const int tz0 = max(0, (z - B::PE + TE) / TE), tz1 = min(g.nt[2] - 1, z / TE);
    const int ty0 = max(0, (y - B::PE + TE) / TE), ty1 = min(g.nt[1] - 1, y / TE);
    const int tx0 = max(0, (x4 - B::XB + 4 + TE - 1) / TE), tx1 = min(g.nt[0] - 1, x4 / TE);
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int tz = tz0; tz <= tz1; tz++)
        for (int ty = ty0; ty <= ty1; ty++) {
            const int trow = (tz * g.nt[1] + ty) * g.nt[0];
            for (int tx = tx0; tx <= tx1; tx++) {
                const int t = trow + tx;
                if (__ldg(tile_start + t) == __ldg(tile_start + t + 1)) continue;
                const float4 v = __ldg(reinterpret_cast<const float4 *>(
                    tb + (size_t)t * B::FLOATS +
                    (((size_t)c * B::PE + (z - TE * tz)) * B::PE + (y - TE * ty)) * B::XB + (x4 - TE * tx)));
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
            }
        }
    return acc;
}

// Atomic-free variant: the four sub-tiles of a tile form a cluster, and the
// tile's padded block goes to its slot of the tile buffer tb (three
// components); k_merge_tiles then writes the grids.
template <int P>
__global__ void __cluster_dims__(4, 1, 1) __launch_bounds__(SubCfg<P>::NT, SE_SUB_MINB)
    k_spread_sub_tb(GP<float> g, int c0, bool stress, const int *__restrict__ tile_start,
                    const float4 *__restrict__ xs, const float4 *__restrict__ fs, const float4 *__restrict__ qs,
                    float *__restrict__ tb) {
    extern __shared__ __align__(16) unsigned char sub_smem_raw[];
    const int tile = blockIdx.x >> 2;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;  // the whole cluster (one tile) returns
    spread_sub_body<P, true>(g, tile, blockIdx.x & 3, beg, end, c0, stress, xs, fs, qs, 1, 0,
                             tb + (size_t)tile * TileBufCfg<P>::FLOATS, 0, 0,
                             *reinterpret_cast<SubSmem<P> *>(sub_smem_raw));
}

// Second pass of the atomic-free flush: every grid point of the corner [0,
// Mt)^3 of the three grids at `grid` is written once from the tile buffer
// (merge_point4), without atomics and without zeroing the grid first, so its
// values do not depend on the order in which CTAs ran.  Thread (threadIdx.x,
// row): the float4 at x = 4 threadIdx.x (+ 4 blockDim.x ...) of x row `row` =
// (c Mt_z + z) Mt_y + y.
template <int P>
__global__ void k_merge_tiles(GP<float> g, const int *__restrict__ tile_start, const float *__restrict__ tb,
                              float *__restrict__ grid, size_t gzs, size_t gcs, bool vec) {
    const size_t row = (size_t)blockIdx.x * blockDim.y + threadIdx.y;
    if (row >= (size_t)3 * g.mt[1] * g.mt[2]) return;
    const int y = (int)(row % g.mt[1]), z = (int)((row / g.mt[1]) % g.mt[2]);
    const int c = (int)(row / ((size_t)g.mt[1] * g.mt[2]));
    float *out = grid + (size_t)c * gcs + (size_t)z * gzs + (size_t)y * g.mf[0];
    for (int x4 = 4 * threadIdx.x; x4 < g.mt[0]; x4 += 4 * blockDim.x) {
        const float4 acc = merge_point4<P>(g, tile_start, tb, c, z, y, x4);
        if (vec && x4 + 3 < g.mt[0]) {
            *reinterpret_cast<float4 *>(out + x4) = acc;
        } else {
            out[x4] = acc.x;
            if (x4 + 1 < g.mt[0]) out[x4 + 1] = acc.y;
            if (x4 + 2 < g.mt[0]) out[x4 + 2] = acc.z;
            if (x4 + 3 < g.mt[0]) out[x4 + 3] = acc.w;
        }
    }
}

// Batches: one CTA per (system, tile, sub-tile) with the right-hand sides
// inside: block b takes sub-tile b mod 4 of item (b / 4) n_rhs of the (system,
// tile, rhs) list (right-hand side innermost) and spreads each right-hand side
// r onto its three grids (the system's grid + 3 r gcs).
template <int P>
__global__ void __launch_bounds__(SubCfg<P>::NT, SE_SUB_MINB)
    k_bspread_sub(const BSys<float> *__restrict__ sys, const int4 *__restrict__ items,
                  const int *__restrict__ tile_start, int n_rhs, const float4 *__restrict__ xs,
                  const float4 *__restrict__ fs) {
    extern __shared__ __align__(16) unsigned char sub_smem_raw[];
    const int4 it = items[(size_t)(blockIdx.x >> 2) * n_rhs];
    const BSys<float> &B = sys[it.x];
    const int key = B.tile_base + it.y;
    const int beg = tile_start[key], end = tile_start[key + 1];
    if (beg == end) return;
    const GP<float> g = B.g;
    for (int r = 0; r < n_rhs; r++)
        spread_sub_body<P>(g, it.y, blockIdx.x & 3, beg, end, 0, false, xs, fs, nullptr, n_rhs, r,
                           B.grid + (size_t)r * 3 * B.gcs, B.gzs, B.gcs,
                           *reinterpret_cast<SubSmem<P> *>(sub_smem_raw));
}

// ---------------------------------------------------------------- gather
// Gather (step 5, eq. u_integr) on the same sub-tiles: thread (cx, cy) loads
// columns (cx, cy) and (cx, cy + 1) of the three inverse-transformed grids into
// registers once per CTA (as z pairs), and for each staged point in key order
// forms the z sums of its two columns with paired FMAs, weights them by wx wy
// and sums over its three components; a warp then reduces two points at a
// time over its lanes (butterfly shuffles) and stores its part of each point
// in a slot of its own, and the parts of the warps are added in a fixed order
// when the batch is written out (no atomics: the result does not depend on
// the order in which warps finish).

template <int P>
struct SubGSmem {
    SubStage<P> S;
    float part[SubCfg<P>::NW][SubCfg<P>::NB][3];  // each warp's part of each point of the batch
    unsigned short list[SubCfg<P>::CAP];
    int wc[SubCfg<P>::NW];
};

// The point's sums over the thread's two columns: v[c] = sum_r wx wy_r sum_k wz_k G[r][c][z_k]
template <int P, int OZ>
__device__ __forceinline__ void subg_point(const SubRec<P> &R, int cx, int cy, const SubAcc<P> &G, float (&v)[3]) {
    constexpr int Q0 = OZ / 2, NP = P / 2 + (OZ & 1);
    static_assert(Q0 + NP <= SubCfg<P>::ZP, "the point's z support stays inside the column");
    float2 d[2][3];
#pragma unroll
    for (int r = 0; r < 2; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) d[r][c] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k2 = 0; k2 < (NP + 1) / 2; k2++) {
        const float4 wv = R.wz[k2];
        const float2 lo = make_float2(wv.x, wv.y), hi = make_float2(wv.z, wv.w);
#pragma unroll
        for (int r = 0; r < 2; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) {
                d[r][c] = __ffma2_rn(lo, G[r][c][Q0 + 2 * k2], d[r][c]);
                if (2 * k2 + 1 < NP) d[r][c] = __ffma2_rn(hi, G[r][c][Q0 + 2 * k2 + 1], d[r][c]);
            }
    }
    const float wxv = R.wx[cx];
    const float2 wyv = *reinterpret_cast<const float2 *>(&R.wy[cy]);
    const float w0 = wxv * wyv.x, w1 = wxv * wyv.y;
#pragma unroll
    for (int c = 0; c < 3; c++) v[c] = fmaf(w1, d[1][c].x + d[1][c].y, w0 * (d[0][c].x + d[0][c].y));
}

// Sum two points' values over the warp's lanes (lanes 0-15 end with point a's,
// 16-31 with point b's) and store them in the warp's slots ia, ib.
__device__ __forceinline__ void subg_reduce2(float (&va)[3], float (&vb)[3], float *pa, float *pb, int lane) {
    const bool up = lane >= 16;
    float t[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float send = up ? va[c] : vb[c], keep = up ? vb[c] : va[c];
        t[c] = keep + __shfl_xor_sync(FULLM, send, 16);
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 3; c++) t[c] += __shfl_xor_sync(FULLM, t[c], o);
    const int c = lane & 15;
    if (c < 3) (up ? pb : pa)[c] = c == 0 ? t[0] : (c == 1 ? t[1] : t[2]);
}

__device__ __forceinline__ void subg_reduce1(float (&va)[3], float *pa, int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 3; c++) va[c] += __shfl_xor_sync(FULLM, va[c], o);
    if (lane < 3) pa[lane] = lane == 0 ? va[0] : (lane == 1 ? va[1] : va[2]);
}

// The batch's records with z offset OZ, OZ + 1, ... whose oy lies in [ylo,
// yhi], two at a time; part: this warp's slots.
template <int P, int OZ>
__device__ __forceinline__ void subg_runs(const SubStage<P> &S, float (*part)[3], int ylo, int yhi, int cx, int cy,
                                          const SubAcc<P> &G, int lane) {
    if constexpr (OZ < SubCfg<P>::TE) {
        const int i0 = S.kst[OZ * SUB + ylo], i1 = S.kst[OZ * SUB + yhi + 1];
        int i = i0;
        for (; i + 1 < i1; i += 2) {
            float va[3], vb[3];
            subg_point<P, OZ>(S.rec[i], cx, cy, G, va);
            subg_point<P, OZ>(S.rec[i + 1], cx, cy, G, vb);
            subg_reduce2(va, vb, part[i], part[i + 1], lane);
        }
        if (i < i1) {
            float va[3];
            subg_point<P, OZ>(S.rec[i], cx, cy, G, va);
            subg_reduce1(va, part[i], lane);
        }
        subg_runs<P, OZ + 1>(S, part, ylo, yhi, cx, cy, G, lane);
    }
}

// One CTA per (tile, sub-tile), block b taking sub-tile b mod 4 of tile b / 4.
// w: the three grids (z-plane stride gzs, component stride gcs); u[perm[n]] =
// the gathered values + self_coef f_orig[perm[n]] (in FP64).
template <int P>
__global__ void __launch_bounds__(SubCfg<P>::NT, SE_SUB_MINB)
    k_gather_sub(GP<float> g, const int *__restrict__ tile_start, const float4 *__restrict__ xs,
                 const int *__restrict__ perm, const float *__restrict__ w, size_t gzs, size_t gcs,
                 const float *__restrict__ f_orig, double self_coef, float *__restrict__ u) {
    using C = SubCfg<P>;
    constexpr int ZP = C::ZP, TE = C::TE;
    extern __shared__ __align__(16) unsigned char subg_smem_raw[];
    SubGSmem<P> &sm = *reinterpret_cast<SubGSmem<P> *>(subg_smem_raw);
    const int tile = blockIdx.x >> 2, sub = blockIdx.x & 3;
    const int beg = tile_start[tile], end = tile_start[tile + 1];
    if (beg == end) return;
    const int tx = tile % g.nt[0], ty = (tile / g.nt[0]) % g.nt[1], tz = tile / (g.nt[0] * g.nt[1]);
    const int sx = sub & 1, sy = sub >> 1;
    const int gx0 = tx * TE + SUB * sx, gy0 = ty * TE + SUB * sy, gz0 = tz * TE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int lr = lane / C::PT;
    const int cyw = warp * C::RW + lr * C::TR;
    const bool own = lr < C::LR && cyw < C::PT;
    const int cx = own ? lane - lr * C::PT : C::PT, cy = own ? cyw : 0;
    const int r0 = warp * C::RW, r1 = min(r0 + C::RW, C::PT) - 1;
    const int ylo = max(0, r0 - (P - 1)), yhi = min(SUB - 1, r1);
    // the thread's two columns of the three grids (zero outside the grids)
    SubAcc<P> G;
    const int gx = gx0 + cx;
#pragma unroll
    for (int r = 0; r < C::TR; r++) {
        const int gy = gy0 + cy + r;
        const bool col = own && cy + r < C::PT && gx < g.mt[0] && gy < g.mt[1];
        const float *b = w + (size_t)gz0 * gzs + (size_t)gy * g.mf[0] + gx;
#pragma unroll
        for (int c = 0; c < 3; c++)
#pragma unroll
            for (int q = 0; q < ZP; q++) {
                const int z0 = 2 * q, z1 = 2 * q + 1;
                const float v0 = (col && gz0 + z0 < g.mt[2]) ? __ldg(b + (size_t)c * gcs + (size_t)z0 * gzs) : 0.0f;
                const float v1 = (col && z1 < C::PZ && gz0 + z1 < g.mt[2])
                                     ? __ldg(b + (size_t)c * gcs + (size_t)z1 * gzs)
                                     : 0.0f;
                G[r][c][q] = make_float2(v0, v1);
            }
    }
    const int *tags = reinterpret_cast<const int *>(xs);
    for (int rb = beg; rb < end; rb += C::CAP) {
        const int cnt = sub_filter<C::NT>(tags, rb, min(C::CAP, end - rb), tx * TE, ty * TE, sx, sy, sm.list,
                                          sm.wc);
        for (int b0 = 0; b0 < cnt; b0 += C::NB) {
            const int nb = min(C::NB, cnt - b0);
            sub_stage<P, true>(sm.S, g, xs, nullptr, nullptr, 1, 0, 0, false, sm.list, rb, b0, nb, gx0, gy0, gz0);
            // every warp's slots start at zero (a warp whose rows no support of a
            // point meets leaves them so)
            for (int i = tid; i < C::NW * C::NB * 3; i += C::NT) (&sm.part[0][0][0])[i] = 0.0f;
            __syncthreads();
            subg_runs<P, 0>(sm.S, sm.part[warp], ylo, yhi, cx, cy, G, lane);
            __syncthreads();
            if (tid < nb) {
                const int n = sm.S.rec[tid].n, m = perm[n];
#pragma unroll
                for (int c = 0; c < 3; c++) {
                    float v = 0.0f;
#pragma unroll
                    for (int k = 0; k < C::NW; k++) v += sm.part[k][tid][c];
                    double o = (double)v;
                    if (self_coef != 0.0) o += self_coef * (double)f_orig[3 * (size_t)m + c];
                    u[3 * (size_t)m + c] = (float)o;
                }
            }
        }
    }
}

template <int P>
cudaError_t run_spread_sub(const GP<float> &g, int ntiles, int c0, bool stress, const int *ts, const float4 *xs,
                           const float4 *fs, const float4 *qs, float *grid, cudaStream_t st) {
    constexpr size_t smem = sizeof(SubSmem<P>);
    cudaError_t e = cudaFuncSetAttribute(k_spread_sub<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const size_t gzs = (size_t)g.mf[0] * g.mf[1], gcs = gzs * g.mf[2];
    k_spread_sub<P><<<4 * ntiles, SubCfg<P>::NT, smem, st>>>(g, c0, stress, ts, xs, fs, qs, grid, gzs, gcs);
    return cudaGetLastError();
}

template <int P>
cudaError_t run_spread_sub_tb(const GP<float> &g, int ntiles, int c0, bool stress, const int *ts, const float4 *xs,
                              const float4 *fs, const float4 *qs, float *tb, cudaStream_t st) {
    constexpr size_t smem = sizeof(SubSmem<P>);
    cudaError_t e =
        cudaFuncSetAttribute(k_spread_sub_tb<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    k_spread_sub_tb<P><<<4 * ntiles, SubCfg<P>::NT, smem, st>>>(g, c0, stress, ts, xs, fs, qs, tb);
    return cudaGetLastError();
}

template <int P>
cudaError_t run_merge_tiles(const GP<float> &g, const int *ts, const float *tb, float *grid, int c0,
                            cudaStream_t st) {
    const size_t gzs = (size_t)g.mf[0] * g.mf[1], gcs = gzs * g.mf[2];
    float *gbase = grid + (size_t)c0 * gcs;
    const bool vec = ((g.mf[0] | gzs | gcs) & 3) == 0 && (reinterpret_cast<size_t>(gbase) & 15) == 0;
    const size_t rows = (size_t)3 * g.mt[1] * g.mt[2];
    const dim3 bs(32, 8);
    k_merge_tiles<P><<<(unsigned)((rows + bs.y - 1) / bs.y), bs, 0, st>>>(g, ts, tb, gbase, gzs, gcs, vec);
    return cudaGetLastError();
}

template <int P>
cudaError_t run_bspread_sub(const BSys<float> *sys, const int4 *items, int nitems, const int *ts, int n_rhs,
                            const float4 *xs, const float4 *fs, cudaStream_t st) {
    constexpr size_t smem = sizeof(SubSmem<P>);
    cudaError_t e = cudaFuncSetAttribute(k_bspread_sub<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    k_bspread_sub<P><<<4 * (nitems / n_rhs), SubCfg<P>::NT, smem, st>>>(sys, items, ts, n_rhs, xs, fs);
    return cudaGetLastError();
}

template <int P>
cudaError_t run_gather_sub(const GP<float> &g, int ntiles, const int *ts, const float4 *xs, const int *perm,
                           const float *w, const float *f_orig, double self_coef, float *u, cudaStream_t st) {
    constexpr size_t smem = sizeof(SubGSmem<P>);
    cudaError_t e = cudaFuncSetAttribute(k_gather_sub<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const size_t gzs = (size_t)g.mf[0] * g.mf[1], gcs = gzs * g.mf[2];
    k_gather_sub<P><<<4 * ntiles, SubCfg<P>::NT, smem, st>>>(g, ts, xs, perm, w, gzs, gcs, f_orig, self_coef, u);
    return cudaGetLastError();
}

}  // namespace

bool sub_supported(int P) { return P == 10 || P == 12; }

cudaError_t launch_gather_sub(const GP<float> &g, int ntiles, const int *tile_start, const float4 *xs,
                              const int *perm, const float *w, const float *f_orig, double self_coef, float *u,
                              cudaStream_t st) {
    if (g.P == 12) return run_gather_sub<12>(g, ntiles, tile_start, xs, perm, w, f_orig, self_coef, u, st);
    if (g.P == 10) return run_gather_sub<10>(g, ntiles, tile_start, xs, perm, w, f_orig, self_coef, u, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_spread_sub(const GP<float> &g, int ntiles, int c0, bool stress, const int *tile_start,
                              const float4 *xs, const float4 *fs, const float4 *qs, float *grid, cudaStream_t st) {
    if (g.P == 12) return run_spread_sub<12>(g, ntiles, c0, stress, tile_start, xs, fs, qs, grid, st);
    if (g.P == 10) return run_spread_sub<10>(g, ntiles, c0, stress, tile_start, xs, fs, qs, grid, st);
    return cudaErrorInvalidValue;
}

size_t tilebuf_floats(int P, int ntiles) {
    switch (P) {
        case 4: return TileBufCfg<4>::FLOATS * (size_t)ntiles;
        case 6: return TileBufCfg<6>::FLOATS * (size_t)ntiles;
        case 8: return TileBufCfg<8>::FLOATS * (size_t)ntiles;
        case 10: return TileBufCfg<10>::FLOATS * (size_t)ntiles;
        case 12: return TileBufCfg<12>::FLOATS * (size_t)ntiles;
        case 14: return TileBufCfg<14>::FLOATS * (size_t)ntiles;
        case 16: return TileBufCfg<16>::FLOATS * (size_t)ntiles;
        default: return 0;
    }
}

cudaError_t launch_merge_tiles(const GP<float> &g, const int *tile_start, const float *tb, float *grid, int c0,
                               cudaStream_t st) {
    switch (g.P) {
        case 4: return run_merge_tiles<4>(g, tile_start, tb, grid, c0, st);
        case 6: return run_merge_tiles<6>(g, tile_start, tb, grid, c0, st);
        case 8: return run_merge_tiles<8>(g, tile_start, tb, grid, c0, st);
        case 10: return run_merge_tiles<10>(g, tile_start, tb, grid, c0, st);
        case 12: return run_merge_tiles<12>(g, tile_start, tb, grid, c0, st);
        case 14: return run_merge_tiles<14>(g, tile_start, tb, grid, c0, st);
        case 16: return run_merge_tiles<16>(g, tile_start, tb, grid, c0, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_spread_sub_tb(const GP<float> &g, int ntiles, int c0, bool stress, const int *tile_start,
                                 const float4 *xs, const float4 *fs, const float4 *qs, float *tb, cudaStream_t st) {
    if (g.P == 12) return run_spread_sub_tb<12>(g, ntiles, c0, stress, tile_start, xs, fs, qs, tb, st);
    if (g.P == 10) return run_spread_sub_tb<10>(g, ntiles, c0, stress, tile_start, xs, fs, qs, tb, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_bspread_sub(const BSys<float> *sys, const int4 *items, int nitems, int P, int n_rhs,
                               const int *tile_start, const float4 *xs, const float4 *fs, cudaStream_t st) {
    if (P == 12) return run_bspread_sub<12>(sys, items, nitems, tile_start, n_rhs, xs, fs, st);
    if (P == 10) return run_bspread_sub<10>(sys, items, nitems, tile_start, n_rhs, xs, fs, st);
    return cudaErrorInvalidValue;
}

}  // namespace se
