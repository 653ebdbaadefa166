// Batched evaluation: S independent systems, each with its own cube, its own
// points and n_rhs right-hand sides, evaluated by one launch per stage over
// all systems (the method of Section 8 applied to every system; the
// precomputed kernel of Section 4.3 is computed once per system and reused
// for all its right-hand sides, as Section 4.3 notes for repeated solves).
//
//   bin (one counting sort over all systems: keys offset per system)
//   zero octants -> spread (items: system x tile x right-hand side)
//   R2C FFTs (one batched cuFFT plan per FFT size class)
//   scale (blocks: system x k-range, all right-hand sides per k-point)
//   C2R FFTs -> gather + self (warp per point, all right-hand sides)
//   real-space sum (clusters of all systems, up to 8 right-hand sides a pass)
//
// Every system gets its own M, xi and rc from the same parameter selection as
// a single plan; P (and the spreading tile) is common to the batch.  The whole
// sequence is captured once into a CUDA graph and replayed while the caller's
// pointers stay the same.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <string>
#include <vector>

#include "se_internal.cuh"

using namespace se;

struct se_batch_s {
    int kernel = 0, prec = 0, S = 0, R = 1;
    int64_t Ntot = 0;
    int P = 0, T_ = 8;
    bool colk = false;  // FP32 register-column spreading and gather
    std::vector<se_plan_s *> sub;  // per system: parameters, geometry, precomputed kernel
    std::vector<int> off_h;        // S + 1 point offsets
    int ntiles_tot = 0, ncells_tot = 0, nrows_tot = 0, nitems = 0, nblk_scale = 0, nblk_zero = 0;
    void *sys_d = nullptr;  // BSys<T>[S]
    void *maps_d = nullptr; // FP32 interleaved grids: S tensor maps of the batched gather
    int *off_d = nullptr, *row_base_d = nullptr, *blk_base_d = nullptr, *zblk_base_d = nullptr;
    int4 *items_d = nullptr;
    int *cl_sys = nullptr;
    Buffers b;
    struct SizeClass {
        int mf[3] = {0, 0, 0}, count = 0;
        void *grid = nullptr, *spec = nullptr, *wgrid = nullptr;
        cufftHandle fwd = 0, inv = 0;
        bool have_fwd = false, have_inv = false;
        // FP32 (ilv): grids interleaved plane by plane, zero-padding-aware transforms
        cufftHandle f2d = 0, i2d = 0, zc = 0;
        size_t G = 0, mt2 = 0;  // grids of the class, nonzero z-planes
    };
    bool ilv = false;
    std::vector<SizeClass> classes;
    void *work = nullptr;
    // CUDA graph of one evaluation, valid for the pointers it was captured with
    bool use_graph = true;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *gx = nullptr, *gf = nullptr;
    void *gu = nullptr;
    int64_t launches = 0;
    cudaStream_t last_stream = nullptr;
    // stage timing (se_batch_set_timing): events around the stages of an
    // evaluation run without the graph
    bool timing = false, timed = false;
    cudaEvent_t ev[8] = {};
};

namespace {

void free_batch(se_batch_s *B) {
    if (!B) return;
    for (auto &e : B->ev)
        if (e) cudaEventDestroy(e);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (auto &c : B->classes) {
        if (c.have_fwd) cufftDestroy(c.fwd);
        if (c.have_inv) cufftDestroy(c.inv);
        if (c.f2d) cufftDestroy(c.f2d);
        if (c.i2d) cufftDestroy(c.i2d);
        if (c.zc) cufftDestroy(c.zc);
        cudaFree(c.grid);
        cudaFree(c.spec);
        cudaFree(c.wgrid);
    }
    void *ptrs[] = {B->work, B->sys_d, B->maps_d, B->off_d, B->row_base_d, B->blk_base_d, B->zblk_base_d, B->items_d,
                    B->cl_sys, B->b.xs_t, B->b.fs_t, B->b.perm_t, B->b.cnt_t, B->b.slot_t, B->b.key_t,
                    B->b.xs_r, B->b.fs_r, B->b.perm_r, B->b.cnt_r, B->b.slot_r, B->b.key_r, B->b.tag_t,
                    B->b.tag_r, B->b.ncl, B->b.clusters, B->b.status};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (se_plan_s *p : B->sub) free_plan(p);
    delete B;
}

template <typename T>
void fill_sys(se_batch_s *B, std::vector<BSys<T>> &sys, const std::vector<int> &tile_base,
              const std::vector<int> &cell_base, const std::vector<int> &row_base, const std::vector<int> &blk_base,
              const std::vector<int> &zblk_base, const std::vector<void *> &grid, const std::vector<void *> &spec,
              const std::vector<void *> &wgrid, const std::vector<std::array<size_t, 4>> &strides) {
    sys.resize(B->S);
    for (int s = 0; s < B->S; s++) {
        se_plan_s *p = B->sub[s];
        BSys<T> &Y = sys[s];
        memset(&Y, 0, sizeof(Y));
        Y.g = gp<T>(p);
        Y.rk = make_rc<T>(p);
        Y.sc = make_scale_const(p);
        Y.ghat = (const T *)p->ghat;
        Y.grid = (T *)grid[s];
        Y.spec = (cplx<T> *)spec[s];
        Y.wgrid = (T *)wgrid[s];
        Y.gzs = strides[s][0];
        Y.gcs = strides[s][1];
        Y.szs = strides[s][2];
        Y.scs = strides[s][3];
        Y.self_coef = (B->kernel == SE_STOKESLET) ? -4.0 * p->xi / sqrt(M_PI) : 0.0;
        Y.off = B->off_h[s];
        Y.n = B->off_h[s + 1] - B->off_h[s];
        Y.tile_base = tile_base[s];
        Y.cell_base = cell_base[s];
        Y.row_base = row_base[s];
        Y.blk_base = blk_base[s];
        Y.zblk_base = zblk_base[s];
    }
}

#define BCK(expr)                                                                        \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return fail(SE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)
#define BCF(expr)                                                                             \
    do {                                                                                      \
        cufftResult _r = (expr);                                                              \
        if (_r != CUFFT_SUCCESS)                                                              \
            return fail(SE_ERR_CUFFT, std::string(#expr) + " failed, code " + std::to_string((int)_r)); \
    } while (0)

template <typename T>
se_status_t enqueue_t(se_batch_s *B, const T *x, const T *f, T *u, cudaStream_t st) {
    const BSys<T> *sys = (const BSys<T> *)B->sys_d;
    const int S = B->S, R = B->R, Ntot = (int)B->Ntot;
    B->launches = 0;
    // stage boundary k (timing only): bin | zero + spread | fft | scale | ifft | gather | real
    auto mark = [&](int k) {
        if (B->timing) cudaEventRecord(B->ev[k], st);
    };
    mark(0);
    BCK(launch_bbin<T>(sys, B->off_d, S, Ntot, R, B->ntiles_tot, B->ncells_tot, x, f, B->b, st, &B->launches));
    mark(1);
    BCK(launch_bzero<T>(sys, B->zblk_base_d, S, B->nblk_zero, R, st));
    if (sizeof(T) == 4 && B->colk)
        BCK(launch_bspread_col((const BSys<float> *)sys, B->items_d, B->nitems, B->P, R, B->b, st));
    else
        BCK(launch_bspread<T>(sys, B->items_d, B->nitems, B->P, B->T_, R, B->b, st));
    B->launches += 2;
    mark(2);
    for (auto &c : B->classes) {
        if (B->ilv) {
            // 2D (y, x) transforms of the nonzero planes of all the class's grids,
            // the spectra's upper z-planes zeroed, then the transform along z
            const size_t plane_c = (size_t)c.mf[1] * (c.mf[0] / 2 + 1);
            BCF(cufftSetStream(c.f2d, st));
            BCF(cufftSetStream(c.zc, st));
            BCF(cufftExecR2C(c.f2d, (cufftReal *)c.grid, (cufftComplex *)c.spec));
            BCK(cudaMemsetAsync((cufftComplex *)c.spec + c.mt2 * c.G * plane_c, 0,
                                (c.mf[2] - c.mt2) * c.G * plane_c * sizeof(cufftComplex), st));
            BCF(cufftExecC2C(c.zc, (cufftComplex *)c.spec, (cufftComplex *)c.spec, CUFFT_FORWARD));
            continue;
        }
        BCF(cufftSetStream(c.fwd, st));
        if (sizeof(T) == 4)
            BCF(cufftExecR2C(c.fwd, (cufftReal *)c.grid, (cufftComplex *)c.spec));
        else
            BCF(cufftExecD2Z(c.fwd, (cufftDoubleReal *)c.grid, (cufftDoubleComplex *)c.spec));
    }
    mark(3);
    BCK(launch_bscale<T>(B->kernel, sys, B->blk_base_d, S, B->nblk_scale, R, st));
    B->launches += 1;
    mark(4);
    for (auto &c : B->classes) {
        if (B->ilv) {
            // back along z, then 2D on only the planes the gather reads
            BCF(cufftSetStream(c.zc, st));
            BCF(cufftSetStream(c.i2d, st));
            BCF(cufftExecC2C(c.zc, (cufftComplex *)c.spec, (cufftComplex *)c.spec, CUFFT_INVERSE));
            BCF(cufftExecC2R(c.i2d, (cufftComplex *)c.spec, (cufftReal *)c.wgrid));
            continue;
        }
        BCF(cufftSetStream(c.inv, st));
        if (sizeof(T) == 4)
            BCF(cufftExecC2R(c.inv, (cufftComplex *)c.spec, (cufftReal *)c.wgrid));
        else
            BCF(cufftExecZ2D(c.inv, (cufftDoubleComplex *)c.spec, (cufftDoubleReal *)c.wgrid));
    }
    mark(5);
    if (sizeof(T) == 4 && B->colk)
        BCK(launch_bgather_col((const BSys<float> *)sys, B->items_d, B->nitems, B->P, R, B->b, (const float *)f,
                               (float *)u, B->maps_d, st));
    else
        BCK(launch_bgather<T>(sys, B->off_d, S, Ntot, B->P, R, B->b, f, u, st));
    B->launches += 1;
    mark(6);
    BCK(launch_breal<T>(B->kernel, sys, B->row_base_d, S, B->nrows_tot, Ntot, R, B->b, B->cl_sys, u, st,
                        &B->launches));
    mark(7);
    if (B->timing) B->timed = true;
    return SE_OK;
}

se_status_t enqueue(se_batch_s *B, const void *x, const void *f, void *u, cudaStream_t st) {
    if (B->prec == SE_FP32) return enqueue_t<float>(B, (const float *)x, (const float *)f, (float *)u, st);
    return enqueue_t<double>(B, (const double *)x, (const double *)f, (double *)u, st);
}

template <typename P_>
cudaError_t bmalloc(P_ **ptr, size_t bytes) {
    return cudaMalloc((void **)ptr, bytes ? bytes : 16);
}

se_status_t create(se_batch_s *B, const int64_t *N_s, const double *box_s, double tol, const se_params_t *params) {
    const int S = B->S, kernel = B->kernel, prec = B->prec, R = B->R;
    // parameters per system, then a common P (the largest chosen)
    std::vector<se_params_t> pr(S);
    int Pmax = 0;
    for (int s = 0; s < S; s++) {
        se_status_t st = choose_params(kernel, prec, N_s[s], box_s[4 * s + 3], tol, params, 0.0, &pr[s], R);
        if (st != SE_OK) return st;
        Pmax = std::max(Pmax, pr[s].P);
    }
    for (int s = 0; s < S; s++) {
        if (pr[s].P == Pmax) continue;
        se_params_t in;
        memset(&in, 0, sizeof(in));
        if (params) in = *params;
        in.P = Pmax;
        se_status_t st = choose_params(kernel, prec, N_s[s], box_s[4 * s + 3], tol, &in, 0.0, &pr[s], R);
        if (st != SE_OK) return st;
    }
    B->P = Pmax;
#ifndef SE_BATCH_FAST_FFT
#define SE_BATCH_FAST_FFT 1
#endif
    // FFT lengths: each system's moved to the fast length around it (below or
    // above, the one of least modelled work), so that the size classes are
    // fewer and their batched transforms faster; explicit M or an FFT cap stay
    const bool fixed = params && (params->M > 0 || params->max_fft > 0 || params->xi > 0);
    for (int s = 0; s < S && SE_BATCH_FAST_FFT && !fixed; s++) {
        const int Mf0 = 2 * (pr[s].M + pr[s].P);
        if (fast_fft_len(Mf0, prec)) continue;
        int lo = Mf0, hi = Mf0;
        while (lo > 2 * (pr[s].P + 2) && !fast_fft_len(lo, prec)) lo -= 2;
        while (!fast_fft_len(hi, prec)) hi += 2;
        double best = 1e300;
        se_params_t pick = pr[s];
        for (int Mf : {lo, hi}) {
            if (!fast_fft_len(Mf, prec) || Mf / 2 - pr[s].P < 2) continue;
            se_params_t in;
            memset(&in, 0, sizeof(in));
            if (params) in = *params;
            in.P = Pmax;
            in.M = Mf / 2 - Pmax;
            se_params_t c;
            if (choose_params(kernel, prec, N_s[s], box_s[4 * s + 3], tol, &in, 0.0, &c, R) != SE_OK) continue;
            const double cost = model_cost(prec, N_s[s], box_s[4 * s + 3], c.P, c.M, c.rc, nullptr, R);
            if (cost < best) {
                best = cost;
                pick = c;
            }
        }
        pr[s] = pick;
    }
    // geometry and the precomputed kernel of every system
    for (int s = 0; s < S; s++) {
        se_plan_s *p = new se_plan_s();
        B->sub.push_back(p);
        if (!(pr[s].xi > 0) || !(pr[s].rc > 0) || pr[s].M < 1)
            return fail(SE_ERR_INVALID_ARG, "batch: invalid parameters for system " + std::to_string(s));
        const double *bx = box_s + 4 * s;
        const double box6[6] = {bx[0], bx[1], bx[2], bx[3], bx[3], bx[3]};
        se_status_t st = setup_plan(p, kernel, prec, N_s[s], box6, pr[s]);
        if (st != SE_OK) return st;
        if (!p->tiled || p->P > 16)
            return fail(SE_ERR_NOT_SUPPORTED, "batch: the support P must be <= 16 (tolerance too small)");
        const RC<double> rk = make_rc<double>(p);
        if ((2 * rk.reach[0] + 1) * (2 * rk.reach[1] + 1) > 121)
            return fail(SE_ERR_NOT_SUPPORTED, "batch: real-space reach above 5 cells");
        if (s > 0 && p->geom.T != B->sub[0]->geom.T)
            return fail(SE_ERR_NOT_SUPPORTED, "batch: spreading tiles differ between systems");
        const size_t O3 = (size_t)(p->mt[0] + 1) * (p->mt[1] + 1) * (p->mt[2] + 1);
        if (bmalloc(&p->ghat64, O3 * sizeof(double)) ||
            (prec == SE_FP32 && bmalloc((float **)&p->ghat, O3 * sizeof(float)))) {
            cudaGetLastError();
            return fail(SE_ERR_OOM, "batch: precompute allocation failed");
        }
        st = precompute(p);
        if (st != SE_OK) return st;
    }
    B->T_ = B->sub[0]->geom.T;
    B->colk = B->sub[0]->colk;
    // offsets and tables
    B->off_h.assign(S + 1, 0);
    for (int s = 0; s < S; s++) B->off_h[s + 1] = B->off_h[s] + (int)N_s[s];
    B->Ntot = B->off_h[S];
    std::vector<int> tile_base(S + 1), cell_base(S + 1), row_base(S + 1), blk_base(S + 1), zblk_base(S + 1);
    std::vector<int4> items;
    for (int s = 0; s < S; s++) {
        se_plan_s *p = B->sub[s];
        tile_base[s + 1] = tile_base[s] + p->ntiles;
        cell_base[s + 1] = cell_base[s] + p->ncells;
        row_base[s + 1] = row_base[s] + p->geom.ncel[1] * p->geom.ncel[2];
        const size_t nk = (size_t)p->mf[2] * p->mf[1] * (p->mf[0] / 2 + 1);
        blk_base[s + 1] = blk_base[s] + (int)((nk + SCALE_BS - 1) / SCALE_BS);
        const size_t zrows = (size_t)3 * R * p->mt[1] * p->mt[2];
        zblk_base[s + 1] = zblk_base[s] + (int)((zrows + 7) / 8);
        for (int t = 0; t < p->ntiles; t++)
            for (int r = 0; r < R; r++) items.push_back(make_int4(s, t, r, 0));
    }
    B->ntiles_tot = tile_base[S];
    B->ncells_tot = cell_base[S];
    B->nrows_tot = row_base[S];
    B->nblk_scale = blk_base[S];
    B->nblk_zero = zblk_base[S];
    B->nitems = (int)items.size();
    // FFT size classes: systems with equal FFT sizes share one batched transform
    std::map<std::array<int, 3>, std::vector<int>> by_mf;
    for (int s = 0; s < S; s++) {
        const int *m = B->sub[s]->mf;
        by_mf[{m[0], m[1], m[2]}].push_back(s);
    }
    const size_t esz = (prec == SE_FP32) ? 4 : 8;
    std::vector<void *> grid(S), spec(S), wgrid(S);
    std::vector<std::array<size_t, 4>> strides(S);
    // FP32 with the register-column and shared-memory kernels: grids of a size
    // class interleaved plane by plane, zero-padding-aware transforms
    B->ilv = (prec == SE_FP32) && B->colk;
    size_t work_max = 0;
    for (auto &kv : by_mf) {
        se_batch_s::SizeClass c;
        for (int d = 0; d < 3; d++) c.mf[d] = kv.first[d];
        c.count = (int)kv.second.size();
        B->classes.push_back(c);
        se_batch_s::SizeClass &C = B->classes.back();
        const size_t Mf3 = (size_t)C.mf[0] * C.mf[1] * C.mf[2], nk = (size_t)C.mf[2] * C.mf[1] * (C.mf[0] / 2 + 1);
        const size_t per = (size_t)3 * R;
        if (B->ilv) {
            C.G = (size_t)C.count * per;
            C.mt2 = (size_t)B->sub[kv.second[0]]->mt[2];
            const size_t plane_r = (size_t)C.mf[1] * C.mf[0], plane_c = (size_t)C.mf[1] * (C.mf[0] / 2 + 1);
            const size_t nreal = C.G * C.mt2 * plane_r;  // [z < mt2][grid][y][x]
            if (bmalloc(&C.grid, nreal * esz) || bmalloc(&C.spec, C.G * C.mf[2] * plane_c * 2 * esz) ||
                bmalloc(&C.wgrid, nreal * esz) || cudaMemset(C.grid, 0, nreal * esz)) {
                cudaGetLastError();
                return fail(SE_ERR_OOM, "batch: grid allocation failed");
            }
            for (int j = 0; j < C.count; j++) {
                const int s = kv.second[j];
                grid[s] = (char *)C.grid + j * per * plane_r * esz;
                spec[s] = (char *)C.spec + j * per * plane_c * 2 * esz;
                wgrid[s] = (char *)C.wgrid + j * per * plane_r * esz;
                strides[s] = {C.G * plane_r, plane_r, C.G * plane_c, plane_c};
            }
            long long n2[2] = {C.mf[1], C.mf[0]}, re2[2] = {C.mf[1], C.mf[0]}, ce2[2] = {C.mf[1], C.mf[0] / 2 + 1};
            long long nz[1] = {C.mf[2]};
            const long long np = (long long)(C.G * C.mt2), ncol = (long long)(C.G * plane_c);
            size_t ws = 0;
            BCF(cufftCreate(&C.f2d));
            BCF(cufftSetAutoAllocation(C.f2d, 0));
            BCF(cufftMakePlanMany64(C.f2d, 2, n2, re2, 1, (long long)plane_r, ce2, 1, (long long)plane_c, CUFFT_R2C,
                                    np, &ws));
            work_max = std::max(work_max, ws);
            BCF(cufftCreate(&C.i2d));
            BCF(cufftSetAutoAllocation(C.i2d, 0));
            BCF(cufftMakePlanMany64(C.i2d, 2, n2, ce2, 1, (long long)plane_c, re2, 1, (long long)plane_r, CUFFT_C2R,
                                    np, &ws));
            work_max = std::max(work_max, ws);
            BCF(cufftCreate(&C.zc));
            BCF(cufftSetAutoAllocation(C.zc, 0));
            BCF(cufftMakePlanMany64(C.zc, 1, nz, nz, ncol, 1, nz, ncol, 1, CUFFT_C2C, ncol, &ws));
            work_max = std::max(work_max, ws);
            continue;
        }
        for (int j = 0; j < C.count; j++)
            strides[kv.second[j]] = {(size_t)C.mf[0] * C.mf[1], Mf3, (size_t)C.mf[1] * (C.mf[0] / 2 + 1), nk};
        if (bmalloc(&C.grid, C.count * per * Mf3 * esz) || bmalloc(&C.spec, C.count * per * nk * 2 * esz) ||
            bmalloc(&C.wgrid, C.count * per * Mf3 * esz) || cudaMemset(C.grid, 0, C.count * per * Mf3 * esz)) {
            cudaGetLastError();
            return fail(SE_ERR_OOM, "batch: grid allocation failed");
        }
        for (int j = 0; j < C.count; j++) {
            const int s = kv.second[j];
            grid[s] = (char *)C.grid + j * per * Mf3 * esz;
            spec[s] = (char *)C.spec + j * per * nk * 2 * esz;
            wgrid[s] = (char *)C.wgrid + j * per * Mf3 * esz;
        }
        long long n[3] = {C.mf[2], C.mf[1], C.mf[0]};
        const long long batch = (long long)C.count * per;
        size_t ws = 0;
        BCF(cufftCreate(&C.fwd));
        C.have_fwd = true;
        BCF(cufftSetAutoAllocation(C.fwd, 0));
        BCF(cufftMakePlanMany64(C.fwd, 3, n, nullptr, 1, (long long)Mf3, nullptr, 1, (long long)nk,
                                prec == SE_FP32 ? CUFFT_R2C : CUFFT_D2Z, batch, &ws));
        work_max = std::max(work_max, ws);
        BCF(cufftCreate(&C.inv));
        C.have_inv = true;
        BCF(cufftSetAutoAllocation(C.inv, 0));
        BCF(cufftMakePlanMany64(C.inv, 3, n, nullptr, 1, (long long)nk, nullptr, 1, (long long)Mf3,
                                prec == SE_FP32 ? CUFFT_C2R : CUFFT_Z2D, batch, &ws));
        work_max = std::max(work_max, ws);
    }
    // the transforms run one after another on one stream: one shared work area
    if (bmalloc(&B->work, work_max)) {
        cudaGetLastError();
        return fail(SE_ERR_OOM, "batch: cuFFT work area allocation failed");
    }
    for (auto &C : B->classes) {
        if (B->ilv) {
            BCF(cufftSetWorkArea(C.f2d, B->work));
            BCF(cufftSetWorkArea(C.i2d, B->work));
            BCF(cufftSetWorkArea(C.zc, B->work));
            continue;
        }
        BCF(cufftSetWorkArea(C.fwd, B->work));
        BCF(cufftSetWorkArea(C.inv, B->work));
    }
    // point buffers
    const size_t Nn = (size_t)B->Ntot, v4 = 4 * esz;
    auto scan_len = [](size_t n) { return n + 2 + (n + 4095) / 4096 + 1; };
    const size_t max_cl = Nn / 4 + B->nrows_tot + 1;  // clusters hold at least 4 targets (or end a row)
    Buffers &b = B->b;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = bmalloc(&b.xs_t, Nn * v4)) || (e = bmalloc(&b.fs_t, Nn * R * v4)) ||
            (e = bmalloc(&b.perm_t, Nn * 4)) || (e = bmalloc(&b.slot_t, Nn * 4)) ||
            (e = bmalloc(&b.key_t, Nn * 4)) || (e = bmalloc(&b.tag_t, Nn * 4)))
            break;
        if ((e = bmalloc(&b.xs_r, Nn * v4)) || (e = bmalloc(&b.fs_r, Nn * R * v4)) ||
            (e = bmalloc(&b.perm_r, Nn * 4)) || (e = bmalloc(&b.slot_r, Nn * 4)) ||
            (e = bmalloc(&b.key_r, Nn * 4)) || (e = bmalloc(&b.tag_r, Nn * 4)))
            break;
        if ((e = bmalloc(&b.cnt_t, scan_len(B->ntiles_tot) * 4)) || (e = bmalloc(&b.cnt_r, scan_len(B->ncells_tot) * 4)) ||
            (e = bmalloc(&b.ncl, scan_len(B->nrows_tot) * 4)) || (e = bmalloc(&b.clusters, max_cl * sizeof(int2))) ||
            (e = bmalloc(&B->cl_sys, max_cl * 4)) || (e = bmalloc(&b.status, 16)))
            break;
        if ((e = cudaMemset(b.status, 0, 16))) break;
        if ((e = bmalloc(&B->off_d, (S + 1) * 4)) || (e = bmalloc(&B->row_base_d, (S + 1) * 4)) ||
            (e = bmalloc(&B->blk_base_d, (S + 1) * 4)) || (e = bmalloc(&B->zblk_base_d, (S + 1) * 4)) ||
            (e = bmalloc(&B->items_d, items.size() * sizeof(int4))))
            break;
        if ((e = cudaMemcpy(B->off_d, B->off_h.data(), (S + 1) * 4, cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(B->row_base_d, row_base.data(), (S + 1) * 4, cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(B->blk_base_d, blk_base.data(), (S + 1) * 4, cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(B->zblk_base_d, zblk_base.data(), (S + 1) * 4, cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(B->items_d, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice)))
            break;
        if (prec == SE_FP32) {
            std::vector<BSys<float>> sys;
            fill_sys<float>(B, sys, tile_base, cell_base, row_base, blk_base, zblk_base, grid, spec, wgrid, strides);
            if (B->ilv) {
                // the batched gather copies its tiles with one tensor map per system
                std::vector<unsigned char> maps(S * TENSOR_MAP_BYTES, 0);
                for (int s = 0; s < S; s++)
                    sys[s].tma = encode_bgather_map(maps.data() + s * TENSOR_MAP_BYTES, sys[s].g, sys[s].wgrid,
                                                    sys[s].gzs, sys[s].gcs, R, B->P) ? 1 : 0;
                if ((e = bmalloc(&B->maps_d, maps.size()))) break;
                if ((e = cudaMemcpy(B->maps_d, maps.data(), maps.size(), cudaMemcpyHostToDevice))) break;
            }
            if ((e = bmalloc(&B->sys_d, S * sizeof(BSys<float>)))) break;
            e = cudaMemcpy(B->sys_d, sys.data(), S * sizeof(BSys<float>), cudaMemcpyHostToDevice);
        } else {
            std::vector<BSys<double>> sys;
            fill_sys<double>(B, sys, tile_base, cell_base, row_base, blk_base, zblk_base, grid, spec, wgrid, strides);
            if ((e = bmalloc(&B->sys_d, S * sizeof(BSys<double>)))) break;
            e = cudaMemcpy(B->sys_d, sys.data(), S * sizeof(BSys<double>), cudaMemcpyHostToDevice);
        }
        if (e) break;
        e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    } while (0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? SE_ERR_OOM : SE_ERR_CUDA,
                    std::string("batch allocation: ") + cudaGetErrorString(e));
    }
    return SE_OK;
}

}  // namespace

extern "C" se_status_t se_batch_create(se_kernel_t kernel, int S, const int64_t *N_s, const double *box_s, int n_rhs,
                                       double tol, se_prec_t prec, const se_params_t *params, se_batch_t *out) {
    if (!out) return fail(SE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (kernel != SE_STOKESLET && kernel != SE_ROTLET)
        return fail(SE_ERR_NOT_SUPPORTED, "se_batch_create: stokeslet and rotlet only");
    if (prec != SE_FP32 && prec != SE_FP64) return fail(SE_ERR_INVALID_ARG, "unknown precision");
    if (S < 1 || !N_s || !box_s) return fail(SE_ERR_INVALID_ARG, "se_batch_create: need S >= 1 systems");
    if (n_rhs < 1 || n_rhs > 64) return fail(SE_ERR_INVALID_ARG, "se_batch_create: n_rhs must be in [1, 64]");
    if (prec == SE_FP64 && erfc_table_init() != cudaSuccess)
        return fail(SE_ERR_CUDA, "the FP64 erfc table could not be copied to the device");
    int64_t tot = 0;
    for (int s = 0; s < S; s++) {
        if (N_s[s] < 1) return fail(SE_ERR_INVALID_ARG, "se_batch_create: every system needs N >= 1");
        if (!(box_s[4 * s + 3] > 0)) return fail(SE_ERR_INVALID_ARG, "se_batch_create: box side must be positive");
        tot += N_s[s];
    }
    if (tot * n_rhs > (int64_t)INT32_MAX / 4) return fail(SE_ERR_INVALID_ARG, "se_batch_create: too many points");
    se_batch_s *B = new se_batch_s();
    B->kernel = kernel;
    B->prec = prec;
    B->S = S;
    B->R = n_rhs;
    se_status_t s = create(B, N_s, box_s, tol, params);
    if (s != SE_OK) {
        free_batch(B);
        return s;
    }
    *out = B;
    return SE_OK;
}

extern "C" se_status_t se_batch_eval(se_batch_t B, const void *x, const void *f, void *u, void *stream) {
    if (!B || !x || !f || !u) return fail(SE_ERR_INVALID_ARG, "se_batch_eval: NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    B->last_stream = st;
    if (!B->use_graph || B->timing) return enqueue(B, x, f, u, st);
    if (!B->exec || B->gx != x || B->gf != f || B->gu != u) {
        if (B->exec) cudaGraphExecDestroy(B->exec);
        if (B->graph) cudaGraphDestroy(B->graph);
        B->exec = nullptr;
        B->graph = nullptr;
        BCK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
        se_status_t s = enqueue(B, x, f, u, B->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(B->cap, &g);
        if (s != SE_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return fail(SE_ERR_CUDA, std::string("se_batch_eval: capture: ") + cudaGetErrorString(e));
        B->graph = g;
        BCK(cudaGraphInstantiate(&B->exec, g, 0));
        B->gx = x;
        B->gf = f;
        B->gu = u;
    }
    BCK(cudaGraphLaunch(B->exec, st));
    return SE_OK;
}

extern "C" se_status_t se_batch_set_timing(se_batch_t B, int on) {
    if (!B) return fail(SE_ERR_INVALID_ARG, "NULL batch");
    if (on && !B->ev[0]) {
        for (auto &e : B->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return fail(SE_ERR_CUDA, "se_batch_set_timing: event");
    }
    B->timing = on != 0;
    B->timed = false;
    return SE_OK;
}

extern "C" int se_batch_stage_times(se_batch_t B, float *ms, int max_n) {
    if (!B || !ms || !B->timed) return 0;
    if (cudaEventSynchronize(B->ev[7]) != cudaSuccess) return 0;
    int n = 0;
    for (int k = 0; k < 7 && n < max_n; k++, n++) {
        float t = 0.0f;
        cudaEventElapsedTime(&t, B->ev[k], B->ev[k + 1]);
        ms[n] = t;
    }
    return n;
}

extern "C" se_status_t se_batch_set_graph(se_batch_t B, int on) {
    if (!B) return fail(SE_ERR_INVALID_ARG, "NULL batch");
    B->use_graph = on != 0;
    return SE_OK;
}

extern "C" se_status_t se_batch_get_params(se_batch_t B, int s, se_params_t *out) {
    if (!B || !out || s < 0 || s >= B->S) return fail(SE_ERR_INVALID_ARG, "se_batch_get_params: bad argument");
    return se_plan_get_params(B->sub[s], out);
}

extern "C" se_status_t se_batch_check(se_batch_t B) {
    if (!B) return fail(SE_ERR_INVALID_ARG, "NULL batch");
    cudaError_t e = B->last_stream ? cudaStreamSynchronize(B->last_stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(SE_ERR_CUDA, std::string("se_batch_check: ") + cudaGetErrorString(e));
    int flags = 0;
    if ((e = cudaMemcpy(&flags, B->b.status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(SE_ERR_CUDA, std::string("se_batch_check: ") + cudaGetErrorString(e));
    cudaMemset(B->b.status, 0, sizeof(int));
    if (flags & FLAG_OOB) return fail(SE_ERR_OUT_OF_BOX, "a point lies outside its system's box");
    if (flags & FLAG_COINCIDENT) return fail(SE_ERR_COINCIDENT, "coincident points were skipped");
    return SE_OK;
}

extern "C" int64_t se_batch_launch_count(se_batch_t B) { return B ? B->launches : -1; }

extern "C" se_status_t se_batch_destroy(se_batch_t B) {
    if (!B) return SE_OK;
    cudaDeviceSynchronize();
    free_batch(B);
    return SE_OK;
}
