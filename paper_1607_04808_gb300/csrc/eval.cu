// Evaluation: u = u^R + u^F + u^self (Section 8), and the gradients of
// L = sum g . u for the backward pass.
//   bin -> spread (step 1) -> R2C FFT (step 2) -> scale (step 3) -> C2R FFT
//   (step 4) -> gather + self (step 5, eq. Slimit) -> real-space sum (Section 6)
#include <algorithm>
#include <string>

#include "se_internal.cuh"

using namespace se;

namespace {

template <typename T>
cufftResult exec_fwd(cufftHandle h, void *in, void *out);
template <>
cufftResult exec_fwd<float>(cufftHandle h, void *in, void *out) {
    return cufftExecR2C(h, (cufftReal *)in, (cufftComplex *)out);
}
template <>
cufftResult exec_fwd<double>(cufftHandle h, void *in, void *out) {
    return cufftExecD2Z(h, (cufftDoubleReal *)in, (cufftDoubleComplex *)out);
}
template <typename T>
cufftResult exec_z(cufftHandle h, void *data, int dir);
template <>
cufftResult exec_z<float>(cufftHandle h, void *data, int dir) {
    return cufftExecC2C(h, (cufftComplex *)data, (cufftComplex *)data, dir);
}
template <>
cufftResult exec_z<double>(cufftHandle h, void *data, int dir) {
    return cufftExecZ2Z(h, (cufftDoubleComplex *)data, (cufftDoubleComplex *)data, dir);
}
template <typename T>
cufftResult exec_inv(cufftHandle h, void *in, void *out);
template <>
cufftResult exec_inv<float>(cufftHandle h, void *in, void *out) {
    return cufftExecC2R(h, (cufftComplex *)in, (cufftReal *)out);
}
template <>
cufftResult exec_inv<double>(cufftHandle h, void *in, void *out) {
    return cufftExecZ2D(h, (cufftDoubleComplex *)in, (cufftDoubleReal *)out);
}

struct StageTimer {
    se_plan_s *p;
    cudaStream_t st;
    int k = 0;
    void mark() {
        if (p->timing && k < 9) cudaEventRecord(p->ev[k++], st);
    }
    // stages: bin, spread, fft, scale, ifft, gather, then the real-space sum
    // split at ev_real into its set-up (cluster list) and its main kernel
    void finish() {
        if (!p->timing || k != 8) return;
        cudaEventSynchronize(p->ev[k - 1]);
        for (int i = 0; i < 6; i++) cudaEventElapsedTime(&p->stage_ms[i], p->ev[i], p->ev[i + 1]);
        cudaEventElapsedTime(&p->stage_ms[6], p->ev[6], p->ev_real);
        cudaEventElapsedTime(&p->stage_ms[7], p->ev_real, p->ev[7]);
        p->n_stage = 8;
    }
};

#define CK(expr)                                                                        \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess)                                                          \
            return fail(SE_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)
#define CF(expr)                                                                              \
    do {                                                                                      \
        cufftResult _r = (expr);                                                              \
        if (_r != CUFFT_SUCCESS)                                                              \
            return fail(SE_ERR_CUFFT, std::string(#expr) + " failed, code " + std::to_string((int)_r)); \
    } while (0)

// Fourier grid w = IFFT(scale(FFT(spread(sources)))) from the tile-sorted sources
// currently held in the plan (fs_t, qs_t).
template <typename T>
se_status_t fourier_grid(se_plan_s *p, cudaStream_t st, void *wout, int nc, StageTimer *tm) {
    CK(launch_spread<T>(p, st, p->b.xs_t, p->b.fs_t, p->b.qs_t, p->grid, nc));
    // periodic plans: the halo of the extended grid folded onto the periodic grid
    if (p->periodic) CK(launch_fold<T>(p, st, p->grid, p->pgrid, nc));
    if (tm) tm->mark();
    if (p->pruned) {
        // zero-padding-aware transforms: 2D (y, x) on the Mtilde nonzero z-planes,
        // the upper z-planes of the spectrum zeroed, then the transform along z;
        // back along z, then 2D on the Mtilde planes the gather reads
        const size_t vol_r = vol(p->geom), plane_c = (size_t)p->mf[1] * (p->mf[0] / 2 + 1);
        const size_t nk = plane_c * p->mf[2], cs = sizeof(cplx<T>);
        CF(cufftSetStream(p->f2d, st));
        CF(cufftSetStream(p->zc, st));
        CF(cufftSetStream(p->i2d, st));
        for (int c = 0; c < nc; c++)
            CF(exec_fwd<T>(p->f2d, (T *)p->grid + c * vol_r, (cplx<T> *)p->spec + c * nk));
        if (sizeof(T) == 4 && p->zw && nc == p->nc) {
            // the z-transforms, the upper planes' zeros and the scaling in one
            // kernel (zfft.cu); the stage times: fft = the 2D transforms, scale =
            // the fused kernel, ifft = the inverse 2D transforms
            if (tm) tm->mark();
            CK(launch_zscale(p, st, p->spec, nc));
            p->launches++;
            if (tm) tm->mark();
            for (int c = 0; c < 3; c++)
                CF(exec_inv<T>(p->i2d, (cplx<T> *)p->spec + c * nk, (T *)wout + c * vol_r));
            if (tm) tm->mark();
            return SE_OK;
        }
        CK(cudaMemset2DAsync((char *)p->spec + p->mt[2] * plane_c * cs, nk * cs, 0,
                             (p->mf[2] - p->mt[2]) * plane_c * cs, nc, st));
        for (int c = 0; c < nc; c++) CF(exec_z<T>(p->zc, (cplx<T> *)p->spec + c * nk, CUFFT_FORWARD));
        if (tm) tm->mark();
        CK(launch_scale<T>(p, st, p->spec, 0));
        if (tm) tm->mark();
        for (int c = 0; c < 3; c++) CF(exec_z<T>(p->zc, (cplx<T> *)p->spec + c * nk, CUFFT_INVERSE));
        for (int c = 0; c < 3; c++)
            CF(exec_inv<T>(p->i2d, (cplx<T> *)p->spec + c * nk, (T *)wout + c * vol_r));
        if (tm) tm->mark();
        return SE_OK;
    }
    cufftHandle fwd = (nc == p->nc) ? p->fwd : p->fwd3;
    CF(cufftSetStream(fwd, st));
    CF(exec_fwd<T>(fwd, p->periodic ? p->pgrid : p->grid, p->spec));
    if (tm) tm->mark();
    CK(launch_scale<T>(p, st, p->spec, 0));
    if (tm) tm->mark();
    CF(cufftSetStream(p->inv, st));
    CF(exec_inv<T>(p->inv, p->spec, p->periodic ? p->pgrid : wout));
    if (p->periodic) CK(launch_unfold<T>(p, st, p->pgrid, wout, 3));
    if (tm) tm->mark();
    return SE_OK;
}

// The forward grid in wgrid now belongs to the sources (x, f, q).
void mark_grid(se_plan_s *p, const void *x, const void *f, const void *q) {
    p->grid_valid = true;
    p->grid_src[0] = x;
    p->grid_src[1] = f;
    p->grid_src[2] = q;
}

bool grid_kept_for(const se_plan_s *p, const void *x, const void *f, const void *q) {
    return p->keep_grid && p->grid_valid && p->grid_src[0] == x && p->grid_src[1] == f && p->grid_src[2] == q;
}

template <typename T>
se_status_t eval_t(se_plan_s *p, const T *x, const T *f, const T *q, T *u, cudaStream_t st) {
    p->last_stream = st;
    p->launches = 0;
    p->grid_valid = false;
    if (p->overlap && !p->timing && p->s_four && real_can_defer(p)) {
        // the Fourier part (spread ... gather, which writes u) on the internal
        // high-priority stream, the real-space sum (into b.rt and b.uj) on st;
        // both read the sorted points, then st adds the real-space sums to u
        CK(launch_bin<T>(p, x, f, q, st));
        CK(cudaEventRecord(p->ev_fork, st));
        CK(cudaStreamWaitEvent(p->s_four, p->ev_fork, 0));
        se_status_t s = fourier_grid<T>(p, p->s_four, p->wgrid, p->nc, nullptr);
        if (s != SE_OK) return s;
        mark_grid(p, x, f, q);
        CK(launch_gather<T>(p, p->s_four, p->wgrid, f, u));
        CK(cudaEventRecord(p->ev_join, p->s_four));
        CK(launch_real<T>(p, st, u, true));
        CK(cudaStreamWaitEvent(st, p->ev_join, 0));
        CK(launch_add_uj<T>(p, st, u));
        return SE_OK;
    }
    StageTimer tm{p, st};
    tm.mark();
    CK(launch_bin<T>(p, x, f, q, st));
    tm.mark();
    se_status_t s = fourier_grid<T>(p, st, p->wgrid, p->nc, &tm);
    if (s != SE_OK) return s;
    mark_grid(p, x, f, q);
    CK(launch_gather<T>(p, st, p->wgrid, f, u));
    tm.mark();
    CK(launch_real<T>(p, st, u));
    tm.mark();
    tm.finish();
    return SE_OK;
}

// Stage timing of se_eval_backward: events around its eight steps (a step it
// skips records an empty interval).
struct BackTimer {
    se_plan_s *p;
    cudaStream_t st;
    int k = 0;
    void mark() {
        if (p->timing && k < 9) cudaEventRecord(p->ev[k++], st);
    }
    void finish() {
        if (!p->timing || k != 9) return;
        cudaEventSynchronize(p->ev[8]);
        for (int i = 0; i < 8; i++) cudaEventElapsedTime(&p->stage_ms[i], p->ev[i], p->ev[i + 1]);
        p->n_stage = 8;
    }
};

template <typename T>
se_status_t backward_t(se_plan_s *p, const T *x, const T *f, const T *q, const T *gu, T *gf, T *gq, T *gx,
                       cudaStream_t st) {
    p->last_stream = st;
    p->launches = 0;
    BackTimer tm{p, st};
    tm.mark();
    const size_t Mf3 = (size_t)p->mf[0] * p->mf[1] * p->mf[2];
    const bool stress = (p->kernel == SE_STRESSLET);
    if (!p->wgrid2) {
        cudaError_t e = cudaMalloc(&p->wgrid2, (stress ? 6 : 3) * Mf3 * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SE_ERR_OOM, "backward: adjoint grid allocation failed");
        }
    }
    if (gx && !p->gsort) {
        cudaError_t e = cudaMalloc(&p->gsort, (size_t)p->N * 4 * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SE_ERR_OOM, "backward: gradient buffer allocation failed");
        }
    }
    // adjoint field from the upstream gradient g: w' = K^T g on the grid (the
    // stokeslet and rotlet multipliers are their own transposes); for the
    // stresslet the symmetric tensor field V_lk = sum_m T_jlk(x_m - y) g_mj
    CK(launch_bin<T>(p, x, gu, nullptr, st));
    tm.mark();
    se_status_t s;
    if (stress) {
        const size_t nk = (size_t)p->mf[2] * p->mf[1] * (p->mf[0] / 2 + 1);
        CK(launch_spread<T>(p, st, p->b.xs_t, p->b.fs_t, nullptr, p->grid, 3));
        if (p->pruned) {
            // the zero-padding-aware transforms of the forward evaluation: three
            // source grids in, the six components of V out (the gathers read
            // only the z < Mtilde planes)
            const size_t plane_c = (size_t)p->mf[1] * (p->mf[0] / 2 + 1), cs = sizeof(cplx<T>);
            CF(cufftSetStream(p->f2d, st));
            CF(cufftSetStream(p->zc, st));
            CF(cufftSetStream(p->i2d, st));
            for (int c = 0; c < 3; c++)
                CF(exec_fwd<T>(p->f2d, (T *)p->grid + c * Mf3, (cplx<T> *)p->spec + c * nk));
            CK(cudaMemset2DAsync((char *)p->spec + p->mt[2] * plane_c * cs, nk * cs, 0,
                                 (p->mf[2] - p->mt[2]) * plane_c * cs, 3, st));
            for (int c = 0; c < 3; c++) CF(exec_z<T>(p->zc, (cplx<T> *)p->spec + c * nk, CUFFT_FORWARD));
            CK(launch_scale_adj_stresslet<T>(p, st, p->spec));
            for (int c = 0; c < 6; c++) CF(exec_z<T>(p->zc, (cplx<T> *)p->spec + c * nk, CUFFT_INVERSE));
            for (int c = 0; c < 6; c++)
                CF(exec_inv<T>(p->i2d, (cplx<T> *)p->spec + c * nk, (T *)p->wgrid2 + c * Mf3));
        } else {
            CF(cufftSetStream(p->fwd3, st));
            CF(exec_fwd<T>(p->fwd3, p->grid, p->spec));
            CK(launch_scale_adj_stresslet<T>(p, st, p->spec));
            CF(cufftSetStream(p->inv, st));
            CF(exec_inv<T>(p->inv, p->spec, p->wgrid2));
            CF(exec_inv<T>(p->inv, (cplx<T> *)p->spec + 3 * nk, (T *)p->wgrid2 + 3 * Mf3));
        }
        tm.mark();
        if (gf || gq) CK(launch_gather_adjT<T>(p, st, p->wgrid2, f, q, gf, gq));
        tm.mark();
        if (gf || gq) CK(launch_real_adjT<T>(p, st, f, q, gf, gq));
        tm.mark();
    } else {
        s = fourier_grid<T>(p, st, p->wgrid2, 3, nullptr);
        if (s != SE_OK) return s;
        tm.mark();
        // transposed operator applied to g: same kernel (S and Omega are symmetric operators)
        if (gf) CK(launch_gather<T>(p, st, p->wgrid2, gu, gf));
        tm.mark();
        if (gf) CK(launch_real<T>(p, st, gf));
        tm.mark();
    }
    if (gx) CK(launch_bin<T>(p, x, f, q, st));
    tm.mark();
    if (gx && !grid_kept_for(p, x, f, q)) {
        // the forward grid, recomputed (the grid of the plan's last evaluation
        // is reused instead when keep-grid is on and the sources are the same)
        p->grid_valid = false;
        s = fourier_grid<T>(p, st, p->wgrid, p->nc, nullptr);
        if (s != SE_OK) return s;
        mark_grid(p, x, f, q);
    }
    tm.mark();
    if (gx) CK(launch_gather_grad<T>(p, st, p->wgrid, p->wgrid2, f, q, gu, gx));
    tm.mark();
    if (gx) CK(launch_real_grad<T>(p, st, gu, gx));
    tm.mark();
    tm.finish();
    return SE_OK;
}

}  // namespace

extern "C" se_status_t se_eval(se_plan_t p, const void *x, const void *f, const void *q, void *u, void *stream) {
    if (!p || !x || !f || !u) return fail(SE_ERR_INVALID_ARG, "se_eval: NULL pointer");
    if (p->kernel == SE_STRESSLET && !q) return fail(SE_ERR_INVALID_ARG, "se_eval: the stresslet needs q");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prec == SE_FP32)
        return eval_t<float>(p, (const float *)x, (const float *)f, (const float *)q, (float *)u, st);
    return eval_t<double>(p, (const double *)x, (const double *)f, (const double *)q, (double *)u, st);
}

extern "C" se_status_t se_eval_real_space(se_plan_t p, const void *x, const void *f, const void *q, void *u,
                                          void *stream) {
    if (!p || !x || !f || !u) return fail(SE_ERR_INVALID_ARG, "se_eval_real_space: NULL pointer");
    if (p->kernel == SE_STRESSLET && !q) return fail(SE_ERR_INVALID_ARG, "se_eval_real_space: the stresslet needs q");
    cudaStream_t st = (cudaStream_t)stream;
    p->last_stream = st;
    p->launches = 0;
    const size_t bytes = (size_t)p->N * 3 * (p->prec == SE_FP32 ? 4 : 8);
    CK(cudaMemsetAsync(u, 0, bytes, st));
    if (p->prec == SE_FP32) {
        CK(launch_bin<float>(p, (const float *)x, (const float *)f, (const float *)q, st));
        CK(launch_real<float>(p, st, (float *)u));
    } else {
        CK(launch_bin<double>(p, (const double *)x, (const double *)f, (const double *)q, st));
        CK(launch_real<double>(p, st, (double *)u));
    }
    return SE_OK;
}

// Room for Nt evaluation targets in the plan's target buffers (grown on demand).
static se_status_t ensure_targets(se_plan_s *p, int64_t Nt) {
    if (Nt <= p->nt_cap) return SE_OK;
    Buffers &b = p->bt;
    void *old[] = {b.xs_t, b.perm_t, b.slot_t, b.key_t, b.tag_t, b.cnt_t, b.xs_r, b.perm_r, b.slot_r, b.key_r,
                   b.tag_r, b.cnt_r, b.ncl, b.clusters};
    cudaDeviceSynchronize();
    for (void *q : old)
        if (q) cudaFree(q);
    b = Buffers();
    p->nt_cap = 0;
    const size_t n = (size_t)Nt, v4 = (p->prec == SE_FP32 ? 16 : 32);
    const size_t nrows = (size_t)p->geom.ncel[1] * p->geom.ncel[2];
    auto scan_len = [](size_t k) { return k + 2 + (k + 4095) / 4096 + 1; };
    cudaError_t e;
    if ((e = cudaMalloc(&b.xs_t, n * v4)) || (e = cudaMalloc(&b.perm_t, n * 4)) || (e = cudaMalloc(&b.slot_t, n * 4)) ||
        (e = cudaMalloc(&b.key_t, n * 4)) || (e = cudaMalloc(&b.tag_t, n * 4)) ||
        (e = cudaMalloc(&b.cnt_t, scan_len(p->ntiles) * 4)) || (e = cudaMalloc(&b.xs_r, n * v4)) ||
        (e = cudaMalloc(&b.perm_r, n * 4)) || (e = cudaMalloc(&b.slot_r, n * 4)) || (e = cudaMalloc(&b.key_r, n * 4)) ||
        (e = cudaMalloc(&b.tag_r, n * 4)) || (e = cudaMalloc(&b.cnt_r, scan_len(p->ncells) * 4)) ||
        (e = cudaMalloc(&b.ncl, scan_len(nrows) * 4)) || (e = cudaMalloc(&b.clusters, (n / 4 + nrows + 1) * sizeof(int2)))) {
        cudaGetLastError();
        return fail(SE_ERR_OOM, "se_eval_targets: target buffer allocation failed");
    }
    b.status = p->b.status;
    p->nt_cap = Nt;
    if (p->deterministic && Nt > p->rs_cap) {
        int *rs = nullptr;
        if (cudaMalloc(&rs, stable_scratch_ints(Nt) * sizeof(int))) {
            cudaGetLastError();
            return fail(SE_ERR_OOM, "se_eval_targets: scratch of the stable bin order");
        }
        cudaFree(p->rs_scratch);
        p->rs_scratch = rs;
        p->rs_cap = Nt;
    }
    return SE_OK;
}

extern "C" se_status_t se_plan_set_deterministic(se_plan_t p, int on) {
    if (!p) return fail(SE_ERR_INVALID_ARG, "se_plan_set_deterministic: NULL plan");
    if (!on) {
        p->deterministic = false;
        return SE_OK;
    }
    if (p->prec != SE_FP32 || p->periodic || !p->colk)
        return fail(SE_ERR_NOT_SUPPORTED,
                    "se_plan_set_deterministic: FP32 free-space plans with the register-column kernels only");
    const int64_t cap = std::max<int64_t>(p->N, p->nt_cap);
    cudaDeviceSynchronize();
    if (cap > p->rs_cap) {
        int *rs = nullptr;
        if (cudaMalloc(&rs, stable_scratch_ints(cap) * sizeof(int))) {
            cudaGetLastError();
            return fail(SE_ERR_OOM, "se_plan_set_deterministic: scratch of the stable bin order");
        }
        cudaFree(p->rs_scratch);
        p->rs_scratch = rs;
        p->rs_cap = cap;
    }
    if (!p->tilebuf && cudaMalloc(&p->tilebuf, tilebuf_floats(p->P, p->ntiles) * sizeof(float))) {
        cudaGetLastError();
        p->tilebuf = nullptr;
        return fail(SE_ERR_OOM, "se_plan_set_deterministic: tile buffer of the atomic-free spreading");
    }
    p->deterministic = true;
    return SE_OK;
}

template <typename T>
se_status_t eval_targets_t(se_plan_s *p, const T *x, const T *f, const T *q, int Nt, const T *xt, T *ut,
                           cudaStream_t st) {
    p->last_stream = st;
    p->launches = 0;
    CK(launch_bin<T>(p, x, f, q, st));
    CK(launch_bin_set<T>(p, p->bt, Nt, xt, nullptr, nullptr, st));
    p->grid_valid = false;
    se_status_t s = fourier_grid<T>(p, st, p->wgrid, p->nc, nullptr);
    if (s != SE_OK) return s;
    mark_grid(p, x, f, q);
    CK(launch_gather_targets<T>(p, st, p->bt, Nt, p->wgrid, ut));
    CK(launch_real_targets<T>(p, st, p->bt, Nt, ut));
    return SE_OK;
}

extern "C" se_status_t se_eval_targets(se_plan_t p, const void *x, const void *f, const void *q, int64_t Nt,
                                       const void *xt, void *ut, void *stream) {
    if (!p || !x || !f || !xt || !ut) return fail(SE_ERR_INVALID_ARG, "se_eval_targets: NULL pointer");
    if (p->kernel == SE_STRESSLET && !q) return fail(SE_ERR_INVALID_ARG, "se_eval_targets: the stresslet needs q");
    if (Nt < 1 || Nt > (int64_t)INT32_MAX / 4) return fail(SE_ERR_INVALID_ARG, "se_eval_targets: Nt out of range");
    if (p->periodic) return fail(SE_ERR_NOT_SUPPORTED, "se_eval_targets: not available for periodic plans");
    se_status_t s = ensure_targets(p, Nt);
    if (s != SE_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prec == SE_FP32)
        return eval_targets_t<float>(p, (const float *)x, (const float *)f, (const float *)q, (int)Nt,
                                     (const float *)xt, (float *)ut, st);
    return eval_targets_t<double>(p, (const double *)x, (const double *)f, (const double *)q, (int)Nt,
                                  (const double *)xt, (double *)ut, st);
}

extern "C" se_status_t se_eval_host(se_plan_t p, const void *x, const void *f, const void *q, void *u,
                                    void *stream) {
    if (!p || !x || !f || !u) return fail(SE_ERR_INVALID_ARG, "se_eval_host: NULL pointer");
    if (p->kernel == SE_STRESSLET && !q) return fail(SE_ERR_INVALID_ARG, "se_eval_host: the stresslet needs q");
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = (size_t)p->N * 3 * (p->prec == SE_FP32 ? 4 : 8);
    if (!p->dx) {
        if (cudaMalloc(&p->dx, bytes) || cudaMalloc(&p->df, bytes) || cudaMalloc(&p->du, bytes) ||
            (p->kernel == SE_STRESSLET && cudaMalloc(&p->dq, bytes))) {
            cudaGetLastError();
            return fail(SE_ERR_OOM, "se_eval_host: staging allocation failed");
        }
    }
    CK(cudaMemcpyAsync(p->dx, x, bytes, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(p->df, f, bytes, cudaMemcpyHostToDevice, st));
    if (q) CK(cudaMemcpyAsync(p->dq, q, bytes, cudaMemcpyHostToDevice, st));
    se_status_t s = se_eval(p, p->dx, p->df, q ? p->dq : nullptr, p->du, stream);
    if (s != SE_OK) return s;
    CK(cudaMemcpyAsync(u, p->du, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SE_OK;
}

extern "C" se_status_t se_eval_backward_q(se_plan_t p, const void *x, const void *f, const void *q,
                                          const void *grad_u, void *grad_f, void *grad_q, void *grad_x,
                                          void *stream) {
    if (!p || !x || !f || !grad_u) return fail(SE_ERR_INVALID_ARG, "se_eval_backward: NULL pointer");
    if (p->kernel == SE_STRESSLET && !q) return fail(SE_ERR_INVALID_ARG, "se_eval_backward: the stresslet needs q");
    if (p->kernel != SE_STRESSLET && grad_q)
        return fail(SE_ERR_INVALID_ARG, "se_eval_backward: grad_q is for the stresslet only");
    if (!grad_f && !grad_q && !grad_x) return SE_OK;
    if (p->periodic) return fail(SE_ERR_NOT_SUPPORTED, "se_eval_backward: not available for periodic plans");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prec == SE_FP32)
        return backward_t<float>(p, (const float *)x, (const float *)f, (const float *)q, (const float *)grad_u,
                                 (float *)grad_f, (float *)grad_q, (float *)grad_x, st);
    return backward_t<double>(p, (const double *)x, (const double *)f, (const double *)q, (const double *)grad_u,
                              (double *)grad_f, (double *)grad_q, (double *)grad_x, st);
}

extern "C" se_status_t se_eval_backward(se_plan_t p, const void *x, const void *f, const void *q, const void *grad_u,
                                        void *grad_f, void *grad_x, void *stream) {
    return se_eval_backward_q(p, x, f, q, grad_u, grad_f, nullptr, grad_x, stream);
}
