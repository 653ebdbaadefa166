// Precomputation of the mollified truncated Green's function (Section 4.3), FP64:
//  1. B^R(k) (eq. BhatR; stokeslet, stresslet) or H^R(k) (eq. HhatR; rotlet) on
//     the oversampled Mg0 x Mg1 x Mg2 grid, k_d = 2 pi kbar_d / (Mg_d h), R the
//     diagonal of the extended box; only the half spectrum kx in [0, Mg0/2] is
//     formed (the data are real and even);
//  2. inverse FFT (complex-to-real), normalised by 1/(Mg0 Mg1 Mg2);
//  3. keep the 2 Mt_d values per dimension centred at zero (j in [-Mt_d, Mt_d-1]),
//     stored wrap-ordered on the (2 Mt0) x (2 Mt1) x (2 Mt2) grid;
//  4. forward FFT (real-to-complex); the result is real and even, so the
//     (Mt0+1)(Mt1+1)(Mt2+1) octant of its real part is all the scaling step needs.
// The data of every step are real and even in each dimension (B^R and H^R are
// radial), so each 3-D transform is taken on the octant (Section 4.3 does not
// prescribe how): three passes of batched 1-D transforms, one per dimension,
// over the octant's lines only, each line extended evenly to the full period,
// its real part kept and, in the first transform, only the Mt_d + 1 outputs
// the truncation keeps.  Against the full 3-D transforms this evaluates B^R on
// an eighth of the points and transforms a quarter of the lines, with the same
// sums; large oversampled grids take it (SE_PRECOMPUTE_OCTANT = 0: never).
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "se_internal.cuh"

namespace se {

namespace {

// Truncated biharmonic transform, with its Taylor series for R k < 1 where the
// closed form cancels (4 pi sum_n (-1)^n k^{2n} R^{2n+4} / ((2n+1)! (2n+4))).
__device__ double bhat_trunc(double k, double R) {
    double x = R * k;
    if (x < 1.0) {
        double s = 0.0, term = R * R * R * R;  // n = 0: R^4 / (1! * 4)
        double fact = 1.0;                      // (2n+1)!
        double pk = 1.0;                        // (kR)^{2n}
        for (int n = 0; n < 12; n++) {
            if (n > 0) {
                fact *= (2.0 * n) * (2.0 * n + 1.0);
                pk *= -x * x;
            }
            s += pk * term / (fact * (2.0 * n + 4.0));
        }
        return 4.0 * M_PI * s;
    }
    double k4 = k * k * k * k;
    return 4.0 * M_PI * ((2.0 - x * x) * cos(x) + 2.0 * x * sin(x) - 2.0) / k4;
}

__device__ double hhat_trunc(double k, double R) {
    if (k == 0.0) return 2.0 * M_PI * R * R;
    double s = sin(R * k / 2.0) / k;
    return 8.0 * M_PI * s * s;
}

struct Dims3 {
    int n[3];
};

__global__ void k_eval_truncated(Dims3 mg, double3 dk, double R, int harmonic, cufftDoubleComplex *out) {
    const int nxh = mg.n[0] / 2 + 1;
    size_t nk = (size_t)mg.n[2] * mg.n[1] * nxh;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nk) return;
    int kx = idx % nxh;
    int ky = (idx / nxh) % mg.n[1];
    int kz = idx / ((size_t)nxh * mg.n[1]);
    int by = (ky < mg.n[1] / 2) ? ky : ky - mg.n[1];
    int bz = (kz < mg.n[2] / 2) ? kz : kz - mg.n[2];
    const double qx = dk.x * kx, qy = dk.y * by, qz = dk.z * bz;
    double kk = sqrt(qx * qx + qy * qy + qz * qz);
    double v = harmonic ? hhat_trunc(kk, R) : bhat_trunc(kk, R);
    out[idx] = make_cuDoubleComplex(v, 0.0);
}

// Gt[j mod Mf] = G[j mod Mg] / (Mg0 Mg1 Mg2) for j_d in [-Mt_d, Mt_d-1]
__global__ void k_truncate(Dims3 mg, Dims3 mt, double scale, const double *G, double *Gt) {
    const int fx = 2 * mt.n[0], fy = 2 * mt.n[1], fz = 2 * mt.n[2];
    size_t n = (size_t)fx * fy * fz;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int ix = idx % fx, iy = (idx / fx) % fy, iz = idx / ((size_t)fx * fy);
    // destination index i holds j = i (i < Mt) or i - Mf (i >= Mt)
    int jx = ix < mt.n[0] ? ix : ix - fx;
    int jy = iy < mt.n[1] ? iy : iy - fy;
    int jz = iz < mt.n[2] ? iz : iz - fz;
    int sx = (jx + mg.n[0]) % mg.n[0], sy = (jy + mg.n[1]) % mg.n[1], sz = (jz + mg.n[2]) % mg.n[2];
    Gt[idx] = G[((size_t)sz * mg.n[1] + sy) * mg.n[0] + sx] * scale;
}

__global__ void k_octant(Dims3 mt, const cufftDoubleComplex *spec, double *oct64, float *oct32) {
    const int fy = 2 * mt.n[1], nxh = mt.n[0] + 1;
    const int ox = mt.n[0] + 1, oy = mt.n[1] + 1, oz = mt.n[2] + 1;
    size_t n = (size_t)ox * oy * oz;
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    int ax = idx % ox, ay = (idx / ox) % oy, az = idx / ((size_t)ox * oy);
    double v = spec[((size_t)az * fy + ay) * nxh + ax].x;
    oct64[idx] = v;
    if (oct32) oct32[idx] = (float)v;
}

// B^R or H^R at kbar_d in [0, Mg_d / 2] (the octant of the even data), x fastest
__global__ void k_eval_octant(Dims3 a, double3 dk, double R, int harmonic, double *out) {
    const size_t n = (size_t)a.n[0] * a.n[1] * a.n[2];
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int x = idx % a.n[0], y = (idx / a.n[0]) % a.n[1], z = idx / ((size_t)a.n[0] * a.n[1]);
    const double qx = dk.x * x, qy = dk.y * y, qz = dk.z * z;
    const double kk = sqrt(qx * qx + qy * qy + qz * qz);
    out[idx] = harmonic ? hhat_trunc(kk, R) : bhat_trunc(kk, R);
}

// Lines of h + 1 values (j = 0 .. h, the fastest dimension of `in`) extended
// evenly to the period 2h: ext[l][i] = in[l][i <= h ? i : 2h - i].
__global__ void k_even_extend(const double *in, int h, size_t L, double *ext) {
    const size_t n = L * 2 * (size_t)h;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const size_t l = idx / (2 * h);
    const int i = (int)(idx - l * 2 * h);
    ext[idx] = in[l * (h + 1) + (i <= h ? i : 2 * h - i)];
}

// The real parts of the lines' transforms (h + 1 complex values per line),
// outputs k < kout, times scale, written with the dimensions rotated: line l
// = s_i m + m_i of the input (dimensions fast, m, s) goes to out[k][s_i][m_i].
__global__ void k_rotate_real(const cufftDoubleComplex *spec, int h, int m, int s, int kout, double scale,
                              double *out) {
    const size_t n = (size_t)kout * s * m;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int mi = idx % m, si = (idx / m) % s, k = idx / ((size_t)m * s);
    out[idx] = spec[((size_t)si * m + mi) * (h + 1) + k].x * scale;
}

// One pass: the transform along the fastest dimension of in (dimensions f = h
// + 1, m, s) of data even in that dimension, outputs k < kout, rotated into out
// (dimensions m, s, kout).  ext, spec: work arrays of at least m s 2h doubles
// and m s (h + 1) complex values.
se_status_t even_pass(const double *in, int h, int m, int s, int kout, double scale, double *ext,
                      cufftDoubleComplex *spec, double *out) {
    const size_t L = (size_t)m * s;
    k_even_extend<<<(unsigned)((L * 2 * h + 255) / 256), 256>>>(in, h, L, ext);
    cufftHandle plan = 0;
    int nn = 2 * h;
    if (cufftPlanMany(&plan, 1, &nn, nullptr, 1, nn, nullptr, 1, h + 1, CUFFT_D2Z, (int)L) != CUFFT_SUCCESS)
        return fail(SE_ERR_CUFFT, "precompute: D2Z line plan failed");
    const cufftResult r = cufftExecD2Z(plan, ext, spec);
    cufftDestroy(plan);
    if (r != CUFFT_SUCCESS) return fail(SE_ERR_CUFFT, "precompute: D2Z lines failed");
    const size_t no = (size_t)kout * s * m;
    k_rotate_real<<<(unsigned)((no + 255) / 256), 256>>>(spec, h, m, s, kout, scale, out);
    return SE_OK;
}

__global__ void k_to_f32(size_t n, const double *in, float *out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

#ifndef SE_PRECOMPUTE_OCTANT
#define SE_PRECOMPUTE_OCTANT 1
#endif

// Steps 1-4 on the octant of the even data.
se_status_t precompute_octant(se_plan_s *p) {
    const int n0 = p->mg[0] / 2, n1 = p->mg[1] / 2, n2 = p->mg[2] / 2;   // half periods of the first transform
    const int t0 = p->mt[0], t1 = p->mt[1], t2 = p->mt[2];                // kept outputs - 1; half periods of the second
    const size_t a_oct = (size_t)(n0 + 1) * (n1 + 1) * (n2 + 1);
    const size_t b1 = (size_t)(t0 + 1) * (n1 + 1) * (n2 + 1), b2 = (size_t)(t0 + 1) * (t1 + 1) * (n2 + 1);
    const size_t g_oct = (size_t)(t0 + 1) * (t1 + 1) * (t2 + 1);
    // work arrays: the extended lines of a pass and their spectra (the largest pass's)
    const size_t L1 = (size_t)(n1 + 1) * (n2 + 1);
    size_t ext_n = std::max({L1 * 2 * n0, (size_t)(n2 + 1) * (t0 + 1) * 2 * n1, (size_t)(t0 + 1) * (t1 + 1) * 2 * n2,
                             (size_t)(t1 + 1) * (t2 + 1) * 2 * t0, (size_t)(t2 + 1) * (t0 + 1) * 2 * t1,
                             (size_t)(t0 + 1) * (t1 + 1) * 2 * t2});
    size_t spec_n = std::max({L1 * (n0 + 1), (size_t)(n2 + 1) * (t0 + 1) * (n1 + 1),
                              (size_t)(t0 + 1) * (t1 + 1) * (n2 + 1), (size_t)(t1 + 1) * (t2 + 1) * (t0 + 1)});
    double *A = nullptr, *B = nullptr, *ext = nullptr;
    cufftDoubleComplex *spec = nullptr;
    auto cleanup = [&]() {
        cudaFree(A);
        cudaFree(B);
        cudaFree(ext);
        cudaFree(spec);
    };
    if (cudaMalloc(&A, std::max(a_oct, b2) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&B, std::max(b1, g_oct) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ext, ext_n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&spec, spec_n * sizeof(cufftDoubleComplex)) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(SE_ERR_OOM, "precompute: device allocation failed");
    }
    const Dims3 a{{n0 + 1, n1 + 1, n2 + 1}};
    const double3 dk = make_double3(2.0 * M_PI / (p->mg[0] * p->h), 2.0 * M_PI / (p->mg[1] * p->h),
                                    2.0 * M_PI / (p->mg[2] * p->h));
    k_eval_octant<<<(unsigned)((a_oct + 255) / 256), 256>>>(a, dk, p->R, p->kernel == SE_ROTLET, A);
    // first transform (inverse, normalised by 1/(Mg0 Mg1 Mg2)): x, y, z passes,
    // keeping j_d in [0, Mt_d] (the wrap-ordered truncation window's octant)
    const double norm = 1.0 / ((double)p->mg[0] * p->mg[1] * p->mg[2]);
    se_status_t st = SE_OK;
    // A [z][y][x] (n0+1 fastest) -> B [jx][z][y]
    if (st == SE_OK) st = even_pass(A, n0, n1 + 1, n2 + 1, t0 + 1, 1.0, ext, spec, B);
    // B [jx][z][y] -> A [jy][jx][z]
    if (st == SE_OK) st = even_pass(B, n1, n2 + 1, t0 + 1, t1 + 1, 1.0, ext, spec, A);
    // A [jy][jx][z] -> B [jz][jy][jx] = G on the octant of the truncation window
    if (st == SE_OK) st = even_pass(A, n2, t0 + 1, t1 + 1, t2 + 1, norm, ext, spec, B);
    // second transform (forward) of G, even with the periods 2 Mt_d: the octant
    // of the real, even result
    if (st == SE_OK) st = even_pass(B, t0, t1 + 1, t2 + 1, t0 + 1, 1.0, ext, spec, A);
    if (st == SE_OK) st = even_pass(A, t1, t2 + 1, t0 + 1, t1 + 1, 1.0, ext, spec, B);
    if (st == SE_OK) st = even_pass(B, t2, t0 + 1, t1 + 1, t2 + 1, 1.0, ext, spec, p->ghat64);
    if (st == SE_OK && p->prec == SE_FP32)
        k_to_f32<<<(unsigned)((g_oct + 255) / 256), 256>>>(g_oct, p->ghat64, (float *)p->ghat);
    const cudaError_t ce = cudaDeviceSynchronize();
    cleanup();
    if (st == SE_OK && ce != cudaSuccess) st = fail(SE_ERR_CUDA, std::string("precompute: ") + cudaGetErrorString(ce));
    return st;
}

// The octant passes from this many points of the oversampled grid on (512^3):
// below it the full 3-D transforms are as fast once warm, and the first
// transform of a new line length in a process costs cuFFT 25 to 75 ms of
// set-up (measured on GB300: FP64 1-D transforms of lengths 252, 350 and 800),
// which the full transforms' kernels do not.  FP64 at 1e-10, N = 1e6 (Mg =
// 800): 158 -> 54 ms (80 ms in a process's first plan); the FP32 plan of the
// same points (Mg = 350) keeps the full transforms (16 ms).
constexpr double OCTANT_MIN_POINTS = 134217728.0;

se_status_t precompute_compute(se_plan_s *p) {
    if (SE_PRECOMPUTE_OCTANT && (double)p->mg[0] * p->mg[1] * p->mg[2] >= OCTANT_MIN_POINTS) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, 0);
        se_status_t st = precompute_octant(p);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        p->precompute_ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (p->prec == SE_FP64 && st == SE_OK) p->ghat = p->ghat64;
        return st;
    }
    const Dims3 mg{{p->mg[0], p->mg[1], p->mg[2]}}, mt{{p->mt[0], p->mt[1], p->mt[2]}};
    const size_t nkg = (size_t)mg.n[2] * mg.n[1] * (mg.n[0] / 2 + 1);
    const size_t ng = (size_t)mg.n[2] * mg.n[1] * mg.n[0];
    const size_t nf = (size_t)p->mf[0] * p->mf[1] * p->mf[2];
    const size_t nkf = (size_t)p->mf[2] * p->mf[1] * (p->mf[0] / 2 + 1);
    cufftDoubleComplex *spec = nullptr;
    double *G = nullptr;
    cufftHandle plan = 0;
    se_status_t st = SE_OK;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, 0);
    auto cleanup = [&]() {
        if (plan) cufftDestroy(plan);
        cudaFree(spec);
        cudaFree(G);
    };
    size_t big = nkg > nkf ? nkg : nkf;
    if (cudaMalloc(&spec, big * sizeof(cufftDoubleComplex)) != cudaSuccess ||
        cudaMalloc(&G, (ng > nf ? ng : nf) * sizeof(double)) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(SE_ERR_OOM, "precompute: device allocation failed");
    }
    const double3 dk = make_double3(2.0 * M_PI / (mg.n[0] * p->h), 2.0 * M_PI / (mg.n[1] * p->h),
                                    2.0 * M_PI / (mg.n[2] * p->h));
    int harmonic = (p->kernel == SE_ROTLET);
    k_eval_truncated<<<(unsigned)((nkg + 255) / 256), 256>>>(mg, dk, p->R, harmonic, spec);
    if (cufftPlan3d(&plan, mg.n[2], mg.n[1], mg.n[0], CUFFT_Z2D) != CUFFT_SUCCESS) {
        cleanup();
        return fail(SE_ERR_CUFFT, "precompute: Z2D plan failed");
    }
    if (cufftExecZ2D(plan, spec, G) != CUFFT_SUCCESS) {
        cleanup();
        return fail(SE_ERR_CUFFT, "precompute: Z2D failed");
    }
    cufftDestroy(plan);
    plan = 0;
    double *Gt = nullptr;
    double *Gt_buf = nullptr;
    if (cudaMalloc(&Gt_buf, nf * sizeof(double)) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(SE_ERR_OOM, "precompute: device allocation failed");
    }
    Gt = Gt_buf;
    k_truncate<<<(unsigned)((nf + 255) / 256), 256>>>(mg, mt, 1.0 / (double)ng, G, Gt);
    if (cufftPlan3d(&plan, p->mf[2], p->mf[1], p->mf[0], CUFFT_D2Z) != CUFFT_SUCCESS) {
        cudaFree(Gt_buf);
        cleanup();
        return fail(SE_ERR_CUFFT, "precompute: D2Z plan failed");
    }
    if (cufftExecD2Z(plan, Gt, spec) != CUFFT_SUCCESS) {
        cudaFree(Gt_buf);
        cleanup();
        return fail(SE_ERR_CUFFT, "precompute: D2Z failed");
    }
    size_t no = (size_t)(mt.n[0] + 1) * (mt.n[1] + 1) * (mt.n[2] + 1);
    k_octant<<<(unsigned)((no + 255) / 256), 256>>>(mt, spec, p->ghat64,
                                                    p->prec == SE_FP32 ? (float *)p->ghat : nullptr);
    cudaError_t ce = cudaDeviceSynchronize();
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    p->precompute_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(Gt_buf);
    cleanup();
    if (ce != cudaSuccess) st = fail(SE_ERR_CUDA, std::string("precompute: ") + cudaGetErrorString(ce));
    if (p->prec == SE_FP64 && st == SE_OK)
        p->ghat = p->ghat64;
    return st;
}

// ---------------------------------------------------------------- cache
// The precomputed octant depends only on the Green's function (harmonic or
// biharmonic), Mg, Mt and h per dimension (R is their diagonal): not on xi, P
// or the points.
// Plans with the same grid reuse it from a host-side cache, and optionally
// from files in a directory (one file per key, written after computing).
struct CacheEntry {
    std::vector<double> oct;
    uint64_t stamp = 0;
};
std::mutex g_cache_mu;
std::map<std::string, CacheEntry> g_cache;
bool g_cache_on = true;
std::string g_cache_dir;
uint64_t g_stamp = 0;
constexpr size_t CACHE_MAX_BYTES = size_t(2) << 30;  // evict the oldest entries beyond 2 GB

std::string cache_key(const se_plan_s *p) {
    uint64_t hb;
    memcpy(&hb, &p->h, sizeof(hb));
    char buf[160];
    snprintf(buf, sizeof(buf), "%s_Mg%dx%dx%d_Mt%dx%dx%d_h%016llx", p->kernel == SE_ROTLET ? "H" : "B", p->mg[0],
             p->mg[1], p->mg[2], p->mt[0], p->mt[1], p->mt[2], (unsigned long long)hb);
    return buf;
}

constexpr uint64_t FILE_MAGIC = 0x5345474841543031ull;  // file format tag

bool read_file(const std::string &path, size_t n, std::vector<double> &out) {
    FILE *fp = fopen(path.c_str(), "rb");
    if (!fp) return false;
    uint64_t hdr[2] = {0, 0};
    bool ok = fread(hdr, sizeof(uint64_t), 2, fp) == 2 && hdr[0] == FILE_MAGIC && hdr[1] == n;
    if (ok) {
        out.resize(n);
        ok = fread(out.data(), sizeof(double), n, fp) == n;
    }
    fclose(fp);
    return ok;
}

void write_file(const std::string &path, const std::vector<double> &v) {
    const std::string tmp = path + ".tmp";
    FILE *fp = fopen(tmp.c_str(), "wb");
    if (!fp) return;
    const uint64_t hdr[2] = {FILE_MAGIC, (uint64_t)v.size()};
    bool ok = fwrite(hdr, sizeof(uint64_t), 2, fp) == 2 && fwrite(v.data(), sizeof(double), v.size(), fp) == v.size();
    ok = (fclose(fp) == 0) && ok;
    if (ok) rename(tmp.c_str(), path.c_str());
    else remove(tmp.c_str());
}

// upload a cached octant into the plan (and its FP32 copy)
se_status_t upload(se_plan_s *p, const std::vector<double> &oct) {
    const size_t n = oct.size();
    if (cudaMemcpy(p->ghat64, oct.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(SE_ERR_CUDA, "precompute: cache upload failed");
    if (p->prec == SE_FP32) {
        std::vector<float> o32(n);
        for (size_t i = 0; i < n; i++) o32[i] = (float)oct[i];
        if (cudaMemcpy(p->ghat, o32.data(), n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(SE_ERR_CUDA, "precompute: cache upload failed");
    } else {
        p->ghat = p->ghat64;
    }
    return SE_OK;
}

}  // namespace

se_status_t precompute(se_plan_s *p) {
    const size_t n = (size_t)(p->mt[0] + 1) * (p->mt[1] + 1) * (p->mt[2] + 1);
    const auto t0 = std::chrono::steady_clock::now();
    const std::string key = cache_key(p);
    std::vector<double> oct;
    bool hit = false;
    std::string dir;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        dir = g_cache_dir;
        if (g_cache_on) {
            auto it = g_cache.find(key);
            if (it != g_cache.end() && it->second.oct.size() == n) {
                oct = it->second.oct;
                it->second.stamp = ++g_stamp;
                hit = true;
            }
        }
    }
    if (!hit && !dir.empty()) hit = read_file(dir + "/se_ghat_" + key + ".bin", n, oct);
    se_status_t st;
    if (hit) {
        st = upload(p, oct);
        p->precompute_cached = true;
    } else {
        st = precompute_compute(p);
        if (st != SE_OK) return st;
        p->precompute_cached = false;
        if (g_cache_on || !dir.empty()) {
            oct.resize(n);
            if (cudaMemcpy(oct.data(), p->ghat64, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(SE_ERR_CUDA, "precompute: cache download failed");
            if (!dir.empty()) write_file(dir + "/se_ghat_" + key + ".bin", oct);
        }
    }
    if (st == SE_OK && g_cache_on && !oct.empty()) {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        CacheEntry &e = g_cache[key];
        if (e.oct.size() != n) e.oct = oct;
        e.stamp = ++g_stamp;
        size_t total = 0;
        for (auto &kv : g_cache) total += kv.second.oct.size() * sizeof(double);
        while (total > CACHE_MAX_BYTES && g_cache.size() > 1) {
            auto oldest = g_cache.begin();
            for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
                if (it->second.stamp < oldest->second.stamp) oldest = it;
            total -= oldest->second.oct.size() * sizeof(double);
            g_cache.erase(oldest);
        }
    }
    if (hit)
        p->precompute_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

void set_precompute_cache(bool memory, const char *dir) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache_on = memory;
    if (!memory) g_cache.clear();
    g_cache_dir = dir ? dir : "";
}

}  // namespace se

using namespace se;

extern "C" se_status_t se_set_precompute_cache(int memory, const char *dir) {
    set_precompute_cache(memory != 0, dir);
    return SE_OK;
}

extern "C" se_status_t se_plan_precompute_info(se_plan_t p, double *ms, int *cached) {
    if (!p) return fail(SE_ERR_INVALID_ARG, "NULL plan");
    if (ms) *ms = p->precompute_ms;
    if (cached) *cached = p->precompute_cached ? 1 : 0;
    return SE_OK;
}
