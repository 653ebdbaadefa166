// Steps 2-4 of Section 5.2 along z, fused (FP32 plans with the
// zero-padding-aware transforms): after the 2-D (y, x) transforms of the
// Mtilde nonzero z-planes, each (ky, kx) column of every source component is
// transformed along z (its upper Mf - Mtilde values are zero, and are not
// read), multiplied by the scaling of eq. gridfcnsc (multiplier.cuh), and
// transformed back; only the Mtilde z-planes the inverse 2-D transforms read
// are written.  One pass over the spectrum instead of the forward z-pass, the
// zeroing of the upper planes, the scaling and the inverse z-pass.
//
// The transforms along z are mixed-radix Stockham transforms (radices 4, 2, 3,
// 5, 7; the FFT lengths of the FP32 plans factor into these) in shared memory:
// a CTA takes CB consecutive kx columns of one ky row, for all components,
// and runs the passes with the twiddles of a table computed in FP64 on the
// host.  The inverse transform is the forward one of the complex conjugate
// (conjugated once more on the way out), unnormalised like cuFFT's (the
// multiplier's constant carries 1/Mf^3).
#include <cmath>
#include <vector>

#include "multiplier.cuh"

namespace se {

namespace {

constexpr int ZF_NT = 256;
constexpr int ZF_LB = 8;  // global loads in flight per thread
// SE_ZF_SMEM_KB: the CTA's shared memory budget (columns per CTA follow from it)
#ifndef SE_ZF_SMEM_KB
#define SE_ZF_SMEM_KB 100
#endif
constexpr size_t ZF_SMEM = SE_ZF_SMEM_KB * 1024;

struct ZRadices {
    int n = 0, np = 0;
    int r[ZF_MAXPASS];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 conj2(float2 a) { return make_float2(a.x, -a.y); }

// cos and sin of 2 pi m / R, m = 1 .. (R - 1) / 2, for the odd radices
__device__ __constant__ const float ZC5[2] = {3.090169944e-01f, -8.090169944e-01f};
__device__ __constant__ const float ZS5[2] = {9.510565163e-01f, 5.877852523e-01f};
__device__ __constant__ const float ZC7[3] = {6.234898019e-01f, -2.225209340e-01f, -9.009688679e-01f};
__device__ __constant__ const float ZS7[3] = {7.818314825e-01f, 9.749279122e-01f, 4.338837391e-01f};

// In-place DFT of size R: X_k = sum_q v_q e^{-2 pi i q k / R}.  Odd R from the
// pairs a_q = v_q + v_{R-q}, d_q = v_q - v_{R-q}:
//   X_k, X_{R-k} = v_0 + sum_q [a_q cos(2 pi q k / R) -+ i d_q sin(2 pi q k / R)].
template <int R>
__device__ __forceinline__ void zdft(float2 (&v)[R]) {
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
        // -i (x + i y) = y - i x
        const float2 md13 = make_float2(d13.y, -d13.x);
        v[0] = cadd(s02, s13);
        v[1] = cadd(d02, md13);
        v[2] = csub(s02, s13);
        v[3] = csub(d02, md13);
    } else {
        constexpr int H = (R - 1) / 2;
        const float *CS = (R == 3) ? nullptr : (R == 5 ? ZC5 : ZC7);
        const float *SN = (R == 3) ? nullptr : (R == 5 ? ZS5 : ZS7);
        float2 a[H], d[H];
#pragma unroll
        for (int q = 1; q <= H; q++) {
            a[q - 1] = cadd(v[q], v[R - q]);
            d[q - 1] = csub(v[q], v[R - q]);
        }
        float2 X[R];
        X[0] = v[0];
#pragma unroll
        for (int q = 0; q < H; q++) X[0] = cadd(X[0], a[q]);
#pragma unroll
        for (int k = 1; k <= H; k++) {
            float2 re = v[0], im = make_float2(0.0f, 0.0f);  // im: sum d_q sin(2 pi q k / R)
#pragma unroll
            for (int q = 1; q <= H; q++) {
                const int m = (q * k) % R, mm = m <= H ? m : R - m;  // cos(2 pi m / R) = cos(2 pi (R - m) / R)
                const float sg = m <= H ? 1.0f : -1.0f;             // sin(2 pi (R - m) / R) = -sin(2 pi m / R)
                const float c = (R == 3) ? -0.5f : CS[mm - 1];
                const float sn = sg * ((R == 3) ? 8.660254038e-01f : SN[mm - 1]);
                re.x = fmaf(a[q - 1].x, c, re.x);
                re.y = fmaf(a[q - 1].y, c, re.y);
                im.x = fmaf(d[q - 1].x, sn, im.x);
                im.y = fmaf(d[q - 1].y, sn, im.y);
            }
            // -i im = (im.y, -im.x)
            X[k] = make_float2(re.x + im.y, re.y - im.x);
            X[R - k] = make_float2(re.x - im.y, re.y + im.x);
        }
#pragma unroll
        for (int k = 0; k < R; k++) v[k] = X[k];
    }
}

// One Stockham pass of radix R over nsig signals of length n (A -> B), Ns
// the product of the earlier passes' radices: butterfly j of a signal reads
// A[j + q n/R], applies the twiddles e^{-2 pi i q (j mod Ns) / (Ns R)} and the
// size-R DFT, and writes B[(j / Ns) Ns R + j mod Ns + q Ns].
template <int R>
__device__ __forceinline__ void zpass(const float2 *A, float2 *B, int n, int Ns, int nsig, const float2 *W) {
    // thread -> butterfly j (fixed for the pass) of signals s0, s0 + sstep, ...
    const int m = n / R, t = n / (Ns * R);
    const int sstep = ZF_NT / m;
    const int s0 = threadIdx.x / m, j = threadIdx.x - s0 * m;
    if (s0 >= sstep) return;  // m does not divide ZF_NT: the last threads idle
    const int k = j % Ns, d = (j / Ns) * Ns * R + k;
    float2 tw[R];
#pragma unroll
    for (int q = 1; q < R; q++) tw[q] = W[q * k * t];
    for (int s = s0; s < nsig; s += sstep) {
        const float2 *a = A + (size_t)s * n + j;
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; q++) v[q] = a[q * m];
        if (Ns > 1) {
#pragma unroll
            for (int q = 1; q < R; q++) v[q] = cmul(v[q], tw[q]);
        }
        zdft<R>(v);
        float2 *o = B + (size_t)s * n + d;
#pragma unroll
        for (int q = 0; q < R; q++) o[q * Ns] = v[q];
    }
}

// The forward transform of nsig signals starting in A (B: scratch of the same
// size); returns the buffer holding the result.
__device__ float2 *zfft(float2 *A, float2 *B, int nsig, const ZRadices &zr, const float2 *W) {
    int Ns = 1;
    for (int p = 0; p < zr.np; p++) {
        const int R = zr.r[p];
        switch (R) {
            case 2: zpass<2>(A, B, zr.n, Ns, nsig, W); break;
            case 3: zpass<3>(A, B, zr.n, Ns, nsig, W); break;
            case 4: zpass<4>(A, B, zr.n, Ns, nsig, W); break;
            case 5: zpass<5>(A, B, zr.n, Ns, nsig, W); break;
            default: zpass<7>(A, B, zr.n, Ns, nsig, W); break;
        }
        __syncthreads();
        float2 *t = A;
        A = B;
        B = t;
        Ns *= R;
    }
    return A;
}

__host__ __device__ bool factor(int n, ZRadices &zr);

// The columns kx = kx0 .. kx0 + cb - 1 of row ky: element (c, kz, ky, kx) of
// the spectra at base + c scs + kz szs + ky nxh + kx (kx < nxh), whose
// z-planes below nz hold the 2-D transforms of the nc source components;
// afterwards the planes below nz of the three output components hold the
// inverse z-transforms of the scaled values.  zsm: n + 2 nc cb n float2 of
// shared memory.
template <int KERNEL>
__device__ __forceinline__ void zscale_body(const ScaleConst &sc, const float *__restrict__ ghat, float2 *base,
                                            size_t scs, size_t szs, int nz, int nc, int cb, const ZRadices &zr,
                                            const float2 *__restrict__ Wg, int ky, int kx0, float2 *zsm) {
    const int n = zr.n, tid = threadIdx.x, nxh = sc.nxh;
    float2 *W = zsm, *A = zsm + n, *B = A + (size_t)nc * cb * n;
    for (int t = tid; t < n; t += ZF_NT) W[t] = Wg[t];
    // the columns' nonzero planes, zeros above (x fastest in global memory):
    // thread -> column col, planes z0, z0 + zstep, ...; ZF_LB loads in flight
    const int zstep = ZF_NT / cb, col = tid % cb, z0 = tid / cb, kx = kx0 + col;
    const bool colok = z0 < zstep && kx < nxh;
    for (int c = 0; c < nc; c++) {
        const float2 *src = base + (size_t)c * scs + (size_t)ky * nxh + kx;
        float2 *dst = A + ((size_t)c * cb + col) * n;
        for (int zb = z0; zb < n && z0 < zstep; zb += ZF_LB * zstep) {
            float2 v[ZF_LB];
#pragma unroll
            for (int u = 0; u < ZF_LB; u++) {
                const int z = zb + u * zstep;
                v[u] = (colok && z < nz) ? src[(size_t)z * szs] : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int u = 0; u < ZF_LB; u++) {
                const int z = zb + u * zstep;
                if (z < n) dst[z] = v[u];
            }
        }
    }
    __syncthreads();
    float2 *F = zfft(A, B, nc * cb, zr, W);
    float2 *S = (F == A) ? B : A;
    // the multiplier at every kz of the columns; the conjugate of the result
    // (the inverse transform as a forward one)
    for (int i0 = tid; i0 < cb * n; i0 += ZF_LB * ZF_NT) {
        float G[ZF_LB];
#pragma unroll
        for (int u = 0; u < ZF_LB; u++) {
            const int i = i0 + u * ZF_NT, cl = i / n, kz = i - cl * n, kxx = kx0 + cl;
            float kv[3];
            G[u] = (i < cb * n && kxx < nxh) ? ghat[kpoint3<float>(sc, kxx, ky, kz, kv)] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < ZF_LB; u++) {
            const int i = i0 + u * ZF_NT, cl = i / n, kz = i - cl * n, kxx = kx0 + cl;
            if (i >= cb * n || kxx >= nxh) continue;
            float kv[3];
            kpoint3<float>(sc, kxx, ky, kz, kv);
            float2 g[6], o[3];
            for (int c = 0; c < nc; c++) g[c] = F[((size_t)c * cb + cl) * n + kz];
            apply_multiplier<float, KERNEL>(sc, kv, G[u], g, o);
#pragma unroll
            for (int j = 0; j < 3; j++) F[((size_t)j * cb + cl) * n + kz] = conj2(o[j]);
        }
    }
    __syncthreads();
    float2 *R = zfft(F, S, 3 * cb, zr, W);
    if (colok) {
        for (int j = 0; j < 3; j++) {
            float2 *dst = base + (size_t)j * scs + (size_t)ky * nxh + kx;
            const float2 *src = R + ((size_t)j * cb + col) * n;
            for (int z = z0; z < nz; z += zstep) dst[(size_t)z * szs] = conj2(src[z]);
        }
    }
}

// One plan: block (bx, ky) takes the columns bx cb .. of row ky of the nc
// spectra of nk points at spec ([kz][ky][kx]).
template <int KERNEL>
__global__ void __launch_bounds__(ZF_NT) k_zscale(ScaleConst sc, const float *__restrict__ ghat, float2 *spec,
                                                  size_t nk, int nz, int nc, int cb, ZRadices zr,
                                                  const float2 *__restrict__ Wg) {
    extern __shared__ __align__(16) float2 zsm[];
    zscale_body<KERNEL>(sc, ghat, spec, nk, (size_t)sc.mf[1] * sc.nxh, nz, nc, cb, zr, Wg, blockIdx.y,
                        blockIdx.x * cb, zsm);
}

__host__ __device__ bool factor(int n, ZRadices &zr) {
    zr.n = n;
    zr.np = 0;
    int m = n;
    const int fs[5] = {4, 2, 3, 5, 7};
    for (int i = 0; i < 5; i++)
        for (const int f = fs[i]; m % f == 0;) {
            if (zr.np == ZF_MAXPASS) return false;
            zr.r[zr.np++] = f;
            m /= f;
        }
    return m == 1;
}

int columns_per_cta(int n, int nc) {
    const size_t per = 2 * (size_t)nc * n * sizeof(float2);
    const size_t room = ZF_SMEM - (size_t)n * sizeof(float2);
    return (int)std::max<size_t>(1, std::min<size_t>(16, room / per));
}

}  // namespace

bool zfuse_supported(int n, int nc) {
    // every pass's butterflies of a signal fit the CTA's threads (n / R <= ZF_NT)
    ZRadices zr;
    return n >= 2 && n <= 2 * ZF_NT && factor(n, zr) && (size_t)n * sizeof(float2) * (1 + 2 * (size_t)nc) <= ZF_SMEM;
}

static void zfuse_table(int n, float2 *w) {
    for (int t = 0; t < n; t++) {
        const double a = -2.0 * M_PI * (double)t / (double)n;
        w[t] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
}

cudaError_t zfuse_twiddles(int n, void **out) {
    std::vector<float2> w(n);
    zfuse_table(n, w.data());
    cudaError_t e = cudaMalloc(out, n * sizeof(float2));
    if (e) return e;
    return cudaMemcpy(*out, w.data(), n * sizeof(float2), cudaMemcpyHostToDevice);
}

cudaError_t launch_zscale(const se_plan_s *p, cudaStream_t st, void *spec, int nc) {
    const ScaleConst sc = make_scale_const(p);
    ZRadices zr;
    if (!p->zw || !zfuse_supported(p->mf[2], nc) || !factor(p->mf[2], zr)) return cudaErrorInvalidValue;
    const int n = p->mf[2], cb = columns_per_cta(n, nc);
    const size_t smem = ((size_t)n + 2 * (size_t)nc * cb * n) * sizeof(float2);
    const size_t nk = (size_t)p->mf[2] * p->mf[1] * sc.nxh;
    const dim3 grid((unsigned)((sc.nxh + cb - 1) / cb), (unsigned)p->mf[1]);
    const float *gh = (const float *)p->ghat;
    float2 *sp = (float2 *)spec;
    const float2 *W = (const float2 *)p->zw;
    cudaError_t e;
    if (p->kernel == SE_STOKESLET) {
        if ((e = cudaFuncSetAttribute(k_zscale<SE_STOKESLET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        k_zscale<SE_STOKESLET><<<grid, ZF_NT, smem, st>>>(sc, gh, sp, nk, p->mt[2], nc, cb, zr, W);
    } else if (p->kernel == SE_STRESSLET) {
        if ((e = cudaFuncSetAttribute(k_zscale<SE_STRESSLET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        k_zscale<SE_STRESSLET><<<grid, ZF_NT, smem, st>>>(sc, gh, sp, nk, p->mt[2], nc, cb, zr, W);
    } else {
        if ((e = cudaFuncSetAttribute(k_zscale<SE_ROTLET>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        k_zscale<SE_ROTLET><<<grid, ZF_NT, smem, st>>>(sc, gh, sp, nk, p->mt[2], nc, cb, zr, W);
    }
    return cudaGetLastError();
}

}  // namespace se
