// se_real_space_noalloc: the screened real-space sum (the same computation as
// se_eval_real_space) for callers that cannot allocate device memory.
//
// Who needs it: code that may not call the device allocator -- a host
// application whose memory arena owns all device memory and forbids outside
// allocations, a plugin that is handed device buffers by its host program, or
// a real-time loop that must never enter cudaMalloc.  Those callers pass their
// inputs and outputs; every temporary (sorted copies of the points, the cell
// list, the cluster list) lives in one file-scope __device__ array of fixed
// size, and the call makes no cudaMalloc, cudaFree or allocating library call.
//
// The first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current; make that first call before
// any stream capture.  Later calls on a stream that is not capturing look the
// address up again (a cheap lookup once the module is loaded), so that a
// context torn down and created again (cudaDeviceReset), which may place the
// array elsewhere, is followed; calls on a capturing stream use the address
// found last.  All calls share the one array: calls whose work
// overlaps on the GPU (different streams, or several host threads) race and
// corrupt each other's results; serialise them.
//
// Limits (checked, SE_ERR_INVALID_ARG beyond them): N <= NOALLOC_MAX_N points,
// and at most NOALLOC_MAX_ROWS rows / NOALLOC_MAX_CELLS cells in the cell list
// (the cell width across rows is rc/5, so L / rc must stay below about 25).
// The array costs NOALLOC_BYTES (about 9 MB) of device memory on every GPU that
// loads the library, for as long as the process lives.
#include <mutex>

#include "se_internal.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_N = 32768;
constexpr int64_t NOALLOC_MAX_ROWS = 128 * 128;
constexpr int64_t NOALLOC_MAX_CELLS = 1 << 18;

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t scan_ints(size_t n) { return n + 2 + (n + 4095) / 4096 + 1; }
// worst case (FP64): six 32-byte point arrays, eight int arrays of N, the two
// scanned count arrays, the cluster list and the status word
constexpr size_t OFF_V4 = 0;
constexpr size_t SZ_V4 = align256(32 * NOALLOC_MAX_N);
constexpr size_t OFF_INT = OFF_V4 + 6 * SZ_V4;
constexpr size_t SZ_INT = align256(4 * NOALLOC_MAX_N);
constexpr size_t OFF_CNT_T = OFF_INT + 8 * SZ_INT;
constexpr size_t SZ_CNT_T = align256(4 * scan_ints(1));
constexpr size_t OFF_CNT_R = OFF_CNT_T + SZ_CNT_T;
constexpr size_t SZ_CNT_R = align256(4 * scan_ints(NOALLOC_MAX_CELLS));
constexpr size_t OFF_NCL = OFF_CNT_R + SZ_CNT_R;
constexpr size_t SZ_NCL = align256(4 * scan_ints(NOALLOC_MAX_ROWS));
constexpr size_t OFF_CL = OFF_NCL + SZ_NCL;
constexpr size_t SZ_CL = align256(8 * (NOALLOC_MAX_N / 4 + NOALLOC_MAX_ROWS + 1));
constexpr size_t OFF_STATUS = OFF_CL + SZ_CL;
constexpr size_t NOALLOC_BYTES = OFF_STATUS + 256;

// The scratch.  In host code this name is only a stand-in for the device
// object: its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

std::mutex g_mu;
void *g_addr[128] = {};  // device address of the scratch, per device ordinal

}  // namespace

using namespace se;

extern "C" se_status_t se_real_space_noalloc(se_kernel_t kernel, se_prec_t prec, int64_t N, const double box[4],
                                             double xi, double rc, const void *x, const void *f, const void *q,
                                             void *u, void *stream) {
    if (kernel < SE_STOKESLET || kernel > SE_ROTLET) return fail(SE_ERR_INVALID_ARG, "unknown kernel");
    if (prec != SE_FP32 && prec != SE_FP64) return fail(SE_ERR_INVALID_ARG, "unknown precision");
    if (N < 1 || N > NOALLOC_MAX_N)
        return fail(SE_ERR_INVALID_ARG, "se_real_space_noalloc: N must be in [1, " + std::to_string(NOALLOC_MAX_N) + "]");
    if (!box || !(box[3] > 0) || !(xi > 0) || !(rc > 0)) return fail(SE_ERR_INVALID_ARG, "invalid box, xi or rc");
    if (!x || !f || !u || (kernel == SE_STRESSLET && !q)) return fail(SE_ERR_INVALID_ARG, "NULL pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 128) return fail(SE_ERR_INVALID_ARG, "device ordinal out of range");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        // look the address up on the first call on this device (the device is
        // current) and again on every call outside a stream capture
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
            (void)cudaGetLastError();
            cs = cudaStreamCaptureStatusActive;  // unknown: keep the address found last
        }
        if (!g_addr[dev] || cs == cudaStreamCaptureStatusNone) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess)
                return fail(SE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_addr[dev] = ptr;
        }
        base = (unsigned char *)g_addr[dev];
    }
    // a plan on the stack: geometry of the cell list only, buffers in the scratch
    se_plan_s p;
    p.erfc_table_off = true;
    p.kernel = kernel;
    p.prec = prec;
    p.N = N;
    for (int d = 0; d < 3; d++) p.x0[d] = box[d];
    for (int d = 0; d < 3; d++) p.len[d] = box[3];
    p.xi = xi;
    p.rc = rc;
    p.P = 2;
    for (int d = 0; d < 3; d++) {
        p.mt[d] = 2;
        p.mf[d] = 4;
    }
    const double L = box[3];
    int ncd = std::max(1, std::min((int)floor(5.0 * L / rc), 200));
    int ncdx = std::max(1, std::min((int)floor(16.0 * L / rc), 1000));
    if ((int64_t)ncd * ncd > NOALLOC_MAX_ROWS)
        return fail(SE_ERR_INVALID_ARG, "se_real_space_noalloc: rc too small for the fixed cell-list size (L/rc <= 25)");
    while ((int64_t)ncd * ncd * ncdx > NOALLOC_MAX_CELLS && ncdx > 1) ncdx--;
    if ((int64_t)ncd * ncd * ncdx > NOALLOC_MAX_CELLS)
        return fail(SE_ERR_INVALID_ARG, "se_real_space_noalloc: cell list exceeds the fixed size");
    const int ncel[3] = {ncdx, ncd, ncd};
    Geom &g = p.geom;
    for (int d = 0; d < 3; d++) {
        g.x0[d] = box[d];
        g.len[d] = L;
        g.mt[d] = 2;
        g.mf[d] = 4;
        g.nt[d] = 1;
        g.ncel[d] = ncel[d];
        g.cw[d] = L / ncel[d];
        g.icw[d] = ncel[d] / L;
    }
    g.h = L;
    g.inv_h = 1.0 / L;
    g.P = 2;
    g.T = 8;
    g.rc = rc;
    g.xi = xi;
    p.ntiles = 1;
    p.ncells = ncd * ncd * ncdx;
    auto fill = [&](auto &G) {
        using TT = std::remove_reference_t<decltype(G.inv_h)>;
        for (int d = 0; d < 3; d++) {
            G.x0[d] = (TT)box[d];
            G.len[d] = (TT)L;
            G.icw[d] = (TT)g.icw[d];
            G.ilen[d] = (TT)(1.0 / L);
            G.cw[d] = (TT)g.cw[d];
            G.mt[d] = 2;
            G.mf[d] = 4;
            G.nt[d] = 1;
            G.ncel[d] = ncel[d];
        }
        G.inv_h = (TT)(1.0 / L);
        G.half_ext = (TT)0;
        G.ah2 = (TT)0;
        G.P = 2;
        G.T_ = 8;
    };
    fill(p.gpf);
    fill(p.gpd);
    p.b.xs_t = base + OFF_V4 + 0 * SZ_V4;
    p.b.fs_t = base + OFF_V4 + 1 * SZ_V4;
    p.b.qs_t = base + OFF_V4 + 2 * SZ_V4;
    p.b.xs_r = base + OFF_V4 + 3 * SZ_V4;
    p.b.fs_r = base + OFF_V4 + 4 * SZ_V4;
    p.b.qs_r = base + OFF_V4 + 5 * SZ_V4;
    int *ints[8];
    for (int k = 0; k < 8; k++) ints[k] = (int *)(base + OFF_INT + k * SZ_INT);
    p.b.perm_t = ints[0];
    p.b.slot_t = ints[1];
    p.b.key_t = ints[2];
    p.b.tag_t = ints[3];
    p.b.perm_r = ints[4];
    p.b.slot_r = ints[5];
    p.b.key_r = ints[6];
    p.b.tag_r = ints[7];
    p.b.cnt_t = (int *)(base + OFF_CNT_T);
    p.b.cnt_r = (int *)(base + OFF_CNT_R);
    p.b.ncl = (int *)(base + OFF_NCL);
    p.b.clusters = (int2 *)(base + OFF_CL);
    p.b.status = (int *)(base + OFF_STATUS);
    // the array keeps the previous call's contents: reset what must start at
    // zero (the counters are cleared inside the binning, the flags here)
    const size_t bytes = (size_t)N * 3 * (prec == SE_FP32 ? 4 : 8);
    if ((e = cudaMemsetAsync(p.b.status, 0, 16, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(u, 0, bytes, st)) != cudaSuccess)
        return fail(SE_ERR_CUDA, std::string("se_real_space_noalloc: ") + cudaGetErrorString(e));
    if (prec == SE_FP32) {
        if ((e = launch_bin<float>(&p, (const float *)x, (const float *)f, (const float *)q, st)) != cudaSuccess ||
            (e = launch_real<float>(&p, st, (float *)u)) != cudaSuccess)
            return fail(SE_ERR_CUDA, std::string("se_real_space_noalloc: ") + cudaGetErrorString(e));
    } else {
        if ((e = launch_bin<double>(&p, (const double *)x, (const double *)f, (const double *)q, st)) != cudaSuccess ||
            (e = launch_real<double>(&p, st, (double *)u)) != cudaSuccess)
            return fail(SE_ERR_CUDA, std::string("se_real_space_noalloc: ") + cudaGetErrorString(e));
    }
    return SE_OK;
}
