// Stable bin order for deterministic evaluations.  The counting sort of the
// binning (Section 6 cell list, Section 5.2 spreading tiles) takes each
// point's slot inside its bin from an atomic counter, so the order of points
// within a bin changes from run to run, and with it the order of the FP32
// sums over a bin's points.  Here the slots are recomputed as the rank of the
// point among the points of its bin with smaller indices: a least-significant
// digit radix sort of the bin keys, 8 bits a pass, each pass a stable counting
// sort (per-block digit counts, one exclusive scan over the digit-major
// table, then a scatter that ranks equal digits by index within the block).
#include "se_internal.cuh"

namespace se {

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int RS_BINS = 256;          // digit values (8 bits)
constexpr int RS_NT = 256;            // threads per block
constexpr int RS_NW = RS_NT / 32;     // warps per block
constexpr int RS_PER = 16;            // elements per thread
constexpr int RS_BLK = RS_NT * RS_PER;  // elements per block

// hist[d * nblk + b] = elements of block b (elements b RS_BLK .. + RS_BLK)
// whose digit is d
__global__ void __launch_bounds__(RS_NT) k_rs_hist(int N, const int *__restrict__ keys, int shift, int nblk,
                                                   int *__restrict__ hist) {
    __shared__ int h[RS_BINS];
    const int tid = threadIdx.x, b = blockIdx.x;
    h[tid] = 0;
    __syncthreads();
    for (int r = 0; r < RS_PER; r++) {
        const int e = b * RS_BLK + r * RS_NT + tid;
        if (e < N) atomicAdd(&h[(keys[e] >> shift) & (RS_BINS - 1)], 1);
    }
    __syncthreads();
    hist[tid * nblk + b] = h[tid];
}

// Stable scatter by digit: element e goes to the start of its digit in this
// block (the scanned table) plus the number of elements of the block with the
// same digit and a smaller index.  The block walks its elements in index
// order, RS_NT at a time: within a warp the rank comes from the lanes with the
// same digit below, across warps from the per-warp counts of the digit.
// vin == nullptr: the values are the element indices.
__global__ void __launch_bounds__(RS_NT) k_rs_scatter(int N, const int *__restrict__ kin, const int *__restrict__ vin,
                                                      int shift, int nblk, const int *__restrict__ hist_scan,
                                                      int *__restrict__ kout, int *__restrict__ vout) {
    __shared__ int run[RS_BINS];
    __shared__ int wc[RS_NW][RS_BINS];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, b = blockIdx.x;
    run[tid] = hist_scan[tid * nblk + b];
    for (int r = 0; r < RS_PER; r++) {
        for (int i = tid; i < RS_NW * RS_BINS; i += RS_NT) (&wc[0][0])[i] = 0;
        __syncthreads();
        const int e = b * RS_BLK + r * RS_NT + tid;
        const bool valid = e < N;
        const int k = valid ? kin[e] : 0;
        const int d = valid ? (k >> shift) & (RS_BINS - 1) : -1;
        const unsigned same = __match_any_sync(FULLM, d);
        const int within = __popc(same & ((1u << lane) - 1u));
        if (valid && within == 0) wc[w][d] = __popc(same);
        __syncthreads();
        if (valid) {
            int pos = run[d] + within;
            for (int v = 0; v < w; v++) pos += wc[v][d];
            kout[pos] = k;
            vout[pos] = vin ? vin[e] : e;
        }
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int v = 0; v < RS_NW; v++) tot += wc[v][tid];
        run[tid] += tot;
        __syncthreads();
    }
}

// slot[i] = position of point i in the key-sorted order minus its bin's start
__global__ void k_rs_slots(int N, const int *__restrict__ skeys, const int *__restrict__ svals,
                           const int *__restrict__ start, int *__restrict__ slot) {
    const int pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= N) return;
    slot[svals[pos]] = pos - start[skeys[pos]];
}

int rs_blocks(int64_t n) { return (int)((n + RS_BLK - 1) / RS_BLK); }

}  // namespace

size_t stable_scratch_ints(int64_t n) {
    const size_t h = (size_t)RS_BINS * rs_blocks(n);
    return 4 * (size_t)n + h + 2 + (h + 4095) / 4096 + 1;
}

cudaError_t launch_stable_slots(int N, const int *keys, int nkeys, const int *start, int *slot, int *scratch,
                                cudaStream_t st, int64_t *launches) {
    if (N <= 0) return cudaSuccess;
    int bits = 1;
    while (bits < 31 && (1 << bits) < nkeys) bits++;
    const int passes = (bits + 7) / 8;
    const int nblk = rs_blocks(N);
    int *kA = scratch, *vA = scratch + N, *kB = scratch + 2 * (size_t)N, *vB = scratch + 3 * (size_t)N;
    int *hist = scratch + 4 * (size_t)N;
    const int *kin = keys, *vin = nullptr;
    for (int ps = 0; ps < passes; ps++) {
        int *ko = (ps & 1) ? kB : kA, *vo = (ps & 1) ? vB : vA;
        k_rs_hist<<<nblk, RS_NT, 0, st>>>(N, kin, 8 * ps, nblk, hist);
        cudaError_t e = launch_scan(hist, RS_BINS * nblk, st);
        if (e) return e;
        k_rs_scatter<<<nblk, RS_NT, 0, st>>>(N, kin, vin, 8 * ps, nblk, hist, ko, vo);
        *launches += 2 + scan_launch_count(RS_BINS * nblk);
        kin = ko;
        vin = vo;
    }
    k_rs_slots<<<(N + 255) / 256, 256, 0, st>>>(N, kin, vin, start, slot);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace se
