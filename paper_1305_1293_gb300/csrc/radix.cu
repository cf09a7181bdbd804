// Data organisation (Step 3 of Section 4.2, Algorithm 3): the windows a propagation
// step produced are gathered into a gap-free pool, here in the order of their edge key
// (instance key base + half-edge id) so that windows on one edge are adjacent for the
// per-edge trimming of Step 4 and the next propagation reads edge records in order.
//
// Hand-written stable LSD radix sort of (32-bit key, 32-bit index) pairs.  The element
// count lives in device memory, so every launch has a fixed grid (graph friendly): block
// b owns the contiguous chunk [b*C, (b+1)*C) with C = ceil(n / gridDim.x).  Per pass:
//   k_rs_hist    - per-block digit counts, stored digit-major
//   k_rs_scan    - one-block exclusive scan of the digit-major table
//   k_rs_scatter - stable scatter: warp ranks from __match_any_sync, warp offsets
//                  from a per-tile shared-memory table, running per-digit offsets.
#include "radix.cuh"

namespace pch {

__device__ __forceinline__ int rs_count(const int* n_ptr, int cap) {
    int n = *n_ptr;
    return n < cap ? n : cap;
}

// Keys of the child arena: invalid slots (he < 0) get ~0u and sort last.
__global__ void k_rs_keys(const int* __restrict__ he, const int* __restrict__ inst, const Inst* __restrict__ insts,
                          const int* n_ptr, int cap, unsigned* key, int* val) {
    int n = rs_count(n_ptr, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int h = he[i];
        key[i] = h < 0 ? ~0u : (unsigned)(insts[inst[i]].keybase + h);
        val[i] = i;
    }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const unsigned* __restrict__ key, const int* n_ptr, int cap,
                                                        int shift, int* hist) {
    __shared__ int h[kRsDigits];
    for (int d = threadIdx.x; d < kRsDigits; d += blockDim.x) h[d] = 0;
    __syncthreads();
    int n = rs_count(n_ptr, cap);
    int C = (n + gridDim.x - 1) / gridDim.x;
    int beg = blockIdx.x * C, end = min(n, beg + C);
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x) atomicAdd(&h[(key[i] >> shift) & (kRsDigits - 1)], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < kRsDigits; d += blockDim.x) hist[d * gridDim.x + blockIdx.x] = h[d];
}

// One block of kRsScanThreads threads scans `total` ints in place.
__global__ void __launch_bounds__(kRsScanThreads) k_rs_scan(int* hist, int total) {
    __shared__ int sh[kRsScanThreads];
    int per = (total + kRsScanThreads - 1) / kRsScanThreads;
    int beg = threadIdx.x * per, end = min(total, beg + per);
    int s = 0;
    for (int i = beg; i < end; ++i) s += hist[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < kRsScanThreads; off <<= 1) {
        int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int run = sh[threadIdx.x] - s;
    for (int i = beg; i < end; ++i) {
        int c = hist[i];
        hist[i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const unsigned* __restrict__ kin, const int* __restrict__ vin,
                                                           unsigned* __restrict__ kout, int* __restrict__ vout,
                                                           const int* n_ptr, int cap, int shift,
                                                           const int* __restrict__ hist) {
    constexpr int W = kRsThreads / 32;
    __shared__ int run[kRsDigits];
    __shared__ int wcnt[W][kRsDigits];
    __shared__ int tot[kRsDigits];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int n = rs_count(n_ptr, cap);
    int C = (n + gridDim.x - 1) / gridDim.x;
    int beg = blockIdx.x * C, end = min(n, beg + C);
    for (int d = threadIdx.x; d < kRsDigits; d += blockDim.x) run[d] = hist[d * gridDim.x + blockIdx.x];
    for (int tile = beg; tile < end; tile += kRsThreads) {
        for (int j = threadIdx.x; j < W * kRsDigits; j += kRsThreads) (&wcnt[0][0])[j] = 0;
        __syncthreads();
        int i = tile + threadIdx.x;
        bool valid = i < end;
        unsigned k = valid ? kin[i] : 0u;
        int v = valid ? vin[i] : 0;
        int digit = valid ? (int)((k >> shift) & (kRsDigits - 1)) : kRsDigits;   // kRsDigits = padding lane
        unsigned peers = __match_any_sync(0xffffffffu, digit);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        for (int d = threadIdx.x; d < kRsDigits; d += kRsThreads) {
            int s = 0;
            for (int w = 0; w < W; ++w) {
                int c = wcnt[w][d];
                wcnt[w][d] = s;
                s += c;
            }
            tot[d] = s;
        }
        __syncthreads();
        if (valid) {
            int pos = run[digit] + wcnt[warp][digit] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRsDigits; d += kRsThreads) run[d] += tot[d];
        __syncthreads();
    }
}

// Sort the child arena by edge key.  Leaves the sorted (key, index) pairs in
// key_buf[passes & 1] / val_buf[passes & 1]; returns that parity.
int launch_sort_children(const WinSoA& arena, const Inst* insts, const int* n_ptr, int cap, int key_bits,
                         unsigned* key_buf[2], int* val_buf[2], int* hist, int blocks, cudaStream_t s) {
    int passes = (key_bits + kRsDigitBits - 1) / kRsDigitBits;
    if (passes < 1) passes = 1;
    int grid0 = blocks * 2;
    k_rs_keys<<<grid0, 256, 0, s>>>(arena.he, arena.inst, insts, n_ptr, cap, key_buf[0], val_buf[0]);
    for (int p = 0; p < passes; ++p) {
        int shift = p * kRsDigitBits;
        k_rs_hist<<<blocks, kRsThreads, 0, s>>>(key_buf[p & 1], n_ptr, cap, shift, hist);
        k_rs_scan<<<1, kRsScanThreads, 0, s>>>(hist, kRsDigits * blocks);
        k_rs_scatter<<<blocks, kRsThreads, 0, s>>>(key_buf[p & 1], val_buf[p & 1], key_buf[(p + 1) & 1],
                                                   val_buf[(p + 1) & 1], n_ptr, cap, shift, hist);
    }
    return passes & 1;
}

}  // namespace pch
