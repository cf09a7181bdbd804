// Data organisation (Step 3 of Section 4.2, Algorithm 3): the windows a propagation
// step produced are gathered into a gap-free pool, grouped by instance (so that the
// append and the selection see one instance per warp), or on request in the order of
// their edge key (instance key base + half-edge id) so that windows on one edge are
// adjacent for the per-edge trimming of Step 4.  A single instance needs no sort.
//
// Hand-written stable LSD radix sort of (32-bit key, 32-bit index) pairs, 8-bit digits.
// The element count n lives in device memory, so every launch has a fixed grid (graph
// friendly); block b owns the contiguous chunk [b*C, (b+1)*C), C = max(kRsChunkMin,
// ceil(n / gridDim.x)), and blocks past the data do nothing.  Per pass, two kernels:
//   k_rs_hist    - digit counts of the block's chunk, one row of 256 per block
//   k_rs_scatter - the block sums the rows before its own (its offset within each digit)
//                  and all rows (digit totals, then their exclusive scan), then scatters
//                  its chunk stably: ranks within a warp from __match_any_sync, warp
//                  offsets from a per-tile shared table, running per-digit offsets.
// Pass 0 reads the keys straight from the child arena (invalid slots sort last).
#include "radix.cuh"

namespace pch {

__device__ __forceinline__ int rs_count(const int* n_ptr, int cap) {
    int n = *n_ptr;
    return n < cap ? n : cap;
}

struct RsChunk {
    int beg, end;
};
__device__ __forceinline__ RsChunk rs_chunk(int n, int b) {
    int C = (n + gridDim.x - 1) / gridDim.x;
    C = C < kRsChunkMin ? kRsChunkMin : C;
    int beg = b * C;
    return {beg < n ? beg : n, min(n, beg + C)};
}

__device__ __forceinline__ int rs_active(int n) {
    int C = (n + gridDim.x - 1) / gridDim.x;
    C = C < kRsChunkMin ? kRsChunkMin : C;
    return (n + C - 1) / C;
}

// Key of arena slot i (pass 0) or the stored key.
__device__ __forceinline__ unsigned rs_key(const RsIn& in, int i) {
    if (in.keys) return in.keys[i];
    int h = in.he[i];
    if (h < 0) return ~0u;
    return in.by_edge ? (unsigned)(in.insts[in.inst[i]].keybase + h) : (unsigned)in.inst[i];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(RsIn in, const int* n_ptr, int cap, int shift, int* hist) {
    __shared__ int h[kRsDigits];
    const int n = rs_count(n_ptr, cap);
    const RsChunk c = rs_chunk(n, blockIdx.x);
    if (c.beg >= c.end) return;
    for (int d = threadIdx.x; d < kRsDigits; d += blockDim.x) h[d] = 0;
    __syncthreads();
    for (int i = c.beg + threadIdx.x; i < c.end; i += blockDim.x) atomicAdd(&h[(rs_key(in, i) >> shift) & (kRsDigits - 1)], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < kRsDigits; d += blockDim.x) hist[blockIdx.x * kRsDigits + d] = h[d];
}

__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(RsIn in, unsigned* __restrict__ kout, int* __restrict__ vout,
                                                           const int* n_ptr, int cap, int shift,
                                                           const int* __restrict__ hist) {
    constexpr int W = kRsThreads / 32;
    static_assert(kRsThreads == kRsDigits, "one thread per digit");
    __shared__ int run[kRsDigits];
    __shared__ int wcnt[W][kRsDigits];
    __shared__ int tot[kRsDigits];
    __shared__ int wsum[W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int n = rs_count(n_ptr, cap);
    const RsChunk c = rs_chunk(n, blockIdx.x);
    if (c.beg >= c.end) return;
    const int active = rs_active(n);
    // this block's offset inside every digit, and the digit totals
    {
        const int d = threadIdx.x;
        int before = 0, total = 0;
        int b = 0;
#pragma unroll 8
        for (b = 0; b < active; ++b) {
            int x = hist[b * kRsDigits + d];
            before += b < (int)blockIdx.x ? x : 0;
            total += x;
        }
        // exclusive scan of the totals over the 256 digits
        int incl = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += wsum[w];
        run[d] = wbase + incl - total + before;
    }
    for (int tile = c.beg; tile < c.end; tile += kRsThreads) {
        for (int j = threadIdx.x; j < W * kRsDigits; j += kRsThreads) (&wcnt[0][0])[j] = 0;
        __syncthreads();
        const int i = tile + threadIdx.x;
        const bool valid = i < c.end;
        const unsigned k = valid ? rs_key(in, i) : 0u;
        const int v = valid ? (in.vals ? in.vals[i] : i) : 0;
        const int digit = valid ? (int)((k >> shift) & (kRsDigits - 1)) : kRsDigits;   // padding lanes group apart
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            const int d = threadIdx.x;
            int s = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                int x = wcnt[w][d];
                wcnt[w][d] = s;
                s += x;
            }
            tot[d] = s;
        }
        __syncthreads();
        if (valid) {
            const int pos = run[digit] + wcnt[warp][digit] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        run[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
}

// Sort the child arena by edge key.  Leaves the sorted (key, index) pairs in
// key_buf[r] / val_buf[r] and returns r.
int launch_sort_children(const WinSoA& arena, const Inst* insts, const int* n_ptr, int cap, int key_bits, int by_edge,
                         unsigned* key_buf[2], int* val_buf[2], int* hist, int blocks, cudaStream_t s) {
    int passes = (key_bits + kRsDigitBits - 1) / kRsDigitBits;
    if (passes < 1) passes = 1;
    int src = -1;   // -1: the arena
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kRsDigitBits;
        const int dst = (src + 1) & 1;
        RsIn in{};
        in.he = arena.he;
        in.inst = arena.inst;
        in.insts = insts;
        in.by_edge = by_edge;
        if (src >= 0) {
            in.keys = key_buf[src];
            in.vals = val_buf[src];
        }
        k_rs_hist<<<blocks, kRsThreads, 0, s>>>(in, n_ptr, cap, shift, hist);
        k_rs_scatter<<<blocks, kRsThreads, 0, s>>>(in, key_buf[dst], val_buf[dst], n_ptr, cap, shift, hist);
        src = dst;
    }
    return src;
}

int sort_kernels_per_pass() { return 2; }

}  // namespace pch
