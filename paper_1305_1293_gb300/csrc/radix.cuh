#pragma once
#include "pch_common.cuh"

namespace pch {

constexpr int kRsDigitBits = 8;
constexpr int kRsDigits = 1 << kRsDigitBits;
constexpr int kRsThreads = 256;
constexpr int kRsChunkMin = 2048;     // elements per sort block at least

// Input of one sort pass: stored (key, index) pairs, or (keys == nullptr) the child arena.
struct RsIn {
    const unsigned* keys;
    const int* vals;
    const int* he;
    const int* inst;
    const Inst* insts;
    int by_edge;    // key = instance key base + half-edge; else the instance
};

int launch_sort_children(const WinSoA& arena, const Inst* insts, const int* n_ptr, int cap, int key_bits, int by_edge,
                         unsigned* key_buf[2], int* val_buf[2], int* hist, int blocks, cudaStream_t s);
int sort_kernels_per_pass();

}  // namespace pch
