#pragma once
#include "pch_common.cuh"

namespace pch {

constexpr int kRsDigitBits = 8;
constexpr int kRsDigits = 1 << kRsDigitBits;
constexpr int kRsThreads = 256;
constexpr int kRsScanThreads = 1024;

int launch_sort_children(const WinSoA& arena, const Inst* insts, const int* n_ptr, int cap, int key_bits,
                         unsigned* key_buf[2], int* val_buf[2], int* hist, int blocks, cudaStream_t s);

}  // namespace pch
