// Host-side internals shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "pch_common.cuh"

namespace pch {

pch_status set_error(pch_status st, const char* fmt, ...);
void clear_error();

struct Workspace;   // solver.cu

}  // namespace pch

struct pch_mesh {
    pch::DevMesh dm;
    int device;
    int n_boundary_he;
    int n_pseudo;
    pch::Workspace* ws;
};

#define PCH_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            return pch::set_error(e_ == cudaErrorMemoryAllocation ? PCH_ERR_OOM : PCH_ERR_CUDA, \
                                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                  __FILE__, __LINE__);                                    \
        }                                                                                 \
    } while (0)

namespace pch {

// Exclusive scan of n ints (device), out may alias in.  Uses tmp of scan_tmp_ints(n).
size_t scan_tmp_ints(int n);
cudaError_t exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s);

// Number of SMs of the current device (cached).
int sm_count();

// Unique id of the calling thread's current CUDA context, 0 if there is none (or the
// driver cannot tell).  Device pointers the library caches across calls are keyed on it,
// so that a pointer from a context that has since been destroyed (cudaDeviceReset, a new
// primary context) is never used again.
unsigned long long current_context_id();

}  // namespace pch
