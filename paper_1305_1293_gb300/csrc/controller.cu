// Learned selection controller: parameters, training kernels (forward, backward, Adam)
// and the FP64 peak microbenchmark.  The network and its role are described in
// controller.cuh; none of this has a counterpart in the paper, which fixes k by hand
// (Section 5.2).
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "pch_host.h"
#include "solver.cuh"

namespace pch {

// Installed controller weights, one device buffer per device, each valid only in the
// context it was allocated in (a reset device loses its weights).
constexpr int kMaxDevices = 64;
struct DevPtrSlot {
    unsigned long long ctx = 0;   // current_context_id() when ptr was obtained; 0 = empty
    float* ptr = nullptr;
};
static DevPtrSlot g_mlp_slot[kMaxDevices];
static std::mutex g_mlp_mu;

// The current device's weights, or nullptr when none were installed in its current
// context: PCH_CONTROL_LEARNED then runs the plain control.
const float* mlp_device_params() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    const DevPtrSlot& sl = g_mlp_slot[dev];
    return (ctx != 0 && sl.ctx == ctx) ? sl.ptr : nullptr;
}

long long default_k() {
    const char* e = std::getenv("PCH_DEFAULT_K");
    if (e) {
        long long v = std::atoll(e);
        if (v > 0) return v;
    }
    return 24576;   // the paper's tuned range 16*2^10 .. 24*2^10 (Section 5.2)
}

int default_hops() {
    const char* e = std::getenv("PCH_DEFAULT_HOPS");
    if (e) {
        int v = std::atoi(e);
        if (v > 0) return v;
    }
    return 32;
}

int default_take_min() {
    const char* e = std::getenv("PCH_TAKE_MIN");
    if (e) {
        int v = std::atoi(e);
        if (v >= 1 && v <= 32) return v;
    }
    return 1;
}

int default_tail_cut() {
    const char* e = std::getenv("PCH_TAIL_CUT");
    if (e) {
        int v = std::atoi(e);
        if (v >= 0) return v;
    }
    return 0;
}

// Resident propagation blocks per SM: 384 threads per SM (12 warps of up to 168
// registers a thread fill the register file), unless PCH_PROP_BLOCKS_PER_SM says otherwise.
int default_prop_blocks_per_sm(int block) {
    const char* e = std::getenv("PCH_PROP_BLOCKS_PER_SM");
    if (e) {
        int v = std::atoi(e);
        if (v > 0 && v <= 32) return v;
    }
    return block >= 384 ? 1 : 384 / block;
}

// ---------------------------------------------------------------- training kernels
// One block of kHidden threads per sample.  act: [n][3][kHidden] post-ReLU activations.
__global__ void __launch_bounds__(kHidden) k_mlp_fwd(const float* __restrict__ p, const float* __restrict__ x, int n,
                                                     float* __restrict__ y, float* __restrict__ act) {
    __shared__ float xs[kFeatures], h0[kHidden], h1[kHidden], h2[kHidden];
    const int t = threadIdx.x;
    for (int b = blockIdx.x; b < n; b += gridDim.x) {
        if (t < kFeatures) xs[t] = x[(size_t)b * kFeatures + t];
        __syncthreads();
        float s = p[kMlpB1 + t];
        for (int i = 0; i < kFeatures; ++i) s = fmaf(p[kMlpW1 + t * kFeatures + i], xs[i], s);
        h0[t] = fmaxf(s, 0.f);
        __syncthreads();
        s = p[kMlpB2 + t];
        for (int i = 0; i < kHidden; ++i) s = fmaf(p[kMlpW2 + t * kHidden + i], h0[i], s);
        h1[t] = fmaxf(s, 0.f);
        __syncthreads();
        s = p[kMlpB3 + t];
        for (int i = 0; i < kHidden; ++i) s = fmaf(p[kMlpW3 + t * kHidden + i], h1[i], s);
        h2[t] = fmaxf(s, 0.f);
        __syncthreads();
        if (act) {
            act[((size_t)b * 3 + 0) * kHidden + t] = h0[t];
            act[((size_t)b * 3 + 1) * kHidden + t] = h1[t];
            act[((size_t)b * 3 + 2) * kHidden + t] = h2[t];
        }
        if (t == 0) {
            float o = p[kMlpB4];
            for (int i = 0; i < kHidden; ++i) o = fmaf(p[kMlpW4 + i], h2[i], o);
            y[b] = o;
        }
        __syncthreads();
    }
}

// Per-sample back-propagation of L = 0.5 mean((y - target)^2): dlt [n][3][kHidden]
// holds dL/dz for each hidden layer's pre-activation; dy[n] = (y - t) / n.
__global__ void __launch_bounds__(kHidden) k_mlp_bwd(const float* __restrict__ p, const float* __restrict__ act,
                                                     const float* __restrict__ y, const float* __restrict__ target,
                                                     int n, float* __restrict__ dlt, float* __restrict__ dy) {
    __shared__ float d2[kHidden], d1[kHidden];
    const int t = threadIdx.x;
    for (int b = blockIdx.x; b < n; b += gridDim.x) {
        const float* a = act + (size_t)b * 3 * kHidden;
        const float e = (y[b] - target[b]) / (float)n;
        if (t == 0) dy[b] = e;
        float v = a[2 * kHidden + t] > 0.f ? e * p[kMlpW4 + t] : 0.f;
        d2[t] = v;
        dlt[((size_t)b * 3 + 2) * kHidden + t] = v;
        __syncthreads();
        float s = 0.f;
        for (int j = 0; j < kHidden; ++j) s = fmaf(p[kMlpW3 + j * kHidden + t], d2[j], s);
        v = a[kHidden + t] > 0.f ? s : 0.f;
        d1[t] = v;
        dlt[((size_t)b * 3 + 1) * kHidden + t] = v;
        __syncthreads();
        s = 0.f;
        for (int j = 0; j < kHidden; ++j) s = fmaf(p[kMlpW2 + j * kHidden + t], d1[j], s);
        dlt[((size_t)b * 3 + 0) * kHidden + t] = a[t] > 0.f ? s : 0.f;
        __syncthreads();
    }
}

// One thread per parameter, sums over the samples in order: deterministic.
__global__ void k_mlp_grad(const float* __restrict__ x, const float* __restrict__ act, const float* __restrict__ dlt,
                           const float* __restrict__ dy, int n, float* __restrict__ grad) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kMlpParams; q += gridDim.x * blockDim.x) {
        float s = 0.f;
        if (q < kMlpB1) {
            int o = (q - kMlpW1) / kFeatures, i = (q - kMlpW1) % kFeatures;
            for (int b = 0; b < n; ++b) s = fmaf(dlt[((size_t)b * 3 + 0) * kHidden + o], x[(size_t)b * kFeatures + i], s);
        } else if (q < kMlpW2) {
            int o = q - kMlpB1;
            for (int b = 0; b < n; ++b) s += dlt[((size_t)b * 3 + 0) * kHidden + o];
        } else if (q < kMlpB2) {
            int o = (q - kMlpW2) / kHidden, i = (q - kMlpW2) % kHidden;
            for (int b = 0; b < n; ++b)
                s = fmaf(dlt[((size_t)b * 3 + 1) * kHidden + o], act[((size_t)b * 3 + 0) * kHidden + i], s);
        } else if (q < kMlpW3) {
            int o = q - kMlpB2;
            for (int b = 0; b < n; ++b) s += dlt[((size_t)b * 3 + 1) * kHidden + o];
        } else if (q < kMlpB3) {
            int o = (q - kMlpW3) / kHidden, i = (q - kMlpW3) % kHidden;
            for (int b = 0; b < n; ++b)
                s = fmaf(dlt[((size_t)b * 3 + 2) * kHidden + o], act[((size_t)b * 3 + 1) * kHidden + i], s);
        } else if (q < kMlpW4) {
            int o = q - kMlpB3;
            for (int b = 0; b < n; ++b) s += dlt[((size_t)b * 3 + 2) * kHidden + o];
        } else if (q < kMlpB4) {
            int i = q - kMlpW4;
            for (int b = 0; b < n; ++b) s = fmaf(dy[b], act[((size_t)b * 3 + 2) * kHidden + i], s);
        } else {
            for (int b = 0; b < n; ++b) s += dy[b];
        }
        grad[q] = s;
    }
}

__global__ void k_mlp_loss(const float* __restrict__ y, const float* __restrict__ target, int n, float* loss) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        double e = (double)y[b] - (double)target[b];
        s += e * e;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(0.5 * sh[0] / n);
}

__global__ void k_mlp_adam(float* p, const float* __restrict__ g, float* m, float* v, int t, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kMlpParams; q += gridDim.x * blockDim.x) {
        float gq = g[q];
        float mq = b1 * m[q] + (1.f - b1) * gq;
        float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    }
}

// ---------------------------------------------------------------- FP64 peak
__global__ void k_dfma_peak(double* out, int iters) {
    double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-3, a2 = a0 + 2e-3, a3 = a0 + 3e-3;
    double a4 = a0 + 4e-3, a5 = a0 + 5e-3, a6 = a0 + 6e-3, a7 = a0 + 7e-3;
    const double m = 0.999999, c = 1e-7;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
        a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
    double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == 12345.678) out[0] = s;   // keep the chains alive
}

}  // namespace pch

using namespace pch;

extern "C" int32_t pch_mlp_num_features(void) { return kFeatures; }
extern "C" int32_t pch_mlp_num_params(void) { return kMlpParams; }

extern "C" pch_status pch_mlp_set_weights(const float* params, int32_t n_params) {
    clear_error();
    if (!params || n_params != kMlpParams) return set_error(PCH_ERR_INVALID_ARG, "expected %d parameters", kMlpParams);
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(params[i])) return set_error(PCH_ERR_INVALID_ARG, "non-finite weight %d", i);
    int dev = 0;
    PCH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(PCH_ERR_INVALID_ARG, "device id %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    DevPtrSlot& sl = g_mlp_slot[dev];
    unsigned long long ctx = current_context_id();
    if (ctx == 0 || sl.ctx != ctx) {
        // first weights in this device's current context (a buffer of an earlier, destroyed
        // context is gone with it and is not freed)
        float* p = nullptr;
        PCH_CUDA(cudaMalloc(&p, sizeof(float) * kMlpParams));
        sl.ptr = p;
        sl.ctx = current_context_id();   // the allocation made the context current
    }
    PCH_CUDA(cudaMemcpy(sl.ptr, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
    return PCH_OK;
}

extern "C" pch_status pch_mlp_forward(const float* params_dev, const float* x_dev, int32_t n, float* y_dev,
                                      void* stream) {
    clear_error();
    if (!params_dev || !x_dev || !y_dev || n <= 0) return set_error(PCH_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    k_mlp_fwd<<<std::min(n, 65535), kHidden, 0, s>>>(params_dev, x_dev, n, y_dev, nullptr);
    PCH_CUDA(cudaGetLastError());
    return PCH_OK;
}

extern "C" pch_status pch_mlp_backward(const float* params_dev, const float* x_dev, const float* target_dev, int32_t n,
                                       float* grad_dev, float* loss_dev, void* stream) {
    clear_error();
    if (!params_dev || !x_dev || !target_dev || !grad_dev || !loss_dev || n <= 0)
        return set_error(PCH_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: activations, deltas, outputs
    float* scratch = nullptr;
    size_t nact = (size_t)n * 3 * kHidden;
    PCH_CUDA(cudaMallocAsync(&scratch, sizeof(float) * (2 * nact + 2 * (size_t)n), s));
    float* act = scratch;
    float* dlt = act + nact;
    float* y = dlt + nact;
    float* dy = y + n;
    int g = std::min(n, 65535);
    k_mlp_fwd<<<g, kHidden, 0, s>>>(params_dev, x_dev, n, y, act);
    k_mlp_bwd<<<g, kHidden, 0, s>>>(params_dev, act, y, target_dev, n, dlt, dy);
    k_mlp_grad<<<(kMlpParams + 255) / 256, 256, 0, s>>>(x_dev, act, dlt, dy, n, grad_dev);
    k_mlp_loss<<<1, 256, 0, s>>>(y, target_dev, n, loss_dev);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(scratch, s);
    PCH_CUDA(e);
    return PCH_OK;
}

extern "C" pch_status pch_mlp_adam(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int32_t t,
                                   float lr, void* stream) {
    clear_error();
    if (!params_dev || !grad_dev || !m_dev || !v_dev || t < 1) return set_error(PCH_ERR_INVALID_ARG, "bad arguments");
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params_dev, grad_dev, m_dev, v_dev, t, lr);
    PCH_CUDA(cudaGetLastError());
    return PCH_OK;
}

extern "C" pch_status pch_measure_fp64_peak(double* tflops) {
    clear_error();
    if (!tflops) return set_error(PCH_ERR_INVALID_ARG, "null output");
    double* out = nullptr;
    PCH_CUDA(cudaMalloc(&out, sizeof(double)));
    const int blocks = sm_count() * 8, threads = 256, iters = 1 << 14;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_dfma_peak<<<blocks, threads>>>(out, 256);   // warm-up
    cudaEventRecord(a);
    k_dfma_peak<<<blocks, threads>>>(out, iters);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    PCH_CUDA(e);
    double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return PCH_OK;
}

// ---------------------------------------------------------------- allocation-free backward
// Scratch of pch_mlp_backward_noalloc, in a file-scope device array instead of a
// cudaMallocAsync buffer: per-sample activations and deltas (3 x 64 floats each), the
// outputs and their errors, for at most kNoAllocMaxSamples samples (6.3 MB).  Every
// GPU that loads the library holds this array until the process exits.
namespace pch {
constexpr int kNoAllocMaxSamples = 4096;
constexpr size_t kNoAllocActFloats = (size_t)kNoAllocMaxSamples * 3 * kHidden;
constexpr size_t kNoAllocFloats = 2 * kNoAllocActFloats + 2 * (size_t)kNoAllocMaxSamples;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];
// Host side: the array's device address, resolved once per device and context (a reset
// device gets a new context, and the array a new address).  The symbol itself is only a
// host-side stand-in and must never be handed to a kernel.
static DevPtrSlot g_noalloc_slot[kMaxDevices];
static std::mutex g_noalloc_mu;
}  // namespace pch

extern "C" pch_status pch_mlp_backward_noalloc(const float* params_dev, const float* x_dev, const float* target_dev,
                                               int32_t n, float* grad_dev, float* loss_dev, void* stream) {
    clear_error();
    if (!params_dev || !x_dev || !target_dev || !grad_dev || !loss_dev || n <= 0)
        return set_error(PCH_ERR_INVALID_ARG, "bad arguments");
    if (n > kNoAllocMaxSamples)
        return set_error(PCH_ERR_CAPACITY, "pch_mlp_backward_noalloc takes at most %d samples (got %d)",
                         kNoAllocMaxSamples, n);
    int dev = 0;
    PCH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(PCH_ERR_INVALID_ARG, "device id %d out of range", dev);
    float* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        DevPtrSlot& sl = g_noalloc_slot[dev];
        const unsigned long long ctx = current_context_id();
        if (ctx != 0 && sl.ctx == ctx) {
            scratch = sl.ptr;
        } else {
            // first call on this device in its current context (the device is current):
            // look the array up
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || p == nullptr)
                return set_error(PCH_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                                 cudaGetErrorString(e));
            scratch = static_cast<float*>(p);
            sl.ptr = scratch;
            sl.ctx = current_context_id();
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* act = scratch;
    float* dlt = act + kNoAllocActFloats;
    float* y = dlt + kNoAllocActFloats;
    float* dy = y + kNoAllocMaxSamples;
    // every scratch element read below is written first by the same call: nothing to clear
    int g = std::min(n, 65535);
    k_mlp_fwd<<<g, kHidden, 0, s>>>(params_dev, x_dev, n, y, act);
    k_mlp_bwd<<<g, kHidden, 0, s>>>(params_dev, act, y, target_dev, n, dlt, dy);
    k_mlp_grad<<<(kMlpParams + 255) / 256, 256, 0, s>>>(x_dev, act, dlt, dy, n, grad_dev);
    k_mlp_loss<<<1, 256, 0, s>>>(y, target_dev, n, loss_dev);
    PCH_CUDA(cudaGetLastError());
    return PCH_OK;
}
