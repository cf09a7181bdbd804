// Learned selection controller: device-side features and inference.
//
// The paper controls each iteration with a fixed window count k (Section 4.2, Step 1;
// the trade-off of Section 5.2, Fig. `fig:parameter`).  This controller replaces the
// fixed k by a 3 x 64 hidden-layer fp32 MLP that maps the frontier statistics of one
// instance to log2 of the number of windows to select, divided by 24.  Any window order
// gives the same distances (Section 4.3, Remark 2), so the controller can change speed,
// never results; a non-finite or out-of-range output falls back to the plain k.
#pragma once
#include "pch_common.cuh"

namespace pch {

// Parameter layout: W1[64][24] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4[1].
constexpr int kMlpW1 = 0;
constexpr int kMlpB1 = kMlpW1 + kHidden * kFeatures;
constexpr int kMlpW2 = kMlpB1 + kHidden;
constexpr int kMlpB2 = kMlpW2 + kHidden * kHidden;
constexpr int kMlpW3 = kMlpB2 + kHidden;
constexpr int kMlpB3 = kMlpW3 + kHidden * kHidden;
constexpr int kMlpW4 = kMlpB3 + kHidden;
constexpr int kMlpB4 = kMlpW4 + kHidden;
constexpr int kMlpParams = kMlpB4 + 1;

// Frontier statistics of one instance at the start of an iteration (row a8):
//  f0      log2(1 + pending) / 20
//  f1..16  cumulative fraction of pending windows within 2^j/4 mean edge lengths of the
//          reference (the nearest pending key), j = 0..15 (octave-coarsened histogram)
//  f17     log2(faces) / 24
//  f18     log2(mean edge length) / 8
//  f19     log2(1 + iteration) / 16
//  f20     children per selected window in the previous iteration / 4
//  f21     log2(1 + front distance / mean edge length) / 16
//  f22     log2(1 + pending / faces) / 8
//  f23     1
__device__ __forceinline__ void controller_features(const InstCtl& c, const Inst& I, const unsigned* hist, int np,
                                                    int it, float* f) {
    f[0] = log2f(1.f + (float)np) / 20.f;
    unsigned run = 0;
    for (int j = 0; j < 16; ++j) {
        for (int b = j * 16; b < (j + 1) * 16; ++b) run += hist[b];
        f[1 + j] = np > 0 ? (float)run / (float)np : 0.f;
    }
    float faces = (float)(I.nh / 3);
    f[17] = log2f(faces) / 24.f;
    f[18] = log2f((float)I.lbar) / 8.f;
    f[19] = log2f(1.f + (float)it) / 16.f;
    f[20] = c.last_ratio / 4.f;
    f[21] = log2f(1.f + (float)(c.ref * I.ilbar)) / 16.f;
    f[22] = log2f(1.f + (float)np / faces) / 8.f;
    f[23] = 1.f;
}

// Block-cooperative forward pass (threads 0..63 compute one neuron each per layer).
// `x` (kFeatures) and `h0`, `h1` (kHidden each) live in shared memory; every thread of
// the block must call it.  Returns the output in *y (shared).
__device__ __forceinline__ void mlp_forward_block(const float* __restrict__ p, const float* x, float* h0, float* h1,
                                                  float* y) {
    const int t = threadIdx.x;
    if (t < kHidden) {
        float s = p[kMlpB1 + t];
        const float* wr = p + kMlpW1 + t * kFeatures;
#pragma unroll 8
        for (int i = 0; i < kFeatures; ++i) s = fmaf(wr[i], x[i], s);
        h0[t] = fmaxf(s, 0.f);
    }
    __syncthreads();
    if (t < kHidden) {
        float s = p[kMlpB2 + t];
        const float* wr = p + kMlpW2 + t * kHidden;
#pragma unroll 8
        for (int i = 0; i < kHidden; ++i) s = fmaf(wr[i], h0[i], s);
        h1[t] = fmaxf(s, 0.f);
    }
    __syncthreads();
    if (t < kHidden) {
        float s = p[kMlpB3 + t];
        const float* wr = p + kMlpW3 + t * kHidden;
#pragma unroll 8
        for (int i = 0; i < kHidden; ++i) s = fmaf(wr[i], h1[i], s);
        h0[t] = fmaxf(s, 0.f) * p[kMlpW4 + t];
    }
    __syncthreads();
    if (t < 32) {
        float s = h0[t] + h0[t + 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (t == 0) *y = s + p[kMlpB4];
    }
    __syncthreads();
}

}  // namespace pch
