// cc_mlp.cuh -- the selector network's forward pass for one sample, shared
// by the batch forward kernel (cc_mlp.cu) and the in-pipeline choice of the
// selected static path (cc_static.cu).  No counterpart in the paper.
//
// Parameter block (floats): mu[16], sigma[16] (input standardisation),
// W1[16][64], b1[64], W2[64][64], b2[64], W3[64][12], b3[12]; ReLU between
// the layers.
#pragma once

#include "cc_internal.h"

namespace ccg {

constexpr int MLP_IN = CC_MLP_IN, MLP_H = CC_MLP_HID, MLP_OUT = CC_MLP_OUT;
constexpr int MLP_O_MU = 0, MLP_O_SIG = MLP_IN, MLP_O_W1 = 2 * MLP_IN, MLP_O_B1 = MLP_O_W1 + MLP_IN * MLP_H,
              MLP_O_W2 = MLP_O_B1 + MLP_H, MLP_O_B2 = MLP_O_W2 + MLP_H * MLP_H, MLP_O_W3 = MLP_O_B2 + MLP_H,
              MLP_O_B3 = MLP_O_W3 + MLP_H * MLP_OUT, MLP_NP = MLP_O_B3 + MLP_OUT;
static_assert(MLP_NP == CC_MLP_NPARAM, "parameter layout");

// One sample by a block of MLP_H threads (t = threadIdx.x < MLP_H).  xin:
// the raw features (any memory); x, h1, h2: shared arrays of MLP_IN, MLP_H,
// MLP_H floats; logits (any memory, MLP_OUT floats) is written by threads
// t < MLP_OUT.  h1 and h2 hold the hidden activations on return.  Every
// thread of the block must call it (it synchronises).
__device__ __forceinline__ void mlp_forward_one(const float *__restrict__ p, const float *xin, float *x, float *h1,
                                                float *h2, float *logits) {
    const int t = threadIdx.x;
    if (t < MLP_IN) {
        float sg = p[MLP_O_SIG + t];
        sg = sg > 1e-6f ? sg : 1e-6f;
        x[t] = (xin[t] - p[MLP_O_MU + t]) / sg;
    }
    __syncthreads();
    float a = p[MLP_O_B1 + t];
    for (int i = 0; i < MLP_IN; ++i) a = fmaf(x[i], p[MLP_O_W1 + i * MLP_H + t], a);
    h1[t] = a > 0.f ? a : 0.f;
    __syncthreads();
    a = p[MLP_O_B2 + t];
    for (int i = 0; i < MLP_H; ++i) a = fmaf(h1[i], p[MLP_O_W2 + i * MLP_H + t], a);
    h2[t] = a > 0.f ? a : 0.f;
    __syncthreads();
    if (t < MLP_OUT) {
        a = p[MLP_O_B3 + t];
        for (int i = 0; i < MLP_H; ++i) a = fmaf(h2[i], p[MLP_O_W3 + i * MLP_OUT + t], a);
        logits[t] = a;
    }
}

// The chosen class: the largest logit, ties to the smallest index.
__device__ __forceinline__ int mlp_argmax(const float *z) {
    int best = 0;
    for (int k = 1; k < MLP_OUT; ++k)
        if (z[k] > z[best]) best = k;
    return best;
}

}  // namespace ccg
