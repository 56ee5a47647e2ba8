// cc_mlp.cu -- the learned variant selector's network (no counterpart in
// the paper, which gives a hand-made decision tree, Section 4.7): a small
// FP32 multilayer perceptron 16 -> 64 -> 64 -> 12 with ReLU, trained on the
// GPU by these kernels.  Nothing here touches connectivity labels; the
// selector only chooses which sampling x finish combination to run.
//
// Parameter block (floats): mu[16], sigma[16] (input standardisation, not
// trained), W1[16][64], b1[64], W2[64][64], b2[64], W3[64][12], b3[12].
// Loss: cross-entropy of softmax(logits) against a soft target
// distribution (targets from measured times, see cc_mlp_soft_targets).
// Gradients are formed per sample, then summed over samples in a fixed
// order, so a training step is deterministic.
#include <cmath>

#include "cc_mlp.cuh"

using namespace ccg;

namespace {

constexpr int IN = MLP_IN, H = MLP_H, OUT = MLP_OUT;
constexpr int O_MU = MLP_O_MU, O_SIG = MLP_O_SIG, O_W1 = MLP_O_W1, O_B1 = MLP_O_B1, O_W2 = MLP_O_W2,
              O_B2 = MLP_O_B2, O_W3 = MLP_O_W3, O_B3 = MLP_O_B3, NP = MLP_NP;
constexpr int O_TRAIN = O_W1;              // first trained parameter
constexpr int NTRAIN = NP - O_TRAIN;

// one block of 64 threads per sample
__global__ void k_mlp_forward(const float *__restrict__ p, const float *__restrict__ X, uint32_t B,
                              float *__restrict__ logits, float *__restrict__ acts) {
    __shared__ float x[IN], h1[H], h2[H];
    const uint32_t s = blockIdx.x;
    if (s >= B) return;
    const int t = threadIdx.x;
    mlp_forward_one(p, X + (size_t)s * IN, x, h1, h2, logits + (size_t)s * OUT);
    if (acts) {
        acts[(size_t)s * 2 * H + t] = h1[t];
        acts[(size_t)s * 2 * H + H + t] = h2[t];
    }
}

// Per-sample gradient of the cross-entropy to soft targets Q:
// dz = softmax(z) - q, back through the layers; written to G[s][NTRAIN]
// (scaled by 1/B) with the per-sample loss.
__global__ void k_mlp_backward(const float *__restrict__ p, const float *__restrict__ X,
                               const float *__restrict__ acts, const float *__restrict__ logits,
                               const float *__restrict__ Q, uint32_t B, float *__restrict__ G,
                               float *__restrict__ loss_s) {
    __shared__ float x[IN], h1[H], h2[H], dz[OUT], dh2[H], dh1[H];
    const uint32_t s = blockIdx.x;
    if (s >= B) return;
    const int t = threadIdx.x;
    const float invB = 1.0f / (float)B;
    if (t < IN) {
        float sg = p[O_SIG + t];
        sg = sg > 1e-6f ? sg : 1e-6f;
        x[t] = (X[(size_t)s * IN + t] - p[O_MU + t]) / sg;
    }
    h1[t] = acts[(size_t)s * 2 * H + t];
    h2[t] = acts[(size_t)s * 2 * H + H + t];
    if (t == 0) {
        const float *z = logits + (size_t)s * OUT;
        float mx = z[0];
        for (int k = 1; k < OUT; ++k) mx = z[k] > mx ? z[k] : mx;
        float se = 0.f;
        for (int k = 0; k < OUT; ++k) se += expf(z[k] - mx);
        const float lse = mx + logf(se);
        float l = 0.f;
        for (int k = 0; k < OUT; ++k) {
            const float q = Q[(size_t)s * OUT + k];
            dz[k] = (expf(z[k] - lse) - q) * invB;
            l -= q * (z[k] - lse);
        }
        loss_s[s] = l;
    }
    __syncthreads();
    // dh2 = W3 dz (masked by ReLU)
    float a = 0.f;
    for (int k = 0; k < OUT; ++k) a = fmaf(p[O_W3 + t * OUT + k], dz[k], a);
    dh2[t] = h2[t] > 0.f ? a : 0.f;
    __syncthreads();
    a = 0.f;
    for (int j = 0; j < H; ++j) a = fmaf(p[O_W2 + t * H + j], dh2[j], a);
    dh1[t] = h1[t] > 0.f ? a : 0.f;
    __syncthreads();
    float *g = G + (size_t)s * NTRAIN;   // g[k] is the gradient of parameter O_TRAIN + k
    for (int idx = t; idx < IN * H; idx += H) g[O_W1 - O_TRAIN + idx] = x[idx / H] * dh1[idx % H];
    g[O_B1 - O_TRAIN + t] = dh1[t];
    for (int idx = t; idx < H * H; idx += H) g[O_W2 - O_TRAIN + idx] = h1[idx / H] * dh2[idx % H];
    g[O_B2 - O_TRAIN + t] = dh2[t];
    for (int idx = t; idx < H * OUT; idx += H) g[O_W3 - O_TRAIN + idx] = h2[idx / OUT] * dz[idx % OUT];
    if (t < OUT) g[O_B3 - O_TRAIN + t] = dz[t];
}

// grads[j] = sum over samples (fixed order); loss = mean of per-sample losses
__global__ void k_mlp_reduce(const float *__restrict__ G, const float *__restrict__ loss_s, uint32_t B,
                             float *__restrict__ grads, float *__restrict__ loss) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < NTRAIN) {
        float a = 0.f;
        for (uint32_t s = 0; s < B; ++s) a += G[(size_t)s * NTRAIN + j];
        grads[O_TRAIN + j] = a;
    } else if (j < (uint32_t)NP) {
        grads[j - NTRAIN] = 0.f;   // mu, sigma are not trained
    }
    if (j == 0 && loss) {
        float l = 0.f;
        for (uint32_t s = 0; s < B; ++s) l += loss_s[s];
        *loss = l / (float)B;
    }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * mhat / (sqrt(vhat) + eps), on the trained parameters only.
__global__ void k_mlp_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, uint32_t step, float lr) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x + O_TRAIN;
    if (j >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mj = b1 * m[j] + (1.f - b1) * g[j];
    const float vj = b2 * v[j] + (1.f - b2) * g[j] * g[j];
    m[j] = mj;
    v[j] = vj;
    const float mh = mj / (1.f - powf(b1, (float)step));
    const float vh = vj / (1.f - powf(b2, (float)step));
    p[j] -= lr * mh / (sqrtf(vh) + eps);
}

// Parameter initialisation: mu = 0, sigma = 1, weights uniform in
// +-sqrt(6 / (fan_in + fan_out)) (Glorot) from counter-based draws, biases 0.
__global__ void k_mlp_init(float *p, uint64_t seed) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NP) return;
    float val = 0.f;
    int fin = 0, fout = 0;
    if (j < O_SIG) val = 0.f;
    else if (j < O_W1) val = 1.f;
    else if (j < O_B1) { fin = IN; fout = H; }
    else if (j < O_W2) val = 0.f;
    else if (j < O_B2) { fin = H; fout = H; }
    else if (j < O_W3) val = 0.f;
    else if (j < O_B3) { fin = H; fout = OUT; }
    else val = 0.f;
    if (fin) {
        const float u = (float)(draw64(seed ^ 0x6D6C7069ull, (uint64_t)j) >> 40) * (1.0f / 16777216.0f);
        const float lim = sqrtf(6.f / (float)(fin + fout));
        val = (2.f * u - 1.f) * lim;
    }
    p[j] = val;
}

// Input standardisation from a training set: mu = mean, sigma = std.
__global__ void k_mlp_norm(float *p, const float *X, uint32_t B) {
    const int t = threadIdx.x;
    if (t >= IN) return;
    float s = 0.f, s2 = 0.f;
    for (uint32_t i = 0; i < B; ++i) {
        const float x = X[(size_t)i * IN + t];
        s += x;
        s2 += x * x;
    }
    const float mu = s / (float)B;
    const float var = s2 / (float)B - mu * mu;
    p[O_MU + t] = mu;
    p[O_SIG + t] = var > 1e-12f ? sqrtf(var) : 1.f;
}

// Soft targets from measured times: r_c = t_c / t_best - 1 (the regret of
// class c), q_c proportional to exp(-r_c / tau).
__global__ void k_mlp_soft_targets(const float *times, uint32_t B, float tau, float *Q) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const float *t = times + (size_t)s * OUT;
    float best = t[0];
    for (int k = 1; k < OUT; ++k) best = t[k] < best ? t[k] : best;
    float z = 0.f, q[OUT];
    for (int k = 0; k < OUT; ++k) {
        q[k] = expf(-(t[k] / best - 1.f) / tau);
        z += q[k];
    }
    for (int k = 0; k < OUT; ++k) Q[(size_t)s * OUT + k] = q[k] / z;
}

__global__ void k_mlp_argmax(const float *logits, uint32_t B, int32_t *cls) {
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    cls[s] = mlp_argmax(logits + (size_t)s * OUT);
}

}  // namespace

extern "C" {

cc_status cc_mlp_init(float *params, uint64_t seed, void *stream) {
    if (!params) return CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        CC_PROF("k_mlp_init", s);
        k_mlp_init<<<(NP + 255) / 256, 256, 0, s>>>(params, seed);
    }
    return from_cuda(cudaGetLastError());
}

cc_status cc_mlp_set_norm(float *params, const float *X, uint32_t B, void *stream) {
    if (!params || !X || B == 0) return CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        CC_PROF("k_mlp_norm", s);
        k_mlp_norm<<<1, 32, 0, s>>>(params, X, B);
    }
    return from_cuda(cudaGetLastError());
}

cc_status cc_mlp_forward(const float *params, const float *X, uint32_t B, float *logits, float *acts, void *stream) {
    if (!params || !X || !logits || B == 0) return B == 0 ? CC_OK : CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        CC_PROF("k_mlp_forward", s);
        k_mlp_forward<<<B, H, 0, s>>>(params, X, B, logits, acts);
    }
    return from_cuda(cudaGetLastError());
}

cc_status cc_mlp_soft_targets(const float *times, uint32_t B, float tau, float *targets, void *stream) {
    if (!times || !targets || !(tau > 0.f)) return CC_ERR_INVALID;
    if (B == 0) return CC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        CC_PROF("k_mlp_soft_targets", s);
        k_mlp_soft_targets<<<(B + 127) / 128, 128, 0, s>>>(times, B, tau, targets);
    }
    return from_cuda(cudaGetLastError());
}

cc_status cc_mlp_backward(const float *params, const float *X, const float *acts, const float *logits,
                          const float *targets, uint32_t B, float *grads, float *loss, void *stream) {
    if (!params || !X || !acts || !logits || !targets || !grads || B == 0) return CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    const size_t og = sc.reserve((size_t)B * NTRAIN * 4), ol = sc.reserve((size_t)B * 4);
    cc_status st = sc.alloc(s);
    if (st != CC_OK) return st;
    {
        CC_PROF("k_mlp_backward", s);
        k_mlp_backward<<<B, H, 0, s>>>(params, X, acts, logits, targets, B, sc.at<float>(og), sc.at<float>(ol));
    }
    {
        CC_PROF("k_mlp_reduce", s);
        k_mlp_reduce<<<(NP + 255) / 256, 256, 0, s>>>(sc.at<float>(og), sc.at<float>(ol), B, grads, loss);
    }
    return from_cuda(cudaGetLastError());
}

cc_status cc_mlp_adam(float *params, const float *grads, float *m, float *v, uint32_t step, float lr, void *stream) {
    if (!params || !grads || !m || !v || step == 0 || !(lr > 0.f)) return CC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        CC_PROF("k_mlp_adam", s);
        k_mlp_adam<<<(NTRAIN + 255) / 256, 256, 0, s>>>(params, grads, m, v, step, lr);
    }
    return from_cuda(cudaGetLastError());
}

cc_status cc_mlp_predict(const float *params, const float *X, uint32_t B, int32_t *class_out, void *stream) {
    if (!params || !X || !class_out) return CC_ERR_INVALID;
    if (B == 0) return CC_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch sc;
    const size_t ol = sc.reserve((size_t)B * OUT * 4);
    cc_status st = sc.alloc(s);
    if (st != CC_OK) return st;
    {
        CC_PROF("k_mlp_forward", s);
        k_mlp_forward<<<B, H, 0, s>>>(params, X, B, sc.at<float>(ol), nullptr);
    }
    {
        CC_PROF("k_mlp_argmax", s);
        k_mlp_argmax<<<(B + 127) / 128, 128, 0, s>>>(sc.at<float>(ol), B, class_out);
    }
    return from_cuda(cudaGetLastError());
}

}  // extern "C"
