// mlp.cu - the learned-alpha predictor: an MLP 4 -> 32 -> 32 -> 1 (tanh hidden layers, FP32)
// with hand-written forward, backward and Adam kernels.
//
// Model layout (floats, see BLTT_ALPHA_MODEL_FLOATS in bltt.h): W1[32][4], b1[32], W2[32][32],
// b2[32], w3[32], b3, then the feature standardisation mean[4], std[4] and the label
// standardisation y_mean, y_std.  The network maps standardised features to the standardised
// label log10(alpha); training minimises the mean squared error over the whole set (full-batch
// Adam, beta1 = 0.9, beta2 = 0.999, eps = 1e-8).  Sums over samples run in a fixed order, so a
// training run is deterministic.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

constexpr int H = 32, F = 4;
constexpr int P_W1 = 0, P_B1 = P_W1 + H * F, P_W2 = P_B1 + H, P_B2 = P_W2 + H * H, P_W3 = P_B2 + H,
              P_B3 = P_W3 + H, NPARAM = P_B3 + 1;
constexpr int P_MEAN = NPARAM, P_STD = P_MEAN + F, P_YM = P_STD + F, P_YS = P_YM + 1,
              MODEL_FLOATS = P_YS + 1;
static_assert(MODEL_FLOATS == BLTT_ALPHA_MODEL_FLOATS, "model layout");

struct Scratch {       // per-sample activations and deltas, [n][H] each
  float *h1, *h2, *d1, *d2, *d3, *loss;
};

// forward for one sample from shared-memory parameters; returns the standardised output
__device__ float forward(const float* p, const float* x, float* h1, float* h2) {
  for (int i = 0; i < H; ++i) {
    float z = p[P_B1 + i];
    for (int j = 0; j < F; ++j) z = fmaf(p[P_W1 + i * F + j], x[j], z);
    h1[i] = tanhf(z);
  }
  for (int i = 0; i < H; ++i) {
    float z = p[P_B2 + i];
    for (int j = 0; j < H; ++j) z = fmaf(p[P_W2 + i * H + j], h1[j], z);
    h2[i] = tanhf(z);
  }
  float y = p[P_B3];
  for (int i = 0; i < H; ++i) y = fmaf(p[P_W3 + i], h2[i], y);
  return y;
}

__device__ void standardise(const float* model, const float* feats, int s, float* x) {
  for (int j = 0; j < F; ++j) x[j] = (feats[s * F + j] - model[P_MEAN + j]) / model[P_STD + j];
}

// per-sample forward + backward (delta) pass; thread per sample
__device__ void fwd_bwd(const float* p, const float* model, const float* feats,
                        const float* labels, int n, const Scratch& sc) {
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    float x[F], h1[H], h2[H];
    standardise(model, feats, s, x);
    const float y = forward(p, x, h1, h2);
    const float t = (labels[s] - model[P_YM]) / model[P_YS];
    const float r = y - t;
    sc.loss[s] = r * r;
    const float d3 = 2.0f * r / (float)n;            // dL/dy for L = mean (y - t)^2
    sc.d3[s] = d3;
    float d2[H];
    for (int i = 0; i < H; ++i) {
      d2[i] = p[P_W3 + i] * d3 * (1.0f - h2[i] * h2[i]);
      sc.h2[s * H + i] = h2[i];
      sc.d2[s * H + i] = d2[i];
      sc.h1[s * H + i] = h1[i];
    }
    for (int j = 0; j < H; ++j) {
      float g = 0.f;
      for (int i = 0; i < H; ++i) g = fmaf(p[P_W2 + i * H + j], d2[i], g);
      sc.d1[s * H + j] = g * (1.0f - h1[j] * h1[j]);
    }
  }
}

// gradient of parameter k: a fixed-order sum over the samples
__device__ float grad_of(int k, const float* model, const float* feats, int n, const Scratch& sc) {
  float g = 0.f;
  if (k < P_B1) {
    const int i = k / F, j = k % F;
    for (int s = 0; s < n; ++s) {
      const float xj = (feats[s * F + j] - model[P_MEAN + j]) / model[P_STD + j];
      g = fmaf(sc.d1[s * H + i], xj, g);
    }
  } else if (k < P_W2) {
    const int i = k - P_B1;
    for (int s = 0; s < n; ++s) g += sc.d1[s * H + i];
  } else if (k < P_B2) {
    const int i = (k - P_W2) / H, j = (k - P_W2) % H;
    for (int s = 0; s < n; ++s) g = fmaf(sc.d2[s * H + i], sc.h1[s * H + j], g);
  } else if (k < P_W3) {
    const int i = k - P_B2;
    for (int s = 0; s < n; ++s) g += sc.d2[s * H + i];
  } else if (k < P_B3) {
    const int i = k - P_W3;
    for (int s = 0; s < n; ++s) g = fmaf(sc.d3[s], sc.h2[s * H + i], g);
  } else {
    for (int s = 0; s < n; ++s) g += sc.d3[s];
  }
  return g;
}

__global__ void k_alpha_grad(const float* model, const float* feats, const float* labels, int n,
                             Scratch sc, float* grad, float* loss) {
  __shared__ float p[NPARAM];
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) p[k] = model[k];
  __syncthreads();
  fwd_bwd(p, model, feats, labels, n, sc);
  __syncthreads();
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) grad[k] = grad_of(k, model, feats, n, sc);
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int s = 0; s < n; ++s) l += sc.loss[s];
    *loss = l / (float)n;
  }
}

// full-batch Adam for `epochs` steps, one block; model[0..NPARAM) is updated in place
__global__ void k_alpha_train(float* model, const float* feats, const float* labels, int n,
                              int epochs, float lr, Scratch sc, float* mstate, float* vstate,
                              float* loss_hist) {
  __shared__ float p[NPARAM];
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  float b1t = 1.f, b2t = 1.f;
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) { mstate[k] = 0.f; vstate[k] = 0.f; }
  for (int ep = 0; ep < epochs; ++ep) {
    __syncthreads();
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) p[k] = model[k];
    __syncthreads();
    fwd_bwd(p, model, feats, labels, n, sc);
    __syncthreads();
    b1t *= b1;
    b2t *= b2;
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) {
      const float g = grad_of(k, model, feats, n, sc);
      const float m = b1 * mstate[k] + (1.f - b1) * g;
      const float v = b2 * vstate[k] + (1.f - b2) * g * g;
      mstate[k] = m;
      vstate[k] = v;
      const float mh = m / (1.f - b1t), vh = v / (1.f - b2t);
      model[k] = p[k] - lr * mh / (sqrtf(vh) + eps);
    }
    if (loss_hist && threadIdx.x == 0) {
      float l = 0.f;
      for (int s = 0; s < n; ++s) l += sc.loss[s];
      loss_hist[ep] = l / (float)n;
    }
  }
}

__global__ void k_alpha_predict(const float* model, const float* feats, int n, float* alpha) {
  __shared__ float p[NPARAM];
  for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) p[k] = model[k];
  __syncthreads();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    float x[F], h1[H], h2[H];
    standardise(model, feats, s, x);
    const float y = forward(p, x, h1, h2);
    const float l10 = y * model[P_YS] + model[P_YM];
    alpha[s] = exp10f(l10);
  }
}

struct DevBuf {
  std::vector<void*> ptrs;
  ~DevBuf() { for (void* q : ptrs) cudaFree(q); }
  template <typename T> T* get(size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    ptrs.push_back(q);
    return static_cast<T*>(q);
  }
};

bool check_model(const float* model) {
  for (int j = 0; j < F; ++j) if (!(model[P_STD + j] > 0.f)) return false;
  return model[P_YS] > 0.f;
}

bool alloc_scratch(DevBuf& db, int n, Scratch& sc) {
  sc.h1 = db.get<float>((size_t)n * H);
  sc.h2 = db.get<float>((size_t)n * H);
  sc.d1 = db.get<float>((size_t)n * H);
  sc.d2 = db.get<float>((size_t)n * H);
  sc.d3 = db.get<float>(n);
  sc.loss = db.get<float>(n);
  return sc.h1 && sc.h2 && sc.d1 && sc.d2 && sc.d3 && sc.loss;
}

}  // namespace

extern "C" {

bltt_status bltt_alpha_grad(const float* model, const float* feats, const float* labels, int n,
                            float* grad_out, float* loss_out) {
  if (!model || !feats || !labels || n < 1 || !grad_out) return BLTT_ERR_INVALID_ARG;
  if (!check_model(model)) return BLTT_ERR_INVALID_ARG;
  DevBuf db;
  float* dm = db.get<float>(MODEL_FLOATS);
  float* df = db.get<float>((size_t)n * F);
  float* dl = db.get<float>(n);
  float* dg = db.get<float>(NPARAM);
  float* dloss = db.get<float>(1);
  Scratch sc{};
  if (!dm || !df || !dl || !dg || !dloss || !alloc_scratch(db, n, sc)) return BLTT_ERR_OOM;
  cudaMemcpy(dm, model, MODEL_FLOATS * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(df, feats, (size_t)n * F * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(dl, labels, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
  k_alpha_grad<<<1, 256>>>(dm, df, dl, n, sc, dg, dloss);
  if (cudaGetLastError() != cudaSuccess) return BLTT_ERR_CUDA;
  if (cudaMemcpy(grad_out, dg, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BLTT_ERR_CUDA;
  if (loss_out) cudaMemcpy(loss_out, dloss, sizeof(float), cudaMemcpyDeviceToHost);
  return BLTT_OK;
}

bltt_status bltt_alpha_train(float* model, const float* feats, const float* labels, int n,
                             int epochs, float lr, float* loss_hist) {
  if (!model || !feats || !labels || n < 1 || epochs < 0 || !(lr > 0.f)) return BLTT_ERR_INVALID_ARG;
  if (!check_model(model)) return BLTT_ERR_INVALID_ARG;
  DevBuf db;
  float* dm = db.get<float>(MODEL_FLOATS);
  float* df = db.get<float>((size_t)n * F);
  float* dl = db.get<float>(n);
  float* ms = db.get<float>(NPARAM);
  float* vs = db.get<float>(NPARAM);
  float* lh = loss_hist ? db.get<float>(std::max(epochs, 1)) : nullptr;
  Scratch sc{};
  if (!dm || !df || !dl || !ms || !vs || (loss_hist && !lh) || !alloc_scratch(db, n, sc))
    return BLTT_ERR_OOM;
  cudaMemcpy(dm, model, MODEL_FLOATS * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(df, feats, (size_t)n * F * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(dl, labels, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
  k_alpha_train<<<1, 256>>>(dm, df, dl, n, epochs, lr, sc, ms, vs, lh);
  if (cudaGetLastError() != cudaSuccess) return BLTT_ERR_CUDA;
  if (cudaMemcpy(model, dm, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BLTT_ERR_CUDA;
  if (loss_hist && epochs > 0)
    cudaMemcpy(loss_hist, lh, epochs * sizeof(float), cudaMemcpyDeviceToHost);
  return BLTT_OK;
}

bltt_status bltt_alpha_predict(const float* model, const float* feats, int n, float* alpha_out) {
  if (!model || !feats || n < 1 || !alpha_out) return BLTT_ERR_INVALID_ARG;
  if (!check_model(model)) return BLTT_ERR_INVALID_ARG;
  DevBuf db;
  float* dm = db.get<float>(MODEL_FLOATS);
  float* df = db.get<float>((size_t)n * F);
  float* da = db.get<float>(n);
  if (!dm || !df || !da) return BLTT_ERR_OOM;
  cudaMemcpy(dm, model, MODEL_FLOATS * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(df, feats, (size_t)n * F * sizeof(float), cudaMemcpyHostToDevice);
  k_alpha_predict<<<(n + 255) / 256, 256>>>(dm, df, n, da);
  if (cudaGetLastError() != cudaSuccess) return BLTT_ERR_CUDA;
  if (cudaMemcpy(alpha_out, da, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return BLTT_ERR_CUDA;
  return BLTT_OK;
}

}  // extern "C"
