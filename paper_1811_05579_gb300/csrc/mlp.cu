// Learned initial guess of the per-cell Newton solve: a small MLP
//   6 inputs -> 64 GELU -> 64 GELU -> 64 GELU -> 1
// with BF16 weights and FP32 accumulation, and its training (forward, backward,
// Adam) on the GPU.  The paper has no learned component: the network only supplies
// the starting point of the scalar Newton iteration of Eq. Tnp1, which still
// converges to the same root (see k_newton in grte1d.cu).
//
// Parameter vector (FP32 master copy, n = 8833):
//   W1[64][6], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[64], b4
// Inputs are the raw features f (log10 T^n, log10 rho*, log10 sigma_eff, log10 eps,
// log10 dt, log10 Cv), standardised with (f - mean)/std; the network predicts the
// standardised target (y - ymean)/ystd, y = log10(T^{n+1}/T^n).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/grte.h"
#include "mlp.cuh"

namespace grte {

constexpr int kIn = GRTE_MLP_IN, kH = GRTE_MLP_HIDDEN;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kH * kH, oW4 = oB3 + kH, oB4 = oW4 + kH, kNP = oB4 + 1;
static_assert(kNP == GRTE_MLP_NPARAMS, "parameter count");

// GELU (tanh form) and its derivative
__device__ __forceinline__ float gelu(float z) {
  const float k = 0.7978845608028654f, c = 0.044715f;
  return 0.5f * z * (1.0f + tanhf(k * (z + c * z * z * z)));
}
__device__ __forceinline__ float gelu_d(float z) {
  const float k = 0.7978845608028654f, c = 0.044715f;
  const float u = k * (z + c * z * z * z);
  const float t = tanhf(u);
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * k * (1.0f + 3.0f * c * z * z);
}

// Forward pass of one sample with weights in shared memory (BF16) and activations in
// a per-thread shared-memory row; returns the standardised output.  z1..z3 keep the
// pre-activations when `keep` is set (for the backward pass).
__device__ float mlp_forward(const __nv_bfloat16* __restrict__ w, const float* __restrict__ xin, float* z1,
                             float* z2, float* z3, float* h1, float* h2, float* h3) {
  for (int j = 0; j < kH; ++j) {
    float acc = __bfloat162float(w[oB1 + j]);
#pragma unroll
    for (int i = 0; i < kIn; ++i) acc += __bfloat162float(w[oW1 + j * kIn + i]) * xin[i];
    z1[j] = acc;
    h1[j] = gelu(acc);
  }
  for (int j = 0; j < kH; ++j) {
    float acc = __bfloat162float(w[oB2 + j]);
    for (int i = 0; i < kH; ++i) acc += __bfloat162float(w[oW2 + j * kH + i]) * h1[i];
    z2[j] = acc;
    h2[j] = gelu(acc);
  }
  for (int j = 0; j < kH; ++j) {
    float acc = __bfloat162float(w[oB3 + j]);
    for (int i = 0; i < kH; ++i) acc += __bfloat162float(w[oW3 + j * kH + i]) * h2[i];
    z3[j] = acc;
    h3[j] = gelu(acc);
  }
  float out = __bfloat162float(w[oB4]);
  for (int i = 0; i < kH; ++i) out += __bfloat162float(w[oW4 + i]) * h3[i];
  return out;
}

constexpr int kMlpThreads = 64;   // samples per block (activations live in shared memory)

struct MlpScratch {
  float z1[kH], z2[kH], z3[kH], h1[kH], h2[kH], h3[kH], x[kIn];
};

__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Forward and (MODE 1) backward of a batch: per-block partial gradients (sum over the
// block's samples of d(loss)/d(param), loss = mean of squared standardised errors)
// are written to part[blockIdx.x][kNP]; MODE 0 writes predictions.  Every lane runs
// the same loops (lanes past n contribute zero), so each gradient contribution is
// summed over the warp by shuffles before one shared-memory atomic per warp.
template <int MODE>
__global__ void __launch_bounds__(kMlpThreads) k_mlp(const __nv_bfloat16* __restrict__ wts, const float* __restrict__ X,
                                                     const float* __restrict__ Y, int64_t n, const float* __restrict__ norm,
                                                     float* __restrict__ out, float* __restrict__ part,
                                                     float* __restrict__ loss_part, float scale) {
  extern __shared__ unsigned char smem_raw[];
  __nv_bfloat16* w = (__nv_bfloat16*)smem_raw;
  float* g = (float*)(smem_raw + ((kNP * 2 + 15) / 16) * 16);
  MlpScratch* scr = (MlpScratch*)(g + (MODE == 1 ? kNP : 0));
  __shared__ float lsum[kMlpThreads];
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) {
    w[i] = wts[i];
    if (MODE == 1) g[i] = 0.0f;
  }
  __syncthreads();
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = s < n;
  const int lane = threadIdx.x & 31;
  MlpScratch& S = scr[threadIdx.x];
  for (int i = 0; i < kIn; ++i) S.x[i] = valid ? (X[s * kIn + i] - norm[i]) / norm[kIn + i] : 0.0f;
  const float o = mlp_forward(w, S.x, S.z1, S.z2, S.z3, S.h1, S.h2, S.h3);
  if (MODE == 0) {
    if (valid) out[s] = o * norm[2 * kIn + 1] + norm[2 * kIn];   // un-standardised prediction
    return;
  }
  const float t = valid ? (Y[s] - norm[2 * kIn]) / norm[2 * kIn + 1] : 0.0f;
  const float d4 = valid ? 2.0f * (o - t) * scale : 0.0f;      // d loss / d out
  const float err2 = valid ? (o - t) * (o - t) : 0.0f;
  auto acc = [&](int idx, float c) {
    c = warp_sum(c);
    if (lane == 0) atomicAdd(&g[idx], c);
  };
  acc(oB4, d4);
  for (int i = 0; i < kH; ++i) {
    acc(oW4 + i, d4 * S.h3[i]);
    S.z3[i] = d4 * __bfloat162float(w[oW4 + i]) * gelu_d(S.z3[i]);   // delta3
  }
  for (int j = 0; j < kH; ++j) {
    const float d3 = S.z3[j];
    acc(oB3 + j, d3);
    for (int i = 0; i < kH; ++i) acc(oW3 + j * kH + i, d3 * S.h2[i]);
  }
  for (int i = 0; i < kH; ++i) {
    float a = 0.0f;
    for (int j = 0; j < kH; ++j) a += __bfloat162float(w[oW3 + j * kH + i]) * S.z3[j];
    S.h3[i] = a * gelu_d(S.z2[i]);                                    // delta2
  }
  for (int j = 0; j < kH; ++j) {
    const float d2 = S.h3[j];
    acc(oB2 + j, d2);
    for (int i = 0; i < kH; ++i) acc(oW2 + j * kH + i, d2 * S.h1[i]);
  }
  for (int i = 0; i < kH; ++i) {
    float a = 0.0f;
    for (int j = 0; j < kH; ++j) a += __bfloat162float(w[oW2 + j * kH + i]) * S.h3[j];
    S.z2[i] = a * gelu_d(S.z1[i]);                                    // delta1
  }
  for (int j = 0; j < kH; ++j) {
    const float d1 = S.z2[j];
    acc(oB1 + j, d1);
    for (int i = 0; i < kIn; ++i) acc(oW1 + j * kIn + i, d1 * S.x[i]);
  }
  lsum[threadIdx.x] = err2;
  __syncthreads();
  for (int i = threadIdx.x; i < kNP; i += blockDim.x) part[(int64_t)blockIdx.x * kNP + i] = g[i];
  if (threadIdx.x == 0) {
    float tt = 0.0f;
    for (int i = 0; i < kMlpThreads; ++i) tt += lsum[i];
    loss_part[blockIdx.x] = tt;
  }
}

// Sum the per-block partial gradients (fixed order) into grad.
__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk, float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNP) return;
  float t = 0.0f;
  for (int b = 0; b < nblk; ++b) t += part[(int64_t)b * kNP + i];
  grad[i] = t;
}

// Adam on the FP32 master copy, then the BF16 working copy.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, float lr, float b1, float b2,
                       float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNP) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  p[i] = pi;
  wb[i] = __float2bfloat16(pi);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kNP) wb[i] = __float2bfloat16(p[i]);
}

size_t mlp_smem_bytes(int mode) {
  return ((kNP * 2 + 15) / 16) * 16 + (mode == 1 ? kNP * sizeof(float) : 0) + kMlpThreads * sizeof(MlpScratch);
}

}  // namespace grte

using namespace grte;

struct grte_mlp {
  float* p = nullptr;        // FP32 master parameters
  float* m = nullptr;
  float* v = nullptr;
  float* g = nullptr;
  __nv_bfloat16* wb = nullptr;
  float* norm = nullptr;     // mean[6], std[6], ymean, ystd
  float hnorm[2 * kIn + 2];
  int64_t adam_t = 0;
  std::string err;
};

static grte_status mfail(grte_mlp_t h, grte_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}
#define MCK(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) return mfail(h, GRTE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace grte {
cudaError_t mlp_guess_launch(grte_mlp_t h, const float* feat, int64_t n, float* y, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int nb = (int)((n + kMlpThreads - 1) / kMlpThreads);
  k_mlp<0><<<nb, kMlpThreads, mlp_smem_bytes(0), stream>>>(h->wb, feat, nullptr, n, h->norm, y, nullptr, nullptr,
                                                            0.0f);
  return cudaGetLastError();
}
}  // namespace grte

extern "C" {

grte_status grte_mlp_create(uint64_t seed, grte_mlp_t* out) {
  if (!out) return GRTE_EINVAL;
  grte_mlp_t h = new (std::nothrow) grte_mlp();
  if (!h) return GRTE_ENOMEM;
  *out = h;
  MCK(cudaMalloc(&h->p, sizeof(float) * kNP));
  MCK(cudaMalloc(&h->m, sizeof(float) * kNP));
  MCK(cudaMalloc(&h->v, sizeof(float) * kNP));
  MCK(cudaMalloc(&h->g, sizeof(float) * kNP));
  MCK(cudaMalloc(&h->wb, sizeof(__nv_bfloat16) * kNP));
  MCK(cudaMalloc(&h->norm, sizeof(float) * (2 * kIn + 2)));
  // He-normal weights, zero biases (seeded, host-side)
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.0f, 1.0f);
  std::vector<float> p(kNP, 0.0f);
  auto fill = [&](int off, int fan_out, int fan_in) {
    const float sd = std::sqrt(2.0f / fan_in);
    for (int i = 0; i < fan_out * fan_in; ++i) p[off + i] = sd * nd(rng);
  };
  fill(oW1, kH, kIn);
  fill(oW2, kH, kH);
  fill(oW3, kH, kH);
  fill(oW4, 1, kH);
  MCK(cudaMemcpy(h->p, p.data(), sizeof(float) * kNP, cudaMemcpyHostToDevice));
  MCK(cudaMemset(h->m, 0, sizeof(float) * kNP));
  MCK(cudaMemset(h->v, 0, sizeof(float) * kNP));
  k_to_bf16<<<(kNP + 255) / 256, 256>>>(h->p, h->wb);
  MCK(cudaGetLastError());
  for (int i = 0; i < kIn; ++i) {
    h->hnorm[i] = 0.0f;
    h->hnorm[kIn + i] = 1.0f;
  }
  h->hnorm[2 * kIn] = 0.0f;
  h->hnorm[2 * kIn + 1] = 1.0f;
  MCK(cudaMemcpy(h->norm, h->hnorm, sizeof(h->hnorm), cudaMemcpyHostToDevice));
  MCK(cudaFuncSetAttribute(k_mlp<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes(0)));
  MCK(cudaFuncSetAttribute(k_mlp<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes(1)));
  return GRTE_OK;
}

void grte_mlp_destroy(grte_mlp_t h) {
  if (!h) return;
  cudaDeviceSynchronize();
  cudaFree(h->p); cudaFree(h->m); cudaFree(h->v); cudaFree(h->g); cudaFree(h->wb); cudaFree(h->norm);
  delete h;
}

const char* grte_mlp_last_error(grte_mlp_t h) { return h ? h->err.c_str() : "null handle"; }

grte_status grte_mlp_set_norm(grte_mlp_t h, const float* mean_in, const float* std_in, float mean_out, float std_out) {
  if (!h || !mean_in || !std_in) return GRTE_EINVAL;
  for (int i = 0; i < kIn; ++i) {
    if (!(std_in[i] > 0.0f)) return mfail(h, GRTE_EINVAL, "std must be > 0");
    h->hnorm[i] = mean_in[i];
    h->hnorm[kIn + i] = std_in[i];
  }
  if (!(std_out > 0.0f)) return mfail(h, GRTE_EINVAL, "std must be > 0");
  h->hnorm[2 * kIn] = mean_out;
  h->hnorm[2 * kIn + 1] = std_out;
  MCK(cudaMemcpy(h->norm, h->hnorm, sizeof(h->hnorm), cudaMemcpyHostToDevice));
  return GRTE_OK;
}

grte_status grte_mlp_get_params(grte_mlp_t h, float* p, size_t n) {
  if (!h || !p || n != (size_t)kNP) return GRTE_EINVAL;
  MCK(cudaMemcpy(p, h->p, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
  return GRTE_OK;
}

grte_status grte_mlp_set_params(grte_mlp_t h, const float* p, size_t n) {
  if (!h || !p || n != (size_t)kNP) return GRTE_EINVAL;
  MCK(cudaMemcpy(h->p, p, sizeof(float) * kNP, cudaMemcpyHostToDevice));
  k_to_bf16<<<(kNP + 255) / 256, 256>>>(h->p, h->wb);
  MCK(cudaGetLastError());
  MCK(cudaDeviceSynchronize());
  return GRTE_OK;
}

// Predictions y (un-standardised) of n raw feature rows X (host arrays).
grte_status grte_mlp_forward(grte_mlp_t h, const float* X, int64_t n, float* y) {
  if (!h || !X || !y || n <= 0) return GRTE_EINVAL;
  float *dX = nullptr, *dY = nullptr;
  MCK(cudaMalloc(&dX, sizeof(float) * n * kIn));
  MCK(cudaMalloc(&dY, sizeof(float) * n));
  MCK(cudaMemcpy(dX, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice));
  const int nb = (int)((n + kMlpThreads - 1) / kMlpThreads);
  k_mlp<0><<<nb, kMlpThreads, mlp_smem_bytes(0)>>>(h->wb, dX, nullptr, n, h->norm, dY, nullptr, nullptr, 0.0f);
  MCK(cudaGetLastError());
  MCK(cudaMemcpy(y, dY, sizeof(float) * n, cudaMemcpyDeviceToHost));
  cudaFree(dX);
  cudaFree(dY);
  return GRTE_OK;
}

static grte_status grad_batch(grte_mlp_t h, const float* dX, const float* dY, int64_t n, float* dpart,
                              float* dlpart, float* loss) {
  const int nb = (int)((n + kMlpThreads - 1) / kMlpThreads);
  k_mlp<1><<<nb, kMlpThreads, mlp_smem_bytes(1)>>>(h->wb, dX, dY, n, h->norm, nullptr, dpart, dlpart,
                                                    1.0f / (float)n);
  MCK(cudaGetLastError());
  k_mlp_reduce<<<(kNP + 255) / 256, 256>>>(dpart, nb, h->g);
  MCK(cudaGetLastError());
  if (loss) {
    std::vector<float> lp(nb);
    MCK(cudaMemcpy(lp.data(), dlpart, sizeof(float) * nb, cudaMemcpyDeviceToHost));
    double t = 0.0;
    for (float v : lp) t += v;
    *loss = (float)(t / n);
  }
  return GRTE_OK;
}

// Gradient of the mean squared standardised error over n samples (host arrays), at
// the current BF16 weights: for checking the backward pass.
grte_status grte_mlp_grad(grte_mlp_t h, const float* X, const float* Y, int64_t n, float* grad, size_t ng,
                          float* loss) {
  if (!h || !X || !Y || !grad || n <= 0 || ng != (size_t)kNP) return GRTE_EINVAL;
  float *dX, *dY, *dpart, *dl;
  const int nb = (int)((n + kMlpThreads - 1) / kMlpThreads);
  MCK(cudaMalloc(&dX, sizeof(float) * n * kIn));
  MCK(cudaMalloc(&dY, sizeof(float) * n));
  MCK(cudaMalloc(&dpart, sizeof(float) * (size_t)nb * kNP));
  MCK(cudaMalloc(&dl, sizeof(float) * nb));
  MCK(cudaMemcpy(dX, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice));
  MCK(cudaMemcpy(dY, Y, sizeof(float) * n, cudaMemcpyHostToDevice));
  grte_status s = grad_batch(h, dX, dY, n, dpart, dl, loss);
  if (s == GRTE_OK) {
    MCK(cudaMemcpy(grad, h->g, sizeof(float) * kNP, cudaMemcpyDeviceToHost));
  }
  cudaFree(dX); cudaFree(dY); cudaFree(dpart); cudaFree(dl);
  return s;
}

// Adam training: `epochs` passes over n samples (host arrays) in mini-batches of
// `batch` (the sample order is a seeded shuffle per epoch); loss = last epoch's mean.
grte_status grte_mlp_train(grte_mlp_t h, const float* X, const float* Y, int64_t n, int epochs, int batch, float lr,
                           uint64_t seed, float* loss) {
  if (!h || !X || !Y || n <= 0 || epochs <= 0 || batch <= 0 || !(lr > 0)) return GRTE_EINVAL;
  std::vector<float> xs((size_t)n * kIn), ys(n);
  std::vector<int64_t> idx(n);
  for (int64_t i = 0; i < n; ++i) idx[i] = i;
  float *dX, *dY, *dpart, *dl;
  const int nbmax = (batch + kMlpThreads - 1) / kMlpThreads;
  MCK(cudaMalloc(&dX, sizeof(float) * n * kIn));
  MCK(cudaMalloc(&dY, sizeof(float) * n));
  MCK(cudaMalloc(&dpart, sizeof(float) * (size_t)nbmax * kNP));
  MCK(cudaMalloc(&dl, sizeof(float) * nbmax));
  std::mt19937_64 rng(seed);
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(idx.begin(), idx.end(), rng);
    for (int64_t i = 0; i < n; ++i) {
      std::memcpy(&xs[i * kIn], &X[idx[i] * kIn], sizeof(float) * kIn);
      ys[i] = Y[idx[i]];
    }
    MCK(cudaMemcpy(dX, xs.data(), sizeof(float) * n * kIn, cudaMemcpyHostToDevice));
    MCK(cudaMemcpy(dY, ys.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    double esum = 0.0;
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int64_t nb = std::min<int64_t>(batch, n - b0);
      float l = 0.0f;
      grte_status s = grad_batch(h, dX + b0 * kIn, dY + b0, nb, dpart, dl, ep == epochs - 1 ? &l : nullptr);
      if (s != GRTE_OK) return s;
      esum += (double)l * nb;
      ++h->adam_t;
      const float b1 = 0.9f, b2 = 0.999f;
      const float bc1 = 1.0f - std::pow(b1, (float)h->adam_t), bc2 = 1.0f - std::pow(b2, (float)h->adam_t);
      k_adam<<<(kNP + 255) / 256, 256>>>(h->p, h->m, h->v, h->g, h->wb, lr, b1, b2, 1e-8f, bc1, bc2);
      MCK(cudaGetLastError());
    }
    last = esum / n;
  }
  MCK(cudaDeviceSynchronize());
  cudaFree(dX); cudaFree(dY); cudaFree(dpart); cudaFree(dl);
  if (loss) *loss = (float)last;
  return GRTE_OK;
}

}  // extern "C"
