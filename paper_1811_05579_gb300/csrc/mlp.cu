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

// ----------------------------------------------------------------------------- tensor cores
// The 64-wide layers, their backward deltas and the weight gradients run on the tensor
// cores: mma.sync m16n8k16, BF16 operands, FP32 accumulation.  The network is "BF16 in,
// FP32 accumulate": the operands of every matrix product are BF16 (the weights, the
// standardised inputs, the activations h1, h2 and the deltas of layers 3, 2, 1 at the
// points where they enter a product); pre-activations, GELU, the output layer, the
// bias gradients and the loss stay FP32.
constexpr int kMlpSamples = 64;            // samples per block
constexpr int kMlpThreads = 128;           // 4 warps, 16 samples each
constexpr int kLd = kH + 8;                // padded row of a BF16 activation tile
constexpr int kLdX = 16 + 8;               // padded row of the input tile (6 used, K = 16)

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A B + D for one 16x16 (A, row-major) x 16x8 (B, column-major) tile
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragments of the m16n8k16 shape from element accessors A(row, k) and B(k, col)
// (lane = 4 g + q: A rows g, g + 8 and k = 2q, 2q + 1, 2q + 8, 2q + 9; B k the same,
// column g; C rows g, g + 8 and columns 2q, 2q + 1).
template <class FA>
__device__ __forceinline__ void frag_a(uint32_t a[4], int lane, FA A) {
  const int g = lane >> 2, q = lane & 3;
  a[0] = pack2(A(g, 2 * q), A(g, 2 * q + 1));
  a[1] = pack2(A(g + 8, 2 * q), A(g + 8, 2 * q + 1));
  a[2] = pack2(A(g, 2 * q + 8), A(g, 2 * q + 9));
  a[3] = pack2(A(g + 8, 2 * q + 8), A(g + 8, 2 * q + 9));
}
template <class FB>
__device__ __forceinline__ void frag_b(uint32_t b[2], int lane, FB B) {
  const int g = lane >> 2, q = lane & 3;
  b[0] = pack2(B(2 * q, g), B(2 * q + 1, g));
  b[1] = pack2(B(2 * q + 8, g), B(2 * q + 9, g));
}

struct MlpTile {   // shared memory of one block
  __nv_bfloat16 w[((kNP + 7) / 8) * 8];    // the BF16 parameter vector
  __nv_bfloat16 w1p[kH][16];               // W1 with K padded 6 -> 16
  __nv_bfloat16 xs[kMlpSamples][kLdX];      // standardised inputs (BF16)
  __nv_bfloat16 h1[kMlpSamples][kLd], h2[kMlpSamples][kLd];
  __nv_bfloat16 d3[kMlpSamples][kLd], d2[kMlpSamples][kLd], d1[kMlpSamples][kLd];
  float z1[kMlpSamples][kH], z2[kMlpSamples][kH], z3[kMlpSamples][kH];   // pre-activations, then deltas
  float d4[kMlpSamples], err2[kMlpSamples];
  float g[kNP];                             // block gradient (MODE 1)
};

// Forward and (MODE 1) backward of 64 samples per block: MODE 0 writes predictions;
// MODE 1 writes the block's gradient (sum over its samples of d(loss)/d(param), loss =
// mean of squared standardised errors, `scale` = 1/n) to part[blockIdx.x][kNP] and its
// summed squared error to loss_part.  Samples past n enter with zero inputs and zero
// output gradient.
template <int MODE>
__global__ void __launch_bounds__(kMlpThreads) k_mlp(const __nv_bfloat16* __restrict__ wts, const float* __restrict__ X,
                                                     const float* __restrict__ Y, int64_t n, const float* __restrict__ norm,
                                                     float* __restrict__ out, float* __restrict__ part,
                                                     float* __restrict__ loss_part, float scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpTile& S = *reinterpret_cast<MlpTile*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int g8 = lane >> 2, q = lane & 3;
  const int64_t s0 = (int64_t)blockIdx.x * kMlpSamples;
  for (int i = tid; i < kNP; i += kMlpThreads) {
    S.w[i] = wts[i];
    if (MODE == 1) S.g[i] = 0.0f;
  }
  for (int i = tid; i < kH * 16; i += kMlpThreads) {
    const int j = i / 16, k = i % 16;
    S.w1p[j][k] = k < kIn ? wts[oW1 + j * kIn + k] : __float2bfloat16(0.0f);
  }
  for (int i = tid; i < kMlpSamples * 16; i += kMlpThreads) {
    const int r = i / 16, k = i % 16;
    const int64_t s = s0 + r;
    float v = 0.0f;
    if (k < kIn && s < n) v = (X[s * kIn + k] - norm[k]) / norm[kIn + k];
    S.xs[r][k] = __float2bfloat16(v);
  }
  __syncthreads();
  const __nv_bfloat16* W = S.w;
  const int r0 = wp * 16;   // this warp's samples
  auto bias = [&](int off, int col) { return __bfloat162float(W[off + col]); };
  // ---- layer 1: Z1 = X W1^T + b1 (K = 16, inputs padded)
  {
    uint32_t a[4];
    frag_a(a, lane, [&](int r, int k) { return S.xs[r0 + r][k]; });
    for (int nt = 0; nt < kH / 8; ++nt) {
      const int c0 = nt * 8 + 2 * q;
      float c[4] = {bias(oB1, c0), bias(oB1, c0 + 1), bias(oB1, c0), bias(oB1, c0 + 1)};
      uint32_t b[2];
      frag_b(b, lane, [&](int k, int col) { return S.w1p[nt * 8 + col][k]; });
      mma16816(c, a, b);
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + g8 + (e >> 1) * 8, col = c0 + (e & 1);
        S.z1[r][col] = c[e];
        S.h1[r][col] = __float2bfloat16(gelu(c[e]));
      }
    }
  }
  __syncwarp();
  // ---- layers 2 and 3: Z = H W^T + b (K = 64)
  auto dense = [&](const __nv_bfloat16 (*H)[kLd], int oW, int oB, float (*Z)[kH], __nv_bfloat16 (*Hn)[kLd],
                   float h3[kH / 8][4]) {
    uint32_t a[4][4];
    for (int kt = 0; kt < 4; ++kt) frag_a(a[kt], lane, [&](int r, int k) { return H[r0 + r][kt * 16 + k]; });
    for (int nt = 0; nt < kH / 8; ++nt) {
      const int c0 = nt * 8 + 2 * q;
      float c[4] = {bias(oB, c0), bias(oB, c0 + 1), bias(oB, c0), bias(oB, c0 + 1)};
      for (int kt = 0; kt < 4; ++kt) {
        uint32_t b[2];
        frag_b(b, lane, [&](int k, int col) { return W[oW + (nt * 8 + col) * kH + kt * 16 + k]; });
        mma16816(c, a[kt], b);
      }
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + g8 + (e >> 1) * 8, col = c0 + (e & 1);
        Z[r][col] = c[e];
        const float hv = gelu(c[e]);
        if (Hn) Hn[r][col] = __float2bfloat16(hv);
        if (h3) h3[nt][e] = hv;
      }
    }
    __syncwarp();
  };
  float h3[kH / 8][4];
  dense(S.h1, oW2, oB2, S.z2, S.h2, nullptr);
  dense(S.h2, oW3, oB3, S.z3, nullptr, h3);
  // ---- output: W4 . h3 + b4 (FP32), rows g and g + 8 of the warp's tile
  float o[2] = {0.0f, 0.0f};
  for (int nt = 0; nt < kH / 8; ++nt)
    for (int e = 0; e < 4; ++e) o[e >> 1] += __bfloat162float(W[oW4 + nt * 8 + 2 * q + (e & 1)]) * h3[nt][e];
  for (int hh = 0; hh < 2; ++hh) {
    o[hh] += __shfl_xor_sync(0xffffffffu, o[hh], 1);
    o[hh] += __shfl_xor_sync(0xffffffffu, o[hh], 2);
    o[hh] += __bfloat162float(W[oB4]);
  }
  if (MODE == 0) {
    if (q == 0)
      for (int hh = 0; hh < 2; ++hh) {
        const int64_t s = s0 + r0 + g8 + hh * 8;
        if (s < n) out[s] = o[hh] * norm[2 * kIn + 1] + norm[2 * kIn];   // un-standardised prediction
      }
    return;
  }
  // ---- backward
  float d4r[2];
  for (int hh = 0; hh < 2; ++hh) {
    const int r = r0 + g8 + hh * 8;
    const int64_t s = s0 + r;
    const bool valid = s < n;
    const float t = valid ? (Y[s] - norm[2 * kIn]) / norm[2 * kIn + 1] : 0.0f;
    d4r[hh] = valid ? 2.0f * (o[hh] - t) * scale : 0.0f;      // d loss / d out
    if (q == 0) {
      S.d4[r] = d4r[hh];
      S.err2[r] = valid ? (o[hh] - t) * (o[hh] - t) : 0.0f;
    }
  }
  // dW4 = sum_s d4 h3 (FP32), delta3 = d4 W4 gelu'(z3)
  for (int nt = 0; nt < kH / 8; ++nt)
    for (int cc = 0; cc < 2; ++cc) {
      const int col = nt * 8 + 2 * q + cc;
      float v = d4r[0] * h3[nt][cc] + d4r[1] * h3[nt][2 + cc];
      for (int off = 4; off < 32; off <<= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (g8 == 0) atomicAdd(&S.g[oW4 + col], v);
      const float w4 = __bfloat162float(W[oW4 + col]);
      for (int hh = 0; hh < 2; ++hh) {
        const int r = r0 + g8 + hh * 8;
        const float dv = d4r[hh] * w4 * gelu_d(S.z3[r][col]);
        S.z3[r][col] = dv;                              // delta3 (FP32)
        S.d3[r][col] = __float2bfloat16(dv);            // its BF16 operand copy
      }
    }
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
    for (int r = 0; r < kMlpSamples; ++r) t += S.d4[r];
    S.g[oB4] = t;
  }
  // dW = delta^T H over the block's 64 samples (K = 64): warp wp owns output rows
  // j = 16 wp .. 16 wp + 15 and all 64 (or the 6 input) columns
  auto wgrad = [&](const __nv_bfloat16 (*Dl)[kLd], const __nv_bfloat16* Hin, int ldh, int ncols, int oW) {
    const int ntiles = (ncols + 7) / 8;
    float acc[kH / 8][4];
    for (int nt = 0; nt < ntiles; ++nt)
      for (int e = 0; e < 4; ++e) acc[nt][e] = 0.0f;
    for (int kt = 0; kt < kMlpSamples / 16; ++kt) {
      uint32_t a[4];
      frag_a(a, lane, [&](int r, int k) { return Dl[kt * 16 + k][r0 + r]; });
      for (int nt = 0; nt < ntiles; ++nt) {
        uint32_t b[2];
        frag_b(b, lane, [&](int k, int col) { return Hin[(kt * 16 + k) * ldh + nt * 8 + col]; });
        mma16816(acc[nt], a, b);
      }
    }
    for (int nt = 0; nt < ntiles; ++nt)
      for (int e = 0; e < 4; ++e) {
        const int j = r0 + g8 + (e >> 1) * 8, i = nt * 8 + 2 * q + (e & 1);
        if (i < ncols) S.g[oW + j * ncols + i] = acc[nt][e];
      }
  };
  // delta_prev = (delta W) gelu'(z_prev) for the warp's 16 samples (K = 64)
  auto dprop = [&](const __nv_bfloat16 (*Dl)[kLd], int oW, float (*Z)[kH], __nv_bfloat16 (*Dn)[kLd]) {
    uint32_t a[4][4];
    for (int kt = 0; kt < 4; ++kt) frag_a(a[kt], lane, [&](int r, int k) { return Dl[r0 + r][kt * 16 + k]; });
    for (int nt = 0; nt < kH / 8; ++nt) {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int kt = 0; kt < 4; ++kt) {
        uint32_t b[2];
        frag_b(b, lane, [&](int k, int col) { return W[oW + (kt * 16 + k) * kH + nt * 8 + col]; });
        mma16816(c, a[kt], b);
      }
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + g8 + (e >> 1) * 8, col = nt * 8 + 2 * q + (e & 1);
        const float dv = c[e] * gelu_d(Z[r][col]);
        Z[r][col] = dv;
        Dn[r][col] = __float2bfloat16(dv);
      }
    }
  };
  auto bgrad = [&](float (*Dz)[kH], int oB) {   // bias gradient: column sums of the FP32 deltas
    if (tid < kH) {
      float t = 0.0f;
      for (int r = 0; r < kMlpSamples; ++r) t += Dz[r][tid];
      S.g[oB + tid] = t;
    }
  };
  wgrad(S.d3, &S.h2[0][0], kLd, kH, oW3);
  bgrad(S.z3, oB3);
  dprop(S.d3, oW3, S.z2, S.d2);
  __syncthreads();
  wgrad(S.d2, &S.h1[0][0], kLd, kH, oW2);
  bgrad(S.z2, oB2);
  dprop(S.d2, oW2, S.z1, S.d1);
  __syncthreads();
  wgrad(S.d1, &S.xs[0][0], kLdX, kIn, oW1);
  bgrad(S.z1, oB1);
  __syncthreads();
  for (int i = tid; i < kNP; i += kMlpThreads) part[(int64_t)blockIdx.x * kNP + i] = S.g[i];
  if (tid == 0) {
    float tt = 0.0f;
    for (int i = 0; i < kMlpSamples; ++i) tt += S.err2[i];
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

size_t mlp_smem_bytes(int) { return sizeof(MlpTile); }

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
  const int nb = (int)((n + kMlpSamples - 1) / kMlpSamples);
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

// Predictions y (un-standardised) of n raw feature rows X, both device arrays, on
// `stream` (NULL: the legacy default stream); asynchronous.
grte_status grte_mlp_forward_device(grte_mlp_t h, const float* X, int64_t n, float* y, void* stream) {
  if (!h || !X || !y || n <= 0) return GRTE_EINVAL;
  MCK(mlp_guess_launch(h, X, n, y, (cudaStream_t)stream));
  return GRTE_OK;
}

// Predictions y (un-standardised) of n raw feature rows X (host arrays).
grte_status grte_mlp_forward(grte_mlp_t h, const float* X, int64_t n, float* y) {
  if (!h || !X || !y || n <= 0) return GRTE_EINVAL;
  float *dX = nullptr, *dY = nullptr;
  MCK(cudaMalloc(&dX, sizeof(float) * n * kIn));
  MCK(cudaMalloc(&dY, sizeof(float) * n));
  MCK(cudaMemcpy(dX, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice));
  const int nb = (int)((n + kMlpSamples - 1) / kMlpSamples);
  k_mlp<0><<<nb, kMlpThreads, mlp_smem_bytes(0)>>>(h->wb, dX, nullptr, n, h->norm, dY, nullptr, nullptr, 0.0f);
  MCK(cudaGetLastError());
  MCK(cudaMemcpy(y, dY, sizeof(float) * n, cudaMemcpyDeviceToHost));
  cudaFree(dX);
  cudaFree(dY);
  return GRTE_OK;
}

static grte_status grad_batch(grte_mlp_t h, const float* dX, const float* dY, int64_t n, float* dpart,
                              float* dlpart, float* loss) {
  const int nb = (int)((n + kMlpSamples - 1) / kMlpSamples);
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
  const int nb = (int)((n + kMlpSamples - 1) / kMlpSamples);
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
  const int nbmax = (batch + kMlpSamples - 1) / kMlpSamples;
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
