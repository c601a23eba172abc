// diff1d.cu - the three-stage diffusion solver of Sec. 2 on the GPU (sm_103a), batched
// over independent 1D instances; FP64.
//
// One step (Eq. limit_U_dis1 - Eq. limit_UT_dis3, fully discrete as Eq. dis-diff; for
// sigma_0/T^3 the fully discrete form after Eq. marshak-diff2):
//   stage 1 (prediction)  (U*_j - U_j)/dt = f_j [k_{j+1} (U*_{j+1} - U*_j) - k_j (U*_j - U*_{j-1})],
//                         f = 4T^3/(4aT^3 + C_v), k_i = a c kappa_i / (D sigma_i dx^2) at node i,
//                         kappa_i = 1 (sigma(x)) or the node mean of T^3 (sigma_0/T^3),
//                         sigma_i the harmonic node mean, k = 0 at the two walls (zero flux):
//                         one tridiagonal solve per instance;
//   stage 2 (correction)  a (T^4 - T_n^4)/dt + C_v (T - T_n)/dt = k*_{j+1} (U*_{j+1} - U*_j) - k*_j (U*_j - U*_{j-1}),
//                         k* with kappa* = the node mean of max(U*, 0)^{3/4} (sigma_0/T^3) or k:
//                         a per-cell quartic, solved by monotone Newton;
//   stage 3 (projection)  U = T^4.
// Kernels: k_dcoef (per cell: U, f, node k), k_dsolve (one CTA per instance: the
// partitioned tridiagonal solver of tridiag.cuh, unknowns in global memory), k_dcorr (per
// cell: the correction's flux and Newton).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "../../include/grte.h"
#include "tridiag.cuh"

namespace grte {
namespace {

constexpr int kDT = 256;   // threads per solve CTA

struct DInst {
  int64_t N, off;          // cells, offset into the cell arrays
  int64_t foff, roff;      // factor / reduced-system offsets
  double dt, dx, a, c, Cv, Dd;
  int kind;
};

struct DDev {
  const DInst* inst;
  double *sig, *T, *U, *f, *k, *Us, *x, *F, *Rd;
  int* status;
};

__device__ __forceinline__ int inst_of(const DInst* in, int n, int64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (in[mid].off <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// per cell: U = T^4, f = 4T^3/(4aT^3 + Cv), k at the cell's left node (0 at the wall)
__global__ void k_dcoef(DDev D, int n_inst, int64_t ncell) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const DInst I = D.inst[inst_of(D.inst, n_inst, g)];
  const int64_t j = g - I.off;
  const double T = D.T[g], T3 = T * T * T;
  D.U[g] = T3 * T;
  D.f[g] = 4.0 * T3 / (4.0 * I.a * T3 + I.Cv);
  double k = 0.0;
  if (j >= 1) {
    const double sl = D.sig[g - 1], sr = D.sig[g];
    const double sn = 2.0 * sl * sr / (sl + sr);
    double kap = 1.0;
    if (I.kind == GRTE_SIGMA_T3) {
      const double Tl = D.T[g - 1];
      kap = 0.5 * (Tl * Tl * Tl + T3);
    }
    k = I.a * I.c * kap / (I.Dd * sn * I.dx * I.dx);
  }
  D.k[g] = k;
  D.x[g] = D.U[g] / I.dt;   // right-hand side of stage 1
}

struct DCoef {   // stage-1 matrix of one instance
  const double *f, *k;
  double idt;
  int64_t N;
  __device__ double kr(int64_t j) const { return j + 1 < N ? k[j + 1] : 0.0; }
  __device__ double a(int64_t j) const { return j > 0 ? -f[j] * k[j] : 0.0; }
  __device__ double c(int64_t j) const { return j + 1 < N ? -f[j] * k[j + 1] : 0.0; }
  __device__ double b(int64_t j) const { return idt + f[j] * (k[j] + kr(j)); }
};

__global__ void __launch_bounds__(kDT) k_dsolve(DDev D) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const DInst I = D.inst[blockIdx.x];
  DCoef cf{D.f + I.off, D.k + I.off, 1.0 / I.dt, I.N};
  XAcc<double, false> xa{D.x + I.off};
  tri_solve<true>(cf, I.N, xa, D.F + I.foff, D.Rd + I.roff, (double*)dsm);
}

// per cell: the correction's flux at U*, then (a/dt) T^4 + (C_v/dt) T = (a/dt) U_n + (C_v/dt) T_n + flux
__global__ void k_dcorr(DDev D, int n_inst, int64_t ncell, int maxit) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= ncell) return;
  const int ii = inst_of(D.inst, n_inst, g);
  const DInst I = D.inst[ii];
  const int64_t j = g - I.off, N = I.N;
  const double* Us = D.x + I.off;   // the solution of stage 1
  auto knode = [&](int64_t i) -> double {   // k* at node i (cells i-1, i)
    if (i < 1 || i > N - 1) return 0.0;
    if (I.kind != GRTE_SIGMA_T3) return D.k[I.off + i];
    const double sl = D.sig[I.off + i - 1], sr = D.sig[I.off + i];
    const double sn = 2.0 * sl * sr / (sl + sr);
    const double kap = 0.5 * (pow(fmax(Us[i - 1], 0.0), 0.75) + pow(fmax(Us[i], 0.0), 0.75));
    return I.a * I.c * kap / (I.Dd * sn * I.dx * I.dx);
  };
  const double uj = Us[j];
  double flux = 0.0;
  if (j + 1 < N) flux += knode(j + 1) * (Us[j + 1] - uj);
  if (j >= 1) flux -= knode(j) * (uj - Us[j - 1]);
  D.Us[g] = uj;
  const double Tn = D.T[g];
  const double A = I.a / I.dt, B = I.Cv / I.dt;
  const double R = A * D.U[g] + B * Tn + flux;
  double t;
  if (!(R > 0.0)) {
    t = 0.0;
    if (R <= 0.0) atomicOr(D.status, 1 << GRTE_ENEGATIVE);
  } else {
    // monotone Newton from T_hi = min((R/A)^{1/4}, R/B) (convex increasing left side)
    t = fmin(sqrt(sqrt(R / A)), R / B);
    int it = 0;
    for (; it < maxit; ++it) {
      const double t2 = t * t;
      const double tn = t - (A * t2 * t2 + B * t - R) / (4.0 * A * t2 * t + B);
      if (!(tn < t)) break;
      t = tn;
    }
    if (it >= maxit) atomicOr(D.status, 1 << GRTE_ENONCONV);
  }
  if (!isfinite(t)) atomicOr(D.status, 1 << GRTE_ENAN);
  D.T[g] = t;
}

}  // namespace
}  // namespace grte

using namespace grte;

struct grte_diff_ctx {
  int n_inst = 0;
  int64_t ncell = 0;
  std::vector<DInst> inst;
  DDev D{};
  DInst* d_inst = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<void*> allocs;
  std::string err;
  int newton_maxit = 60;
};

static grte_status dfail(grte_diff_t h, grte_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}
#define DCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return dfail(h, GRTE_ECUDA, cudaGetErrorString(e_));    \
  } while (0)

template <typename T>
static bool dalloc_d(grte_diff_t h, T** p, int64_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * (size_t)std::max<int64_t>(n, 1)) != cudaSuccess) return false;
  h->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

extern "C" {

void grte_diff_destroy(grte_diff_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* grte_diff_last_error(grte_diff_t h) { return h ? h->err.c_str() : "null handle"; }

grte_status grte_diff_create(int n_inst, const grte_diffusion1d* in, void* stream, grte_diff_t* out) {
  if (!out) return GRTE_EINVAL;
  *out = nullptr;
  if (n_inst <= 0 || !in) return GRTE_EINVAL;
  grte_diff_t h = new (std::nothrow) grte_diff_ctx();
  if (!h) return GRTE_ENOMEM;
  *out = h;
  int64_t off = 0, foff = 0, roff = 0;
  for (int i = 0; i < n_inst; ++i) {
    const grte_diffusion1d& p = in[i];
    if (p.nx < 2 || p.nx > (1 << 24)) return dfail(h, GRTE_EINVAL, "nx must be in [2, 2^24]");
    if (!p.sigma) return dfail(h, GRTE_EINVAL, "sigma is NULL");
    if (p.sigma_kind != GRTE_SIGMA_CONST && p.sigma_kind != GRTE_SIGMA_T3) return dfail(h, GRTE_EINVAL, "bad sigma_kind");
    if (!(p.x1 > p.x0) || !(p.dt > 0) || !(p.a > 0) || !(p.c > 0) || !(p.Cv > 0))
      return dfail(h, GRTE_EINVAL, "x1 > x0, dt, a, c, Cv must be positive");
    for (int64_t j = 0; j < p.nx; ++j)
      if (!(p.sigma[j] > 0.0) || !std::isfinite(p.sigma[j])) return dfail(h, GRTE_EINVAL, "sigma must be positive");
    DInst I{};
    I.N = p.nx;
    I.off = off;
    I.foff = foff;
    I.roff = roff;
    I.dt = p.dt;
    I.dx = (p.x1 - p.x0) / (double)p.nx;
    I.a = p.a;
    I.c = p.c;
    I.Cv = p.Cv;
    I.Dd = p.dd > 0 ? p.dd : 3.0;
    I.kind = p.sigma_kind;
    h->inst.push_back(I);
    off += p.nx;
    foff += tri_fac_size(p.nx, kDT);
    roff += tri_red_size(p.nx, kDT);
  }
  h->n_inst = n_inst;
  h->ncell = off;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    DCK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  DDev& D = h->D;
  const int64_t nc = off;
  if (!(dalloc_d(h, &h->d_inst, n_inst) && dalloc_d(h, &D.sig, nc) && dalloc_d(h, &D.T, nc) &&
        dalloc_d(h, &D.U, nc) && dalloc_d(h, &D.f, nc) && dalloc_d(h, &D.k, nc) && dalloc_d(h, &D.Us, nc) &&
        dalloc_d(h, &D.x, nc) && dalloc_d(h, &D.F, foff) && dalloc_d(h, &D.Rd, roff) &&
        dalloc_d(h, &D.status, 1)))
    return dfail(h, GRTE_ENOMEM, "cudaMalloc failed");
  D.inst = h->d_inst;
  DCK(cudaMemcpyAsync(h->d_inst, h->inst.data(), sizeof(DInst) * n_inst, cudaMemcpyHostToDevice, h->stream));
  for (int i = 0; i < n_inst; ++i)
    DCK(cudaMemcpyAsync(D.sig + h->inst[i].off, in[i].sigma, sizeof(double) * in[i].nx, cudaMemcpyHostToDevice,
                        h->stream));
  DCK(cudaMemsetAsync(D.status, 0, sizeof(int), h->stream));
  DCK(cudaMemsetAsync(D.T, 0, sizeof(double) * nc, h->stream));
  DCK(cudaStreamSynchronize(h->stream));
  return GRTE_OK;
}

grte_status grte_diff_set_T(grte_diff_t h, int inst, const double* T, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !T) return dfail(h, GRTE_EINVAL, "bad instance or NULL T");
  const DInst& I = h->inst[inst];
  if (len != (size_t)I.N) return dfail(h, GRTE_EINVAL, "len must equal nx");
  for (size_t j = 0; j < len; ++j)
    if (!(T[j] >= 0.0) || !std::isfinite(T[j])) return dfail(h, GRTE_EINVAL, "T must be finite and >= 0");
  DCK(cudaMemcpyAsync(h->D.T + I.off, T, sizeof(double) * I.N, cudaMemcpyHostToDevice, h->stream));
  DCK(cudaStreamSynchronize(h->stream));
  return GRTE_OK;
}

grte_status grte_diff_step(grte_diff_t h, int64_t nsteps) {
  if (!h) return GRTE_EINVAL;
  if (nsteps < 0) return dfail(h, GRTE_EINVAL, "nsteps < 0");
  const unsigned cb = 256, cg = (unsigned)((h->ncell + cb - 1) / cb);
  const size_t smem = (size_t)tri_smem_bytes(kDT, true, 8);
  for (int64_t n = 0; n < nsteps; ++n) {
    k_dcoef<<<cg, cb, 0, h->stream>>>(h->D, h->n_inst, h->ncell);
    k_dsolve<<<(unsigned)h->n_inst, kDT, smem, h->stream>>>(h->D);
    k_dcorr<<<cg, cb, 0, h->stream>>>(h->D, h->n_inst, h->ncell, h->newton_maxit);
  }
  DCK(cudaGetLastError());
  return GRTE_OK;
}

static grte_status dstatus(grte_diff_t h) {
  int s = 0;
  DCK(cudaStreamSynchronize(h->stream));
  DCK(cudaMemcpy(&s, h->D.status, sizeof(int), cudaMemcpyDeviceToHost));
  for (int code : {GRTE_ENAN, GRTE_ENONCONV, GRTE_ENEGATIVE})
    if (s & (1 << code)) return dfail(h, (grte_status)code, "device reported status " + std::to_string(code));
  return GRTE_OK;
}

grte_status grte_diff_sync(grte_diff_t h) {
  if (!h) return GRTE_EINVAL;
  const grte_status s = dstatus(h);
  if (s != GRTE_OK && s != GRTE_ECUDA) DCK(cudaMemset(h->D.status, 0, sizeof(int)));
  return s;
}

static grte_status dget(grte_diff_t h, int inst, const double* src, double* out, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !out) return dfail(h, GRTE_EINVAL, "bad instance or NULL output");
  const DInst& I = h->inst[inst];
  if (len != (size_t)I.N) return dfail(h, GRTE_EINVAL, "len must equal nx");
  DCK(cudaStreamSynchronize(h->stream));
  DCK(cudaMemcpy(out, src + I.off, sizeof(double) * I.N, cudaMemcpyDeviceToHost));
  return dstatus(h);
}

grte_status grte_diff_get_T(grte_diff_t h, int inst, double* T, size_t len) {
  return h ? dget(h, inst, h->D.T, T, len) : GRTE_EINVAL;
}
grte_status grte_diff_get_Ustar(grte_diff_t h, int inst, double* U, size_t len) {
  return h ? dget(h, inst, h->D.Us, U, len) : GRTE_EINVAL;
}

}  // extern "C"
