// Aggregation multigrid for the cell-centred rho system of the 2D prediction
// preconditioner (a 3x3-stencil operator on the Nx x Ny cells).
//
// The operator comes from the vertex-averaged streaming derivatives of the 2D scheme:
// summed over a symmetric quadrature, the vertex gradient followed by the cell
// divergence couples a cell to its four diagonal neighbours only, so the cells split
// into two weakly coupled colour classes ((p + q) even / odd) and the checkerboard-
// modulated smooth modes are near-null modes as well as the smooth ones.  Plain 2x2
// aggregation sums that mode to zero; here every coarse cell carries one unknown per
// colour class, the aggregate of the fine unknowns of that colour in its 2x2 block
// (level 0: the one or two cells of the colour; above: the same-colour unknowns of
// the four child cells).  Coarse operators are Galerkin products P^T S P with the
// piecewise-constant P; they stay 3x3 stencils, with two colours: 18 couplings per
// unknown.  Smoother: two damped Jacobi sweeps before and after the coarse correction
// (damping 0.8).  The coarsest level (<= 64 unknowns) is inverted densely (Gauss-
// Jordan, no pivoting: the operators are diagonally dominant) once per setup.
//
// Layout: level 0 unknown = cell q*nx + p, coefficients [pos][cell] with pos = (dy+1)*3
// + (dx+1); level >= 1 unknown u = colour*ncell + cell, coefficients [pos*2 + colour'][u].
// Periodic axes wrap; a coarse offset is taken modulo the coarse size and stored at
// 0, +1 or -1 in that order of preference (on a periodic axis of one or two coarse
// cells several offsets name the same cell: the stencil apply sums them, so storing
// each coupling once is enough).
#pragma once
#include <cstdint>

namespace grte2 {
namespace mg {

constexpr int kThreadsMg = 256;
constexpr int kDenseMax = 64;
constexpr double kOmega = 0.8;

struct Level {
  int nx, ny, ncomp, perx, pery;
  int64_t ncell, n;
  double* coef;    // ncomp 1: [9][n]; ncomp 2: [18][n]
  double* idiag;   // [n], 0 for an empty aggregate
  double *x, *xt, *b;
};

__device__ __forceinline__ int nbr(int p, int d, int n, int per) {
  const int r = p + d;
  if (per) return r < 0 ? r + n : (r >= n ? r - n : r);
  return (r < 0 || r >= n) ? -1 : r;
}

__device__ __forceinline__ int coarse_off(int Pn, int P, int cn, int per) {
  if (!per) return Pn - P;
  int d = (Pn - P) % cn;
  if (d < 0) d += cn;
  return d == 0 ? 0 : (d == 1 ? 1 : -1);
}

// index in the coarse level C of the aggregate of fine unknown (p, q, colour col)
__device__ __forceinline__ int64_t agg_of(const Level& C, int p, int q, int col) {
  return (int64_t)col * C.ncell + (int64_t)(q >> 1) * C.nx + (p >> 1);
}

// (S x)_u, with x read as x[v] + xc[agg(v)] when xc is given (fused prolongation)
template <int NC>
__device__ double apply_row(const Level& L, const double* __restrict__ x, const double* __restrict__ xc,
                            const Level& C, int64_t u, int p, int q) {
  double s = 0.0;
#pragma unroll
  for (int t = 0; t < 9 * NC; ++t) {
    const double a = L.coef[(int64_t)t * L.n + u];
    if (a == 0.0) continue;
    const int pos = NC == 1 ? t : (t >> 1);
    const int pn = nbr(p, pos % 3 - 1, L.nx, L.perx), qn = nbr(q, pos / 3 - 1, L.ny, L.pery);
    if (pn < 0 || qn < 0) continue;
    const int col = NC == 1 ? ((pn + qn) & 1) : (t & 1);
    const int64_t v = (NC == 1 ? 0 : (int64_t)col * L.ncell) + (int64_t)qn * L.nx + pn;
    double xv = x[v];
    if (xc) xv += xc[agg_of(C, pn, qn, col)];
    s += a * xv;
  }
  return s;
}

template <int NC>
__device__ __forceinline__ void unknown_pos(const Level& L, int64_t u, int& p, int& q, int& col) {
  const int64_t cell = NC == 1 ? u : u % L.ncell;
  p = (int)(cell % L.nx);
  q = (int)(cell / L.nx);
  col = NC == 1 ? ((p + q) & 1) : (int)(u / L.ncell);
}

// first sweep from x = 0
__global__ void mg_jacobi0(Level L) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= L.n) return;
  L.x[u] = kOmega * L.b[u] * L.idiag[u];
}

// xout = xi + omega D^{-1} (b - S xi), xi = xin (+ P xc)
template <int NC>
__global__ void mg_jacobi(Level L, const double* __restrict__ xin, double* __restrict__ xout,
                          const double* __restrict__ xc, Level C) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= L.n) return;
  int p, q, col;
  unknown_pos<NC>(L, u, p, q, col);
  double xi = xin[u];
  if (xc) xi += xc[agg_of(C, p, q, col)];
  const double r = L.b[u] - apply_row<NC>(L, xin, xc, C, u, p, q);
  xout[u] = xi + kOmega * r * L.idiag[u];
}

// C.b[U] = sum over the members u of U of (b - S x)_u
template <int NC>
__global__ void mg_restrict(Level F, const double* __restrict__ x, Level C) {
  const int64_t U = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (U >= C.n) return;
  const int col = (int)(U / C.ncell);
  const int64_t cell = U - (int64_t)col * C.ncell;
  const int P = (int)(cell % C.nx), Q = (int)(cell / C.nx);
  double s = 0.0;
  for (int b = 0; b < 4; ++b) {
    const int p = 2 * P + (b & 1), q = 2 * Q + (b >> 1);
    if (p >= F.nx || q >= F.ny) continue;
    if (NC == 1 && ((p + q) & 1) != col) continue;
    const int64_t u = (NC == 1 ? 0 : (int64_t)col * F.ncell) + (int64_t)q * F.nx + p;
    s += F.b[u] - apply_row<NC>(F, x, nullptr, C, u, p, q);
  }
  C.b[U] = s;
}

// Galerkin coarse operator C = P^T F P
template <int NC>
__global__ void mg_galerkin(Level F, Level C) {
  const int64_t U = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (U >= C.n) return;
  const int col = (int)(U / C.ncell);
  const int64_t cell = U - (int64_t)col * C.ncell;
  const int P = (int)(cell % C.nx), Q = (int)(cell / C.nx);
  double acc[18];
#pragma unroll
  for (int t = 0; t < 18; ++t) acc[t] = 0.0;
  for (int b = 0; b < 4; ++b) {
    const int p = 2 * P + (b & 1), q = 2 * Q + (b >> 1);
    if (p >= F.nx || q >= F.ny) continue;
    if (NC == 1 && ((p + q) & 1) != col) continue;
    const int64_t u = (NC == 1 ? 0 : (int64_t)col * F.ncell) + (int64_t)q * F.nx + p;
#pragma unroll
    for (int t = 0; t < 9 * NC; ++t) {
      const double a = F.coef[(int64_t)t * F.n + u];
      if (a == 0.0) continue;
      const int pos = NC == 1 ? t : (t >> 1);
      const int pn = nbr(p, pos % 3 - 1, F.nx, F.perx), qn = nbr(q, pos / 3 - 1, F.ny, F.pery);
      if (pn < 0 || qn < 0) continue;
      const int cc = NC == 1 ? ((pn + qn) & 1) : (t & 1);
      const int dX = coarse_off(pn >> 1, P, C.nx, C.perx), dY = coarse_off(qn >> 1, Q, C.ny, C.pery);
      acc[((dY + 1) * 3 + dX + 1) * 2 + cc] += a;
    }
  }
#pragma unroll
  for (int t = 0; t < 18; ++t) C.coef[(int64_t)t * C.n + U] = acc[t];
  const double d = acc[4 * 2 + col];
  C.idiag[U] = d != 0.0 ? 1.0 / d : 0.0;
}

__global__ void mg_idiag0(Level L) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= L.n) return;
  const double d = L.coef[4 * L.n + u];
  L.idiag[u] = d != 0.0 ? 1.0 / d : 0.0;
}

// Dense inverse of the coarsest level's operator (one block): M (n x n, scratch) is
// assembled from the stencil, a zero row (empty aggregate) gets a unit diagonal, and
// Gauss-Jordan on [M | I] leaves the inverse in inv.
template <int NC>
__global__ void mg_dense_inverse(Level L, double* __restrict__ M, double* __restrict__ inv) {
  __shared__ double fac[kDenseMax];
  const int n = (int)L.n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    M[i] = 0.0;
    inv[i] = (i / n == i % n) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int u = threadIdx.x; u < n; u += blockDim.x) {
    int p, q, col;
    unknown_pos<NC>(L, u, p, q, col);
    for (int t = 0; t < 9 * NC; ++t) {
      const double a = L.coef[(int64_t)t * L.n + u];
      if (a == 0.0) continue;
      const int pos = NC == 1 ? t : (t >> 1);
      const int pn = nbr(p, pos % 3 - 1, L.nx, L.perx), qn = nbr(q, pos / 3 - 1, L.ny, L.pery);
      if (pn < 0 || qn < 0) continue;
      const int cc = NC == 1 ? ((pn + qn) & 1) : (t & 1);
      const int v = (NC == 1 ? 0 : cc * (int)L.ncell) + qn * L.nx + pn;
      M[u * n + v] += a;
    }
    if (M[u * n + u] == 0.0) M[u * n + u] = 1.0;
  }
  __syncthreads();
  for (int col = 0; col < n; ++col) {
    const double piv = M[col * n + col];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      M[col * n + j] /= piv;
      inv[col * n + j] /= piv;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) fac[r] = r == col ? 0.0 : M[r * n + col];
    __syncthreads();
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
      const int r = i / n, j = i % n;
      if (r == col) continue;
      M[i] -= fac[r] * M[col * n + j];
      inv[i] -= fac[r] * inv[col * n + j];
    }
    __syncthreads();
  }
}

// x = inv b on the coarsest level (one block)
__global__ void mg_dense_apply(Level L, const double* __restrict__ inv) {
  const int n = (int)L.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += inv[i * n + j] * L.b[j];
    L.x[i] = s;
  }
}

}  // namespace mg
}  // namespace grte2
