// Per-pair multigrid preconditioner for the 2D correction substep (GRTE_PREC2D_CORR_MG).
//
// Correction substep 2 solves, for every direction pair k, (A + G_k) E_k = r_k on the
// cells (Eq. dis-cor1/2 in the dimension-by-dimension form of Sec. 4): A the per-cell
// diagonal, G_k the streaming operator along Omega_k through the vertex-averaged
// differences, a 3x3 stencil per pair.  Where A is small against G_k (hot, optically thin
// cells at small eps) the pair system is a strongly anisotropic diffusion along Omega_k,
// and a per-cell (Jacobi) preconditioner needs a number of Krylov iterations that grows
// ~3x per grid doubling.  This preconditioner replaces (A + G_k)^{-1} by one V-cycle of an
// aggregation multigrid per pair, all K pairs batched:
//   - level 0: the pair's 3x3 stencil, recovered by probing the operator once per solve
//     (cells coloured so that no two cells of a 3x3 neighbourhood share a colour);
//   - coarser levels: 2x2 aggregates, Galerkin products P^T S P with the piecewise-
//     constant P (they stay 3x3 stencils), down to lines of <= 2 cells;
//   - smoother: zebra line relaxation, y lines then x lines before the coarse correction,
//     x lines then y lines after it; on the coarsest level kCoarseSweeps such pairs.
// The lines are tridiagonal solves (Thomas, one thread per line).  A thread walks its line
// along the slow index of the layout, so that a warp's 32 lines read adjacent addresses:
// y lines in the row-major copy (cell q nx + p), x lines in a transposed copy (p ny + q)
// with its own transposed stencil; the iterate and the right side are transposed between
// the two.  Periodic axes: a line's wrap coupling and the neighbour lines across the
// wrap are taken from the current iterate (the line solve itself is not cyclic).
// Arithmetic in binary32: a preconditioner's rounding only changes the Krylov iteration,
// not the converged solution (every restart forms the binary64 residual).
#pragma once
#include <cstdint>

namespace grte2 {
namespace mp {

constexpr int kThreadsMp = 256;
constexpr int kCoarseSweeps = 4;

struct PLevel {
  int nx, ny, K, perx, pery;
  int64_t n;          // cells per pair
  float* cr;          // [K][9][n] row-major stencil, pos = (dy + 1) * 3 + dx + 1
  float* ct;          // [K][9][n] transposed: cell p ny + q, pos = (dx + 1) * 3 + dy + 1
  float *x, *xt;      // [K][n] iterate, row-major / transposed
  float *b, *bt;      // [K][n] right side, row-major / transposed
  float* cp;          // [K][n] Thomas scratch
};

__device__ __forceinline__ int pnbr(int p, int d, int n, int per) {
  const int r = p + d;
  if (per) return r < 0 ? r + n : (r >= n ? r - n : r);
  return (r < 0 || r >= n) ? -1 : r;
}

__device__ __forceinline__ int pcoarse_off(int Pn, int P, int cn, int per) {
  if (!per) return Pn - P;
  int d = (Pn - P) % cn;
  if (d < 0) d += cn;
  return d == 0 ? 0 : (d == 1 ? 1 : -1);
}

// Zebra line relaxation in one layout: lines along the slow axis (ns cells), one line per
// fast index i of the given parity (nf lines per pair); coef holds the stencil in the
// layout's own positions pos = (ds + 1) * 3 + df + 1.  The line's own unknowns are
// replaced by the solution of its tridiagonal system with the other lines (and a
// periodic slow axis's wrap coupling) at their current values.
__global__ void mp_line(const float* __restrict__ coef, float* __restrict__ x, const float* __restrict__ b,
                        float* __restrict__ cp, int nf, int ns, int K, int perf, int pers, int parity) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int half = (nf - parity + 1) / 2;   // lines of this parity per pair
  if (t >= (int64_t)K * half) return;
  const int k = (int)(t / half);
  const int i = parity + 2 * (int)(t - (int64_t)k * half);
  const int64_t n = (int64_t)nf * ns;
  const float* C = coef + (int64_t)k * 9 * n;
  float* X = x + (int64_t)k * n;
  const float* B = b + (int64_t)k * n;
  float* CP = cp + (int64_t)k * n;
  const int il = pnbr(i, -1, nf, perf), ir = pnbr(i, 1, nf, perf);
  // wrap values of a periodic slow axis, read before the line is overwritten
  const float xw_first = pers ? X[i] : 0.0f, xw_last = pers ? X[(int64_t)(ns - 1) * nf + i] : 0.0f;
  float cprev = 0.0f, dprev = 0.0f;
  for (int j = 0; j < ns; ++j) {
    const int64_t e = (int64_t)j * nf + i;
    float r = B[e];
    // the neighbour lines (fast offset -1, +1) at slow offsets -1, 0, +1
#pragma unroll
    for (int ds = -1; ds <= 1; ++ds) {
      const int jn = pnbr(j, ds, ns, pers);
      if (jn < 0) continue;
#pragma unroll
      for (int df = -1; df <= 1; df += 2) {
        const int in = df < 0 ? il : ir;
        if (in < 0) continue;
        const float a = C[(int64_t)((ds + 1) * 3 + df + 1) * n + e];
        r -= a * X[(int64_t)jn * nf + in];
      }
    }
    float a = C[(int64_t)1 * n + e], c = C[(int64_t)7 * n + e];
    const float bb = C[(int64_t)4 * n + e];
    if (j == 0) {
      if (pers) r -= a * xw_last;
      a = 0.0f;
    }
    if (j == ns - 1) {
      if (pers) r -= c * xw_first;
      c = 0.0f;
    }
    const float den = bb - a * cprev;
    const float inv = 1.0f / den;
    cprev = c * inv;
    dprev = (r - a * dprev) * inv;
    CP[e] = cprev;
    X[e] = dprev;
  }
  float xn = dprev;
  for (int j = ns - 2; j >= 0; --j) {
    const int64_t e = (int64_t)j * nf + i;
    xn = X[e] - CP[e] * xn;
    X[e] = xn;
  }
}

// out[k][p * ny + q] = in[k][q * nx + p] (tiled through shared memory)
__global__ void mp_transpose(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int K) {
  __shared__ float tile[32][33];
  const int k = blockIdx.z;
  const int64_t n = (int64_t)nx * ny;
  const int p0 = blockIdx.x * 32, q0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int q = q0 + r, p = p0 + threadIdx.x;
    if (q < ny && p < nx) tile[r][threadIdx.x] = in[(int64_t)k * n + (int64_t)q * nx + p];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int p = p0 + r, q = q0 + threadIdx.x;
    if (p < nx && q < ny) out[(int64_t)k * n + (int64_t)p * ny + q] = tile[threadIdx.x][r];
  }
  (void)K;
}

// the transposed stencil: ct[k][(dx+1)*3 + dy+1][p ny + q] = cr[k][(dy+1)*3 + dx+1][q nx + p]
__global__ void mp_stencil_t(PLevel L) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)L.K * L.n) return;
  const int k = (int)(t / L.n);
  const int64_t c = t - (int64_t)k * L.n;
  const int p = (int)(c % L.nx), q = (int)(c / L.nx);
  const int64_t ct = (int64_t)p * L.ny + q;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx)
      L.ct[((int64_t)k * 9 + (dx + 1) * 3 + dy + 1) * L.n + ct] = L.cr[((int64_t)k * 9 + (dy + 1) * 3 + dx + 1) * L.n + c];
}

// (S x)_c for pair k at cell (p, q), row-major
__device__ __forceinline__ float mp_apply(const PLevel& L, const float* __restrict__ X, const float* __restrict__ C,
                                          int p, int q, int64_t c) {
  float s = 0.0f;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    const int qn = pnbr(q, dy, L.ny, L.pery);
    if (qn < 0) continue;
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int pn = pnbr(p, dx, L.nx, L.perx);
      if (pn < 0) continue;
      s += C[(int64_t)((dy + 1) * 3 + dx + 1) * L.n + c] * X[(int64_t)qn * L.nx + pn];
    }
  }
  return s;
}

// coarse right side: C.b[k][U] = sum over the 2x2 members of (b - S x); C.x = 0
__global__ void mp_restrict(PLevel F, PLevel Cl) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)Cl.K * Cl.n) return;
  const int k = (int)(t / Cl.n);
  const int64_t U = t - (int64_t)k * Cl.n;
  const int P = (int)(U % Cl.nx), Q = (int)(U / Cl.nx);
  const float* X = F.x + (int64_t)k * F.n;
  const float* B = F.b + (int64_t)k * F.n;
  const float* Cf = F.cr + (int64_t)k * 9 * F.n;
  float s = 0.0f;
  for (int m = 0; m < 4; ++m) {
    const int p = 2 * P + (m & 1), q = 2 * Q + (m >> 1);
    if (p >= F.nx || q >= F.ny) continue;
    const int64_t c = (int64_t)q * F.nx + p;
    s += B[c] - mp_apply(F, X, Cf, p, q, c);
  }
  Cl.b[t] = s;
  Cl.x[t] = 0.0f;
}

// F.x += P C.x (piecewise constant)
__global__ void mp_prolong(PLevel F, PLevel Cl) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)F.K * F.n) return;
  const int k = (int)(t / F.n);
  const int64_t c = t - (int64_t)k * F.n;
  const int p = (int)(c % F.nx), q = (int)(c / F.nx);
  F.x[t] += Cl.x[(int64_t)k * Cl.n + (int64_t)(q >> 1) * Cl.nx + (p >> 1)];
}

// Galerkin coarse stencil C = P^T F P per pair
__global__ void mp_galerkin(PLevel F, PLevel Cl) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)Cl.K * Cl.n) return;
  const int k = (int)(t / Cl.n);
  const int64_t U = t - (int64_t)k * Cl.n;
  const int P = (int)(U % Cl.nx), Q = (int)(U / Cl.nx);
  const float* Cf = F.cr + (int64_t)k * 9 * F.n;
  float acc[9];
#pragma unroll
  for (int s = 0; s < 9; ++s) acc[s] = 0.0f;
  for (int m = 0; m < 4; ++m) {
    const int p = 2 * P + (m & 1), q = 2 * Q + (m >> 1);
    if (p >= F.nx || q >= F.ny) continue;
    const int64_t c = (int64_t)q * F.nx + p;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int qn = pnbr(q, dy, F.ny, F.pery);
      if (qn < 0) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int pn = pnbr(p, dx, F.nx, F.perx);
        if (pn < 0) continue;
        const float a = Cf[(int64_t)((dy + 1) * 3 + dx + 1) * F.n + c];
        const int dX = pcoarse_off(pn >> 1, P, Cl.nx, Cl.perx), dY = pcoarse_off(qn >> 1, Q, Cl.ny, Cl.pery);
        acc[(dY + 1) * 3 + dX + 1] += a;
      }
    }
  }
#pragma unroll
  for (int s = 0; s < 9; ++s) Cl.cr[((int64_t)k * 9 + s) * Cl.n + U] = acc[s];
}

}  // namespace mp
}  // namespace grte2
