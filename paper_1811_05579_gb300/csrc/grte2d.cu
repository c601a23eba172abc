// GB300 (sm_103a) implementation of one step of the AP scheme for the gray radiative
// transfer equation (Tang, Wang, Zhang, arXiv:1811.05579) on a 2D grid: the 1D
// scheme (Algorithm 2 of Sec. 4, sigma_0/T^3 form of Sec. 5) taken direction by
// direction, as declared in include/grte.h (grte2d_*).
//
// Unknowns: E (pairs k, cells) and O (pairs k, vertices), U and T per cell.  The
// streaming operators are applied matrix-free by two stencil kernels: a vertex pass
// (node equation O = o - d D_k E at vertices that carry one, the inflow-wall and
// corner expressions elsewhere) and a cell pass (kappa D*_k O, a cell beside an
// inflow wall taking its wall side from Eq. bc-pre with its own E).  The prediction
// (Eq. dis-pre / Eq. dis-pre-marshak) is solved for (e, rho), E = rho + e, by
// restarted GMRES with an exact per-cell angular block solve as left preconditioner;
// the temperature (Eq. Tnp1) by monotone Newton per cell; correction substep 2
// (Eq. dis-cor) by GMRES on the stacked pair systems; projection (Eq. dis-proj).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/grte.h"

// NVTX range over a host-side stage of a step (shown by Nsight Systems and other NVTX
// tools; free when none is attached)
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace
#include "mg2d.cuh"
#include "mgpair2d.cuh"
#include "mlp.cuh"

namespace grte2 {

constexpr double kGuessGate2 = 1.1220184543019633;   // 10^0.05: learned-start gate (k2_newton)
constexpr int kMgStageCycles = 4;   // restart cycles of the multigrid-preconditioned stage
constexpr double kMixedRtol = 1e-11; // mixed precision: floor of the Krylov tolerance
constexpr double kInnerReduce = 1e-5; // mixed precision: residual reduction of one binary32 cycle

constexpr int kMaxPairs = 64;
constexpr int kMaxRestart2 = 64;
constexpr int kThreads = 256;
constexpr int kRedBlocks = 304;   // 2 x 152 SMs: blocks of the first reduction stage
constexpr int kDotBlocks = 304;   // 2 x 152: blocks of the Gram-Schmidt dot products (one wave)
constexpr int kAxpyBlocks = 1216; // 8 x 152: blocks of the streaming vector updates

struct G2 {
  int Nx, Ny, K, bcx, bcy, kind;   // kind: GRTE_SIGMA_CONST or GRTE_SIGMA_T3 (sigma_0/T^p)
  double p;                        // the exponent of sigma_0/T^p (3 for GRTE_SIGMA_T3)
  int64_t nc, nv;
  double dx, dy, eps, dt, a, c, Cv;
  double bx0, bx1, by0, by1;
  double h2x, h2y, te;   // 1/(2 dx), 1/(2 dy), 2/eps (no divisions in the stencils)
};

struct D2 {
  G2 g;
  const double *mu, *eta, *w, *sig;
  double *T, *U, *E, *O;                      // state; E [k][cell], O [k][vertex]
  double *kc, *A, *alpha, *s, *gam;           // per cell at the current temperature
  double *dv, *odv;                           // per vertex: d and d eps^2/(c dt) (node-equation vertices)
  double *rho_n, *Us, *Fdiv, *rho_s, *newton_its, *acU;
  double *wsc, *iwsc;   // per-cell scale of the Krylov unknowns (k2_weights) and its inverse
  double *gd, *gdi, *pdi;   // [k][cell] diagonal g_k of G_k, 1/(A + g_k); [cell] inverse rho pivot
  int* status;
  int newton_maxit;
  // learned Newton start: per-cell features (6 floats), predicted and logged targets
  float *feat, *guess, *ytrue;
  int use_guess, log_samples, start_prev;
};

__device__ __forceinline__ void flag2(int* status, int code) { atomicOr(status, 1 << code); }

__device__ __forceinline__ int cell_of(const G2& g, int p, int q) {
  if (g.bcx == GRTE_BC_PERIODIC) p = (p + g.Nx) % g.Nx;
  if (g.bcy == GRTE_BC_PERIODIC) q = (q + g.Ny) % g.Ny;
  if (p < 0 || p >= g.Nx || q < 0 || q >= g.Ny) return -1;
  return q * g.Nx + p;
}

// 0: node equation (inside, or a periodic copy), 2: inflow x wall, 3: inflow y wall, 4: corner
__device__ __forceinline__ int vkind(const G2& g, int i, int j) {
  const bool onx = g.bcx == GRTE_BC_INFLOW && (i == 0 || i == g.Nx);
  const bool ony = g.bcy == GRTE_BC_INFLOW && (j == 0 || j == g.Ny);
  return onx && ony ? 4 : onx ? 2 : ony ? 3 : 0;
}

// ----------------------------------------------------------------------------- coefficients
// Per cell at temperature T (Eq. dis-pre: kappa = 1, theta = T^3; Eq. dis-pre-marshak:
// kappa = T^3, theta = 1; sigma_0/T^p: kappa = T^p, theta = T^{3-p}): s, gamma,
// A = kappa/(c dt) + sig/eps^2, alpha = kappa/(c dt) + s.
__global__ void k2_coef(D2 D) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const double T = D.T[c], sg = D.sig[c];
  const double T3 = T * T * T;
  const double kc = g.kind == GRTE_SIGMA_CONST ? 1.0 : (g.p == 3.0 ? T3 : pow(T, g.p));
  const double th = g.kind == GRTE_SIGMA_CONST ? T3 : (g.p == 3.0 ? 1.0 : pow(T, 3.0 - g.p));
  const double e2 = g.eps * g.eps;
  const double s = sg * g.Cv / (g.Cv * e2 + 4.0 * sg * th * g.dt * g.a * g.c);
  D.kc[c] = kc;
  D.s[c] = s;
  D.gam[c] = 4.0 * sg * th * g.dt / (e2 * g.Cv);
  D.A[c] = kc / (g.c * g.dt) + sg / e2;
  D.alpha[c] = kc / (g.c * g.dt) + s;
}

// Per vertex with a node equation: kappa = mean of the four cells, sig = their harmonic
// mean, d = kappa/(kappa eps^2/(c dt) + sig), od = d eps^2/(c dt).  0 at wall vertices.
__global__ void k2_vcoef(D2 D) {
  const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (v >= g.nv) return;
  const int i = (int)(v % (g.Nx + 1)), j = (int)(v / (g.Nx + 1));
  double d = 0.0;
  if (vkind(g, i, j) == 0) {
    const int cs[4] = {cell_of(g, i - 1, j - 1), cell_of(g, i, j - 1), cell_of(g, i - 1, j), cell_of(g, i, j)};
    double kv = 0.0, inv = 0.0;
    bool pos = true;
    for (int q = 0; q < 4; ++q) {
      kv += 0.25 * D.kc[cs[q]];
      const double sg = D.sig[cs[q]];
      if (sg > 0.0) inv += 1.0 / sg; else pos = false;
    }
    const double sv = pos ? 4.0 / inv : 0.0;
    d = kv > 0.0 ? kv / (kv * g.eps * g.eps / (g.c * g.dt) + sv) : 0.0;
  }
  D.dv[v] = d;
  D.odv[v] = d * g.eps * g.eps / (g.c * g.dt);
}

__global__ void k2_rho(D2 D, const double* __restrict__ E, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= D.g.nc) return;
  double r = 0.0;
  for (int k = 0; k < D.g.K; ++k) r += D.w[k] * E[(int64_t)k * D.g.nc + c];
  out[c] = r;
}

__global__ void k2_acU(D2 D) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= D.g.nc) return;
  const double t = D.T[c];
  D.acU[c] = D.g.a * D.g.c * (t * t) * (t * t);
}

// ----------------------------------------------------------------------------- stencils
// Coefficients the Krylov-loop stencils read, in precision S: binary64 (the D2 arrays)
// or, in the mixed mode's binary32 Krylov cycles, float copies made once per solve
// (cell, vertex and preconditioner values) and per restart (the Krylov cell scale).
template <typename S>
struct CV {
  const S *mu, *eta, *w;         // [K]
  const S *kc, *A, *alpha;       // [cell]
  const S* dv;                   // [vertex]
  const S *gd, *gdi, *pdi;       // [k][cell], [k][cell], [cell]
  const S *wsc, *iwsc;           // [cell]
  S h2x, h2y, te;
};

// Per-pair cell field u_k(c) = (uk[k*ks + c] + ub[c]) * sc[c] (any part may be absent).
template <typename S>
struct UFieldT {
  const S* uk;
  int64_t ks;
  const S* ub;
  const S* sc = nullptr;
  __device__ __forceinline__ S at(int k, int c) const {
    S v = S(0);
    if (uk) v += uk[(int64_t)k * ks + c];
    if (ub) v += ub[c];
    return sc ? v * sc[c] : v;
  }
  __device__ __forceinline__ bool any() const { return uk || ub; }
};
using UField = UFieldT<double>;

// O at a node-equation vertex: o - d (D_k u)  (o = d eps^2 O^n/(c dt) with data).
template <typename S, bool DATA>
__device__ S O_node(const D2& D, const CV<S>& cv, const UFieldT<S>& u, int k, int i, int j) {
  const G2& g = D.g;
  const int64_t v = (int64_t)j * (g.Nx + 1) + i;
  S r = S(0);
  if constexpr (DATA) r = D.odv[v] * D.O[(int64_t)k * g.nv + v];
  if (u.any()) {
    const int c00 = cell_of(g, i - 1, j - 1), c10 = cell_of(g, i, j - 1), c01 = cell_of(g, i - 1, j),
              c11 = cell_of(g, i, j);
    const S u00 = u.at(k, c00), u10 = u.at(k, c10), u01 = u.at(k, c01), u11 = u.at(k, c11);
    const S grad = cv.mu[k] * ((u10 + u11) - (u00 + u01)) * cv.h2x + cv.eta[k] * ((u01 + u11) - (u00 + u10)) * cv.h2y;
    r -= cv.dv[v] * grad;
  }
  return r;
}

// Wall expression (Eq. bc-pre along the normal of `axis` at vertex (i, j)):
//   Omega_k enters:  O = 2/eps (b - E_wall) - O_inner;  else  O = 2/eps (E_wall - b) - O_inner.
template <typename S, bool DATA>
__device__ S O_wall(const D2& D, const CV<S>& cv, const UFieldT<S>& u, int k, int i, int j, int axis, S Oinner) {
  const G2& g = D.g;
  S comp;
  double b;
  int side, ca, cb;
  if (axis == 0) {
    side = i == 0 ? 0 : 1;
    comp = cv.mu[k];
    b = side == 0 ? g.bx0 : g.bx1;
    const int p = side == 0 ? 0 : g.Nx - 1;
    ca = cell_of(g, p, j - 1);
    cb = cell_of(g, p, j);
  } else {
    side = j == 0 ? 0 : 1;
    comp = cv.eta[k];
    b = side == 0 ? g.by0 : g.by1;
    const int q = side == 0 ? 0 : g.Ny - 1;
    ca = cell_of(g, i - 1, q);
    cb = cell_of(g, i, q);
  }
  const bool enters = side == 0 ? comp > S(0) : comp < S(0);
  const S sgn = enters ? S(1) : S(-1);
  S Ew = S(0);
  if (u.any()) {
    int n = 0;
    if (ca >= 0) { Ew += u.at(k, ca); ++n; }
    if (cb >= 0) { Ew += u.at(k, cb); ++n; }
    if (n == 2) Ew *= S(0.5);
  }
  S bd = S(0);
  if constexpr (DATA) bd = b;
  return sgn * cv.te * (bd - Ew) - Oinner;
}

template <typename S, bool DATA>
__device__ S O_at(const D2& D, const CV<S>& cv, const UFieldT<S>& u, int k, int i, int j) {
  const G2& g = D.g;
  const int kind = vkind(g, i, j);
  if (kind == 0) return O_node<S, DATA>(D, cv, u, k, i, j);
  const int ii = i == 0 ? 1 : g.Nx - 1, jj = j == 0 ? 1 : g.Ny - 1;
  if (kind == 2) return O_wall<S, DATA>(D, cv, u, k, i, j, 0, O_node<S, DATA>(D, cv, u, k, ii, j));
  if (kind == 3) return O_wall<S, DATA>(D, cv, u, k, i, j, 1, O_node<S, DATA>(D, cv, u, k, i, jj));
  // corner: mean of the two walls; each wall's inner vertex lies on the other wall
  const S Oin_x = O_wall<S, DATA>(D, cv, u, k, ii, j, 1, O_node<S, DATA>(D, cv, u, k, ii, jj));
  const S Oin_y = O_wall<S, DATA>(D, cv, u, k, i, jj, 0, O_node<S, DATA>(D, cv, u, k, ii, jj));
  return S(0.5) * (O_wall<S, DATA>(D, cv, u, k, i, j, 0, Oin_x) + O_wall<S, DATA>(D, cv, u, k, i, j, 1, Oin_y));
}

// V[k][v] = O_k at every vertex for the field u (and the data part with DATA); one
// thread per (pair, vertex), consecutive threads on consecutive vertices.
template <typename S, bool DATA>
__global__ void k2_vertex(D2 D, CV<S> cv, UFieldT<S> u, S* __restrict__ V) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (t >= (int64_t)g.K * g.nv) return;
  const int tt = (int)t, nv = (int)g.nv;   // K nv < 2^31 (checked at creation)
  const int k = tt / nv, v = tt - k * nv;
  const int j = v / (g.Nx + 1), i = v - j * (g.Nx + 1);
  V[t] = O_at<S, DATA>(D, cv, u, k, i, j);
}

// The correction's flux (sigma_0/T^3) at the inflow walls: each inflow-wall vertex takes
// the prediction's value shifted by the change at its inner vertex (the indices clamped
// into the interior along the inflow axes), V = Vp + (V_in - Vp_in); Vp holds the
// prediction's vertex values.  Inner vertices are never wall vertices (Nx, Ny >= 2).
__global__ void k2_wallshift(D2 D, double* __restrict__ V, const double* __restrict__ Vp) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (t >= (int64_t)g.K * g.nv) return;
  const int64_t k = t / g.nv, v = t - k * g.nv;
  const int j = (int)(v / (g.Nx + 1)), i = (int)(v - (int64_t)j * (g.Nx + 1));
  if (vkind(g, i, j) == 0) return;
  const int ii = g.bcx == GRTE_BC_INFLOW ? min(max(i, 1), g.Nx - 1) : i;
  const int jj = g.bcy == GRTE_BC_INFLOW ? min(max(j, 1), g.Ny - 1) : j;
  const int64_t vin = k * g.nv + (int64_t)jj * (g.Nx + 1) + ii;
  V[t] = Vp[t] + (V[vin] - Vp[vin]);
}

enum { C_MV_PRED = 0, C_MV_CORR = 1, C_DIVK = 2, C_FDIV = 3 };

// Side weights of cell (p, q) for pair k: the streaming derivative of O at the cell is
//   mu/(2 dx) [wL (O00 + O01) + wR (O10 + O11)] + eta/(2 dy) [wB (O00 + O10) + wT (O01 + O11)]
//   + ed E_cell + bt,
// with (wL, wR, wB, wT) = (-1, 1, -1, 1) inside.  A cell beside an inflow wall applies
// Eq. bc-pre to its own wall side as the 1D wall cell does: the low x side becomes
// s 2/eps (b - E_cell) - (high side), i.e. mu (2 R - s 2/eps (b - E_cell))/dx, and
// likewise for the other sides (s = +1 if Omega_k enters there, else -1).
template <typename S>
struct CellSides {
  S wL, wR, wB, wT, ed, bt;
};

template <typename S>
__device__ __forceinline__ CellSides<S> cell_sides(const D2& D, const CV<S>& cv, int k, int p, int q) {
  const G2& g = D.g;
  CellSides<S> cs{S(-1), S(1), S(-1), S(1), S(0), S(0)};
  const S mu = cv.mu[k], eta = cv.eta[k], te = cv.te, ix = S(2) * cv.h2x, iy = S(2) * cv.h2y;
  if (g.bcx == GRTE_BC_INFLOW) {
    if (p == 0) {
      const S s = mu > S(0) ? S(1) : S(-1);   // Omega_k enters at x = 0 when mu > 0
      cs.wL = S(0);
      cs.wR = S(2);
      cs.ed += mu * s * te * ix;
      cs.bt -= mu * s * te * S(g.bx0) * ix;
    }
    if (p == g.Nx - 1) {
      const S s = mu < S(0) ? S(1) : S(-1);
      if (p != 0) cs.wL = S(-2);
      cs.wR = S(0);
      cs.ed -= mu * s * te * ix;
      cs.bt += mu * s * te * S(g.bx1) * ix;
    }
  }
  if (g.bcy == GRTE_BC_INFLOW) {
    if (q == 0) {
      const S s = eta > S(0) ? S(1) : S(-1);
      cs.wB = S(0);
      cs.wT = S(2);
      cs.ed += eta * s * te * iy;
      cs.bt -= eta * s * te * S(g.by0) * iy;
    }
    if (q == g.Ny - 1) {
      const S s = eta < S(0) ? S(1) : S(-1);
      if (q != 0) cs.wB = S(-2);
      cs.wT = S(0);
      cs.ed -= eta * s * te * iy;
      cs.bt += eta * s * te * S(g.by1) * iy;
    }
  }
  return cs;
}

// Streaming derivative of O_k at cell c (cell_sides), for pair k.
template <typename S, bool DATA>
__device__ __forceinline__ S cell_div(const D2& D, const CV<S>& cv, const S* __restrict__ V, const UFieldT<S>& u,
                                      int k, int64_t c) {
  const G2& g = D.g;
  const int ci = (int)c;
  const int q = ci / g.Nx, p = ci - q * g.Nx;
  const int64_t v00 = (int64_t)q * (g.Nx + 1) + p, v10 = v00 + 1, v01 = v00 + g.Nx + 1, v11 = v01 + 1;
  const S* Vk = V + (int64_t)k * g.nv;
  const bool wall = (g.bcx == GRTE_BC_INFLOW && (p == 0 || p == g.Nx - 1)) ||
                    (g.bcy == GRTE_BC_INFLOW && (q == 0 || q == g.Ny - 1));
  if (!wall)
    return cv.mu[k] * ((Vk[v10] + Vk[v11]) - (Vk[v00] + Vk[v01])) * cv.h2x +
           cv.eta[k] * ((Vk[v01] + Vk[v11]) - (Vk[v00] + Vk[v10])) * cv.h2y;
  const CellSides<S> cs = cell_sides<S>(D, cv, k, p, q);
  S div = cv.mu[k] * cv.h2x * (cs.wL * (Vk[v00] + Vk[v01]) + cs.wR * (Vk[v10] + Vk[v11])) +
          cv.eta[k] * cv.h2y * (cs.wB * (Vk[v00] + Vk[v10]) + cs.wT * (Vk[v01] + Vk[v11]));
  if (u.any()) div += cs.ed * u.at(k, (int)c);
  if constexpr (DATA) div += cs.bt;
  return div;
}

// The correction's flux per pair at cell c (sigma_0/T^3): cell_div over V, except that a
// cell beside an inflow wall takes the part along that wall's normal from the
// prediction's vertex values Vn (so that, as in 1D, its flux across the wall and the
// opposite side is the prediction's; the part along the wall reads V).
__global__ void k2_fdiv_corr(D2 D, CV<double> cv, const double* __restrict__ V, const double* __restrict__ Vn,
                             UField u, double* __restrict__ tk) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (t >= (int64_t)g.K * g.nc) return;
  const int tt = (int)t, nc = (int)g.nc;
  const int k = tt / nc, ci = tt - k * nc;
  const int q = ci / g.Nx, p = ci - q * g.Nx;
  const bool xw = g.bcx == GRTE_BC_INFLOW && (p == 0 || p == g.Nx - 1);
  const bool yw = g.bcy == GRTE_BC_INFLOW && (q == 0 || q == g.Ny - 1);
  if (!xw && !yw) {
    tk[t] = cell_div<double, true>(D, cv, V, u, k, ci);
    return;
  }
  const int64_t v00 = (int64_t)q * (g.Nx + 1) + p, v10 = v00 + 1, v01 = v00 + g.Nx + 1, v11 = v01 + 1;
  const double* Vx = (xw ? Vn : V) + (int64_t)k * g.nv;
  const double* Vy = (yw ? Vn : V) + (int64_t)k * g.nv;
  const CellSides<double> cs = cell_sides<double>(D, cv, k, p, q);
  tk[t] = cv.mu[k] * cv.h2x * (cs.wL * (Vx[v00] + Vx[v01]) + cs.wR * (Vx[v10] + Vx[v11])) +
          cv.eta[k] * cv.h2y * (cs.wB * (Vy[v00] + Vy[v10]) + cs.wT * (Vy[v01] + Vy[v11])) +
          cs.ed * u.at(k, ci) + cs.bt;
}

// Cell pass over the vertex values V (computed from the same field u, with the data
// part when DATA), one thread per (pair, cell):
//   C_MV_PRED: y_k = A z_k + alpha z_rho + kappa S_k,  t_k = kappa S_k (for the rho row)
//   C_MV_CORR: y_k = A z_k + kappa S_k
//   C_DIVK:    y_k = kappa S_k
//   C_FDIV:    t_k = S_k
// S_k the streaming derivative of O_k at the cell (cell_sides).  z is read scaled by
// zs[c] when zs is given (the Krylov unknowns are cell-scaled).  The sums over pairs
// (rho row, C_FDIV) are k2_cellsum.
template <typename S, int MODE, bool DATA>
__global__ void k2_cell(D2 D, CV<S> cv, const S* __restrict__ V, UFieldT<S> u, const S* __restrict__ z,
                        S* __restrict__ y, const S* __restrict__ zs, S* __restrict__ tk) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (t >= (int64_t)g.K * g.nc) return;
  const int tt = (int)t, nc = (int)g.nc;
  const int k = tt / nc;
  const int64_t c = tt - k * nc;
  const S div = cell_div<S, DATA>(D, cv, V, u, k, c);
  const S kc = cv.kc[c];
  const S f = zs ? zs[c] : S(1);
  if (MODE == C_MV_PRED) {
    y[t] = cv.A[c] * f * z[t] + cv.alpha[c] * f * z[(int64_t)g.K * g.nc + c] + kc * div;
    tk[t] = kc * div;
  } else if (MODE == C_MV_CORR) {
    y[t] = cv.A[c] * f * z[t] + kc * div;
  } else if (MODE == C_DIVK) {
    y[t] = kc * div;
  } else {
    tk[t] = div;
  }
}

// Per-cell sums over pairs (fixed order): C_MV_PRED: y_rho = alpha z_rho + sum_k w_k t_k;
// C_FDIV: y = sum_k w_k t_k.
template <typename S, int MODE>
__global__ void k2_cellsum(D2 D, CV<S> cv, const S* __restrict__ tk, const S* __restrict__ z, S* __restrict__ y,
                           const S* __restrict__ zs) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  S acc = S(0);
  for (int k = 0; k < g.K; ++k) acc += cv.w[k] * tk[(int64_t)k * g.nc + c];
  if (MODE == C_MV_PRED) {
    const S f = zs ? zs[c] : S(1);
    y[(int64_t)g.K * g.nc + c] = cv.alpha[c] * f * z[(int64_t)g.K * g.nc + c] + acc;
  } else {
    y[c] = acc;
  }
}

// Diagonal of G_k at cell c (for the preconditioner): the node-equation vertices of
// the cell contribute kappa (side weight) (D* coefficient) (-d) (D_k coefficient), a
// wall cell its own E term kappa ed; wall vertices of an opposite side (corner cells)
// are left out.
__device__ double gdiag(const D2& D, const CV<double>& cv, int k, int p, int q) {
  const G2& g = D.g;
  const CellSides<double> cs = cell_sides<double>(D, cv, k, p, q);
  const double mx = D.mu[k] * g.h2x, ey = D.eta[k] * g.h2y;
  const int di[4] = {0, 1, 0, 1}, dj[4] = {0, 0, 1, 1};
  // D* coefficient of vertex t of the cell with the side weights
  const double cst[4] = {cs.wL * mx + cs.wB * ey, cs.wR * mx + cs.wB * ey, cs.wL * mx + cs.wT * ey,
                         cs.wR * mx + cs.wT * ey};
  const double a = mx + ey, b = mx - ey;
  const double cgr[4] = {a, -b, b, -a};   // D_k coefficient of this cell at vertex t
  double r = cs.ed;
  for (int t = 0; t < 4; ++t) {
    const int i = p + di[t], j = q + dj[t];
    if (vkind(g, i, j) != 0) continue;
    const int64_t v = (int64_t)j * (g.Nx + 1) + i;
    r += cst[t] * (-D.dv[v] * cgr[t]);
  }
  return D.kc[q * g.Nx + p] * r;
}

// Left preconditioner.  Prediction: per cell, the angular block of the matrix with G_k
// replaced by its diagonal g_k (an arrow matrix), solved exactly:
//   rho = [r_rho - sum_k w_k g_k r_k/(A+g_k)] / [alpha + sum_k w_k g_k (A - alpha)/(A+g_k)],
//   e_k = (r_k - (alpha + g_k) rho)/(A + g_k).
// Correction: z_k = r_k/(A + g_k).  The result is multiplied by the cell's Krylov
// scale w (the GMRES runs on w-scaled unknowns: D_w P^{-1} M D_w^{-1}).
// (the diagonals g_k and the reciprocals come from k2_gdiag, once per solve)
template <typename S, bool PRED>
__global__ void k2_prec(D2 D, CV<S> cv, const S* __restrict__ r, S* __restrict__ z) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const S ws = cv.wsc[c];
  if (!PRED) {
    for (int k = 0; k < g.K; ++k) z[(int64_t)k * g.nc + c] = ws * r[(int64_t)k * g.nc + c] * cv.gdi[(int64_t)k * g.nc + c];
    return;
  }
  const S al = cv.alpha[c];
  S num = r[(int64_t)g.K * g.nc + c];
  for (int k = 0; k < g.K; ++k) {
    const int64_t o = (int64_t)k * g.nc + c;
    num -= cv.w[k] * cv.gd[o] * r[o] * cv.gdi[o];
  }
  const S rho = num * cv.pdi[c];
  z[(int64_t)g.K * g.nc + c] = ws * rho;
  for (int k = 0; k < g.K; ++k) {
    const int64_t o = (int64_t)k * g.nc + c;
    z[o] = ws * (r[o] - (al + cv.gd[o]) * rho) * cv.gdi[o];
  }
}

// ----------------------------------------------------------------------------- Schur preconditioner
// Prediction preconditioner with the cells coupled (GRTE_PREC2D_MULTIGRID): block elimination of
// the (e, rho) system with (A + G_k)^{-1} replaced by its diagonal D_k = 1/(A + g_k),
//   f   = r_rho - sum_k w_k G_k D_k r_k
//   rho = S^{-1} f,   S = alpha + sum_k w_k G_k D_k beta   (beta = A - alpha)
//   e_k = D_k (r_k - alpha rho - G_k rho),
// with G_k applied exactly (vertex and cell passes) and S^{-1} one multigrid V-cycle
// (mg2d.cuh).  S is a 3x3 stencil on the cells, recovered once per solve by probing:
// the cells are coloured so that no two cells of a 3x3 neighbourhood share a colour,
// and S applied to the indicator of one colour gives, at every cell, the coupling to
// the one cell of that colour next to it.

// Colour of cell i along an axis of n cells: i mod 3, except on a periodic axis whose
// length is not a multiple of 3, where the sequence ends with 0 1 2 3 (n = 1 mod 3) or
// 0 1 2 3 0 1 2 3 (n = 2 mod 3) so that any three cyclically consecutive cells differ
// (n = 5 needs five colours, n <= 2 one per cell).
__host__ __device__ inline int axis_colour(int i, int n, int per) {
  if (!per || n % 3 == 0) return i % 3;
  if (n <= 2 || n == 5) return i;
  if (n % 3 == 1) return i < n - 4 ? i % 3 : i - (n - 4);
  return i < n - 8 ? i % 3 : (i - (n - 8)) % 4;
}
__host__ __device__ inline int axis_ncolours(int n, int per) {
  if (!per || n % 3 == 0) return n < 3 ? n : 3;
  if (n <= 2 || n == 5) return n;
  return 4;
}

// probe input: e_k = D_k beta on the cells of colour (cx, cy), 0 elsewhere
__global__ void k2_probe_in(D2 D, int cx, int cy, double* __restrict__ e) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (t >= (int64_t)g.K * g.nc) return;
  const int c = (int)(t % g.nc), p = c % g.Nx, q = c / g.Nx;
  const bool on = axis_colour(p, g.Nx, g.bcx == GRTE_BC_PERIODIC) == cx &&
                  axis_colour(q, g.Ny, g.bcy == GRTE_BC_PERIODIC) == cy;
  e[t] = on ? D.gdi[t] * (D.A[c] - D.alpha[c]) : 0.0;
}

// probe output: sum_k w_k tk (+ alpha on the diagonal) stored at the stencil position of
// the cell of colour (cx, cy) in the 3x3 neighbourhood (positions tried in the order
// 0, +1, -1 per axis: on a periodic axis of one or two cells several positions name the
// same cell and the coupling is stored once)
__global__ void k2_probe_out(D2 D, int cx, int cy, const double* __restrict__ tk, double* __restrict__ S0) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const int px = g.bcx == GRTE_BC_PERIODIC, py = g.bcy == GRTE_BC_PERIODIC;
  const int p = (int)(c % g.Nx), q = (int)(c / g.Nx);
  double v = 0.0;
  for (int k = 0; k < g.K; ++k) v += D.w[k] * tk[(int64_t)k * g.nc + c];
  const int order[3] = {0, 1, -1};
  for (int a = 0; a < 3; ++a) {
    const int dy = order[a], qn = mg::nbr(q, dy, g.Ny, py);
    if (qn < 0 || axis_colour(qn, g.Ny, py) != cy) continue;
    for (int b = 0; b < 3; ++b) {
      const int dx = order[b], pn = mg::nbr(p, dx, g.Nx, px);
      if (pn < 0 || axis_colour(pn, g.Nx, px) != cx) continue;
      if (pn == p && qn == q) v += D.alpha[c];
      S0[(int64_t)((dy + 1) * 3 + dx + 1) * g.nc + c] = v;
      return;
    }
  }
}

// Per-pair multigrid of the correction (mgpair2d.cuh): probe input e_k = 1 on the cells of
// colour (cx, cy) for every pair
__global__ void k2_mp_probe_in(D2 D, int cx, int cy, double* __restrict__ e) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (t >= (int64_t)g.K * g.nc) return;
  const int c = (int)(t % g.nc), p = c % g.Nx, q = c / g.Nx;
  e[t] = (axis_colour(p, g.Nx, g.bcx == GRTE_BC_PERIODIC) == cx && axis_colour(q, g.Ny, g.bcy == GRTE_BC_PERIODIC) == cy)
             ? 1.0 : 0.0;
}

// probe output: (A + G_k) e at cell c is the coupling of c to the one cell of colour
// (cx, cy) in its 3x3 neighbourhood, stored at that position of pair k's stencil
// (positions tried in the order 0, +1, -1 per axis, as for the prediction's stencil)
__global__ void k2_mp_probe_out(D2 D, int cx, int cy, const double* __restrict__ y, float* __restrict__ cr) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (t >= (int64_t)g.K * g.nc) return;
  const int k = (int)(t / g.nc);
  const int64_t c = t - (int64_t)k * g.nc;
  const int px = g.bcx == GRTE_BC_PERIODIC, py = g.bcy == GRTE_BC_PERIODIC;
  const int p = (int)(c % g.Nx), q = (int)(c / g.Nx);
  const int order[3] = {0, 1, -1};
  for (int a = 0; a < 3; ++a) {
    const int dy = order[a], qn = mg::nbr(q, dy, g.Ny, py);
    if (qn < 0 || axis_colour(qn, g.Ny, py) != cy) continue;
    for (int b = 0; b < 3; ++b) {
      const int dx = order[b], pn = mg::nbr(p, dx, g.Nx, px);
      if (pn < 0 || axis_colour(pn, g.Nx, px) != cx) continue;
      cr[((int64_t)k * 9 + (dy + 1) * 3 + dx + 1) * g.nc + c] = (float)y[t];
      return;
    }
  }
}

// the finest level's right side from a residual r (any type), and z = w x (the cell's
// Krylov scale)
template <typename S>
__global__ void k2_mp_in(int64_t n, const S* __restrict__ r, float* __restrict__ b) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)r[t];
}
template <typename S>
__global__ void k2_mp_out(D2 D, CV<S> cv, const float* __restrict__ x, S* __restrict__ z) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)D.g.K * D.g.nc) return;
  z[t] = cv.wsc[t % D.g.nc] * (S)x[t];
}

// et_k = D_k r_k
__global__ void k2_pc_et(D2 D, const double* __restrict__ r, double* __restrict__ et) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)D.g.K * D.g.nc) return;
  et[t] = D.gdi[t] * r[t];
}

// f = r_rho - sum_k w_k tk
__global__ void k2_pc_rhs(D2 D, const double* __restrict__ r, const double* __restrict__ tk, double* __restrict__ f) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  double s = r[(int64_t)g.K * g.nc + c];
  for (int k = 0; k < g.K; ++k) s -= D.w[k] * tk[(int64_t)k * g.nc + c];
  f[c] = s;
}

// z_k = w D_k (r_k - alpha rho - tk), z_rho = w rho  (tk = G_k rho; w the Krylov scale)
__global__ void k2_pc_final(D2 D, const double* __restrict__ r, const double* __restrict__ rho,
                            const double* __restrict__ tk, double* __restrict__ z) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  const int64_t ne = (int64_t)g.K * g.nc;
  if (t >= ne + g.nc) return;
  const int64_t c = t % g.nc;
  z[t] = t < ne ? D.wsc[c] * D.gdi[t] * (r[t] - D.alpha[c] * rho[c] - tk[t]) : D.wsc[c] * rho[c];
}

// gd[k][c] = diagonal of G_k at cell c (for the preconditioner), at the current coefficients
// and the reciprocals the preconditioner needs: gdi = 1/(A + g_k) and, per cell, the
// inverse of the arrow block's rho pivot alpha + sum_k w_k g_k (A - alpha)/(A + g_k).
__global__ void k2_gdiag(D2 D, CV<double> cv) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const int p = (int)(c % g.Nx), q = (int)(c / g.Nx);
  const double A = D.A[c], al = D.alpha[c];
  double den = al;
  for (int k = 0; k < g.K; ++k) {
    const int64_t o = (int64_t)k * g.nc + c;
    const double gk = gdiag(D, cv, k, p, q), inv = 1.0 / (A + gk);
    D.gd[o] = gk;
    D.gdi[o] = inv;
    den += D.w[k] * gk * (A - al) * inv;
  }
  D.pdi[c] = 1.0 / den;
}

// Krylov scale per cell from a magnitude field src: s = |src| + 1e-13 max|src| (or
// s = max|src| for every cell with uniform), w = f/s (f = 1 in the prediction, eps in the correction, whose unknown E_J enters
// E as eps E_J).
__global__ void k2_maxabs(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  double t = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    t = fmax(t, fabs(x[j]));
  for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmax(m, red[q]);
    part[blockIdx.x] = m;
  }
}

__global__ void k2_weights(D2 D, const double* __restrict__ src, double f, const double* __restrict__ part, int nb,
                           int uniform) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= D.g.nc) return;
  double m = 0.0;
  for (int b = 0; b < nb; ++b) m = fmax(m, part[b]);
  const double s = (uniform ? m : fabs(src[c]) + 1e-13 * m) + 1e-300;
  D.wsc[c] = f / s;
  D.iwsc[c] = s / f;
}

// magnitude of E^{n+1} per cell for the correction's scale: max(a c U, |rho*|)
__global__ void k2_corrscale(D2 D, double* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= D.g.nc) return;
  out[c] = fmax(D.acU[c], fabs(D.rho_s[c]));
}

// x[k][c] *= sc[c] over nvec stacked per-cell blocks
__global__ void k2_cellscale(double* __restrict__ x, const double* __restrict__ sc, int nvec, int64_t nc) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const double f = sc[c];
  for (int k = 0; k < nvec; ++k) x[(int64_t)k * nc + c] *= f;
}

// ----------------------------------------------------------------------------- right-hand sides
// Prediction: b_k = kappa E^n_k/(c dt) + s a c U^n - phi_k,
//             b_rho = kappa rho^n/(c dt) + s a c U^n - sum_k w_k phi_k;
// initial iterate e_k = E^n_k - rho^n, rho = rho^n.
__global__ void k2_rhs_pred(D2 D, const double* __restrict__ phi, double* __restrict__ b, double* __restrict__ x) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const double cdt = g.c * g.dt, sac = D.s[c] * g.a * g.c * D.U[c], kc = D.kc[c], rn = D.rho_n[c];
  double ps = 0.0;
  for (int k = 0; k < g.K; ++k) {
    const int64_t o = (int64_t)k * g.nc + c;
    b[o] = kc * D.E[o] / cdt + sac - phi[o];
    x[o] = D.E[o] - rn;
    ps += D.w[k] * phi[o];
  }
  b[(int64_t)g.K * g.nc + c] = kc * rn / cdt + sac - ps;
  x[(int64_t)g.K * g.nc + c] = rn;
}

// The correction's flux (sigma_0/T^3): the vertex coefficients of Eq. dis-cor-marshak1 take
// the multiplier V* = max(U*, 0)^{3/4} in place of the prediction's kappa = (T^n)^3;
// kc is set to V* here for k2_vcoef, and k2_coef restores it at T^{n+1} for substep 2.
__global__ void k2_vstar(D2 D) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= D.g.nc) return;
  D.kc[c] = pow(fmax(D.Us[c], 0.0), 0.25 * D.g.p);
}

// E*_k = rho + e_k, U* = (U^n + gamma rho)/(1 + gamma a c), rho* kept.
__global__ void k2_finish_pred(D2 D, const double* __restrict__ x, double* __restrict__ Es) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const double rho = x[(int64_t)g.K * g.nc + c];
  for (int k = 0; k < g.K; ++k) Es[(int64_t)k * g.nc + c] = rho + x[(int64_t)k * g.nc + c];
  D.rho_s[c] = rho;
  D.Us[c] = (D.U[c] + D.gam[c] * rho) / (1.0 + D.gam[c] * g.a * g.c);
}

// Correction: b_k = [kappa (E^n_k - a c U)/(c dt) - (G_k a c U) - phi_k]/eps, x = 0.
__global__ void k2_rhs_corr(D2 D, const double* __restrict__ GU, const double* __restrict__ phi,
                            double* __restrict__ b, double* __restrict__ x) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const double cdt = g.c * g.dt, kc = D.kc[c], acU = D.acU[c];
  for (int k = 0; k < g.K; ++k) {
    const int64_t o = (int64_t)k * g.nc + c;
    b[o] = (kc * (D.E[o] - acU) / cdt - GU[o] - phi[o]) / g.eps;
    x[o] = 0.0;
  }
}

// E^{n+1} = a c U + eps E_J (Eq. dis-proj), U = T^4
__global__ void k2_project(D2 D, const double* __restrict__ EJ) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const double acU = D.acU[c];
  for (int k = 0; k < g.K; ++k) {
    const int64_t o = (int64_t)k * g.nc + c;
    D.E[o] = acU + g.eps * EJ[o];
  }
  const double t = D.T[c];
  D.U[c] = (t * t) * (t * t);
}

// ----------------------------------------------------------------------------- Newton
// Features of the learned Newton start per cell (after the prediction), as in 1D:
// log10 T^n, log10 rho*, log10 sigma_eff, log10 eps, log10 dt, log10 Cv.
__global__ void k2_newton_feat(D2 D) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const double Tn = D.T[c], t3 = Tn * Tn * Tn;
  const double sig_eff = g.kind == GRTE_SIGMA_CONST ? D.sig[c]
                                                    : D.sig[c] / fmax(g.p == 3.0 ? t3 : pow(Tn, g.p), 1e-300);
  auto lg = [](double x) { return (float)log10(fmin(fmax(x, 1e-300), 1e300)); };
  float* f = D.feat + 6 * c;
  f[0] = lg(Tn);
  f[1] = lg(D.rho_s[c]);
  f[2] = lg(sig_eff);
  f[3] = lg(g.eps);
  f[4] = lg(g.dt);
  f[5] = lg(g.Cv);
}

// Eq. Tnp1 (sigma_0/T^3: Eq. dis-cor-marshak4 + 5) multiplied by sig:
//   A T^4 + B T = R,  A = sig a/dt,  B = sig Cv/dt + eps^2 kap Cv/(c dt^2),
//   R = sig (rho^n/(c dt) - Fdiv) + B T^n,  kap = 1 or max(U*, 0)^{3/4};
// Newton from T_hi = min((R/A)^{1/4}, R/B) decreases monotonically to the root.  With
// a learned start (network output y = log10(T^{n+1}/T^n), guess T^n 10^y, used where
// it lies more than 12% below T_hi: elsewhere T_hi is within the network's error of
// the root) or the previous-T
// start, one Newton step from the guess lands at or above the root (convex left
// side); the learned one is clamped to T_hi.
__global__ void k2_newton(D2 D) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const G2& g = D.g;
  if (c >= g.nc) return;
  const double sg = D.sig[c], Tn = D.T[c];
  const double kap = g.kind == GRTE_SIGMA_CONST ? 1.0 : pow(fmax(D.Us[c], 0.0), 0.25 * g.p);
  const double A = sg * g.a / g.dt;
  const double B = sg * g.Cv / g.dt + g.eps * g.eps * kap * g.Cv / (g.c * g.dt * g.dt);
  const double R = sg * (D.rho_n[c] / (g.c * g.dt) - D.Fdiv[c]) + B * Tn;
  double T = Tn;
  int its = 0;
  if (A == 0.0 && B == 0.0) {
    T = Tn;
  } else if (!(R > 0.0)) {
    T = 0.0;
    flag2(D.status, R <= 0.0 ? GRTE_ENEGATIVE : GRTE_ENAN);
  } else {
    double t = A > 0.0 ? sqrt(sqrt(R / A)) : INFINITY;
    if (B > 0.0) t = fmin(t, R / B);
    const double gl = D.use_guess ? Tn * exp10((double)D.guess[c]) : 0.0;
    const bool learned = D.use_guess && isfinite(gl) && gl > 0.0 && gl * kGuessGate2 < t;
    if (learned || D.start_prev) {
      const double gs = learned ? gl : Tn;
      if (isfinite(gs) && gs > 0.0) {
        const double g2 = gs * gs;
        const double t1 = gs - (A * g2 * g2 + B * gs - R) / (4.0 * A * g2 * gs + B);
        if (isfinite(t1) && t1 > 0.0) t = learned ? fmin(t, t1) : t1;
        ++its;
      }
    }
    for (its = its + 1; its <= D.newton_maxit; ++its) {
      const double t2 = t * t;
      const double f = A * t2 * t2 + B * t - R;
      const double fp = 4.0 * A * t2 * t + B;
      const double tn = t - f / fp;
      if (!(tn < t)) break;
      t = tn;
    }
    if (its > D.newton_maxit) flag2(D.status, GRTE_ENONCONV);
    T = t;
  }
  D.T[c] = T;
  D.newton_its[c] = (double)its;
  if (D.log_samples) D.ytrue[c] = (T > 0.0 && Tn > 0.0) ? (float)log10(T / Tn) : 0.0f;
}

// ----------------------------------------------------------------------------- vector kernels
// Partial dot products of w with V_0..V_{nvec-1} (stride n): one value per (block, vec),
// fixed order; k2_reduce sums the block partials (one block per value).  The vectors go
// in chunks of C (w read once per chunk), each thread keeping C sums in the vectors'
// precision S; the block sums are binary64.  All C loads of an element are issued
// unconditionally (a chunk's missing vectors read its last one and are masked out), so
// they are in flight together; the warp sums are formed in S and widened once.
template <typename S, int C>
__global__ void __launch_bounds__(kThreads, 2) k2_mdot(const S* __restrict__ w, const S* __restrict__ V, int nvec,
                                                     int64_t n, double* __restrict__ part) {
  __shared__ double red[kThreads / 32][C];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i0 = 0; i0 < nvec; i0 += C) {
    const int nv = min(C, nvec - i0);
    const S* Vb = V + (int64_t)i0 * n;
    S acc[C];
#pragma unroll
    for (int t = 0; t < C; ++t) acc[t] = S(0);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      const S wj = w[j];
      S vt[C];
#pragma unroll
      for (int t = 0; t < C; ++t) vt[t] = Vb[(int64_t)min(t, nv - 1) * n + j];
#pragma unroll
      for (int t = 0; t < C; ++t) acc[t] = t < nv ? fma(wj, vt[t], acc[t]) : acc[t];
    }
#pragma unroll
    for (int t = 0; t < C; ++t) {
      S v = acc[t];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid][t] = (double)v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nv; t += blockDim.x) {
      double u = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) u += red[q][t];
      part[(int64_t)(i0 + t) * gridDim.x + blockIdx.x] = u;
    }
    __syncthreads();
  }
}

__global__ void k2_reduce(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) t += part[(int64_t)blockIdx.x * nb + b];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    out[blockIdx.x] = s;
  }
}

// k2_reduce for the Gram-Schmidt coefficients: coef[b] = sum of value b's partials and
// the Hessenberg column hcol[b] (+)= coef[b] (first pass: assign)
__global__ void k2_reduce_h(const double* __restrict__ part, int nb, double* __restrict__ coef,
                            double* __restrict__ hcol, int assign) {
  __shared__ double red[kThreads / 32];
  double t = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) t += part[(int64_t)blockIdx.x * nb + b];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    coef[blockIdx.x] = s;
    hcol[blockIdx.x] = assign ? s : hcol[blockIdx.x] + s;
  }
}

// w -= sum_i coef[i] V_i (coefficients staged in shared memory in the vectors' precision,
// four independent partial sums per element); with NORM also the block partials of
// |w|^2 of the result (binary64).
template <typename S, bool NORM>
__global__ void __launch_bounds__(kThreads) k2_maxpy(S* __restrict__ w, const S* __restrict__ V,
                                                      const double* __restrict__ coef, int nvec, int64_t n,
                                                      double* __restrict__ part) {
  __shared__ S cf[kMaxRestart2 + 1];
  __shared__ double red[kThreads / 32];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) cf[i] = S(coef[i]);
  __syncthreads();
  S nrm = S(0);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    S t0 = w[j], t1 = S(0), t2 = S(0), t3 = S(0);
    int i = 0;
    for (; i + 4 <= nvec; i += 4) {
      t0 = fma(-cf[i], V[(int64_t)i * n + j], t0);
      t1 = fma(-cf[i + 1], V[(int64_t)(i + 1) * n + j], t1);
      t2 = fma(-cf[i + 2], V[(int64_t)(i + 2) * n + j], t2);
      t3 = fma(-cf[i + 3], V[(int64_t)(i + 3) * n + j], t3);
    }
    for (; i < nvec; ++i) t0 = fma(-cf[i], V[(int64_t)i * n + j], t0);
    const S r = (t0 + t1) + (t2 + t3);
    w[j] = r;
    if (NORM) nrm = fma(r, r, nrm);
  }
  if (NORM) {
    double v = nrm;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double u = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) u += red[q];
      part[blockIdx.x] = u;
    }
  }
}

// x += sum_i coef[i] V_i (x binary64; binary32 basis vectors: the combination is formed
// in binary32 and added once)
template <typename S>
__global__ void k2_update(double* __restrict__ x, const S* __restrict__ V, const double* __restrict__ coef, int nvec,
                          int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(S) == 8) {
      double t = x[j];
      for (int i = 0; i < nvec; ++i) t += coef[i] * V[(int64_t)i * n + j];
      x[j] = t;
    } else {
      S t = S(0);
      for (int i = 0; i < nvec; ++i) t = fma(S(coef[i]), V[(int64_t)i * n + j], t);
      x[j] += (double)t;
    }
  }
}

template <typename S>
__global__ void k2_scale(S* __restrict__ x, double s, int64_t n) {
  const S f = S(s);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    x[j] *= f;
}

// binary32 copy dst = src * f
__global__ void k2_tof(const double* __restrict__ src, float* __restrict__ dst, int64_t n, double f) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = (float)(src[j] * f);
}

// y = b - y
__global__ void k2_bminus(const double* __restrict__ b, double* __restrict__ y, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    y[j] = b[j] - y[j];
}

__global__ void k2_energy(D2 D, double* __restrict__ part) {
  __shared__ double red[kThreads / 32];
  const G2& g = D.g;
  double t = 0.0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < g.nc; c += (int64_t)gridDim.x * blockDim.x) {
    double rho = 0.0;
    for (int k = 0; k < g.K; ++k) rho += D.w[k] * D.E[(int64_t)k * g.nc + c];
    t += g.dx * g.dy * (rho / g.c + g.Cv * D.T[c]);
  }
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    part[blockIdx.x] = s;
  }
}

// Level-symmetric S8 pairs for 2D (80 directions on the sphere: cosine levels
// mu_i^2 = (1 + 6 i)/21, i = 0..3; per octant the permutations of the level triples
// (0,0,3), (0,1,2), (1,1,1), three weight classes fixed by the moments sum w = 1,
// sum w mu^4 = 1/5, sum w mu^6 = 1/7; the 40 directions with a positive third cosine,
// projected on the plane, form 20 pairs; each pair is represented by its member with
// mu > 0 and weighs its two members).  Sorted by (mu, eta).
static void s8_pairs(std::vector<double>& mu, std::vector<double>& eta, std::vector<double>& w) {
  double m[4], lv[4];
  for (int i = 0; i < 4; ++i) {
    m[i] = (1.0 + 6.0 * i) / 21.0;
    lv[i] = std::sqrt(m[i]);
  }
  struct Dir { int a, b, c, cls; };
  std::vector<Dir> oct;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c)
        if (a + b + c == 3) {
          int s[3] = {a, b, c};
          std::sort(s, s + 3);
          const int cls = (s[0] == 0 && s[1] == 0) ? 0 : (s[0] == 1 && s[1] == 1) ? 2 : 1;
          oct.push_back({a, b, c, cls});
        }
  double M[3][4] = {{0}};
  for (const Dir& d : oct) {
    M[0][d.cls] += 8.0;
    M[1][d.cls] += 8.0 * m[d.a] * m[d.a];
    M[2][d.cls] += 8.0 * m[d.a] * m[d.a] * m[d.a];
  }
  M[0][3] = 1.0;
  M[1][3] = 1.0 / 5.0;
  M[2][3] = 1.0 / 7.0;
  for (int col = 0; col < 3; ++col) {   // Gauss-Jordan with partial pivoting on 3x3
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
    for (int cc = 0; cc < 4; ++cc) std::swap(M[col][cc], M[piv][cc]);
    for (int r = 0; r < 3; ++r) {
      if (r == col) continue;
      const double f = M[r][col] / M[col][col];
      for (int cc = 0; cc < 4; ++cc) M[r][cc] -= f * M[col][cc];
    }
  }
  const double wc[3] = {M[0][3] / M[0][0], M[1][3] / M[1][1], M[2][3] / M[2][2]};
  struct P { double mu, eta, w; };
  std::vector<P> ps;
  double tot = 0.0;
  // the member with mu > 0 and third cosine > 0 of each pair; the pair's weight is that
  // of (mu, eta, xi) plus that of (-mu, -eta, xi)
  for (int sy = 0; sy < 2; ++sy)
    for (const Dir& d : oct) {
      const double x = lv[d.a], y = (sy == 0 ? 1.0 : -1.0) * lv[d.b];
      ps.push_back({x, y, 2.0 * wc[d.cls]});
      tot += 2.0 * wc[d.cls];
    }
  std::sort(ps.begin(), ps.end(), [](const P& l, const P& r) { return l.mu < r.mu || (l.mu == r.mu && l.eta < r.eta); });
  mu.clear(); eta.clear(); w.clear();
  for (const P& p : ps) {
    mu.push_back(p.mu);
    eta.push_back(p.eta);
    w.push_back(p.w / tot);
  }
}

}  // namespace grte2

// =============================================================================== host
using namespace grte2;

// Kernel launches made by this thread (every launch site increments it); grte2d_step
// reports the difference over the call in grte_stats_t.launches.
static thread_local int64_t tl_launches = 0;

struct grte2d_ctx {
  D2 D{};
  G2 g{};
  grte_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool state_set = false;
  std::vector<double> hmu, heta, hw;
  std::vector<void*> allocs;
  std::string err;
  grte_stats_t stats{};
  int host_flags = 0;   // statuses found on the host (a solve that missed its tolerance)
  int m = 30;
  double *V = nullptr, *phi = nullptr, *GU = nullptr, *Es = nullptr;
  double *b = nullptr, *x = nullptr, *Kr = nullptr, *Kt = nullptr, *Kbasis = nullptr;
  double *part = nullptr, *dots = nullptr, *coef = nullptr, *cscale = nullptr, *hcol = nullptr;
  double* tk = nullptr;   // [k][cell] per-pair cell values summed by k2_cellsum
  grte_mlp_t mlp = nullptr;   // learned Newton start (not owned)
  CV<double> cv{};            // the binary64 coefficient view of D
  // mixed precision: binary32 copies of the coefficients (cv32) and the binary32 Krylov
  // cycle's buffers (basis, matrix-vector product, vertex values, per-pair cell values)
  bool mixed = false;
  CV<float> cv32{};
  float *mu32 = nullptr, *eta32 = nullptr, *w32 = nullptr, *kc32 = nullptr, *A32 = nullptr, *alpha32 = nullptr;
  float *dv32 = nullptr, *gd32 = nullptr, *gdi32 = nullptr, *pdi32 = nullptr, *wsc32 = nullptr, *iwsc32 = nullptr;
  float *V32 = nullptr, *Kr32 = nullptr, *Vv32 = nullptr, *tk32 = nullptr;
  std::vector<mg::Level> mgl;        // multigrid levels of the Schur preconditioner (empty: per-cell block only)
  double *mg_M = nullptr, *mg_inv = nullptr;   // coarsest level: dense scratch and inverse
  // correction substep 2: per-pair multigrid (GRTE_PREC2D_CORR_MG), its V-cycle as one graph
  std::vector<mp::PLevel> mpl;
  cudaGraphExec_t mp_graph = nullptr;
  double* mp_probe = nullptr;   // [k][cell] probe input
  int mp_nodes = 0;             // kernel launches of one V-cycle graph
  double *dmu = nullptr, *deta = nullptr, *dw = nullptr, *dsig = nullptr;
};

static grte_status fail2(grte2d_t h, grte_status s, const std::string& m) {
  if (h) h->err = m;
  return s;
}
#define CK2(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail2(h, GRTE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static unsigned grid_of(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

template <typename T>
static bool alloc2(grte2d_t h, T** p, int64_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, sizeof(T) * (size_t)std::max<int64_t>(n, 1)) != cudaSuccess) return false;
  cudaMemset(q, 0, sizeof(T) * (size_t)std::max<int64_t>(n, 1));
  h->allocs.push_back(q);
  *p = (T*)q;
  return true;
}

template <typename S>
static void launch_mdot(const S* w, const S* V, int nvec, int64_t n, double* part, cudaStream_t st) {
  if (nvec <= 4) tl_launches++, k2_mdot<S, 4><<<kDotBlocks, kThreads, 0, st>>>(w, V, nvec, n, part);
  else if (nvec <= 8) tl_launches++, k2_mdot<S, 8><<<kDotBlocks, kThreads, 0, st>>>(w, V, nvec, n, part);
  else tl_launches++, k2_mdot<S, 16><<<kDotBlocks, kThreads, 0, st>>>(w, V, nvec, n, part);
}

// dots[i] = <w, V_i>, i < nvec, returned on the host.
static grte_status mdot(grte2d_t h, const double* w, const double* V, int nvec, int64_t n, double* host) {
  cudaStream_t st = h->stream;
  launch_mdot<double>(w, V, nvec, n, h->part, st);
  tl_launches++, k2_reduce<<<nvec, kThreads, 0, st>>>(h->part, kDotBlocks, h->dots);
  CK2(cudaGetLastError());
  CK2(cudaMemcpyAsync(host, h->dots, sizeof(double) * nvec, cudaMemcpyDeviceToHost, st));
  CK2(cudaStreamSynchronize(st));
  return GRTE_OK;
}

// y = M x (pred: the (e, rho) matrix; corr: the stacked A + G_k), through the vertex
// and cell passes.  The Krylov unknowns are w-scaled: they are unscaled on the way in.
static void apply_M(grte2d_t h, bool pred, const double* xin, double* y) {
  D2& D = h->D;
  cudaStream_t st = h->stream;
  UField u{xin, D.g.nc, pred ? xin + (int64_t)D.g.K * D.g.nc : nullptr, D.iwsc};
  const int64_t K = D.g.K;
  tl_launches++, k2_vertex<double, false><<<grid_of(K * D.g.nv), kThreads, 0, st>>>(D, h->cv, u, h->V);
  if (pred) {
    tl_launches++, k2_cell<double, C_MV_PRED, false><<<grid_of(K * D.g.nc), kThreads, 0, st>>>(D, h->cv, h->V, u, xin, y, D.iwsc, h->tk);
    tl_launches++, k2_cellsum<double, C_MV_PRED><<<grid_of(D.g.nc), kThreads, 0, st>>>(D, h->cv, h->tk, xin, y, D.iwsc);
  } else {
    tl_launches++, k2_cell<double, C_MV_CORR, false><<<grid_of(K * D.g.nc), kThreads, 0, st>>>(D, h->cv, h->V, u, xin, y, D.iwsc, h->tk);
  }
}

// binary32 matrix and block preconditioner (mixed precision Krylov cycles)
static void apply_M32(grte2d_t h, bool pred, const float* xin, float* y) {
  D2& D = h->D;
  cudaStream_t st = h->stream;
  const int64_t K = D.g.K, nc = D.g.nc;
  UFieldT<float> u{xin, nc, pred ? xin + K * nc : nullptr, h->cv32.iwsc};
  tl_launches++, k2_vertex<float, false><<<grid_of(K * D.g.nv), kThreads, 0, st>>>(D, h->cv32, u, h->Vv32);
  if (pred) {
    tl_launches++, k2_cell<float, C_MV_PRED, false><<<grid_of(K * nc), kThreads, 0, st>>>(D, h->cv32, h->Vv32, u, xin, y,
                                                                         h->cv32.iwsc, h->tk32);
    tl_launches++, k2_cellsum<float, C_MV_PRED><<<grid_of(nc), kThreads, 0, st>>>(D, h->cv32, h->tk32, xin, y, h->cv32.iwsc);
  } else {
    tl_launches++, k2_cell<float, C_MV_CORR, false><<<grid_of(K * nc), kThreads, 0, st>>>(D, h->cv32, h->Vv32, u, xin, y,
                                                                         h->cv32.iwsc, h->tk32);
  }
}

// One V-cycle of the per-pair multigrid on level l (right side in mpl[l].b, iterate in
// mpl[l].x, zero on entry); returns the kernels launched.  Issued once under stream capture.
static int mp_vcycle(grte2d_t h, size_t l) {
  cudaStream_t st = h->stream;
  const mp::PLevel& L = h->mpl[l];
  const bool coarsest = l + 1 == h->mpl.size();
  int nl = 0;
  const dim3 tb(32, 8);
  const dim3 trc((L.nx + 31) / 32, (L.ny + 31) / 32, L.K), tcr((L.ny + 31) / 32, (L.nx + 31) / 32, L.K);
  mp::mp_transpose<<<trc, tb, 0, st>>>(L.b, L.bt, L.nx, L.ny, L.K);
  ++nl;
  auto lines = [&](const float* coef, float* x, const float* b, int nf, int ns, int perf, int pers) {
    for (int par = 0; par < 2; ++par) {
      const int64_t nt = (int64_t)L.K * ((nf - par + 1) / 2);
      if (nt == 0) continue;
      mp::mp_line<<<(unsigned)((nt + mp::kThreadsMp - 1) / mp::kThreadsMp), mp::kThreadsMp, 0, st>>>(
          coef, x, b, L.cp, nf, ns, L.K, perf, pers, par);
      ++nl;
    }
  };
  auto sweep_y = [&]() { lines(L.cr, L.x, L.b, L.nx, L.ny, L.perx, L.pery); };
  auto sweep_x = [&]() {
    mp::mp_transpose<<<trc, tb, 0, st>>>(L.x, L.xt, L.nx, L.ny, L.K);
    lines(L.ct, L.xt, L.bt, L.ny, L.nx, L.pery, L.perx);
    mp::mp_transpose<<<tcr, tb, 0, st>>>(L.xt, L.x, L.ny, L.nx, L.K);
    nl += 2;
  };
  for (int sw = 0; sw < (coarsest ? mp::kCoarseSweeps : 1); ++sw) {
    sweep_y();
    sweep_x();
  }
  if (!coarsest) {
    const mp::PLevel& C = h->mpl[l + 1];
    mp::mp_restrict<<<grid_of((int64_t)C.K * C.n), kThreads, 0, st>>>(L, C);
    ++nl;
    nl += mp_vcycle(h, l + 1);
    mp::mp_prolong<<<grid_of((int64_t)L.K * L.n), kThreads, 0, st>>>(L, C);
    ++nl;
    sweep_x();
    sweep_y();
  }
  return nl;
}

// Per solve: the finest level's stencils by probing the correction operator, the Galerkin
// levels and the transposed copies; the V-cycle graph is captured on first use (its
// buffers are fixed for the handle's lifetime).
static grte_status mp_setup(grte2d_t h) {
  D2& D = h->D;
  const G2& g = D.g;
  cudaStream_t st = h->stream;
  const int64_t K = g.K, nc = g.nc;
  mp::PLevel& L0 = h->mpl[0];
  const int px = g.bcx == GRTE_BC_PERIODIC, py = g.bcy == GRTE_BC_PERIODIC;
  const int ncx = axis_ncolours(g.Nx, px), ncy = axis_ncolours(g.Ny, py);
  CK2(cudaMemsetAsync(L0.cr, 0, sizeof(float) * 9 * K * nc, st));
  for (int cy = 0; cy < ncy; ++cy)
    for (int cx = 0; cx < ncx; ++cx) {
      tl_launches++, k2_mp_probe_in<<<grid_of(K * nc), kThreads, 0, st>>>(D, cx, cy, h->mp_probe);
      tl_launches++, k2_vertex<double, false><<<grid_of(K * g.nv), kThreads, 0, st>>>(D, h->cv, UField{h->mp_probe, nc, nullptr}, h->V);
      tl_launches++, k2_cell<double, C_MV_CORR, false><<<grid_of(K * nc), kThreads, 0, st>>>(
          D, h->cv, h->V, UField{h->mp_probe, nc, nullptr}, h->mp_probe, h->Kr, nullptr, h->tk);
      tl_launches++, k2_mp_probe_out<<<grid_of(K * nc), kThreads, 0, st>>>(D, cx, cy, h->Kr, L0.cr);
    }
  for (size_t l = 0; l < h->mpl.size(); ++l) {
    const mp::PLevel& L = h->mpl[l];
    if (l > 0) tl_launches++, mp::mp_galerkin<<<grid_of((int64_t)L.K * L.n), kThreads, 0, st>>>(h->mpl[l - 1], L);
    tl_launches++, mp::mp_stencil_t<<<grid_of((int64_t)L.K * L.n), kThreads, 0, st>>>(L);
  }
  CK2(cudaGetLastError());
  if (!h->mp_graph) {
    cudaGraph_t gr = nullptr;
    CK2(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(L0.x, 0, sizeof(float) * K * nc, st);
    h->mp_nodes = mp_vcycle(h, 0);
    CK2(cudaStreamEndCapture(st, &gr));
    const cudaError_t e = cudaGraphInstantiate(&h->mp_graph, gr, 0);
    cudaGraphDestroy(gr);
    CK2(e);
  }
  return GRTE_OK;
}

// z = w V-cycle(r) per pair (correction, GRTE_PREC2D_CORR_MG)
template <typename S>
static void mp_apply(grte2d_t h, const CV<S>& cv, const S* r, S* z) {
  const int64_t n = h->D.g.K * h->D.g.nc;
  cudaStream_t st = h->stream;
  tl_launches++, k2_mp_in<S><<<grid_of(n), kThreads, 0, st>>>(n, r, h->mpl[0].b);
  cudaGraphLaunch(h->mp_graph, st);
  tl_launches += h->mp_nodes;
  tl_launches++, k2_mp_out<S><<<grid_of(n), kThreads, 0, st>>>(h->D, cv, h->mpl[0].x, z);
}

static void apply_P32(grte2d_t h, bool pred, const float* r, float* z) {
  if (!pred && h->mp_graph) {
    mp_apply<float>(h, h->cv32, r, z);
    return;
  }
  if (pred) tl_launches++, k2_prec<float, true><<<grid_of(h->D.g.nc), kThreads, 0, h->stream>>>(h->D, h->cv32, r, z);
  else tl_launches++, k2_prec<float, false><<<grid_of(h->D.g.nc), kThreads, 0, h->stream>>>(h->D, h->cv32, r, z);
}

static void tof(grte2d_t h, const double* src, float* dst, int64_t n) {
  tl_launches++, k2_tof<<<kAxpyBlocks, kThreads, 0, h->stream>>>(src, dst, n, 1.0);
}

// binary32 copies of the coefficients a solve's Krylov cycles read (after k2_gdiag)
static void mirror_coefficients(grte2d_t h) {
  if (!h->mixed) return;
  const D2& D = h->D;
  const int64_t K = D.g.K, nc = D.g.nc;
  tof(h, D.kc, h->kc32, nc);
  tof(h, D.A, h->A32, nc);
  tof(h, D.alpha, h->alpha32, nc);
  tof(h, D.dv, h->dv32, D.g.nv);
  tof(h, D.gd, h->gd32, K * nc);
  tof(h, D.gdi, h->gdi32, K * nc);
  tof(h, D.pdi, h->pdi32, nc);
}

// One V-cycle on level l (right side in mgl[l].b); returns the buffer holding the result.
static const double* mg_vcycle(grte2d_t h, size_t l) {
  cudaStream_t st = h->stream;
  mg::Level& L = h->mgl[l];
  const unsigned gb = grid_of(L.n);
  if (l + 1 == h->mgl.size()) {
    tl_launches++, mg::mg_dense_apply<<<1, mg::kThreadsMg, 0, st>>>(L, h->mg_inv);
    return L.x;
  }
  mg::Level& C = h->mgl[l + 1];
  const unsigned gcb = grid_of(C.n);
  tl_launches++, mg::mg_jacobi0<<<gb, kThreads, 0, st>>>(L);
  if (L.ncomp == 1) {
    tl_launches++, mg::mg_jacobi<1><<<gb, kThreads, 0, st>>>(L, L.x, L.xt, nullptr, C);
    tl_launches++, mg::mg_restrict<1><<<gcb, kThreads, 0, st>>>(L, L.xt, C);
  } else {
    tl_launches++, mg::mg_jacobi<2><<<gb, kThreads, 0, st>>>(L, L.x, L.xt, nullptr, C);
    tl_launches++, mg::mg_restrict<2><<<gcb, kThreads, 0, st>>>(L, L.xt, C);
  }
  const double* xc = mg_vcycle(h, l + 1);
  if (L.ncomp == 1) {
    tl_launches++, mg::mg_jacobi<1><<<gb, kThreads, 0, st>>>(L, L.xt, L.x, xc, C);
    tl_launches++, mg::mg_jacobi<1><<<gb, kThreads, 0, st>>>(L, L.x, L.xt, nullptr, C);
  } else {
    tl_launches++, mg::mg_jacobi<2><<<gb, kThreads, 0, st>>>(L, L.xt, L.x, xc, C);
    tl_launches++, mg::mg_jacobi<2><<<gb, kThreads, 0, st>>>(L, L.x, L.xt, nullptr, C);
  }
  return L.xt;
}

// Probe S (3x3 stencil into level 0) at the current coefficients and build the
// coarse levels; after k2_gdiag.
static void mg_setup(grte2d_t h) {
  D2& D = h->D;
  const G2& g = D.g;
  cudaStream_t st = h->stream;
  const int64_t K = g.K, nc = g.nc;
  mg::Level& L0 = h->mgl[0];
  cudaMemsetAsync(L0.coef, 0, sizeof(double) * 9 * nc, st);
  const int px = g.bcx == GRTE_BC_PERIODIC, py = g.bcy == GRTE_BC_PERIODIC;
  const int ncx = axis_ncolours(g.Nx, px), ncy = axis_ncolours(g.Ny, py);
  for (int cy = 0; cy < ncy; ++cy)
    for (int cx = 0; cx < ncx; ++cx) {
      tl_launches++, k2_probe_in<<<grid_of(K * nc), kThreads, 0, st>>>(D, cx, cy, h->Kt);
      tl_launches++, k2_vertex<double, false><<<grid_of(K * g.nv), kThreads, 0, st>>>(D, h->cv, UField{h->Kt, nc, nullptr}, h->V);
      tl_launches++, k2_cell<double, C_DIVK, false><<<grid_of(K * nc), kThreads, 0, st>>>(D, h->cv, h->V, UField{h->Kt, nc, nullptr}, nullptr,
                                                                   h->tk, nullptr, nullptr);
      tl_launches++, k2_probe_out<<<grid_of(nc), kThreads, 0, st>>>(D, cx, cy, h->tk, L0.coef);
    }
  tl_launches++, mg::mg_idiag0<<<grid_of(nc), kThreads, 0, st>>>(L0);
  for (size_t l = 0; l + 1 < h->mgl.size(); ++l) {
    mg::Level &F = h->mgl[l], &C = h->mgl[l + 1];
    if (F.ncomp == 1) tl_launches++, mg::mg_galerkin<1><<<grid_of(C.n), kThreads, 0, st>>>(F, C);
    else tl_launches++, mg::mg_galerkin<2><<<grid_of(C.n), kThreads, 0, st>>>(F, C);
  }
  mg::Level& Lc = h->mgl.back();
  if (Lc.ncomp == 1) tl_launches++, mg::mg_dense_inverse<1><<<1, mg::kThreadsMg, 0, st>>>(Lc, h->mg_M, h->mg_inv);
  else tl_launches++, mg::mg_dense_inverse<2><<<1, mg::kThreadsMg, 0, st>>>(Lc, h->mg_M, h->mg_inv);
}

static void apply_P(grte2d_t h, bool pred, bool use_mg, const double* r, double* z) {
  D2& D = h->D;
  cudaStream_t st = h->stream;
  if (!pred) {
    if (h->mp_graph) mp_apply<double>(h, h->cv, r, z);
    else tl_launches++, k2_prec<double, false><<<grid_of(D.g.nc), kThreads, 0, st>>>(D, h->cv, r, z);
    return;
  }
  if (!use_mg) {
    tl_launches++, k2_prec<double, true><<<grid_of(D.g.nc), kThreads, 0, st>>>(D, h->cv, r, z);
    return;
  }
  const int64_t K = D.g.K, nc = D.g.nc;
  tl_launches++, k2_pc_et<<<grid_of(K * nc), kThreads, 0, st>>>(D, r, h->Kt);
  tl_launches++, k2_vertex<double, false><<<grid_of(K * D.g.nv), kThreads, 0, st>>>(D, h->cv, UField{h->Kt, nc, nullptr}, h->V);
  tl_launches++, k2_cell<double, C_DIVK, false><<<grid_of(K * nc), kThreads, 0, st>>>(D, h->cv, h->V, UField{h->Kt, nc, nullptr}, nullptr, h->tk,
                                                               nullptr, nullptr);
  tl_launches++, k2_pc_rhs<<<grid_of(nc), kThreads, 0, st>>>(D, r, h->tk, h->mgl[0].b);
  const double* rho = mg_vcycle(h, 0);
  tl_launches++, k2_vertex<double, false><<<grid_of(K * D.g.nv), kThreads, 0, st>>>(D, h->cv, UField{nullptr, 0, rho}, h->V);
  tl_launches++, k2_cell<double, C_DIVK, false><<<grid_of(K * nc), kThreads, 0, st>>>(D, h->cv, h->V, UField{nullptr, 0, rho}, nullptr, h->tk,
                                                               nullptr, nullptr);
  tl_launches++, k2_pc_final<<<grid_of((K + 1) * nc), kThreads, 0, st>>>(D, r, rho, h->tk, z);
}

// One Arnoldi step in precision S: w = V_{j+1} = D_w P^{-1} M D_w^{-1} V_j (binary32: the
// binary32 matrix and block preconditioner), orthogonalised against V_0..V_j by classical
// Gram-Schmidt (the coefficients stay on the device; the last pass's update also gives
// |w|^2); hc receives the Hessenberg column, hc[j+1] = |w|^2 (w not normalised).
template <typename S>
static grte_status arnoldi_step(grte2d_t h, bool pred, bool mg_stage, S* V, int j, int64_t n, std::vector<double>& hc) {
  cudaStream_t st = h->stream;
  S* vj = V + (int64_t)j * n;
  S* w = V + (int64_t)(j + 1) * n;
  if constexpr (sizeof(S) == 8) {
    apply_M(h, pred, vj, h->Kr);
    apply_P(h, pred, mg_stage, h->Kr, w);
  } else {
    apply_M32(h, pred, vj, h->Kr32);
    apply_P32(h, pred, h->Kr32, w);
  }
  // binary32 cycles: one pass (a cycle only has to gain 1e5 and the binary64 restart
  // corrects what the basis's loss of orthogonality costs); binary64: two passes
  const int passes = sizeof(S) == 4 ? 1 : 2;
  for (int pass = 0; pass < passes; ++pass) {
    launch_mdot<S>(w, V, j + 1, n, h->part, st);
    tl_launches++, k2_reduce_h<<<j + 1, kThreads, 0, st>>>(h->part, kDotBlocks, h->coef, h->hcol, pass == 0);
    if (pass + 1 < passes) {
      tl_launches++, k2_maxpy<S, false><<<kAxpyBlocks, kThreads, 0, st>>>(w, V, h->coef, j + 1, n, nullptr);
    } else {
      tl_launches++, k2_maxpy<S, true><<<kAxpyBlocks, kThreads, 0, st>>>(w, V, h->coef, j + 1, n, h->part);
      tl_launches++, k2_reduce<<<1, kThreads, 0, st>>>(h->part, kAxpyBlocks, h->hcol + j + 1);
    }
  }
  CK2(cudaGetLastError());
  CK2(cudaMemcpyAsync(hc.data(), h->hcol, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, st));
  CK2(cudaStreamSynchronize(st));
  return GRTE_OK;
}

// Restarted GMRES(m) with left preconditioning on M x = b (x holds the initial
// iterate).  Each restart cycle runs on the cell-scaled unknowns y = D_w x, D_w the
// diagonal of the per-cell scale w computed from the current iterate (prediction:
// w = 1/|rho|; correction: w = eps/max(a c U, |rho*|)), a similarity transform
// D_w P^{-1} M D_w^{-1} that keeps the preconditioned spectrum.  In those units every
// cell's unknowns are O(1), so the test |D_w P^{-1}(b - M x)|_2 <= rtol sqrt(n_cells)
// bounds the residual of every cell relative to the cell's own magnitude (RMS).
//
// Mixed precision: every restart still forms the residual and updates x in binary64,
// but the cycle's Krylov process (basis, matrix, block preconditioner, Gram-Schmidt)
// runs in binary32 and ends once it has reduced the residual by kInnerReduce (about
// the most a binary32 cycle can do reliably): restarted GMRES as iterative refinement,
// whose accuracy is set by the binary64 residual.  rtol is floored at kMixedRtol (the
// test is an RMS over cells; 1e-9 left single cells ~1e-5 off in T at 512^2).
//
// mg_stage (prediction, multigrid preconditioner, binary64): the same iteration with
// one scale for all cells (w = 1/max|rho|).  The multigrid couples the cells, and
// under per-cell scales its error terms from hot cells into cold ones are multiplied by
// the ratio of their magnitudes (up to ~1e8 across a front), which stalls the
// iteration; with one scale it converges in a few iterations to rtol relative to the
// largest cell.  It ends there, or when a restart no longer gains 4x, or a cycle stops
// falling (less than 2x over four iterations after a 1e6 reduction), and never flags
// ENONCONV: the per-cell scaled solve with the per-cell block preconditioner then runs
// from its iterate and decides convergence (the cold, opaque cells it still has to fix
// are nearly local).
static grte_status gmres2(grte2d_t h, bool pred, bool mg_stage, int64_t n, int& iters) {
  cudaStream_t st = h->stream;
  D2& D = h->D;
  const int nblk = pred ? D.g.K + 1 : D.g.K;
  const unsigned gc = grid_of(D.g.nc);
  const int m = h->m;
  double* V = h->Kbasis;
  const bool f32 = h->mixed && !mg_stage;
  std::vector<double> H((size_t)(m + 1) * m, 0.0), g(m + 1), cs(m), sn(m), yv(m);
  const unsigned vb = kAxpyBlocks;
  const double rtol = h->mixed ? std::max(h->opt.krylov_rtol, kMixedRtol) : h->opt.krylov_rtol;
  const double thr = rtol * std::sqrt((double)D.g.nc);
  const int maxcycles = mg_stage ? kMgStageCycles : h->opt.krylov_maxcycles;
  grte_status s = GRTE_OK;
  iters = 0;
  auto set_scale = [&]() {
    const double* src = pred ? h->x + (int64_t)D.g.K * D.g.nc : h->cscale;
    tl_launches++, k2_maxabs<<<kRedBlocks, kThreads, 0, st>>>(src, D.g.nc, h->part);
    tl_launches++, k2_weights<<<gc, kThreads, 0, st>>>(D, src, pred ? 1.0 : D.g.eps, h->part, kRedBlocks, mg_stage ? 1 : 0);
    if (f32) {
      tof(h, D.wsc, h->wsc32, D.g.nc);
      tof(h, D.iwsc, h->iwsc32, D.g.nc);
    }
  };
  // the true scaled residual of the unscaled x, into V_0; returns its norm
  auto residual = [&](double* beta) -> grte_status {
    set_scale();
    tl_launches++, k2_cellscale<<<gc, kThreads, 0, st>>>(h->x, D.wsc, nblk, D.g.nc);   // x -> y
    apply_M(h, pred, h->x, h->Kr);
    tl_launches++, k2_bminus<<<vb, kThreads, 0, st>>>(h->b, h->Kr, n);
    apply_P(h, pred, mg_stage, h->Kr, V);
    double b2 = 0.0;
    grte_status r = mdot(h, V, V, 1, n, &b2);
    *beta = std::sqrt(b2);
    return r;
  };
  // a restart cycle that did not reduce the residual 4x while it is below 1e-9 (RMS per
  // cell) has reached the rounding floor of the residual evaluation (in cold, very
  // opaque cells the rows are sums of terms far larger than the residual)
  const double stall = 1e-9 * std::sqrt((double)D.g.nc);
  double prev = INFINITY;
  for (int cycle = 0; cycle <= maxcycles; ++cycle) {
    double beta = 0.0;
    if ((s = residual(&beta)) != GRTE_OK) return s;
    if (!std::isfinite(beta)) return fail2(h, GRTE_ENAN, "GMRES: non-finite residual");
    const bool floor_reached = mg_stage ? beta >= 0.25 * prev : (beta <= stall && beta >= 0.25 * prev);
    prev = beta;
    if (beta <= thr || floor_reached || cycle == maxcycles) {
      if (floor_reached) beta = 0.0;
      tl_launches++, k2_cellscale<<<gc, kThreads, 0, st>>>(h->x, D.iwsc, nblk, D.g.nc);  // y -> x
      if (!mg_stage && !(beta <= thr)) h->host_flags |= 1 << GRTE_ENONCONV;
      return GRTE_OK;
    }
    if (f32) tl_launches++, k2_tof<<<vb, kThreads, 0, st>>>(V, h->V32, n, 1.0 / beta);
    else tl_launches++, k2_scale<double><<<vb, kThreads, 0, st>>>(V, 1.0 / beta, n);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int kk = 0;
    for (int j = 0; j < m; ++j) {
      std::vector<double> hc(j + 2, 0.0);
      s = f32 ? arnoldi_step<float>(h, pred, mg_stage, h->V32, j, n, hc)
              : arnoldi_step<double>(h, pred, mg_stage, V, j, n, hc);
      if (s != GRTE_OK) return s;
      const double hn = std::sqrt(hc[j + 1]);
      hc[j + 1] = hn;
      ++iters;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
        hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
        hc[i] = t;
      }
      const double rr = std::hypot(hc[j], hc[j + 1]);
      cs[j] = rr > 0.0 ? hc[j] / rr : 1.0;
      sn[j] = rr > 0.0 ? hc[j + 1] / rr : 0.0;
      hc[j] = rr;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hc[i];
      kk = j + 1;
      if (hn > 0.0) {
        if (f32) tl_launches++, k2_scale<float><<<vb, kThreads, 0, st>>>(h->V32 + (int64_t)(j + 1) * n, 1.0 / hn, n);
        else tl_launches++, k2_scale<double><<<vb, kThreads, 0, st>>>(V + (int64_t)(j + 1) * n, 1.0 / hn, n);
      }
      const double gj = std::fabs(g[j + 1]);
      if (gj <= 0.5 * thr || hn == 0.0) break;
      if (f32 && gj <= kInnerReduce * beta) break;
      if (mg_stage && j >= 4 && gj <= 1e-6 * beta && gj > 0.5 * std::fabs(g[j - 3])) break;
    }
    for (int i = kk - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < kk; ++l) t -= H[(size_t)i * m + l] * yv[l];
      yv[i] = t / H[(size_t)i * m + i];
    }
    CK2(cudaMemcpyAsync(h->coef, yv.data(), sizeof(double) * kk, cudaMemcpyHostToDevice, st));
    if (f32) tl_launches++, k2_update<float><<<vb, kThreads, 0, st>>>(h->x, h->V32, h->coef, kk, n);
    else tl_launches++, k2_update<double><<<vb, kThreads, 0, st>>>(h->x, V, h->coef, kk, n);
    tl_launches++, k2_cellscale<<<gc, kThreads, 0, st>>>(h->x, D.iwsc, nblk, D.g.nc);    // y -> x
    CK2(cudaStreamSynchronize(st));
    CK2(cudaGetLastError());
  }
  return GRTE_OK;
}

static grte_status step2(grte2d_t h) {
  NvtxRange nv_("grte2d: step");
  D2& D = h->D;
  const G2& g = D.g;
  cudaStream_t st = h->stream;
  const unsigned gc = grid_of(g.nc), gv = grid_of(g.nv);
  const unsigned gvk = grid_of((int64_t)g.K * g.nv), gck = grid_of((int64_t)g.K * g.nc);
  const int64_t K = g.K, nc = g.nc;
  int its = 0;
  // prediction at T^n
  tl_launches++, k2_coef<<<gc, kThreads, 0, st>>>(D);
  tl_launches++, k2_vcoef<<<gv, kThreads, 0, st>>>(D);
  tl_launches++, k2_rho<<<gc, kThreads, 0, st>>>(D, D.E, D.rho_n);
  tl_launches++, k2_vertex<double, true><<<gvk, kThreads, 0, st>>>(D, h->cv, UField{nullptr, 0, nullptr}, h->V);
  tl_launches++, k2_cell<double, C_DIVK, true><<<gck, kThreads, 0, st>>>(D, h->cv, h->V, UField{nullptr, 0, nullptr}, nullptr, h->phi, nullptr, nullptr);
  tl_launches++, k2_rhs_pred<<<gc, kThreads, 0, st>>>(D, h->phi, h->b, h->x);
  tl_launches++, k2_gdiag<<<gc, kThreads, 0, st>>>(D, h->cv);
  mirror_coefficients(h);
  if (!h->mgl.empty()) mg_setup(h);
  CK2(cudaGetLastError());
  grte_status s = GRTE_OK;
  if (!h->mgl.empty()) {
    s = gmres2(h, true, true, (K + 1) * nc, its);
    if (s != GRTE_OK) return s;
    h->stats.krylov_iters += its;
    h->stats.krylov_iters_mg += its;
  }
  s = gmres2(h, true, false, (K + 1) * nc, its);
  if (s != GRTE_OK) return s;
  h->stats.krylov_iters += its;
  tl_launches++, k2_finish_pred<<<gc, kThreads, 0, st>>>(D, h->x, h->Es);
  // the flux term of the temperature equation: O from E* by the vertex map, with the
  // prediction's coefficients (sigma(x)) or those of V* = (U*)^{3/4} (sigma_0/T^3)
  if (g.kind == GRTE_SIGMA_T3) {
    // the prediction's vertex values (the Krylov basis is free until the correction's
    // solve: it holds (m+1)(K+1) nc >= K nv values), then those of V*; the inflow walls
    // shifted (k2_wallshift) and the wall-normal parts of the wall cells taken from the
    // prediction's (k2_fdiv_corr)
    double* Vp = h->Kbasis;
    tl_launches++, k2_vertex<double, true><<<gvk, kThreads, 0, st>>>(D, h->cv, UField{h->Es, nc, nullptr}, Vp);
    tl_launches++, k2_vstar<<<gc, kThreads, 0, st>>>(D);
    tl_launches++, k2_vcoef<<<gv, kThreads, 0, st>>>(D);
    tl_launches++, k2_vertex<double, true><<<gvk, kThreads, 0, st>>>(D, h->cv, UField{h->Es, nc, nullptr}, h->V);
    tl_launches++, k2_wallshift<<<gvk, kThreads, 0, st>>>(D, h->V, Vp);
    tl_launches++, k2_fdiv_corr<<<gck, kThreads, 0, st>>>(D, h->cv, h->V, Vp, UField{h->Es, nc, nullptr}, h->tk);
  } else {
    tl_launches++, k2_vertex<double, true><<<gvk, kThreads, 0, st>>>(D, h->cv, UField{h->Es, nc, nullptr}, h->V);
    tl_launches++, k2_cell<double, C_FDIV, true><<<gck, kThreads, 0, st>>>(D, h->cv, h->V, UField{h->Es, nc, nullptr}, nullptr, nullptr, nullptr, h->tk);
  }
  tl_launches++, k2_cellsum<double, C_FDIV><<<gc, kThreads, 0, st>>>(D, h->cv, h->tk, nullptr, D.Fdiv, nullptr);
  if (D.use_guess || D.log_samples) tl_launches++, k2_newton_feat<<<gc, kThreads, 0, st>>>(D);
  if (D.use_guess) {
    tl_launches++;   // the network's guess: one kernel
    cudaError_t e = grte::mlp_guess_launch(h->mlp, D.feat, nc, D.guess, st);
    if (e != cudaSuccess) return fail2(h, GRTE_ECUDA, std::string("mlp guess: ") + cudaGetErrorString(e));
  }
  tl_launches++, k2_newton<<<gc, kThreads, 0, st>>>(D);
  // correction substep 2 at T^{n+1}
  tl_launches++, k2_coef<<<gc, kThreads, 0, st>>>(D);
  tl_launches++, k2_vcoef<<<gv, kThreads, 0, st>>>(D);
  tl_launches++, k2_acU<<<gc, kThreads, 0, st>>>(D);
  tl_launches++, k2_vertex<double, true><<<gvk, kThreads, 0, st>>>(D, h->cv, UField{nullptr, 0, nullptr}, h->V);
  tl_launches++, k2_cell<double, C_DIVK, true><<<gck, kThreads, 0, st>>>(D, h->cv, h->V, UField{nullptr, 0, nullptr}, nullptr, h->phi, nullptr, nullptr);
  tl_launches++, k2_vertex<double, false><<<gvk, kThreads, 0, st>>>(D, h->cv, UField{nullptr, 0, D.acU}, h->V);
  tl_launches++, k2_cell<double, C_DIVK, false><<<gck, kThreads, 0, st>>>(D, h->cv, h->V, UField{nullptr, 0, D.acU}, nullptr, h->GU, nullptr, nullptr);
  tl_launches++, k2_rhs_corr<<<gc, kThreads, 0, st>>>(D, h->GU, h->phi, h->b, h->x);
  tl_launches++, k2_corrscale<<<gc, kThreads, 0, st>>>(D, h->cscale);
  tl_launches++, k2_gdiag<<<gc, kThreads, 0, st>>>(D, h->cv);
  mirror_coefficients(h);
  CK2(cudaGetLastError());
  if (!h->mpl.empty() && (s = mp_setup(h)) != GRTE_OK) return s;
  its = 0;
  s = gmres2(h, false, false, K * nc, its);
  if (s != GRTE_OK) return s;
  h->stats.krylov_iters += its;
  h->stats.krylov_iters_corr += its;
  // projection: E = a c U + eps E_J, O from E (vertex map with the O^n data), U = T^4
  tl_launches++, k2_project<<<gc, kThreads, 0, st>>>(D, h->x);
  tl_launches++, k2_vertex<double, true><<<gvk, kThreads, 0, st>>>(D, h->cv, UField{D.E, nc, nullptr}, h->V);
  CK2(cudaMemcpyAsync(D.O, h->V, sizeof(double) * K * g.nv, cudaMemcpyDeviceToDevice, st));
  CK2(cudaGetLastError());
  return GRTE_OK;
}

extern "C" {

void grte2d_destroy(grte2d_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->mp_graph) cudaGraphExecDestroy(h->mp_graph);
  for (void* p : h->allocs) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* grte2d_last_error(grte2d_t h) { return h ? h->err.c_str() : "null handle"; }

grte_status grte2d_create(const grte_instance2d* p, const grte_options* opt, grte2d_t* out) {
  if (!out) return GRTE_EINVAL;
  *out = nullptr;
  if (!p) return GRTE_EINVAL;
  grte2d_t h = new (std::nothrow) grte2d_ctx();
  if (!h) return GRTE_ENOMEM;
  *out = h;
  grte_default_options(&h->opt);
  if (opt) h->opt = *opt;
  h->m = h->opt.krylov_restart == 10 ? 30 : h->opt.krylov_restart;
  if (h->m < 1 || h->m > kMaxRestart2) return fail2(h, GRTE_EINVAL, "krylov_restart out of range [1,64]");
  if (!(h->opt.krylov_rtol > 0) || h->opt.krylov_maxcycles < 1 || h->opt.newton_maxit < 1)
    return fail2(h, GRTE_EINVAL, "bad solver options");
  if (p->nx < 2 || p->ny < 2 || p->nx > 32768 || p->ny > 32768) return fail2(h, GRTE_EINVAL, "nx, ny must be in [2, 32768]");
  if ((int64_t)std::max(p->n_pair, 20) * (p->nx + 1) * (p->ny + 1) >= (int64_t)1 << 31)
    return fail2(h, GRTE_EINVAL, "n_pair * (nx+1) * (ny+1) must be below 2^31");
  if (!p->sigma) return fail2(h, GRTE_EINVAL, "sigma is NULL");
  if (p->sigma_kind != GRTE_SIGMA_CONST && p->sigma_kind != GRTE_SIGMA_T3 && p->sigma_kind != GRTE_SIGMA_POW)
    return fail2(h, GRTE_EINVAL, "bad sigma_kind");
  if (p->sigma_kind == GRTE_SIGMA_POW && !(p->sigma_p >= 0.0 && p->sigma_p <= 3.0))
    return fail2(h, GRTE_EINVAL, "sigma_p must be in [0, 3]");
  for (int bc : {p->bc_x, p->bc_y})
    if (bc != GRTE_BC_INFLOW && bc != GRTE_BC_PERIODIC) return fail2(h, GRTE_EINVAL, "bc must be INFLOW or PERIODIC");
  if (!(p->lx > 0) || !(p->ly > 0) || !(p->dt > 0) || !(p->a > 0) || !(p->c > 0) || !(p->Cv > 0) || !(p->eps > 0))
    return fail2(h, GRTE_EINVAL, "lx, ly, dt, a, c, Cv, eps must be positive");
  if (p->n_pair < 0 || p->n_pair > kMaxPairs) return fail2(h, GRTE_EINVAL, "n_pair must be in [0, 64]");
  if (p->n_pair == 0) {
    s8_pairs(h->hmu, h->heta, h->hw);
  } else {
    if (!p->mu || !p->eta || !p->w) return fail2(h, GRTE_EINVAL, "mu, eta, w required when n_pair > 0");
    h->hmu.assign(p->mu, p->mu + p->n_pair);
    h->heta.assign(p->eta, p->eta + p->n_pair);
    h->hw.assign(p->w, p->w + p->n_pair);
    double sw = 0.0;
    for (int k = 0; k < p->n_pair; ++k) {
      if (!(h->hw[k] > 0.0)) return fail2(h, GRTE_EINVAL, "weights must be positive");
      if (p->bc_x == GRTE_BC_INFLOW && h->hmu[k] == 0.0) return fail2(h, GRTE_EINVAL, "mu = 0 with an inflow x axis");
      if (p->bc_y == GRTE_BC_INFLOW && h->heta[k] == 0.0) return fail2(h, GRTE_EINVAL, "eta = 0 with an inflow y axis");
      sw += h->hw[k];
    }
    for (double& v : h->hw) v /= sw;
  }
  G2& g = h->g;
  g.Nx = (int)p->nx;
  g.Ny = (int)p->ny;
  g.K = (int)h->hmu.size();
  g.bcx = p->bc_x;
  g.bcy = p->bc_y;
  g.kind = p->sigma_kind == GRTE_SIGMA_CONST ? GRTE_SIGMA_CONST : GRTE_SIGMA_T3;
  g.p = p->sigma_kind == GRTE_SIGMA_POW ? p->sigma_p : 3.0;
  g.nc = p->nx * p->ny;
  g.nv = (p->nx + 1) * (p->ny + 1);
  g.dx = p->lx / (double)p->nx;
  g.dy = p->ly / (double)p->ny;
  g.eps = p->eps; g.dt = p->dt; g.a = p->a; g.c = p->c; g.Cv = p->Cv;
  g.bx0 = p->b_x0; g.bx1 = p->b_x1; g.by0 = p->b_y0; g.by1 = p->b_y1;
  g.h2x = 1.0 / (2.0 * g.dx);
  g.h2y = 1.0 / (2.0 * g.dy);
  g.te = 2.0 / g.eps;
  for (int64_t c = 0; c < g.nc; ++c)
    if (!(p->sigma[c] >= 0.0) || !std::isfinite(p->sigma[c])) return fail2(h, GRTE_EINVAL, "sigma must be finite and >= 0");
  if (h->opt.stream) {
    h->stream = (cudaStream_t)h->opt.stream;
  } else {
    CK2(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  D2& D = h->D;
  D.g = g;
  D.newton_maxit = h->opt.newton_maxit;
  const int64_t K = g.K, nc = g.nc, nv = g.nv, nz = (K + 1) * nc;
  bool ok = alloc2(h, &h->dmu, K) && alloc2(h, &h->deta, K) && alloc2(h, &h->dw, K) && alloc2(h, &h->dsig, nc) &&
            alloc2(h, &D.T, nc) && alloc2(h, &D.U, nc) && alloc2(h, &D.E, K * nc) && alloc2(h, &D.O, K * nv) &&
            alloc2(h, &D.kc, nc) && alloc2(h, &D.A, nc) && alloc2(h, &D.alpha, nc) && alloc2(h, &D.s, nc) &&
            alloc2(h, &D.gam, nc) && alloc2(h, &D.dv, nv) && alloc2(h, &D.odv, nv) && alloc2(h, &D.rho_n, nc) &&
            alloc2(h, &D.Us, nc) && alloc2(h, &D.Fdiv, nc) && alloc2(h, &D.rho_s, nc) &&
            alloc2(h, &D.newton_its, nc) && alloc2(h, &D.acU, nc) && alloc2(h, &D.status, 1) &&
            alloc2(h, &D.wsc, nc) && alloc2(h, &D.iwsc, nc) && alloc2(h, &D.gd, K * nc) && alloc2(h, &D.gdi, K * nc) && alloc2(h, &D.pdi, nc) &&
            alloc2(h, &h->V, K * nv) && alloc2(h, &h->phi, K * nc) && alloc2(h, &h->GU, K * nc) &&
            alloc2(h, &h->Es, K * nc) && alloc2(h, &h->b, nz) && alloc2(h, &h->x, nz) && alloc2(h, &h->Kr, nz) &&
            alloc2(h, &h->Kt, nz) && alloc2(h, &h->Kbasis, (int64_t)(h->m + 1) * nz) &&
            alloc2(h, &h->part, (int64_t)kAxpyBlocks * (kMaxRestart2 + 1)) && alloc2(h, &h->dots, kMaxRestart2 + 1) &&
            alloc2(h, &h->coef, kMaxRestart2 + 1) && alloc2(h, &h->cscale, nc) &&
            alloc2(h, &h->hcol, kMaxRestart2 + 2) && alloc2(h, &h->tk, K * nc);
  if (!ok) return fail2(h, GRTE_ENOMEM, "cudaMalloc failed");
  if (h->opt.prec2d & ~(GRTE_PREC2D_MULTIGRID | GRTE_PREC2D_CORR_MG))
    return fail2(h, GRTE_EINVAL, "prec2d: a set of GRTE_PREC2D_MULTIGRID and GRTE_PREC2D_CORR_MG");
  if (h->opt.prec2d & GRTE_PREC2D_CORR_MG) {
    // levels of 2x2 aggregates down to lines of <= 2 cells in both axes
    mp::PLevel L{};
    L.nx = g.Nx; L.ny = g.Ny; L.K = (int)K;
    L.perx = g.bcx == GRTE_BC_PERIODIC; L.pery = g.bcy == GRTE_BC_PERIODIC;
    for (;;) {
      L.n = (int64_t)L.nx * L.ny;
      const int64_t kn = K * L.n;
      if (!alloc2(h, &L.cr, 9 * kn) || !alloc2(h, &L.ct, 9 * kn) || !alloc2(h, &L.x, kn) || !alloc2(h, &L.xt, kn) ||
          !alloc2(h, &L.b, kn) || !alloc2(h, &L.bt, kn) || !alloc2(h, &L.cp, kn))
        return fail2(h, GRTE_ENOMEM, "cudaMalloc pair multigrid");
      h->mpl.push_back(L);
      if (L.nx <= 2 && L.ny <= 2) break;
      L.nx = (L.nx + 1) / 2;
      L.ny = (L.ny + 1) / 2;
    }
    if (!alloc2(h, &h->mp_probe, K * nc)) return fail2(h, GRTE_ENOMEM, "cudaMalloc pair multigrid");
  }
  if (h->opt.prec2d & GRTE_PREC2D_MULTIGRID) {
    // level 0: the cells (one unknown each); then 2x2 aggregation with one unknown per
    // colour class, until the level has at most mg::kDenseMax unknowns
    mg::Level L{};
    L.nx = g.Nx; L.ny = g.Ny; L.ncomp = 1;
    L.perx = g.bcx == GRTE_BC_PERIODIC; L.pery = g.bcy == GRTE_BC_PERIODIC;
    for (;;) {
      L.ncell = (int64_t)L.nx * L.ny;
      L.n = L.ncell * L.ncomp;
      if (!alloc2(h, &L.coef, 9 * L.ncomp * L.n) || !alloc2(h, &L.idiag, L.n) || !alloc2(h, &L.x, L.n) ||
          !alloc2(h, &L.xt, L.n) || !alloc2(h, &L.b, L.n))
        return fail2(h, GRTE_ENOMEM, "cudaMalloc multigrid");
      h->mgl.push_back(L);
      if (L.n <= mg::kDenseMax) break;
      L.nx = (L.nx + 1) / 2;
      L.ny = (L.ny + 1) / 2;
      L.ncomp = 2;
    }
    if (!alloc2(h, &h->mg_M, mg::kDenseMax * mg::kDenseMax) || !alloc2(h, &h->mg_inv, mg::kDenseMax * mg::kDenseMax))
      return fail2(h, GRTE_ENOMEM, "cudaMalloc multigrid");
  }
  D.mu = h->dmu; D.eta = h->deta; D.w = h->dw; D.sig = h->dsig;
  h->cv = CV<double>{D.mu, D.eta, D.w, D.kc, D.A, D.alpha, D.dv, D.gd, D.gdi, D.pdi, D.wsc, D.iwsc,
                     g.h2x, g.h2y, g.te};
  if (h->opt.precision == GRTE_MIXED) {
    h->mixed = true;
    const int64_t nvk = K * nv;
    bool okf = alloc2(h, &h->mu32, K) && alloc2(h, &h->eta32, K) && alloc2(h, &h->w32, K) &&
               alloc2(h, &h->kc32, nc) && alloc2(h, &h->A32, nc) && alloc2(h, &h->alpha32, nc) &&
               alloc2(h, &h->dv32, nv) && alloc2(h, &h->gd32, K * nc) && alloc2(h, &h->gdi32, K * nc) &&
               alloc2(h, &h->pdi32, nc) && alloc2(h, &h->wsc32, nc) && alloc2(h, &h->iwsc32, nc) &&
               alloc2(h, &h->V32, (int64_t)(h->m + 1) * nz) && alloc2(h, &h->Kr32, nz) &&
               alloc2(h, &h->Vv32, nvk) && alloc2(h, &h->tk32, K * nc);
    if (!okf) return fail2(h, GRTE_ENOMEM, "cudaMalloc binary32 buffers");
    std::vector<float> f(K);
    for (int64_t k = 0; k < K; ++k) f[k] = (float)h->hmu[k];
    CK2(cudaMemcpy(h->mu32, f.data(), sizeof(float) * K, cudaMemcpyHostToDevice));
    for (int64_t k = 0; k < K; ++k) f[k] = (float)h->heta[k];
    CK2(cudaMemcpy(h->eta32, f.data(), sizeof(float) * K, cudaMemcpyHostToDevice));
    for (int64_t k = 0; k < K; ++k) f[k] = (float)h->hw[k];
    CK2(cudaMemcpy(h->w32, f.data(), sizeof(float) * K, cudaMemcpyHostToDevice));
    h->cv32 = CV<float>{h->mu32, h->eta32, h->w32, h->kc32, h->A32, h->alpha32, h->dv32, h->gd32, h->gdi32,
                        h->pdi32, h->wsc32, h->iwsc32, (float)g.h2x, (float)g.h2y, (float)g.te};
  } else if (h->opt.precision != GRTE_FP64) {
    return fail2(h, GRTE_EINVAL, "precision must be GRTE_FP64 or GRTE_MIXED");
  }
  CK2(cudaMemcpy(h->dmu, h->hmu.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
  CK2(cudaMemcpy(h->deta, h->heta.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
  CK2(cudaMemcpy(h->dw, h->hw.data(), sizeof(double) * K, cudaMemcpyHostToDevice));
  CK2(cudaMemcpy(h->dsig, p->sigma, sizeof(double) * nc, cudaMemcpyHostToDevice));
  return GRTE_OK;
}

grte_status grte2d_set_state(grte2d_t h, const double* T, const double* E, const double* O) {
  if (!h) return GRTE_EINVAL;
  if (!T) return fail2(h, GRTE_EINVAL, "T is NULL");
  if ((E == nullptr) != (O == nullptr)) return fail2(h, GRTE_EINVAL, "E and O must both be given or both NULL");
  const G2& g = h->g;
  const int64_t K = g.K, nc = g.nc, nv = g.nv;
  std::vector<double> hE(K * nc), hO(K * nv, 0.0), hU(nc);
  for (int64_t c = 0; c < nc; ++c) {
    if (!(T[c] >= 0.0) || !std::isfinite(T[c])) return fail2(h, GRTE_EINVAL, "T must be finite and >= 0");
    hU[c] = (T[c] * T[c]) * (T[c] * T[c]);
  }
  for (int64_t k = 0; k < K; ++k) {
    for (int64_t c = 0; c < nc; ++c) hE[k * nc + c] = E ? E[c * K + k] : g.a * g.c * hU[c];
    if (O)
      for (int64_t v = 0; v < nv; ++v) hO[k * nv + v] = O[v * K + k];
  }
  D2& D = h->D;
  CK2(cudaStreamSynchronize(h->stream));
  CK2(cudaMemcpy(D.T, T, sizeof(double) * nc, cudaMemcpyHostToDevice));
  CK2(cudaMemcpy(D.U, hU.data(), sizeof(double) * nc, cudaMemcpyHostToDevice));
  CK2(cudaMemcpy(D.E, hE.data(), sizeof(double) * K * nc, cudaMemcpyHostToDevice));
  CK2(cudaMemcpy(D.O, hO.data(), sizeof(double) * K * nv, cudaMemcpyHostToDevice));
  CK2(cudaMemset(D.status, 0, sizeof(int)));
  h->host_flags = 0;
  h->state_set = true;
  return GRTE_OK;
}

static grte_status status2(grte2d_t h) {
  int s = 0;
  CK2(cudaStreamSynchronize(h->stream));
  CK2(cudaMemcpy(&s, h->D.status, sizeof(int), cudaMemcpyDeviceToHost));
  s |= h->host_flags;
  h->stats.status_flags = s;
  for (int code : {GRTE_ENAN, GRTE_ENONCONV, GRTE_ENEGATIVE, GRTE_ETIMEOUT})
    if (s & (1 << code)) return fail2(h, (grte_status)code, "device reported status " + std::to_string(code));
  return GRTE_OK;
}

grte_status grte2d_step(grte2d_t h, int64_t n) {
  NvtxRange nv_("grte2d_step");
  if (!h) return GRTE_EINVAL;
  if (!h->state_set) return fail2(h, GRTE_ESTATE, "state not set");
  if (n < 0) return fail2(h, GRTE_EINVAL, "n < 0");
  h->stats.krylov_iters = 0;
  h->stats.krylov_iters_corr = 0;
  h->stats.krylov_iters_mg = 0;
  const int64_t l0 = tl_launches;
  for (int64_t i = 0; i < n; ++i) {
    grte_status s = step2(h);
    h->stats.launches = tl_launches - l0;
    if (s != GRTE_OK) return s;
    h->stats.steps += 1;
  }
  return status2(h);
}

static grte_status get2(grte2d_t h, const double* src, int64_t count, double* out, size_t len) {
  if (!out || len != (size_t)count) return fail2(h, GRTE_EINVAL, "bad output length");
  CK2(cudaStreamSynchronize(h->stream));
  CK2(cudaMemcpy(out, src, sizeof(double) * count, cudaMemcpyDeviceToHost));
  return status2(h);
}

grte_status grte2d_get_T(grte2d_t h, double* T, size_t len) {
  if (!h) return GRTE_EINVAL;
  return get2(h, h->D.T, h->g.nc, T, len);
}

grte_status grte2d_get_E(grte2d_t h, double* E, size_t len) {
  if (!h) return GRTE_EINVAL;
  const int64_t K = h->g.K, nc = h->g.nc;
  if (!E || len != (size_t)(K * nc)) return fail2(h, GRTE_EINVAL, "len must be nx*ny*K");
  std::vector<double> t(K * nc);
  grte_status s = get2(h, h->D.E, K * nc, t.data(), t.size());
  for (int64_t k = 0; k < K; ++k)
    for (int64_t c = 0; c < nc; ++c) E[c * K + k] = t[k * nc + c];
  return s;
}

grte_status grte2d_get_O(grte2d_t h, double* O, size_t len) {
  if (!h) return GRTE_EINVAL;
  const int64_t K = h->g.K, nv = h->g.nv;
  if (!O || len != (size_t)(K * nv)) return fail2(h, GRTE_EINVAL, "len must be (nx+1)*(ny+1)*K");
  std::vector<double> t(K * nv);
  grte_status s = get2(h, h->D.O, K * nv, t.data(), t.size());
  for (int64_t k = 0; k < K; ++k)
    for (int64_t v = 0; v < nv; ++v) O[v * K + k] = t[k * nv + v];
  return s;
}

grte_status grte2d_get_stage(grte2d_t h, int which, double* out, size_t len) {
  if (!h) return GRTE_EINVAL;
  const double* src = which == 0 ? h->D.Us : which == 1 ? h->D.Fdiv : which == 2 ? h->D.rho_s
                    : which == 3 ? h->D.newton_its : nullptr;
  if (!src) return fail2(h, GRTE_EINVAL, "which must be 0..3");
  return get2(h, src, h->g.nc, out, len);
}

grte_status grte2d_get_quadrature(grte2d_t h, double* mu, double* eta, double* w, size_t K) {
  if (!h) return GRTE_EINVAL;
  if (!mu || !eta || !w || K != h->hmu.size()) return fail2(h, GRTE_EINVAL, "K must equal the pair count");
  std::copy(h->hmu.begin(), h->hmu.end(), mu);
  std::copy(h->heta.begin(), h->heta.end(), eta);
  std::copy(h->hw.begin(), h->hw.end(), w);
  return GRTE_OK;
}

grte_status grte2d_get_energy(grte2d_t h, double* e) {
  if (!h) return GRTE_EINVAL;
  if (!e) return fail2(h, GRTE_EINVAL, "e is NULL");
  tl_launches++, k2_energy<<<kRedBlocks, kThreads, 0, h->stream>>>(h->D, h->part);
  tl_launches++, k2_reduce<<<1, kThreads, 0, h->stream>>>(h->part, kRedBlocks, h->dots);
  CK2(cudaGetLastError());
  CK2(cudaMemcpyAsync(e, h->dots, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK2(cudaStreamSynchronize(h->stream));
  return GRTE_OK;
}

static grte_status ensure_feat2(grte2d_t h) {
  D2& D = h->D;
  if (!D.feat) {
    const int64_t nc = h->g.nc;
    if (!alloc2(h, &D.feat, 6 * nc) || !alloc2(h, &D.guess, nc) || !alloc2(h, &D.ytrue, nc))
      return fail2(h, GRTE_ENOMEM, "cudaMalloc features");
  }
  return GRTE_OK;
}

grte_status grte2d_set_guess(grte2d_t h, grte_mlp_t m) {
  if (!h) return GRTE_EINVAL;
  CK2(cudaStreamSynchronize(h->stream));
  if (m) {
    grte_status s = ensure_feat2(h);
    if (s != GRTE_OK) return s;
  }
  h->mlp = m;
  h->D.use_guess = m ? 1 : 0;
  h->D.start_prev = 0;
  return GRTE_OK;
}

grte_status grte2d_set_newton_start(grte2d_t h, int mode) {
  if (!h) return GRTE_EINVAL;
  if (mode != GRTE_START_BOUND && mode != GRTE_START_PREVIOUS && mode != GRTE_START_LEARNED)
    return fail2(h, GRTE_EINVAL, "bad start mode");
  if (mode == GRTE_START_LEARNED && !h->mlp) return fail2(h, GRTE_ESTATE, "no network set (grte2d_set_guess)");
  CK2(cudaStreamSynchronize(h->stream));
  h->D.start_prev = mode == GRTE_START_PREVIOUS ? 1 : 0;
  h->D.use_guess = mode == GRTE_START_LEARNED ? 1 : 0;
  return GRTE_OK;
}

grte_status grte2d_set_sample_logging(grte2d_t h, int on) {
  if (!h) return GRTE_EINVAL;
  CK2(cudaStreamSynchronize(h->stream));
  if (on) {
    grte_status s = ensure_feat2(h);
    if (s != GRTE_OK) return s;
  }
  h->D.log_samples = on ? 1 : 0;
  return GRTE_OK;
}

grte_status grte2d_get_newton_samples(grte2d_t h, float* X, float* y, size_t n) {
  if (!h) return GRTE_EINVAL;
  if (!X || !y || n != (size_t)h->g.nc) return fail2(h, GRTE_EINVAL, "n must be nx*ny");
  if (!h->D.log_samples) return fail2(h, GRTE_ESTATE, "sample logging is off");
  CK2(cudaStreamSynchronize(h->stream));
  CK2(cudaMemcpy(X, h->D.feat, sizeof(float) * 6 * n, cudaMemcpyDeviceToHost));
  CK2(cudaMemcpy(y, h->D.ytrue, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return GRTE_OK;
}

grte_status grte2d_stats(grte2d_t h, grte_stats_t* st) {
  if (!h || !st) return GRTE_EINVAL;
  std::vector<double> its(h->g.nc);
  CK2(cudaStreamSynchronize(h->stream));
  CK2(cudaMemcpy(its.data(), h->D.newton_its, sizeof(double) * h->g.nc, cudaMemcpyDeviceToHost));
  double mx = 0.0, sum = 0.0;
  for (double v : its) { mx = std::max(mx, v); sum += v; }
  h->stats.newton_iters_max = (int64_t)mx;
  h->stats.newton_iters_mean = sum / (double)h->g.nc;
  grte_status s = status2(h);
  *st = h->stats;
  return s;
}

// ----------------------------------------------------------------------------- one create
grte_status grte_create(const grte_grid* grid, const grte_quadrature* quad, const grte_opacity* opac,
                        double a, double c, double Cv, double eps, const grte_bc* bc,
                        const grte_options* opt, grte_handle* out) {
  if (!out) return GRTE_EINVAL;
  out->dim = 0;
  out->ncell = 0;
  out->h1 = nullptr;
  out->h2 = nullptr;
  if (!grid || !opac || !bc) return GRTE_EINVAL;
  const bool custom = quad && quad->mu;
  if (grid->dim == 1) {
    const int64_t nx = grid->nx;
    if (nx < 2) return GRTE_EINVAL;
    const int n_dir = (quad && quad->n_dir) ? quad->n_dir : 16;
    if (n_dir < 2 || n_dir % 2) return GRTE_EINVAL;
    const int M = n_dir / 2;
    if (custom && !quad->w) return GRTE_EINVAL;
    if (bc->kind[0] != bc->kind[1] || (bc->kind[0] != GRTE_BC_INFLOW && bc->kind[0] != GRTE_BC_REFLECT))
      return GRTE_EINVAL;
    std::vector<double> sig(nx), bL(M), bR(M);
    for (int64_t j = 0; j < nx; ++j) sig[j] = opac->sigma0 ? opac->sigma0[j] : opac->sigma0_scalar;
    for (int k = 0; k < M; ++k) {
      bL[k] = bc->b[0] ? bc->b[0][k] : bc->b_iso[0];
      bR[k] = bc->b[1] ? bc->b[1][k] : bc->b_iso[1];
    }
    grte_instance1d p{};
    p.nx = nx;
    p.n_angle = M;
    p.v = custom ? quad->mu : nullptr;
    p.w = custom ? quad->w : nullptr;
    p.sigma = sig.data();
    p.sigma_kind = opac->kind;
    p.sigma_p = opac->sigma_p;
    p.bc = bc->kind[0];
    p.bL = bL.data();
    p.bR = bR.data();
    p.x0 = grid->x0;
    p.x1 = grid->x1;
    p.dt = grid->dt;
    p.a = a;
    p.c = c;
    p.Cv = Cv;
    p.eps = eps;
    grte_t h = nullptr;
    const grte_status s = grte_create_1d(1, &p, opt, &h);
    if (s != GRTE_OK) {
      grte_destroy(h);
      return s;
    }
    out->dim = 1;
    out->ncell = nx;
    out->h1 = h;
    return GRTE_OK;
  }
  if (grid->dim != 2) return GRTE_EINVAL;
  if (grid->x0 != 0.0 || grid->y0 != 0.0) return GRTE_EINVAL;
  if (bc->kind[0] != bc->kind[1] || bc->kind[2] != bc->kind[3]) return GRTE_EINVAL;
  const int n_dir = (quad && quad->n_dir) ? quad->n_dir : 40;
  if (!custom && n_dir != 40) return GRTE_EINVAL;
  if (custom && (!quad->eta || !quad->w || n_dir < 2 || n_dir % 2)) return GRTE_EINVAL;
  const int64_t nc = grid->nx * grid->ny;
  if (grid->nx < 2 || grid->ny < 2) return GRTE_EINVAL;
  std::vector<double> sig(nc);
  for (int64_t q = 0; q < nc; ++q) sig[q] = opac->sigma0 ? opac->sigma0[q] : opac->sigma0_scalar;
  grte_instance2d p{};
  p.nx = grid->nx;
  p.ny = grid->ny;
  p.n_pair = custom ? n_dir / 2 : 0;
  p.mu = custom ? quad->mu : nullptr;
  p.eta = custom ? quad->eta : nullptr;
  p.w = custom ? quad->w : nullptr;
  p.sigma = sig.data();
  p.sigma_kind = opac->kind;
  p.sigma_p = opac->sigma_p;
  p.bc_x = bc->kind[0];
  p.bc_y = bc->kind[2];
  p.b_x0 = bc->b_iso[0];
  p.b_x1 = bc->b_iso[1];
  p.b_y0 = bc->b_iso[2];
  p.b_y1 = bc->b_iso[3];
  p.lx = grid->x1;
  p.ly = grid->y1;
  p.dt = grid->dt;
  p.a = a;
  p.c = c;
  p.Cv = Cv;
  p.eps = eps;
  grte2d_t h = nullptr;
  const grte_status s = grte2d_create(&p, opt, &h);
  if (s != GRTE_OK) {
    grte2d_destroy(h);
    return s;
  }
  out->dim = 2;
  out->ncell = nc;
  out->h2 = h;
  return GRTE_OK;
}

grte_status grte_handle_set_initial(grte_handle* h, const double* T, size_t len) {
  if (!h || !T || len != (size_t)h->ncell) return GRTE_EINVAL;
  if (h->dim == 1) return grte_set_state(h->h1, 0, T, nullptr, nullptr);
  if (h->dim == 2) return grte2d_set_state(h->h2, T, nullptr, nullptr);
  return GRTE_EINVAL;
}

grte_status grte_handle_step(grte_handle* h, int64_t n) {
  if (!h) return GRTE_EINVAL;
  if (h->dim == 1) return grte_step(h->h1, n);
  if (h->dim == 2) return grte2d_step(h->h2, n);
  return GRTE_EINVAL;
}

grte_status grte_handle_sync(grte_handle* h) {
  if (!h) return GRTE_EINVAL;
  if (h->dim == 1) return grte_sync(h->h1);
  if (h->dim == 2) return GRTE_OK;   // 2D steps are synchronous and report their status
  return GRTE_EINVAL;
}

grte_status grte_handle_get_T(grte_handle* h, double* T, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (h->dim == 1) return grte_get_T(h->h1, 0, T, len);
  if (h->dim == 2) return grte2d_get_T(h->h2, T, len);
  return GRTE_EINVAL;
}

void grte_handle_destroy(grte_handle* h) {
  if (!h) return;
  if (h->h1) grte_destroy(h->h1);
  if (h->h2) grte2d_destroy(h->h2);
  h->h1 = nullptr;
  h->h2 = nullptr;
  h->dim = 0;
  h->ncell = 0;
}

}  // extern "C"
