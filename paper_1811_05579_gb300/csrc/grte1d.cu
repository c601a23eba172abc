// GB300 (sm_103a) implementation of one step of the 1D AP scheme for the gray
// radiative transfer equation (Tang, Wang, Zhang, arXiv:1811.05579): Algorithm 2 of
// Sec. 4 (sigma(x)) and its sigma_0/T^3 form of Sec. 5, for many independent
// instances at once.  The C ABI is declared in include/grte.h.
//
// Formulation (exact rewrite of the paper's equations, see the per-kernel comments):
// per angle line (instance, k) the even part is split as E = rho + e with
// rho = sum_k w_k E_k; O is eliminated with the node equation and the wall rows, U*
// with the U equation.  The prediction (Eq. dis-pre / Eq. dis-pre-marshak) becomes
//   e-equation  (A + G_k) e_k = h_k - alpha rho - G_k rho       (tridiagonal per line)
//   conservation  alpha rho + sum_k w_k [G_k(rho + e_k) + phi_k] = kappa rho^n/(c dt) + s a c U^n
// and is solved for rho by GMRES whose matrix-vector product is M independent
// tridiagonal line solves (factorised once per step and reused), preconditioned by
// the same construction with a single effective angle (sum_k w_k G_k), which is one
// more tridiagonal solve per instance.  The temperature equation (Eq. Tnp1) is a
// per-cell quartic solved by monotone Newton; correction substep 2 (Eq. dis-cor) is
// one tridiagonal solve per line in E_J with the same operator family; projection
// (Eq. dis-proj) is fused into that kernel's epilogue.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
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
#include "mlp.cuh"
#include "tridiag.cuh"

namespace grte {

namespace cg = cooperative_groups;
constexpr double kGuessGate = 1.1220184543019633;   // 10^0.05: learned-start gate (k_newton)
constexpr int kMaxRestart = 16;

struct Inst {
  int N, M, kind, bc;      // kind: GRTE_SIGMA_CONST or GRTE_SIGMA_T3 (sigma_0/T^p, p below)
  double p;                // the exponent of sigma_0/T^p (3 for GRTE_SIGMA_T3)
  double eps, dt, dx, a, c, Cv;
  double wv, wv2;          // sum_k w_k v_k, sum_k w_k v_k^2
  double two_eps, inv_eps; // 2/eps, 1/eps
  // derived per-instance constants (inst_derive), so that no per-cell kernel divides by them
  double rdx, e2cdt;       // 1/dx, eps^2/(c dt)
  double rcdt, reps2, rdx2; // 1/(c dt), 1/eps^2, 1/dx^2
  double gamc, gbc;        // 4 dt/(eps^2 Cv), 2/(eps dx)
  double adt, cvdt, ekc;   // a/dt, Cv/dt, eps^2 Cv/(c dt^2)
  double bLflux, bRflux;   // sum_k w_k v_k b_L,k and sum_k w_k v_k b_R,k
  int64_t cell_off;        // per-cell arrays
  int64_t elem_off;        // E-like arrays, line k at elem_off + k*N
  int64_t nelem_off;       // O-like arrays, line k at nelem_off + k*(N+1)
  int64_t red_off;         // reduced-system storage of the preconditioner
  int ang_off;             // v, w, bL, bR
  int line_off;            // first line of this instance
  int64_t fd_off;          // fused solve: the instance's staged data terms (floats)
};

// The derived constants of an instance from eps, dt, dx, c and Cv.
static void inst_derive(Inst& I) {
  I.two_eps = 2.0 / I.eps;
  I.inv_eps = 1.0 / I.eps;
  I.rdx = 1.0 / I.dx;
  I.e2cdt = I.eps * I.eps / (I.c * I.dt);
  I.rcdt = 1.0 / (I.c * I.dt);
  I.reps2 = 1.0 / (I.eps * I.eps);
  I.rdx2 = 1.0 / (I.dx * I.dx);
  I.gamc = 4.0 * I.dt / (I.eps * I.eps * I.Cv);
  I.gbc = 2.0 / (I.eps * I.dx);
  I.adt = I.a / I.dt;
  I.cvdt = I.Cv / I.dt;
  I.ekc = I.eps * I.eps * I.Cv / (I.c * I.dt * I.dt);
}

struct Line {
  int inst, k;
  int64_t red_off;         // reduced-system storage of this line
  int64_t f_off;           // factor storage of this line (tri_fac_size values)
};

// Per-cell coefficient arrays (length = total cells) for one operator family.
struct CellCoef {
  double *kc, *s, *alpha, *A, *gam, *gl, *gu, *gb, *dl;  // dl_j = d at the left node of cell j
  // products and reciprocals precomputed per cell so that no line kernel divides:
  double *od;    // dl_j eps^2/(c dt): o_j = od_j O^n_j
  double *dlx;   // dl_j / dx
  double *kcd;   // kappa_j/(c dt)
  double *kdx;   // kappa_j / dx
  double *sac;   // s_j a c
  double *ralpha;  // 1/alpha_j
  double *ratio;   // (A_j - alpha_j)/alpha_j = beta/alpha
  double *fR, *fL; // m^R d_{j+1}/dx, m^L d_j/dx (streaming flux of a per-cell field, unscaled by kappa)
  double *gbx;     // 2/eps in the inflow wall cells, else 0
  // the correction's flux (sigma_0/T^3) at the iterate of the last data pass: at the
  // left node of each cell d*/dx and d* eps^2/(c dt), d* the node coefficient of
  // V* = (U*)^{3/4} (Eq. dis-cor-marshak1 with the predicted data)
  double *dsx, *ods;
  // mixed path: the preconditioner's last step z = r/alpha - zc u_j + zl u_{j-1} + zr u_{j+1}
  // (z = (r - Gbar u)/alpha, Gbar u = wv2 [gl (u_j - u_{j-1}) + gu (u_j - u_{j+1})] + wv gb u_j)
  double *zl, *zc, *zr;
};

// Binary32 copies of the per-cell values that the line and Krylov kernels use per
// element in the mixed mode (each converted once per cell, so that no per-element
// work touches the FP64 pipe).  Null in the FP64 mode.
struct CellF {
  float *A, *gl, *gu, *gb, *od, *dlx, *kcd, *kdx, *ratio, *ralpha, *alpha;
  float *kcde, *kdxe, *dlxe;    // kcd/eps, kdx/eps, dlx*eps (correction substep 2)
  float *fR, *fL, *gbx;         // rho-part flux coefficients (fused Krylov passes)
  float *dsx, *ods;             // binary32 copies of cf.dsx, cf.ods
  float *P1, *P2, *P3, *Frho;   // per-cell parts of a prediction pass
  float *Q1, *Q2, *gU;          // per-cell parts of correction substep 2
};

struct Dev {
  Inst* inst;
  Line* lines;
  double *v, *w, *bL, *bR;
  // state: per element the deviation Eh = E - a c U (E = a c U + Eh) and O, in the
  // bulk type of the precision mode (double or float); per cell T, U in double
  void *Eh, *O;
  double *T, *U, *sig;
  // per-cell
  double *rho_n, *rho_s, *Fs, *Us, *newton_its;
  double* Fc;      // the correction's flux (sigma_0/T^3: with V* = (U*)^{3/4}; sigma(x): = Fs)
  // per-cell parts of a line pass, computed once per cell in double
  double *P1, *P2, *P3, *Frho, *gU, *Q1, *Q2;
  double *gwork;   // per-cell double work vector of the Krylov kernels
  double *Swall;   // per (instance, angle): the two inflow-wall flux contributions in double
  CellCoef cf;
  CellF fc;
  // per-element work (bulk type)
  void *xb, *S, *F, *Rd, *onode;
  void* S2;        // per element: the correction's e/o flux part (sigma_0/T^3 data passes)
  // preconditioner factors
  double *pF, *pRd, *pG, *pH, *gw, *pInv;
  // GMRES
  double *gx, *gV, *gz, *gH, *gg, *gcs, *gsn, *gbeta, *gxn;
  int *gactive, *gk, *gdone, *gits, *gcycles, *gestconv;
  int* status;
  double* energy;   // 3 per instance
  // learned Newton guess: per-cell features (6 floats), predicted and logged targets
  float *feat, *guess, *ytrue;
  float* fdata;     // fused solve: data terms of the prediction, [slice cell][32 angles]
  int use_guess, log_samples;
  int start_prev;   // 1: Newton starts one step from T^n instead of the closed-form bound
  int m;  // restart length
  int maxcycles;  // restart cycles per step before ENONCONV
  double rtol, stall, wfloor;
  int mixed;
  int newton_maxit;
};

__device__ __forceinline__ void flag(int* status, int inst, int code) { atomicOr(status + inst, 1 << code); }

// The per-cell array of the bulk type R: the double original or its binary32 copy.
template <typename R>
__device__ __forceinline__ const R* pick(const double* d, const float* f);
template <>
__device__ __forceinline__ const double* pick<double>(const double* d, const float*) { return d; }
template <>
__device__ __forceinline__ const float* pick<float>(const double*, const float* f) { return f; }

// Arithmetic type of the Krylov vectors, preconditioner and Gram-Schmidt for a bulk
// type: double in both modes.  (With binary32 Krylov vectors the mixed mode's second
// restart accepted iterates whose wall-cell temperature was off by ~1e-5.)
template <typename R>
struct KryT { using type = double; };

// ----------------------------------------------------------------------------- cells
// Per-cell coefficients at temperature Tc (T^n for the prediction, T^{n+1} for
// correction substep 2).  kappa/theta as in Eq. dis-pre (sigma(x): kappa = 1,
// theta = T^3) or Eq. dis-pre-marshak (sigma_0/T^3: kappa = T^3 with node means,
// theta = 1).  d_i = kappa_i / (kappa_i eps^2/(c dt) + sig_i) with sig_i the
// harmonic mean of the two cells; gl/gu/gb are the tridiagonal streaming operator
// G (per unit v^2 and v) of kappa v (O_{j+1} - O_j)/dx after eliminating O.
__global__ void __launch_bounds__(256) k_cell_coef(Dev D, int n_inst, const int64_t* __restrict__ cell_inst_start,
                                                   int64_t ncell, int use_new_T) {
  // every node coefficient d_i once per block (launched with 256 threads): thread t computes
  // the left node of its cell, the right node is the next thread's (the block's last thread
  // computes its own)
  __shared__ double dn_s[256];
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = gid < ncell;
  // locate instance by binary search over cell offsets
  int lo = 0, hi = n_inst - 1;
  const int64_t gq = live ? gid : ncell - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (cell_inst_start[mid] <= gq) lo = mid; else hi = mid - 1;
  }
  const Inst I = D.inst[lo];
  const int64_t j = gq - I.cell_off;
  const int N = I.N;
  const double* T = D.T;   // T^n or T^{n+1}, whichever the caller has placed there
  (void)use_new_T;
  auto kap = [&](int64_t jj) -> double {
    if (I.kind == GRTE_SIGMA_CONST) return 1.0;
    double t = T[I.cell_off + jj];
    return I.p == 3.0 ? t * t * t : pow(t, I.p);
  };
  auto sig = [&](int64_t jj) -> double { return D.sig[I.cell_off + jj]; };
  // d_i = kn/(kn eps^2/(c dt) + sn), sn = 2 sl sr/(sl + sr): one division as
  // kn (sl + sr)/(kn eps^2/(c dt) (sl + sr) + 2 sl sr)
  auto dnode = [&](int64_t i) -> double {  // interior node i (1..N-1)
    const double kn = (I.kind == GRTE_SIGMA_CONST) ? 1.0 : 0.5 * (kap(i - 1) + kap(i));
    const double sl = sig(i - 1), sr = sig(i);
    if (sl > 0.0 && sr > 0.0) {
      const double ss = sl + sr;
      return kn * ss / (kn * I.e2cdt * ss + 2.0 * sl * sr);
    }
    return kn / (kn * I.e2cdt);
  };
  const double dl = (j >= 1) ? dnode(j) : 0.0;
  dn_s[threadIdx.x] = dl;
  __syncthreads();
  if (!live) return;
  const double dr = (j <= N - 2) ? ((threadIdx.x + 1 < blockDim.x) ? dn_s[threadIdx.x + 1] : dnode(j + 1)) : 0.0;
  const double kc = kap(j);
  const double sj = sig(j);
  const double Tj = T[gid];
  // theta: T^3 (sigma(x)); T^{3-p} for sigma_0/T^p (1 at p = 3)
  const double theta = (I.kind == GRTE_SIGMA_CONST) ? Tj * Tj * Tj : (I.p == 3.0 ? 1.0 : pow(Tj, 3.0 - I.p));
  const double eps2 = I.eps * I.eps;
  const double s = sj * I.Cv / (I.Cv * eps2 + 4.0 * sj * theta * I.dt * I.a * I.c);
  const bool inflow = I.bc == GRTE_BC_INFLOW;
  const double mL = (inflow && j == N - 1) ? 2.0 : 1.0;
  const double mR = (inflow && j == 0) ? 2.0 : 1.0;
  const bool wallc = inflow && (j == 0 || j == N - 1);
  const double kcd = kc * I.rcdt;
  const double alpha = kcd + s;
  const double ralpha = 1.0 / alpha;
  const double A = kcd + sj * I.reps2;
  const double gl = kc * mL * dl * I.rdx2, gu = kc * mR * dr * I.rdx2;
  const double gb = wallc ? kc * I.gbc : 0.0;
  const double od = dl * I.e2cdt, dlx = dl * I.rdx, kdx = kc * I.rdx;
  const double ratio = (sj * I.reps2 - s) * ralpha;
  const double fR = mR * dr * I.rdx, fL = mL * dl * I.rdx;
  const double gbx = wallc ? I.two_eps : 0.0;
  D.cf.kc[gid] = kc;
  D.cf.s[gid] = s;
  D.cf.alpha[gid] = alpha;
  D.cf.A[gid] = A;
  D.cf.gam[gid] = sj * theta * I.gamc;
  D.cf.gl[gid] = gl;
  D.cf.gu[gid] = gu;
  D.cf.gb[gid] = gb;
  D.cf.dl[gid] = dl;
  D.cf.od[gid] = od;
  D.cf.dlx[gid] = dlx;
  D.cf.kcd[gid] = kcd;
  D.cf.kdx[gid] = kdx;
  D.cf.sac[gid] = s * I.a * I.c;
  D.cf.ralpha[gid] = ralpha;
  D.cf.ratio[gid] = ratio;
  D.cf.fR[gid] = fR;
  D.cf.fL[gid] = fL;
  D.cf.gbx[gid] = gbx;
  if (D.mixed) {
    const CellF& f = D.fc;
    f.A[gid] = (float)A;
    f.gl[gid] = (float)gl;
    f.gu[gid] = (float)gu;
    f.gb[gid] = (float)gb;
    f.od[gid] = (float)od;
    f.dlx[gid] = (float)dlx;
    f.kcd[gid] = (float)kcd;
    f.kdx[gid] = (float)kdx;
    f.ratio[gid] = (float)ratio;
    f.ralpha[gid] = (float)ralpha;
    f.alpha[gid] = (float)alpha;
    f.kcde[gid] = (float)(kcd * I.inv_eps);
    f.kdxe[gid] = (float)(kdx * I.inv_eps);
    D.cf.zl[gid] = I.wv2 * gl * ralpha;
    D.cf.zr[gid] = I.wv2 * gu * ralpha;
    D.cf.zc[gid] = (I.wv2 * (gl + gu) + I.wv * gb) * ralpha;
    f.dlxe[gid] = (float)(dlx * I.eps);
    f.fR[gid] = (float)fR;
    f.fL[gid] = (float)fL;
    f.gbx[gid] = (float)gbx;
  }
}

__device__ __forceinline__ int inst_of(const int64_t* __restrict__ cell_inst_start, int n_inst, int64_t gid) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (cell_inst_start[mid] <= gid) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// a / b in binary64 from a binary32 reciprocal and one residual correction (relative error
// ~1e-14, a few binary64 operations instead of the divide sequence); outside the binary32
// range the plain division.
__device__ __forceinline__ double q_div(double a, double b) {
  if (!(fabs(b) > 1e-30 && fabs(b) < 1e30)) return a / b;
  const double r = (double)__frcp_rn((float)b);
  const double q = a * r;
  return q + (a - q * b) * r;
}

// u^{3/4} for u >= 0: y = u^{3/4} from binary32, then two Newton steps on y^4 = u^3
// (quadratic convergence from ~2^-22 to binary64 rounding).  The binary32 quantities
// u^{3/2} and 4 y^3 = 4 u^{9/4} stay normal for 1e-16 < u < 1e16; outside, the library power.
__device__ __forceinline__ double q_pow34(double u) {
  if (u == 0.0) return 0.0;
  if (!(u > 1e-16 && u < 1e16)) return pow(u, 0.75);
  const float uf = (float)u;
  double y = (double)sqrtf(uf * sqrtf(uf));
  const double u3 = u * u * u;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double y2 = y * y;
    y -= (y2 * y2 - u3) * (double)__frcp_rn((float)(4.0 * y2 * y));
  }
  return y;
}

// rho^n = sum_k w_k E^n_k = a c U^n + sum_k w_k Eh_k (sum_k w_k = 1), fixed angle order.
template <typename R>
__global__ void k_rho(Dev D, int n_inst, const int64_t* __restrict__ cell_inst_start, int64_t ncell,
                      double* __restrict__ out) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= ncell) return;
  const Inst I = D.inst[inst_of(cell_inst_start, n_inst, gid)];
  const int64_t j = gid - I.cell_off;
  const R* Eh = (const R*)D.Eh;
  double acc = 0.0;
  for (int k = 0; k < I.M; ++k) acc += D.w[I.ang_off + k] * (double)Eh[I.elem_off + (int64_t)k * I.N + j];
  out[gid] = I.a * I.c * D.U[gid] + acc;
}

// Per-cell parts of a prediction pass at the per-cell vector x (double, once per
// cell, so that the line kernels only combine them with per-angle factors):
//   P1 = -alpha x (+ s a c U^n + kappa/(c dt) a c U^n for a data pass)
//   P2 = (Gint x)_j,  P3 = gb_j x_j  (G_k x = v^2 P2 + v P3)
//   Frho = sum_k w_k v_k (O_{j+1,k} - O_{j,k}) of the rho part of O:
//          wv2 [fR (x_j - x_{j+1}) + fL (x_j - x_{j-1})] + wv gbx x_j
//          (data pass: minus 2/eps sum_k w_k v_k b at the inflow walls).
// X: type of the input vector (double for the iterate, the bulk type for a Krylov
// direction).
template <typename X>
__device__ __forceinline__ void cellpart_cell(const Dev& D, const Inst& I, int64_t gid, int64_t j,
                                              const X* __restrict__ x, int full) {
  const int64_t N = I.N;
  const double xj = x[j], xl = j > 0 ? (double)x[j - 1] : 0.0, xr = j < N - 1 ? (double)x[j + 1] : 0.0;
  double p1 = -D.cf.alpha[gid] * xj;
  if (full) p1 += (D.cf.sac[gid] + D.cf.kcd[gid] * I.a * I.c) * D.U[gid];
  const double p2 = D.cf.gl[gid] * (xj - xl) + D.cf.gu[gid] * (xj - xr);
  const double p3 = D.cf.gb[gid] * xj;
  double fr = I.wv2 * (D.cf.fR[gid] * (xj - xr) + D.cf.fL[gid] * (xj - xl)) + I.wv * D.cf.gbx[gid] * xj;
  if (full && I.bc == GRTE_BC_INFLOW) {
    if (j == 0) fr -= I.two_eps * I.bLflux;
    if (j == N - 1) fr -= I.two_eps * I.bRflux;
  }
  D.P1[gid] = p1;
  D.P2[gid] = p2;
  D.P3[gid] = p3;
  D.Frho[gid] = fr;
  if (D.mixed) {
    D.fc.P1[gid] = (float)p1;
    D.fc.P2[gid] = (float)p2;
    D.fc.P3[gid] = (float)p3;
    D.fc.Frho[gid] = (float)fr;
  }
  if (full && I.kind == GRTE_SIGMA_T3) {
    // node coefficient of the correction's flux at this cell's left node (interior
    // nodes): d* = V*/(V* eps^2/(c dt) + sig), V* = mean over the two cells of
    // max(U*, 0)^{3/4}, U* = (U^n + gam x)/(1 + gam a c)
    double ds = 0.0;
    if (j >= 1) {
      const double ac = I.a * I.c;
      const double ul = (D.U[gid - 1] + D.cf.gam[gid - 1] * xl) / (1.0 + D.cf.gam[gid - 1] * ac);
      const double ur = (D.U[gid] + D.cf.gam[gid] * xj) / (1.0 + D.cf.gam[gid] * ac);
      const double e4 = 0.25 * I.p;   // V* = max(U*, 0)^{p/4}
      const double vn = I.p == 3.0 ? 0.5 * (q_pow34(fmax(ul, 0.0)) + q_pow34(fmax(ur, 0.0)))
                                   : 0.5 * (pow(fmax(ul, 0.0), e4) + pow(fmax(ur, 0.0), e4));
      const double sl = D.sig[gid - 1], sr = D.sig[gid];
      const double sn = (sl > 0.0 && sr > 0.0) ? 2.0 * sl * sr / (sl + sr) : 0.0;
      const double den = vn * I.e2cdt + sn;
      ds = den > 0.0 ? vn / den : 0.0;
    }
    D.cf.dsx[gid] = ds * I.rdx;
    D.cf.ods[gid] = ds * I.e2cdt;
    if (D.mixed) {
      D.fc.dsx[gid] = (float)(ds * I.rdx);
      D.fc.ods[gid] = (float)(ds * I.e2cdt);
    }
  }
}

template <typename X>
__global__ void k_cellpart_pred(Dev D, int n_inst, const int64_t* __restrict__ cell_inst_start, int64_t ncell,
                                const X* __restrict__ xvec, int full) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= ncell) return;
  const int ii = inst_of(cell_inst_start, n_inst, gid);
  const Inst I = D.inst[ii];
  if (!full && !D.gactive[ii]) return;
  cellpart_cell<X>(D, I, gid, gid - I.cell_off, xvec + I.cell_off, full);
}

// Per-cell parts of correction substep 2 at T^{n+1} (U^n still in D.U):
//   Q1 = kappa/(c dt) a c (U^n - U^{n+1}) / eps,
//   gU_j = d_j/dx a c (U^{n+1}_j - U^{n+1}_{j-1}) at node j (0 at the wall node),
//   Q2 = gU_{j+1} - gU_j (interior; the wall cells are formed in double by the line kernel).
__global__ void k_cellpart_corr(Dev D, int n_inst, const int64_t* __restrict__ cell_inst_start, int64_t ncell) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= ncell) return;
  const Inst I = D.inst[inst_of(cell_inst_start, n_inst, gid)];
  const int64_t j = gid - I.cell_off, N = I.N;
  const double* T = D.T + I.cell_off;
  auto U1 = [&](int64_t jj) { const double t = T[jj]; const double t2 = t * t; return t2 * t2; };
  const double ac = I.a * I.c;
  D.Q1[gid] = D.cf.kcd[gid] * ac * (D.U[gid] - U1(j)) * I.inv_eps;
  const double gl = (j >= 1) ? D.cf.dlx[gid] * ac * (U1(j) - U1(j - 1)) : 0.0;
  const double gr = (j <= N - 2) ? D.cf.dlx[gid + 1] * ac * (U1(j + 1) - U1(j)) : 0.0;
  D.gU[gid] = gl;
  D.Q2[gid] = gr - gl;
  if (D.mixed) {
    D.fc.Q1[gid] = (float)D.Q1[gid];
    D.fc.Q2[gid] = (float)(gr - gl);
    D.fc.gU[gid] = (float)gl;
  }
}

// ----------------------------------------------------------------------------- lines
template <typename R>
struct LineCoef {  // A + v^2 Gint + v Gbdry of one line, in the bulk type R
  const R *A, *gl, *gu, *gb;
  R v, v2;
  int64_t N;
  __device__ R a(int64_t j) const { return j > 0 ? -v2 * gl[j] : R(0); }
  __device__ R c(int64_t j) const { return j < N - 1 ? -v2 * gu[j] : R(0); }
  __device__ R b(int64_t j) const { return A[j] + v2 * (gl[j] + gu[j]) + v * gb[j]; }
};

enum { PRED_FULL_FACTOR = 0, PRED_FULL = 1, PRED_HOM = 2 };

// Shared-memory layout of a line CTA: [x (padded), if XS] [reduced system].
template <typename R, bool XS>
__device__ __forceinline__ XAcc<R, XS> line_x(unsigned char* dsm, R* xglob) {
  return XAcc<R, XS>{XS ? (R*)dsm : xglob};
}
template <typename R, bool XS>
__device__ __forceinline__ R* line_red(unsigned char* dsm, int64_t N) {
  const int64_t off = XS ? ((tri_xs_len(N) * (int64_t)sizeof(R) + 15) / 16) * 16 : 0;
  return (R*)(dsm + off);
}

// One prediction pass over a line (instance, k) for the per-cell vector x (rho or a
// Krylov direction): right-hand side of the e-equation
//   r = h_k - alpha x - G_k x = P1 - v^2 P2 - v P3 + kappa/(c dt) Eh^n_k - kappa v D_k/dx
// (D_k = o_{j+1} - o_j, o_i = d_i eps^2 O^n_i/(c dt), Eq. dis-pre1; walls Eq. bc-pre),
// tridiagonal solve for e_k in R, and the e/o part of w_k v_k (O_{j+1,k} - O_{j,k})
// into S (the rho part is Frho, per cell in double).  In the two wall cells the
// right-hand side and the flux are formed in double: there (2/eps)(b - x) is an
// O(eps) difference of O(1) numbers.  HOM passes carry no data.  NT threads per
// line; with XS the line's unknowns stay in shared memory for the whole pass (only
// the flux leaves the CTA), else they live in the global scratch xb.
template <int MODE, typename R, int NT, bool XS>
__global__ void __launch_bounds__(NT, 1024 / NT) k_pred_line(Dev D, const void* __restrict__ xvec) {
  using XT = typename std::conditional<MODE == PRED_HOM, typename KryT<R>::type, double>::type;   // Krylov direction or iterate
  extern __shared__ __align__(16) unsigned char dsm[];
  const Line L = D.lines[blockIdx.x];
  const Inst I = D.inst[L.inst];
  if (MODE == PRED_HOM && !D.gactive[L.inst]) return;
  const int64_t N = I.N;
  const int k = L.k;
  const double v = D.v[I.ang_off + k], w = D.w[I.ang_off + k];
  const bool inflow = I.bc == GRTE_BC_INFLOW;
  const double bL = (MODE == PRED_HOM || !inflow) ? 0.0 : D.bL[I.ang_off + k];
  const double bR = (MODE == PRED_HOM || !inflow) ? 0.0 : D.bR[I.ang_off + k];
  const int64_t co = I.cell_off, eo = I.elem_off + (int64_t)k * N, oo = I.nelem_off + (int64_t)k * (N + 1);
  const XT* x = (const XT*)xvec + co;
  const XAcc<R, XS> xb = line_x<R, XS>(dsm, (R*)D.xb + eo);
  // per-cell values in the bulk type for the per-element work
  const R *P1r = pick<R>(D.P1, D.fc.P1) + co, *P2r = pick<R>(D.P2, D.fc.P2) + co,
          *P3r = pick<R>(D.P3, D.fc.P3) + co, *kcdr = pick<R>(D.cf.kcd, D.fc.kcd) + co,
          *kdxr = pick<R>(D.cf.kdx, D.fc.kdx) + co, *odr = pick<R>(D.cf.od, D.fc.od) + co,
          *dlxr = pick<R>(D.cf.dlx, D.fc.dlx) + co;
  // double originals for the two inflow wall cells
  const double *gl = D.cf.gl + co, *gu = D.cf.gu + co, *gb = D.cf.gb + co, *dlx = D.cf.dlx + co,
               *kcd = D.cf.kcd + co, *kdx = D.cf.kdx + co, *P1 = D.P1 + co, *P2 = D.P2 + co;
  const R* Ehn = (const R*)D.Eh + eo;
  const R* On = (const R*)D.O + oo;
  const double v2 = v * v;
  const R vr = R(v), v2r = R(v2);
  const double two_eps = I.two_eps;
  auto onode = [&](int64_t i) -> R {   // o_i in R
    if (MODE == PRED_HOM) return R(0);
    if (i <= 0 || i >= N) return R(0);
    return odr[i] * On[i];
  };
  // right-hand side of an inflow wall row, in double:
  // -v gb x + kappa v (2/eps) b/dx = kappa v (2/eps)(b - x)/dx is an O(eps) difference
  auto wall_rhs = [&](int64_t j) -> double {
    const double b = (j == 0) ? bL : bR;
    double r = P1[j] - v2 * P2[j] + kdx[j] * v * two_eps * (b - (double)x[j]);
    if (MODE != PRED_HOM) {
      const double o = (j == 0) ? 2.0 * (double)onode(1) : -2.0 * (double)onode(N - 1);
      r += kcd[j] * (double)Ehn[j] - kdx[j] * v * o;
    }
    return r;
  };
#pragma unroll 4
  for (int64_t j = threadIdx.x; j < N; j += NT) {
    const bool wall = inflow && (j == 0 || j == N - 1);
    if (!wall) {
      R r = P1r[j] - v2r * P2r[j] - vr * P3r[j];
      if (MODE != PRED_HOM) r += kcdr[j] * Ehn[j] - kdxr[j] * vr * (onode(j + 1) - onode(j));
      xb[j] = r;
    } else {
      xb[j] = R(wall_rhs(j));
    }
  }
  __syncthreads();
  LineCoef<R> cfl{pick<R>(D.cf.A, D.fc.A) + co, pick<R>(D.cf.gl, D.fc.gl) + co, pick<R>(D.cf.gu, D.fc.gu) + co,
                  pick<R>(D.cf.gb, D.fc.gb) + co, vr, v2r, N};
  R* F = (R*)D.F + L.f_off;
  R* Rd = (R*)D.Rd + L.red_off;
  R* red = line_red<R, XS>(dsm, N);
  if (MODE == PRED_FULL_FACTOR) tri_solve<true>(cfl, N, xb, F, Rd, red);
  else tri_solve<false>(cfl, N, xb, F, Rd, red);
  // the wall unknowns enter the wall flux multiplied by 2/eps: re-solve their rows in
  // double from the neighbours (the rows are dominated by v gb ~ 1/eps, so the
  // neighbour's bulk-precision error is damped by |c/b|)
  __shared__ double ew[2];
  if (inflow && threadIdx.x == 0) {
    const double b0 = D.cf.A[co] + v2 * (gl[0] + gu[0]) + v * gb[0];
    ew[0] = (wall_rhs(0) + v2 * gu[0] * (double)xb[1]) / b0;
    const double bN = D.cf.A[co + N - 1] + v2 * (gl[N - 1] + gu[N - 1]) + v * gb[N - 1];
    ew[1] = (wall_rhs(N - 1) + v2 * gl[N - 1] * (double)xb[N - 2]) / bN;
  }
  __syncthreads();
  // e/o part of w_k v_k (O_{j+1,k} - O_{j,k}):
  //   O^eo_i = o_i - d_i v (e_i - e_{i-1})/dx (interior nodes)
  //   j = 0:   2 O^eo_1 + (2/eps) e_0       (the b_L and x parts are in Frho)
  //   j = N-1: (2/eps) e_{N-1} - 2 O^eo_{N-1}
  R* Sk = (R*)D.S + eo;
  const R wvr = R(w * v);
  // the correction's flux (sigma_0/T^3 data passes): the same with the node coefficient
  // d* of V* = (U*)^{3/4} (cf.dsx = d*/dx, cf.ods = d* eps^2/(c dt), from the per-cell parts)
  const bool corr = MODE != PRED_HOM && I.kind == GRTE_SIGMA_T3;
  if (inflow && threadIdx.x == 0) {   // wall cells: e/o flux in double, kept in Swall
    const double eL = ew[0], eR = ew[1];
    const double e1 = (N > 2) ? (double)xb[1] : eR, eN2 = (N > 2) ? (double)xb[N - 2] : eL;
    const double O1 = (double)onode(1) - dlx[1] * v * (e1 - eL);
    const double ON1 = (double)onode(N - 1) - dlx[N - 1] * v * (eR - eN2);
    D.Swall[2 * (I.ang_off + k) + 0] = w * v * (2.0 * O1 + two_eps * eL);
    D.Swall[2 * (I.ang_off + k) + 1] = w * v * (two_eps * eR - 2.0 * ON1);
  }
  if (corr) {
    R* S2k = (R*)D.S2 + eo;
    const R *dsxr = pick<R>(D.cf.dsx, D.fc.dsx) + co, *odsr = pick<R>(D.cf.ods, D.fc.ods) + co;
    for (int64_t j = threadIdx.x; j < N; j += NT) {
      auto Oc = [&](int64_t i) -> R { return odsr[i] * On[i] - dsxr[i] * vr * (xb[i] - xb[i - 1]); };
      // (the inflow wall cells keep the prediction's flux: not read there)
      const R OR = (j + 1 <= N - 1) ? Oc(j + 1) : R(0);
      const R OL = (j >= 1) ? Oc(j) : R(0);
      S2k[j] = wvr * (OR - OL);
    }
  }
#pragma unroll 4
  for (int64_t j = threadIdx.x; j < N; j += NT) {
    auto Oeo = [&](int64_t i) -> R { return onode(i) - dlxr[i] * vr * (xb[i] - xb[i - 1]); };
    R val;
    if (inflow && (j == 0 || j == N - 1)) {
      val = R(0);                       // in Swall
    } else {
      const R OR = (j + 1 <= N - 1) ? Oeo(j + 1) : R(0);
      const R OL = (j >= 1) ? Oeo(j) : R(0);
      val = OR - OL;
    }
    Sk[j] = wvr * val;
  }
}

// ----------------------------------------------------------------------------- instance (GMRES)
// The per-instance Krylov work runs on a thread-block cluster of kCL CTAs: each CTA
// owns a contiguous slice of the instance's cells; dot products are reduced through
// distributed shared memory (fixed rank order, so every CTA gets the same value);
// the preconditioner's tridiagonal solve is partitioned across the cluster by the
// spike method (local solves plus a 2*kCL interface system).
constexpr int kCL = 8;

template <typename K>
struct PrecCoef {  // A + (A/alpha) (wv2 Gint + wv Gbdry), evaluated in double, stored in K
  const double *A, *gl, *gu, *gb, *ralpha;
  double wv, wv2;
  int64_t N;
  __device__ double f(int64_t j) const { return A[j] * ralpha[j]; }
  __device__ K a(int64_t j) const { return j > 0 ? K(-f(j) * wv2 * gl[j]) : K(0); }
  __device__ K c(int64_t j) const { return j < N - 1 ? K(-f(j) * wv2 * gu[j]) : K(0); }
  __device__ K b(int64_t j) const { return K(A[j] + f(j) * (wv2 * (gl[j] + gu[j]) + wv * gb[j])); }
};

template <typename K>
struct SliceCoef {  // the rows [c0, c0+n) of a system, decoupled from the rest
  PrecCoef<K> p;
  int64_t c0, n;
  __device__ K a(int64_t j) const { return j > 0 ? p.a(c0 + j) : K(0); }
  __device__ K c(int64_t j) const { return j < n - 1 ? p.c(c0 + j) : K(0); }
  __device__ K b(int64_t j) const { return p.b(c0 + j); }
};

struct Slice {
  int nact;        // CTAs that own cells (>= 1)
  int64_t c0, n;   // this CTA's cells [c0, c0+n) (n = 0 if rank >= nact)
};

__device__ __forceinline__ Slice slice_of(int64_t N, int rank) {
  Slice sl;
  int64_t half = N / 2;
  sl.nact = (int)(half < kCL ? half : kCL);
  if (rank >= sl.nact) { sl.c0 = N; sl.n = 0; return sl; }
  const int64_t base = N / sl.nact, rem = N % sl.nact;
  sl.c0 = rank * base + (rank < rem ? rank : rem);
  sl.n = base + (rank < rem ? 1 : 0);
  return sl;
}

// Reduced-system storage of the preconditioner: kCL slices, each tri_red_size(slice).
__host__ __device__ inline int64_t prec_red_size(int64_t N) {
  int64_t half = N / 2;
  int nact = (int)(half < kCL ? half : kCL);
  int64_t base = N / nact;
  return (int64_t)kCL * tri_red_size(base + 1, kTriThreads);
}
// Factor storage of the preconditioner slices: slice (instance ii, rank) starts at
// 5 (cell_off + c0 + (ii kCL + rank) kTriThreads), room for tri_fac_size(n, kTriThreads).
__host__ __device__ inline int64_t prec_fac_off(int64_t cell_off, int64_t c0, int ii, int rank) {
  return 5 * (cell_off + c0 + ((int64_t)ii * kCL + rank) * kTriThreads);
}

struct GmresSmem {
  double tri[4 * 2 * kTriThreads];   // reduced system of the slice solves
  double red[32];
  double part[2][kMaxRestart + 2];   // double-buffered partial sums exchanged by DSMEM
  double ends[6];                    // y_first, y_last, g_first, g_last, h_first, h_last
  double xlr[2];                     // interface values left of and right of this slice
  double hcol[kMaxRestart + 2];
  double y[kMaxRestart];
  double gj[2 * kCL][4 * kCL];          // Gauss-Jordan workspace of the interface system
  double yv[2 * kCL];                   // gathered slice-end values
  double redm[32][kMaxRestart + 2];     // per-warp partials of a multi-value reduction
};

__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];   // same order in every thread
  return t;
}

// Sum nv per-CTA partial values over the cluster (fixed rank order).  `buf` selects
// the half of the double buffer; two consecutive calls must use different halves.
__device__ void cluster_sums(cg::cluster_group& cl, GmresSmem& sm, int buf, const double* mine, int nv,
                             double* out) {
  if (threadIdx.x < nv) sm.part[buf][threadIdx.x] = mine[threadIdx.x];
  cl.sync();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int r = 0; r < kCL; ++r) t += cl.map_shared_rank(&sm.part[buf][0], r)[threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// Max of nv per-CTA values over the cluster.
__device__ void cluster_maxs(cg::cluster_group& cl, GmresSmem& sm, int buf, const double* mine, int nv,
                             double* out) {
  if (threadIdx.x < nv) sm.part[buf][threadIdx.x] = mine[threadIdx.x];
  cl.sync();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int r = 0; r < kCL; ++r) t = fmax(t, cl.map_shared_rank(&sm.part[buf][0], r)[threadIdx.x]);
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

__device__ double cta_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t = fmax(t, red[i]);
  return t;
}

// z = P^{-1} r on this CTA's slice, P the single-effective-angle Schur operator:
//   u = (A + (A/alpha) Gbar)^{-1} (beta/alpha) r,  z = (r - Gbar u)/alpha,
//   Gbar = sum_k w_k G_k, beta = A - alpha.
// The tridiagonal solve is split over the cluster: each slice solves its own rows
// (y), and in FACTOR mode also the two spike vectors g, h (its response to the
// coupling with the neighbouring slices); the 2*nact end values then give the
// slice-boundary unknowns, and u = y - u_left g - u_right h.
// K: arithmetic type of the Krylov vectors (the bulk type); RT: type of r.
template <bool FACTOR, bool XS, typename K, typename RT>
__device__ void prec_apply_cl(const Dev& D, const Inst& I, const Slice& sl, int rank, cg::cluster_group& cl,
                              const RT* r, K* z, K* work, K* wsm, GmresSmem& sm) {
  const int64_t N = I.N, co = I.cell_off, c0 = sl.c0, n = sl.n;
  const double *A = D.cf.A + co, *gl = D.cf.gl + co, *gu = D.cf.gu + co, *gb = D.cf.gb + co,
               *ralpha = D.cf.ralpha + co;
  const K *ratio_k = pick<K>(D.cf.ratio, D.fc.ratio) + co, *ralpha_k = pick<K>(D.cf.ralpha, D.fc.ralpha) + co,
          *gl_k = pick<K>(D.cf.gl, D.fc.gl) + co, *gu_k = pick<K>(D.cf.gu, D.fc.gu) + co,
          *gb_k = pick<K>(D.cf.gb, D.fc.gb) + co;
  K* pg = (K*)D.pG + co;
  K* ph = (K*)D.pH + co;
  PrecCoef<K> pc{A, gl, gu, gb, ralpha, I.wv, I.wv2, N};
  SliceCoef<K> sc{pc, c0, n};
  K* F = (K*)D.pF + prec_fac_off(co, c0, blockIdx.x / kCL, rank);
  K* Rd = (K*)D.pRd + I.red_off + (int64_t)rank * (prec_red_size(N) / kCL);
  K* red = (K*)sm.tri;
  // the slice's unknowns: shared memory (XS) or the global work vector
  const XAcc<K, XS> wx{XS ? wsm : work + c0};
  const XAcc<K, false> gx{pg + c0}, hx{ph + c0};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) wx[j] = ratio_k[c0 + j] * K(r[c0 + j]);
  __syncthreads();
  if (n > 0) {
    tri_solve<FACTOR>(sc, n, wx, F, Rd, red);
    if (FACTOR) {
      for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
        pg[c0 + j] = (j == 0) ? pc.a(c0) : K(0);
        ph[c0 + j] = (j == n - 1) ? pc.c(c0 + n - 1) : K(0);
      }
      __syncthreads();
      tri_solve<false>(sc, n, gx, F, Rd, red);
      tri_solve<false>(sc, n, hx, F, Rd, red);
    }
    if (threadIdx.x == 0) {
      sm.ends[0] = (double)wx[0];
      sm.ends[1] = (double)wx[n - 1];
      sm.ends[2] = (double)pg[c0];
      sm.ends[3] = (double)pg[c0 + n - 1];
      sm.ends[4] = (double)ph[c0];
      sm.ends[5] = (double)ph[c0 + n - 1];
    }
  }
  cl.sync();
  // interface unknowns X[2q] = u at the first cell of slice q, X[2q+1] = at its last:
  //   X[2q]   + g_first(q) X[2q-1] + h_first(q) X[2q+2] = y_first(q)
  //   X[2q+1] + g_last(q)  X[2q-1] + h_last(q)  X[2q+2] = y_last(q)
  // The matrix depends only on the operator: FACTOR inverts it once per step (one
  // warp, Gauss-Jordan with partial pivoting) and stores the two rows this slice
  // needs; every apply is then two short dot products.
  const int na = sl.nact, m2 = 2 * na;
  double* inv_rows = D.pInv + ((int64_t)blockIdx.x) * 2 * (2 * kCL);
  if (FACTOR && threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int w2 = 2 * m2;
    for (int idx = lane; idx < m2 * w2; idx += 32) {
      const int i = idx / w2, j = idx % w2;
      sm.gj[i][j] = 0.0;
    }
    __syncwarp();
    if (lane < m2) {
      const int q = lane / 2, t = lane % 2;
      const double* e = cl.map_shared_rank(&sm.ends[0], q);
      sm.gj[lane][lane] = 1.0;
      if (q > 0) sm.gj[lane][2 * q - 1] += e[2 + t];
      if (q < na - 1) sm.gj[lane][2 * q + 2] += e[4 + t];
      sm.gj[lane][m2 + lane] = 1.0;
    }
    __syncwarp();
    for (int col = 0; col < m2; ++col) {
      int piv = col;
      if (lane == 0)
        for (int i = col + 1; i < m2; ++i)
          if (fabs(sm.gj[i][col]) > fabs(sm.gj[piv][col])) piv = i;
      piv = __shfl_sync(0xffffffffu, piv, 0);
      if (piv != col)
        for (int j = lane; j < w2; j += 32) {
          const double t = sm.gj[col][j];
          sm.gj[col][j] = sm.gj[piv][j];
          sm.gj[piv][j] = t;
        }
      __syncwarp();
      const double ip = 1.0 / sm.gj[col][col];
      __syncwarp();
      for (int j = lane; j < w2; j += 32) sm.gj[col][j] *= ip;
      __syncwarp();
      double f = (lane < m2 && lane != col) ? sm.gj[lane][col] : 0.0;
      __syncwarp();
      for (int i = 0; i < m2; ++i) {
        const double fi = __shfl_sync(0xffffffffu, f, i);
        if (i != col && fi != 0.0)
          for (int j = lane; j < w2; j += 32) sm.gj[i][j] -= fi * sm.gj[col][j];
      }
      __syncwarp();
    }
    // rows 2 rank - 1 and 2 rank + 2 of the inverse (columns m2 .. 2 m2 - 1)
    for (int j = lane; j < m2; j += 32) {
      inv_rows[j] = (rank > 0 && rank < na) ? sm.gj[2 * rank - 1][m2 + j] : 0.0;
      inv_rows[2 * kCL + j] = (rank < na - 1) ? sm.gj[2 * rank + 2][m2 + j] : 0.0;
    }
  }
  if (threadIdx.x < m2) {
    const int q = threadIdx.x / 2, t = threadIdx.x % 2;
    sm.yv[threadIdx.x] = cl.map_shared_rank(&sm.ends[0], q)[t];
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double acc = 0.0;
    const double* row = inv_rows + threadIdx.x * 2 * kCL;
    for (int j = 0; j < m2; ++j) acc += row[j] * sm.yv[j];
    sm.xlr[threadIdx.x] = acc;
  }
  __syncthreads();
  const K ul = K(sm.xlr[0]), ur = K(sm.xlr[1]);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) wx[j] = wx[j] - ul * pg[c0 + j] - ur * ph[c0 + j];
  __syncthreads();
  const K wv2 = K(I.wv2), wv = K(I.wv);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const int64_t g = c0 + j;
    const K uj = wx[j];
    const K uL = g > 0 ? (j > 0 ? wx[j - 1] : ul) : K(0);
    const K uR = g < N - 1 ? (j < n - 1 ? wx[j + 1] : ur) : K(0);
    const K Gu = wv2 * (gl_k[g] * (uj - uL) + gu_k[g] * (uj - uR)) + wv * gb_k[g] * uj;
    z[g] = (K(r[g]) - Gu) * ralpha_k[g];
  }
  __syncthreads();
}

// F_j = sum_k w_k v_k (O_{j+1,k} - O_{j,k}) of a pass: the per-cell rho part plus the
// per-angle e/o parts, 16 loads issued together, four partial sums (type A) combined
// in a fixed order; the two inflow wall cells sum their double wall fluxes.
template <typename R, typename A = R>
__device__ __forceinline__ A eo_sum(const Dev& D, const Inst& I, int64_t j) {
  const R* S = (const R*)D.S + I.elem_off + j;
  const int64_t N = I.N;
  A p[4] = {A(0), A(0), A(0), A(0)};
  int k = 0;
  for (; k + 16 <= I.M; k += 16) {
    R t[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) t[q] = S[(int64_t)(k + q) * N];
#pragma unroll
    for (int q = 0; q < 16; ++q) p[q & 3] += A(t[q]);
  }
  for (; k < I.M; ++k) p[k & 3] += A(S[(int64_t)k * N]);
  return (p[0] + p[1]) + (p[2] + p[3]);
}

__device__ __forceinline__ bool wall_cell(const Inst& I, int64_t j) {
  return I.bc == GRTE_BC_INFLOW && (j == 0 || j == I.N - 1);
}

__device__ __forceinline__ double wall_sum(const Dev& D, const Inst& I, int64_t j) {
  const int side = (j == 0) ? 0 : 1;
  double acc = 0.0;
  for (int k = 0; k < I.M; ++k) acc += D.Swall[2 * (I.ang_off + k) + side];
  return acc;
}

// in double (true residual): each e/o part converted and summed in double
template <typename R>
__device__ __forceinline__ double flux_sum(const Dev& D, const Inst& I, int64_t j) {
  const double fr = D.Frho[I.cell_off + j];
  if (wall_cell(I, j)) return fr + wall_sum(D, I, j);
  return fr + eo_sum<R, double>(D, I, j);
}

// in the bulk type (Krylov directions)
template <typename R>
__device__ __forceinline__ R flux_sum_k(const Dev& D, const Inst& I, int64_t j) {
  if (wall_cell(I, j)) return R(D.Frho[I.cell_off + j] + wall_sum(D, I, j));
  return pick<R>(D.Frho, D.fc.Frho)[I.cell_off + j] + eo_sum<R>(D, I, j);
}

// The correction's flux at a cell j that is not an inflow wall cell (sigma_0/T^3, the
// node coefficients d* of the data pass that just ran at the iterate x): its rho part
//   wv2 [d*_{j+1} (x_j - x_{j+1}) + d*_j (x_j - x_{j-1})]/dx
// plus the per-angle e/o parts S2 (in double).  The inflow wall cells keep the
// prediction's flux (the wall node takes the prediction's value shifted by the change at
// the adjacent node).
template <typename R>
__device__ __forceinline__ double corr_flux_sum(const Dev& D, const Inst& I, int64_t j, const double* x) {
  const int64_t N = I.N, co = I.cell_off;
  const double xj = x[j], xl = j > 0 ? x[j - 1] : 0.0, xr = j < N - 1 ? x[j + 1] : 0.0;
  const double dR = j < N - 1 ? D.cf.dsx[co + j + 1] : 0.0, dL = D.cf.dsx[co + j];
  const double f = I.wv2 * (dR * (xj - xr) + dL * (xj - xl));
  const R* S = (const R*)D.S2 + I.elem_off + j;
  double acc = 0.0;
  for (int k = 0; k < I.M; ++k) acc += (double)S[(int64_t)k * N];
  return f + acc;
}

enum { G_RESTART_FIRST = 0, G_RESTART = 1, G_ARNOLDI = 2, G_UPDATE = 3 };


// GMRES bookkeeping, one cluster per instance (restart length m, left
// preconditioned).  Vectors live in global memory: x (iterate), V[0..m] (Krylov
// basis), z (scratch).  Scalars (H, g, Givens) are computed identically by every
// CTA; rank 0 stores them.
template <int MODE, typename R, bool XS>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kTriThreads) k_gmres(Dev D, int jcol) {
  using K = typename KryT<R>::type;   // arithmetic of the Krylov vectors
  // FP64 mode: the per-cell parts of the next pass are formed here (no separate launch)
  constexpr bool FUSED_PARTS = sizeof(R) == 8;
  __shared__ GmresSmem sm;
  extern __shared__ __align__(16) unsigned char gdsm[];   // the slice's unknowns (XS)
  K* wsm = (K*)gdsm;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int ii = blockIdx.x / kCL;
  const Inst I = D.inst[ii];
  const int64_t N = I.N, co = I.cell_off;
  const Slice sl = slice_of(N, rank);
  const int64_t c0 = sl.c0, n = sl.n;
  const int m = D.m;
  double* x = D.gx + co;           // iterate, double
  double* zd = D.gz + co;          // scratch as double (residual) ...
  K* zk = (K*)D.gz + co;           // ... or as K (a preconditioner input)
  K* work = (K*)D.gwork + co;
  const int64_t ncell_tot = D.gz - D.gx;     // gz = gx + ncell_total (allocation layout)
  auto Vi = [&](int i) { return (K*)D.gV + (int64_t)i * ncell_tot + co; };
  double* H = D.gH + (int64_t)ii * (kMaxRestart + 1) * kMaxRestart;
  double* g = D.gg + (int64_t)ii * (kMaxRestart + 1);
  double* cs = D.gcs + (int64_t)ii * kMaxRestart;
  double* sn = D.gsn + (int64_t)ii * kMaxRestart;
  const double *alpha = D.cf.alpha + co, *kcd = D.cf.kcd + co, *kdx = D.cf.kdx + co, *sac = D.cf.sac + co;

  if (MODE == G_RESTART_FIRST || MODE == G_RESTART) {
    if (MODE == G_RESTART && D.gdone[ii]) return;        // uniform over the cluster
    // the previous restart's values, read before any CTA of the cluster can overwrite
    // them (rank 0 stores the new ones below): every CTA takes the same decision
    const double beta_prev = D.gbeta[ii];
    const int cycles_prev = D.gcycles[ii];
    // r = -R(x) from the FULL pass that just ran at x
    double* r = zd;
    for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) {
      const double fl = flux_sum<R>(D, I, j);
      const double Rj = alpha[j] * x[j] - kcd[j] * D.rho_n[co + j] - sac[j] * D.U[co + j] + kdx[j] * fl;
      r[j] = -Rj;
      D.Fs[co + j] = fl;                    // F* of the current iterate (final at convergence)
      D.Fc[co + j] = (I.kind == GRTE_SIGMA_T3 && !wall_cell(I, j)) ? corr_flux_sum<R>(D, I, j, x) : fl;
    }
    // per-cell weights of the stopping test: the preconditioned residual relative to
    // |x_j| (floor wfloor max|x|: 1e-13 in FP64, 1e-8 with binary32 line solves), so
    // that the test bounds every cell's relative correction and not only the large
    // cells' share of a 2-norm
    double xm = 0.0;
    for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) xm = fmax(xm, fabs(x[j]));
    xm = cta_max(xm, sm.red);
    __shared__ double xms[1];
    cluster_maxs(cl, sm, 0, &xm, 1, xms);
    for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x)
      D.gw[co + j] = 1.0 / (fabs(x[j]) + D.wfloor * xms[0] + 1e-300);
    __syncthreads();
    K* v0 = Vi(0);
    if (MODE == G_RESTART_FIRST) prec_apply_cl<true, XS, K, double>(D, I, sl, rank, cl, r, v0, work, wsm, sm);
    else prec_apply_cl<false, XS, K, double>(D, I, sl, rank, cl, r, v0, work, wsm, sm);
    double loc[3] = {0.0, 0.0, 0.0};
    K ss = K(0);
    for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) {
      const K vj = v0[j];
      ss += vj * vj;
      loc[1] += x[j] * x[j];
      loc[2] = fmax(loc[2], fabs((double)vj) * D.gw[co + j]);
    }
    loc[0] = (double)ss;
    loc[0] = cta_sum(loc[0], sm.red);
    loc[1] = cta_sum(loc[1], sm.red);
    loc[2] = cta_max(loc[2], sm.red);
    __shared__ double tots[2], tmax[1];
    cluster_sums(cl, sm, 1, loc, 2, tots);
    cluster_maxs(cl, sm, 0, loc + 2, 1, tmax);
    const double nrm = sqrt(tots[0]), xn = sqrt(tots[1]);
    const double rinf = tmax[0];
    // Converged when every cell's relative preconditioned correction is below rtol.
    // Restarted GMRES cannot go below the rounding floor of the residual evaluation
    // itself (a sum of terms much larger than the residual): a restart cycle that
    // did not reduce it by 4x while it is below 1e-9 has reached that floor.
    bool conv = !(rinf > D.rtol);   // also true for rinf == 0
    if (MODE == G_RESTART && !conv && rinf <= D.stall &&
        (rinf >= 0.25 * beta_prev || (D.mixed && cycles_prev >= 1))) conv = true;
    if (rank == 0 && threadIdx.x == 0) {
      if (MODE == G_RESTART) D.gcycles[ii] += 1;
      D.gbeta[ii] = rinf;
      D.gxn[ii] = xn;
      D.gestconv[ii] = 0;
      if (conv) {
        D.gactive[ii] = 0;
        D.gdone[ii] = 1;
      } else {
        D.gactive[ii] = 1;
        D.gdone[ii] = 0;
        g[0] = nrm;
        for (int i = 1; i <= m; ++i) g[i] = 0.0;
        D.gk[ii] = 0;
      }
      if (!isfinite(nrm)) flag(D.status, ii, GRTE_ENAN);
    }
    if (!conv) {
      const K inv = K(1.0 / nrm);
      for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) v0[j] *= inv;
    }
    cl.sync();   // no CTA leaves while another may still read its shared memory
    // per-cell parts of the first direction pass (V_0 of the neighbouring slices is
    // complete after the cluster barrier)
    // (FP64 mode only: in the mixed mode the per-cell kernel runs on all SMs instead,
    // since this kernel's FP64 rate on one cluster per instance would be the limit)
    if (FUSED_PARTS && !conv)
      for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) cellpart_cell<K>(D, I, co + j, j, v0, 0);
    return;
  }

  if (MODE == G_ARNOLDI) {
    if (!D.gactive[ii]) return;                           // uniform over the cluster
    // g[jcol] is rotated by rank 0 at the end of this step: read it now, before the
    // cluster barriers below, so that no CTA can see the rotated value and every CTA
    // takes the same continue/stop decision
    const double g_jcol = g[jcol];
    // C v_j = alpha v_j + kappa/dx * sum_k S_k  (the HOM pass just ran on v_j)
    const K* vj = Vi(jcol);
    K* cv = zk;
    const K *alpha_k = pick<K>(D.cf.alpha, D.fc.alpha) + co, *kdx_k = pick<K>(D.cf.kdx, D.fc.kdx) + co;
    for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x)
      cv[j] = alpha_k[j] * vj[j] + kdx_k[j] * K(flux_sum_k<R>(D, I, j));
    __syncthreads();
    K* wv = Vi(jcol + 1);
    prec_apply_cl<false, XS, K, K>(D, I, sl, rank, cl, cv, wv, work, wsm, sm);
    // classical Gram-Schmidt, twice (CGS2): two cluster reductions instead of j+1
    __shared__ double dots[kMaxRestart + 2];
    __shared__ double hc[kMaxRestart + 2];   // Hessenberg column (thread 0 finishes it)
    __shared__ int cont_s;                   // 1: another Arnoldi step follows
    if (threadIdx.x <= jcol + 1) hc[threadIdx.x] = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      // all jcol+1 dot products in one sweep and one CTA reduction
      // per-thread partial sums in K, reductions in double
      K lk[kMaxRestart + 1];
      double loc[kMaxRestart + 1];
      for (int i = 0; i <= jcol; ++i) lk[i] = K(0);
      for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) {
        const K wj = wv[j];
        for (int i = 0; i <= jcol; ++i) lk[i] += wj * Vi(i)[j];
      }
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int i = 0; i <= jcol; ++i) {
        double v = (double)lk[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sm.redm[wid][i] = v;
      }
      __syncthreads();
      for (int i = 0; i <= jcol; ++i) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sm.redm[w][i];   // same order in every thread
        loc[i] = t;
      }
      __syncthreads();
      cluster_sums(cl, sm, pass, loc, jcol + 1, dots);
      for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) {
        K t = wv[j];
        for (int i = 0; i <= jcol; ++i) t -= K(dots[i]) * Vi(i)[j];
        wv[j] = t;
      }
      if (threadIdx.x <= jcol) hc[threadIdx.x] += dots[threadIdx.x];
      __syncthreads();
    }
    K l1 = K(0);
    for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) l1 += wv[j] * wv[j];
    double loc1 = cta_sum((double)l1, sm.red);
    __shared__ double nn[1];
    cluster_sums(cl, sm, 0, &loc1, 1, nn);
    const double nrm = sqrt(nn[0]);
    if (threadIdx.x == 0) {
      hc[jcol + 1] = nrm;
      for (int i = 0; i < jcol; ++i) {           // previous Givens rotations
        const double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
        hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
        hc[i] = t;
      }
      const double a0 = hc[jcol], b0 = hc[jcol + 1];
      const double rr = hypot(a0, b0);
      const double c0g = rr > 0.0 ? a0 / rr : 1.0, s0g = rr > 0.0 ? b0 / rr : 0.0;
      hc[jcol] = rr;
      const double gj = g_jcol;
      const double gnext = -s0g * gj;
      // GMRES's own (2-norm) estimate; the per-cell test runs on the true residual.
      // Every CTA takes the same decision (its inputs are cluster-wide values).
      const bool est = fabs(gnext) <= 0.05 * D.rtol * D.gxn[ii];
      const bool stop = est || nrm == 0.0 || jcol + 1 >= m;
      cont_s = stop ? 0 : 1;
      if (rank == 0) {
        cs[jcol] = c0g;
        sn[jcol] = s0g;
        g[jcol + 1] = gnext;
        g[jcol] = c0g * gj;
        for (int i = 0; i <= jcol; ++i) H[i * kMaxRestart + jcol] = hc[i];
        D.gk[ii] = jcol + 1;
        D.gits[ii] += 1;
        if (est) D.gestconv[ii] = 1;
        if (stop) D.gactive[ii] = 0;
      }
    }
    const K inv = K(nrm > 0.0 ? 1.0 / nrm : 0.0);
    for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) wv[j] *= inv;
    cl.sync();
    // per-cell parts of the next direction pass (V_{j+1} complete after the barrier)
    if (FUSED_PARTS && cont_s)
      for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) cellpart_cell<K>(D, I, co + j, j, wv, 0);
    return;
  }

  if (MODE == G_UPDATE) {
    if (D.gdone[ii]) return;
    const int kk = D.gk[ii];
    if (threadIdx.x == 0) {
      for (int i = kk - 1; i >= 0; --i) {
        double t = g[i];
        for (int l = i + 1; l < kk; ++l) t -= H[i * kMaxRestart + l] * sm.y[l];
        sm.y[i] = t / H[i * kMaxRestart + i];
      }
    }
    __syncthreads();
    for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) {
      double t = x[j];
      for (int i = 0; i < kk; ++i) t += sm.y[i] * (double)Vi(i)[j];
      x[j] = t;
    }
    if (FUSED_PARTS) {
      cl.sync();
      // per-cell parts of the data pass at the updated iterate
      for (int64_t j = c0 + threadIdx.x; j < c0 + n; j += blockDim.x) cellpart_cell<double>(D, I, co + j, j, x, 1);
    }
    return;
  }
}

// ----------------------------------------------------------------------------- Newton
// Correction substep 1 (Eq. Tnp1; sigma_0/T^3: sum of Eq. dis-cor-marshak4/5),
// multiplied through by sig:  A T^4 + B T = R,
//   A = sig a/dt,  B = sig Cv/dt + eps^2 kap Cv/(c dt^2),  R = sig (rho^n/(c dt) - F*/dx) + B T^n,
// kap = 1 (sigma(x)) or K* = max(U*,0)^{3/4} (sigma_0/T^3).  Newton from
// T_hi = min((R/A)^{1/4}, R/B) decreases monotonically to the unique root
// (convex increasing left side); it stops when the iterate stops decreasing.
// Raw features of the learned Newton guess for each cell (after the prediction):
// log10 T^n, log10 rho*, log10 sigma_eff, log10 eps, log10 dt, log10 Cv.
__global__ void k_newton_feat(Dev D, int n_inst, const int64_t* __restrict__ cell_inst_start, int64_t ncell) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= ncell) return;
  const Inst I = D.inst[inst_of(cell_inst_start, n_inst, gid)];
  const double Tn = D.T[gid];
  const double rho = D.gx[gid];
  const double t3 = Tn * Tn * Tn;
  const double sig_eff = (I.kind == GRTE_SIGMA_CONST)
                            ? D.sig[gid]
                            : D.sig[gid] / fmax(I.p == 3.0 ? t3 : pow(Tn, I.p), 1e-300);
  auto lg = [](double x) { return (float)log10(fmin(fmax(x, 1e-300), 1e300)); };
  float* f = D.feat + 6 * gid;
  f[0] = lg(Tn);
  f[1] = lg(rho);
  f[2] = lg(sig_eff);
  f[3] = lg(I.eps);
  f[4] = lg(I.dt);
  f[5] = lg(I.Cv);
}

__global__ void k_newton(Dev D, int n_inst, const int64_t* __restrict__ cell_inst_start, int64_t ncell) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= ncell) return;
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (cell_inst_start[mid] <= gid) lo = mid; else hi = mid - 1;
  }
  const Inst I = D.inst[lo];
  const double rho = D.gx[gid];
  const double gam = D.cf.gam[gid];
  const double Un = D.U[gid];
  const double Us = (Un + gam * rho) / (1.0 + gam * I.a * I.c);
  D.Us[gid] = Us;
  D.rho_s[gid] = rho;
  const double sig = D.sig[gid];
  const double kap = (I.kind == GRTE_SIGMA_CONST) ? 1.0
                     : (I.p == 3.0 ? q_pow34(fmax(Us, 0.0)) : pow(fmax(Us, 0.0), 0.25 * I.p));
  const double A = sig * I.adt;
  const double B = sig * I.cvdt + kap * I.ekc;
  const double Tn = D.T[gid];
  // the correction's flux (sigma_0/T^3: with V* = (U*)^{3/4}; sigma(x): the prediction's F*)
  const double R = sig * (D.rho_n[gid] * I.rcdt - D.Fc[gid] * I.rdx) + B * Tn;
  double T;
  int its = 0;
  if (A == 0.0 && B == 0.0) {
    T = Tn;
  } else if (!(R > 0.0)) {
    T = 0.0;
    if (R <= 0.0) flag(D.status, lo, GRTE_ENEGATIVE);
  } else {
    double t = INFINITY;
    if (A > 0.0) t = sqrt(sqrt(R / A));
    if (B > 0.0) t = fmin(t, R / B);
    // the learned guess gl is used where it lies more than 10^0.05 - 1 (about 12%)
    // below the closed-form bound: there the bound starts far above the root (a front
    // cell).  Elsewhere the bound is within the network's few-percent error of the root
    // (the root lies below both) and is kept, so that noise does not cost the extra
    // guess step.
    const double gl = D.use_guess ? Tn * exp10((double)D.guess[gid]) : 0.0;
    const bool learned = D.use_guess && isfinite(gl) && gl > 0.0 && gl * kGuessGate < t;
    if (learned || D.start_prev) {
      // learned (or previous-T) start: one Newton step from any positive guess lands
      // at or above the root (convex left side).  The learned start is clamped to the
      // closed-form bound, so its residual is never larger than the plain start's; the
      // previous-T start is kept unclamped (the textbook start, for comparison).
      const double g = learned ? gl : Tn;
      if (isfinite(g) && g > 0.0) {
        const double g2 = g * g;
        const double t1 = g - (A * g2 * g2 + B * g - R) / (4.0 * A * g2 * g + B);
        if (isfinite(t1) && t1 > 0.0) t = learned ? fmin(t, t1) : t1;
        ++its;
      }
    }
    for (its = its + 1; its <= D.newton_maxit; ++its) {
      const double t2 = t * t;
      const double f = A * t2 * t2 + B * t - R;
      const double fp = 4.0 * A * t2 * t + B;
      const double tn = t - q_div(f, fp);
      if (!(tn < t)) break;
      t = tn;
    }
    if (its > D.newton_maxit) flag(D.status, lo, GRTE_ENONCONV);
    T = t;
  }
  if (!isfinite(T) || !isfinite(R)) flag(D.status, lo, GRTE_ENAN);
  D.newton_its[gid] = its;
  D.T[gid] = T;            // T^{n+1}
  if (D.log_samples) D.ytrue[gid] = (T > 0.0 && Tn > 0.0) ? (float)log10(T / Tn) : 0.0f;
}

// ----------------------------------------------------------------------------- correction
// Correction substep 2 (Eq. dis-cor1/2 with Eq. dis-cor4; Eq. dis-cor-marshak1/2
// with Eq. 9171 and K -> (T^{n+1})^3) and projection (Eq. dis-proj), one line per
// CTA.  With U = (T^{n+1})^4 and O eliminated by the node equation,
//   O_i = o'_i - d_i eps v (E_J,i - E_J,i-1)/dx,  o'_i = d_i [eps^2 O^n_i/(c dt) - a c v (U_i - U_{i-1})/dx],
// the cell equation divided by eps reads (A + v^2 Gint + v Gbdry) E_J = rhs with the
// coefficients of k_cell_coef at T^{n+1}; the walls use O_{J,0} = 2/eps (b_L - E_0) - O_1
// and O_{J,N} = 2/eps (E_{N-1} - b_R) - O_{N-1}.  Then E^{n+1} = a c U + eps E_J,
// O^{n+1} = O_J (in place: each CTA owns its line).
// Per-angle parts in R; the U parts (Q1, gU, Q2) come in double from
// k_cellpart_corr, and the two inflow wall cells are formed in double.  NT and XS as
// in k_pred_line.  With dry != 0 the state is left unchanged (the solve runs, the
// projection is not stored): a side-effect-free pass for timing.
template <typename R, int NT, bool XS>
__global__ void __launch_bounds__(NT, 1024 / NT) k_corr_line(Dev D, int dry) {
  extern __shared__ __align__(16) unsigned char dsm[];
  const Line L = D.lines[blockIdx.x];
  const Inst I = D.inst[L.inst];
  const int64_t N = I.N;
  const int k = L.k;
  const double v = D.v[I.ang_off + k];
  const double eps = I.eps, ac = I.a * I.c;
  const bool inflow = I.bc == GRTE_BC_INFLOW;
  const double bL = inflow ? D.bL[I.ang_off + k] : 0.0, bR = inflow ? D.bR[I.ang_off + k] : 0.0;
  const int64_t co = I.cell_off, eo = I.elem_off + (int64_t)k * N, oo = I.nelem_off + (int64_t)k * (N + 1);
  R* Eh = (R*)D.Eh + eo;
  R* O = (R*)D.O + oo;
  const double* T = D.T + co;   // T^{n+1}
  const double* Un = D.U + co;  // U^n
  const XAcc<R, XS> xb = line_x<R, XS>(dsm, (R*)D.xb + eo);
  R* on = (R*)D.onode + oo;
  const double *dlx = D.cf.dlx + co, *kcd = D.cf.kcd + co, *kdx = D.cf.kdx + co, *Q1 = D.Q1 + co,
               *Q2 = D.Q2 + co, *gU = D.gU + co;
  const double two_eps = I.two_eps, inv_eps = I.inv_eps;
  const R vr = R(v), v2r = R(v * v);
  constexpr bool F32 = sizeof(R) == 4;
  const R* odr = pick<R>(D.cf.od, D.fc.od) + co;
  auto U1 = [&](int64_t j) { const double t = T[j]; const double t2 = t * t; return t2 * t2; };
  for (int64_t i = threadIdx.x; i <= N; i += NT)
    on[i] = (i >= 1 && i <= N - 1) ? odr[i] * O[i] : R(0);   // eps^2 d O^n/(c dt) part of o'
  __syncthreads();
  for (int64_t j = threadIdx.x; j < N; j += NT) {
    const bool wall = inflow && (j == 0 || j == N - 1);
    if (!wall) {
      if constexpr (F32) {
        const int64_t g = co + j;
        const R ke = (R)D.fc.kdxe[g];
        xb[j] = D.fc.Q1[g] + D.fc.kcde[g] * Eh[j] - ke * vr * (on[j + 1] - on[j]) + ke * v2r * D.fc.Q2[g];
      } else {
        xb[j] = R(Q1[j]) + R(kcd[j] * inv_eps) * Eh[j] - R(kdx[j] * v * inv_eps) * (on[j + 1] - on[j]) +
                R(kdx[j] * v * v * inv_eps) * R(Q2[j]);
      }
    } else {
      double Dj;
      if (j == 0) Dj = 2.0 * ((double)on[1] - v * gU[1]) - two_eps * (bL - ac * U1(0));
      else Dj = two_eps * (ac * U1(N - 1) - bR) - 2.0 * ((double)on[N - 1] - v * gU[N - 1]);
      xb[j] = R((kcd[j] * ((double)Eh[j] + ac * (Un[j] - U1(j))) - kdx[j] * v * Dj) * inv_eps);
    }
  }
  __syncthreads();
  LineCoef<R> cfl{pick<R>(D.cf.A, D.fc.A) + co, pick<R>(D.cf.gl, D.fc.gl) + co, pick<R>(D.cf.gu, D.fc.gu) + co,
                  pick<R>(D.cf.gb, D.fc.gb) + co, vr, v2r, N};
  tri_solve<true>(cfl, N, xb, (R*)D.F + L.f_off, (R*)D.Rd + L.red_off, line_red<R, XS>(dsm, N));
  if (dry) return;
  // projection: O^{n+1} = O_J, Eh^{n+1} = eps E_J (E^{n+1} = a c U^{n+1} + Eh^{n+1})
  const R epsr = R(eps);
  for (int64_t i = threadIdx.x; i <= N; i += NT) {
    auto Oint = [&](int64_t n) -> R {
      if constexpr (F32) return on[n] - vr * D.fc.gU[co + n] - D.fc.dlxe[co + n] * vr * (xb[n] - xb[n - 1]);
      else return on[n] - vr * R(gU[n]) - R(dlx[n] * eps) * vr * (xb[n] - xb[n - 1]);
    };
    R Oi;
    if (i >= 1 && i <= N - 1) Oi = Oint(i);
    else if (!inflow) Oi = R(0);
    else if (i == 0) Oi = R(two_eps * (bL - ac * U1(0)) - 2.0 * (double)xb[0] - (double)Oint(1));
    else Oi = R(two_eps * (ac * U1(N - 1) - bR) + 2.0 * (double)xb[N - 1] - (double)Oint(N - 1));
    O[i] = Oi;
  }
  for (int64_t j = threadIdx.x; j < N; j += NT) Eh[j] = epsr * xb[j];
}

// Energy sums of one instance per CTA (FP64, fixed reduction order):
//   acc[0] = sum_j dx (rho_j/c + Cv T_j)                     (energy now)
//   acc[1] += dt sum_j F*_j                                  (wall flux of the prediction)
//   acc[2] += dt sum_j eps^2/(c sig_j dt + eps^2) (F*_j - F^{n+1}_j)   (Eq. semiconservative defect)
template <typename R>
__global__ void __launch_bounds__(kTriThreads) k_energy(Dev D, int accumulate) {
  __shared__ double red[32];
  const int ii = blockIdx.x;
  const Inst I = D.inst[ii];
  const int64_t N = I.N, co = I.cell_off;
  double e = 0.0, f = 0.0, dft = 0.0;
  const double eps2 = I.eps * I.eps, cdt = I.c * I.dt;
  for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
    double rho = I.a * I.c * D.U[co + j], Fn = 0.0;
    for (int k = 0; k < I.M; ++k) {
      const double w = D.w[I.ang_off + k], v = D.v[I.ang_off + k];
      rho += w * (double)((const R*)D.Eh)[I.elem_off + (int64_t)k * N + j];
      const R* O = (const R*)D.O + I.nelem_off + (int64_t)k * (N + 1);
      Fn += w * v * ((double)O[j + 1] - (double)O[j]);
    }
    e += I.dx * (rho / I.c + I.Cv * D.T[co + j]);
    const double Fs = D.Fs[co + j];
    f += Fs;
    dft += eps2 / (cdt * D.sig[co + j] + eps2) * (Fs - Fn);
  }
  e = cta_sum(e, red);
  f = cta_sum(f, red);
  dft = cta_sum(dft, red);
  if (threadIdx.x == 0) {
    D.energy[3 * ii + 0] = e;
    if (accumulate) {
      D.energy[3 * ii + 1] += I.dt * f;
      D.energy[3 * ii + 2] += I.dt * dft;
    }
  }
}

// U^{n+1} = (T^{n+1})^4 (Eq. dis-proj1)
__global__ void k_project_U(Dev D, int64_t ncell) {
  int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid >= ncell) return;
  const double t = D.T[gid];
  D.U[gid] = (t * t) * (t * t);
}

}  // namespace grte

#include "fused1d.cuh"

// =============================================================================== host
using namespace grte;

struct grte_ctx {
  int n_inst = 0;
  std::vector<Inst> inst;
  std::vector<Line> lines;
  std::vector<double> hv, hw;
  int64_t ncell = 0, nelem = 0, nnelem = 0, nred = 0, npred = 0, nlines = 0;
  grte_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool state_set = false;
  std::vector<char> inst_set;
  Dev D{};
  int64_t* d_cell_start = nullptr;
  Inst* d_inst = nullptr;
  Line* d_lines = nullptr;
  std::vector<void*> allocs;
  std::string err;
  grte_stats_t stats{};
  int* h_flags = nullptr;   // pinned: gdone per instance
  // per-kernel event timing
  uint32_t prof_mask = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  int64_t launches = 0;
  grte_mlp_t mlp = nullptr;   // learned Newton guess (not owned)
  // line solves: threads per CTA (0 until chosen), unknowns in shared memory or not
  int nt = 0;
  bool xs = false;
  int64_t maxN = 0;
  // Krylov kernels: largest preconditioner slice, slice unknowns in shared memory or not
  int64_t max_slice = 0;
  bool gxs = false;
  // captured step (after the first step): graph, executable, device counters
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int* d_cycles = nullptr;          // restart cycles of the current step
  long long* d_acc = nullptr;       // Krylov iterations, cycles, iterations run, condition kernels run
  int64_t graph_fixed_launches = 0;
  double tune_ms[3] = {-1.0, -1.0, -1.0};
  // fused prediction solve: instances grouped by cluster size 1, 2, 4, 8, 16
  bool fused = false;
  int* d_finst = nullptr;
  int fcnt[5] = {0, 0, 0, 0, 0}, foff[5] = {0, 0, 0, 0, 0};
  cudaEvent_t ev_state = nullptr;   // grte_get_T_device: the caller's stream waits on it
};

// The captured step depends on values passed by value to its kernels (the device
// description, the Newton start, the learned guess): setters that change them drop it.
static void drop_step_graph(grte_t h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->graph_exec = nullptr;
  h->graph = nullptr;
}

static cudaEvent_t pool_event(grte_t h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// Launch wrapper: counts launches and, for profiled kernel ids, brackets the launch
// with an event pair on the handle's stream.
#define LAUNCH(kid, ...)                                                         \
  do {                                                                           \
    const bool prof_ = (h->prof_mask >> (kid)) & 1u;                             \
    cudaEvent_t e0_ = nullptr, e1_ = nullptr;                                    \
    if (prof_) { e0_ = pool_event(h); e1_ = pool_event(h); cudaEventRecord(e0_, st); } \
    __VA_ARGS__;                                                                 \
    if (prof_) { cudaEventRecord(e1_, st); h->prof_ev.push_back({(kid), {e0_, e1_}}); } \
    ++h->launches;                                                               \
  } while (0)

static grte_status fail(grte_t h, grte_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}
#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return fail(h, GRTE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static int g_fail_alloc_after = -1;   // < 0: off (grte_test_fail_alloc_after)

template <typename T>
static cudaError_t dalloc(grte_t h, T** p, int64_t n) {
  void* q = nullptr;
  // test hook (grte_test_fail_alloc_after): the allocation after the given count fails
  if (g_fail_alloc_after >= 0 && g_fail_alloc_after-- == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  cudaError_t e = cudaMalloc(&q, sizeof(T) * (size_t)std::max<int64_t>(n, 1));
  if (e == cudaSuccess) {
    h->allocs.push_back(q);
    cudaMemset(q, 0, sizeof(T) * (size_t)std::max<int64_t>(n, 1));
  }
  *p = (T*)q;
  return e;
}

// ----------------------------------------------------------------------------- line launches
// Dynamic shared memory of a line CTA: the padded unknowns of the longest line (when
// they stay in shared memory) and the reduced system.
static int64_t line_smem(const grte_ctx* h, int nt, bool factor) {
  const int es = h->opt.precision == GRTE_MIXED ? 4 : 8;
  return (h->xs ? (tri_xs_len(h->maxN) * es + 15) / 16 * 16 : 0) + tri_smem_bytes(nt, factor, es);
}

static int g_smem_optin = 0;   // largest dynamic shared memory a line kernel may request
static int g_gmres_dyn = 0;    // largest dynamic shared memory a Krylov kernel may request

static bool line_fits(const grte_ctx* h, int nt) {
  const int es = h->opt.precision == GRTE_MIXED ? 4 : 8;
  const int64_t need = (tri_xs_len(h->maxN) * es + 15) / 16 * 16 + tri_smem_bytes(nt, true, es);
  return need <= g_smem_optin;
}

template <class K>
static cudaError_t smem_attr(K k, int bytes) {
  return cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename R, int NT, bool XS>
static cudaError_t line_attrs_one(int bytes) {
  cudaError_t e = smem_attr(k_pred_line<PRED_FULL_FACTOR, R, NT, XS>, bytes);
  if (e == cudaSuccess) e = smem_attr(k_pred_line<PRED_FULL, R, NT, XS>, bytes);
  if (e == cudaSuccess) e = smem_attr(k_pred_line<PRED_HOM, R, NT, XS>, bytes);
  if (e == cudaSuccess) e = smem_attr(k_corr_line<R, NT, XS>, bytes);
  return e;
}

// Allow every line kernel the device's opt-in shared memory (less a margin for the
// kernels' static shared memory); once per device.
static cudaError_t line_kernel_attrs() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const int bytes = optin - 256;
  e = line_attrs_one<double, 256, false>(bytes);
  if (e == cudaSuccess) e = line_attrs_one<double, 256, true>(bytes);
  if (e == cudaSuccess) e = line_attrs_one<double, 512, true>(bytes);
  if (e == cudaSuccess) e = line_attrs_one<double, 1024, true>(bytes);
  if (e == cudaSuccess) e = line_attrs_one<float, 256, false>(bytes);
  if (e == cudaSuccess) e = line_attrs_one<float, 256, true>(bytes);
  if (e == cudaSuccess) e = line_attrs_one<float, 512, true>(bytes);
  if (e == cudaSuccess) e = line_attrs_one<float, 1024, true>(bytes);
  if (e != cudaSuccess) return e;
  g_smem_optin = bytes;
  // Krylov kernels: the opt-in size less their static shared memory
  int gdyn = bytes;
  auto gm = [&](const void* f) {
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
    if (e == cudaSuccess) gdyn = std::min(gdyn, bytes - (int)fa.sharedSizeBytes);
  };
  const void* gk[] = {(const void*)k_gmres<G_RESTART_FIRST, double, true>, (const void*)k_gmres<G_RESTART, double, true>,
                      (const void*)k_gmres<G_ARNOLDI, double, true>, (const void*)k_gmres<G_UPDATE, double, true>,
                      (const void*)k_gmres<G_RESTART_FIRST, float, true>, (const void*)k_gmres<G_RESTART, float, true>,
                      (const void*)k_gmres<G_ARNOLDI, float, true>, (const void*)k_gmres<G_UPDATE, float, true>};
  for (const void* f : gk) gm(f);
  for (const void* f : gk)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, gdyn);
  if (e != cudaSuccess) return e;
  g_gmres_dyn = gdyn;
  if (dev >= 0 && dev < 64) done[dev] = true;
  return cudaSuccess;
}

static int64_t gmres_dyn_smem(const grte_ctx* h) {
  return h->gxs ? (tri_xs_len(h->max_slice) * 8 + 15) / 16 * 16 : 0;
}
template <int MODE, typename R>
static void gmres_launch(grte_ctx* h, int jcol) {
  const unsigned grid = (unsigned)(h->n_inst * kCL);
  if (h->gxs) k_gmres<MODE, R, true><<<grid, kTriThreads, (size_t)gmres_dyn_smem(h), h->stream>>>(h->D, jcol);
  else k_gmres<MODE, R, false><<<grid, kTriThreads, 0, h->stream>>>(h->D, jcol);
}

template <int MODE, typename R, int NT, bool XS>
static void pred_launch(grte_ctx* h, const void* x) {
  k_pred_line<MODE, R, NT, XS><<<(unsigned)h->nlines, NT, (size_t)line_smem(h, NT, MODE == PRED_FULL_FACTOR),
                                 h->stream>>>(h->D, x);
}
template <int MODE, typename R>
static void pred_pass(grte_ctx* h, const void* x) {
  if (!h->xs) return pred_launch<MODE, R, 256, false>(h, x);
  switch (h->nt) {
    case 1024: pred_launch<MODE, R, 1024, true>(h, x); break;
    case 512: pred_launch<MODE, R, 512, true>(h, x); break;
    default: pred_launch<MODE, R, 256, true>(h, x); break;
  }
}
template <typename R, int NT, bool XS>
static void corr_launch(grte_ctx* h, int dry) {
  k_corr_line<R, NT, XS><<<(unsigned)h->nlines, NT, (size_t)line_smem(h, NT, true), h->stream>>>(h->D, dry);
}
template <typename R>
static void corr_pass(grte_ctx* h, int dry) {
  if (!h->xs) return corr_launch<R, 256, false>(h, dry);
  switch (h->nt) {
    case 1024: corr_launch<R, 1024, true>(h, dry); break;
    case 512: corr_launch<R, 512, true>(h, dry); break;
    default: corr_launch<R, 256, true>(h, dry); break;
  }
}

// ----------------------------------------------------------------------------- fused launches
// Cluster size of an instance in the fused prediction solve: one 512-cell slice per CTA,
// rounded up to a power of two (class index 0..4 for 1, 2, 4, 8, 16 CTAs).
static int fused_class(int64_t nx) {
  const int64_t q = (nx + kFS - 1) / kFS;
  int c = 0;
  while ((1 << c) < q) ++c;
  return c;
}

static bool fused_fits(const Inst& I) { return I.N >= 64 && I.N <= (int64_t)kFQ * kFS && I.M <= 32; }

// Kernel attributes of the fused solve (once per device): its shared memory and the
// non-portable cluster size 16.
// Dynamic shared memory of the fused kernel: the struct and the slice's Krylov basis
// V_0..V_m (m = restart length).
static size_t fused_smem(int m) { return sizeof(FSmem) + (size_t)(m + 1) * kFS * sizeof(double); }
static int g_fused_optin = 0;   // the device's opt-in shared memory per block

static cudaError_t fused_attrs() {
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_pred_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)k_pred_fused, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) g_fused_optin = optin;
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

static void fused_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at, int Qc, int nclusters, int m,
                         cudaStream_t st) {
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3((unsigned)(nclusters * Qc), 1, 1);
  cfg.blockDim = dim3(kFT, 1, 1);
  cfg.dynamicSmemBytes = fused_smem(m);
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)Qc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
}

// 1 if a cluster of Qc CTAs of the fused kernel can be resident on this device.
static cudaError_t fused_schedulable(int Qc, int m, bool* ok) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  fused_config(cfg, at, Qc, 1, m, nullptr);
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&n, (const void*)k_pred_fused, &cfg);
  *ok = e == cudaSuccess && n >= 1;
  return e;
}

static cudaError_t fused_launch(grte_ctx* h, int c) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  fused_config(cfg, at, 1 << c, h->fcnt[c], h->D.m, h->stream);
  return cudaLaunchKernelEx(&cfg, k_pred_fused, h->D, (const int*)(h->d_finst + h->foff[c]));
}

// Krylov iterations and restart cycles of the fused solve, accumulated over graph replays.
__global__ void k_fused_stats(const int* __restrict__ gits, const int* __restrict__ gcycles, int n, long long* acc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    long long a = 0, b = 0;
    for (int i = 0; i < n; ++i) {
      a += gits[i];
      b += gcycles[i];
    }
    acc[0] += a;
    acc[1] += b;
  }
}

// Autotuner of the line solves: times, for 256, 512 and 1024 threads per line (those
// whose shared memory fits), one factor pass, four solve passes and one correction
// pass (dry: the state is not touched) on this handle's own instances, twice, and
// keeps the thread count with the smallest second time.  Needs the per-cell parts of
// the current step (k_cell_coef, k_cellpart_pred) on the stream; synchronises.
template <typename R>
static cudaError_t autotune_lines(grte_ctx* h) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) { cudaEventDestroy(e0); return e; }
  int best = 256;
  float best_ms = 3.0e38f;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    const int nt = 256 << i;
    h->tune_ms[i] = -1.0;
    if (!line_fits(h, nt)) continue;
    h->nt = nt;
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, h->stream);
      pred_pass<PRED_FULL_FACTOR, R>(h, h->D.gx);
      for (int q = 0; q < 4; ++q) pred_pass<PRED_FULL, R>(h, h->D.gx);
      corr_pass<R>(h, 1);
      cudaEventRecord(e1, h->stream);
      e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e != cudaSuccess) break;
    h->tune_ms[i] = ms;
    if (ms < best_ms) { best_ms = ms; best = nt; }
  }
  h->nt = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

// Gauss-Legendre nodes on [-1,1] by Newton on P_n (three-term recurrence); the
// positive half, weights normalised to sum 1 (= int_0^1 dv).
static void gauss_legendre_half(int n, std::vector<double>& v, std::vector<double>& w) {
  const int M = n / 2;
  v.resize(M);
  w.resize(M);
  for (int i = 0; i < M; ++i) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
    }
    v[M - 1 - i] = x;                       // increasing order
    w[M - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

extern "C" {

void grte_default_options(grte_options* o) {
  if (!o) return;
  o->precision = GRTE_FP64;
  o->krylov_rtol = 1e-13;
  o->krylov_restart = 10;
  o->krylov_maxcycles = 30;
  o->newton_maxit = 60;
  o->energy_every = 0;
  o->stream = nullptr;
  o->line_threads = 0;
  o->use_graph = 1;
  o->prec2d = 0;
  o->solver1d = GRTE_SOLVER_AUTO;
}

const char* grte_last_error(grte_t h) { return h ? h->err.c_str() : "null handle"; }

void grte_destroy(grte_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_step_graph(h);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_flags) cudaFreeHost(h->h_flags);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->ev_state) cudaEventDestroy(h->ev_state);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

void grte_test_fail_alloc_after(int n) { g_fail_alloc_after = n < 0 ? -1 : n; }

grte_status grte_create_1d(int n_inst, const grte_instance1d* in, const grte_options* opt, grte_t* out) {
  if (!out) return GRTE_EINVAL;
  *out = nullptr;
  if (n_inst <= 0 || !in) return GRTE_EINVAL;
  grte_t h = new (std::nothrow) grte_ctx();
  if (!h) return GRTE_ENOMEM;
  grte_default_options(&h->opt);
  if (opt) h->opt = *opt;
  auto bad = [&](const std::string& m) { grte_status s = fail(h, GRTE_EINVAL, m); *out = h; return s; };
  auto nomem = [&](const std::string& m) { grte_status s = fail(h, GRTE_ENOMEM, m); *out = h; return s; };
  if (h->opt.precision != GRTE_FP64 && h->opt.precision != GRTE_MIXED) return bad("precision must be GRTE_FP64 or GRTE_MIXED");
  if (h->opt.krylov_restart < 1 || h->opt.krylov_restart > kMaxRestart) return bad("krylov_restart out of range [1,16]");
  if (h->opt.krylov_maxcycles < 1 || h->opt.newton_maxit < 1 || !(h->opt.krylov_rtol > 0)) return bad("bad solver options");
  h->n_inst = n_inst;
  int64_t coff = 0, eoff = 0, noff = 0, roff = 0, poff = 0, foff = 0;
  int aoff = 0, loff = 0;
  if (h->opt.line_threads != 0 && h->opt.line_threads != 256 && h->opt.line_threads != 512 &&
      h->opt.line_threads != 1024)
    return bad("line_threads must be 0, 256, 512 or 1024");
  for (int i = 0; i < n_inst; ++i) {
    const grte_instance1d& p = in[i];
    if (p.nx < 2 || p.nx > (1 << 24)) return bad("nx must be in [2, 2^24]");
    if (p.n_angle < 1 || p.n_angle > 4096) return bad("n_angle must be in [1, 4096]");
    if (!p.sigma) return bad("sigma is NULL");
    if (p.sigma_kind != GRTE_SIGMA_CONST && p.sigma_kind != GRTE_SIGMA_T3 && p.sigma_kind != GRTE_SIGMA_POW)
      return bad("bad sigma_kind");
    if (p.sigma_kind == GRTE_SIGMA_POW && !(p.sigma_p >= 0.0 && p.sigma_p <= 3.0))
      return bad("sigma_p must be in [0, 3]");
    if (p.bc != GRTE_BC_INFLOW && p.bc != GRTE_BC_REFLECT) return bad("bad bc");
    if (!(p.x1 > p.x0) || !(p.dt > 0) || !(p.a > 0) || !(p.c > 0) || !(p.Cv > 0) || !(p.eps > 0))
      return bad("x1 > x0, dt, a, c, Cv, eps must be positive");
    if ((p.v == nullptr) != (p.w == nullptr)) return bad("v and w must both be given or both NULL");
    std::vector<double> v, w;
    if (p.v) {
      v.assign(p.v, p.v + p.n_angle);
      w.assign(p.w, p.w + p.n_angle);
    } else {
      gauss_legendre_half(2 * p.n_angle, v, w);
    }
    double sw = 0.0;
    for (int k = 0; k < p.n_angle; ++k) {
      if (!(v[k] > 0.0 && v[k] <= 1.0) || !(w[k] > 0.0)) return bad("angles must lie in (0,1], weights > 0");
      sw += w[k];
    }
    for (int k = 0; k < p.n_angle; ++k) w[k] /= sw;   // sum_k w_k = 1 exactly as possible
    for (int64_t j = 0; j < p.nx; ++j)
      if (!(p.sigma[j] >= 0.0) || !std::isfinite(p.sigma[j])) return bad("sigma must be finite and >= 0");
    Inst I{};
    I.N = (int)p.nx;
    I.M = p.n_angle;
    I.kind = p.sigma_kind == GRTE_SIGMA_CONST ? GRTE_SIGMA_CONST : GRTE_SIGMA_T3;
    I.p = p.sigma_kind == GRTE_SIGMA_POW ? p.sigma_p : 3.0;
    I.bc = p.bc;
    I.eps = p.eps;
    I.dt = p.dt;
    I.dx = (p.x1 - p.x0) / (double)p.nx;
    I.a = p.a;
    I.c = p.c;
    I.Cv = p.Cv;
    double wv = 0, wv2 = 0;
    for (int k = 0; k < p.n_angle; ++k) {
      wv += w[k] * v[k];
      wv2 += w[k] * v[k] * v[k];
    }
    I.wv = wv;
    I.wv2 = wv2;
    I.two_eps = 2.0 / p.eps;
    {
      double fl = 0.0, fr = 0.0;
      for (int k = 0; k < p.n_angle; ++k) {
        if (p.bc == GRTE_BC_INFLOW && p.bL) fl += w[k] * v[k] * p.bL[k];
        if (p.bc == GRTE_BC_INFLOW && p.bR) fr += w[k] * v[k] * p.bR[k];
      }
      I.bLflux = fl;
      I.bRflux = fr;
    }
    I.inv_eps = 1.0 / p.eps;
    inst_derive(I);
    I.cell_off = coff;
    I.elem_off = eoff;
    I.nelem_off = noff;
    I.red_off = poff;
    I.ang_off = aoff;
    I.line_off = loff;
    for (int k = 0; k < p.n_angle; ++k) {
      h->lines.push_back(Line{i, k, roff, foff});
      roff += tri_red_size(p.nx, kTriMaxNT);
      foff += 5 * (p.nx + std::min<int64_t>(p.nx / 2, kTriMaxNT));   // >= tri_fac_size(nx, nt), nt <= 1024
    }
    h->maxN = std::max<int64_t>(h->maxN, p.nx);
    {
      const int64_t nact = std::min<int64_t>(p.nx / 2, kCL);
      h->max_slice = std::max<int64_t>(h->max_slice, p.nx / nact + 1);
    }
    poff += prec_red_size(p.nx);
    coff += p.nx;
    eoff += p.nx * p.n_angle;
    noff += (p.nx + 1) * p.n_angle;
    aoff += p.n_angle;
    loff += p.n_angle;
    h->inst.push_back(I);
    h->hv.insert(h->hv.end(), v.begin(), v.end());
    h->hw.insert(h->hw.end(), w.begin(), w.end());
  }
  h->ncell = coff;
  h->nlines = (int64_t)h->lines.size();
  h->nelem = eoff;
  h->nnelem = noff;
  h->nred = roff;
  h->npred = poff;
  *out = h;
  if (h->opt.stream) {
    h->stream = (cudaStream_t)h->opt.stream;
  } else {
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  CK(cudaEventCreateWithFlags(&h->ev_state, cudaEventDisableTiming));
  Dev& D = h->D;
  const int m = h->opt.krylov_restart;
  D.m = m;
  D.maxcycles = h->opt.krylov_maxcycles;
  // binary32 line solves and Krylov vectors leave noise in the residual of cells far
  // below the maximum: the mixed mode floors the tolerance at 1e-9, measures cells
  // below 1e-6 of the maximum against that floor, and accepts a second restart below
  // 1e-4 (FP64: a restart that stalls below 1e-9)
  const bool mixed = h->opt.precision == GRTE_MIXED;
  D.rtol = mixed ? std::max(h->opt.krylov_rtol, 1e-9) : h->opt.krylov_rtol;
  D.stall = mixed ? 1e-4 : 1e-9;
  D.wfloor = mixed ? 1e-6 : 1e-13;
  D.mixed = mixed ? 1 : 0;
  const int64_t es = mixed ? 4 : 8;   // bytes per bulk element
  D.newton_maxit = h->opt.newton_maxit;
  const int64_t nc = h->ncell, ne = h->nelem, nn = h->nnelem, na = aoff;
#define AL(ptr, n) do { if (dalloc(h, &(ptr), (n)) != cudaSuccess) return nomem("cudaMalloc failed for " #ptr); } while (0)
  AL(h->d_inst, n_inst);
  AL(h->d_lines, (int64_t)h->lines.size());
  AL(h->d_cell_start, n_inst);
  AL(D.v, na); AL(D.w, na); AL(D.bL, na); AL(D.bR, na);
  { char* p_; if (dalloc(h, &p_, es * ne) != cudaSuccess) return nomem("cudaMalloc Eh"); D.Eh = p_; }
  { char* p_; if (dalloc(h, &p_, es * nn) != cudaSuccess) return nomem("cudaMalloc O"); D.O = p_; }
  AL(D.T, nc); AL(D.U, nc); AL(D.sig, nc);
  AL(D.P1, nc); AL(D.P2, nc); AL(D.P3, nc); AL(D.Frho, nc); AL(D.gU, nc); AL(D.Q1, nc); AL(D.Q2, nc);
  AL(D.gwork, nc);
  AL(D.Swall, 2 * na);
  AL(D.rho_n, nc); AL(D.rho_s, nc); AL(D.Fs, nc); AL(D.Us, nc); AL(D.newton_its, nc); AL(D.Fc, nc);
  AL(D.cf.kc, nc); AL(D.cf.s, nc); AL(D.cf.alpha, nc); AL(D.cf.A, nc); AL(D.cf.gam, nc);
  AL(D.cf.gl, nc); AL(D.cf.gu, nc); AL(D.cf.gb, nc); AL(D.cf.dl, nc);
  AL(D.cf.od, nc); AL(D.cf.dlx, nc); AL(D.cf.kcd, nc); AL(D.cf.kdx, nc); AL(D.cf.sac, nc);
  AL(D.cf.ralpha, nc); AL(D.cf.ratio, nc); AL(D.cf.fR, nc); AL(D.cf.fL, nc); AL(D.cf.gbx, nc);
  AL(D.cf.dsx, nc); AL(D.cf.ods, nc);
  if (mixed) {
    CellF& f = D.fc;
    AL(f.A, nc); AL(f.gl, nc); AL(f.gu, nc); AL(f.gb, nc); AL(f.od, nc); AL(f.dlx, nc); AL(f.kcd, nc);
    AL(f.kdx, nc); AL(f.ratio, nc); AL(f.ralpha, nc); AL(f.alpha, nc); AL(f.kcde, nc); AL(f.kdxe, nc);
    AL(f.dlxe, nc); AL(f.P1, nc); AL(f.P2, nc); AL(f.P3, nc); AL(f.Frho, nc); AL(f.Q1, nc); AL(f.Q2, nc);
    AL(f.gU, nc); AL(f.fR, nc); AL(f.fL, nc); AL(f.gbx, nc); AL(f.dsx, nc); AL(f.ods, nc);
    AL(D.cf.zl, nc); AL(D.cf.zc, nc); AL(D.cf.zr, nc);
  }
  {
    char* p_;
    if (dalloc(h, &p_, es * ne) != cudaSuccess) return nomem("cudaMalloc xb"); D.xb = p_;
    if (dalloc(h, &p_, es * ne) != cudaSuccess) return nomem("cudaMalloc S"); D.S = p_;
    if (dalloc(h, &p_, es * ne) != cudaSuccess) return nomem("cudaMalloc S2"); D.S2 = p_;
    if (dalloc(h, &p_, es * foff) != cudaSuccess) return nomem("cudaMalloc F"); D.F = p_;
    if (dalloc(h, &p_, es * h->nred) != cudaSuccess) return nomem("cudaMalloc Rd"); D.Rd = p_;
    if (dalloc(h, &p_, es * nn) != cudaSuccess) return nomem("cudaMalloc onode"); D.onode = p_;
  }
  AL(D.pF, 5 * (nc + (int64_t)n_inst * kCL * kTriThreads)); AL(D.pRd, h->npred); AL(D.pG, nc); AL(D.pH, nc); AL(D.gw, nc);
  AL(D.pInv, (int64_t)n_inst * kCL * 2 * (2 * kCL));
  // x, z contiguous so that the GMRES kernel can recover the total cell count
  double* xz = nullptr;
  AL(xz, 2 * nc);
  D.gx = xz;
  D.gz = xz + nc;
  AL(D.gV, (int64_t)(m + 1) * nc);
  AL(D.gH, (int64_t)n_inst * (kMaxRestart + 1) * kMaxRestart);
  AL(D.gg, (int64_t)n_inst * (kMaxRestart + 1));
  AL(D.gcs, (int64_t)n_inst * kMaxRestart);
  AL(D.gsn, (int64_t)n_inst * kMaxRestart);
  AL(D.gbeta, n_inst);
  AL(D.gxn, n_inst);
  AL(D.gactive, n_inst); AL(D.gk, n_inst); AL(D.gdone, n_inst); AL(D.gits, n_inst); AL(D.gcycles, n_inst);
  AL(D.gestconv, n_inst);
  AL(D.status, n_inst);
  AL(D.energy, 3 * (int64_t)n_inst);
  AL(h->d_cycles, 1);
  AL(h->d_acc, 4);
#undef AL
  D.inst = h->d_inst;
  D.lines = h->d_lines;
  std::vector<int64_t> cstart(n_inst);
  std::vector<double> hbL(na, 0.0), hbR(na, 0.0), hsig(nc);
  for (int i = 0; i < n_inst; ++i) {
    const Inst& I = h->inst[i];
    cstart[i] = I.cell_off;
    for (int k = 0; k < I.M; ++k) {
      hbL[I.ang_off + k] = in[i].bL ? in[i].bL[k] : 0.0;
      hbR[I.ang_off + k] = in[i].bR ? in[i].bR[k] : 0.0;
    }
    std::memcpy(hsig.data() + I.cell_off, in[i].sigma, sizeof(double) * I.N);
  }
  CK(cudaMemcpy(h->d_inst, h->inst.data(), sizeof(Inst) * n_inst, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_lines, h->lines.data(), sizeof(Line) * h->lines.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_cell_start, cstart.data(), sizeof(int64_t) * n_inst, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(D.v, h->hv.data(), sizeof(double) * na, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(D.w, h->hw.data(), sizeof(double) * na, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(D.bL, hbL.data(), sizeof(double) * na, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(D.bR, hbR.data(), sizeof(double) * na, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(D.sig, hsig.data(), sizeof(double) * nc, cudaMemcpyHostToDevice));
  CK(cudaMallocHost(&h->h_flags, sizeof(int) * n_inst));
  h->inst_set.assign(n_inst, 0);
  CK(line_kernel_attrs());
  // line solves: unknowns in shared memory when the largest line fits at 256 threads
  h->xs = line_fits(h, 256);
  h->gxs = (tri_xs_len(h->max_slice) * 8 + 15) / 16 * 16 <= g_gmres_dyn;
  if (h->opt.line_threads != 0) h->nt = (h->xs && line_fits(h, h->opt.line_threads)) ? h->opt.line_threads : 256;
  else if (!h->xs) h->nt = 256;   // nothing to tune: the global-memory variant runs at 256
  // fused prediction solve: mixed precision, every instance within the slice limits, and a
  // device that can hold the clusters
  if (mixed && h->opt.solver1d == GRTE_SOLVER_AUTO) {
    bool ok = std::all_of(h->inst.begin(), h->inst.end(), [](const Inst& I) { return fused_fits(I); });
    if (ok) CK(fused_attrs());
    ok = ok && fused_smem(m) <= (size_t)g_fused_optin;
    std::vector<std::vector<int>> cls(5);
    if (ok)
      for (int i = 0; i < n_inst; ++i) cls[fused_class(h->inst[i].N)].push_back(i);
    for (int c = 0; c < 5 && ok; ++c) {
      if (cls[c].empty()) continue;
      bool sched = false;
      CK(fused_schedulable(1 << c, m, &sched));
      ok = sched;
    }
    if (ok) {
      std::vector<int> order;
      for (int c = 0; c < 5; ++c) {
        h->foff[c] = (int)order.size();
        h->fcnt[c] = (int)cls[c].size();
        order.insert(order.end(), cls[c].begin(), cls[c].end());
      }
      int64_t fd = 0;
      for (int i = 0; i < n_inst; ++i) {
        h->inst[i].fd_off = fd;
        fd += (int64_t)(1 << fused_class(h->inst[i].N)) * kFS * 32;
      }
      if (dalloc(h, &h->d_finst, n_inst) != cudaSuccess) return nomem("cudaMalloc finst");
      if (dalloc(h, &D.fdata, fd) != cudaSuccess) return nomem("cudaMalloc fdata");
      CK(cudaMemcpy(h->d_finst, order.data(), sizeof(int) * n_inst, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(h->d_inst, h->inst.data(), sizeof(Inst) * n_inst, cudaMemcpyHostToDevice));
      h->fused = true;
    }
  }
  return GRTE_OK;
}

grte_status grte_set_state(grte_t h, int inst, const double* T, const double* E, const double* O) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !T) return fail(h, GRTE_EINVAL, "bad instance or T NULL");
  if ((E == nullptr) != (O == nullptr)) return fail(h, GRTE_EINVAL, "E and O must both be given or both NULL");
  const Inst& I = h->inst[inst];
  const int64_t N = I.N, M = I.M;
  std::vector<double> hE(N * M), hO((N + 1) * M), hU(N);
  for (int64_t j = 0; j < N; ++j) {
    if (!(T[j] >= 0.0) || !std::isfinite(T[j])) return fail(h, GRTE_EINVAL, "T must be finite and >= 0");
    hU[j] = (T[j] * T[j]) * (T[j] * T[j]);
  }
  // device layout: line-major, E stored as its deviation Eh = E - a c U
  for (int64_t k = 0; k < M; ++k) {
    for (int64_t j = 0; j < N; ++j) hE[k * N + j] = E ? E[j * M + k] - I.a * I.c * hU[j] : 0.0;
    for (int64_t i = 0; i <= N; ++i) hO[k * (N + 1) + i] = O ? O[i * M + k] : 0.0;
  }
  Dev& D = h->D;
  CK(cudaMemcpyAsync(D.T + I.cell_off, T, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(D.U + I.cell_off, hU.data(), sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
  if (h->opt.precision == GRTE_MIXED) {
    std::vector<float> fE(hE.begin(), hE.end()), fO(hO.begin(), hO.end());
    CK(cudaMemcpyAsync((float*)D.Eh + I.elem_off, fE.data(), sizeof(float) * N * M, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync((float*)D.O + I.nelem_off, fO.data(), sizeof(float) * (N + 1) * M, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  } else {
    CK(cudaMemcpyAsync((double*)D.Eh + I.elem_off, hE.data(), sizeof(double) * N * M, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync((double*)D.O + I.nelem_off, hO.data(), sizeof(double) * (N + 1) * M, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  h->inst_set[inst] = 1;
  h->state_set = std::all_of(h->inst_set.begin(), h->inst_set.end(), [](char c) { return c != 0; });
  return GRTE_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- one step
// The step is built from four pieces shared by the eager path (host loop over the
// Krylov iterations) and the CUDA graph (device-side conditionals):
//   prologue  coefficients at T^n, rho^n, x = rho^n, factor pass, first restart
//   iteration cellpart(V_j), direction pass, Arnoldi step j
//   tail      update x, cellpart(x), data pass, restart (residual, stopping test)
//   epilogue  Newton (Eq. Tnp1), coefficients at T^{n+1}, substep 2 and projection
struct StepGeom {
  int ni;
  int64_t nc, vstride;
  unsigned cgrid;
  static constexpr int cb = 256;
};
static StepGeom step_geom(grte_t h) {
  StepGeom g;
  g.ni = h->n_inst;
  g.nc = h->ncell;
  g.vstride = h->D.gz - h->D.gx;   // cell stride of the Krylov basis (as in k_gmres)
  g.cgrid = (unsigned)((g.nc + StepGeom::cb - 1) / StepGeom::cb);
  return g;
}

template <typename R>
static grte_status step_prologue(grte_t h, bool allow_tune) {
  NvtxRange nv_("grte: prologue (coefficients, rho^n, factor pass, first restart)");
  Dev& D = h->D;
  cudaStream_t st = h->stream;
  const StepGeom G = step_geom(h);
  LAUNCH(GRTE_K_CELL_COEF, k_cell_coef<<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, 0));
  LAUNCH(GRTE_K_RHO, k_rho<R><<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, D.rho_n));
  CK(cudaMemcpyAsync(D.gx, D.rho_n, sizeof(double) * G.nc, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(D.gits, 0, sizeof(int) * G.ni, st));
  CK(cudaMemsetAsync(D.gcycles, 0, sizeof(int) * G.ni, st));
  if (h->d_cycles) CK(cudaMemsetAsync(h->d_cycles, 0, sizeof(int), st));
  LAUNCH(GRTE_K_CELL_COEF, k_cellpart_pred<double><<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, D.gx, 1));
  if (h->nt == 0) {
    if (!allow_tune) return fail(h, GRTE_ESTATE, "line solves not tuned");
    cudaError_t e = autotune_lines<R>(h);
    if (e != cudaSuccess) return fail(h, GRTE_ECUDA, std::string("line autotune: ") + cudaGetErrorString(e));
  }
  LAUNCH(GRTE_K_PRED_FACTOR, (pred_pass<PRED_FULL_FACTOR, R>(h, D.gx)));
  LAUNCH(GRTE_K_GMRES, (gmres_launch<G_RESTART_FIRST, R>(h, 0)));
  return GRTE_OK;
}

template <typename R>
static void step_iteration(grte_t h, int j) {
  using K = typename KryT<R>::type;
  Dev& D = h->D;
  cudaStream_t st = h->stream;
  const StepGeom G = step_geom(h);
  const K* vj = (const K*)D.gV + (int64_t)j * G.vstride;   // Krylov direction
  // per-cell parts of the pass: in FP64 k_gmres forms them, in the mixed mode this kernel
  if (sizeof(R) == 4)
    LAUNCH(GRTE_K_CELL_COEF, k_cellpart_pred<K><<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, vj, 0));
  LAUNCH(GRTE_K_PRED_HOM, (pred_pass<PRED_HOM, R>(h, vj)));
  LAUNCH(GRTE_K_GMRES, (gmres_launch<G_ARNOLDI, R>(h, j)));
}

template <typename R>
static void step_tail(grte_t h) {
  Dev& D = h->D;
  cudaStream_t st = h->stream;
  const StepGeom G = step_geom(h);
  LAUNCH(GRTE_K_GMRES, (gmres_launch<G_UPDATE, R>(h, 0)));   // FP64: also the per-cell parts at x
  if (sizeof(R) == 4)
    LAUNCH(GRTE_K_CELL_COEF, k_cellpart_pred<double><<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, D.gx, 1));
  LAUNCH(GRTE_K_PRED_FULL, (pred_pass<PRED_FULL, R>(h, D.gx)));
  LAUNCH(GRTE_K_GMRES, (gmres_launch<G_RESTART, R>(h, 0)));
}

template <typename R>
static grte_status step_epilogue(grte_t h) {
  NvtxRange nv_("grte: Newton, correction, projection");
  Dev& D = h->D;
  cudaStream_t st = h->stream;
  const StepGeom G = step_geom(h);
  // correction substep 1 (per-cell Newton); T now holds T^{n+1}
  if (D.use_guess || D.log_samples)
    LAUNCH(GRTE_K_NEWTON, k_newton_feat<<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc));
  if (D.use_guess) {
    cudaError_t e = mlp_guess_launch(h->mlp, D.feat, G.nc, D.guess, st);
    if (e != cudaSuccess) return fail(h, GRTE_ECUDA, std::string("mlp guess: ") + cudaGetErrorString(e));
    ++h->launches;
  }
  LAUNCH(GRTE_K_NEWTON, k_newton<<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc));
  // correction substep 2 + projection at T^{n+1}
  LAUNCH(GRTE_K_CELL_COEF, k_cell_coef<<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, 1));
  LAUNCH(GRTE_K_CELL_COEF, k_cellpart_corr<<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc));
  LAUNCH(GRTE_K_CORR, corr_pass<R>(h, 0));
  LAUNCH(GRTE_K_PROJECT, k_project_U<<<G.cgrid, G.cb, 0, st>>>(D, G.nc));
  if (h->opt.energy_every > 0) LAUNCH(GRTE_K_ENERGY, k_energy<R><<<G.ni, kTriThreads, 0, st>>>(D, 1));
  CK(cudaGetLastError());
  return GRTE_OK;
}

// One step with the fused prediction solve: coefficients and rho^n, one persistent launch
// per cluster size for the whole GMRES solve, then Newton, correction and projection.
template <typename R>
static grte_status step_fused(grte_t h, bool allow_tune) {
  NvtxRange nv_("grte: step (one-kernel prediction solve)");
  Dev& D = h->D;
  cudaStream_t st = h->stream;
  const StepGeom G = step_geom(h);
  LAUNCH(GRTE_K_CELL_COEF, k_cell_coef<<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, 0));
  LAUNCH(GRTE_K_RHO, k_rho<R><<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, D.rho_n));
  CK(cudaMemcpyAsync(D.gx, D.rho_n, sizeof(double) * G.nc, cudaMemcpyDeviceToDevice, st));
  for (int c = 0; c < 5; ++c) {
    if (!h->fcnt[c]) continue;
    cudaError_t e = cudaSuccess;
    LAUNCH(GRTE_K_PRED_SOLVE, e = fused_launch(h, c));
    CK(e);
  }
  if (h->nt == 0) {
    if (!allow_tune) return fail(h, GRTE_ESTATE, "line solves not tuned");
    // the correction's line solves are tuned on this step's per-cell parts
    LAUNCH(GRTE_K_CELL_COEF, k_cellpart_pred<double><<<G.cgrid, G.cb, 0, st>>>(D, G.ni, h->d_cell_start, G.nc, D.gx, 1));
    cudaError_t e = autotune_lines<R>(h);
    if (e != cudaSuccess) return fail(h, GRTE_ECUDA, std::string("line autotune: ") + cudaGetErrorString(e));
  }
  return step_epilogue<R>(h);
}

template <typename R>
static grte_status build_fused_graph(grte_t h) {
  cudaStream_t st = h->stream;
  if (h->prof_mask != 0) return fail(h, GRTE_ESTATE, "graph capture while profiling");
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return fail(h, GRTE_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  const int64_t l0 = h->launches;
  grte_status s = step_fused<R>(h, false);
  if (s == GRTE_OK) k_fused_stats<<<1, 32, 0, st>>>(h->D.gits, h->D.gcycles, h->n_inst, h->d_acc);
  h->graph_fixed_launches = h->launches - l0 + 1;
  h->launches = l0;
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &graph);
  if (s != GRTE_OK) { if (graph) cudaGraphDestroy(graph); return s; }
  if (e2 == cudaSuccess) e2 = cudaGetLastError();
  if (e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(h, GRTE_ECUDA, std::string("fused step capture: ") + cudaGetErrorString(e2));
  }
  cudaGraphExec_t ex = nullptr;
  e2 = cudaGraphInstantiate(&ex, graph, 0);
  if (e2 != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(h, GRTE_ECUDA, std::string("fused step instantiate: ") + cudaGetErrorString(e2));
  }
  h->graph = graph;
  h->graph_exec = ex;
  return GRTE_OK;
}

// ENONCONV for every instance whose prediction solve is not done (restart limit).
__global__ void k_flag_undone(const int* __restrict__ gdone, int* status, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!gdone[i]) atomicOr(status + i, 1 << GRTE_ENONCONV);
}

// Eager step: the host reads the solver flags between launches.
template <typename R>
static grte_status step_once(grte_t h) {
  Dev& D = h->D;
  cudaStream_t st = h->stream;
  const int ni = h->n_inst;
  grte_status s0 = step_prologue<R>(h, true);
  if (s0 != GRTE_OK) return s0;
  int cycles = 0;
  for (;;) {
    for (int j = 0; j < D.m; ++j) {
      step_iteration<R>(h, j);
      // a Krylov direction pass costs far more than a round trip: after the first
      // iteration, stop launching once no instance is still iterating
      if (j >= 1 && j + 1 < D.m) {
        CK(cudaMemcpyAsync(h->h_flags, D.gactive, sizeof(int) * ni, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        bool any = false;
        for (int i = 0; i < ni; ++i) any = any || h->h_flags[i];
        if (!any) break;
      }
    }
    step_tail<R>(h);
    ++cycles;
    CK(cudaMemcpyAsync(h->h_flags, D.gdone, sizeof(int) * ni, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool all = true;
    for (int i = 0; i < ni; ++i) all = all && h->h_flags[i];
    if (all) break;
    if (cycles >= h->opt.krylov_maxcycles) {
      // flag the instances that did not converge (on the handle's stream)
      k_flag_undone<<<1, 256, 0, st>>>(D.gdone, D.status, ni);
      CK(cudaGetLastError());
      break;
    }
  }
  h->stats.krylov_cycles += cycles;
  return step_epilogue<R>(h);
}

// ----------------------------------------------------------------------------- graph
// Device-side control of the captured step.  k_cond_active sets an IF node's
// condition to "some instance is still iterating"; k_cond_cycle counts restart
// cycles and sets the WHILE node's condition to "some instance is not done and the
// cycle limit is not reached" (flagging the instances left undone at the limit);
// k_step_stats accumulates the step's Krylov iterations and cycles.
__global__ void k_cond_active(cudaGraphConditionalHandle hnd, const int* __restrict__ gactive, int n, long long* acc) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (gactive[i]) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    acc[3] += 1;            // condition kernels run
    if (any) acc[2] += 1;   // Krylov iterations run
    cudaGraphSetConditional(hnd, any ? 1u : 0u);
  }
}

__global__ void k_cond_cycle(cudaGraphConditionalHandle hnd, const int* __restrict__ gdone, int* status, int n,
                             int* cycles, int maxcycles, int count) {
  __shared__ int undone;
  if (threadIdx.x == 0) undone = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!gdone[i]) undone = 1;
  __syncthreads();
  const int c = *cycles + count;   // every thread reads before thread 0 writes
  __syncthreads();
  bool go = undone != 0;
  if (go && c >= maxcycles) {
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (!gdone[i]) atomicOr(status + i, 1 << GRTE_ENONCONV);
    go = false;
  }
  if (threadIdx.x == 0) {
    *cycles = c;
    cudaGraphSetConditional(hnd, go ? 1u : 0u);
  }
}

__global__ void k_step_stats(const int* __restrict__ gits, int n, const int* __restrict__ cycles,
                             long long* acc) {
  long long t = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) t += gits[i];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __shared__ long long red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    acc[0] += s;
    acc[1] += *cycles;
  }
}

// Add a conditional node at the current end of the capture on stream st and return
// its body graph; further captures on st depend on the node.
static cudaError_t capture_conditional(cudaStream_t st, cudaGraphConditionalHandle hnd, cudaGraphConditionalNodeType type,
                                       cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorIllegalState;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = hnd;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, ed, nd, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

static cudaError_t capture_graph_of(cudaStream_t st, cudaGraph_t* g) {
  cudaStreamCaptureStatus cs;
  return cudaStreamGetCaptureInfo(st, &cs, nullptr, g, nullptr, nullptr, nullptr);
}

// Capture the Krylov iterations j..m-1 as nested IF nodes on stream st:
//   cond_active(h_j); IF(h_j) { iteration j; cond_active(h_j+1); IF(h_j+1) { ... } }
template <typename R>
static grte_status capture_iterations(grte_t h, cudaStream_t st, int j, std::vector<cudaStream_t>& aux) {
  Dev& D = h->D;
  cudaGraph_t g = nullptr;
  CK(capture_graph_of(st, &g));
  cudaGraphConditionalHandle hc;
  CK(cudaGraphConditionalHandleCreate(&hc, g, 0, 0));
  k_cond_active<<<1, 256, 0, st>>>(hc, D.gactive, h->n_inst, h->d_acc);
  CK(cudaGetLastError());
  cudaGraph_t body = nullptr;
  CK(capture_conditional(st, hc, cudaGraphCondTypeIf, &body));
  cudaStream_t sb = aux[j];
  CK(cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  cudaStream_t keep = h->stream;
  h->stream = sb;
  step_iteration<R>(h, j);
  grte_status s = GRTE_OK;
  if (j + 1 < D.m) s = capture_iterations<R>(h, sb, j + 1, aux);
  h->stream = keep;
  cudaGraph_t out = nullptr;
  cudaError_t e = cudaStreamEndCapture(sb, &out);
  if (s != GRTE_OK) return s;
  CK(e);
  return GRTE_OK;
}

// Build the executable graph of one step (after the line solves are tuned).
template <typename R>
static grte_status build_step_graph(grte_t h) {
  Dev& D = h->D;
  cudaStream_t st = h->stream;
  std::vector<cudaStream_t> aux(D.m + 1, nullptr);
  for (auto& a : aux) CK(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
  auto drop = [&]() { for (auto& a : aux) if (a) cudaStreamDestroy(a); };
  const bool prof = h->prof_mask != 0;
  if (prof) { drop(); return fail(h, GRTE_ESTATE, "graph capture while profiling"); }
  grte_status s = GRTE_OK;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) { drop(); return fail(h, GRTE_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e)); }
  const int64_t l0 = h->launches;
  int64_t fixed = 0;
  do {
    s = step_prologue<R>(h, false);
    if (s != GRTE_OK) break;
    fixed += h->launches - l0;
    cudaGraph_t g = nullptr;
    if ((e = capture_graph_of(st, &g)) != cudaSuccess) break;
    cudaGraphConditionalHandle hw;
    if ((e = cudaGraphConditionalHandleCreate(&hw, g, 0, 0)) != cudaSuccess) break;
    k_cond_cycle<<<1, 256, 0, st>>>(hw, D.gdone, D.status, h->n_inst, h->d_cycles, h->opt.krylov_maxcycles, 0);
    cudaGraph_t wbody = nullptr;
    if ((e = capture_conditional(st, hw, cudaGraphCondTypeWhile, &wbody)) != cudaSuccess) break;
    cudaStream_t sw = aux[D.m];
    if ((e = cudaStreamBeginCaptureToGraph(sw, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) != cudaSuccess) break;
    h->stream = sw;
    s = capture_iterations<R>(h, sw, 0, aux);
    if (s == GRTE_OK) {
      step_tail<R>(h);
      k_cond_cycle<<<1, 256, 0, sw>>>(hw, D.gdone, D.status, h->n_inst, h->d_cycles, h->opt.krylov_maxcycles, 1);
    }
    h->stream = st;
    cudaGraph_t wout = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(sw, &wout);
    if (s != GRTE_OK) break;
    if ((e = e2) != cudaSuccess) break;
    const int64_t l1 = h->launches;
    s = step_epilogue<R>(h);
    if (s != GRTE_OK) break;
    fixed += h->launches - l1 + 2;   // + the first cycle condition and the statistics
    k_step_stats<<<1, 256, 0, st>>>(D.gits, h->n_inst, h->d_cycles, h->d_acc);
  } while (0);
  h->launches = l0;
  h->graph_fixed_launches = fixed;
  h->stream = st;
  cudaError_t e3 = cudaStreamEndCapture(st, &graph);
  drop();
  if (s != GRTE_OK) { if (graph) cudaGraphDestroy(graph); return s; }
  if (e == cudaSuccess) e = e3;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(h, GRTE_ECUDA, std::string("step graph capture: ") + cudaGetErrorString(e));
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(h, GRTE_ECUDA, std::string("step graph instantiate: ") + cudaGetErrorString(e));
  }
  h->graph = graph;
  h->graph_exec = ex;
  return GRTE_OK;
}

extern "C" {

grte_status grte_step(grte_t h, int64_t nsteps) {
  NvtxRange nv_("grte_step");
  if (!h) return GRTE_EINVAL;
  if (!h->state_set) return fail(h, GRTE_ESTATE, "state not set for every instance");
  if (nsteps < 0) return fail(h, GRTE_EINVAL, "nsteps < 0");
  h->stats.krylov_cycles = 0;
  h->stats.krylov_iters = 0;
  h->launches = 0;
  const bool mixed = h->opt.precision == GRTE_MIXED;
  int64_t its = 0, cyc = 0, ngraph = 0;
  std::vector<int> hits(h->n_inst);
  CK(cudaMemsetAsync(h->d_acc, 0, 4 * sizeof(long long), h->stream));
  if (h->fused) {
    std::vector<int> hcyc(h->n_inst);
    for (int64_t n = 0; n < nsteps; ++n) {
      const bool use_graph = h->opt.use_graph && h->nt != 0 && h->prof_mask == 0;
      if (use_graph) {
        if (!h->graph_exec) {
          grte_status s = build_fused_graph<float>(h);
          if (s != GRTE_OK) return s;
        }
        CK(cudaGraphLaunch(h->graph_exec, h->stream));
        ++ngraph;
      } else {
        grte_status s = step_fused<float>(h, true);
        if (s != GRTE_OK) return s;
        CK(cudaMemcpyAsync(hits.data(), h->D.gits, sizeof(int) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaMemcpyAsync(hcyc.data(), h->D.gcycles, sizeof(int) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int v : hits) its += v;
        for (int v : hcyc) cyc += v;
      }
      h->stats.steps += 1;
    }
    if (ngraph > 0) {
      long long acc[4] = {0, 0, 0, 0};
      CK(cudaMemcpyAsync(acc, h->d_acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      its += acc[0];
      cyc += acc[1];
      h->launches += ngraph * h->graph_fixed_launches;
    }
    h->stats.krylov_iters = its;
    h->stats.krylov_cycles = cyc;
    return GRTE_OK;
  }
  for (int64_t n = 0; n < nsteps; ++n) {
    // graph path: after the first (tuning) step, when not profiling
    const bool use_graph = h->opt.use_graph && h->nt != 0 && h->prof_mask == 0;
    if (use_graph) {
      if (!h->graph_exec) {
        grte_status s = mixed ? build_step_graph<float>(h) : build_step_graph<double>(h);
        if (s != GRTE_OK) return s;
      }
      CK(cudaGraphLaunch(h->graph_exec, h->stream));
      ++ngraph;
    } else {
      const int64_t c0 = h->stats.krylov_cycles;
      grte_status s = mixed ? step_once<float>(h) : step_once<double>(h);
      if (s != GRTE_OK) return s;
      cyc += h->stats.krylov_cycles - c0;
      CK(cudaMemcpyAsync(hits.data(), h->D.gits, sizeof(int) * h->n_inst, cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int v : hits) its += v;
    }
    h->stats.steps += 1;
  }
  if (ngraph > 0) {
    long long acc[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(acc, h->d_acc, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    its += acc[0];
    cyc += acc[1];
    // kernels run by the graph steps: the fixed ones, per cycle the tail (mixed 4, FP64 3)
    // and its condition kernel, every condition kernel of the iterations, and per
    // iteration run the direction pass and the Arnoldi step (mixed: also the per-cell parts)
    const int64_t per_cycle = mixed ? 5 : 4, per_iter = mixed ? 3 : 2;
    h->launches += ngraph * h->graph_fixed_launches + acc[1] * per_cycle + acc[3] + acc[2] * per_iter;
  }
  h->stats.krylov_iters = its;
  h->stats.krylov_cycles = cyc;
  return GRTE_OK;
}

static grte_status device_status(grte_t h) {
  std::vector<int> s(h->n_inst);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(s.data(), h->D.status, sizeof(int) * h->n_inst, cudaMemcpyDeviceToHost));
  int64_t all = 0;
  for (int v : s) all |= v;
  h->stats.status_flags = all;
  for (int code : {GRTE_ENAN, GRTE_ENONCONV, GRTE_ENEGATIVE, GRTE_ETIMEOUT})
    if (all & (1 << code)) return fail(h, (grte_status)code, "device reported status " + std::to_string(code));
  return GRTE_OK;
}

grte_status grte_sync(grte_t h) {
  if (!h) return GRTE_EINVAL;
  const grte_status s = device_status(h);
  // reported once: the per-instance flags are cleared for the steps that follow
  if (s != GRTE_OK && s != GRTE_ECUDA) CK(cudaMemset(h->D.status, 0, sizeof(int) * h->n_inst));
  return s;
}

static grte_status get_cells(grte_t h, int inst, const double* src, double* out, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !out) return fail(h, GRTE_EINVAL, "bad instance or NULL output");
  const Inst& I = h->inst[inst];
  if (len != (size_t)I.N) return fail(h, GRTE_EINVAL, "len must equal nx");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(out, src + I.cell_off, sizeof(double) * I.N, cudaMemcpyDeviceToHost));
  return device_status(h);
}

grte_status grte_get_T(grte_t h, int inst, double* T, size_t len) {
  if (!h) return GRTE_EINVAL;
  return get_cells(h, inst, h->D.T, T, len);
}

grte_status grte_get_stage(grte_t h, int inst, int which, double* out, size_t len) {
  if (!h) return GRTE_EINVAL;
  const double* src = which == 0 ? h->D.Us : which == 1 ? h->D.Fs : which == 2 ? h->D.rho_s
                    : which == 3 ? h->D.newton_its : which == 4 ? h->D.Fc : nullptr;
  if (!src) return fail(h, GRTE_EINVAL, "which must be 0..4");
  return get_cells(h, inst, src, out, len);
}

// Copy n bulk elements from device offset `off` (in elements) of `base` into doubles.
static grte_status copy_bulk(grte_t h, const void* base, int64_t off, int64_t n, double* out) {
  CK(cudaStreamSynchronize(h->stream));
  if (h->opt.precision == GRTE_MIXED) {
    std::vector<float> t(n);
    CK(cudaMemcpy(t.data(), (const float*)base + off, sizeof(float) * n, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i) out[i] = t[i];
  } else {
    CK(cudaMemcpy(out, (const double*)base + off, sizeof(double) * n, cudaMemcpyDeviceToHost));
  }
  return GRTE_OK;
}

grte_status grte_get_E(grte_t h, int inst, double* E, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !E) return fail(h, GRTE_EINVAL, "bad instance or NULL output");
  const Inst& I = h->inst[inst];
  if (len != (size_t)I.N * I.M) return fail(h, GRTE_EINVAL, "len must equal nx*M");
  std::vector<double> t((size_t)I.N * I.M), U(I.N);
  grte_status s = copy_bulk(h, h->D.Eh, I.elem_off, (int64_t)t.size(), t.data());
  if (s != GRTE_OK) return s;
  CK(cudaMemcpy(U.data(), h->D.U + I.cell_off, sizeof(double) * I.N, cudaMemcpyDeviceToHost));
  for (int64_t k = 0; k < I.M; ++k)
    for (int64_t j = 0; j < I.N; ++j) E[j * I.M + k] = I.a * I.c * U[j] + t[k * I.N + j];
  return device_status(h);
}

grte_status grte_get_O(grte_t h, int inst, double* O, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !O) return fail(h, GRTE_EINVAL, "bad instance or NULL output");
  const Inst& I = h->inst[inst];
  if (len != (size_t)(I.N + 1) * I.M) return fail(h, GRTE_EINVAL, "len must equal (nx+1)*M");
  std::vector<double> t((size_t)(I.N + 1) * I.M);
  grte_status s = copy_bulk(h, h->D.O, I.nelem_off, (int64_t)t.size(), t.data());
  if (s != GRTE_OK) return s;
  for (int64_t k = 0; k < I.M; ++k)
    for (int64_t i = 0; i <= I.N; ++i) O[i * I.M + k] = t[k * (I.N + 1) + i];
  return device_status(h);
}

grte_status grte_get_rho(grte_t h, int inst, double* rho, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !rho) return fail(h, GRTE_EINVAL, "bad instance or NULL output");
  const Inst& I = h->inst[inst];
  if (len != (size_t)I.N) return fail(h, GRTE_EINVAL, "len must equal nx");
  std::vector<double> E((size_t)I.N * I.M);
  grte_status s = grte_get_E(h, inst, E.data(), E.size());
  if (s != GRTE_OK && s != GRTE_ENEGATIVE) return s;
  for (int64_t j = 0; j < I.N; ++j) {
    double acc = 0.0;
    for (int k = 0; k < I.M; ++k) acc += h->hw[I.ang_off + k] * E[j * I.M + k];
    rho[j] = acc;
  }
  return s;
}

grte_status grte_get_I(grte_t h, int inst, double* Ipos, double* Ineg, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !Ipos || !Ineg) return fail(h, GRTE_EINVAL, "bad instance or NULL output");
  const Inst& I = h->inst[inst];
  if (len != (size_t)I.N * I.M) return fail(h, GRTE_EINVAL, "len must equal nx*M");
  std::vector<double> E((size_t)I.N * I.M), O((size_t)(I.N + 1) * I.M);
  grte_status s = grte_get_E(h, inst, E.data(), E.size());
  if (s != GRTE_OK && s != GRTE_ENEGATIVE) return s;
  s = grte_get_O(h, inst, O.data(), O.size());
  if (s != GRTE_OK && s != GRTE_ENEGATIVE) return s;
  for (int64_t j = 0; j < I.N; ++j)
    for (int k = 0; k < I.M; ++k) {
      const double oc = 0.5 * (O[j * I.M + k] + O[(j + 1) * I.M + k]);
      Ipos[j * I.M + k] = E[j * I.M + k] + I.eps * oc;
      Ineg[j * I.M + k] = E[j * I.M + k] - I.eps * oc;
    }
  return s;
}

// Checkpoint blob: a header, the per-instance sizes, the energy sums and the raw device
// state (T, U in binary64; Eh = E - a c U and O in the handle's bulk type), so that a
// restored handle continues bit for bit.
namespace {
struct BlobHead {
  char magic[8];
  uint32_t version, dim, precision, n_inst;
  int64_t steps;
};
constexpr char kBlobMagic[8] = {'G', 'R', 'T', 'E', 'S', 'T', '1', 'D'};
}  // namespace

static size_t blob_size(grte_t h) {
  const size_t es = h->opt.precision == GRTE_MIXED ? 4 : 8;
  size_t n = sizeof(BlobHead) + sizeof(int64_t) * 2 * h->n_inst + sizeof(double) * 3 * h->n_inst;
  for (const Inst& I : h->inst) n += sizeof(double) * 2 * I.N + es * (I.N * I.M + (I.N + 1) * I.M);
  return n;
}

grte_status grte_get_state(grte_t h, void* buf, size_t* len) {
  if (!h || !len) return GRTE_EINVAL;
  const size_t need = blob_size(h);
  if (!buf) {
    *len = need;
    return GRTE_OK;
  }
  if (*len < need) return fail(h, GRTE_EINVAL, "buffer smaller than the state (query the size with buf = NULL)");
  if (!h->state_set) return fail(h, GRTE_ESTATE, "state not set");
  CK(cudaStreamSynchronize(h->stream));
  unsigned char* p = (unsigned char*)buf;
  BlobHead hd{};
  memcpy(hd.magic, kBlobMagic, 8);
  hd.version = 1;
  hd.dim = 1;
  hd.precision = (uint32_t)h->opt.precision;
  hd.n_inst = (uint32_t)h->n_inst;
  hd.steps = h->stats.steps;
  memcpy(p, &hd, sizeof hd);
  p += sizeof hd;
  for (const Inst& I : h->inst) {
    const int64_t nm[2] = {I.N, I.M};
    memcpy(p, nm, sizeof nm);
    p += sizeof nm;
  }
  CK(cudaMemcpy(p, h->D.energy, sizeof(double) * 3 * h->n_inst, cudaMemcpyDeviceToHost));
  p += sizeof(double) * 3 * h->n_inst;
  const size_t es = h->opt.precision == GRTE_MIXED ? 4 : 8;
  for (const Inst& I : h->inst) {
    CK(cudaMemcpy(p, h->D.T + I.cell_off, sizeof(double) * I.N, cudaMemcpyDeviceToHost));
    p += sizeof(double) * I.N;
    CK(cudaMemcpy(p, h->D.U + I.cell_off, sizeof(double) * I.N, cudaMemcpyDeviceToHost));
    p += sizeof(double) * I.N;
    CK(cudaMemcpy(p, (const char*)h->D.Eh + es * I.elem_off, es * I.N * I.M, cudaMemcpyDeviceToHost));
    p += es * I.N * I.M;
    CK(cudaMemcpy(p, (const char*)h->D.O + es * I.nelem_off, es * (I.N + 1) * I.M, cudaMemcpyDeviceToHost));
    p += es * (I.N + 1) * I.M;
  }
  *len = need;
  return device_status(h);
}

grte_status grte_restore_state(grte_t h, const void* buf, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (!buf || len != blob_size(h)) return fail(h, GRTE_EINVAL, "blob size does not match this handle");
  const unsigned char* p = (const unsigned char*)buf;
  BlobHead hd;
  memcpy(&hd, p, sizeof hd);
  p += sizeof hd;
  if (memcmp(hd.magic, kBlobMagic, 8) != 0 || hd.version != 1 || hd.dim != 1)
    return fail(h, GRTE_EINVAL, "not a 1D state blob of this library");
  if (hd.precision != (uint32_t)h->opt.precision || hd.n_inst != (uint32_t)h->n_inst)
    return fail(h, GRTE_EINVAL, "blob precision or instance count differs from this handle");
  for (const Inst& I : h->inst) {
    int64_t nm[2];
    memcpy(nm, p, sizeof nm);
    p += sizeof nm;
    if (nm[0] != I.N || nm[1] != I.M) return fail(h, GRTE_EINVAL, "blob instance sizes differ from this handle");
  }
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(h->D.energy, p, sizeof(double) * 3 * h->n_inst, cudaMemcpyHostToDevice));
  p += sizeof(double) * 3 * h->n_inst;
  const size_t es = h->opt.precision == GRTE_MIXED ? 4 : 8;
  for (const Inst& I : h->inst) {
    CK(cudaMemcpy(h->D.T + I.cell_off, p, sizeof(double) * I.N, cudaMemcpyHostToDevice));
    p += sizeof(double) * I.N;
    CK(cudaMemcpy(h->D.U + I.cell_off, p, sizeof(double) * I.N, cudaMemcpyHostToDevice));
    p += sizeof(double) * I.N;
    CK(cudaMemcpy((char*)h->D.Eh + es * I.elem_off, p, es * I.N * I.M, cudaMemcpyHostToDevice));
    p += es * I.N * I.M;
    CK(cudaMemcpy((char*)h->D.O + es * I.nelem_off, p, es * (I.N + 1) * I.M, cudaMemcpyHostToDevice));
    p += es * (I.N + 1) * I.M;
  }
  h->stats.steps = hd.steps;
  std::fill(h->inst_set.begin(), h->inst_set.end(), (char)1);
  h->state_set = true;
  return GRTE_OK;
}

grte_status grte_get_T_device(grte_t h, int inst, double* dptr, size_t len, void* stream) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !dptr) return fail(h, GRTE_EINVAL, "bad instance or NULL output");
  const Inst& I = h->inst[inst];
  if (len != (size_t)I.N) return fail(h, GRTE_EINVAL, "len must equal nx");
  cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
  if (st != h->stream) {
    // the copy waits for the handle's queued steps, on the caller's stream
    CK(cudaEventRecord(h->ev_state, h->stream));
    CK(cudaStreamWaitEvent(st, h->ev_state, 0));
  }
  CK(cudaMemcpyAsync(dptr, h->D.T + I.cell_off, sizeof(double) * I.N, cudaMemcpyDeviceToDevice, st));
  return GRTE_OK;
}

grte_status grte_get_energy(grte_t h, int inst, double* out, size_t n) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !out || n != 3) return fail(h, GRTE_EINVAL, "bad instance, NULL output or n != 3");
  if (!h->state_set) return fail(h, GRTE_ESTATE, "state not set");
  // refresh the energy of the current state; the accumulated terms are untouched
  if (h->opt.precision == GRTE_MIXED) k_energy<float><<<h->n_inst, kTriThreads, 0, h->stream>>>(h->D, 0);
  else k_energy<double><<<h->n_inst, kTriThreads, 0, h->stream>>>(h->D, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(out, h->D.energy + 3 * inst, sizeof(double) * 3, cudaMemcpyDeviceToHost));
  return GRTE_OK;
}

grte_status grte_get_quadrature(grte_t h, int inst, double* v, double* w, size_t len) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !v || !w) return fail(h, GRTE_EINVAL, "bad instance or NULL output");
  const Inst& I = h->inst[inst];
  if (len != (size_t)I.M) return fail(h, GRTE_EINVAL, "len must equal n_angle");
  std::memcpy(v, h->hv.data() + I.ang_off, sizeof(double) * I.M);
  std::memcpy(w, h->hw.data() + I.ang_off, sizeof(double) * I.M);
  return GRTE_OK;
}

grte_status grte_stats(grte_t h, grte_stats_t* st) {
  if (!h || !st) return GRTE_EINVAL;
  std::vector<double> its(h->ncell);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(its.data(), h->D.newton_its, sizeof(double) * h->ncell, cudaMemcpyDeviceToHost));
  double mx = 0, sum = 0;
  for (double v : its) {
    mx = std::max(mx, v);
    sum += v;
  }
  h->stats.newton_iters_max = (int64_t)mx;
  h->stats.newton_iters_mean = h->ncell ? sum / h->ncell : 0.0;
  h->stats.line_threads = h->nt;
  h->stats.line_smem = h->xs ? 1 : 0;
  grte_status s = device_status(h);
  *st = h->stats;
  return s;
}

grte_status grte_get_tuning(grte_t h, int* line_threads, double* ms, size_t n) {
  if (!h) return GRTE_EINVAL;
  if (!line_threads || !ms || n < 3) return fail(h, GRTE_EINVAL, "need line_threads and ms[3]");
  *line_threads = h->nt;
  for (int i = 0; i < 3; ++i) ms[i] = h->tune_ms[i];
  return GRTE_OK;
}

grte_status grte_profile_begin(grte_t h, uint32_t kernel_mask) {
  if (!h) return GRTE_EINVAL;
  CK(cudaStreamSynchronize(h->stream));
  h->prof_ev.clear();
  h->ev_used = 0;
  h->prof_mask = kernel_mask;
  return GRTE_OK;
}

grte_status grte_profile_end(grte_t h, double* ms, int64_t* launches, size_t n) {
  if (!h) return GRTE_EINVAL;
  if (!ms || !launches || n < (size_t)GRTE_NKERNELS) return fail(h, GRTE_EINVAL, "need GRTE_NKERNELS outputs");
  CK(cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < n; ++i) { ms[i] = 0.0; launches[i] = 0; }
  for (auto& pe : h->prof_ev) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, pe.second.first, pe.second.second));
    ms[pe.first] += t;
    launches[pe.first] += 1;
  }
  h->prof_ev.clear();
  h->ev_used = 0;
  h->prof_mask = 0;
  return GRTE_OK;
}

int64_t grte_last_launches(grte_t h) { return h ? h->launches : 0; }

static grte_status ensure_feat(grte_t h) {
  Dev& D = h->D;
  if (!D.feat) {
    if (dalloc(h, &D.feat, 6 * h->ncell) != cudaSuccess) return fail(h, GRTE_ENOMEM, "cudaMalloc feat");
    if (dalloc(h, &D.guess, h->ncell) != cudaSuccess) return fail(h, GRTE_ENOMEM, "cudaMalloc guess");
    if (dalloc(h, &D.ytrue, h->ncell) != cudaSuccess) return fail(h, GRTE_ENOMEM, "cudaMalloc ytrue");
  }
  return GRTE_OK;
}

grte_status grte_set_guess(grte_t h, grte_mlp_t m) {
  if (!h) return GRTE_EINVAL;
  drop_step_graph(h);
  CK(cudaStreamSynchronize(h->stream));
  if (m) {
    grte_status s = ensure_feat(h);
    if (s != GRTE_OK) return s;
  }
  h->mlp = m;
  h->D.use_guess = m ? 1 : 0;
  h->D.start_prev = 0;
  return GRTE_OK;
}

grte_status grte_set_newton_start(grte_t h, int mode) {
  if (!h) return GRTE_EINVAL;
  drop_step_graph(h);
  if (mode != GRTE_START_BOUND && mode != GRTE_START_PREVIOUS && mode != GRTE_START_LEARNED)
    return fail(h, GRTE_EINVAL, "bad start mode");
  if (mode == GRTE_START_LEARNED && !h->mlp) return fail(h, GRTE_ESTATE, "no network set (grte_set_guess)");
  CK(cudaStreamSynchronize(h->stream));
  h->D.start_prev = mode == GRTE_START_PREVIOUS ? 1 : 0;
  h->D.use_guess = mode == GRTE_START_LEARNED ? 1 : 0;
  return GRTE_OK;
}

grte_status grte_set_sample_logging(grte_t h, int on) {
  if (!h) return GRTE_EINVAL;
  drop_step_graph(h);
  CK(cudaStreamSynchronize(h->stream));
  if (on) {
    grte_status s = ensure_feat(h);
    if (s != GRTE_OK) return s;
  }
  h->D.log_samples = on ? 1 : 0;
  return GRTE_OK;
}

grte_status grte_get_newton_samples(grte_t h, int inst, float* X, float* y, size_t nx) {
  if (!h) return GRTE_EINVAL;
  if (inst < 0 || inst >= h->n_inst || !X || !y) return fail(h, GRTE_EINVAL, "bad instance or NULL output");
  const Inst& I = h->inst[inst];
  if (nx != (size_t)I.N) return fail(h, GRTE_EINVAL, "nx must equal the instance's cell count");
  if (!h->D.log_samples) return fail(h, GRTE_ESTATE, "sample logging is off");
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(X, h->D.feat + 6 * I.cell_off, sizeof(float) * 6 * I.N, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(y, h->D.ytrue + I.cell_off, sizeof(float) * I.N, cudaMemcpyDeviceToHost));
  return GRTE_OK;
}

}  // extern "C"

// =============================================================================== no-allocation step
// grte_step1d_noalloc: the steps of grte_step for one FP64 instance whose state lives
// in caller-owned device memory, with every work buffer carved out of one file-scope
// device array (no cudaMalloc, cudaFree or other allocating call on any path).
namespace grte {
constexpr int64_t kNaMaxCells = 4096;
constexpr int kNaMaxAngles = 32;
constexpr int64_t kNaMaxElems = 65536;                      // nx * n_angle
constexpr int64_t kNaMaxNodeElems = kNaMaxElems + kNaMaxAngles;
constexpr int64_t kNaCellArrays = 42;                       // per-cell double arrays (40 + the x/z pair)
constexpr int64_t kNaAlign = 256;
__host__ __device__ constexpr int64_t na_round(int64_t b) { return (b + kNaAlign - 1) / kNaAlign * kNaAlign; }
// line solves run at kTriThreads threads here: per line at most 2 kTriThreads reduced
// equations and 9 PCR levels
constexpr int64_t kNaRedLine = 10 * 2 * (2 * kTriThreads) + 2 * kTriThreads;   // >= tri_red_size(n, kTriThreads)
constexpr int64_t kNaFacLine = 5 * kTriThreads;   // tri_fac_size(n, kTriThreads) <= 5 n + kNaFacLine
constexpr int64_t kNaBytes =
    kNaCellArrays * na_round(8 * kNaMaxCells) +                     // per-cell arrays
    na_round(8 * 5 * (kNaMaxCells + kCL * kTriThreads)) +           // preconditioner factors
    na_round(8 * kCL * kNaRedLine) +                                // preconditioner reduced systems
    na_round(8 * (kMaxRestart + 1) * kNaMaxCells) +                 // Krylov basis
    na_round(8 * kNaMaxElems) * 4 +                                 // Eh, xb, S, S2
    na_round(8 * (5 * kNaMaxElems + kNaMaxAngles * kNaFacLine)) +   // line factors
    na_round(8 * kNaMaxNodeElems) +                                 // node scratch
    na_round(8 * kNaMaxAngles * kNaRedLine) +                        // line reduced systems
    na_round(8 * 4 * kNaMaxAngles) + na_round(8 * 2 * kNaMaxAngles) +   // v, w, bL, bR; Swall
    na_round(8 * ((kMaxRestart + 1) * kMaxRestart + 3 * kMaxRestart + 8 + kCL * 2 * 2 * kCL)) +
    na_round(4 * 16) + na_round(sizeof(Inst)) + na_round(sizeof(Line) * kNaMaxAngles) + na_round(8);
}  // namespace grte

// Work memory of grte_step1d_noalloc: kNaBytes = 11,198,464 bytes (about 11.2 MB),
// held by every GPU that loads the library until the process exits.  Calls share it
// (see include/grte.h, which states the same figure; the assertion keeps the two in
// step when the layout changes).
static_assert(grte::kNaBytes == 11198464, "no-alloc work memory size changed: update the documented figure");
static __device__ __align__(256) unsigned char g_noalloc_scratch[grte::kNaBytes];
static void* g_noalloc_base[64];   // device address of g_noalloc_scratch, per device

namespace grte {
__global__ void k_na_prepare(const double* __restrict__ T, const double* __restrict__ E, double* __restrict__ U,
                             double* __restrict__ Eh, int64_t N, int M, double ac) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid < N) {
    const double t = T[gid];
    U[gid] = (t * t) * (t * t);
  }
  if (gid < N * M) {
    const double t = T[gid % N];
    Eh[gid] = E[gid] - ac * ((t * t) * (t * t));
  }
}
__global__ void k_na_finish(const double* __restrict__ U, const double* __restrict__ Eh, double* __restrict__ E,
                            int64_t N, int M, double ac) {
  const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (gid < N * M) E[gid] = ac * U[gid % N] + Eh[gid];
}

// Gauss-Legendre, positive half, into fixed arrays (n <= 2 kNaMaxAngles).
static void gl_half_fixed(int n, double* v, double* w) {
  const int M = n / 2;
  for (int i = 0; i < M; ++i) {
    double x = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      const double d = p1 / dp;
      x -= d;
      if (fabs(d) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    v[M - 1 - i] = x;
    w[M - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}
}  // namespace grte

extern "C" grte_status grte_step1d_noalloc(const grte_instance1d* p, const grte_options* opt, double* T,
                                           double* E, double* O, int64_t nsteps, void* stream) {
  using namespace grte;
  if (!p || !T || !E || !O || nsteps < 0) return GRTE_EINVAL;
  grte_options o;
  grte_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != GRTE_FP64) return GRTE_EINVAL;
  if (o.krylov_restart < 1 || o.krylov_restart > kMaxRestart || o.krylov_maxcycles < 1 || o.newton_maxit < 1 ||
      !(o.krylov_rtol > 0))
    return GRTE_EINVAL;
  const int64_t N = p->nx;
  const int M = p->n_angle;
  // size limits of the static work memory
  if (N < 2 || N > kNaMaxCells || M < 1 || M > kNaMaxAngles || N * M > kNaMaxElems) return GRTE_EINVAL;
  if (!p->sigma || (p->sigma_kind != GRTE_SIGMA_CONST && p->sigma_kind != GRTE_SIGMA_T3 &&
                    !(p->sigma_kind == GRTE_SIGMA_POW && p->sigma_p >= 0.0 && p->sigma_p <= 3.0)) ||
      (p->bc != GRTE_BC_INFLOW && p->bc != GRTE_BC_REFLECT))
    return GRTE_EINVAL;
  if (!(p->x1 > p->x0) || !(p->dt > 0) || !(p->a > 0) || !(p->c > 0) || !(p->Cv > 0) || !(p->eps > 0))
    return GRTE_EINVAL;
  if ((p->v == nullptr) != (p->w == nullptr)) return GRTE_EINVAL;
  double v[kNaMaxAngles], w[kNaMaxAngles], bL[kNaMaxAngles], bR[kNaMaxAngles];
  if (p->v) {
    for (int k = 0; k < M; ++k) { v[k] = p->v[k]; w[k] = p->w[k]; }
  } else {
    gl_half_fixed(2 * M, v, w);
  }
  double sw = 0.0;
  for (int k = 0; k < M; ++k) {
    if (!(v[k] > 0.0 && v[k] <= 1.0) || !(w[k] > 0.0)) return GRTE_EINVAL;
    sw += w[k];
  }
  for (int k = 0; k < M; ++k) w[k] /= sw;
  for (int64_t j = 0; j < N; ++j)
    if (!(p->sigma[j] >= 0.0) || !std::isfinite(p->sigma[j])) return GRTE_EINVAL;
  Inst I{};
  I.N = (int)N; I.M = M; I.bc = p->bc; I.eps = p->eps; I.dt = p->dt;
  I.kind = p->sigma_kind == GRTE_SIGMA_CONST ? GRTE_SIGMA_CONST : GRTE_SIGMA_T3;
  I.p = p->sigma_kind == GRTE_SIGMA_POW ? p->sigma_p : 3.0;
  I.dx = (p->x1 - p->x0) / (double)N; I.a = p->a; I.c = p->c; I.Cv = p->Cv;
  double wv = 0, wv2 = 0, fl = 0, fr = 0;
  for (int k = 0; k < M; ++k) {
    bL[k] = (p->bc == GRTE_BC_INFLOW && p->bL) ? p->bL[k] : 0.0;
    bR[k] = (p->bc == GRTE_BC_INFLOW && p->bR) ? p->bR[k] : 0.0;
    wv += w[k] * v[k];
    wv2 += w[k] * v[k] * v[k];
    fl += w[k] * v[k] * bL[k];
    fr += w[k] * v[k] * bR[k];
  }
  I.wv = wv; I.wv2 = wv2; I.bLflux = fl; I.bRflux = fr;
  inst_derive(I);
  I.cell_off = 0; I.elem_off = 0; I.nelem_off = 0; I.red_off = 0; I.ang_off = 0; I.line_off = 0;
  Line lines[kNaMaxAngles];
  for (int k = 0; k < M; ++k) lines[k] = Line{0, k, (int64_t)k * kNaRedLine, (int64_t)k * (5 * N + kNaFacLine)};

  // device address of the static work memory: looked up once per device, with the
  // device current (the host-side symbol is not a device address)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GRTE_ECUDA;
  if (!g_noalloc_base[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return GRTE_ECUDA;
    g_noalloc_base[dev] = ptr;
  }
  unsigned char* cur = (unsigned char*)g_noalloc_base[dev];
  auto take = [&](int64_t bytes) { unsigned char* q = cur; cur += na_round(bytes); return (void*)q; };
  Dev D{};
  double** cells[kNaCellArrays - 2] = {&D.U, &D.sig, &D.rho_n, &D.rho_s, &D.Fs, &D.Us, &D.newton_its, &D.P1, &D.P2,
                                   &D.P3, &D.Frho, &D.gU, &D.Q1, &D.Q2, &D.gwork, &D.cf.kc, &D.cf.s,
                                   &D.cf.alpha, &D.cf.A, &D.cf.gam, &D.cf.gl, &D.cf.gu, &D.cf.gb, &D.cf.dl,
                                   &D.cf.od, &D.cf.dlx, &D.cf.kcd, &D.cf.kdx, &D.cf.sac, &D.cf.ralpha,
                                   &D.cf.ratio, &D.cf.fR, &D.cf.fL, &D.cf.gbx, &D.pG, &D.pH, &D.gw,
                                   &D.cf.dsx, &D.cf.ods, &D.Fc};
  for (int i = 0; i < kNaCellArrays - 2; ++i) *cells[i] = (double*)take(8 * kNaMaxCells);
  // x and z of the Krylov kernels are adjacent: the kernels take the cell stride of
  // the basis as gz - gx, here kNaMaxCells
  D.gx = (double*)take(8 * 2 * kNaMaxCells);
  D.gz = D.gx + kNaMaxCells;
  D.pF = (double*)take(8 * 5 * (kNaMaxCells + kCL * kTriThreads));
  D.pRd = (double*)take(8 * kCL * kNaRedLine);
  D.gV = (double*)take(8 * (kMaxRestart + 1) * kNaMaxCells);
  D.Eh = take(8 * kNaMaxElems);
  D.xb = take(8 * kNaMaxElems);
  D.S = take(8 * kNaMaxElems);
  D.S2 = take(8 * kNaMaxElems);
  D.F = take(8 * (5 * kNaMaxElems + kNaMaxAngles * kNaFacLine));
  D.onode = take(8 * kNaMaxNodeElems);
  D.Rd = take(8 * kNaMaxAngles * kNaRedLine);
  double* vw = (double*)take(8 * 4 * kNaMaxAngles);
  D.v = vw; D.w = vw + kNaMaxAngles; D.bL = vw + 2 * kNaMaxAngles; D.bR = vw + 3 * kNaMaxAngles;
  D.Swall = (double*)take(8 * 2 * kNaMaxAngles);
  double* small = (double*)take(8 * ((kMaxRestart + 1) * kMaxRestart + 3 * kMaxRestart + 8 + kCL * 2 * 2 * kCL));
  D.gH = small;
  D.gg = D.gH + (kMaxRestart + 1) * kMaxRestart;
  D.gcs = D.gg + kMaxRestart + 1;
  D.gsn = D.gcs + kMaxRestart;
  D.gbeta = D.gsn + kMaxRestart;
  D.gxn = D.gbeta + 1;
  D.energy = D.gxn + 1;
  D.pInv = D.energy + 4;
  int* ints = (int*)take(4 * 16);
  D.gactive = ints; D.gk = ints + 1; D.gdone = ints + 2; D.gits = ints + 3; D.gcycles = ints + 4;
  D.gestconv = ints + 5; D.status = ints + 6;
  Inst* d_inst = (Inst*)take(sizeof(Inst));
  Line* d_lines = (Line*)take(sizeof(Line) * kNaMaxAngles);
  int64_t* d_cell_start = (int64_t*)take(8);
  if (cur - (unsigned char*)g_noalloc_base[dev] > kNaBytes) return GRTE_ENOMEM;   // layout check
  D.T = T;
  D.O = O;
  D.inst = d_inst;
  D.lines = d_lines;
  D.m = o.krylov_restart;
  D.maxcycles = o.krylov_maxcycles;
  D.rtol = o.krylov_rtol;
  D.stall = 1e-9;
  D.wfloor = 1e-13;
  D.mixed = 0;
  D.newton_maxit = o.newton_maxit;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t zero64 = 0;
#define NA(call) do { if ((call) != cudaSuccess) return GRTE_ECUDA; } while (0)
  NA(cudaMemcpyAsync(d_inst, &I, sizeof(Inst), cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync(d_lines, lines, sizeof(Line) * M, cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync(d_cell_start, &zero64, 8, cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync(D.v, v, 8 * M, cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync(D.w, w, 8 * M, cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync(D.bL, bL, 8 * M, cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync(D.bR, bR, 8 * M, cudaMemcpyHostToDevice, st));
  NA(cudaMemcpyAsync(D.sig, p->sigma, 8 * N, cudaMemcpyHostToDevice, st));
  // what must start at zero: statuses, counters, energy sums, Krylov scalars
  NA(cudaMemsetAsync(ints, 0, 4 * 16, st));
  NA(cudaMemsetAsync(small, 0, 8 * ((kMaxRestart + 1) * kMaxRestart + 3 * kMaxRestart + 8 + kCL * 2 * 2 * kCL), st));
  const double ac = p->a * p->c;
  const unsigned eb = (unsigned)((N * M + 255) / 256);
  k_na_prepare<<<eb, 256, 0, st>>>(T, E, D.U, (double*)D.Eh, N, M, ac);
  NA(cudaGetLastError());
  // a handle that lives on this stack frame and refers only to the memory above
  grte_ctx ctx;
  ctx.n_inst = 1;
  ctx.ncell = N;
  ctx.nelem = N * M;
  ctx.nnelem = (N + 1) * M;
  ctx.nlines = M;
  ctx.opt = o;
  ctx.opt.energy_every = 0;
  ctx.stream = st;
  ctx.D = D;
  ctx.d_cell_start = d_cell_start;
  ctx.d_inst = d_inst;
  ctx.d_lines = d_lines;
  int flag_buf[1] = {0};
  ctx.h_flags = flag_buf;
  ctx.state_set = true;
  // line solves at kTriThreads threads, unknowns in shared memory when they fit
  if (line_kernel_attrs() != cudaSuccess) { ctx.h_flags = nullptr; return GRTE_ECUDA; }
  ctx.maxN = N;
  ctx.xs = line_fits(&ctx, kTriThreads);
  ctx.max_slice = N / std::min<int64_t>(N / 2, kCL) + 1;
  ctx.gxs = (tri_xs_len(ctx.max_slice) * 8 + 15) / 16 * 16 <= g_gmres_dyn;
  ctx.nt = kTriThreads;
  for (int64_t n = 0; n < nsteps; ++n) {
    grte_status s = step_once<double>(&ctx);
    if (s != GRTE_OK) { ctx.h_flags = nullptr; return s; }
  }
  ctx.h_flags = nullptr;   // not owned
  k_na_finish<<<eb, 256, 0, st>>>(D.U, (const double*)D.Eh, E, N, M, ac);
  NA(cudaGetLastError());
  int status = 0;
  NA(cudaMemcpyAsync(&status, D.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA(cudaStreamSynchronize(st));
#undef NA
  for (int code : {GRTE_ENAN, GRTE_ENONCONV, GRTE_ENEGATIVE, GRTE_ETIMEOUT})
    if (status & (1 << code)) return (grte_status)code;
  return GRTE_OK;
}
