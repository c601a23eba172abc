// CTA-cooperative partitioned tridiagonal solver (sm_103a).
//
// Solves  a_j x_{j-1} + b_j x_j + c_j x_{j+1} = r_j,  j = 0..n-1  (a_0 = c_{n-1} = 0)
// for strictly diagonally dominant systems (no pivoting).  The n unknowns are cut
// into P contiguous chunks (one per thread).  Each thread eliminates its chunk's
// interior so that the interior unknowns depend only on the chunk's first and last
// unknowns; the 2P first/last unknowns form a tridiagonal reduced system (a Schur
// complement, still diagonally dominant) that the CTA solves by parallel cyclic
// reduction in shared memory; each thread then back-substitutes its interior.
//
// FACTOR mode also stores everything that depends on the matrix only (per element:
// 1/den, c-hat, c-check, a-check; per system: the PCR multipliers and the final
// reciprocal diagonal), so later SOLVE calls with the same matrix do only the
// right-hand-side recurrences: 5 flops per element plus 2 per reduced equation and
// PCR level.
//
// The right-hand side is read from x[] and the solution written back to x[] (global
// memory, unit stride).  Storage sizes: 4*n values in F, tri_red_size(n) in Rd.
#pragma once
#include <cstdint>

namespace grte {

constexpr int kTriThreads = 256;          // threads (and at most this many chunks) per CTA
constexpr int kTriMaxRed = 2 * kTriThreads;
constexpr int kB = 8;                     // elements per block of the serial sweeps
constexpr int kMaxLevels = 10;            // PCR levels for up to 2*kTriThreads reduced equations

__host__ __device__ inline int tri_chunks(int64_t n) {
  int64_t p = n / 2;
  return (int)(p < kTriThreads ? p : kTriThreads);
}
__host__ __device__ inline int tri_levels(int nr) {
  int L = 0;
  while ((1 << L) < nr) ++L;
  return L;
}
__host__ __device__ inline int64_t tri_red_size(int64_t n) {
  int nr = 2 * tri_chunks(n);
  return (int64_t)tri_levels(nr) * 2 * nr + nr;
}

template <typename R>
struct TriSmem {
  R a[2][kTriMaxRed];
  R b[2][kTriMaxRed];
  R c[2][kTriMaxRed];
  R r[2][kTriMaxRed];
};

// Coefficient provider interface (Cf): R a(int64_t j), b(j), c(j); a(0) and c(n-1)
// must be 0.  b() is called in FACTOR mode only.
template <bool FACTOR, typename R, class Cf>
__device__ void tri_solve(const Cf& cf, int64_t n, R* __restrict__ x, R* __restrict__ F,
                          R* __restrict__ Rd, TriSmem<R>& sm) {
  const int P = tri_chunks(n);
  const int nr = 2 * P;
  const int L = tri_levels(nr);
  const int tid = threadIdx.x;
  R* f_inv = F;
  R* f_ch = F + n;
  R* f_cc = F + 2 * n;
  R* f_ac = F + 3 * n;
  const int64_t base = n / P;
  const int64_t rem = n % P;

  // ---- phase A: chunk elimination -------------------------------------------------
  if (tid < P) {
    const int64_t s = tid * base + (tid < rem ? tid : rem);
    const int64_t len = base + (tid < rem ? 1 : 0);
    const int64_t e = s + len - 1;
    R rs, re, As = 0, Bs = 0, Cs = 0, Ae = 0, Be = 0, Ce = 0;
    if (len >= 3) {
      // down sweep over the interior s+1..e-1:
      //   x_j = rhat_j - chat_j x_{j+1} - ahat_j x_s
      // The recurrences are serial, so the loads of each block of kB elements are
      // issued together ahead of the dependent arithmetic (one memory latency per
      // block instead of one per element).
      R rh = 0, ch = 0, ah = 0;
      int64_t j = s + 1;
      if (FACTOR) {
        for (; j <= e - 1; ++j) {
          const R aj = cf.a(j), bj = cf.b(j), cj = cf.c(j), rj = x[j];
          const R den = (j == s + 1) ? bj : bj - aj * ch;
          const R inv = R(1) / den;
          ah = (j == s + 1) ? aj * inv : -aj * ah * inv;
          ch = cj * inv;
          f_inv[j] = inv;
          f_ch[j] = ch;
          f_ac[j] = ah;            // a-hat for now; becomes a-check in the up sweep
          rh = (j == s + 1) ? rj * inv : (rj - aj * rh) * inv;
          x[j] = rh;
        }
      } else {
        rh = x[j] * f_inv[j];
        x[j] = rh;
        ++j;
        for (; j + kB - 1 <= e - 1; j += kB) {
          R xv[kB], iv[kB], av[kB];
#pragma unroll
          for (int u = 0; u < kB; ++u) {
            xv[u] = x[j + u];
            iv[u] = f_inv[j + u];
            av[u] = cf.a(j + u);
          }
#pragma unroll
          for (int u = 0; u < kB; ++u) {
            rh = (xv[u] - av[u] * rh) * iv[u];
            xv[u] = rh;
          }
#pragma unroll
          for (int u = 0; u < kB; ++u) x[j + u] = xv[u];
        }
        for (; j <= e - 1; ++j) {
          rh = (x[j] - cf.a(j) * rh) * f_inv[j];
          x[j] = rh;
        }
      }
      // up sweep: x_j = rcheck_j - ccheck_j x_e - acheck_j x_s
      R rc = x[e - 1];
      if (FACTOR) {
        R cc = f_ch[e - 1], ac = f_ac[e - 1];
        f_cc[e - 1] = cc;
        for (int64_t jj = e - 2; jj >= s + 1; --jj) {
          const R chj = f_ch[jj];
          rc = x[jj] - chj * rc;
          x[jj] = rc;
          cc = -chj * cc;
          ac = f_ac[jj] - chj * ac;
          f_cc[jj] = cc;
          f_ac[jj] = ac;
        }
      } else {
        int64_t jj = e - 2;
        for (; jj - (kB - 1) >= s + 1; jj -= kB) {
          R xv[kB], cv[kB];
#pragma unroll
          for (int u = 0; u < kB; ++u) {
            xv[u] = x[jj - u];
            cv[u] = f_ch[jj - u];
          }
#pragma unroll
          for (int u = 0; u < kB; ++u) {
            rc = xv[u] - cv[u] * rc;
            xv[u] = rc;
          }
#pragma unroll
          for (int u = 0; u < kB; ++u) x[jj - u] = xv[u];
        }
        for (; jj >= s + 1; --jj) {
          rc = x[jj] - f_ch[jj] * rc;
          x[jj] = rc;
        }
      }
      // reduced rows of x_s and x_e
      R cS = cf.c(s), aE = cf.a(e);
      rs = x[s] - cS * x[s + 1];           // x[s+1] holds rcheck_{s+1}
      re = x[e] - aE * x[e - 1];           // x[e-1] holds rhat_{e-1} (= rcheck_{e-1})
      if (FACTOR) {
        As = cf.a(s);
        Bs = cf.b(s) - cS * f_ac[s + 1];
        Cs = -cS * f_cc[s + 1];
        Ae = -aE * f_ac[e - 1];           // a-hat_{e-1} = a-check_{e-1}
        Be = cf.b(e) - aE * f_ch[e - 1];
        Ce = cf.c(e);
      }
    } else {  // len == 2: no interior
      rs = x[s];
      re = x[e];
      if (FACTOR) {
        As = cf.a(s); Bs = cf.b(s); Cs = cf.c(s);
        Ae = cf.a(e); Be = cf.b(e); Ce = cf.c(e);
      }
    }
    sm.r[0][2 * tid] = rs;
    sm.r[0][2 * tid + 1] = re;
    if (FACTOR) {
      sm.a[0][2 * tid] = As; sm.b[0][2 * tid] = Bs; sm.c[0][2 * tid] = Cs;
      sm.a[0][2 * tid + 1] = Ae; sm.b[0][2 * tid + 1] = Be; sm.c[0][2 * tid + 1] = Ce;
    }
  }
  __syncthreads();

  // ---- phase B: parallel cyclic reduction on the nr reduced equations -----------
  // SOLVE mode: every level's multipliers of this thread's equations are loaded
  // before the first level (one memory latency instead of one per level)
  R pk1[kMaxLevels][2], pk2[kMaxLevels][2];
  if (!FACTOR) {
#pragma unroll
    for (int l = 0; l < kMaxLevels; ++l)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = tid + q * blockDim.x;
        if (l < L && i < nr) {
          pk1[l][q] = Rd[(int64_t)l * 2 * nr + i];
          pk2[l][q] = Rd[(int64_t)l * 2 * nr + nr + i];
        }
      }
  }
  int cur = 0;
#pragma unroll
  for (int l = 0; l < kMaxLevels; ++l) {
    if (l >= L) break;
    const int st = 1 << l;
    R* k1s = Rd + (int64_t)l * 2 * nr;
    R* k2s = k1s + nr;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int i = tid + q * blockDim.x;
      if (i >= nr) continue;
      const bool hasL = i - st >= 0, hasR = i + st < nr;
      R k1, k2;
      if (FACTOR) {
        k1 = hasL ? sm.a[cur][i] / sm.b[cur][i - st] : R(0);
        k2 = hasR ? sm.c[cur][i] / sm.b[cur][i + st] : R(0);
        k1s[i] = k1;
        k2s[i] = k2;
        sm.a[cur ^ 1][i] = hasL ? -sm.a[cur][i - st] * k1 : R(0);
        sm.c[cur ^ 1][i] = hasR ? -sm.c[cur][i + st] * k2 : R(0);
        R bn = sm.b[cur][i];
        if (hasL) bn -= sm.c[cur][i - st] * k1;
        if (hasR) bn -= sm.a[cur][i + st] * k2;
        sm.b[cur ^ 1][i] = bn;
      } else {
        k1 = pk1[l][q];
        k2 = pk2[l][q];
      }
      R rn = sm.r[cur][i];
      if (hasL) rn -= sm.r[cur][i - st] * k1;
      if (hasR) rn -= sm.r[cur][i + st] * k2;
      sm.r[cur ^ 1][i] = rn;
    }
    __syncthreads();
    cur ^= 1;
  }
  R* ib = Rd + (int64_t)L * 2 * nr;
  for (int i = tid; i < nr; i += blockDim.x) {
    R inv;
    if (FACTOR) {
      inv = R(1) / sm.b[cur][i];
      ib[i] = inv;
    } else {
      inv = ib[i];
    }
    sm.r[cur][i] *= inv;
  }
  __syncthreads();

  // ---- phase C: back substitution ---------------------------------------------------
  if (tid < P) {
    const int64_t s = tid * base + (tid < rem ? tid : rem);
    const int64_t len = base + (tid < rem ? 1 : 0);
    const int64_t e = s + len - 1;
    const R xs = sm.r[cur][2 * tid], xe = sm.r[cur][2 * tid + 1];
    x[s] = xs;
    x[e] = xe;
#pragma unroll 4
    for (int64_t j = s + 1; j <= e - 1; ++j) x[j] = x[j] - f_cc[j] * xe - f_ac[j] * xs;
  }
  __syncthreads();
}

}  // namespace grte
