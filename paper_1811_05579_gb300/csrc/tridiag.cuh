// CTA-cooperative partitioned tridiagonal solver (sm_103a).
//
// Solves  a_j x_{j-1} + b_j x_j + c_j x_{j+1} = r_j,  j = 0..n-1  (a_0 = c_{n-1} = 0)
// for strictly diagonally dominant systems (no pivoting).  The n unknowns are cut
// into P contiguous chunks (one per thread, P <= blockDim.x).  Each thread eliminates
// its chunk's interior so that the interior unknowns depend only on the chunk's first
// and last unknowns; the 2P first/last unknowns form a tridiagonal reduced system (a
// Schur complement, still diagonally dominant) that the CTA solves by parallel cyclic
// reduction (PCR) in shared memory; each thread then back-substitutes its interior.
//
// FACTOR mode also stores everything that depends on the matrix only, so that later
// SOLVE calls with the same matrix do only the right-hand-side recurrences (5 flops
// per element plus 2 per reduced equation and PCR level) and never evaluate the
// coefficients.  Factor storage is chunk-interleaved: element u of chunk t sits at
// u*P + t, so the P threads' u-th elements are adjacent and every factor load or
// store of a warp is one contiguous segment.  Five arrays of tri_fac_stride(n, nt)
// values each: 1/den, a (plus c of the chunk's first row in slot 0), c-hat, c-check,
// a-check.  PCR multipliers and the final reciprocal diagonal take tri_red_size(n, nt).
//
// The right-hand side is read from x and the solution written back to x through an
// accessor: shared memory (padded by one slot per 32 so that the threads' chunk
// walks hit distinct banks) or global memory (unit stride).
#pragma once
#include <cstdint>

namespace grte {

constexpr int kTriThreads = 256;          // threads per CTA of the preconditioner slices
constexpr int kTriMaxNT = 1024;           // largest thread count of a line CTA
constexpr int kMaxLevels = 11;            // PCR levels for up to 2*kTriMaxNT reduced equations
constexpr int kB = 8;                     // elements per block of the serial sweeps
constexpr int kPcrAhead = 4;              // PCR levels whose multipliers are loaded ahead

__host__ __device__ inline int tri_chunks(int64_t n, int nt) {
  int64_t p = n / 2;
  return (int)(p < nt ? p : nt);
}
__host__ __device__ inline int tri_levels(int nr) {
  int L = 0;
  while ((1 << L) < nr) ++L;
  return L;
}
__host__ __device__ inline int64_t tri_red_size(int64_t n, int nt) {
  int nr = 2 * tri_chunks(n, nt);
  return (int64_t)tri_levels(nr) * 2 * nr + nr;
}
// values per factor array (>= n; <= n + min(n/2, nt))
__host__ __device__ inline int64_t tri_fac_stride(int64_t n, int nt) {
  const int64_t P = tri_chunks(n, nt);
  return (n / P + 1) * P;
}
__host__ __device__ inline int64_t tri_fac_size(int64_t n, int nt) { return 5 * tri_fac_stride(n, nt); }
// shared-memory bytes of the reduced system: FACTOR keeps a, b, c, r (in place), SOLVE
// a double-buffered r
__host__ __device__ inline int64_t tri_smem_bytes(int nt, bool factor, int elem) {
  return (int64_t)(factor ? 4 : 2) * 2 * nt * elem;
}
// padded length of a shared-memory x of n values
__host__ __device__ inline int64_t tri_xs_len(int64_t n) { return n + (n >> 5) + 1; }

template <typename R, bool SM>
struct XAcc {
  R* p;
  __device__ __forceinline__ R& operator[](int64_t j) const { return SM ? p[j + (j >> 5)] : p[j]; }
};

// Coefficient provider interface (Cf): R a(int64_t j), b(j), c(j); a(0) and c(n-1)
// must be 0.  Called in FACTOR mode only.  `red` points at tri_smem_bytes(blockDim.x,
// FACTOR, sizeof(R)) bytes of shared memory.
template <bool FACTOR, typename R, class Cf, class X>
__device__ void tri_solve(const Cf& cf, int64_t n, const X& x, R* __restrict__ F, R* __restrict__ Rd, R* red) {
  const int nt = blockDim.x;
  const int P = tri_chunks(n, nt);
  const int nr = 2 * P;
  const int L = tri_levels(nr);
  const int tid = threadIdx.x;
  const int64_t fs = tri_fac_stride(n, nt);
  R* f_inv = F;
  R* f_a = F + fs;
  R* f_ch = F + 2 * fs;
  R* f_cc = F + 3 * fs;
  R* f_ac = F + 4 * fs;
  const int64_t base = n / P;
  const int64_t rem = n % P;
  // shared reduced system: FACTOR a|b|c|r, SOLVE r0|r1
  R* sa = red;
  R* sb = red + nr;
  R* sc = red + 2 * nr;
  R* sr = FACTOR ? red + 3 * nr : red;

  // ---- phase A: chunk elimination -------------------------------------------------
  if (tid < P) {
    const int64_t s = tid * base + (tid < rem ? tid : rem);
    const int64_t len = base + (tid < rem ? 1 : 0);   // >= 2
    const int64_t e = s + len - 1;
    auto fi = [&](int64_t u) { return u * P + tid; };
    R rs, re, As = 0, Bs = 0, Cs = 0, Ae = 0, Be = 0, Ce = 0;
    if (len >= 3) {
      // down sweep over the interior u = 1..len-2:
      //   x_j = rhat_j - chat_j x_{j+1} - ahat_j x_s
      R rh = 0, ch = 0, ah = 0;
      if (FACTOR) {
        for (int64_t u = 1; u <= len - 2; ++u) {
          const int64_t j = s + u;
          const R aj = cf.a(j), bj = cf.b(j), cj = cf.c(j), rj = x[j];
          const R den = (u == 1) ? bj : bj - aj * ch;
          const R inv = R(1) / den;
          ah = (u == 1) ? aj * inv : -aj * ah * inv;
          ch = cj * inv;
          f_inv[fi(u)] = inv;
          f_a[fi(u)] = aj;
          f_ch[fi(u)] = ch;
          f_ac[fi(u)] = ah;        // a-hat for now; becomes a-check in the up sweep
          rh = (u == 1) ? rj * inv : (rj - aj * rh) * inv;
          x[j] = rh;
        }
      } else {
        // the recurrences are serial: the loads of a block of kB elements are issued
        // together ahead of the dependent arithmetic
        rh = x[s + 1] * f_inv[fi(1)];
        x[s + 1] = rh;
        int64_t u = 2;
        for (; u + kB - 1 <= len - 2; u += kB) {
          R xv[kB], iv[kB], av[kB];
#pragma unroll
          for (int q = 0; q < kB; ++q) {
            xv[q] = x[s + u + q];
            iv[q] = f_inv[fi(u + q)];
            av[q] = f_a[fi(u + q)];
          }
#pragma unroll
          for (int q = 0; q < kB; ++q) {
            rh = (xv[q] - av[q] * rh) * iv[q];
            xv[q] = rh;
          }
#pragma unroll
          for (int q = 0; q < kB; ++q) x[s + u + q] = xv[q];
        }
        for (; u <= len - 2; ++u) {
          rh = (x[s + u] - f_a[fi(u)] * rh) * f_inv[fi(u)];
          x[s + u] = rh;
        }
      }
      // up sweep: x_j = rcheck_j - ccheck_j x_e - acheck_j x_s
      R rc = x[e - 1];
      if (FACTOR) {
        R cc = f_ch[fi(len - 2)], ac = f_ac[fi(len - 2)];
        f_cc[fi(len - 2)] = cc;
        for (int64_t u = len - 3; u >= 1; --u) {
          const R chj = f_ch[fi(u)];
          rc = x[s + u] - chj * rc;
          x[s + u] = rc;
          cc = -chj * cc;
          ac = f_ac[fi(u)] - chj * ac;
          f_cc[fi(u)] = cc;
          f_ac[fi(u)] = ac;
        }
      } else {
        int64_t u = len - 3;
        for (; u - (kB - 1) >= 1; u -= kB) {
          R xv[kB], cv[kB];
#pragma unroll
          for (int q = 0; q < kB; ++q) {
            xv[q] = x[s + u - q];
            cv[q] = f_ch[fi(u - q)];
          }
#pragma unroll
          for (int q = 0; q < kB; ++q) {
            rc = xv[q] - cv[q] * rc;
            xv[q] = rc;
          }
#pragma unroll
          for (int q = 0; q < kB; ++q) x[s + u - q] = xv[q];
        }
        for (; u >= 1; --u) {
          rc = x[s + u] - f_ch[fi(u)] * rc;
          x[s + u] = rc;
        }
      }
      // reduced rows of x_s and x_e; c_s and a_e are kept in the unused slots
      // f_ch[slot 0] and f_a[slot len-1] for the SOLVE calls
      R cS, aE;
      if (FACTOR) {
        cS = cf.c(s);
        aE = cf.a(e);
        f_ch[fi(0)] = cS;
        f_a[fi(len - 1)] = aE;
      } else {
        cS = f_ch[fi(0)];
        aE = f_a[fi(len - 1)];
      }
      rs = x[s] - cS * x[s + 1];           // x[s+1] holds rcheck_{s+1}
      re = x[e] - aE * x[e - 1];           // x[e-1] holds rhat_{e-1} (= rcheck_{e-1})
      if (FACTOR) {
        As = cf.a(s);
        Bs = cf.b(s) - cS * f_ac[fi(1)];
        Cs = -cS * f_cc[fi(1)];
        Ae = -aE * f_ac[fi(len - 2)];     // a-hat_{e-1} = a-check_{e-1}
        Be = cf.b(e) - aE * f_ch[fi(len - 2)];
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
    sr[2 * tid] = rs;
    sr[2 * tid + 1] = re;
    if (FACTOR) {
      sa[2 * tid] = As; sb[2 * tid] = Bs; sc[2 * tid] = Cs;
      sa[2 * tid + 1] = Ae; sb[2 * tid + 1] = Be; sc[2 * tid + 1] = Ce;
    }
  }
  __syncthreads();

  // ---- phase B: parallel cyclic reduction on the nr reduced equations -----------
  // thread tid owns equations tid and tid + nt (nr <= 2 nt)
  R* ib = Rd + (int64_t)L * 2 * nr;
  if (FACTOR) {
    // in place: every level reads its neighbours into registers, then writes
    for (int l = 0; l < L; ++l) {
      const int st = 1 << l;
      R* k1s = Rd + (int64_t)l * 2 * nr;
      R* k2s = k1s + nr;
      R na[2], nb[2], nc[2], nrr[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = tid + q * nt;
        if (i >= nr) continue;
        const bool hasL = i - st >= 0, hasR = i + st < nr;
        const R k1 = hasL ? sa[i] / sb[i - st] : R(0);
        const R k2 = hasR ? sc[i] / sb[i + st] : R(0);
        k1s[i] = k1;
        k2s[i] = k2;
        na[q] = hasL ? -sa[i - st] * k1 : R(0);
        nc[q] = hasR ? -sc[i + st] * k2 : R(0);
        R bn = sb[i], rn = sr[i];
        if (hasL) { bn -= sc[i - st] * k1; rn -= sr[i - st] * k1; }
        if (hasR) { bn -= sa[i + st] * k2; rn -= sr[i + st] * k2; }
        nb[q] = bn;
        nrr[q] = rn;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = tid + q * nt;
        if (i >= nr) continue;
        sa[i] = na[q]; sb[i] = nb[q]; sc[i] = nc[q]; sr[i] = nrr[q];
      }
      __syncthreads();
    }
    for (int i = tid; i < nr; i += nt) {
      const R inv = R(1) / sb[i];
      ib[i] = inv;
      sr[i] *= inv;
    }
  } else {
    // double-buffered r; the multipliers of level l + kPcrAhead are loaded while
    // level l runs (a ring of registers, indices fixed by the full unroll)
    R k1r[kPcrAhead][2], k2r[kPcrAhead][2];
#pragma unroll
    for (int l = 0; l < kPcrAhead; ++l)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = tid + q * nt;
        if (l < L && i < nr) {
          k1r[l][q] = Rd[(int64_t)l * 2 * nr + i];
          k2r[l][q] = Rd[(int64_t)l * 2 * nr + nr + i];
        }
      }
    R* rc = sr;
    R* rn = sr + nr;
#pragma unroll
    for (int l = 0; l < kMaxLevels; ++l) {
      if (l >= L) break;
      const int st = 1 << l;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int i = tid + q * nt;
        if (i >= nr) continue;
        const R k1 = k1r[l % kPcrAhead][q], k2 = k2r[l % kPcrAhead][q];
        R v = rc[i];
        if (i - st >= 0) v -= rc[i - st] * k1;
        if (i + st < nr) v -= rc[i + st] * k2;
        rn[i] = v;
        const int la = l + kPcrAhead;
        if (la < L) {
          k1r[l % kPcrAhead][q] = Rd[(int64_t)la * 2 * nr + i];
          k2r[l % kPcrAhead][q] = Rd[(int64_t)la * 2 * nr + nr + i];
        }
      }
      __syncthreads();
      R* t = rc; rc = rn; rn = t;
    }
    for (int i = tid; i < nr; i += nt) rc[i] *= ib[i];
    sr = rc;
  }
  __syncthreads();

  // ---- phase C: back substitution ---------------------------------------------------
  if (tid < P) {
    const int64_t s = tid * base + (tid < rem ? tid : rem);
    const int64_t len = base + (tid < rem ? 1 : 0);
    const int64_t e = s + len - 1;
    const R xs = sr[2 * tid], xe = sr[2 * tid + 1];
    x[s] = xs;
    x[e] = xe;
#pragma unroll 4
    for (int64_t u = 1; u <= len - 2; ++u) {
      const int64_t k = u * P + tid;
      x[s + u] = x[s + u] - f_cc[k] * xe - f_ac[k] * xs;
    }
  }
  __syncthreads();
}

}  // namespace grte
