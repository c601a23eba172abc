// fused1d.cuh - the prediction solve of one 1D time step as one persistent kernel per
// instance (GB300, sm_103a).  Included by grte1d.cu inside namespace grte.
//
// What it computes is what the line-kernel path computes: the prediction of Algorithm 2
// (Eq. dis-pre, Eq. dis-pre-marshak, wall rows Eq. bc-pre) written on (rho, e), E = rho + e,
//   e-equation     (A + G_k) e_k = h_k - alpha rho - G_k rho        (tridiagonal per angle)
//   conservation   R(rho) = alpha rho - kappa rho^n/(c dt) - s a c U^n + kappa/dx F(rho) = 0,
//                  F_j = sum_k w_k v_k (O_{j+1,k} - O_{j,k}),
// solved for rho by restarted GMRES left-preconditioned by the single-effective-angle Schur
// operator P = alpha + Gbar (A + Gbar)^{-1} beta (Gbar = sum_k w_k G_k, beta = A - alpha).
// Its outputs are the converged rho* (D.gx), F* (D.Fs) and the flux the temperature
// equation takes (D.Fc: for sigma_0/T^3 the flux of Eq. dis-cor-marshak1 with the node
// coefficients of V* = max(U*, 0)^{3/4} at the converged iterate, the inflow wall cells
// keeping F*; for sigma(x) F* itself), read by the Newton kernel.
//
// How it runs: one thread-block cluster of Q CTAs per instance (Q in {1,2,4,8,16}), CTA q
// owning the 512-cell slice [512 q, 512 q + 512) (cells past nx are decoupled identity rows).
// The cluster runs every restart cycle, Arnoldi step, line pass and preconditioner
// application of the solve without leaving the kernel; control decisions are taken from
// cluster-wide sums reduced in a fixed rank order, so every CTA takes the same branch.
//   - A line pass (the product behind one GMRES matrix-vector product) keeps the unknowns of
//     all angles of the slice in shared memory: warp w owns cells [32 w, 32 w + 32), lane k
//     the angle v_k (M <= 32).  Each thread eliminates its 32-cell chunk with the tridiagonal
//     coefficients recomputed from per-cell arrays held in shared memory (binary32), so a pass
//     reads no per-element data besides the state (data passes only).  The chunks' end rows
//     form a 32-row tridiagonal system per angle, solved by parallel cyclic reduction (PCR)
//     together with its two unit spikes; the slices' 2x2 Schur complements then form a
//     2Q-row interface system per angle, gathered through distributed shared memory and
//     solved by PCR in every CTA; each thread finally back-substitutes its chunk.
//   - The angular sums of the flux are reduced per cell in shared memory in a fixed order.
//   - The Krylov vectors (binary64) live in global memory, one slice per CTA; dot products
//     are block sums then cluster sums in rank order (bit-reproducible).
//   - The preconditioner is one tridiagonal solve per instance in binary64, run by warp 0 of
//     every CTA on its slice with the same chunk / PCR / interface construction.
// Mixed precision only (binary32 line passes, binary64 per-cell parts, Krylov vectors,
// preconditioner, the two inflow wall rows and the true residual's angular sums).

namespace grte {

constexpr int kFL = 32;           // cells per chunk (one thread's serial sweep)
constexpr int kFW = 16;           // chunks (warps) per slice
constexpr int kFS = kFL * kFW;    // cells per slice (one CTA)
constexpr int kFT = 32 * kFW;     // threads per CTA
constexpr int kFQ = 16;           // largest cluster: nx <= kFQ * kFS
constexpr int kFR = 2 * kFW;      // reduced rows per angle and slice
constexpr int kFX = 33;           // padded row length of the slice's unknowns
constexpr int kFPL = kFS / 32;    // cells per lane of the preconditioner's warp (16)
constexpr int kPW = 4;            // preconditioner sub-chunk warps (4 cells each per lane)
static_assert(kFPL == 4 * kPW, "the preconditioner's two levels assume 16 = 4 x 4 cells per lane");

struct FSmem {
  float x[kFS][kFX];                                   // unknowns of the slice, [cell][angle]
  // per-cell binary32 arrays of the slice with one halo cell each side (index j - c0 + 1)
  // the line coefficients packed (x: A, y: gl, z: gu, w: gb), one load per sweep step
  float4 lc[kFS + 2];
  float od[kFS + 2], dlx[kFS + 2], kcd[kFS + 2], kdx[kFS + 2];
  float P1[kFS], P2[kFS], P3[kFS];                      // per-cell parts of the pass
  // reduced systems: [row][angle]
  float ra[kFR][33], rb[kFR][33], rc[kFR][33], rr[kFR][33], rg[kFR][33], rh[kFR][33];
  float ends[2][4][32];                                 // published: S11 S12 S21 S22 (double-buffered)
  float endr[2][2][32];                                 // published: r'_F, r'_L
  float coup[2][2][32];                                 // published: a at the first cell, c at the last
  float xlr[2][32];                                     // e at c0 - 1 and at c0 + kFS, per angle
  float vk[32], v2k[32], wvk[32], wvkl[32];            // per-angle constants (0 past M); wvkl:
                                                        // w v - wvk (binary32 low part)
  double vkd[32], wvkd[32];
  double wib[2][32], wgn[2][32], won[2][32], wdl[2];   // inflow wall rows (f_load_cells)
  double fl[kFS];                                       // flux sums of the last pass
  double fdat[kFS];                                     // data part of the flux (data passes)
  // the correction's flux (sigma_0/T^3): node coefficients d* of V* = (U*)^{3/4} at the
  // nodes c0 + t (t = 0..kFS), the node moments Om = sum_k w_k v_k O^n, the flux per cell
  double Om[kFS + 1];                                  // node moments of O^n (sigma_0/T^3 data)
  double pu[kFS];                                       // preconditioner solution (slice)
  // binary64 preconditioner, factored once per solve: chunk sweeps [u][lane] (u = 1..kFPL-2),
  // the reduced 64-row system's PCR multipliers and unit spikes, the interface's multipliers
  double pxr[kFPL][32], pinv[kFPL][32], pa[kFPL][32], pch[kFPL][32], pah[kFPL][32];
  double pcs[32], pae[32];
  double pc0[kPW][32], pa3[kPW][32];                  // level A: c at a sub-chunk's first cell, a at its last
  double pk1[6][64], pk2[6][64], pib[64], pgv[64], phv[64];
  double ik1[5][32], ik2[5][32], iib[32];
  double pS[4], paf, pcl;
  float wgt[kFS];                                       // stopping-test weights
  double zv[kFS];                                       // preconditioner input (slice)
  double sc[4];                                         // scalars computed once (thread 0)
  long long xmw[kFW];                                   // per-warp max |x| (bit patterns)
  double xmx[2];                                        // the slice's max |x|, per restart parity
  double xmall;                                         // the cluster's max |x|
  double wall[2][32];                                   // wall-row right-hand sides (double)
  double red[kFW][kMaxRestart + 2];                     // per-warp partial sums
  double part[2][kMaxRestart + 2];                      // cluster partials (double-buffered)
  double sums[kMaxRestart + 2];
  // binary64 preconditioner: reduced rows of the 32 lane chunks (64 rows), interface
  double pe[2][6];                                      // published: S11 S12 S21 S22 r'F r'L
  double pcoup[2][2];
  double pxl[2];
  // GMRES state (identical in every CTA)
  double H[(kMaxRestart + 1) * kMaxRestart], hinv[kMaxRestart], g[kMaxRestart + 1], cs[kMaxRestart],
      sn[kMaxRestart],
      y[kMaxRestart], hc[kMaxRestart + 2];
  int stop;
};
// V* and d* of the correction's flux (f_pass) are kept as binary64 over the reduced-system
// arrays after the line solve: ra..rb and rc..rr must be adjacent and 8-byte aligned
static_assert(offsetof(FSmem, ra) % 8 == 0 && offsetof(FSmem, rc) % 8 == 0, "alignment");
static_assert(offsetof(FSmem, rb) == offsetof(FSmem, ra) + sizeof(FSmem::ra) &&
              offsetof(FSmem, rc) == offsetof(FSmem, rb) + sizeof(FSmem::rb) &&
              offsetof(FSmem, rr) == offsetof(FSmem, rc) + sizeof(FSmem::rc), "layout");
static_assert(2 * sizeof(FSmem::ra) >= (kFS + 2) * sizeof(double), "room for V*");

// Per-CTA geometry.
struct FGeo {
  int ii, q, Q;         // instance, slice, slices in the cluster
  int64_t c0, co;       // first cell of the slice (instance-local), instance cell offset
  int N, M;
};

// Cluster reductions.  The binary64 pipe is the scarce resource (one warp instruction
// holds a sub-partition's pipe for many cycles), so the slice part runs on warps 0..3, one
// per sub-partition, each thread accumulating 4 cells; a warp then reduces its S values
// with a reduce-scatter butterfly (S - 1 + 5 - log2 S additions per lane instead of 5 S),
// and the 16 ranks' partials are combined by a 16-lane butterfly per value.  Maxima are of
// non-negative terms (or NaN), taken as integer maxima of the binary64 bit patterns (order
// preserving for x >= 0; a NaN wins), off the binary64 pipe.  The order of the additions
// is fixed, so every CTA of the cluster gets the same bits.
constexpr int kGW = 4;                 // warps of the slice part
constexpr int kGC = kFS / (32 * kGW);  // cells per thread (4)

// In-warp reduce-scatter of S (a power of two <= 16) values per lane: on return a[0] holds
// the warp sum of value vi, and the lanes whose low 5 - log2 S bits are 0 hold distinct vi.
template <int S>
__device__ __forceinline__ double f_warp_rs(double (&a)[S], int lane, int& vi) {
  int base = 0, o = 16;
#pragma unroll
  for (int h = S / 2; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int s2 = 0; s2 < h; ++s2) {
      const double send = up ? a[s2] : a[s2 + h];
      const double keep = up ? a[s2 + h] : a[s2];
      a[s2] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    if (up) base += h;
  }
  for (; o >= 1; o >>= 1) a[0] += __shfl_xor_sync(0xffffffffu, a[0], o);
  vi = base;
  return a[0];
}

// Warp part of the slice sums for S slots (ns <= S live): writes sm.red[wid][0..ns-1].
template <int S, class FS>
__device__ __forceinline__ void f_slice_rs(FSmem& sm, int ns, FS sterm) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  double a[S];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    a[i] = 0.0;
    if (i < ns) {
#pragma unroll
      for (int c = 0; c < kGC; ++c) a[i] += sterm(i, t + c * 32 * kGW);
    }
  }
  int vi;
  const double r = f_warp_rs<S>(a, lane, vi);
  constexpr int lowbits = 32 / S - 1;
  if ((lane & lowbits) == 0 && vi < ns) sm.red[wid][vi] = r;
}

// ns <= NS sums of sterm(i, c) (i < ns) and, if MX, the maximum of mterm(c) >= 0 over the
// cluster's cells (c the slice cell); results in sm.sums[0..ns-1] and sm.sums[ns] for every
// thread.  Every thread takes part; par selects the half of the double buffer.
template <int NS, bool MX, class FS, class FM>
__device__ void f_reduce(FSmem& sm, cg::cluster_group& cl, int& par, int ns, FS sterm, FM mterm) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  if (wid < kGW) {
    if (NS > 0 && ns > 0) {
      if (NS <= 1 || ns <= 1) f_slice_rs<1>(sm, ns, sterm);
      else if (NS <= 2 || ns <= 2) f_slice_rs<(NS < 2 ? 1 : 2)>(sm, ns, sterm);
      else if (NS <= 4 || ns <= 4) f_slice_rs<(NS < 4 ? 1 : 4)>(sm, ns, sterm);
      else if (NS <= 8 || ns <= 8) f_slice_rs<(NS < 8 ? 1 : 8)>(sm, ns, sterm);
      else f_slice_rs<(NS < 16 ? 1 : 16)>(sm, ns, sterm);
    }
    if (MX) {
      long long m = 0;
#pragma unroll
      for (int c = 0; c < kGC; ++c) m = max(m, __double_as_longlong(mterm(t + c * 32 * kGW)));
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) sm.red[wid][ns] = __longlong_as_double(m);
    }
  }
  __syncthreads();
  const int nv = ns + (MX ? 1 : 0);
  if (t < nv) {
    double v;
    if (MX && t == ns) {
      long long m = __double_as_longlong(sm.red[0][t]);
#pragma unroll
      for (int w2 = 1; w2 < kGW; ++w2) m = max(m, __double_as_longlong(sm.red[w2][t]));
      v = __longlong_as_double(m);
    } else {
      v = (sm.red[0][t] + sm.red[1][t]) + (sm.red[2][t] + sm.red[3][t]);
    }
    sm.part[par][t] = v;
  }
  cl.sync();
  // 16 lanes per value, lane r reading rank r's partial
  if (wid < (nv + 1) / 2) {
    const int i = t >> 4, r = t & 15;
    const unsigned hm = (lane < 16) ? 0x0000ffffu : 0xffff0000u;   // this lane's 16-lane group
    const int Q = (int)cl.num_blocks();
    const double* src = cl.map_shared_rank(&sm.part[par][0], r < Q ? r : 0);
    const bool live = i < nv && r < Q;
    const double pv = live ? src[i] : 0.0;
    if (MX && i == ns) {
      long long m = __double_as_longlong(pv);
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(hm, m, o));
      if (r == 0) sm.sums[i] = __longlong_as_double(m);
    } else {
      double a = pv;
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) a += __shfl_xor_sync(hm, a, o);
      if (r == 0 && i < nv) sm.sums[i] = a;
    }
  }
  par ^= 1;
  __syncthreads();
}

// Approximate binary32 reciprocal (rcp.approx.ftz: within 1 ulp) for the chunk sweeps,
// whose pivots are O(1) and positive.
__device__ __forceinline__ float f_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Tridiagonal coefficients of line k at the slice-local cell jl (halo index):
//   a = -v^2 gl, b = A + v^2 (gl + gu) + v gb, c = -v^2 gu   (LineCoef).
__device__ __forceinline__ void f_coef(const FSmem& sm, int jl, float v, float v2, float& a, float& b, float& c) {
  const float4 q = sm.lc[jl];
  a = -v2 * q.y;
  c = -v2 * q.z;
  b = fmaf(v, q.w, fmaf(v2, q.y + q.z, q.x));
}

// PCR on n <= kFR rows of (ra, rb, rc) with NR right-hand sides (rr; rg, rh) for every
// angle, in place: on return rr (rg, rh) hold the solutions.  Warp w takes the angles w and
// w + kFW with lane = row; the rows are kept scaled to a unit diagonal, so a level takes the
// neighbours' (a, c, r) by shuffles and one reciprocal.  The arrays are padded to 33
// columns, so that a warp's column reads hit 32 banks.  Every thread takes part.
template <int NR>
__device__ __forceinline__ void f_pcr(FSmem& sm, int n) {
  static_assert(2 * kFW == 32, "two angles per warp");
  const int i = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool live = i < n;
  float a[2], c[2], r[2][NR];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = w + h * kFW;
    if (live) {
      const float ib = __frcp_rn(sm.rb[i][k]);
      a[h] = sm.ra[i][k] * ib;
      c[h] = sm.rc[i][k] * ib;
      r[h][0] = sm.rr[i][k] * ib;
      if (NR > 1) r[h][1] = sm.rg[i][k] * ib;
      if (NR > 2) r[h][2] = sm.rh[i][k] * ib;
    } else {
      a[h] = c[h] = 0.0f;
#pragma unroll
      for (int j = 0; j < NR; ++j) r[h][j] = 0.0f;
    }
  }
  for (int st = 1; st < n; st <<= 1) {
    const bool hl = i >= st, hr = i + st < n;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float al = __shfl_up_sync(0xffffffffu, a[h], st), cl = __shfl_up_sync(0xffffffffu, c[h], st);
      float ar = __shfl_down_sync(0xffffffffu, a[h], st), cr = __shfl_down_sync(0xffffffffu, c[h], st);
      float rl[NR], rr[NR];
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        rl[j] = __shfl_up_sync(0xffffffffu, r[h][j], st);
        rr[j] = __shfl_down_sync(0xffffffffu, r[h][j], st);
      }
      // row i - a_i row_{i-st} - c_i row_{i+st} (unit diagonals), then rescaled
      const float k1 = hl ? a[h] : 0.0f, k2 = hr ? c[h] : 0.0f;
      const float nb = 1.0f - k1 * cl - k2 * ar;
      const float ib = __frcp_rn(nb);
      a[h] = -k1 * al * ib;
      c[h] = -k2 * cr * ib;
#pragma unroll
      for (int j = 0; j < NR; ++j) r[h][j] = (r[h][j] - k1 * rl[j] - k2 * rr[j]) * ib;
    }
  }
  if (live) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = w + h * kFW;
      sm.rr[i][k] = r[h][0];
      if (NR > 1) sm.rg[i][k] = r[h][1];
      if (NR > 2) sm.rh[i][k] = r[h][2];
    }
  }
  __syncthreads();
}

// Solve the M line systems (A + G_k) e_k = x_k of the instance for the right-hand sides in
// sm.x (this CTA's slice), in place.  sm.xlr receives e at the neighbouring cells c0 - 1
// and c0 + kFS.  All threads of all CTAs of the cluster take part.
__device__ void f_line_solve(FSmem& sm, cg::cluster_group& cl, const FGeo& G, int& par) {
  const int k = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float v = sm.vk[k], v2 = sm.v2k[k];
  const int row0 = w * kFL;
  // (1) backward elimination of the chunk's interior from its last cell:
  //     x_u = rt_u - at_u x_{u-1} - ct_u x_e, down to u = 1 (the S row's partner)
  float rt = 0.0f, at = 0.0f, ct = 0.0f;
#pragma unroll
  for (int u = kFL - 2; u >= 1; --u) {
    float a, b, c;
    f_coef(sm, row0 + u + 1, v, v2, a, b, c);
    const float r = sm.x[row0 + u][k];
    float den, num, ctv;
    if (u == kFL - 2) {
      den = b;
      num = r;
      ctv = c;
    } else {
      den = fmaf(-c, at, b);
      num = fmaf(-c, rt, r);
      ctv = -c * ct;
    }
    const float inv = f_rcp(den);
    rt = num * inv;
    at = a * inv;
    ct = ctv * inv;
  }
  // (2) forward elimination: x_u = rh_u - ch_u x_{u+1} - ah_u x_s (rh_u kept in sm.x)
  float rhp = 0.0f, chp = 0.0f, ahp = 0.0f;
#pragma unroll
  for (int u = 1; u <= kFL - 2; ++u) {
    float a, b, c;
    f_coef(sm, row0 + u + 1, v, v2, a, b, c);
    const float r = sm.x[row0 + u][k];
    float den, ahv, num;
    if (u == 1) {
      den = b;
      ahv = a;
      num = r;
    } else {
      den = fmaf(-a, chp, b);
      ahv = -a * ahp;
      num = fmaf(-a, rhp, r);
    }
    const float inv = f_rcp(den);
    chp = c * inv;
    ahp = ahv * inv;
    rhp = num * inv;
    sm.x[row0 + u][k] = rhp;
  }
  {
    float as, bs, cs, ae, be, ce;
    f_coef(sm, row0 + 1, v, v2, as, bs, cs);
    f_coef(sm, row0 + kFL, v, v2, ae, be, ce);
    const float rs = sm.x[row0][k], re = sm.x[row0 + kFL - 1][k];
    // S row: a_s x_{s-1} + b_s x_s + c_s x_1, x_1 = rt - at x_s - ct x_e
    sm.ra[2 * w][k] = (w == 0) ? 0.0f : as;
    sm.rb[2 * w][k] = fmaf(-cs, at, bs);
    sm.rc[2 * w][k] = -cs * ct;
    sm.rr[2 * w][k] = fmaf(-cs, rt, rs);
    // E row: a_e x_{e-1} + b_e x_e + c_e x_{e+1}, x_{e-1} = rh - ch x_e - ah x_s
    sm.ra[2 * w + 1][k] = -ae * ahp;
    sm.rb[2 * w + 1][k] = fmaf(-ae, chp, be);
    sm.rc[2 * w + 1][k] = (w == kFW - 1) ? 0.0f : ce;
    sm.rr[2 * w + 1][k] = fmaf(-ae, rhp, re);
    sm.rg[2 * w][k] = (w == 0) ? 1.0f : 0.0f;          // unit spikes of the slice's reduced system
    sm.rg[2 * w + 1][k] = 0.0f;
    sm.rh[2 * w][k] = 0.0f;
    sm.rh[2 * w + 1][k] = (w == kFW - 1) ? 1.0f : 0.0f;
    if (w == 0) sm.coup[par][0][k] = as;               // a at the slice's first cell
    if (w == kFW - 1) sm.coup[par][1][k] = ce;         // c at its last cell
  }
  __syncthreads();
  f_pcr<3>(sm, kFR);
  // the slice's 2x2 Schur complement on (first, last): S = Z^{-1}, Z = [[g0, h0], [g1, h1]]
  if (w == 0) {
    const float z00 = sm.rg[0][k], z0n = sm.rh[0][k], zn0 = sm.rg[kFR - 1][k], znn = sm.rh[kFR - 1][k];
    const float det = z00 * znn - z0n * zn0;
    const float id = __frcp_rn(det);
    const float S11 = znn * id, S12 = -z0n * id, S21 = -zn0 * id, S22 = z00 * id;
    const float y0 = sm.rr[0][k], y1 = sm.rr[kFR - 1][k];
    sm.ends[par][0][k] = S11;
    sm.ends[par][1][k] = S12;
    sm.ends[par][2][k] = S21;
    sm.ends[par][3][k] = S22;
    sm.endr[par][0][k] = S11 * y0 + S12 * y1;
    sm.endr[par][1][k] = S21 * y0 + S22 * y1;
  }
  cl.sync();
  // interface system of all slices, rows [F_0, L_0, F_1, L_1, ...] per angle:
  //   a_q L_{q-1} + S11 F_q + S12 L_q = r'_F,   S21 F_q + S22 L_q + c_q F_{q+1} = r'_L
  // (built in every CTA from the gathered values into ra..rr; the slice's own y, g, h
  // are kept in rr/rg/rh until then)
  const int Q = G.Q, n2 = 2 * Q;
  float yk[2] = {0.0f, 0.0f}, gk[2] = {0.0f, 0.0f}, hk[2] = {0.0f, 0.0f};
  {
    const int r0 = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int i = r0 + p * kFW;
      yk[p] = sm.rr[i][k];
      gk[p] = sm.rg[i][k];
      hk[p] = sm.rh[i][k];
    }
  }
  __syncthreads();
  {
    // two items (row, angle) per thread, every remote load issued before the stores
    static_assert(2 * kFT >= 2 * kFQ * 32, "interface gather: two items per thread");
    float va[2], vb[2], vc[2], vr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = threadIdx.x + h * kFT;
      const int i = idx >> 5, kk = idx & 31, qq = i >> 1, side = i & 1;
      va[h] = vb[h] = vc[h] = vr[h] = 0.0f;
      if (idx < n2 * 32) {
        const float* e = cl.map_shared_rank(&sm.ends[par][0][0], qq);
        const float* er = cl.map_shared_rank(&sm.endr[par][0][0], qq);
        const float* cp = cl.map_shared_rank(&sm.coup[par][0][0], qq);
        if (side == 0) {
          va[h] = (qq > 0) ? cp[kk] : 0.0f;
          vb[h] = e[0 * 32 + kk];
          vc[h] = e[1 * 32 + kk];
          vr[h] = er[0 * 32 + kk];
        } else {
          va[h] = e[2 * 32 + kk];
          vb[h] = e[3 * 32 + kk];
          vc[h] = (qq < Q - 1) ? cp[32 + kk] : 0.0f;
          vr[h] = er[1 * 32 + kk];
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = threadIdx.x + h * kFT;
      if (idx < n2 * 32) {
        const int i = idx >> 5, kk = idx & 31;
        sm.ra[i][kk] = va[h];
        sm.rb[i][kk] = vb[h];
        sm.rc[i][kk] = vc[h];
        sm.rr[i][kk] = vr[h];
      }
    }
  }
  __syncthreads();
  // this CTA's couplings (read before the interface solve reuses the arrays)
  const float a_first = sm.coup[par][0][k], c_last = sm.coup[par][1][k];
  f_pcr<1>(sm, n2);
  const float Lp = (G.q > 0) ? sm.rr[2 * G.q - 1][k] : 0.0f;
  const float Fn = (G.q < Q - 1) ? sm.rr[2 * G.q + 2][k] : 0.0f;
  __syncthreads();
  if (w == 0) {
    sm.xlr[0][k] = Lp;
    sm.xlr[1][k] = Fn;
  }
  // the slice's reduced solution: y - L_{q-1} a g - F_{q+1} c h
  {
    const int r0 = threadIdx.x >> 5;
    const float la = Lp * a_first, fc = Fn * c_last;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int i = r0 + p * kFW;
      sm.rr[i][k] = yk[p] - la * gk[p] - fc * hk[p];
    }
  }
  par ^= 1;
  __syncthreads();
  // back substitution of the chunk: the forward factors ch, ah (matrix only) recomputed
  // into registers, then x_u = rh_u - ch_u x_{u+1} - ah_u x_s from the last cell down
  const float xs = sm.rr[2 * w][k], xe = sm.rr[2 * w + 1][k];
  float ch[kFL - 2], ah[kFL - 2];
  {
    float chv = 0.0f, ahv = 0.0f;
#pragma unroll
    for (int u = 1; u <= kFL - 2; ++u) {
      float a, b, c;
      f_coef(sm, row0 + u + 1, v, v2, a, b, c);
      const float den = (u == 1) ? b : fmaf(-a, chv, b);
      const float inv = f_rcp(den);
      ahv = ((u == 1) ? a : -a * ahv) * inv;
      chv = c * inv;
      ch[u - 1] = chv;
      ah[u - 1] = ahv;
    }
  }
  sm.x[row0][k] = xs;
  sm.x[row0 + kFL - 1][k] = xe;
  float xn = xe;
#pragma unroll
  for (int u = kFL - 2; u >= 1; --u) {
    xn = fmaf(-ch[u - 1], xn, fmaf(-ah[u - 1], xs, sm.x[row0 + u][k]));
    sm.x[row0 + u][k] = xn;
  }
  __syncthreads();
}

// Load the slice's per-cell binary32 arrays (with halos) and the angle constants.
__device__ void f_load_cells(FSmem& sm, const Dev& D, const Inst& I, const FGeo& G) {
  for (int t = threadIdx.x; t < kFS + 2; t += kFT) {
    const int64_t j = G.c0 + t - 1;
    const bool in = j >= 0 && j < G.N;
    const int64_t g = G.co + j;
    sm.lc[t] = in ? make_float4(D.fc.A[g], D.fc.gl[g], D.fc.gu[g], D.fc.gb[g]) : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    sm.od[t] = in ? D.fc.od[g] : 0.0f;
    sm.dlx[t] = in ? D.fc.dlx[g] : 0.0f;
    sm.kcd[t] = in ? D.fc.kcd[g] : 0.0f;
    sm.kdx[t] = in ? D.fc.kdx[g] : 0.0f;
  }
  if (threadIdx.x < 32) {
    const int k = threadIdx.x;
    const bool ka = k < G.M;
    const double v = ka ? D.v[I.ang_off + k] : 0.0, w = ka ? D.w[I.ang_off + k] : 0.0;
    sm.vk[k] = (float)v;
    sm.v2k[k] = (float)(v * v);
    sm.wvk[k] = (float)(w * v);
    sm.wvkl[k] = (float)(w * v - (double)(float)(w * v));
    sm.vkd[k] = v;
    sm.wvkd[k] = w * v;
    // inflow wall rows of this slice (per angle, fixed for the solve): 1/b of the wall
    // row, its neighbour coefficient over b, and o^n at the node next to the wall
    if (I.bc == GRTE_BC_INFLOW) {
      for (int side = 0; side < 2; ++side) {
        const int64_t jw = side == 0 ? 0 : G.N - 1;
        if (!(jw >= G.c0 && jw < G.c0 + kFS)) continue;
        const int64_t g = G.co + jw, ni = side == 0 ? 1 : G.N - 1;
        const double v2 = v * v;
        const double bw = D.cf.A[g] + v2 * (D.cf.gl[g] + D.cf.gu[g]) + v * D.cf.gb[g];
        sm.wib[side][k] = ka ? 1.0 / bw : 0.0;
        sm.wgn[side][k] = ka ? v2 * (side == 0 ? D.cf.gu[g] : D.cf.gl[g]) / bw : 0.0;
        const float* Ok = (const float*)D.O + I.nelem_off + (int64_t)k * (G.N + 1);
        sm.won[side][k] = ka ? (double)(D.fc.od[G.co + ni] * Ok[ni]) : 0.0;
        if (k == 0) sm.wdl[side] = D.cf.dlx[G.co + ni];
      }
    }
  }
  __syncthreads();
}

// Per-cell parts of a pass at the per-cell vector xg (instance-local, global, complete):
//   P1 = -alpha x (+ (s a c + kappa a c/(c dt)) U^n on data passes), P2 = Gint x, P3 = gb x,
//   fl = Frho = wv2 [fR (x_j - x_{j+1}) + fL (x_j - x_{j-1})] + wv gbx x_j
//        (data passes: minus 2/eps sum_k w_k v_k b at the inflow walls).
// X: the per-cell vector.  Data passes: the iterate, an instance-local global vector.
// Krylov passes: a direction, slice-local in shared memory, whose values at the two
// neighbouring cells are read from the neighbouring CTAs (distributed shared memory).
struct FVec {
  const double* p;   // FULL: instance-local global; HOM: slice-local shared
  double left, right;   // HOM: the values at c0 - 1 and c0 + kFS
};

template <bool FULL>
__device__ __forceinline__ double f_x(const FVec& X, const FGeo& G, int64_t j) {
  if (FULL) return X.p[j];
  const int64_t t = j - G.c0;
  return t < 0 ? X.left : (t >= kFS ? X.right : X.p[t]);
}

// f_div: a / b in binary64 from a binary32 reciprocal and one residual correction (q_div)
__device__ __forceinline__ double f_div(double a, double b) { return q_div(a, b); }

// sqrt(q) and 1/sqrt(q) in binary64 for q >= 0 without the binary64 square root and divide
// sequences: y = 1/sqrt(q) from a binary32 seed refined by two Newton-Raphson steps
// y <- y (3 - q y^2)/2 (quadratic convergence: ~2^-22 -> ~2^-44 -> binary64 rounding), and
// sqrt(q) = q y.  Outside the seed's range (and for 0, inf, NaN) the plain operations.
__device__ __forceinline__ void f_sqrt_pair(double q, double& r, double& ir) {
  if (!(q > 1e-36 && q < 1e36)) {
    r = sqrt(q);
    ir = 1.0 / r;
    return;
  }
  double y = (double)rsqrtf((float)q);
  y = y * fma(-0.5 * q, y * y, 1.5);
  y = y * fma(-0.5 * q, y * y, 1.5);
  r = q * y;
  ir = y;
}

// The multiplier of the correction's flux (sigma_0/T^3, Eq. dis-cor-marshak1 with the
// predicted data) in cell i for the iterate rho = X:
//   V* = max(U*, 0)^{3/4},  U* = (U^n + gam rho)/(1 + gam a c)  (Eq. dis-pre3);
// y = u^{3/4} from binary32, then one Newton step on y^4 = u^3 in binary64.
__device__ __forceinline__ double f_vstar(const Dev& D, const Inst& I, const FGeo& G, const FVec& X, int64_t i) {
  const int64_t g = G.co + i;
  const double gam = D.cf.gam[g];
  const double u = fmax(f_div(D.U[g] + gam * f_x<true>(X, G, i), 1.0 + gam * (I.a * I.c)), 0.0);
  if (u == 0.0) return 0.0;
  if (I.p != 3.0) return pow(u, 0.25 * I.p);          // sigma_0/T^p, p != 3: V* = u^{p/4}
  // outside the range where u^{3/2} and 4 y^3 = 4 u^{9/4} are normal binary32 numbers
  if (!(u > 1e-16 && u < 1e16)) return pow(u, 0.75);
  const float uf = (float)u;
  const double y = (double)sqrtf(uf * sqrtf(uf));
  const double y2 = y * y, u2 = u * u;
  return y - (y2 * y2 - u2 * u) * (double)__frcp_rn((float)(4.0 * y2 * y));
}

// Node coefficient of the correction's flux at node i from the multipliers of its two
// cells: d*_i = V*_i/(V*_i eps^2/(c dt) + sig_i), V*_i the mean of the two cells, sig_i
// their harmonic mean; 0 at the wall nodes and past the grid.
__device__ __forceinline__ double f_dnode(const Dev& D, const Inst& I, const FGeo& G, int64_t i, double vl,
                                          double vr) {
  if (i < 1 || i > G.N - 1) return 0.0;
  const double sl = D.sig[G.co + i - 1], sr = D.sig[G.co + i];
  const double sn = (sl > 0.0 && sr > 0.0) ? f_div(2.0 * sl * sr, sl + sr) : 0.0;
  const double vn = 0.5 * (vl + vr);
  const double den = vn * I.e2cdt + sn;
  return den > 0.0 ? f_div(vn, den) : 0.0;
}

template <bool FULL>
__device__ void f_cellparts(FSmem& sm, const Dev& D, const Inst& I, const FGeo& G, const FVec& X) {
  const int t = threadIdx.x;
  const int64_t j = G.c0 + t;
  const bool wallc = I.bc == GRTE_BC_INFLOW && (j == 0 || j == G.N - 1);
  if (!FULL && j < G.N && !wallc) {
    // a Krylov direction's parts are used in binary32: formed in binary32 (the binary64
    // pipe is the scarce one) from the direction and the binary32 coefficient copies
    const int64_t g = G.co + j, N = G.N;
    const float xj = (float)f_x<FULL>(X, G, j), xl = j > 0 ? (float)f_x<FULL>(X, G, j - 1) : 0.0f,
                xr = j < N - 1 ? (float)f_x<FULL>(X, G, j + 1) : 0.0f;
    const float4 q = sm.lc[t + 1];
    const float gl = q.y, gu = q.z;
    sm.P1[t] = -D.fc.alpha[g] * xj;
    sm.P2[t] = gl * (xj - xl) + gu * (xj - xr);
    sm.P3[t] = q.w * xj;
    sm.fl[t] = (double)((float)I.wv2 * (D.fc.fR[g] * (xj - xr) + D.fc.fL[g] * (xj - xl)) +
                        (float)I.wv * D.fc.gbx[g] * xj);
    return;
  }
  if (j < G.N) {
    const int64_t g = G.co + j, N = G.N;
    const double xj = f_x<FULL>(X, G, j), xl = j > 0 ? f_x<FULL>(X, G, j - 1) : 0.0,
                 xr = j < N - 1 ? f_x<FULL>(X, G, j + 1) : 0.0;
    double p1 = -D.cf.alpha[g] * xj;
    if (FULL) p1 += (D.cf.sac[g] + D.cf.kcd[g] * I.a * I.c) * D.U[g];
    const double p2 = D.cf.gl[g] * (xj - xl) + D.cf.gu[g] * (xj - xr);
    const double p3 = D.cf.gb[g] * xj;
    double fr = I.wv2 * (D.cf.fR[g] * (xj - xr) + D.cf.fL[g] * (xj - xl)) + I.wv * D.cf.gbx[g] * xj;
    if (FULL && I.bc == GRTE_BC_INFLOW) {
      if (j == 0) fr -= I.two_eps * I.bLflux;
      if (j == N - 1) fr -= I.two_eps * I.bRflux;
    }
    sm.P1[t] = (float)p1;
    sm.P2[t] = (float)p2;
    sm.P3[t] = (float)p3;
    // (here: data passes, and the inflow wall cells of Krylov passes, whose rho part
    // cancels against the e/o wall sum to O(eps), both carrying the factor 2/eps)
    sm.fl[t] = fr;
  } else {
    sm.P1[t] = 0.0f;
    sm.P2[t] = 0.0f;
    sm.P3[t] = 0.0f;
    sm.fl[t] = 0.0;
  }
}

// hi + lo += (wh + wl) d in binary32 pairs: the product's rounding error from an fma, the
// weight's low part, and the addition's error (Knuth's two-sum) carried in lo; the pair holds
// the sum to about 2^-44 of the terms' magnitudes without the binary64 pipe.
__device__ __forceinline__ void f_acc2(float& hi, float& lo, float wh, float wl, float d) {
  const float p = __fmul_rn(wh, d);
  const float e = fmaf(wl, d, fmaf(wh, d, -p));
  const float sN = __fadd_rn(hi, p);
  const float bb = __fsub_rn(sN, hi);
  lo += (__fsub_rn(hi, __fsub_rn(sN, bb)) + __fsub_rn(p, bb)) + e;
  hi = sN;
}

// Data part of a data pass: the right-hand side terms kappa/(c dt) Eh^n - kappa v/dx (o_{j+1} - o_j)
// (o_i = d_i eps^2 O^n_i/(c dt) at interior nodes, 0 at the walls) into sm.x, and the data
// part of the flux sum_k w_k v_k (o_{j+1,k} - o_{j,k}) into sm.fdat (not at inflow wall cells).
// The data do not change within a step: the first data pass of a solve (stage = true) reads
// the angle-major state (warp w loads the 32 cells of its chunk for 8 angles at a time,
// coalesced rows, written transposed), keeps fdat in shared memory and the transposed terms
// in D.fdata; the later data passes read them back with lane = angle (coalesced).
__device__ void f_stage_data(FSmem& sm, const Dev& D, const Inst& I, const FGeo& G, bool stage) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* fd = D.fdata + I.fd_off + (G.c0 + w * kFL) * 32;
  if (!stage) {
#pragma unroll 8
    for (int u = 0; u < kFL; ++u) sm.x[w * kFL + u][lane] = fd[u * 32 + lane];
    __syncwarp();
    return;
  }
  const int64_t N = G.N, j = G.c0 + w * kFL + lane;
  const int jl = w * kFL + lane + 1;
  const float* Eh = (const float*)D.Eh + I.elem_off;
  const float* On = (const float*)D.O + I.nelem_off;
  const bool real = j < N;
  const bool wallc = I.bc == GRTE_BC_INFLOW && (j == 0 || j == N - 1);
  const float kcd = sm.kcd[jl], kdx = sm.kdx[jl], odj = sm.od[jl], odr = sm.od[jl + 1];
  const bool nj = j >= 1 && j <= N - 1, nr = j + 1 >= 1 && j + 1 <= N - 1;
  float fh = 0.0f, fo = 0.0f, oh = 0.0f, oo = 0.0f, rh = 0.0f, ro = 0.0f;   // (hi, lo) sums
  constexpr int B = 8;
  for (int k0 = 0; k0 < 32; k0 += B) {
    float e[B], oj[B], orr[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int kk = k0 + q;
      const bool ka = kk < G.M;
      const float* Ek = Eh + (int64_t)kk * N;
      const float* Ok = On + (int64_t)kk * (N + 1);
      e[q] = (ka && real) ? Ek[j] : 0.0f;
      oj[q] = (ka && nj) ? Ok[j] : 0.0f;
      orr[q] = (ka && lane == 31 && nr) ? Ok[j + 1] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < B; ++q) {
      const int kk = k0 + q;
      const float o0 = odj * oj[q];
      float o1 = __shfl_down_sync(0xffffffffu, o0, 1);
      if (lane == 31) o1 = odr * orr[q];
      const float Dj = o1 - o0;
      const float d = real ? fmaf(kcd, e[q], -kdx * sm.vk[kk] * Dj) : 0.0f;
      sm.x[w * kFL + lane][kk] = d;
      const float wh = sm.wvk[kk], wl = sm.wvkl[kk];
      if (real && !wallc) f_acc2(fh, fo, wh, wl, Dj);
      f_acc2(oh, oo, wh, wl, oj[q]);
      if (lane == 31) f_acc2(rh, ro, wh, wl, orr[q]);
    }
  }
  sm.fdat[w * kFL + lane] = (double)fh + (double)fo;
  sm.Om[w * kFL + lane] = (double)oh + (double)oo;   // node c0 + t (interior nodes; 0 elsewhere)
  if (w == kFW - 1 && lane == 31) sm.Om[kFS] = (double)rh + (double)ro;
  __syncwarp();
#pragma unroll 8
  for (int u = 0; u < kFL; ++u) fd[u * 32 + lane] = sm.x[w * kFL + u][lane];
  __syncwarp();
}

// Right-hand side of the inflow wall row j (0 or N-1) for angle k in binary64:
//   P1 - v^2 P2 + kappa v (2/eps)(b - x)/dx  [+ kappa/(c dt) Eh^n - kappa v o/dx on data passes,
//   o = 2 o_1 (left) or -2 o_{N-1} (right)] (the O(eps) difference is formed in double).
template <bool FULL>
__device__ double f_wall_rhs(const Dev& D, const Inst& I, const FGeo& G, const FVec& X, int64_t j, int k) {
  const int64_t N = G.N, g = G.co + j;
  const double v = D.v[I.ang_off + k], v2 = v * v;
  const double xj = f_x<FULL>(X, G, j), xl = j > 0 ? f_x<FULL>(X, G, j - 1) : 0.0,
               xr = j < N - 1 ? f_x<FULL>(X, G, j + 1) : 0.0;
  double p1 = -D.cf.alpha[g] * xj;
  if (FULL) p1 += (D.cf.sac[g] + D.cf.kcd[g] * I.a * I.c) * D.U[g];
  const double p2 = D.cf.gl[g] * (xj - xl) + D.cf.gu[g] * (xj - xr);
  const double b = FULL ? ((j == 0) ? D.bL[I.ang_off + k] : D.bR[I.ang_off + k]) : 0.0;
  double r = p1 - v2 * p2 + D.cf.kdx[g] * v * I.two_eps * (b - xj);
  if (FULL) {
    const float* Ok = (const float*)D.O + I.nelem_off + (int64_t)k * (N + 1);
    const float* Ek = (const float*)D.Eh + I.elem_off + (int64_t)k * N;
    const int64_t ni = (j == 0) ? 1 : N - 1;
    const double on = (double)(D.fc.od[G.co + ni] * Ok[ni]);
    const double o = (j == 0) ? 2.0 * on : -2.0 * on;
    r += D.cf.kcd[g] * (double)Ek[j] - D.cf.kdx[g] * v * o;
  }
  return r;
}

// One line pass at the per-cell vector xg (FULL: the iterate, with the data terms; HOM: a
// Krylov direction).  On return sm.fl[t] holds F_j for the slice's cells (double; HOM:
// the binary32 sum widened).  xg must be complete in global memory (a cluster barrier
// precedes the call inside).
template <bool FULL>
__device__ void f_pass(FSmem& sm, cg::cluster_group& cl, const Dev& D, const Inst& I, const FGeo& G,
                       const double* xg, int& par, bool stage = false) {
  cl.sync();   // xg complete on every slice (halo reads)
  FVec X{xg, 0.0, 0.0};
  if (!FULL) {
    // the direction's values next to the slice, from the neighbouring CTAs' shared memory
    if (G.q > 0) X.left = cl.map_shared_rank(const_cast<double*>(xg), G.q - 1)[kFS - 1];
    if (G.q < G.Q - 1) X.right = cl.map_shared_rank(const_cast<double*>(xg), G.q + 1)[0];
  }
  const int k = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t N = G.N;
  f_cellparts<FULL>(sm, D, I, G, X);
  if (FULL) f_stage_data(sm, D, I, G, stage);
  __syncthreads();
  const bool inflow = I.bc == GRTE_BC_INFLOW;
  const float v = sm.vk[k], v2 = sm.v2k[k];
  // right-hand sides r = P1 - v^2 P2 - v P3 (+ data) of the chunk
#pragma unroll 4
  for (int u = 0; u < kFL; ++u) {
    const int t = w * kFL + u;
    float r = fmaf(-v, sm.P3[t], fmaf(-v2, sm.P2[t], sm.P1[t]));
    if (FULL) r += sm.x[t][k];
    sm.x[t][k] = (k < G.M) ? r : 0.0f;
  }
  // inflow wall rows in double
  if (inflow && k < G.M) {
    for (int side = 0; side < 2; ++side) {
      const int64_t jw = side == 0 ? 0 : N - 1;
      const int64_t tl = jw - G.c0;
      if (tl >= 0 && tl < kFS && (int)(tl / kFL) == w) {
        const double r = f_wall_rhs<FULL>(D, I, G, X, jw, k);
        sm.wall[side][k] = r;
        sm.x[tl][k] = (float)r;
      }
    }
  }
  __syncthreads();
  f_line_solve(sm, cl, G, par);
  // inflow walls: e re-solved in double from the neighbour; e/o wall flux in double
  if (inflow && w == 0) {
    for (int side = 0; side < 2; ++side) {
      const int64_t jw = side == 0 ? 0 : N - 1;
      const int64_t tl = jw - G.c0;
      if (!(tl >= 0 && tl < kFS)) continue;
      double sw = 0.0;
      if (k < G.M) {
        const double vd = sm.vkd[k];
        // neighbour value (float solution) and the node term next to the wall
        const int64_t jn = side == 0 ? 1 : N - 2;
        const int64_t tn = jn - G.c0;
        const double en = (tn >= 0) ? (double)sm.x[tn][k] : (double)sm.xlr[0][k];
        const double ew = sm.wall[side][k] * sm.wib[side][k] + sm.wgn[side][k] * en;
        const double on = FULL ? sm.won[side][k] : 0.0;
        const double dl = sm.wdl[side];
        if (side == 0) {
          const double O1 = on - dl * vd * (en - ew);
          sw = sm.wvkd[k] * (2.0 * O1 + I.two_eps * ew);
        } else {
          const double ON1 = on - dl * vd * (ew - en);
          sw = sm.wvkd[k] * (I.two_eps * ew - 2.0 * ON1);
        }
      }
      for (int o = 16; o > 0; o >>= 1) sw += __shfl_xor_sync(0xffffffffu, sw, o);
      if (k == 0) sm.fl[tl] += sw;
    }
  }
  // e/o flux of every interior cell without the data part, summed over the angles by the
  // cell's own thread (reads its row and the two neighbouring rows of sm.x):
  //   sum_k -w_k v_k^2 [dlx_{j+1} (e_{j+1} - e_j) - dlx_j (e_j - e_{j-1})]  (nodes 1..N-1)
  {
    const int t = threadIdx.x;
    const int64_t j = G.c0 + t;
    if (j < N && !(inflow && (j == 0 || j == N - 1))) {
      const float dR = (j + 1 <= N - 1) ? sm.dlx[t + 2] : 0.0f;
      const float dL = (j >= 1) ? sm.dlx[t + 1] : 0.0f;
      const float* xl = (t > 0) ? &sm.x[t - 1][0] : &sm.xlr[0][0];
      const float* xr = (t < kFS - 1) ? &sm.x[t + 1][0] : &sm.xlr[1][0];
      if (FULL) {
        // compensated binary32 sum (Knuth's two-sum): the rounding error of every addition
        // is carried in lo, so hi + lo holds the sum to about 2^-48 relative
        float hi = 0.0f, lo = 0.0f;
        for (int kk = 0; kk < G.M; ++kk) {
          const float ej = sm.x[t][kk];
          const float wv2k = -sm.wvk[kk] * sm.vk[kk];
          const float a = wv2k * (dR * (xr[kk] - ej) - dL * (ej - xl[kk]));
          const float sN = hi + a;
          const float bb = sN - hi;
          lo += (hi - (sN - bb)) + (a - bb);
          hi = sN;
        }
        sm.fl[t] += sm.fdat[t] + ((double)hi + (double)lo);
      } else {
        float acc = (float)sm.fl[t];
        for (int kk = 0; kk < G.M; ++kk) {
          const float ej = sm.x[t][kk];
          acc += -sm.wvk[kk] * sm.vk[kk] * (dR * (xr[kk] - ej) - dL * (ej - xl[kk]));
        }
        sm.fl[t] = (double)acc;
      }
    }
  }
  __syncthreads();
}

// Right-hand side of row il (and row ir) of a 64-row system held two rows per lane of
// warp 0 (rows 2 lane, 2 lane + 1 in v0, v1).
__device__ __forceinline__ double f_row(double v0, double v1, int i) {
  const int src = (i < 0 ? 0 : (i > 63 ? 63 : i));
  const double a = __shfl_sync(0xffffffffu, v0, src >> 1), b = __shfl_sync(0xffffffffu, v1, src >> 1);
  return (src & 1) ? b : a;
}

// Cell slot (within a lane's 16-cell chunk) of row i of the preconditioner's level-B
// system: the end cells 0, 3, 4, 7, ..., 15 of the four sub-chunks.
__device__ __forceinline__ int f_pcb(int i) { return 4 * (i >> 1) + 3 * (i & 1); }

// The single-effective-angle Schur operator of the preconditioner (binary64):
//   P = alpha + Gbar (A + Gbar)^{-1} beta, applied as  u = (A + (A/alpha) Gbar)^{-1} (beta/alpha) r,
//   z = (r - Gbar u)/alpha,  Gbar = sum_k w_k G_k, beta = A - alpha.
// The tridiagonal matrix T = A + (A/alpha) Gbar is the same for every application of a solve:
// f_prec_factor eliminates it once and f_prec then solves with the stored factors, without
// divisions.  A slice's 512 cells are 32 chunks of 16 (one per lane), each of four 4-cell
// sub-chunks.  Level A (warps 0..3, one per sub-partition: the binary64 pipe is the scarce
// resource) eliminates each sub-chunk's two interior cells, leaving an 8-row system per
// chunk; level B (warp 0) eliminates its six interior rows, leaving the 64 chunk-end rows,
// solved by PCR with two unit spikes; then the slice's 2x2 Schur complement and, in every
// CTA, the 2Q-row interface system of the cluster (PCR multipliers stored per level).
__device__ void f_prec_coef(const Dev& D, const Inst& I, const FGeo& G, int64_t j, double& a, double& b,
                            double& c) {
  if (j >= G.N) { a = 0.0; b = 1.0; c = 0.0; return; }
  const int64_t g = G.co + j;
  const double f = D.cf.A[g] * D.cf.ralpha[g];
  const double l = D.cf.gl[g], u = D.cf.gu[g];
  a = j > 0 ? -f * I.wv2 * l : 0.0;
  c = j < G.N - 1 ? -f * I.wv2 * u : 0.0;
  b = D.cf.A[g] + f * (I.wv2 * (l + u) + I.wv * D.cf.gb[g]);
}

__device__ void f_prec_factor(FSmem& sm, cg::cluster_group& cl, const Dev& D, const Inst& I, const FGeo& G,
                              int& par) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool w0 = threadIdx.x < 32;
  // level A (warps 0..3, one per sub-partition): sub-chunk w (cells 4w..4w+3) of lane l's
  // 16-cell chunk; its two interior cells eliminated, its end rows become rows 2w, 2w+1 of
  // the chunk's 8-row level-B system, kept as (a, b, c) in the free reduced-system arrays
  double* const lb = reinterpret_cast<double*>(&sm.ra[0][0]);   // [3][8][32]
  if (w < kPW) {
    const int u0 = 4 * w;
    const int64_t s = G.c0 + lane * kFPL + u0;
    double a0, b0, c0, a1, b1, c1, a2, b2, c2, a3, b3, c3;
    f_prec_coef(D, I, G, s, a0, b0, c0);
    f_prec_coef(D, I, G, s + 1, a1, b1, c1);
    f_prec_coef(D, I, G, s + 2, a2, b2, c2);
    f_prec_coef(D, I, G, s + 3, a3, b3, c3);
    const double i1 = 1.0 / b1;
    const double ah1 = a1 * i1, ch1 = c1 * i1;
    const double i2 = 1.0 / (b2 - a2 * ch1);
    const double ah2 = -a2 * ah1 * i2, ch2 = c2 * i2;
    sm.pinv[u0 + 1][lane] = i1;
    sm.pa[u0 + 1][lane] = a1;
    sm.pch[u0 + 1][lane] = ch1;
    sm.pah[u0 + 1][lane] = ah1;
    sm.pinv[u0 + 2][lane] = i2;
    sm.pa[u0 + 2][lane] = a2;
    sm.pch[u0 + 2][lane] = ch2;
    sm.pah[u0 + 2][lane] = ah2;
    sm.pc0[w][lane] = c0;
    sm.pa3[w][lane] = a3;
    // x_1 = rc - cc x_e - ac x_s
    const double cc = -ch1 * ch2, ac = ah1 - ch1 * ah2;
    lb[(0 * 8 + 2 * w) * 32 + lane] = a0;
    lb[(1 * 8 + 2 * w) * 32 + lane] = b0 - c0 * ac;
    lb[(2 * 8 + 2 * w) * 32 + lane] = -c0 * cc;
    lb[(0 * 8 + 2 * w + 1) * 32 + lane] = -a3 * ah2;
    lb[(1 * 8 + 2 * w + 1) * 32 + lane] = b3 - a3 * ch2;
    lb[(2 * 8 + 2 * w + 1) * 32 + lane] = c3;
  }
  __syncthreads();
  if (w0) {
    // level B (warp 0): the 8 rows' interior (rows 1..6, cells f_pcb(1..6)) eliminated;
    // factors stored at those cells' slots
    double a[8], b[8], c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      a[i] = lb[(0 * 8 + i) * 32 + lane];
      b[i] = lb[(1 * 8 + i) * 32 + lane];
      c[i] = lb[(2 * 8 + i) * 32 + lane];
    }
    double chv[8], ahv[8];
    double chp = 0.0, ahp = 0.0;
#pragma unroll
    for (int i = 1; i <= 6; ++i) {
      const double den = (i == 1) ? b[i] : b[i] - a[i] * chp;
      const double inv = 1.0 / den;
      ahp = ((i == 1) ? a[i] : -a[i] * ahp) * inv;
      chp = c[i] * inv;
      const int u = f_pcb(i);
      sm.pinv[u][lane] = inv;
      sm.pa[u][lane] = a[i];
      sm.pch[u][lane] = chp;
      sm.pah[u][lane] = ahp;
      chv[i] = chp;
      ahv[i] = ahp;
    }
    double cc = chv[6], ac = ahv[6];
#pragma unroll
    for (int i = 5; i >= 1; --i) {
      cc = -chv[i] * cc;
      ac = ahv[i] - chv[i] * ac;
    }
    const double as = a[0], bs = b[0], cs = c[0], ae = a[7], be = b[7], ce = c[7];
    sm.pcs[lane] = cs;
    sm.pae[lane] = ae;
    double ra0 = (lane == 0) ? 0.0 : as, rb0 = bs - cs * ac, rc0 = -cs * cc;
    double ra1 = -ae * ahv[6], rb1 = be - ae * chv[6];
    double rc1 = (lane == 31) ? 0.0 : ce;
    double g0 = (lane == 0) ? 1.0 : 0.0, g1 = 0.0, h0 = 0.0, h1 = (lane == 31) ? 1.0 : 0.0;
    const double af = __shfl_sync(0xffffffffu, as, 0), cl_ = __shfl_sync(0xffffffffu, ce, 31);
    for (int l = 0, st = 1; st < 64; ++l, st <<= 1) {
      double na[2], nb[2], nc[2], ng[2], nh[2];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int i = 2 * lane + p, il = i - st, ir = i + st;
        const bool hl = il >= 0, hr = ir < 64;
        const double Lb = f_row(rb0, rb1, il), La = f_row(ra0, ra1, il), Lc = f_row(rc0, rc1, il);
        const double Lg = f_row(g0, g1, il), Lh = f_row(h0, h1, il);
        const double Rb = f_row(rb0, rb1, ir), Ra = f_row(ra0, ra1, ir), Rc = f_row(rc0, rc1, ir);
        const double Rg = f_row(g0, g1, ir), Rh = f_row(h0, h1, ir);
        const double a = p ? ra1 : ra0, b = p ? rb1 : rb0, c = p ? rc1 : rc0;
        const double k1 = hl ? a / Lb : 0.0, k2 = hr ? c / Rb : 0.0;
        sm.pk1[l][i] = k1;
        sm.pk2[l][i] = k2;
        na[p] = hl ? -La * k1 : 0.0;
        nc[p] = hr ? -Rc * k2 : 0.0;
        nb[p] = b - (hl ? Lc * k1 : 0.0) - (hr ? Ra * k2 : 0.0);
        ng[p] = (p ? g1 : g0) - (hl ? Lg * k1 : 0.0) - (hr ? Rg * k2 : 0.0);
        nh[p] = (p ? h1 : h0) - (hl ? Lh * k1 : 0.0) - (hr ? Rh * k2 : 0.0);
      }
      ra0 = na[0]; ra1 = na[1]; rb0 = nb[0]; rb1 = nb[1]; rc0 = nc[0]; rc1 = nc[1];
      g0 = ng[0]; g1 = ng[1]; h0 = nh[0]; h1 = nh[1];
    }
    const double i0 = 1.0 / rb0, i1 = 1.0 / rb1;
    sm.pib[2 * lane] = i0;
    sm.pib[2 * lane + 1] = i1;
    g0 *= i0; h0 *= i0; g1 *= i1; h1 *= i1;
    sm.pgv[2 * lane] = g0;
    sm.pgv[2 * lane + 1] = g1;
    sm.phv[2 * lane] = h0;
    sm.phv[2 * lane + 1] = h1;
    // the slice's 2x2 Schur complement on (first, last): S = Z^{-1}, Z = [[g0, h0], [g63, h63]]
    const double z00 = __shfl_sync(0xffffffffu, g0, 0), z0n = __shfl_sync(0xffffffffu, h0, 0);
    const double zn0 = __shfl_sync(0xffffffffu, g1, 31), znn = __shfl_sync(0xffffffffu, h1, 31);
    if (lane == 0) {
      const double id = 1.0 / (z00 * znn - z0n * zn0);
      sm.pS[0] = znn * id;
      sm.pS[1] = -z0n * id;
      sm.pS[2] = -zn0 * id;
      sm.pS[3] = z00 * id;
      sm.paf = af;
      sm.pcl = cl_;
      for (int q = 0; q < 4; ++q) sm.pe[par][q] = sm.pS[q];
      sm.pcoup[par][0] = af;
      sm.pcoup[par][1] = cl_;
    }
  }
  cl.sync();
  if (w0) {
    // interface rows [F_0, L_0, F_1, L_1, ...]: a_q L_{q-1} + S11 F_q + S12 L_q (F rows),
    // S21 F_q + S22 L_q + c_q F_{q+1} (L rows); PCR multipliers stored per level
    const int Q = G.Q, n2 = 2 * Q;
    double ia = 0.0, ib = 1.0, ic = 0.0;
    if (lane < n2) {
      const int qq = lane >> 1;
      const double* pe = cl.map_shared_rank(&sm.pe[par][0], qq);
      const double* pc = cl.map_shared_rank(&sm.pcoup[par][0], qq);
      if ((lane & 1) == 0) {
        ia = qq > 0 ? pc[0] : 0.0;
        ib = pe[0];
        ic = pe[1];
      } else {
        ia = pe[2];
        ib = pe[3];
        ic = qq < Q - 1 ? pc[1] : 0.0;
      }
    }
    for (int l = 0, st = 1; st < n2; ++l, st <<= 1) {
      const int il = lane - st, irr = lane + st;
      const int sl = il >= 0 ? il : 0, sr = irr < n2 ? irr : 0;
      const double Lb = __shfl_sync(0xffffffffu, ib, sl), La = __shfl_sync(0xffffffffu, ia, sl);
      const double Lc = __shfl_sync(0xffffffffu, ic, sl);
      const double Rb = __shfl_sync(0xffffffffu, ib, sr), Ra = __shfl_sync(0xffffffffu, ia, sr);
      const double Rc = __shfl_sync(0xffffffffu, ic, sr);
      const bool hl = il >= 0, hr = irr < n2;
      const double k1 = hl ? ia / Lb : 0.0, k2 = hr ? ic / Rb : 0.0;
      if (lane < n2) {
        sm.ik1[l][lane] = k1;
        sm.ik2[l][lane] = k2;
        const double na = hl ? -La * k1 : 0.0, nc = hr ? -Rc * k2 : 0.0;
        const double nb = ib - (hl ? Lc * k1 : 0.0) - (hr ? Ra * k2 : 0.0);
        ia = na;
        ib = nb;
        ic = nc;
      }
    }
    sm.iib[lane] = (lane < n2) ? 1.0 / ib : 0.0;
  }
  par ^= 1;
  __syncthreads();
}

// z = P^{-1} rin on the slice with the factors of f_prec_factor (binary64).  rin and z:
// slice-local vectors in shared memory (cell c0 + t at index t).
__device__ void f_prec(FSmem& sm, cg::cluster_group& cl, const Dev& D, const Inst& I, const FGeo& G,
                       const double* rin, double* z, int& par) {
  const int64_t N = G.N, co = G.co;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool w0 = threadIdx.x < 32;
  double y0 = 0.0, y1 = 0.0;
  // level A (warps 0..3): the sub-chunk's scaled right-hand side, its forward sweep (rh at
  // the interior slots) and its two level-B right-hand sides (at the end slots)
  if (w < kPW) {
    const int u0 = 4 * w, tl = lane * kFPL + u0;
    const int64_t s = G.c0 + tl;
    double r[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) r[v] = (s + v < N) ? D.cf.ratio[co + s + v] * rin[tl + v] : 0.0;
    const double rh1 = r[1] * sm.pinv[u0 + 1][lane];
    const double rh2 = (r[2] - sm.pa[u0 + 2][lane] * rh1) * sm.pinv[u0 + 2][lane];
    const double rc = rh1 - sm.pch[u0 + 1][lane] * rh2;
    sm.pxr[u0][lane] = r[0] - sm.pc0[w][lane] * rc;
    sm.pxr[u0 + 1][lane] = rh1;
    sm.pxr[u0 + 2][lane] = rh2;
    sm.pxr[u0 + 3][lane] = r[3] - sm.pa3[w][lane] * rh2;
  }
  __syncthreads();
  if (w0) {
    // level B (warp 0): forward sweep of the 8 rows, then the chunk's two reduced rows
    double rb[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) rb[i] = sm.pxr[f_pcb(i)][lane];
    double rhv[8];
    double rh = 0.0;
#pragma unroll
    for (int i = 1; i <= 6; ++i) {
      const int u = f_pcb(i);
      rh = (i == 1 ? rb[1] : rb[i] - sm.pa[u][lane] * rh) * sm.pinv[u][lane];
      rhv[i] = rh;
      sm.pxr[u][lane] = rh;
    }
    double rc = rhv[6];
#pragma unroll
    for (int i = 5; i >= 1; --i) rc = rhv[i] - sm.pch[f_pcb(i)][lane] * rc;
    double r0 = rb[0] - sm.pcs[lane] * rc, r1 = rb[7] - sm.pae[lane] * rhv[6];
    for (int l = 0, st = 1; st < 64; ++l, st <<= 1) {
      double nr[2];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int i = 2 * lane + p;
        const double Lr = f_row(r0, r1, i - st), Rr = f_row(r0, r1, i + st);
        nr[p] = (p ? r1 : r0) - sm.pk1[l][i] * Lr - sm.pk2[l][i] * Rr;
      }
      r0 = nr[0];
      r1 = nr[1];
    }
    y0 = r0 * sm.pib[2 * lane];
    y1 = r1 * sm.pib[2 * lane + 1];
    const double ya = __shfl_sync(0xffffffffu, y0, 0), yb = __shfl_sync(0xffffffffu, y1, 31);
    if (lane == 0) {
      sm.pe[par][4] = sm.pS[0] * ya + sm.pS[1] * yb;
      sm.pe[par][5] = sm.pS[2] * ya + sm.pS[3] * yb;
    }
  }
  cl.sync();   // every slice's reduced right-hand side published
  if (w0) {
    const int Q = G.Q, n2 = 2 * Q;
    double ir = 0.0;
    if (lane < n2) ir = cl.map_shared_rank(&sm.pe[par][0], lane >> 1)[4 + (lane & 1)];
    for (int l = 0, st = 1; st < n2; ++l, st <<= 1) {
      const int il = lane - st, irr = lane + st;
      const double Lr = __shfl_sync(0xffffffffu, ir, il >= 0 ? il : 0);
      const double Rr = __shfl_sync(0xffffffffu, ir, irr < n2 ? irr : 0);
      if (lane < n2) ir = ir - sm.ik1[l][lane] * Lr - sm.ik2[l][lane] * Rr;
    }
    const double X = ir * sm.iib[lane];
    const int sLp = G.q > 0 ? 2 * G.q - 1 : 0, sFn = G.q < Q - 1 ? 2 * G.q + 2 : 0;
    const double XL = __shfl_sync(0xffffffffu, X, sLp), XF = __shfl_sync(0xffffffffu, X, sFn);
    const double Lp = G.q > 0 ? XL : 0.0, Fn = G.q < Q - 1 ? XF : 0.0;
    const double la = Lp * sm.paf, fc = Fn * sm.pcl;
    const double xs = y0 - la * sm.pgv[2 * lane] - fc * sm.phv[2 * lane];
    const double xe = y1 - la * sm.pgv[2 * lane + 1] - fc * sm.phv[2 * lane + 1];
    sm.pu[lane * kFPL] = xs;
    sm.pu[lane * kFPL + kFPL - 1] = xe;
    // level B back substitution (cells 3, 4, 7, ..., 12)
    double xn = xe;
#pragma unroll
    for (int i = 6; i >= 1; --i) {
      const int u = f_pcb(i);
      xn = sm.pxr[u][lane] - sm.pch[u][lane] * xn - sm.pah[u][lane] * xs;
      sm.pu[lane * kFPL + u] = xn;
    }
    if (lane == 0) {
      sm.pxl[0] = Lp;
      sm.pxl[1] = Fn;
    }
  }
  __syncthreads();
  // level A back substitution (warps 0..3): the sub-chunk's two interior cells
  if (w < kPW) {
    const int u0 = 4 * w, tl = lane * kFPL + u0;
    const double xs = sm.pu[tl], xe = sm.pu[tl + 3];
    const double x2 = sm.pxr[u0 + 2][lane] - sm.pch[u0 + 2][lane] * xe - sm.pah[u0 + 2][lane] * xs;
    const double x1 = sm.pxr[u0 + 1][lane] - sm.pch[u0 + 1][lane] * x2 - sm.pah[u0 + 1][lane] * xs;
    sm.pu[tl + 1] = x1;
    sm.pu[tl + 2] = x2;
  }
  par ^= 1;
  __syncthreads();
  // z = (r - Gbar u)/alpha, Gbar u = wv2 [gl (u_j - u_{j-1}) + gu (u_j - u_{j+1})] + wv gb u_j,
  // from the per-cell coefficients zl, zc, zr (cell coefficient kernel)
  {
    const int t = threadIdx.x;
    const int64_t j = G.c0 + t;
    if (j < N) {
      const int64_t g = co + j;
      const double uj = sm.pu[t];
      const double uL = j > 0 ? (t > 0 ? sm.pu[t - 1] : sm.pxl[0]) : 0.0;
      const double uR = j < N - 1 ? (t < kFS - 1 ? sm.pu[t + 1] : sm.pxl[1]) : 0.0;
      z[t] = rin[t] * D.cf.ralpha[g] - D.cf.zc[g] * uj + D.cf.zl[g] * uL + D.cf.zr[g] * uR;
    } else {
      z[t] = 0.0;
    }
  }
  __syncthreads();
}

// The flux the temperature equation of the sigma_0/T^3 correction takes (Eq. dis-cor-marshak1
// with the predicted data; f_vstar, f_dnode), written to D.Fc for the slice's cells that
// are not inflow wall cells (those keep F*, written with it).  Called once, after the
// solve: the last data pass ran at the converged iterate X, and its angular unknowns
// (E* - rho*) are still in sm.x with the neighbours' edge values in sm.xlr.  Node
// coefficients in binary64 (the rho part needs them so); the e/o part as a compensated
// binary32 sum like the prediction's.  V* and d* live in the reduced-system arrays,
// free after the line solves.
__device__ void f_corr_flux(FSmem& sm, const Dev& D, const Inst& I, const FGeo& G, const FVec& X) {
  const int64_t N = G.N;
  const bool inflow = I.bc == GRTE_BC_INFLOW;
  double* const vst = reinterpret_cast<double*>(&sm.ra[0][0]);   // kFS + 2 cell values (ra, rb)
  double* const dsd = reinterpret_cast<double*>(&sm.rc[0][0]);   // kFS + 1 node values (rc, rr)
  const int t = threadIdx.x;
  const int64_t j = G.c0 + t;
  __syncthreads();
  vst[t + 1] = j < N ? f_vstar(D, I, G, X, j) : 0.0;
  if (t == 0) vst[0] = (j > 0 && j <= N) ? f_vstar(D, I, G, X, j - 1) : 0.0;
  if (t == kFS - 1) vst[kFS + 1] = j + 1 < N ? f_vstar(D, I, G, X, j + 1) : 0.0;
  __syncthreads();
  dsd[t] = f_dnode(D, I, G, j, vst[t], vst[t + 1]);
  if (t == kFS - 1) dsd[kFS] = f_dnode(D, I, G, j + 1, vst[kFS], vst[kFS + 1]);
  __syncthreads();
  if (j < N && !(inflow && (j == 0 || j == N - 1))) {
    const double xj = f_x<true>(X, G, j), xl = j > 0 ? f_x<true>(X, G, j - 1) : 0.0,
                 xr = j < N - 1 ? f_x<true>(X, G, j + 1) : 0.0;
    const double dL = dsd[t], dR = dsd[t + 1];
    // rho and data parts
    double fc = I.wv2 * (dR * (xj - xr) + dL * (xj - xl)) * I.rdx + I.e2cdt * (dR * sm.Om[t + 1] - dL * sm.Om[t]);
    // e/o part: sum_k -w_k v_k^2 [d*_{j+1}(e_{j+1} - e_j) - d*_j (e_j - e_{j-1})]/dx
    const float idxf = __frcp_rn((float)I.dx);
    const float dRc = (float)dR * idxf, dLc = (float)dL * idxf;
    const float* xlw = (t > 0) ? &sm.x[t - 1][0] : &sm.xlr[0][0];
    const float* xrw = (t < kFS - 1) ? &sm.x[t + 1][0] : &sm.xlr[1][0];
    float hc = 0.0f, lc = 0.0f;
    for (int kk = 0; kk < G.M; ++kk) {
      const float ej = sm.x[t][kk];
      const float a = -sm.wvk[kk] * sm.vk[kk] * (dRc * (xrw[kk] - ej) - dLc * (ej - xlw[kk]));
      const float sN = hc + a;
      const float bb = sN - hc;
      lc += (hc - (sN - bb)) + (a - bb);
      hc = sN;
    }
    D.Fc[G.co + j] = fc + ((double)hc + (double)lc);
  }
  __syncthreads();
}

// The whole prediction solve of one instance per cluster.  blockIdx.x / Q indexes
// D.finst (the instances of this launch's cluster size).
__global__ void __launch_bounds__(kFT, 1) k_pred_fused(Dev D, const int* __restrict__ finst) {
  extern __shared__ __align__(16) unsigned char fdsm[];
  FSmem& sm = *reinterpret_cast<FSmem*>(fdsm);
  cg::cluster_group cl = cg::this_cluster();
  FGeo G;
  G.Q = (int)cl.num_blocks();
  G.q = (int)cl.block_rank();
  G.ii = finst[blockIdx.x / G.Q];
  const Inst I = D.inst[G.ii];
  G.N = I.N;
  G.M = I.M;
  G.c0 = (int64_t)G.q * kFS;
  G.co = I.cell_off;
  const int ii = G.ii;
  const int64_t N = G.N, co = G.co;
  const int t = threadIdx.x;
  const int64_t j = G.c0 + t;
  const bool real = j < N;
  const int m = D.m;
  double* x = D.gx + co;
  // the slice's Krylov basis V_0..V_m in shared memory after the struct (cell c0 + t at t)
  double* Vs = reinterpret_cast<double*>(fdsm + sizeof(FSmem));
  auto Vi = [&](int i) { return Vs + (int64_t)i * kFS; };
  double* zv = sm.zv;
  int par = 0;
  f_load_cells(sm, D, I, G);
  f_prec_factor(sm, cl, D, I, G, par);
  int cycles = 0, its = 0, stag = 0;
  double beta_prev = 0.0;
  bool first = true;
  int xpar = 0;
  for (;;) {
    // ---- restart: true residual at x, preconditioned, stopping test --------------------
    // the slice's max |x| (x >= 0 bit patterns as integers: order preserving), published
    // before the pass's opening cluster barrier, which also makes it visible to the others
    {
      long long mx = real ? __double_as_longlong(fabs(x[j])) : 0;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((t & 31) == 0) sm.xmw[t >> 5] = mx;
      __syncthreads();
      if (t == 0) {
        long long a = sm.xmw[0];
        for (int w2 = 1; w2 < kFW; ++w2) a = max(a, sm.xmw[w2]);
        sm.xmx[xpar] = __longlong_as_double(a);
      }
    }
    f_pass<true>(sm, cl, D, I, G, x, par, first);
    if (real) {
      const int64_t g = co + j;
      const double fl = sm.fl[t];
      const double R = D.cf.alpha[g] * x[j] - D.cf.kcd[g] * D.rho_n[g] - D.cf.sac[g] * D.U[g] + D.cf.kdx[g] * fl;
      zv[t] = -R;
      D.Fs[g] = fl;
      D.Fc[g] = fl;   // sigma_0/T^3: replaced after the solve (f_corr_flux) except at inflow walls
    } else {
      zv[t] = 0.0;
    }
    // the cluster's max |x|: every slice's value, published before the pass's barrier
    if (t < 32) {
      const int lane = t;
      long long mx = lane < G.Q ? __double_as_longlong(cl.map_shared_rank(&sm.xmx[xpar], lane)[0]) : 0;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) sm.xmall = __longlong_as_double(mx);
    }
    __syncthreads();
    const double xmax = sm.xmall;
    xpar ^= 1;
    sm.wgt[t] = real ? __frcp_rn((float)(fabs(x[j]) + D.wfloor * xmax + 1e-300)) : 0.0f;
    __syncthreads();
    double* v0 = Vi(0);
    f_prec(sm, cl, D, I, G, zv, v0, par);
    {
      // |v0|^2 and |x|^2, and the weighted maximum of v0 (the stopping test), in one pass
      f_reduce<2, true>(
          sm, cl, par, 2,
          [&](int i, int c) {
            if (G.c0 + c >= N) return 0.0;
            const double a = i == 0 ? v0[c] : x[G.c0 + c];
            return a * a;
          },
          [&](int c) { return fabs(v0[c]) * (double)sm.wgt[c]; });
      if (t == 0) {
        double r, ir;
        f_sqrt_pair(sm.sums[0], r, ir);
        sm.sc[0] = r;
        sm.sc[2] = ir;
        sm.sc[3] = sm.sums[2];
      } else if (t == 32) {   // another sub-partition's binary64 pipe
        double r, ir;
        f_sqrt_pair(sm.sums[1], r, ir);
        sm.sc[1] = r;
      }
      __syncthreads();
      const double nrm = sm.sc[0], xn = sm.sc[1], inv_nrm = sm.sc[2], rinf_c = sm.sc[3];
      bool conv = !(rinf_c > D.rtol);
      if (!first && !conv && rinf_c <= D.stall && (rinf_c >= 0.25 * beta_prev || (D.mixed && cycles >= 2)))
        conv = true;
      // stagnation above the stall level (two restart cycles in a row that each reduced
      // the residual by less than 10%: the binary32 passes' rounding floor lies above the
      // tolerance, e.g. a cell near zero beside a hot one): the solve ends, unconverged
      bool stagnant = false;
      if (!first && !conv) {
        stag = (rinf_c >= 0.9 * beta_prev) ? stag + 1 : 0;
        stagnant = stag >= 2;
      }
      beta_prev = rinf_c;
      if (!isfinite(nrm)) {
        if (G.q == 0 && t == 0) flag(D.status, ii, GRTE_ENAN);
        conv = true;
      }
      if (conv) break;
      if (cycles >= D.maxcycles || stagnant) {
        if (G.q == 0 && t == 0) flag(D.status, ii, GRTE_ENONCONV);
        break;
      }
      ++cycles;
      first = false;
      // ---- restart cycle: Arnoldi with CGS2 ---------------------------------------------
      if (t == 0) {
        sm.g[0] = nrm;
        for (int i = 1; i <= m; ++i) sm.g[i] = 0.0;
      }
      v0[t] *= inv_nrm;
      __syncthreads();
      int kk = 0;
      for (int jc = 0; jc < m; ++jc) {
        const double* vj = Vi(jc);
        f_pass<false>(sm, cl, D, I, G, vj, par);
        // C v_j = alpha v_j + kappa/dx F(v_j), preconditioned into V_{j+1}
        if (real) {
          const int64_t g = co + j;
          zv[t] = D.cf.alpha[g] * vj[t] + D.cf.kdx[g] * sm.fl[t];
        } else {
          zv[t] = 0.0;
        }
        __syncthreads();
        double* wv = Vi(jc + 1);
        f_prec(sm, cl, D, I, G, zv, wv, par);
        // classical Gram-Schmidt, twice (CGS2): per pass one block sum of the jc + 1 dot
        // products w.V_i and one cluster sum; the Hessenberg column accumulates in shared
        // memory.  The second pass also sums |w1|^2, and |w2|^2 = |w1|^2 - |h2|^2 (V
        // orthonormal): exact to rounding while |h2|^2 is small against |w1|^2, which it is
        // after a first pass unless w lies almost in span(V); otherwise a separate sum.
        for (int pass = 0; pass < 2; ++pass) {
          const int nd = jc + 1 + pass;   // the dot products, and |w1|^2 in the second pass
          f_reduce<kMaxRestart + 1, false>(
              sm, cl, par, nd, [&](int i, int c) { return wv[c] * (i <= jc ? Vi(i)[c] : wv[c]); },
              [](int) { return 0.0; });
          {
            double wj = wv[t];
#pragma unroll
            for (int i = 0; i < kMaxRestart; ++i) {
              if (i > jc) break;
              wj -= sm.sums[i] * Vi(i)[t];
            }
            wv[t] = wj;
          }
          if (t <= jc) sm.hc[t] = (pass == 0 ? 0.0 : sm.hc[t]) + sm.sums[t];
          if (pass == 1 && t == 0) {
            double h2 = 0.0;
            for (int i = 0; i <= jc; ++i) h2 += sm.sums[i] * sm.sums[i];
            const double w1 = sm.sums[jc + 1];
            const bool pyth = h2 <= 1e-4 * w1;
            sm.sc[2] = pyth ? 1.0 : 0.0;
            if (pyth) {
              double r, ir;
              f_sqrt_pair(w1 - h2, r, ir);
              sm.sc[0] = r;
              sm.sc[1] = r > 0.0 ? ir : 0.0;
            }
          }
          __syncthreads();
        }
        if (sm.sc[2] == 0.0) {
          f_reduce<1, false>(sm, cl, par, 1, [&](int, int c) { return wv[c] * wv[c]; }, [](int) { return 0.0; });
          if (t == 0) {
            double r, ir;
            f_sqrt_pair(sm.sums[0], r, ir);
            sm.sc[0] = r;
            sm.sc[1] = r > 0.0 ? ir : 0.0;
          }
          __syncthreads();
        }
        const double nrmw = sm.sc[0];
        // Givens rotations and the GMRES residual estimate (thread 0; shared with all)
        if (t == 0) {
          double* hc = sm.hc;
          hc[jc + 1] = nrmw;
          for (int i = 0; i < jc; ++i) {
            const double tq = sm.cs[i] * hc[i] + sm.sn[i] * hc[i + 1];
            hc[i + 1] = -sm.sn[i] * hc[i] + sm.cs[i] * hc[i + 1];
            hc[i] = tq;
          }
          const double a0 = hc[jc], b0 = hc[jc + 1];
          const double q = a0 * a0 + b0 * b0;
          double rr, irr;
          if (q > 1e-36 && q < 1e36) {
            f_sqrt_pair(q, rr, irr);
          } else {
            rr = hypot(a0, b0);
            irr = 1.0 / rr;
          }
          const double c0g = rr > 0.0 ? a0 * irr : 1.0, s0g = rr > 0.0 ? b0 * irr : 0.0;
          hc[jc] = rr;
          sm.hinv[jc] = irr;   // 1/H[jc][jc] for the triangular solve
          const double gj = sm.g[jc];
          const double gnext = -s0g * gj;
          sm.cs[jc] = c0g;
          sm.sn[jc] = s0g;
          sm.g[jc + 1] = gnext;
          sm.g[jc] = c0g * gj;
          for (int i = 0; i <= jc; ++i) sm.H[i * kMaxRestart + jc] = hc[i];
          const bool est = fabs(gnext) <= 0.05 * D.rtol * xn;
          sm.stop = (est || nrmw == 0.0 || jc + 1 >= m) ? 1 : 0;
        }
        wv[t] *= sm.sc[1];
        __syncthreads();
        ++its;
        kk = jc + 1;
        if (sm.stop) break;
      }
      // x += V y, H y = g (upper triangular, kk columns)
      if (t == 0) {
        for (int i = kk - 1; i >= 0; --i) {
          double tq = sm.g[i];
          for (int l = i + 1; l < kk; ++l) tq -= sm.H[i * kMaxRestart + l] * sm.y[l];
          sm.y[i] = tq * sm.hinv[i];
        }
      }
      __syncthreads();
      if (real) {
        double tq = x[j];
#pragma unroll
        for (int i = 0; i < kMaxRestart; ++i) {
          if (i >= kk) break;
          tq += sm.y[i] * Vi(i)[t];
        }
        x[j] = tq;
      }
      __syncthreads();
    }
  }
  // the correction's flux at the converged iterate (sigma_0/T^3)
  if (I.kind == GRTE_SIGMA_T3) f_corr_flux(sm, D, I, G, FVec{x, 0.0, 0.0});
  if (G.q == 0 && t == 0) {
    D.gits[ii] = its;
    D.gcycles[ii] = cycles;
  }
  cl.sync();   // no CTA leaves while another may read its shared memory
}

}  // namespace grte
