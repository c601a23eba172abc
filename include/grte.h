/*
 * grte.h - C ABI of the GB300 (sm_103a) implementation of the asymptotic-preserving
 * prediction / correction / projection scheme for the nonlinear gray radiative
 * transfer equation (Tang, Wang, Zhang, arXiv:1811.05579).
 *
 * Scope: the 1D even/odd staggered scheme of Sec. 4 (Algorithm 2) for a
 * temperature-independent opacity sigma(x), and its sigma_0(x)/T^3 form of Sec. 5,
 * for any number of independent slab instances advanced together.
 *
 * Conventions (every entry point):
 *  - Plain C types only.  Pointers marked "host" are read or written on the host and
 *    copied; the library keeps no reference to them after the call returns.
 *  - Pointers marked "device" are CUDA device addresses owned by the caller.
 *  - Every call returns a grte_status and never aborts the process.  A failed call
 *    leaves a message readable with grte_last_error().  Size arguments are checked
 *    against the exact size the call needs (GRTE_EINVAL otherwise).
 *  - Steps are launched asynchronously on the handle's stream.  Problems found on
 *    the device (non-converged Krylov or Newton solve, negative right-hand side of
 *    the temperature equation, NaN) are recorded per instance and reported, sticky,
 *    by the grte_get_* calls and grte_sync(), which synchronise the stream;
 *    grte_sync() clears them once reported.
 *  - Layout of the angular unknowns in device memory: per instance, angle-major
 *    lines, E[k][j] (k = 0..M-1 positive angles, j = 0..nx-1 cells) and
 *    O[k][i] (i = 0..nx nodes).  Host copies returned by grte_get_E/O use the
 *    cell-major order [j][k] / [i][k].
 */
#ifndef GRTE_H
#define GRTE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grte_ctx* grte_t;

typedef enum {
  GRTE_OK = 0,
  GRTE_EINVAL = 1,     /* bad argument (size, range, NULL, state)                    */
  GRTE_ENOMEM = 2,     /* device or host allocation failed                           */
  GRTE_ECUDA = 3,      /* a CUDA runtime call failed                                 */
  GRTE_ENONCONV = 4,   /* a Krylov or Newton solve did not reach its tolerance       */
  GRTE_ENEGATIVE = 5,  /* right-hand side R <= 0 in the temperature equation: T = 0  */
  GRTE_ENAN = 6,       /* NaN or Inf met in the state                                */
  GRTE_ETIMEOUT = 7,   /* a device-side wait gave up                                 */
  GRTE_ESTATE = 8      /* handle used before its state was set                       */
} grte_status;

enum { GRTE_SIGMA_CONST = 0, /* sigma(x), independent of T (Sec. 4)            */
       GRTE_SIGMA_T3 = 1,    /* sigma_0(x) / T^3 (Sec. 5, Eq. marshak00)        */
       GRTE_SIGMA_POW = 2    /* sigma_0(x) / T^p, 0 <= p <= 3 (sigma_p): the Sec. 5 form with
                                kappa = T^p, theta = T^{3-p}, V* = (U*)^{p/4} in the
                                correction (p = 3: GRTE_SIGMA_T3; p = 0: GRTE_SIGMA_CONST) */ };
enum { GRTE_BC_INFLOW = 0,   /* I(0,v) = b_L(v), I(L,-v) = b_R(-v), v > 0 (Eq. BC1d, Eq. bc-pre) */
       GRTE_BC_REFLECT = 1,  /* I(wall, v) = I(wall, -v): odd part zero at the walls (1D)        */
       GRTE_BC_PERIODIC = 2  /* 2D only: the axis wraps around                                   */ };
enum { GRTE_FP64 = 0,        /* every per-element operation in binary64                         */
       GRTE_MIXED = 1        /* angular bulk in binary32; per-cell Newton and sums in binary64   */ };

/* One 1D slab instance on [x0, x1] with nx uniform cells (Sec. 4, Eq. E000/O000). */
typedef struct {
  int64_t nx;            /* cells, >= 2                                                      */
  int n_angle;           /* M, positive angles (the quadrature has 2M directions +-v_k)       */
  const double* v;       /* host, M angles in (0,1], or NULL: Gauss-Legendre with 2M nodes   */
  const double* w;       /* host, M weights summing to 1 (= int_0^1 dv), or NULL with v NULL */
  const double* sigma;   /* host, nx values of sigma(x) (CONST) or sigma_0(x) (T3), >= 0     */
  int sigma_kind;        /* GRTE_SIGMA_CONST or GRTE_SIGMA_T3                                */
  int bc;                /* GRTE_BC_INFLOW or GRTE_BC_REFLECT                                */
  const double* bL;      /* host, M values I(x0, +v_k) (INFLOW only; NULL = 0)               */
  const double* bR;      /* host, M values I(x1, -v_k) (INFLOW only; NULL = 0)               */
  double x0, x1;         /* slab, x1 > x0                                                    */
  double dt;             /* time step > 0                                                    */
  double a, c, Cv;       /* radiation constant, light speed, heat capacity (> 0)            */
  double eps;            /* scaled mean free path epsilon > 0                                */
  double sigma_p;        /* the exponent p of GRTE_SIGMA_POW (ignored otherwise)              */
} grte_instance1d;

typedef struct {
  int precision;         /* GRTE_FP64 (default) or GRTE_MIXED                                */
  double krylov_rtol;    /* prediction solve stops when every cell's preconditioned residual
                            is <= rtol |rho_j| (1e-13), or when a restart cycle stalls below
                            1e-9 (the rounding floor of the residual).  MIXED: rtol is
                            floored at 1e-9, cells below 1e-6 max|rho| are measured against
                            that floor, and a second restart below 1e-4 ends the solve; in
                            the one-kernel solve (solver1d) two restart cycles in a row that
                            each reduce the residual by less than 10% above that level end
                            it with GRTE_ENONCONV (the binary32 rounding floor lies above the
                            tolerance there)                                                   */
  int krylov_restart;    /* GMRES restart length (10)                                        */
  int krylov_maxcycles;  /* GMRES restart cycles per step before GRTE_ENONCONV (30)           */
  int newton_maxit;      /* per-cell Newton iterations before GRTE_ENONCONV (60)             */
  int energy_every;      /* 1: accumulate the energy sums of grte_get_energy every step; 0 off */
  void* stream;          /* cudaStream_t to run on; NULL: the library makes its own          */
  int line_threads;      /* threads per line solve: 0 (default) = autotune at the first step
                            (times the line kernels at 256, 512 and 1024 threads on this
                            handle's instances and keeps the fastest), or 256, 512, 1024    */
  int use_graph;         /* 1 (default): from the second step on, each step is one CUDA graph
                            launch (captured once; the Krylov loop runs under device-side
                            conditional nodes, no host round trip inside a step).  Steps
                            taken while per-kernel profiling is on run eagerly.  0: eager    */
  int prec2d;            /* 2D preconditioners, a bit set.  Prediction: GRTE_PREC2D_BLOCK
                            (0, default): the per-cell angular block (cells uncoupled);
                            GRTE_PREC2D_MULTIGRID (bit 0): first a solve preconditioned by
                            block elimination of the (e, rho) system with the per-cell
                            diagonal of each pair operator and one multigrid V-cycle on the
                            cells' rho Schur complement (one scale for all cells), then the
                            per-cell scaled solve with the block preconditioner.  Correction
                            substep 2: the per-cell diagonal (default), or with
                            GRTE_PREC2D_CORR_MG (bit 1) one V-cycle per direction pair of a
                            2x2-aggregation multigrid with zebra x/y line smoothers (binary32;
                            about 23 floats per cell and pair on the finest level).  Ignored
                            by the 1D path                                                 */
  int solver1d;          /* 1D prediction solve: GRTE_SOLVER_AUTO (default): in GRTE_MIXED, when
                            every instance has 64 <= nx <= 8192 and n_angle <= 32 and the
                            restart length is at most 11 (its Krylov basis is held in shared
                            memory), the whole
                            solve of an instance runs in one persistent kernel on a cluster of
                            up to 16 CTAs (the angular unknowns of each 512-cell slice held in
                            shared memory), else the line kernels; GRTE_SOLVER_LINES: always
                            the line kernels (one launch per line pass and Krylov step)      */
} grte_options;
enum { GRTE_SOLVER_AUTO = 0, GRTE_SOLVER_LINES = 1 };

/* Statistics of the last grte_step call (summed over its steps and instances). */
typedef struct {
  int64_t steps;             /* steps taken by the handle so far                   */
  int64_t krylov_iters;      /* GMRES iterations in the last grte_step call        */
  int64_t krylov_cycles;     /* GMRES restart cycles in the last grte_step call    */
  int64_t newton_iters_max;  /* largest per-cell Newton count in the last step     */
  double newton_iters_mean;  /* mean per-cell Newton count in the last step        */
  int64_t status_flags;      /* OR over instances of (1 << grte_status) seen       */
  int64_t line_threads;      /* threads per line solve in use (0 before the first step) */
  int64_t line_smem;         /* 1: the line unknowns stay in shared memory           */
  int64_t krylov_iters_corr; /* 2D: the part of krylov_iters spent in the correction
                                substep (the rest is the prediction); 1D: 0          */
  int64_t krylov_iters_mg;   /* 2D: the part of the prediction's iterations taken with
                                the multigrid preconditioner; 1D: 0                  */
  int64_t launches;          /* 2D: kernels launched by the last grte2d_step call (1D:
                                0; see grte_last_launches)                           */
} grte_stats_t;

/* Fill *opt with the defaults. */
void grte_default_options(grte_options* opt);

/* Create a handle for n_inst independent 1D instances (Sec. 4 / Sec. 5).  All
 * inputs are copied.  opt may be NULL (defaults).  The state is unset until
 * grte_set_state().  Errors: EINVAL (bad sizes/values), ENOMEM, ECUDA. */
grte_status grte_create_1d(int n_inst, const grte_instance1d* inst, const grte_options* opt,
                           grte_t* out);

/* Set the state of instance `inst` from host arrays: T (nx), and either
 * E (nx*M, [j][k]) and O ((nx+1)*M, [i][k]), or E = O = NULL for the equilibrium
 * I = a c T^4 (E = a c T^4, O = 0).  U is set to T^4 (Algorithm 2 input). */
grte_status grte_set_state(grte_t h, int inst, const double* T, const double* E, const double* O);

/* Checkpoint / restore.  grte_get_state writes an opaque blob of the handle's whole
 * state: the raw device arrays T, U (binary64) and E - a c U, O (in the handle's bulk
 * type), the energy sums of grte_get_energy and the step count, behind a header with
 * the precision and every instance's (nx, n_angle).  buf: host, *len bytes; with
 * buf = NULL only *len is set to the size needed.  grte_restore_state loads such a blob
 * into a handle created with the same instances and precision; steps taken after a
 * restore are bit-identical to the steps the saved handle would have taken (the blob
 * holds every value a step reads).  Errors: EINVAL (size, header, precision or
 * instance sizes differ; *len too small), ESTATE (state unset). */
grte_status grte_get_state(grte_t h, void* buf, size_t* len);
grte_status grte_restore_state(grte_t h, const void* buf, size_t len);

/* T of instance `inst` (nx values, binary64) copied into the caller's device buffer
 * dptr (device) on the caller's CUDA stream (NULL: the handle's stream), after the
 * handle's queued steps (the caller's stream waits for them); asynchronous, no host
 * round trip (zero-copy hand-off to frameworks holding the device memory).  Errors:
 * EINVAL (bad instance, NULL dptr, len != nx). */
grte_status grte_get_T_device(grte_t h, int inst, double* dptr, size_t len, void* stream);

/* Advance every instance by nsteps steps of Algorithm 2 (asynchronous). */
grte_status grte_step(grte_t h, int64_t nsteps);

/* Wait for the stream; return the first device-side status (ENAN, ENONCONV, ENEGATIVE in
 * that order) recorded by the steps since the last grte_sync, then clear it: a status is
 * sticky (every grte_get_* call reports it too) until grte_sync has returned it. */
grte_status grte_sync(grte_t h);

/* Copy results of instance `inst` to host arrays (synchronises).  len = element count. */
grte_status grte_get_T(grte_t h, int inst, double* T, size_t len);           /* nx              */
grte_status grte_get_rho(grte_t h, int inst, double* rho, size_t len);       /* nx, rho = <I> = sum_k w_k E_k */
grte_status grte_get_E(grte_t h, int inst, double* E, size_t len);           /* nx*M,  [j][k]   */
grte_status grte_get_O(grte_t h, int inst, double* O, size_t len);           /* (nx+1)*M, [i][k] */
/* Cell-centre intensities I(+v_k) = E + eps (O_j + O_{j+1})/2 and I(-v_k) = E - eps(...), [j][k]. */
grte_status grte_get_I(grte_t h, int inst, double* Ipos, double* Ineg, size_t len);
/* Intermediate per-cell results of the last step: which = 0 U*, 1 F* =
 * sum_k w_k v_k (O*_{j+1,k} - O*_{j,k}), 2 rho*, 3 Newton iterations (as double),
 * 4 the flux that correction substep 1 takes (sigma(x): F*; sigma_0/T^3: the flux of
 * Eq. dis-cor-marshak1 at the predicted data with V* = max(U*,0)^{3/4}). */
grte_status grte_get_stage(grte_t h, int inst, int which, double* out, size_t len);
/* Energy diagnostics of instance `inst` (FP64 sums on the device; Eq. energybalance and
 * Eq. semiconservative of Sec. 3, 1D): out[0] = sum_j dx (rho_j/c + Cv T_j) now;
 * out[1] = sum over the steps taken with energy_every = 1 of dt sum_j F*_j (the
 * telescoped wall flux sum_k w_k v_k (O*_N - O*_0) of the prediction);
 * out[2] = sum over those steps of dt sum_j eps^2/(c sig_j dt + eps^2) (F*_j - F^{n+1}_j),
 * F = sum_k w_k v_k (O_{j+1,k} - O_{j,k}).  For a T-independent sigma
 * out[0] + out[1] - out[2] is constant in time (n = 3). */
grte_status grte_get_energy(grte_t h, int inst, double* out, size_t n);
/* Quadrature actually used by instance `inst` (M values each). */
grte_status grte_get_quadrature(grte_t h, int inst, double* v, double* w, size_t len);

grte_status grte_stats(grte_t h, grte_stats_t* st);

/* Line-solver tuning of the handle: *line_threads as in grte_stats_t, and ms[i] the
 * timed cost (factor pass + 4 solve passes + correction pass, ms) of candidate
 * 256 << i (i = 0..2; -1: not timed or not feasible).  n >= 3.  Errors: EINVAL. */
grte_status grte_get_tuning(grte_t h, int* line_threads, double* ms, size_t n);

/* Kernel ids for per-kernel timing. */
enum { GRTE_K_CELL_COEF = 0, GRTE_K_RHO = 1, GRTE_K_PRED_FACTOR = 2, GRTE_K_PRED_HOM = 3,
       GRTE_K_PRED_FULL = 4, GRTE_K_GMRES = 5, GRTE_K_NEWTON = 6, GRTE_K_CORR = 7,
       GRTE_K_PROJECT = 8, GRTE_K_ENERGY = 9, GRTE_K_PRED_SOLVE = 10, GRTE_NKERNELS = 11 };
/* Start recording a CUDA event pair around every launch of the kernels whose bit
 * (1 << id) is set in kernel_mask, on the handle's stream (device-side timing). */
grte_status grte_profile_begin(grte_t h, uint32_t kernel_mask);
/* Stop recording, synchronise, and return per kernel id the summed event time (ms)
 * and the launch count; n must be >= GRTE_NKERNELS (host arrays). */
grte_status grte_profile_end(grte_t h, double* ms, int64_t* launches, size_t n);
/* Kernel launches issued by the last grte_step call (all kernels, profiled or not). */
int64_t grte_last_launches(grte_t h);
const char* grte_last_error(grte_t h);
void grte_destroy(grte_t h);   /* NULL is a no-op */

/* Testing hook: the (n+1)-th device allocation of the 1D handle calls from now on fails
 * as if the device were out of memory (grte_create_1d then returns GRTE_ENOMEM, with the
 * handle in *out for grte_last_error and grte_destroy); n < 0 switches it off. */
void grte_test_fail_alloc_after(int n);

/* ---- Learned initial guess of the per-cell Newton solve --------------------------------
 * The paper solves the per-cell quartic of Eq. Tnp1 with "standard iterative solvers";
 * it has no learned component.  This optional part supplies Newton's starting point from
 * a small network 6 -> 64 -> 64 -> 64 -> 1 (GELU, BF16 weights, FP32 accumulation)
 * trained on the GPU on (local state -> converged T^{n+1}) pairs that the scheme itself
 * produces.  Newton still runs to convergence from the guess (one Newton step from any
 * positive guess lands at or above the root of the convex quartic, and the start is
 * clamped to the plain upper bound min((R/A)^{1/4}, R/B), so the residual can only shrink),
 * so the converged T is the same as without the guess.
 * Raw features, per cell: log10 T^n, log10 rho*, log10 sigma_eff (sigma or sigma_0/T^3),
 * log10 eps, log10 dt, log10 Cv; target y = log10(T^{n+1}/T^n). */
enum { GRTE_MLP_IN = 6, GRTE_MLP_HIDDEN = 64, GRTE_MLP_NPARAMS = 8833 };
typedef struct grte_mlp* grte_mlp_t;
/* He-normal weights from `seed`, zero biases, identity standardisation. */
grte_status grte_mlp_create(uint64_t seed, grte_mlp_t* out);
void grte_mlp_destroy(grte_mlp_t m);   /* NULL is a no-op */
const char* grte_mlp_last_error(grte_mlp_t m);
/* Standardisation: network input (f - mean_in)/std_in, output y = out*std_out + mean_out. */
grte_status grte_mlp_set_norm(grte_mlp_t m, const float* mean_in, const float* std_in, float mean_out, float std_out);
/* FP32 master parameters, layout W1[64][6] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4 (host). */
grte_status grte_mlp_get_params(grte_mlp_t m, float* p, size_t n);
grte_status grte_mlp_set_params(grte_mlp_t m, const float* p, size_t n);
/* y[i] (un-standardised) for n raw feature rows X[i*6 .. i*6+5] (host arrays). */
grte_status grte_mlp_forward(grte_mlp_t m, const float* X, int64_t n, float* y);
/* The same on device arrays X (n x 6) and y (n) on a CUDA stream (NULL: the default
 * stream); asynchronous (the inference the Newton kernels use). */
grte_status grte_mlp_forward_device(grte_mlp_t m, const float* X, int64_t n, float* y, void* stream);
/* Gradient (n_grad = GRTE_MLP_NPARAMS) of the mean squared standardised error at the current
 * BF16 weights, and that loss (host arrays). */
grte_status grte_mlp_grad(grte_mlp_t m, const float* X, const float* y, int64_t n, float* grad, size_t n_grad,
                          float* loss);
/* Adam (lr, beta 0.9/0.999) over `epochs` seeded shuffles of the n samples in mini-batches. */
grte_status grte_mlp_train(grte_mlp_t m, const float* X, const float* y, int64_t n, int epochs, int batch, float lr,
                           uint64_t seed, float* loss);
/* Use `m` (not owned; keep it alive while the handle steps) for Newton's starting point in
 * every later step of h; NULL restores the plain start. */
grte_status grte_set_guess(grte_t h, grte_mlp_t m);
/* Newton's starting point: BOUND (default) min((R/A)^{1/4}, R/B), from which Newton
 * decreases monotonically to the root; PREVIOUS one Newton step from T^n (the textbook
 * start); LEARNED one Newton step from the network's guess, clamped to BOUND (set by
 * grte_set_guess), in the cells where the guess lies more than 10^0.05 - 1 (about 12%)
 * below BOUND (elsewhere BOUND is within the network's error of the root and is kept).
 * All three converge to the same root. */
enum { GRTE_PREC2D_BLOCK = 0, GRTE_PREC2D_MULTIGRID = 1, GRTE_PREC2D_CORR_MG = 2 };
enum { GRTE_START_BOUND = 0, GRTE_START_PREVIOUS = 1, GRTE_START_LEARNED = 2 };
grte_status grte_set_newton_start(grte_t h, int mode);
/* 1: record the features and the converged target of every cell at each step (the last
 * step's are returned by grte_get_newton_samples); 0: off. */
grte_status grte_set_sample_logging(grte_t h, int on);
grte_status grte_get_newton_samples(grte_t h, int inst, float* X, float* y, size_t nx);

/* Steps without any allocation (the paper has no counterpart; this is a service to
 * callers that cannot allocate device memory - for instance code running inside a
 * memory pool or allocator callback, under a strict memory budget, or in a process
 * whose allocator must not be re-entered).  It advances ONE instance `inst` by
 * nsteps steps of grte_step (FP64 only; opt may be NULL; opt->stream is ignored and
 * `stream` is used), with the state in caller-owned device memory, updated in place:
 *   T  device, nx doubles;
 *   E  device, nx*M doubles, line-major E[k*nx + j] (the device layout of grte.h);
 *   O  device, (nx+1)*M doubles, line-major O[k*(nx+1) + i].
 * No cudaMalloc, cudaFree or other allocating call is made: every work buffer is
 * carved from one static device array of 11,198,464 bytes (about 11.2 MB) that every GPU loading this
 * library holds until the process exits.  Limits: nx <= 4096, n_angle <= 32,
 * nx*n_angle <= 65536; larger sizes return GRTE_EINVAL.  The first call on a device
 * looks up the device address of that array (cudaGetSymbolAddress, with the device
 * current), so make that first call before any stream capture.  All calls share the
 * array and each call clears what must start at zero (statuses, counters, Krylov
 * scalars); calls whose execution overlaps on the GPU race with each other.  Returns
 * the same statuses as grte_step + grte_sync (synchronises `stream`). */
grte_status grte_step1d_noalloc(const grte_instance1d* inst, const grte_options* opt, double* T, double* E,
                                double* O, int64_t nsteps, void* stream);

/* ----------------------------------------------------------------------------------
 * 2D instances.  The paper derives the scheme in 1D and extends it direction by
 * direction (Sec. 4); the 2D form used here: E (and U, T) at the centres of an
 * nx x ny cell grid, O at its (nx+1) x (ny+1) vertices, for K pairs of directions
 * (Omega_k, -Omega_k) with Omega_k = (mu_k, eta_k).  The streaming derivative of E
 * at a vertex is the mean of the two cell differences across it, that of O at a
 * cell the mean of the two vertex differences along each side; node, cell and U
 * equations, Newton and correction are those of the 1D scheme (Eq. dis-pre,
 * Eq. dis-pre-marshak, Eq. Tnp1, Eq. dis-cor, Eq. dis-proj).  A cell beside an inflow
 * wall applies Eq. bc-pre to its own wall side, as the 1D wall cell does (side =
 * s 2/eps (b - E_cell) - opposite side); a wall vertex itself uses the same relation
 * along the normal with E the mean of the two wall cells beside it, and a corner of two
 * inflow walls takes the mean of the two walls' values.
 *
 * Linear solves: the prediction by GMRES on (e, rho) (E = rho + e, as in 1D) with the
 * matrix applied by stencil kernels and an exact per-cell angular block solve as
 * preconditioner (optionally preceded by a multigrid-preconditioned stage, prec2d);
 * correction substep 2 by GMRES on the K stacked pair systems (Jacobi preconditioned).
 * Both run on unknowns scaled per cell by the cell's own magnitude, so that the stopping
 * test holds in every cell.  GRTE_FP64: binary64 throughout; GRTE_MIXED: binary32
 * Krylov cycles inside binary64 restarts (grte2d_create).
 * -------------------------------------------------------------------------------- */
typedef struct grte2d_ctx* grte2d_t;

typedef struct {
  int64_t nx, ny;        /* cells per axis, >= 2 each                                        */
  int n_pair;            /* K; 0: the built-in level-symmetric S8 set (20 pairs)             */
  const double* mu;      /* host, K x-cosines (n_pair > 0), nonzero where x is an inflow axis */
  const double* eta;     /* host, K y-cosines, nonzero where y is an inflow axis              */
  const double* w;       /* host, K pair weights > 0 (renormalised to sum 1)                  */
  const double* sigma;   /* host, nx*ny values, row-major [j*nx + i] (j: y index), >= 0       */
  int sigma_kind;        /* GRTE_SIGMA_CONST or GRTE_SIGMA_T3                                 */
  int bc_x, bc_y;        /* GRTE_BC_INFLOW or GRTE_BC_PERIODIC per axis                       */
  double b_x0, b_x1;     /* isotropic inflow intensity on x = 0 and x = lx (INFLOW; 0: vacuum) */
  double b_y0, b_y1;     /* the same on y = 0 and y = ly                                      */
  double lx, ly;         /* domain [0, lx] x [0, ly]                                          */
  double dt, a, c, Cv, eps;
  double sigma_p;        /* the exponent p of GRTE_SIGMA_POW (ignored otherwise)              */
} grte_instance2d;

/* Create a 2D handle (inputs copied; opt may be NULL: precision, krylov_rtol (root mean
 * square over cells of the preconditioned residual relative to each cell's own
 * magnitude, default 1e-13; a restart cycle that stalls below 1e-9, the rounding floor
 * of the residual, is accepted too), krylov_restart (up to 64; 30 if the 1D default 10
 * is given), krylov_maxcycles, newton_maxit, stream and prec2d apply).  GRTE_MIXED: each
 * restart forms the residual and updates the unknowns in binary64, but the cycle's
 * Krylov process (basis, matrix, block preconditioner, Gram-Schmidt) runs in binary32
 * and ends after a 1e5 reduction of the residual (iterative refinement); krylov_rtol is
 * floored at 1e-11; coefficients, Newton and the energy sums stay binary64.  The state is
 * unset until grte2d_set_state.  Errors: EINVAL, ENOMEM, ECUDA. */
grte_status grte2d_create(const grte_instance2d* inst, const grte_options* opt, grte2d_t* out);
/* T: nx*ny; E: nx*ny*K as [cell][k] and O: (nx+1)*(ny+1)*K as [vertex][k] (vertex
 * index j*(nx+1) + i), or E = O = NULL for the equilibrium I = a c T^4. */
grte_status grte2d_set_state(grte2d_t h, const double* T, const double* E, const double* O);
/* Advance n steps (synchronous).  Statuses as grte_step + grte_sync. */
grte_status grte2d_step(grte2d_t h, int64_t n);
grte_status grte2d_get_T(grte2d_t h, double* T, size_t len);           /* len = nx*ny          */
grte_status grte2d_get_E(grte2d_t h, double* E, size_t len);           /* len = nx*ny*K        */
grte_status grte2d_get_O(grte2d_t h, double* O, size_t len);           /* len = (nx+1)(ny+1)K  */
/* which: 0 U*, 1 the flux term of the temperature equation (Eq. Tnp1): sum_k w_k (D*_k O_k)
 * with O from the predicted E* by the vertex map of the prediction (sigma(x)) or of the
 * multiplier V* = (U*)^{3/4} (sigma_0/T^3, Eq. dis-cor-marshak1), 2 rho*, 3 Newton
 * iterations; len = nx*ny. */
grte_status grte2d_get_stage(grte2d_t h, int which, double* out, size_t len);
grte_status grte2d_get_quadrature(grte2d_t h, double* mu, double* eta, double* w, size_t K);
/* Total energy sum over cells dx dy (rho/c + Cv T) of the current state. */
grte_status grte2d_get_energy(grte2d_t h, double* e);
grte_status grte2d_stats(grte2d_t h, grte_stats_t* st);
/* Learned Newton start on a 2D handle, as grte_set_guess / grte_set_newton_start /
 * grte_set_sample_logging / grte_get_newton_samples (n = nx*ny; the features are the
 * same six per cell). */
grte_status grte2d_set_guess(grte2d_t h, grte_mlp_t mlp);
grte_status grte2d_set_newton_start(grte2d_t h, int mode);
grte_status grte2d_set_sample_logging(grte2d_t h, int on);
grte_status grte2d_get_newton_samples(grte2d_t h, float* X, float* y, size_t n);
const char* grte2d_last_error(grte2d_t h);
void grte2d_destroy(grte2d_t h);

/* ----------------------------------------------------------------------------------
 * One create call for both dimensions: the problem of Eq. radiative_transport on a
 * uniform grid in 1D (Sec. 4) or 2D, described by grid, quadrature, opacity, the
 * constants a, c, C_v, eps and the boundary conditions.  It builds a 1D handle with one
 * instance (grte_create_1d) or a 2D handle (grte2d_create) and returns it in a
 * grte_handle; the dimension-specific calls stay available on h1 / h2.
 * -------------------------------------------------------------------------------- */
typedef struct {
  int dim;                 /* 1 or 2                                                         */
  int64_t nx, ny;          /* cells per axis (ny ignored in 1D)                              */
  double x0, x1;           /* domain along x (1D: the slab; 2D: x0 must be 0)                */
  double y0, y1;           /* domain along y (2D; y0 must be 0)                              */
  double dt;               /* time step                                                      */
} grte_grid;
typedef struct {
  int n_dir;               /* directions: 1D 2M (+-v_k), 2D 2K (+-Omega_k), or 0 for the
                              default (1D: 16 Gauss-Legendre; 2D: S8, 40)                     */
  const double* mu;        /* host or NULL (built-in): 1D the M positive cosines v_k; 2D the K
                              x-cosines of the pairs                                          */
  const double* eta;       /* host, 2D: the K y-cosines (NULL with mu NULL)                   */
  const double* w;         /* host, M or K weights (NULL with mu NULL)                        */
} grte_quadrature;
typedef struct {
  int kind;                /* GRTE_SIGMA_CONST, GRTE_SIGMA_T3 or GRTE_SIGMA_POW              */
  const double* sigma0;    /* host, one value per cell (2D row-major [j*nx + i]), or NULL     */
  double sigma0_scalar;    /* used when sigma0 is NULL                                       */
  double sigma_p;          /* the exponent p of GRTE_SIGMA_POW                              */
} grte_opacity;
typedef struct {
  int kind[4];             /* edges x0, x1, y0, y1: GRTE_BC_INFLOW, GRTE_BC_REFLECT (1D, both
                              walls), GRTE_BC_PERIODIC (2D, both edges of an axis)            */
  double b_iso[4];         /* isotropic inflow intensity per edge (0: vacuum)                */
  const double* b[4];      /* host, 1D only: per positive angle values on x0 / x1 (M each), or
                              NULL for b_iso                                                  */
} grte_bc;
typedef struct {
  int dim;
  int64_t ncell;           /* nx (1D) or nx*ny (2D)                                          */
  grte_t h1;               /* dim 1: a one-instance 1D handle                                */
  grte2d_t h2;             /* dim 2                                                          */
} grte_handle;

/* Errors: EINVAL (bad description, as grte_create_1d / grte2d_create), ENOMEM, ECUDA; on
 * failure out holds no handle (the partial one is destroyed; the message is lost). */
grte_status grte_create(const grte_grid* grid, const grte_quadrature* quad, const grte_opacity* opac,
                        double a, double c, double Cv, double eps, const grte_bc* bc,
                        const grte_options* opt, grte_handle* out);
/* Initial state: the equilibrium I = a c T^4 for the given T (nx or nx*ny values, host). */
grte_status grte_handle_set_initial(grte_handle* h, const double* T, size_t len);
grte_status grte_handle_step(grte_handle* h, int64_t n);
grte_status grte_handle_sync(grte_handle* h);
grte_status grte_handle_get_T(grte_handle* h, double* T, size_t len);   /* nx or nx*ny, host */
void grte_handle_destroy(grte_handle* h);                              /* NULL is a no-op */

/* ----------------------------------------------------------------------------------
 * The three-stage diffusion solver of Sec. 2 (Eq. limit_U_dis1 - Eq. limit_UT_dis3, fully
 * discrete as Eq. dis-diff; for sigma_0/T^3 the fully discrete form after Eq.
 * marshak-diff2) for the limit equation a dT^4/dt + C_v dT/dt = div(a c/(D sigma) grad T^4)
 * (Eq. limit_T; sigma_0/T^3: a c T^3/(D sigma_0)), batched over independent 1D instances,
 * FP64: per step one tridiagonal solve per instance for U* (prediction), the per-cell
 * quartic for T^{n+1} by monotone Newton (correction; the flux with the node mean of
 * (U*)^{3/4} for sigma_0/T^3) and U = T^4 (projection).  Zero-flux walls.
 * -------------------------------------------------------------------------------- */
typedef struct grte_diff_ctx* grte_diff_t;
typedef struct {
  int64_t nx;              /* cells, >= 2                                                    */
  const double* sigma;     /* host, nx values of sigma (CONST) or sigma_0 (T3), > 0          */
  int sigma_kind;          /* GRTE_SIGMA_CONST or GRTE_SIGMA_T3                              */
  double x0, x1, dt, a, c, Cv;
  double dd;               /* D_d of Eq. limit_T (0: 3, the 1D value)                        */
} grte_diffusion1d;

/* Errors: EINVAL, ENOMEM, ECUDA (the handle is returned in *out for grte_diff_last_error
 * and grte_diff_destroy).  stream: a cudaStream_t or NULL (own stream). */
grte_status grte_diff_create(int n_inst, const grte_diffusion1d* inst, void* stream, grte_diff_t* out);
grte_status grte_diff_set_T(grte_diff_t h, int inst, const double* T, size_t len);   /* host, nx */
grte_status grte_diff_step(grte_diff_t h, int64_t nsteps);                            /* async */
/* Statuses of the steps since the last grte_diff_sync (ENAN, ENONCONV, ENEGATIVE: a cell
 * whose right-hand side reached R <= 0, set to T = 0), then cleared. */
grte_status grte_diff_sync(grte_diff_t h);
grte_status grte_diff_get_T(grte_diff_t h, int inst, double* T, size_t len);         /* host, nx */
grte_status grte_diff_get_Ustar(grte_diff_t h, int inst, double* U, size_t len);     /* last U* */
const char* grte_diff_last_error(grte_diff_t h);
void grte_diff_destroy(grte_diff_t h);

#ifdef __cplusplus
}
#endif
#endif
