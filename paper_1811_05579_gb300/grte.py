"""Thin ctypes binding of the C ABI in include/grte.h (argument marshalling only).

Every step of the scheme runs in the CUDA library `libgrte.so` built in-tree by
`paper_1811_05579_gb300.build.build_library()`.  Importing this module loads that
library and raises if it is missing; there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgrte.so")

GRTE_OK = 0
GRTE_EINVAL, GRTE_ENOMEM, GRTE_ECUDA, GRTE_ENONCONV, GRTE_ENEGATIVE, GRTE_ENAN, GRTE_ETIMEOUT, GRTE_ESTATE = range(1, 9)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONCONV", 5: "ENEGATIVE",
                6: "ENAN", 7: "ETIMEOUT", 8: "ESTATE"}
SIGMA_CONST, SIGMA_T3, SIGMA_POW = 0, 1, 2
BC_INFLOW, BC_REFLECT, BC_PERIODIC = 0, 1, 2
FP64, MIXED = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)


class Instance1D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("n_angle", ctypes.c_int), ("v", _dp), ("w", _dp),
                ("sigma", _dp), ("sigma_kind", ctypes.c_int), ("bc", ctypes.c_int),
                ("bL", _dp), ("bR", _dp), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("dt", ctypes.c_double), ("a", ctypes.c_double), ("c", ctypes.c_double),
                ("Cv", ctypes.c_double), ("eps", ctypes.c_double), ("sigma_p", ctypes.c_double)]


class Instance2D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("n_pair", ctypes.c_int), ("mu", _dp),
                ("eta", _dp), ("w", _dp), ("sigma", _dp), ("sigma_kind", ctypes.c_int), ("bc_x", ctypes.c_int),
                ("bc_y", ctypes.c_int), ("b_x0", ctypes.c_double), ("b_x1", ctypes.c_double),
                ("b_y0", ctypes.c_double), ("b_y1", ctypes.c_double), ("lx", ctypes.c_double),
                ("ly", ctypes.c_double), ("dt", ctypes.c_double), ("a", ctypes.c_double), ("c", ctypes.c_double),
                ("Cv", ctypes.c_double), ("eps", ctypes.c_double), ("sigma_p", ctypes.c_double)]


class GridS(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double), ("dt", ctypes.c_double)]


class QuadS(ctypes.Structure):
    _fields_ = [("n_dir", ctypes.c_int), ("mu", _dp), ("eta", _dp), ("w", _dp)]


class OpacS(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("sigma0", _dp), ("sigma0_scalar", ctypes.c_double),
                ("sigma_p", ctypes.c_double)]


class BcS(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 4), ("b_iso", ctypes.c_double * 4), ("b", _dp * 4)]


class HandleS(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("ncell", ctypes.c_int64), ("h1", ctypes.c_void_p), ("h2", ctypes.c_void_p)]


class Diffusion1D(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("sigma", _dp), ("sigma_kind", ctypes.c_int), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("dt", ctypes.c_double), ("a", ctypes.c_double), ("c", ctypes.c_double),
                ("Cv", ctypes.c_double), ("dd", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("krylov_rtol", ctypes.c_double),
                ("krylov_restart", ctypes.c_int), ("krylov_maxcycles", ctypes.c_int),
                ("newton_maxit", ctypes.c_int), ("energy_every", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("line_threads", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("prec2d", ctypes.c_int), ("solver1d", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("krylov_iters", ctypes.c_int64),
                ("krylov_cycles", ctypes.c_int64), ("newton_iters_max", ctypes.c_int64),
                ("newton_iters_mean", ctypes.c_double), ("status_flags", ctypes.c_int64),
                ("line_threads", ctypes.c_int64), ("line_smem", ctypes.c_int64),
                ("krylov_iters_corr", ctypes.c_int64), ("krylov_iters_mg", ctypes.c_int64),
                ("launches", ctypes.c_int64)]


EXPORTED = ["grte_default_options", "grte_create_1d", "grte_set_state", "grte_step", "grte_sync",
            "grte_get_T", "grte_get_rho", "grte_get_E", "grte_get_O", "grte_get_I", "grte_get_stage",
            "grte_get_quadrature", "grte_stats", "grte_last_error", "grte_destroy",
            "grte_profile_begin", "grte_profile_end", "grte_last_launches", "grte_get_energy",
            "grte_step1d_noalloc", "grte_mlp_create", "grte_mlp_destroy", "grte_mlp_last_error",
            "grte_mlp_set_norm", "grte_mlp_get_params", "grte_mlp_set_params", "grte_mlp_forward",
            "grte_mlp_grad", "grte_mlp_train", "grte_set_guess", "grte_set_sample_logging",
            "grte_get_newton_samples", "grte_set_newton_start", "grte_get_tuning", "grte2d_create",
            "grte2d_set_state", "grte2d_step", "grte2d_get_T", "grte2d_get_E", "grte2d_get_O", "grte2d_get_stage",
            "grte2d_get_quadrature", "grte2d_get_energy", "grte2d_stats", "grte2d_last_error", "grte2d_destroy",
            "grte2d_set_guess", "grte2d_set_newton_start", "grte2d_set_sample_logging",
            "grte2d_get_newton_samples", "grte_get_state", "grte_restore_state", "grte_get_T_device",
            "grte_test_fail_alloc_after", "grte_create", "grte_handle_set_initial", "grte_handle_step",
            "grte_handle_sync", "grte_handle_get_T", "grte_handle_destroy", "grte_diff_create", "grte_diff_set_T",
            "grte_diff_step", "grte_diff_sync", "grte_diff_get_T", "grte_diff_get_Ustar", "grte_diff_last_error",
            "grte_diff_destroy", "grte_mlp_forward_device"]
START_BOUND, START_PREVIOUS, START_LEARNED = 0, 1, 2
PREC2D_BLOCK, PREC2D_MULTIGRID, PREC2D_CORR_MG = 0, 1, 2   # prec2d bits: prediction MG, correction MG
MLP_NPARAMS = 8833
_fp = ctypes.POINTER(ctypes.c_float)
KERNELS = ["cell_coef", "rho", "pred_factor", "pred_hom", "pred_full", "gmres", "newton", "corr",
           "project", "energy", "pred_solve"]
SOLVER_AUTO, SOLVER_LINES = 0, 1


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError("libgrte.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    lib.grte_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.grte_default_options.restype = None
    lib.grte_create_1d.argtypes = [ctypes.c_int, ctypes.POINTER(Instance1D), ctypes.POINTER(Options),
                                   ctypes.POINTER(ctypes.c_void_p)]
    lib.grte_set_state.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, _dp]
    lib.grte_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    lib.grte_sync.argtypes = [ctypes.c_void_p]
    for name in ("grte_get_T", "grte_get_rho", "grte_get_E", "grte_get_O"):
        getattr(lib, name).argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_size_t]
    lib.grte_get_I.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, ctypes.c_size_t]
    lib.grte_get_stage.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_size_t]
    lib.grte_get_quadrature.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, ctypes.c_size_t]
    lib.grte_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(Stats)]
    lib.grte_last_error.argtypes = [ctypes.c_void_p]
    lib.grte_last_error.restype = ctypes.c_char_p
    lib.grte_destroy.argtypes = [ctypes.c_void_p]
    lib.grte_destroy.restype = None
    lib.grte_profile_begin.argtypes = [ctypes.c_void_p, ctypes.c_uint32]
    lib.grte_profile_end.argtypes = [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_int64), ctypes.c_size_t]
    lib.grte_last_launches.argtypes = [ctypes.c_void_p]
    lib.grte_last_launches.restype = ctypes.c_int64
    lib.grte_get_energy.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_size_t]
    lib.grte_get_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    lib.grte_restore_state.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]
    lib.grte_get_T_device.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.c_void_p]
    lib.grte_test_fail_alloc_after.argtypes = [ctypes.c_int]
    lib.grte_test_fail_alloc_after.restype = None
    lib.grte_create.argtypes = [ctypes.POINTER(GridS), ctypes.POINTER(QuadS), ctypes.POINTER(OpacS), ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.POINTER(BcS),
                                ctypes.POINTER(Options), ctypes.POINTER(HandleS)]
    lib.grte_handle_set_initial.argtypes = [ctypes.POINTER(HandleS), _dp, ctypes.c_size_t]
    lib.grte_handle_step.argtypes = [ctypes.POINTER(HandleS), ctypes.c_int64]
    lib.grte_handle_sync.argtypes = [ctypes.POINTER(HandleS)]
    lib.grte_handle_get_T.argtypes = [ctypes.POINTER(HandleS), _dp, ctypes.c_size_t]
    lib.grte_handle_destroy.argtypes = [ctypes.POINTER(HandleS)]
    lib.grte_handle_destroy.restype = None
    lib.grte_diff_create.argtypes = [ctypes.c_int, ctypes.POINTER(Diffusion1D), ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]
    lib.grte_diff_set_T.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_size_t]
    lib.grte_diff_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    lib.grte_diff_sync.argtypes = [ctypes.c_void_p]
    lib.grte_diff_get_T.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_size_t]
    lib.grte_diff_get_Ustar.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_size_t]
    lib.grte_diff_last_error.argtypes = [ctypes.c_void_p]
    lib.grte_diff_last_error.restype = ctypes.c_char_p
    lib.grte_diff_destroy.argtypes = [ctypes.c_void_p]
    lib.grte_diff_destroy.restype = None
    lib.grte_mlp_create.argtypes = [ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]
    lib.grte_mlp_destroy.argtypes = [ctypes.c_void_p]
    lib.grte_mlp_destroy.restype = None
    lib.grte_mlp_last_error.argtypes = [ctypes.c_void_p]
    lib.grte_mlp_last_error.restype = ctypes.c_char_p
    lib.grte_mlp_set_norm.argtypes = [ctypes.c_void_p, _fp, _fp, ctypes.c_float, ctypes.c_float]
    lib.grte_mlp_get_params.argtypes = [ctypes.c_void_p, _fp, ctypes.c_size_t]
    lib.grte_mlp_set_params.argtypes = [ctypes.c_void_p, _fp, ctypes.c_size_t]
    lib.grte_mlp_forward.argtypes = [ctypes.c_void_p, _fp, ctypes.c_int64, _fp]
    lib.grte_mlp_forward_device.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p]
    lib.grte_mlp_grad.argtypes = [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, _fp, ctypes.c_size_t, _fp]
    lib.grte_mlp_train.argtypes = [ctypes.c_void_p, _fp, _fp, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_float, ctypes.c_uint64, _fp]
    lib.grte_set_guess.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.grte_set_sample_logging.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.grte_set_newton_start.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.grte_get_newton_samples.argtypes = [ctypes.c_void_p, ctypes.c_int, _fp, _fp, ctypes.c_size_t]
    lib.grte_step1d_noalloc.argtypes = [ctypes.POINTER(Instance1D), ctypes.POINTER(Options), ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.grte2d_create.argtypes = [ctypes.POINTER(Instance2D), ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_void_p)]
    lib.grte2d_set_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
    lib.grte2d_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    for name in ("grte2d_get_T", "grte2d_get_E", "grte2d_get_O"):
        getattr(lib, name).argtypes = [ctypes.c_void_p, _dp, ctypes.c_size_t]
    lib.grte2d_get_stage.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_size_t]
    lib.grte2d_get_quadrature.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_size_t]
    lib.grte2d_get_energy.argtypes = [ctypes.c_void_p, _dp]
    lib.grte2d_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(Stats)]
    lib.grte2d_last_error.argtypes = [ctypes.c_void_p]
    lib.grte2d_last_error.restype = ctypes.c_char_p
    lib.grte2d_destroy.argtypes = [ctypes.c_void_p]
    lib.grte2d_destroy.restype = None
    lib.grte2d_set_guess.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.grte2d_set_newton_start.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.grte2d_set_sample_logging.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.grte2d_get_newton_samples.argtypes = [ctypes.c_void_p, _fp, _fp, ctypes.c_size_t]
    return lib


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        _LIB = load_library()
    return _LIB


class GrteError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def _ptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def instance_struct(p, keep):
    """Fill an Instance1D from a spec dict (arrays kept alive in `keep`)."""
    sig = _f64(np.broadcast_to(p["sigma"], (p["nx"],)))
    v = _f64(p.get("v"))
    w = _f64(p.get("w"))
    M = p["n_angle"]
    bL = _f64(np.broadcast_to(p.get("bL", 0.0), (M,)))
    bR = _f64(np.broadcast_to(p.get("bR", 0.0), (M,)))
    keep += [sig, v, w, bL, bR]
    return Instance1D(p["nx"], M, _ptr(v), _ptr(w), _ptr(sig), p.get("kind", SIGMA_T3),
                      p.get("bc", BC_INFLOW), _ptr(bL), _ptr(bR), p.get("x0", 0.0),
                      p.get("x1", 1.0), p["dt"], p.get("a", 1.0), p.get("c", 1.0),
                      p.get("Cv", 1.0), p["eps"], p.get("p", 3.0))


def step1d_noalloc(spec, T_ptr, E_ptr, O_ptr, nsteps, stream=None, options=None):
    """grte_step1d_noalloc on caller-owned device buffers (device addresses as ints):
    T (nx), E (nx*M, line-major) and O ((nx+1)*M, line-major), updated in place.
    options: None (the library's defaults) or a dict of grte_options fields."""
    keep = []
    inst = instance_struct(spec, keep)
    opt = None
    if options is not None:
        opt = Options()
        lib().grte_default_options(ctypes.byref(opt))
        for k, v in options.items():
            setattr(opt, k, v)
        opt = ctypes.byref(opt)
    return lib().grte_step1d_noalloc(ctypes.byref(inst), opt, T_ptr, E_ptr, O_ptr, nsteps, stream)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fptr(a):
    return a.ctypes.data_as(_fp)


class MLP:
    """Learned Newton guess network (grte_mlp_*)."""

    def __init__(self, seed=0):
        h = ctypes.c_void_p()
        st = lib().grte_mlp_create(seed, ctypes.byref(h))
        self.h = h
        if st != GRTE_OK:
            raise GrteError(st, "grte_mlp_create")

    def _check(self, st):
        if st != GRTE_OK:
            raise GrteError(st, lib().grte_mlp_last_error(self.h).decode())

    def close(self):
        if self.h is not None:
            lib().grte_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_norm(self, mean_in, std_in, mean_out, std_out):
        mi, si = _f32(mean_in), _f32(std_in)
        self._check(lib().grte_mlp_set_norm(self.h, _fptr(mi), _fptr(si), float(mean_out), float(std_out)))

    def params(self):
        p = np.empty(MLP_NPARAMS, dtype=np.float32)
        self._check(lib().grte_mlp_get_params(self.h, _fptr(p), p.size))
        return p

    def set_params(self, p):
        p = _f32(p)
        self._check(lib().grte_mlp_set_params(self.h, _fptr(p), p.size))

    def forward(self, X):
        X = _f32(X)
        y = np.empty(X.shape[0], dtype=np.float32)
        self._check(lib().grte_mlp_forward(self.h, _fptr(X), X.shape[0], _fptr(y)))
        return y

    def forward_device(self, x_ptr, n, y_ptr, stream=None):
        """Inference on device arrays (addresses as ints) on `stream` (asynchronous)."""
        self._check(lib().grte_mlp_forward_device(self.h, ctypes.c_void_p(x_ptr), n, ctypes.c_void_p(y_ptr),
                                                  ctypes.c_void_p(stream) if stream else None))

    def grad(self, X, Y):
        X, Y = _f32(X), _f32(Y)
        g = np.empty(MLP_NPARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        self._check(lib().grte_mlp_grad(self.h, _fptr(X), _fptr(Y), X.shape[0], _fptr(g), g.size,
                                        ctypes.byref(loss)))
        return float(loss.value), g

    def train(self, X, Y, epochs=10, batch=1024, lr=1e-3, seed=0):
        X, Y = _f32(X), _f32(Y)
        loss = ctypes.c_float()
        self._check(lib().grte_mlp_train(self.h, _fptr(X), _fptr(Y), X.shape[0], epochs, batch, lr, seed,
                                         ctypes.byref(loss)))
        return float(loss.value)


class Grte:
    """Handle over n independent 1D instances (grte_create_1d)."""

    def __init__(self, instances, precision=FP64, krylov_rtol=1e-13, krylov_restart=10,
                 krylov_maxcycles=30, newton_maxit=60, energy_every=0, stream=None, line_threads=0,
                 use_graph=True, solver1d=SOLVER_AUTO):
        L = lib()
        self._keep = []
        arr = (Instance1D * len(instances))()
        self.specs = []
        for i, p in enumerate(instances):
            sig = _f64(np.broadcast_to(p["sigma"], (p["nx"],)))
            v = _f64(p.get("v"))
            w = _f64(p.get("w"))
            M = p["n_angle"]
            bL = _f64(np.broadcast_to(p.get("bL", 0.0), (M,)))
            bR = _f64(np.broadcast_to(p.get("bR", 0.0), (M,)))
            self._keep += [sig, v, w, bL, bR]
            arr[i] = Instance1D(p["nx"], M, _ptr(v), _ptr(w), _ptr(sig), p.get("kind", SIGMA_T3),
                                p.get("bc", BC_INFLOW), _ptr(bL), _ptr(bR), p.get("x0", 0.0),
                                p.get("x1", 1.0), p["dt"], p.get("a", 1.0), p.get("c", 1.0),
                                p.get("Cv", 1.0), p["eps"], p.get("p", 3.0))
            self.specs.append(dict(nx=int(p["nx"]), M=int(M), eps=float(p["eps"])))
        opt = Options()
        L.grte_default_options(ctypes.byref(opt))
        opt.precision = precision
        opt.krylov_rtol = krylov_rtol
        opt.krylov_restart = krylov_restart
        opt.krylov_maxcycles = krylov_maxcycles
        opt.newton_maxit = newton_maxit
        opt.energy_every = energy_every
        opt.stream = stream
        opt.line_threads = line_threads
        opt.use_graph = 1 if use_graph else 0
        opt.solver1d = solver1d
        h = ctypes.c_void_p()
        st = L.grte_create_1d(len(instances), arr, ctypes.byref(opt), ctypes.byref(h))
        self.h = h
        if st != GRTE_OK:
            msg = L.grte_last_error(h).decode() if h.value else "create failed"
            L.grte_destroy(h)
            self.h = None
            raise GrteError(st, msg)

    def _check(self, st, allow=()):
        if st != GRTE_OK and st not in allow:
            raise GrteError(st, lib().grte_last_error(self.h).decode())
        return st

    def close(self):
        if self.h is not None:
            lib().grte_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, inst, T, E=None, O=None):
        T, E, O = _f64(T), _f64(E), _f64(O)
        return self._check(lib().grte_set_state(self.h, inst, _ptr(T), _ptr(E), _ptr(O)))

    def step(self, n=1):
        return self._check(lib().grte_step(self.h, n))

    def sync(self, allow=()):
        return self._check(lib().grte_sync(self.h), allow)

    def _get(self, fn, inst, shape, allow):
        out = np.empty(shape, dtype=np.float64)
        self._check(fn(self.h, inst, _ptr(out), out.size), allow)
        return out

    def T(self, inst, allow=()):
        return self._get(lib().grte_get_T, inst, self.specs[inst]["nx"], allow)

    def rho(self, inst, allow=()):
        return self._get(lib().grte_get_rho, inst, self.specs[inst]["nx"], allow)

    def E(self, inst, allow=()):
        s = self.specs[inst]
        return self._get(lib().grte_get_E, inst, (s["nx"], s["M"]), allow)

    def get_state(self, allow=()):
        """The opaque checkpoint blob of the whole handle (bytes)."""
        n = ctypes.c_size_t(0)
        self._check(lib().grte_get_state(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(lib().grte_get_state(self.h, buf, ctypes.byref(n)), allow)
        return buf.raw[:n.value]

    def restore_state(self, blob):
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        return self._check(lib().grte_restore_state(self.h, buf, len(blob)))

    def T_device(self, inst, dptr, n, stream=None):
        """Copy T of `inst` into the device buffer at address dptr (n doubles) on `stream`."""
        return self._check(lib().grte_get_T_device(self.h, inst, ctypes.c_void_p(dptr), n,
                                                   ctypes.c_void_p(stream) if stream else None))

    def O(self, inst, allow=()):
        s = self.specs[inst]
        return self._get(lib().grte_get_O, inst, (s["nx"] + 1, s["M"]), allow)

    def I(self, inst, allow=()):
        s = self.specs[inst]
        ip = np.empty((s["nx"], s["M"]))
        im = np.empty((s["nx"], s["M"]))
        self._check(lib().grte_get_I(self.h, inst, _ptr(ip), _ptr(im), ip.size), allow)
        return ip, im

    def stage(self, inst, which, allow=()):
        out = np.empty(self.specs[inst]["nx"])
        self._check(lib().grte_get_stage(self.h, inst, which, _ptr(out), out.size), allow)
        return out

    def energy(self, inst):
        out = np.empty(3)
        self._check(lib().grte_get_energy(self.h, inst, _ptr(out), 3))
        return out

    def quadrature(self, inst):
        M = self.specs[inst]["M"]
        v = np.empty(M)
        w = np.empty(M)
        self._check(lib().grte_get_quadrature(self.h, inst, _ptr(v), _ptr(w), M))
        return v, w

    def profile_begin(self, kernels):
        mask = 0
        for k in kernels:
            mask |= 1 << KERNELS.index(k)
        return self._check(lib().grte_profile_begin(self.h, mask))

    def profile_end(self):
        n = len(KERNELS)
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        self._check(lib().grte_profile_end(self.h, _ptr(ms), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNELS) if cnt[i]}

    def last_launches(self):
        return int(lib().grte_last_launches(self.h))

    def set_guess(self, mlp):
        return self._check(lib().grte_set_guess(self.h, mlp.h if mlp is not None else None))

    def set_newton_start(self, mode):
        return self._check(lib().grte_set_newton_start(self.h, mode))

    def set_sample_logging(self, on):
        return self._check(lib().grte_set_sample_logging(self.h, 1 if on else 0))

    def newton_samples(self, inst):
        nx = self.specs[inst]["nx"]
        X = np.empty((nx, 6), dtype=np.float32)
        y = np.empty(nx, dtype=np.float32)
        self._check(lib().grte_get_newton_samples(self.h, inst, _fptr(X), _fptr(y), nx))
        return X, y

    def tuning(self):
        """(threads per line solve, {candidate threads: timed ms}) of the autotuner."""
        nt = ctypes.c_int()
        ms = np.full(3, -1.0)
        self._check(lib().grte_get_tuning(self.h, ctypes.byref(nt), _ptr(ms), 3))
        return int(nt.value), {256 << i: float(ms[i]) for i in range(3) if ms[i] >= 0}

    def stats(self, allow=()):
        s = Stats()
        self._check(lib().grte_stats(self.h, ctypes.byref(s)), allow)
        return {f: getattr(s, f) for f, _ in Stats._fields_}


class Grte2D:
    """One 2D instance (grte2d_create): cells nx x ny ([j][i] row-major), vertices
    (nx+1) x (ny+1), K direction pairs (the built-in S8 set when mu is None)."""

    def __init__(self, nx, ny, sigma, dt, eps, kind=SIGMA_T3, bc_x=BC_INFLOW, bc_y=BC_INFLOW, b_x0=0.0, b_x1=0.0,
                 b_y0=0.0, b_y1=0.0, mu=None, eta=None, w=None, lx=1.0, ly=1.0, a=1.0, c=1.0, Cv=1.0,
                 krylov_rtol=1e-13, krylov_restart=30, krylov_maxcycles=30, newton_maxit=60, stream=None,
                 prec=0, precision=FP64, p=3.0):
        L = lib()
        sig = _f64(np.broadcast_to(np.asarray(sigma, dtype=np.float64).ravel(), (nx * ny,)))
        mu, eta, w = _f64(mu), _f64(eta), _f64(w)
        self._keep = [sig, mu, eta, w]
        K = 0 if mu is None else mu.size
        inst = Instance2D(nx, ny, K, _ptr(mu), _ptr(eta), _ptr(w), _ptr(sig), kind, bc_x, bc_y, b_x0, b_x1, b_y0,
                          b_y1, lx, ly, dt, a, c, Cv, eps, p)
        opt = Options()
        L.grte_default_options(ctypes.byref(opt))
        opt.krylov_rtol = krylov_rtol
        opt.krylov_restart = krylov_restart
        opt.krylov_maxcycles = krylov_maxcycles
        opt.newton_maxit = newton_maxit
        opt.stream = stream
        opt.prec2d = prec
        opt.precision = precision
        h = ctypes.c_void_p()
        st = L.grte2d_create(ctypes.byref(inst), ctypes.byref(opt), ctypes.byref(h))
        self.h = h
        if st != GRTE_OK:
            msg = L.grte2d_last_error(h).decode() if h.value else "create failed"
            L.grte2d_destroy(h)
            self.h = None
            raise GrteError(st, msg)
        self.nx, self.ny = nx, ny
        self.nc, self.nv = nx * ny, (nx + 1) * (ny + 1)
        self.K = K if K else 20

    def _check(self, st, allow=()):
        if st != GRTE_OK and st not in allow:
            raise GrteError(st, lib().grte2d_last_error(self.h).decode())
        return st

    def close(self):
        if self.h is not None:
            lib().grte2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, T, E=None, O=None):
        T = _f64(np.ravel(T))
        E = None if E is None else _f64(E)
        O = None if O is None else _f64(O)
        return self._check(lib().grte2d_set_state(self.h, _ptr(T), _ptr(E), _ptr(O)))

    def step(self, n=1, allow=()):
        return self._check(lib().grte2d_step(self.h, n), allow)

    def T(self, allow=()):
        out = np.empty(self.nc)
        self._check(lib().grte2d_get_T(self.h, _ptr(out), out.size), allow)
        return out

    def E(self, allow=()):
        out = np.empty((self.nc, self.K))
        self._check(lib().grte2d_get_E(self.h, _ptr(out), out.size), allow)
        return out

    def O(self, allow=()):
        out = np.empty((self.nv, self.K))
        self._check(lib().grte2d_get_O(self.h, _ptr(out), out.size), allow)
        return out

    def stage(self, which, allow=()):
        out = np.empty(self.nc)
        self._check(lib().grte2d_get_stage(self.h, which, _ptr(out), out.size), allow)
        return out

    def quadrature(self):
        mu, eta, w = np.empty(self.K), np.empty(self.K), np.empty(self.K)
        self._check(lib().grte2d_get_quadrature(self.h, _ptr(mu), _ptr(eta), _ptr(w), self.K))
        return mu, eta, w

    def energy(self):
        e = np.zeros(1)
        self._check(lib().grte2d_get_energy(self.h, _ptr(e)))
        return float(e[0])

    def set_guess(self, mlp):
        return self._check(lib().grte2d_set_guess(self.h, mlp.h if mlp is not None else None))

    def set_newton_start(self, mode):
        return self._check(lib().grte2d_set_newton_start(self.h, mode))

    def set_sample_logging(self, on):
        return self._check(lib().grte2d_set_sample_logging(self.h, 1 if on else 0))

    def newton_samples(self):
        X = np.empty((self.nc, 6), dtype=np.float32)
        y = np.empty(self.nc, dtype=np.float32)
        self._check(lib().grte2d_get_newton_samples(self.h, _fptr(X), _fptr(y), self.nc))
        return X, y

    def stats(self, allow=()):
        s = Stats()
        self._check(lib().grte2d_stats(self.h, ctypes.byref(s)), allow)
        return {f: getattr(s, f) for f, _ in Stats._fields_}


class Problem:
    """grte_create: one problem of either dimension (grid dim 1 or 2), driven through the
    dimension-independent grte_handle_* calls."""

    def __init__(self, dim, nx, dt, eps, sigma0, kind=SIGMA_T3, ny=0, x0=0.0, x1=1.0, y1=1.0, n_dir=0,
                 mu=None, eta=None, w=None, bc_kind=(BC_INFLOW,) * 4, b_iso=(0.0,) * 4, a=1.0, c=1.0, Cv=1.0,
                 precision=FP64, p=3.0):
        L = lib()
        self._keep = []
        sig = np.asarray(sigma0, dtype=np.float64)
        scalar = sig.ndim == 0
        sig = None if scalar else np.ascontiguousarray(sig.ravel())
        arrs = [None if x is None else _f64(x) for x in (mu, eta, w)]
        self._keep += [sig] + arrs
        grid = GridS(dim, nx, ny, x0, x1, 0.0, y1, dt)
        quad = QuadS(n_dir, *[_ptr(x) for x in arrs])
        opac = OpacS(kind, _ptr(sig), float(sigma0) if scalar else 0.0, float(p))
        bc = BcS((ctypes.c_int * 4)(*bc_kind), (ctypes.c_double * 4)(*b_iso), (_dp * 4)(None, None, None, None))
        opt = Options()
        L.grte_default_options(ctypes.byref(opt))
        opt.precision = precision
        self.hs = HandleS()
        st = L.grte_create(ctypes.byref(grid), ctypes.byref(quad), ctypes.byref(opac), a, c, Cv, eps,
                           ctypes.byref(bc), ctypes.byref(opt), ctypes.byref(self.hs))
        if st != GRTE_OK:
            raise GrteError(st, "grte_create failed")

    def set_initial(self, T):
        T = _f64(T)
        st = lib().grte_handle_set_initial(ctypes.byref(self.hs), _ptr(T), T.size)
        if st != GRTE_OK:
            raise GrteError(st, "grte_handle_set_initial failed")

    def step(self, n=1):
        return lib().grte_handle_step(ctypes.byref(self.hs), n)

    def sync(self):
        return lib().grte_handle_sync(ctypes.byref(self.hs))

    def T(self, allow=()):
        out = np.empty(self.hs.ncell)
        st = lib().grte_handle_get_T(ctypes.byref(self.hs), _ptr(out), out.size)
        if st != GRTE_OK and st not in allow:
            raise GrteError(st, "grte_handle_get_T failed")
        return out

    def close(self):
        if self.hs.dim:
            lib().grte_handle_destroy(ctypes.byref(self.hs))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Diffusion:
    """The three-stage diffusion solver of Sec. 2 (grte_diff_*): instances are dicts with
    nx, sigma, kind (SIGMA_CONST / SIGMA_T3), dt and optionally x0, x1, a, c, Cv, dd."""

    def __init__(self, instances, stream=None):
        L = lib()
        arr = (Diffusion1D * len(instances))()
        self._keep = []
        self.nx = []
        for i, p in enumerate(instances):
            sig = _f64(np.broadcast_to(p["sigma"], (p["nx"],)))
            self._keep.append(sig)
            arr[i] = Diffusion1D(p["nx"], _ptr(sig), p.get("kind", SIGMA_CONST), p.get("x0", 0.0), p.get("x1", 1.0),
                                 p["dt"], p.get("a", 1.0), p.get("c", 1.0), p.get("Cv", 1.0), p.get("dd", 0.0))
            self.nx.append(int(p["nx"]))
        h = ctypes.c_void_p()
        st = L.grte_diff_create(len(instances), arr, stream, ctypes.byref(h))
        self.h = h
        if st != GRTE_OK:
            msg = L.grte_diff_last_error(h).decode() if h.value else "create failed"
            L.grte_diff_destroy(h)
            self.h = None
            raise GrteError(st, msg)

    def _check(self, st, allow=()):
        if st != GRTE_OK and st not in allow:
            raise GrteError(st, lib().grte_diff_last_error(self.h).decode())
        return st

    def set_T(self, inst, T):
        T = _f64(T)
        return self._check(lib().grte_diff_set_T(self.h, inst, _ptr(T), T.size))

    def step(self, n=1):
        return self._check(lib().grte_diff_step(self.h, n))

    def sync(self, allow=()):
        return self._check(lib().grte_diff_sync(self.h), allow)

    def T(self, inst, allow=()):
        out = np.empty(self.nx[inst])
        self._check(lib().grte_diff_get_T(self.h, inst, _ptr(out), out.size), allow)
        return out

    def Ustar(self, inst, allow=()):
        out = np.empty(self.nx[inst])
        self._check(lib().grte_diff_get_Ustar(self.h, inst, _ptr(out), out.size), allow)
        return out

    def close(self):
        if self.h is not None:
            lib().grte_diff_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
