"""Seeded synthetic inputs for the GRTE workloads (no scheme arithmetic here).

Every random input is drawn from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", 2014): state += 0x9E3779B97F4A7C15 and the output
mix z = (z ^ z>>30) * 0xBF58476D1CE4E5B9, z = (z ^ z>>27) * 0x94D049BB133111EB,
z ^ z>>31; uniform doubles are the top 53 bits times 2^-53.  The same stream feeds
the CUDA path and the CPU oracle, so both see identical inputs.

The workloads are the 1D slab problems of the paper's numerical section scaled to
the sizes measured here; see the recipe of each function.
"""
import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed):
        self.state = int(seed) & _MASK

    def next_u64(self):
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, n=None):
        """Uniform doubles in [0, 1)."""
        if n is None:
            return (self.next_u64() >> 11) * (1.0 / (1 << 53))
        # the same stream, n draws at once: state_k = state + k * golden (mod 2^64)
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * np.uint64(_GOLDEN)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * _GOLDEN) & _MASK
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))

    def normal(self, n):
        """Standard normals by Box-Muller."""
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:n]


BASE_SEED = 1811055790

SIGMA_CONST = 0   # sigma(x) independent of T
SIGMA_T3 = 1      # sigma_0(x) / T^3
BC_INFLOW = 0
BC_REFLECT = 1


@dataclass
class Instance1D:
    """Inputs of one 1D slab problem on [0, 1] (cells j = 0..nx-1)."""
    nx: int
    n_dir: int                 # total directions (+-v pairs): n_dir/2 positive angles
    eps: float
    dt: float
    sigma: np.ndarray          # (nx,) sigma(x) or sigma_0(x)
    T0: np.ndarray             # (nx,) initial temperature; I = a c T0^4 initially
    kind: int = SIGMA_T3
    bc: int = BC_INFLOW
    bL: float = 1.0            # isotropic inflow intensity I(0, v > 0) (a c 1^4 with a = c = 1)
    bR: float = 0.0            # isotropic inflow intensity I(1, v < 0)
    a: float = 1.0
    c: float = 1.0
    Cv: float = 1.0
    steps: int = 1
    name: str = ""
    length: float = 1.0        # slab [0, length]


def marshak_1d(nx=128, n_dir=16, eps=1e-3, sigma0=1.0, T_in=1e-2, cfl=0.5, t_end=0.5):
    """1D slab, sigma = sigma0/T^3, T_in everywhere, left inflow a c 1^4 for v > 0,
    right vacuum; dt = cfl * dx, run to t_end (128 cells, 16 directions, eps 1e-3:
    the Marshak-wave setting of the paper's nonlinear-opacity section at a small
    eps)."""
    dx = 1.0 / nx
    dt = cfl * dx
    return Instance1D(nx=nx, n_dir=n_dir, eps=eps, dt=dt, sigma=np.full(nx, sigma0),
                      T0=np.full(nx, T_in), kind=SIGMA_T3, bc=BC_INFLOW, bL=1.0, bR=0.0,
                      steps=int(round(t_end / dt)), name="marshak1d_nx%d_nv%d" % (nx, n_dir))


def marshak_dimensional(dt_s, nx=50, t_end_ns=0.02, n_dir=16):
    """The Marshak wave with units of the last example of Sec. 6: c = 29.98 cm/ns,
    a = 0.01372 GJ/(cm^3 keV^4), C_v = 0.3 GJ/(cm^3 keV), sigma = 300/T^3 cm^-1 (eps = 1),
    slab [0, 0.02] cm, T(0, t) = 1 keV (isotropic inflow a c 1^4), vacuum on the right,
    T(x, 0) = (1 - tanh(1000 (x - 0.0024)))/2 keV with I = a c T^4; time in ns, dt_s in
    seconds.  The paper gives neither dx nor the final time: nx = 50 (dx = 4e-4 cm) is a
    grid on which the oracle is stable at all three of its time steps."""
    L = 0.02
    a, c, Cv = 0.01372, 29.98, 0.3
    x = (np.arange(nx) + 0.5) * L / nx
    T0 = 0.5 * (1.0 - np.tanh((x - 0.0024) * 1000.0))
    dt = dt_s * 1e9
    return Instance1D(nx=nx, n_dir=n_dir, eps=1.0, dt=dt, sigma=np.full(nx, 300.0), T0=T0, kind=SIGMA_T3,
                      bc=BC_INFLOW, bL=a * c, bR=0.0, a=a, c=c, Cv=Cv, steps=int(round(t_end_ns / dt)),
                      name="marshak_dim_dt%.1e" % dt_s, length=L)


def smoothed_log_uniform_T(rng, nx, lo=1e-3, hi=1e-2, width=65, passes=3):
    """log10 T_j ~ U[log10 lo, log10 hi] iid, then `passes` centred box filters of
    `width` cells (clamped at the ends) on log10 T."""
    g = math.log10(lo) + (math.log10(hi) - math.log10(lo)) * rng.uniform(nx)
    h = width // 2
    for _ in range(passes):
        pad = np.concatenate([np.full(h, g[0]), g, np.full(h, g[-1])])
        cs = np.concatenate([[0.0], np.cumsum(pad)])
        g = (cs[width:] - cs[:-width]) / width
    return 10.0 ** g


def slab_1d_runs(nx=8192, n_dir=64, cfl=0.5, steps=10000, seed=None):
    """The six (sigma0, eps) runs: sigma0 in {1, 10} x eps in {1, 1e-2, 1e-4},
    sigma = sigma0/T^3, T_in log-uniform in [1e-3, 1e-2] then smoothed (one seeded
    field shared by the six runs), left inflow a c 1^4, right vacuum, dt = cfl dx."""
    rng = SplitMix64(BASE_SEED + 1 if seed is None else seed)
    T0 = smoothed_log_uniform_T(rng, nx)
    dx = 1.0 / nx
    out = []
    for sigma0 in (1.0, 10.0):
        for eps in (1.0, 1e-2, 1e-4):
            out.append(Instance1D(nx=nx, n_dir=n_dir, eps=eps, dt=cfl * dx,
                                  sigma=np.full(nx, sigma0), T0=T0.copy(), kind=SIGMA_T3,
                                  bc=BC_INFLOW, bL=1.0, bR=0.0, steps=steps,
                                  name="slab_s%g_e%g" % (sigma0, eps)))
    return out


def batched_1d(n_inst=256, seed=None, steps=1000, cfl=0.5, smooth_T=True,
               nx_range=(256, 8192), n_dirs=(16, 32, 64)):
    """Independent 1D instances of uneven sizes: nx = round(exp U[ln 256, ln 8192]),
    n_dir uniform over {16, 32, 64}, eps = 10^U[-5, 0], sigma0 ~ U[0.5, 50],
    sigma = sigma0/T^3, T_in smoothed log-uniform (or 1e-2 everywhere), dt = cfl dx."""
    rng = SplitMix64(BASE_SEED + 3 if seed is None else seed)
    out = []
    for i in range(n_inst):
        nx = int(round(math.exp(math.log(nx_range[0]) + (math.log(nx_range[1]) - math.log(nx_range[0])) * rng.uniform())))
        n_dir = n_dirs[min(int(rng.uniform() * len(n_dirs)), len(n_dirs) - 1)]
        eps = 10.0 ** (-5.0 + 5.0 * rng.uniform())
        sigma0 = 0.5 + 49.5 * rng.uniform()
        T0 = smoothed_log_uniform_T(rng, nx) if smooth_T else np.full(nx, 1e-2)
        out.append(Instance1D(nx=nx, n_dir=n_dir, eps=eps, dt=cfl / nx, sigma=np.full(nx, sigma0),
                              T0=T0, kind=SIGMA_T3, bc=BC_INFLOW, bL=1.0, bR=0.0, steps=steps,
                              name="batch%03d" % i))
    return out


def free_streaming_1d(nx=128, n_dir=16, seed=None, cfl=0.5):
    """sigma = 0, eps = 1, I_in(x, v) = sum_{m=1..3} alpha_m sin(2 pi m x + phi_m)(1+v)/2 + 1.5
    with alpha_m ~ U[0, 0.3], phi_m ~ U[0, 2 pi) seeded; left inflow I_in(0, v),
    right inflow I_in(1, -v).  Returns (instance, alpha, phi)."""
    rng = SplitMix64(BASE_SEED + 11 if seed is None else seed)
    alpha = 0.3 * rng.uniform(3)
    phi = 2 * np.pi * rng.uniform(3)
    dx = 1.0 / nx
    inst = Instance1D(nx=nx, n_dir=n_dir, eps=1.0, dt=cfl * dx, sigma=np.zeros(nx),
                      T0=np.ones(nx), kind=SIGMA_CONST, bc=BC_INFLOW, name="freestream")
    return inst, alpha, phi


def free_streaming_intensity(x, v, alpha, phi):
    """I_in(x, v) of free_streaming_1d (x, v broadcastable)."""
    s = 0.0
    for m in range(3):
        s = s + alpha[m] * np.sin(2 * np.pi * (m + 1) * x + phi[m])
    return s * (1.0 + v) / 2.0 + 1.5


def random_state_1d(rng, nx, M, scale_T=(0.05, 1.0)):
    """Generic non-equilibrium seeded state for parity tests: T log-uniform in
    scale_T, E = T^4 (1 + 0.1 u), O = 0.2 (u - 1/2) with u uniform."""
    lo, hi = scale_T
    T = 10.0 ** (math.log10(lo) + (math.log10(hi) - math.log10(lo)) * rng.uniform(nx))
    E = (T ** 4)[:, None] * (1.0 + 0.1 * rng.uniform(nx * M).reshape(nx, M))
    O = 0.2 * (rng.uniform((nx + 1) * M).reshape(nx + 1, M) - 0.5)
    return T, E, O


# ----------------------------------------------------------------------------- 2D

def checkerboard_sigma_2d(nx, ny=None, blocks=8, lo=1.0, hi=100.0):
    """sigma_0 per cell ([j][i], row-major) of the 2D checkerboard: lo on the 'black',
    hi on the 'white' blocks of a blocks x blocks board, block (0, 0) black."""
    ny = nx if ny is None else ny
    i = np.arange(nx) // max(nx // blocks, 1)
    j = np.arange(ny) // max(ny // blocks, 1)
    return np.where(((i[None, :] + j[:, None]) % 2) == 0, lo, hi).astype(np.float64)


def lognormal_sigma_2d(n, seed=BASE_SEED + 5, sd_cells=8.0):
    """sigma_0 per cell of the random-smooth 2D workload: exp(g), where g is an iid
    N(0, 1) field on the periodic n x n grid, filtered by a separable Gaussian of
    standard deviation sd_cells (taps to 4 sd, wrapped), then shifted and scaled to
    zero mean and unit variance, so that sigma_0 is log-normal with mu = 0, s = 1."""
    z = SplitMix64(seed).normal(n * n).reshape(n, n)
    r = int(math.ceil(4 * sd_cells))
    taps = np.exp(-0.5 * (np.arange(-r, r + 1) / sd_cells) ** 2)
    taps /= taps.sum()
    for ax in (0, 1):
        z = sum(t * np.roll(z, d, axis=ax) for d, t in zip(range(-r, r + 1), taps))
    g = (z - z.mean()) / z.std()
    return np.exp(g)
