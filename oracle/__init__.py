"""Plain serial FP64 CPU oracle for the AP prediction/correction/projection scheme.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, links or runs anything in this package.  Only the tests,
`__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference` legs of
`bench.py` may use it.

Each module follows the paper (Tang, Wang, Zhang, "Accurate front capturing
asymptotic preserving scheme for nonlinear gray radiative transfer equation",
arXiv:1811.05579) and cites the section / equation it writes out:

  quadrature  - angular quadrature sets (velocity discretisation of Sec. 4):
                Gauss-Legendre in 1D, level-symmetric S8 pairs in 2D
  scalar      - the per-cell quartic of the correction step (Eq. Tnp1)
  grte1d      - Algorithm 2 (Sec. 4) and its sigma/T^3 form (Sec. 5) in 1D, the latter
                for a general exponent sigma_0/T^p
  grte2d      - the same scheme on a 2D grid (direction by direction, Sec. 4; the
                reading of the 2D discretisation is in that module's header)
  diffusion1d - the three-stage diffusion solver (Sec. 2, Eq. dis-diff) and the
                fully implicit limit solvers (Sec. 6, Eq. imp_T and diff_solver)
  mlp         - the network of the learned Newton start in FP64, in its BF16 form
                (weights and every product's operands rounded to bfloat16, as the
                library's tensor-core kernels compute it; forward and gradient)

The linear systems are solved exactly by direct elimination (block-tridiagonal
Gaussian elimination, sparse LU); iterative solvers are not used anywhere here.
"""
