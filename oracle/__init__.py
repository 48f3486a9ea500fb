"""FP64 CPU oracle for band-limited PDE-constrained LDDMM with SL-RK integration.

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously-correct statement of
what the GPU library computes (arxiv 2006.06823, Secs. 2-3). Only the test suite, the
``smoke()`` check and the benchmark's CPU-baseline / reference arms may import it. The GPU
product path never imports, links or calls anything here, and this package imports nothing
from the GPU package. It shares no code with the CUDA path.

Modules
  spectral  band-limited projection pi, inclusion iota, spectral derivatives, L~ (Sec. 2.2)
  interp    trilinear and periodic cubic B-spline interpolation (Sec. 3.1, Sec. 4.2)
  sl        SL characteristics and the Table 1 transport equations, Heun (SL-RK) steps (Sec. 3)
  variants  energy, gradient and Gauss-Newton Hessian-vector products (Sec. 2.3.1-2.3.3)
  spatial   the three variants in the spatial domain (Sec. 2.1, SL-RK in Omega): velocity on
            the grid, spectral derivatives and L by numpy's FFT, voxel-mean L2 product
  gnk       PCG with preconditioner L~^-1, Gauss-Newton update, line search (Sec. 2.1-2.2)
  multilevel  two-level preconditioner (coarse half-grid Gauss-Newton solve on the low
            modes, L~^-1 on the rest) and flexible PCG (Secs. 6-7 name it as future work)

Parity status: every function here is pinned by a ``-m "not gpu"`` test against a closed
form, an invariant, a library routine or brute force. ``gnk.register`` is pinned as a driver
on quadratic model problems (each Gauss-Newton step meets its forcing term, the Armijo
halving lands on the closed-form step, the stop rules), but the registration it produces on
the LDDMM problem has no exact answer: parity unpinned beyond the pins on its parts
(objective, gradient-vs-finite-difference, Hessian symmetry, PCG closed form).
"""
