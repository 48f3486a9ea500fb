"""Seeded problem builders shared by the tests (inputs from the generator and the oracle)."""
import numpy as np

from oracle import sl as SL
from oracle import spectral as S
from oracle import variants as Vn
from paper_2006_06823_b300 import synth


def scaled_velocity(K, K_gen, seed, shape, max_vox):
    """Random BL velocity scaled (with the oracle's iota) to max |v| = max_vox voxels."""
    vt = synth.random_velocity_coeffs(K, K_gen, seed)
    nz, ny, nx = shape
    v = S.include(vt, shape) * (np.array([nx, ny, nz]) / (2 * np.pi))[:, None, None, None]
    return vt * (max_vox / np.sqrt((v ** 2).sum(0)).max())


def voxel_velocity(vt, shape):
    nz, ny, nx = shape
    return S.include(vt, shape) * (np.array([nx, ny, nz]) / (2 * np.pi))[:, None, None, None]


def blob_pair(shape, K, seed=0, max_vox=3.0, order=1, nt_warp=10):
    """Small-workload pair: fixed = Gaussian blobs, moving = fixed warped by a random
    stationary BL velocity (8^3 modes, max displacement max_vox) with the oracle."""
    I1 = synth.gaussian_blobs(shape, seed=seed)
    vt = scaled_velocity(K, 8, seed + 1, shape, max_vox)
    I0 = SL.sl_transport(I1, voxel_velocity(vt, shape), nt_warp, +1, order)
    return I0, I1


def oracle_problem(shape, K, variant, order, nt=10, seed=0, sigma2=0.01):
    I0, I1 = blob_pair(shape, K, seed=seed, order=order)
    p = Vn.Params(K=K, nt=nt, order=order, variant=variant, sigma2=sigma2)
    return Vn.Problem(I0, I1, p)


# The bench-path parity workload: the paper-scale phantom recipe on a 96 x 112 x 96 grid (nx a
# multiple of 16, so the x stages of pi and iota run on the tensor cores), K = 32.
BENCH_SHAPE = (96, 112, 96)   # nz, ny, nx
BENCH_K = 32


def bench_phantom_problem(order, nt, noisy=True):
    """The ellipsoid phantom warped by a random band-limited velocity (8 nx / 192 voxels max
    displacement, the oracle's transport), with N(0, 0.01) noise on both images if `noisy`;
    deformation-state variant."""
    shape = BENCH_SHAPE
    nz, ny, nx = shape
    fixed = synth.ellipsoid_phantom(shape)
    vt = scaled_velocity(BENCH_K, BENCH_K, 1, shape, 8.0 * nx / 192)
    moving = SL.sl_transport(fixed, voxel_velocity(vt, shape), 10, +1, 1)
    I0 = synth.add_noise(moving, seed=2) if noisy else moving
    I1 = synth.add_noise(fixed, seed=3) if noisy else fixed
    return Vn.Problem(I0, I1, Vn.Params(K=BENCH_K, nt=nt, order=order, variant=Vn.DEFSTATE,
                                        sigma2=0.01))


def bench_velocity():
    """The velocity at which the bench-path gradient and Hessian are compared."""
    return scaled_velocity(BENCH_K, BENCH_K, 5, BENCH_SHAPE, 2.0)


def first_direction(g32, alpha, s):
    """The first PCG direction L~^{-1}(-g) of a Gauss-Newton step from a complex64 gradient,
    as the complex128 values of its complex64 rounding (what the GPU receives)."""
    p = S.apply_Linv(-np.asarray(g32, dtype=np.complex64).astype(np.complex128), alpha, s)
    return p.astype(np.complex64).astype(np.complex128)


def small_phantom_problem(order, nt, shape=(32, 32, 32), K=16):
    """The same recipe on a small grid (the registration follows the oracle there)."""
    nz, ny, nx = shape
    fixed = synth.ellipsoid_phantom(shape)
    vt = scaled_velocity(K, K, 1, shape, 8.0 * nx / 192)
    moving = SL.sl_transport(fixed, voxel_velocity(vt, shape), 10, +1, 1)
    I0 = synth.add_noise(moving, seed=2)
    I1 = synth.add_noise(fixed, seed=3)
    return Vn.Problem(I0, I1, Vn.Params(K=K, nt=nt, order=order, variant=Vn.DEFSTATE, sigma2=0.01))


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
