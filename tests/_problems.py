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


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
