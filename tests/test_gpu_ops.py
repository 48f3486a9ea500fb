"""GPU parity of the stand-alone hot-path operators against the FP64 oracle (C ABI calls).

Tolerances: FP32 arithmetic against FP64; <= 1e-5 relative L2 per SL step (the stated
per-step bound), a few 1e-6 for the partial-DFT projection and inclusion (sums of at most
nx + ny + nz FP32 products with FP64-evaluated twiddles).
"""
import numpy as np
import pytest

from oracle import interp as I
from oracle import sl as SL
from oracle import spectral as S
from paper_2006_06823_b300 import synth
from _problems import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402

CASES = [((16, 16, 16), 8), ((20, 24, 36), 10), ((18, 22, 37), 12), ((33, 40, 64), 32),
         ((8, 8, 8), 4),
         ((64, 66, 64), 64),   # the largest band the library accepts (K = 64)
         # Y stages on the tensor cores: iota's in two blocks of 72 positions; K = 48
         ((20, 144, 32), 16), ((48, 112, 48), 48)]


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def devc(c):
    return torch.as_tensor(np.ascontiguousarray(c).astype(np.complex64), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64 if t.dtype == torch.float32 else np.complex128)


@pytest.mark.parametrize("shape,K", CASES)
@pytest.mark.parametrize("ncomp", [1, 3])
def test_bl_project_matches_oracle(shape, K, ncomp):
    f = synth.random_field(shape, seed=11, ncomp=ncomp)
    c = host(L.bl_project(dev(f), K))
    ref = S.project(f, K)
    assert rel_l2(c, ref) < 3e-6
    # Hermitian output, zero slot-0 planes
    np.testing.assert_allclose(S.hermitian_part(c), c, atol=1e-7 * np.abs(ref).max())
    assert np.abs(c[:, 0]).max() == 0 and np.abs(c[:, :, 0]).max() == 0 and np.abs(c[..., 0]).max() == 0


@pytest.mark.parametrize("shape,K", CASES)
@pytest.mark.parametrize("deriv", [-1, 0, 1, 2])
def test_bl_include_matches_oracle(shape, K, deriv):
    c = synth.random_coeffs(K, seed=12, ncomp=3, decay_power=0.5)
    f = host(L.bl_include(devc(c), shape, deriv_axis=deriv))
    src = c if deriv < 0 else np.stack([S.deriv(ci, deriv) for ci in c])
    assert rel_l2(f, S.include(src, shape)) < 3e-6


@pytest.mark.parametrize("shape,K", CASES[:3])
def test_bl_include_bspline_coefficients(shape, K):
    c = synth.random_coeffs(K, seed=13, ncomp=2)
    f = host(L.bl_include(devc(c), shape, bspline=True))
    ref = I.bspline_prefilter(S.include(c, shape))
    assert rel_l2(f, ref) < 3e-6


def test_projection_of_inclusion_is_identity_on_the_band():
    shape, K = (24, 28, 32), 16
    c = synth.random_coeffs(K, seed=14, ncomp=3)
    back = host(L.bl_project(L.bl_include(devc(c), shape), K))
    assert rel_l2(back, c) < 3e-6


@pytest.mark.parametrize("shape", [(16, 16, 16), (20, 24, 37)])
@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("direction", [1, -1])
def test_characteristics_match_oracle(shape, order, direction):
    V = synth.random_displacement(shape, seed=15, max_vox=12.0, smooth=3.0)
    D = host(L.sl_characteristics(dev(V), 0.2, direction, order))
    ref = SL.departure_offsets(V, 0.2, direction, order)
    assert rel_l2(D, ref) < 2e-6


@pytest.mark.parametrize("direction", [1, -1])
def test_interpolation_cells_of_the_departure_points_are_bit_exact(direction):
    """Index-valued result: the cell j + floor(D) each departure point falls in equals the
    oracle's wherever the fraction of D is not within 1e-4 of a cell boundary (the FP32 and
    FP64 offsets differ by ~1e-5 voxels, so only points that close to a boundary may differ)."""
    shape = (20, 24, 37)
    V = synth.random_displacement(shape, seed=15, max_vox=12.0, smooth=3.0)
    D = L.sl_characteristics(dev(V), 0.2, direction, 1).cpu().numpy().astype(np.float64)
    ref = SL.departure_offsets(V, 0.2, direction, 1)
    frac = ref - np.floor(ref)
    clear = (frac > 1e-4) & (frac < 1 - 1e-4)
    assert clear.mean() > 0.99
    assert np.array_equal(np.floor(D)[clear].astype(np.int64), np.floor(ref)[clear].astype(np.int64))


@pytest.mark.parametrize("shape", [(16, 16, 16), (20, 24, 37), (33, 40, 64)])
@pytest.mark.parametrize("order", [1, 3])
@pytest.mark.parametrize("direction", [1, -1])
@pytest.mark.parametrize("ncomp", [1, 3])
def test_sl_transport_matches_oracle(shape, order, direction, ncomp):
    nt = 5
    V = synth.random_displacement(shape, seed=16, max_vox=15.0, smooth=3.0)
    f = synth.random_field(shape, seed=17, ncomp=ncomp, smooth=1.5)
    out = host(L.sl_transport(dev(V), dev(f), nt, direction, order))
    ref = np.stack([SL.sl_transport(fc, V, nt, direction, order) for fc in f])
    assert rel_l2(out, ref) < nt * 1e-5


def test_zero_velocity_transport_is_bit_exact_identity():
    shape = (12, 10, 14)
    f = dev(synth.random_field(shape, seed=18))
    out = L.sl_transport(torch.zeros((3,) + shape, device="cuda"), f, 4, 1, L.INTERP_LINEAR)
    assert torch.equal(out, f)


def test_integer_constant_velocity_is_an_exact_roll():
    shape = (8, 6, 10)
    f = synth.random_field(shape, seed=19)
    nt = 4
    V = np.zeros((3,) + shape)
    V[0] += 2 * nt
    V[2] -= nt
    out = host(L.sl_transport(dev(V), dev(f), nt, 1, L.INTERP_LINEAR))
    np.testing.assert_array_equal(out, np.roll(f.astype(np.float32), (-nt, 2 * nt), axis=(1, 3)))


def test_transport_in_place_alias():
    shape = (16, 18, 20)
    V = dev(synth.random_displacement(shape, seed=20, max_vox=4.0))
    f = dev(synth.random_field(shape, seed=21, smooth=1.0))
    ref = L.sl_transport(V, f.clone(), 3, 1, L.INTERP_LINEAR)
    g = f.clone()
    L.sl_transport(V, g, 3, 1, L.INTERP_LINEAR, out=g)
    assert torch.equal(g, ref)


def test_invalid_arguments_raise():
    with pytest.raises(L.LddmmError):
        L.bl_project(torch.zeros((1, 8, 8, 8), device="cuda"), 10)  # K > n
    with pytest.raises(L.LddmmError):
        L.bl_project(torch.zeros((1, 8, 8, 8), device="cuda"), 5)   # odd K


# shapes that take the tensor-core x stages (K a multiple of 16, nx a multiple of 4; iota also
# needs nx a multiple of 16): ragged row counts, a partial last K chunk, K = 16 and 32
TC_CASES = [((33, 40, 64), 32), ((20, 24, 48), 16), ((40, 36, 100), 32), ((18, 20, 80), 16),
            ((34, 36, 256), 32),   # nx = 256: the shallower tensor-core rings
            ((64, 64, 64), 64)]    # pi's x stage with all 128 rows of the M = 128 A operand


@pytest.mark.parametrize("shape,K", TC_CASES)
@pytest.mark.parametrize("precision", [L.PREC_FP32, L.PREC_FP32_SIMT])
def test_bl_project_tensor_core_and_simt_paths_match_oracle(shape, K, precision):
    f = synth.random_field(shape, seed=51, ncomp=3)
    c = host(L.bl_project(dev(f), K, precision=precision))
    assert rel_l2(c, S.project(f, K)) < 3e-6
    assert L.device_error() == 0


@pytest.mark.parametrize("shape,K", TC_CASES)
@pytest.mark.parametrize("precision", [L.PREC_FP32, L.PREC_FP32_SIMT])
@pytest.mark.parametrize("deriv", [-1, 1])
def test_bl_include_tensor_core_and_simt_paths_match_oracle(shape, K, precision, deriv):
    c = synth.random_coeffs(K, seed=52, ncomp=3, decay_power=0.5)
    f = host(L.bl_include(devc(c), shape, deriv_axis=deriv, precision=precision))
    src = c if deriv < 0 else np.stack([S.deriv(ci, deriv) for ci in c])
    assert rel_l2(f, S.include(src, shape)) < 3e-6
    assert L.device_error() == 0


@pytest.mark.parametrize("shape,K", TC_CASES + [((96, 112, 96), 32)])
def test_bf16x3_projection_and_inclusion_error_is_bounded(shape, K):
    """Mixed-precision spectral path: BF16 hi + lo split products with FP32 accumulation.
    hi and lo each carry 8 mantissa bits, so the represented operands are exact to ~2^-17
    and the lo*lo product that the row-GEMM stages drop is ~2^-18 relative (pi's transposed x
    stage keeps it): results stay within ~1e-5 of FP64."""
    f = synth.random_field(shape, seed=53, ncomp=3)
    c = host(L.bl_project(dev(f), K, precision=L.PREC_BF16X3))
    e_pi = rel_l2(c, S.project(f, K))
    cc = synth.random_coeffs(K, seed=54, ncomp=3, decay_power=0.5)
    g = host(L.bl_include(devc(cc), shape, precision=L.PREC_BF16X3))
    e_io = rel_l2(g, S.include(cc, shape))
    assert e_pi < 5e-5 and e_io < 5e-5, (e_pi, e_io)
    assert L.device_error() == 0
