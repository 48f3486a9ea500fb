"""The BF16-storage transport (lddmm_sl_transport_bf16) against the FP64 oracle. Its error is
that of the storage roundings, bounded here from first principles: the field is rounded to
BF16 (relative 2^-9) after every step, and these errors are averaged, not amplified, by
trilinear interpolation, so they add up to at most about sqrt(nt) 2^-9 in relative L2 (a factor
2 is allowed for); BF16 offsets are off by up to 2^-9 |D| in every step, the same displacement
each step, which moves the result by nt 2^-9 max|D| voxels, i.e. a relative change of at most
nt 2^-9 max|D| rms|grad m| / rms|m|."""
import numpy as np
import pytest

from oracle import sl as SL
from paper_2006_06823_b300 import synth
from _problems import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402


@pytest.mark.parametrize("shape,nt", [((32, 40, 48), 10), ((33, 17, 40), 4)])
@pytest.mark.parametrize("offsets_bf16", [False, True])
def test_bf16_storage_transport_error_is_the_storage_roundings(shape, nt, offsets_bf16):
    V = synth.random_displacement(shape, seed=21, max_vox=6.0, smooth=3.0)
    f = synth.random_field(shape, seed=22, smooth=2.0)[0]
    ref = SL.sl_transport(f, V, nt, +1, 1)
    Vt = torch.as_tensor(V, dtype=torch.float32, device="cuda")
    ft = torch.as_tensor(f, dtype=torch.float32, device="cuda")
    out = L.sl_transport_bf16(Vt, ft, nt, L.FORWARD, offsets_bf16).cpu().numpy()
    fp32 = L.sl_transport(Vt, ft, nt, L.FORWARD, L.INTERP_LINEAR).cpu().numpy()
    u = 2.0 ** -9
    bound = 2 * np.sqrt(nt) * u
    if offsets_bf16:
        dmax = np.abs(SL.departure_offsets(V, 1.0 / nt, +1, 1)).max()
        g = np.stack(np.gradient(f))
        bound += nt * u * dmax * np.sqrt((g ** 2).sum(0).mean()) / np.sqrt((f ** 2).mean())
    err = rel_l2(out, ref)
    assert err < bound, (err, bound)
    assert rel_l2(out, fp32) < bound
    # the FP32-storage transport is far tighter: the BF16 form is measurably rounded
    assert rel_l2(fp32, ref) < 1e-5
