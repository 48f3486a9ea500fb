"""The persistent batched SL transport (lddmm_sl_transport_batch): many pairs of different
grids in one cooperative launch. Each pair's result must equal the single-pair transport's bit
for bit (the same per-voxel arithmetic), and the single-pair transport has oracle parity; one
pair is also checked against the FP64 oracle directly. The bounded grid barrier is exercised
with its self-test form: the barrier waits for one block more than the launch has, every wait
runs out after its short bound, the call returns ETIMEOUT, and the next call works."""
import numpy as np
import pytest

from oracle import sl as SL
from paper_2006_06823_b300 import synth
from _problems import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402

GRIDS = [(16, 16, 16), (20, 24, 36), (33, 17, 40), (64, 64, 64), (8, 9, 10), (48, 40, 32)]


def _pairs(seed0=0):
    vels, fields = [], []
    for i, shape in enumerate(GRIDS):
        V = synth.random_displacement(shape, seed=seed0 + 2 * i, max_vox=6.0, smooth=3.0)
        f = synth.random_field(shape, seed=seed0 + 2 * i + 1, smooth=1.0)[0]
        vels.append(torch.as_tensor(V, dtype=torch.float32, device="cuda"))
        fields.append(torch.as_tensor(f, dtype=torch.float32, device="cuda"))
    return vels, fields


@pytest.mark.parametrize("nt,direction", [(5, L.FORWARD), (4, L.BACKWARD), (1, L.FORWARD)])
def test_batch_equals_the_single_pair_transport_bit_for_bit(nt, direction):
    vels, fields = _pairs()
    outs = L.sl_transport_batch(vels, fields, nt, direction)
    for v, f, o in zip(vels, fields, outs):
        ref = L.sl_transport(v, f, nt, direction, L.INTERP_LINEAR)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)


def test_batch_matches_the_oracle():
    vels, fields = _pairs(seed0=100)
    outs = L.sl_transport_batch(vels, fields, 3, L.FORWARD)
    for i in (0, 2):
        ref = SL.sl_transport(fields[i].cpu().numpy().astype(np.float64),
                              vels[i].cpu().numpy().astype(np.float64), 3, +1, 1)
        assert rel_l2(outs[i].cpu().numpy(), ref) < 3e-6


def test_inactive_pairs_are_left_untouched():
    vels, fields = _pairs(seed0=200)
    outs = [torch.full_like(f, 7.0) for f in fields]
    active = torch.tensor([1, 0, 1, 0, 1, 1], dtype=torch.int32, device="cuda")
    L.sl_transport_batch(vels, fields, 2, L.FORWARD, outs=outs, active=active)
    for i, (v, f, o) in enumerate(zip(vels, fields, outs)):
        if active[i]:
            assert torch.equal(o, L.sl_transport(v, f, 2, L.FORWARD, L.INTERP_LINEAR))
        else:
            assert bool((o == 7.0).all())


def test_barrier_wait_runs_out_and_the_next_call_works():
    vels, fields = _pairs(seed0=300)
    with pytest.raises(L.LddmmError) as e:
        L.sl_transport_batch(vels, fields, 2, L.FORWARD, wait_seconds=-0.05)
    assert e.value.code == L.ETIMEOUT
    outs = L.sl_transport_batch(vels, fields, 2, L.FORWARD)
    for v, f, o in zip(vels, fields, outs):
        assert torch.equal(o, L.sl_transport(v, f, 2, L.FORWARD, L.INTERP_LINEAR))
