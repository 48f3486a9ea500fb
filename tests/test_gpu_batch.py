"""Batched registration, graph-captured Hessian products and the autotuner, through the C ABI.

Graph replay and block-shape choice change only how the same kernels are launched, so results
must match the eager single-pair path exactly (the reductions are deterministic)."""
import numpy as np
import pytest

from oracle import variants as Vn
from _problems import oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402


def _ctx(prob, stream=None, **kw):
    nz, ny, nx = prob.shape
    p = prob.p
    I0 = torch.as_tensor(prob.I0, dtype=torch.float32, device="cuda")
    I1 = torch.as_tensor(prob.I1, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    if stream is None:
        ctx = L.Context(nx, ny, nz, p.K, nt=p.nt, variant=p.variant, interp=p.order,
                        sigma2=p.sigma2, **kw)
        ctx.set_images(I0, I1)
    else:
        with torch.cuda.stream(stream):
            ctx = L.Context(nx, ny, nz, p.K, nt=p.nt, variant=p.variant, interp=p.order,
                            sigma2=p.sigma2, **kw)
            ctx.set_images(I0, I1)
    torch.cuda.synchronize()
    return ctx


PAIRS = [((16, 16, 16), 8, 0), ((20, 24, 16), 8, 1), ((16, 16, 16), 8, 2), ((24, 16, 20), 10, 3)]


def test_batch_matches_sequential_registrations():
    probs = [oracle_problem(s, K, Vn.DEFSTATE, 1, nt=4, seed=seed) for s, K, seed in PAIRS]
    seq = []
    for prob in probs:
        with _ctx(prob, max_gn=3, max_pcg=5) as ctx:
            v, rep = ctx.register()
            seq.append((v.cpu().numpy(), rep))
    streams = [torch.cuda.Stream() for _ in probs]
    ctxs = [_ctx(prob, st, max_gn=3, max_pcg=5) for prob, st in zip(probs, streams)]
    vs = [c.zeros_cube() for c in ctxs]
    torch.cuda.synchronize()
    reps = L.register_batch(ctxs, vs, max_threads=4)
    torch.cuda.synchronize()
    for (v0, r0), v1, r1 in zip(seq, vs, reps):
        assert r1["gn_iters"] == r0["gn_iters"] and r1["pcg_iters_total"] == r0["pcg_iters_total"]
        assert r1["E"] == pytest.approx(r0["E"], rel=1e-12)
        np.testing.assert_array_equal(v1.cpu().numpy(), v0)
    for c in ctxs:
        c.close()
    assert L.device_error() == 0


def test_graph_replay_and_autotuned_blocks_give_identical_registrations():
    prob = oracle_problem((24, 20, 28), 8, Vn.DEFSTATE, 1, nt=4, seed=5)
    with _ctx(prob, max_gn=2, max_pcg=6) as ctx:
        v0, r0 = ctx.register()
        v0 = v0.cpu().numpy()
        ctx.set_option(L.OPT_GRAPHS, 1)
        n0 = L.launch_count()
        v1, r1 = ctx.register()
        n1 = L.launch_count()
        bx = ctx.autotune()
        assert bx in (16, 32, 64, 128, 256)
        v2, r2 = ctx.register()
    np.testing.assert_array_equal(v1.cpu().numpy(), v0)
    np.testing.assert_array_equal(v2.cpu().numpy(), v0)
    assert r1["pcg_iters_total"] == r0["pcg_iters_total"] == r2["pcg_iters_total"]
    assert n1 - n0 > 100  # graph replays are counted as launches too


def test_autotune_cache_round_trip(tmp_path):
    prob = oracle_problem((16, 16, 16), 8, Vn.DEFSTATE, 1, nt=2, seed=6)
    path = str(tmp_path / "tune.json")
    with _ctx(prob) as ctx:
        bx = ctx.autotune(path)
    text = open(path).read()
    assert '"16x16x16/i1"' in text
    with _ctx(prob) as ctx:
        assert ctx.autotune(path) == bx
