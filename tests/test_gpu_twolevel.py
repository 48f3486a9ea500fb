"""GPU parity of the two-level preconditioner (LDDMM_OPT_TWO_LEVEL: a half-grid Gauss-Newton
solve on the low modes, scaled L~^{-1} on the rest, flexible outer PCG; the multi-level
preconditioner Secs. 6-7 name as the way to a faster PCG of Sec. 2.2) against the oracle's
``gnk.register(two_level=m)``, through the C ABI."""
import numpy as np
import pytest

from oracle import gnk
from oracle import variants as Vn
from _problems import oracle_problem

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def context(prob, images=True, **kw):
    nz, ny, nx = prob.shape
    p = prob.p
    ctx = L.Context(nx, ny, nz, p.K, nt=p.nt, variant=p.variant, interp=p.order, alpha=p.alpha,
                    s=p.s, sigma2=p.sigma2, **kw)
    if images:
        ctx.set_images(dev(prob.I0), dev(prob.I1))
    return ctx


# a non-cubic grid (coarse 10 x 12 x 8) checks the axes of the image restriction
CASES = [((16, 16, 16), Vn.DEFSTATE, 1), ((16, 16, 16), Vn.IMAGE, 1),
         ((16, 24, 20), Vn.DEFSTATE, 3), ((16, 24, 20), Vn.STATE, 1)]


@pytest.mark.parametrize("shape,variant,order", CASES)
def test_two_level_registration_matches_oracle(shape, variant, order):
    prob = oracle_problem(shape, 8, variant, order, nt=5)
    v_o, rep_o = gnk.register(prob, max_gn=3, max_pcg=5, two_level=4)
    with context(prob, max_gn=3, max_pcg=5) as ctx:
        ctx.set_option(L.OPT_TWO_LEVEL, 4)
        v, rep = ctx.register()
    assert rep_o.pcg_inner_total > 0
    assert rep["gn_iters"] == rep_o.gn_iters
    assert rep["pcg_iters_total"] == rep_o.pcg_iters_total
    assert rep["pcg_inner_total"] == rep_o.pcg_inner_total
    assert rep["stop_reason"] == rep_o.stop_reason
    assert rep["E"] == pytest.approx(rep_o.E, rel=1e-3)
    assert rep["mse_rel"] == pytest.approx(rep_o.mse_rel, rel=1e-3)


def test_option_order_and_switching_off():
    """Images set before or after the option give the same result (the coarse images follow
    lddmm_set_images); value 0 returns to the spectral preconditioner bit for bit."""
    prob = oracle_problem((16, 16, 16), 8, Vn.DEFSTATE, 1, nt=4)
    kw = dict(max_gn=2, max_pcg=4)
    with context(prob, images=False, **kw) as a, context(prob, **kw) as b, \
            context(prob, **kw) as plain:
        a.set_option(L.OPT_TWO_LEVEL, 3)
        a.set_images(dev(prob.I0), dev(prob.I1))
        b.set_option(L.OPT_TWO_LEVEL, 3)
        va, ra = a.register()
        vb, rb = b.register()
        assert torch.equal(va, vb)
        assert (ra["pcg_iters_total"], ra["pcg_inner_total"]) == (rb["pcg_iters_total"],
                                                                   rb["pcg_inner_total"])
        b.set_option(L.OPT_TWO_LEVEL, 0)
        vb0, rb0 = b.register()
        vp, rp = plain.register()
        assert torch.equal(vb0, vp)
        assert rb0["pcg_inner_total"] == 0 and rb0["pcg_iters_total"] == rp["pcg_iters_total"]


@pytest.mark.parametrize("kw,value", [
    (dict(spatial=True), 2),            # band-limited only
    (dict(nonstationary=True), 2),      # stationary only
    (dict(K=6), 2),                     # K >= 8
    (dict(), -1), (dict(), 1001),       # value range
])
def test_option_validation(kw, value):
    K = kw.pop("K", 8)
    ctx = L.Context(16, 16, 16, K, nt=4, **kw)
    with pytest.raises(L.LddmmError) as e:
        ctx.set_option(L.OPT_TWO_LEVEL, value)
    assert e.value.code == L.EINVAL
    ctx.set_option(L.OPT_GRAPHS, 1)     # the context stays usable
    ctx.close()


def test_odd_grid_is_refused():
    ctx = L.Context(16, 17, 16, 8, nt=4)
    with pytest.raises(L.LddmmError) as e:
        ctx.set_option(L.OPT_TWO_LEVEL, 2)
    assert e.value.code == L.EINVAL
    ctx.close()


def test_batch_with_two_level_matches_sequential_registrations():
    """lddmm_register_batch runs each pair's coarse level on that pair's stream: results equal
    the sequential two-level registrations bit for bit."""
    probs = [oracle_problem((16, 16, 16), 8, Vn.DEFSTATE, 1, nt=4, seed=0),
             oracle_problem((16, 24, 20), 8, Vn.IMAGE, 1, nt=4, seed=1)]
    kw = dict(max_gn=2, max_pcg=4)
    seq = []
    for prob in probs:
        with context(prob, **kw) as ctx:
            ctx.set_option(L.OPT_TWO_LEVEL, 3)
            v, rep = ctx.register()
            seq.append((v.cpu().numpy(), rep))
    streams = [torch.cuda.Stream() for _ in probs]
    ctxs = []
    for prob, st in zip(probs, streams):
        with torch.cuda.stream(st):
            ctx = context(prob, **kw)
            ctx.set_option(L.OPT_TWO_LEVEL, 3)
        ctxs.append(ctx)
    vs = [c.zeros_cube() for c in ctxs]
    torch.cuda.synchronize()
    reps = L.register_batch(ctxs, vs, max_threads=2)
    torch.cuda.synchronize()
    for (v0, r0), v1, r1 in zip(seq, vs, reps):
        assert (r1["pcg_iters_total"], r1["pcg_inner_total"]) == (r0["pcg_iters_total"],
                                                                   r0["pcg_inner_total"])
        np.testing.assert_array_equal(v1.cpu().numpy(), v0)
    for c in ctxs:
        c.close()
    assert L.device_error() == 0
