"""Failure detection without a GPU fault: a device-side wait that nothing completes gives up
within its bound and reports LDDMM_ETIMEOUT through the device error word (the CUDA context
stays usable), and a workspace cap turns an over-budget context into LDDMM_ENOMEM before the
allocation is made."""
import time

import numpy as np
import pytest

from oracle import spectral as S
from paper_2006_06823_b300 import synth
from _problems import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402


def test_bounded_wait_gives_up_with_etimeout_and_the_context_stays_usable():
    assert L.device_error() == 0
    t0 = time.perf_counter()
    status = L.selftest_wait(0.05)
    elapsed = time.perf_counter() - t0
    assert status == L.ETIMEOUT
    assert elapsed >= 0.05
    assert L.device_error() == L.ETIMEOUT     # read and cleared ...
    assert L.device_error() == 0              # ... once
    # the context still runs the tensor-core kernels that use the same wait routine
    f = synth.random_field((16, 20, 32), seed=61, ncomp=3)
    c = L.bl_project(torch.as_tensor(f, dtype=torch.float32, device="cuda"), 16)
    assert rel_l2(c.cpu().numpy().astype(np.complex128), S.project(f, 16)) < 3e-6
    assert L.device_error() == 0


def test_workspace_limit_refuses_an_over_budget_context_and_admits_one_within_it():
    try:
        ctx = L.Context(16, 16, 16, 8, nt=4)
        need = ctx.workspace_bytes()
        ctx.close()
        assert need > 0
        L.set_workspace_limit(need - 1)
        with pytest.raises(L.LddmmError) as e:
            L.Context(16, 16, 16, 8, nt=4)
        assert e.value.code == L.ENOMEM
        L.set_workspace_limit(need)
        ctx = L.Context(16, 16, 16, 8, nt=4)
        assert ctx.workspace_bytes() == need
        # the coarse level of the two-level preconditioner is a context of its own, far smaller
        ctx.set_option(L.OPT_TWO_LEVEL, 2)
        ctx.close()
    finally:
        L.set_workspace_limit(0)
