"""The allocation-free projection entry point (lddmm_bl_project_noalloc).

Some callers cannot let a library allocate device memory: a host framework that owns all
device memory through its own pool, a service held to a memory budget reserved up front,
or a latency-critical loop that cannot afford the allocator. For them the library offers
a projection that works in a fixed scratch array compiled into the library. This test
calls it through the C ABI twice in a row (different inputs, so stale contents of the
shared scratch would show) and compares each result with the regular, allocating
lddmm_bl_project, within the projection tolerance used by the other GPU tests. The file is
named to run last, so a failure here does not hide the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402
from paper_2006_06823_b300 import synth  # noqa: E402


def _project(fn, f, K):
    C, nz, ny, nx = f.shape
    out = torch.empty((C, K, K, K), dtype=torch.complex64, device="cuda")
    rc = fn(nx, ny, nz, K, ctypes.c_void_p(f.data_ptr()), C, ctypes.c_void_p(out.data_ptr()),
            L.PREC_FP32, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.OK, L.load().lddmm_last_error()
    return out


@pytest.mark.parametrize("shape,K,ncomp", [((40, 48, 36), 16, 3), ((192, 224, 192), 32, 3)])
def test_noalloc_projection_matches_the_allocating_one_twice_in_a_row(shape, K, ncomp):
    lib = L.load()
    for seed in (41, 42):
        f = torch.as_tensor(synth.random_field(shape, seed=seed, ncomp=ncomp),
                            dtype=torch.float32, device="cuda")
        ref = _project(lib.lddmm_bl_project, f, K)
        got = _project(lib.lddmm_bl_project_noalloc, f, K)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.linalg.norm(g - r) <= 3e-6 * np.linalg.norm(r)


def test_noalloc_projection_rejects_problems_beyond_its_scratch():
    lib = L.load()
    f = torch.zeros(16, device="cuda")
    rc = lib.lddmm_bl_project_noalloc(512, 512, 256, 32, ctypes.c_void_p(f.data_ptr()), 3,
                                      ctypes.c_void_p(f.data_ptr()), L.PREC_FP32, None)
    assert rc == L.EINVAL
    assert b"scratch" in lib.lddmm_last_error()
