"""The allocation-free projection entry point (lddmm_bl_project_noalloc).

Some callers cannot let a library allocate device memory: a host framework that owns all
device memory through its own pool, a service held to a memory budget reserved up front,
or a latency-critical loop that cannot afford the allocator. For them the library offers
a projection that works in a fixed scratch array compiled into the library. This test
calls it through the C ABI twice in a row (different inputs, so stale contents of the
shared scratch would show) and compares each result with the regular, allocating
lddmm_bl_project at the same precision form, within the projection tolerance used by the
other GPU tests; every precision form the entry point accepts is covered, since each puts
different operand images and stage buffers into the fixed array. It also checks the
defining property: after a warm-up call (which takes the scratch address once), a call
leaves the high-water mark of the device's default memory pool where it was. The file is
named to run last, so a failure here does not hide the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402
from paper_2006_06823_b300 import synth  # noqa: E402

# relative L2 between the two entry points: the same kernels on the same inputs, so equal
# up to the order of the partial sums that do not depend on where the scratch lives
TOL = {L.PREC_FP32: 3e-6, L.PREC_BF16X3: 3e-6, L.PREC_FP32_SIMT: 3e-6}


def _project(fn, f, K, prec):
    C, nz, ny, nx = f.shape
    out = torch.empty((C, K, K, K), dtype=torch.complex64, device="cuda")
    rc = fn(nx, ny, nz, K, ctypes.c_void_p(f.data_ptr()), C, ctypes.c_void_p(out.data_ptr()),
            prec, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.OK, L.load().lddmm_last_error()
    return out


@pytest.mark.parametrize("prec", [L.PREC_FP32, L.PREC_BF16X3, L.PREC_FP32_SIMT])
@pytest.mark.parametrize("shape,K,ncomp", [((40, 48, 36), 16, 3), ((192, 224, 192), 32, 3)])
def test_noalloc_projection_matches_the_allocating_one_twice_in_a_row(shape, K, ncomp, prec):
    lib = L.load()
    for seed in (41, 42):
        f = torch.as_tensor(synth.random_field(shape, seed=seed, ncomp=ncomp),
                            dtype=torch.float32, device="cuda")
        ref = _project(lib.lddmm_bl_project, f, K, prec)
        got = _project(lib.lddmm_bl_project_noalloc, f, K, prec)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.linalg.norm(g - r) <= TOL[prec] * np.linalg.norm(r)


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcudart not found")


def test_noalloc_projection_takes_no_pool_memory():
    """UsedMemHigh of the device's default pool (the stream-ordered allocator's high-water
    mark) is reset after a warm-up call and read again after the measured call: the
    allocating projection raises it, the allocation-free one must not."""
    rt = _cudart()
    lib = L.load()
    shape, K = (96, 112, 96), 32
    f = torch.as_tensor(synth.random_field(shape, seed=5, ncomp=3), dtype=torch.float32,
                        device="cuda")
    out = torch.empty((3, K, K, K), dtype=torch.complex64, device="cuda")
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    USED_MEM_HIGH = 8                 # cudaMemPoolAttrUsedMemHigh

    def high_after(fn):
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, USED_MEM_HIGH, ctypes.byref(zero)) == 0
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        nz, ny, nx = shape
        rc = fn(nx, ny, nz, K, ctypes.c_void_p(f.data_ptr()), 3,
                ctypes.c_void_p(out.data_ptr()), L.PREC_FP32, st)
        assert rc == L.OK, lib.lddmm_last_error()
        torch.cuda.synchronize()
        high = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, USED_MEM_HIGH, ctypes.byref(high)) == 0
        return high.value

    _ = high_after(lib.lddmm_bl_project_noalloc)       # warm-up: takes the scratch address
    assert high_after(lib.lddmm_bl_project) > 0        # the pool does see the regular call
    assert high_after(lib.lddmm_bl_project_noalloc) == 0


def test_noalloc_projection_rejects_problems_beyond_its_scratch():
    lib = L.load()
    f = torch.zeros(16, device="cuda")
    rc = lib.lddmm_bl_project_noalloc(512, 512, 256, 32, ctypes.c_void_p(f.data_ptr()), 3,
                                      ctypes.c_void_p(f.data_ptr()), L.PREC_FP32, None)
    assert rc == L.EINVAL
    assert b"scratch" in lib.lddmm_last_error()
