"""Parity at the paper-scale grid (192 x 224 x 192, K = 32) in the benchmark's launch
configuration, on outputs the oracle computes one by one (sampled modes and voxels) or on
a single full-grid step."""
import numpy as np
import pytest

from oracle import sl as SL
from paper_2006_06823_b300 import synth
from _problems import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2006_06823_b300 as L  # noqa: E402

SHAPE = (192, 224, 192)   # nz, ny, nx
K = 32


def _coords():
    nz, ny, nx = SHAPE
    return (2 * np.pi * np.arange(nx) / nx, 2 * np.pi * np.arange(ny) / ny,
            2 * np.pi * np.arange(nz) / nz)


def test_projection_sampled_modes():
    f = synth.random_field(SHAPE, seed=31)[0]
    c = L.bl_project(torch.as_tensor(f, dtype=torch.float32, device="cuda"), K)[0].cpu().numpy()
    xs, ys, zs = _coords()
    rng = synth.rng(32)
    h = K // 2
    modes = [(h, h, h), (1, 1, 1), (K - 1, K - 1, K - 1), (h, 1, K - 1)]
    modes += [tuple(rng.integers(1, K, 3)) for _ in range(8)]
    for jz, jy, jx in modes:
        kx, ky, kz = jx - h, jy - h, jz - h
        # the definition: mean over voxels of f e^{-i k.x}, summed one mode at a time
        ex = np.exp(-1j * kx * xs)[None, None, :]
        ey = np.exp(-1j * ky * ys)[None, :, None]
        ez = np.exp(-1j * kz * zs)[:, None, None]
        ref = np.mean(f * ex * ey * ez)
        # the x and Y stages add in the tensor core's FP32 accumulator: the mean mode (k = 0,
        # 8.3M same-sign terms) carries up to 3.3e-6 relative, every other mode less
        assert abs(c[jz, jy, jx] - ref) < 4e-6 * max(abs(ref), np.abs(f).mean() * 1e-2), (jz, jy, jx)


def test_inclusion_sampled_voxels():
    c = synth.random_coeffs(K, seed=33, ncomp=1, decay_power=0.5)[0]
    f = L.bl_include(torch.as_tensor(c.astype(np.complex64), device="cuda"), SHAPE)[0].cpu().numpy()
    rng = synth.rng(34)
    nz, ny, nx = SHAPE
    idx = np.stack([rng.integers(0, n, 300) for n in (nz, ny, nx)], 1)
    h = K // 2
    k = np.arange(K) - h
    sel = np.argwhere(np.ones((K, K, K), bool)[1:, 1:, 1:]) + 1
    coef = c[sel[:, 0], sel[:, 1], sel[:, 2]]
    kz, ky, kx = k[sel[:, 0]], k[sel[:, 1]], k[sel[:, 2]]
    for z, y, x in idx:
        phase = kx * 2 * np.pi * x / nx + ky * 2 * np.pi * y / ny + kz * 2 * np.pi * z / nz
        ref = np.real(np.sum(coef * np.exp(1j * phase)))
        assert abs(f[z, y, x] - ref) < 2e-6 * np.abs(c).sum() ** 0.5 + 1e-6 * abs(ref)


def test_transport_one_full_grid_step():
    V = synth.random_displacement(SHAPE, seed=35, max_vox=8.0, smooth=6.0)
    f = synth.ellipsoid_phantom(SHAPE)
    Vt = torch.as_tensor(V, dtype=torch.float32, device="cuda")
    ft = torch.as_tensor(f, dtype=torch.float32, device="cuda")
    out = L.sl_transport(Vt, ft, 1, L.FORWARD, L.INTERP_LINEAR).cpu().numpy()
    ref = SL.sl_transport(f, V, 1, +1, 1)
    assert rel_l2(out, ref) < 1e-5


def test_mixed_precision_256_phantom():
    """Mixed-precision forms on a 256^3 phantom (the paper-scale recipe on a cubic grid):
    pi and iota in each spectral precision against the FP64 oracle's (numpy-FFT) pi/iota, and
    one registration per form with its GN / PCG counts and final energy against the plain
    FP32 form. With LDDMM_REPORT_DIR set the numbers go to mixed_precision_256.json."""
    import json
    import os
    from oracle import spectral as S
    shape = (256, 256, 256)
    nz, ny, nx = shape
    fixed = synth.ellipsoid_phantom(shape)
    fd = torch.as_tensor(fixed, dtype=torch.float32, device="cuda")
    ref_c = S.project(fixed, K)
    ref_f = S.include(ref_c, shape)
    out = {"operators": {}, "registration": {}}
    for name, prec in (("fp32_tensor", L.PREC_FP32), ("fp32_simt", L.PREC_FP32_SIMT),
                       ("bf16x3", L.PREC_BF16X3)):
        c = L.bl_project(fd, K, precision=prec)[0].cpu().numpy().astype(np.complex128)
        f = L.bl_include(torch.as_tensor(ref_c.astype(np.complex64), device="cuda")[None], shape,
                         precision=prec)[0].cpu().numpy().astype(np.float64)
        out["operators"][name] = {"pi_rel_l2": rel_l2(c, ref_c), "iota_rel_l2": rel_l2(f, ref_f)}
    for name, r in out["operators"].items():
        bound = 5e-5 if name == "bf16x3" else 3e-6
        assert r["pi_rel_l2"] < bound and r["iota_rel_l2"] < bound, (name, r)
    # moving = phantom transported along a random band-limited velocity (8 voxels max)
    vt = synth.random_velocity_coeffs(K, K, seed=1)
    v = L.bl_include(torch.as_tensor(vt.astype(np.complex64), device="cuda"), shape)
    V = v * (torch.tensor([nx, ny, nz], dtype=torch.float32, device="cuda").view(3, 1, 1, 1)
             / (2 * np.pi))
    V *= 8.0 / V.pow(2).sum(0).sqrt().max()
    moving = L.sl_transport(V, fd, 10, L.FORWARD, L.INTERP_LINEAR)
    for name, prec in (("fp32_simt", L.PREC_FP32_SIMT), ("fp32_tensor", L.PREC_FP32),
                       ("bf16x3", L.PREC_BF16X3), ("bf16x3_jbf16", L.PREC_BF16X3_JBF16)):
        with L.Context(nx, ny, nz, K, nt=10, variant=L.V_DEFSTATE, interp=L.INTERP_LINEAR,
                       max_gn=10, max_pcg=20, gtol=1e-3, precision=prec) as ctx:
            ctx.set_images(moving, fd)
            _, rep = ctx.register()
        out["registration"][name] = {k: rep[k] for k in ("gn_iters", "pcg_iters_total", "E",
                                                         "grad_rel_l2", "seconds")}
    base = out["registration"]["fp32_simt"]
    for name, r in out["registration"].items():
        r["E_rel_diff_vs_fp32_simt"] = abs(r["E"] - base["E"]) / abs(base["E"])
    rd = os.environ.get("LDDMM_REPORT_DIR")
    if rd:
        os.makedirs(rd, exist_ok=True)
        json.dump(out, open(os.path.join(rd, "mixed_precision_256.json"), "w"), indent=1)
    for name, r in out["registration"].items():
        assert r["E_rel_diff_vs_fp32_simt"] < 1e-3, (name, r)
