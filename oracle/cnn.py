"""FP64 reference of the warm-start network's layers (3-D convolutions and friends).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The learned warm start has no basis in the paper; this module is the plain statement of the
layers the GPU network uses, so that its forward pass and its gradients can be checked:
  conv3x3x3 with zero padding:  out[co][x] = b[co] + sum_{ci, t} w[co][ci][t] in[ci][x + o(t)]
  its input gradient:           din[ci][x] = sum_{co, t} w[co][ci][t] dout[co][x - o(t)]
  its weight gradient:          dw[co][ci][t] = sum_x dout[co][x] in[ci][x + o(t)]
  2x average pooling, 2x nearest upsampling, ReLU, mean squared error.
Arrays are [C][D][D][D] (one sample) or [B][C][D][D][D]; tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)
for offsets o(t) = (dz, dy, dx) in {-1, 0, 1}^3.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x, dz, dy, dx):
    """y[.., z, y, x] = x[.., z + dz, y + dy, x + dx] with zeros outside the volume."""
    out = np.zeros_like(x)
    D0, D1, D2 = x.shape[-3:]

    def sl(d, n):  # (destination, source) ranges along one axis
        if d >= 0:
            return slice(0, n - d), slice(d, n)
        return slice(-d, n), slice(0, n + d)

    (oz, iz), (oy, iy), (ox, ix) = sl(dz, D0), sl(dy, D1), sl(dx, D2)
    out[..., oz, oy, ox] = x[..., iz, iy, ix]
    return out


def conv3d(x, w, b=None):
    """x [Cin][D^3], w [Cout][Cin][27] -> [Cout][D^3] (zero padding, stride 1)."""
    x = np.asarray(x, dtype=np.float64)
    cout = w.shape[0]
    out = np.zeros((cout,) + x.shape[1:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        xs = _shift(x, dz, dy, dx)
        out += np.tensordot(w[:, :, t], xs, axes=(1, 0))
    if b is not None:
        out += b[:, None, None, None]
    return out


def conv3d_dgrad(dout, w):
    """Gradient of sum(dout * conv3d(x, w)) with respect to x."""
    din = np.zeros((w.shape[1],) + dout.shape[1:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        din += _shift(np.tensordot(w[:, :, t].T, dout, axes=(1, 0)), -dz, -dy, -dx)
    return din


def conv3d_wgrad(dout, x):
    """Gradient of sum(dout * conv3d(x, w)) with respect to w ([Cout][Cin][27]) and b."""
    dw = np.zeros((dout.shape[0], x.shape[0], 27))
    for t, (dz, dy, dx) in enumerate(TAPS):
        dw[:, :, t] = np.tensordot(dout, _shift(x, dz, dy, dx), axes=([1, 2, 3], [1, 2, 3]))
    return dw, dout.sum(axis=(1, 2, 3))


def conv3d_loops(x, w, b):
    """conv3d by explicit loops over every output voxel (tiny inputs; a pin for conv3d)."""
    cin, D0, D1, D2 = x.shape
    out = np.zeros((w.shape[0], D0, D1, D2))
    for co in range(w.shape[0]):
        for z in range(D0):
            for y in range(D1):
                for xx in range(D2):
                    s = b[co]
                    for t, (dz, dy, dx) in enumerate(TAPS):
                        zz, yy, xi = z + dz, y + dy, xx + dx
                        if 0 <= zz < D0 and 0 <= yy < D1 and 0 <= xi < D2:
                            s += np.dot(w[co, :, t], x[:, zz, yy, xi])
                    out[co, z, y, xx] = s
    return out


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x):
    C, D0, D1, D2 = x.shape
    return x.reshape(C, D0 // 2, 2, D1 // 2, 2, D2 // 2, 2).mean(axis=(2, 4, 6))


def avgpool2_grad(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 1), 2, 2), 2, 3) / 8.0


def upsample2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 1), 2, 2), 2, 3)


def upsample2_grad(dy):
    C, D0, D1, D2 = dy.shape
    return dy.reshape(C, D0 // 2, 2, D1 // 2, 2, D2 // 2, 2).sum(axis=(2, 4, 6))


# ---------------------------------------------------------------- the warm-start network
def layer_specs(base_channels=16):
    """(name, cin, cout) of the 13 convolutions, in forward order (levels 0..3 down, 2..0 up)."""
    c = base_channels
    return [("e0a", 2, c), ("e0b", c, c), ("e1a", c, 2 * c), ("e1b", 2 * c, 2 * c),
            ("e2a", 2 * c, 4 * c), ("e2b", 4 * c, 4 * c), ("e3a", 4 * c, 8 * c),
            ("e3b", 8 * c, 8 * c), ("d2a", 12 * c, 4 * c), ("d2b", 4 * c, 4 * c),
            ("d1a", 6 * c, 2 * c), ("d1b", 2 * c, 2 * c), ("out", 2 * c, 3)]


def round_bf16(a):
    """Round to the nearest bfloat16 value (8 significant bits, ties to even), returned as
    float64. Written from the format's definition: keep the top 16 bits of the IEEE float32
    pattern after adding 0x7FFF plus the lowest kept bit."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x, storage=None):
    """Network forward for one sample x [2][D^3] (D divisible by 8). Returns (y, cache):
    y [3][(D/2)^3], the velocity on the half-resolution grid (no activation on the output).

    storage="bf16" models a network that stores its input and every activation it keeps
    (ReLU outputs, pooled maps; upsampling copies) in bfloat16, each rounded once from the
    exact value; the output stays unrounded. storage=None is the FP64 network."""
    P = params
    cache = {}
    R = round_bf16 if storage == "bf16" else (lambda a: a)

    def cv(name, inp, act=True):
        pre = conv3d(inp, P[name + ".w"], P[name + ".b"])
        cache[name] = (inp, pre)
        return R(relu(pre)) if act else pre

    x = R(x)
    e0 = cv("e0b", cv("e0a", x))                    # D
    e1 = cv("e1b", cv("e1a", R(avgpool2(e0))))      # D/2
    e2 = cv("e2b", cv("e2a", R(avgpool2(e1))))      # D/4
    e3 = cv("e3b", cv("e3a", R(avgpool2(e2))))      # D/8
    d2 = cv("d2b", cv("d2a", np.concatenate([upsample2(e3), e2])))   # D/4
    d1 = cv("d1b", cv("d1a", np.concatenate([upsample2(d2), e1])))   # D/2
    y = cv("out", d1, act=False)
    cache["shapes"] = (e0.shape, e1.shape, e2.shape, e3.shape)
    return y, cache


def backward(params, cache, dy):
    """Gradients of sum(dy * y) for every parameter (dict name -> array)."""
    P = params
    g = {}

    def bcv(name, dout, act=True):
        inp, pre = cache[name]
        if act:
            dout = dout * (pre > 0)
        dw, db = conv3d_wgrad(dout, inp)
        g[name + ".w"], g[name + ".b"] = dw, db
        return conv3d_dgrad(dout, P[name + ".w"])

    c4 = cache["e3b"][1].shape[0]
    dd1 = bcv("d1a", bcv("d1b", bcv("out", dy, act=False)))
    c_up1 = cache["d2b"][1].shape[0]
    dd2_up, de1 = dd1[:c_up1], dd1[c_up1:]
    dd2 = bcv("d2a", bcv("d2b", upsample2_grad(dd2_up)))
    de3_up, de2 = dd2[:c4], dd2[c4:]
    de3 = bcv("e3a", bcv("e3b", upsample2_grad(de3_up)))
    de2 = de2 + avgpool2_grad(de3)
    de2 = bcv("e2a", bcv("e2b", de2))
    de1 = de1 + avgpool2_grad(de2)
    de1 = bcv("e1a", bcv("e1b", de1))
    de0 = avgpool2_grad(de1)
    bcv("e0a", bcv("e0b", de0))
    return g


def init_params(seed_rng, base_channels=16):
    """He-style initialisation (random numbers come from the caller's generator)."""
    P = {}
    for name, cin, cout in layer_specs(base_channels):
        std = np.sqrt(2.0 / (cin * 27))
        P[name + ".w"] = seed_rng.standard_normal((cout, cin, 27)) * std
        P[name + ".b"] = np.zeros(cout)
    return P


def mse(y, target):
    """Mean squared error and its gradient with respect to y."""
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size
