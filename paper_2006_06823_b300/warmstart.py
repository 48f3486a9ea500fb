"""Learned Gauss-Newton warm start: training data, training and evaluation.

The paper's solver starts every registration from v~ = 0. Here a 3-D convolutional
encoder-decoder (``Net``, kernels in ``csrc/cnn.cu``) is trained on registrations that the
plain method itself produces, and its prediction is handed to the same solver as the
initial velocity. The solver always finishes the job; its stopping test keeps the
cold-start reference ||g(0)|| (the library computes it when the initial velocity is not
zero), so a warm start has to reach the same relative residual as a cold one.

Two workloads. ``phantom``: the paper-scale recipe itself (the noisy ellipsoid phantom of
the benchmark, moving = phantom transported along a random 32^3-mode band-limited velocity of
8 voxels maximum displacement, N(0, 0.01) noise on both images; velocity seed s, noise seeds
s + 1, s + 2). ``blobs`` (the default, noise-free):

Workload (the small workload's recipe scaled to the paper-scale grid): the fixed image is
the Gaussian-blob phantom (``synth.gaussian_blobs`` scaled to the grid), the moving image
is the fixed one transported by the library for nt steps along a random stationary
band-limited velocity (8^3 generated modes, decay (1 + |k|^2)^-2) scaled to a maximum
displacement of 8 voxels (the paper-scale workload's displacement). Every pair comes from
one seed. Targets are iota_{(D/2)^3}(v~_GN), the solver's solution on the network's output
grid (exact: the band K <= D/2 fits that grid), inputs the band-limited resampling of the
pair to D^3.

    python -m paper_2006_06823_b300.warmstart --train-pairs 1000 --eval-pairs 200 --out DIR

writes DIR/warmstart_params.npz (weights), DIR/warmstart_eval.json (per-pair cold / warm
reports and their summary) and DIR/warmstart_train.json (loss curve).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

import paper_2006_06823_b300 as L
from paper_2006_06823_b300 import synth

SHAPE = (192, 224, 192)          # nz, ny, nx
K = 32
NT = 10
SOLVER = dict(nt=NT, variant=L.V_DEFSTATE, interp=L.INTERP_LINEAR, alpha=0.0025, s=2,
              sigma2=0.01, max_gn=10, max_pcg=20, gtol=1e-3)
NET_D, NET_C = 64, 16
MAX_VOX = 8.0          # maximum displacement of the generating velocity, voxels
EVAL_MAX_GN = 30       # GN cap of the evaluation (both arms), so both can reach gtol
TRAIN_SEED0, EVAL_SEED0 = 100_000, 900_000
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                       "warmstart_d64_c16.npz")
# the same network trained on the paper-scale (noisy ellipsoid-phantom) recipe
WEIGHTS_PHANTOM = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                               "warmstart_phantom_d64_c16.npz")


def make_pair(seed, shape=SHAPE, K=K, nt=NT, max_vox=None):
    """(I0, I1) float32 device images of one seed: I1 = blobs, I0 = I1 transported along
    the seed's random band-limited velocity (library kernels), scaled to a maximum
    displacement of max_vox voxels (default MAX_VOX)."""
    import torch
    nz, ny, nx = shape
    if max_vox is None:
        max_vox = MAX_VOX
    I1 = synth.gaussian_blobs_device(shape, seed, "cuda")
    vt = synth.random_velocity_coeffs(K, 8, seed + 1)
    vt_d = torch.as_tensor(vt.astype(np.complex64), device="cuda")
    v = L.bl_include(vt_d, shape)
    to_vox = torch.tensor([nx, ny, nz], dtype=torch.float32, device="cuda").view(3, 1, 1, 1) / (2 * math.pi)
    V = v * to_vox
    V *= max_vox / V.pow(2).sum(0).sqrt().max()
    I0 = L.sl_transport(V, I1, nt, L.FORWARD, L.INTERP_LINEAR)
    return I0.contiguous(), I1


_PHANTOM = {}


def phantom_fixed(shape=SHAPE):
    """The paper-scale workload's fixed image (ellipsoid phantom, no noise) on the device,
    built once per grid."""
    import torch
    if shape not in _PHANTOM:
        _PHANTOM[shape] = torch.as_tensor(synth.ellipsoid_phantom(shape), dtype=torch.float32,
                                          device="cuda")
    return _PHANTOM[shape]


def make_phantom_pair(vel_seed, noise_seeds, shape=SHAPE, K=K, nt=NT, max_vox=None,
                      host_noise=False):
    """(I0, I1) of the paper-scale workload's recipe: I1 = phantom + noise, I0 = phantom
    transported (library kernels) along the seed's random band-limited velocity (K^3 generated
    modes, (1 + |k|^2)^-2, max_vox voxels max) + noise, N(0, 0.01) on both. host_noise draws
    the noise with ``synth.add_noise`` (the benchmark's pair), else with a seeded device
    generator (training pairs)."""
    import torch
    nz, ny, nx = shape
    if max_vox is None:
        max_vox = MAX_VOX
    fixed = phantom_fixed(shape)
    vt = synth.random_velocity_coeffs(K, K, vel_seed)
    v = L.bl_include(torch.as_tensor(vt.astype(np.complex64), device="cuda"), shape)
    to_vox = torch.tensor([nx, ny, nz], dtype=torch.float32, device="cuda").view(3, 1, 1, 1) / (2 * math.pi)
    V = v * to_vox
    V *= max_vox / V.pow(2).sum(0).sqrt().max()
    moving = L.sl_transport(V, fixed, nt, L.FORWARD, L.INTERP_LINEAR)
    if host_noise:
        I0 = synth.add_noise(moving.cpu().numpy().astype(np.float64), seed=noise_seeds[0])
        I1 = synth.add_noise(fixed.cpu().numpy().astype(np.float64), seed=noise_seeds[1])
        return (torch.as_tensor(I0, dtype=torch.float32, device="cuda"),
                torch.as_tensor(I1, dtype=torch.float32, device="cuda"))
    out = []
    for img, sd in zip((moving, fixed), noise_seeds):
        g = torch.Generator(device="cuda")
        g.manual_seed(int(sd))
        out.append((img + 0.1 * torch.randn(img.shape, generator=g, device="cuda")).contiguous())
    return out[0], out[1]


def make_workload_pair(workload, seed, max_vox=None):
    """One pair of the named workload from one seed: 'blobs' (the warm-start workload) or
    'phantom' (the paper-scale recipe; velocity seed = seed, noise seeds seed + 1, seed + 2)."""
    if workload == "phantom":
        return make_phantom_pair(seed, (seed + 1, seed + 2), max_vox=max_vox)
    return make_pair(seed, max_vox=max_vox)


def save_params(net, path):
    """Weights as BF16 bit patterns (what the kernels use) and biases as FP32."""
    p = net.get_params().cpu().numpy()
    import torch
    bits = torch.from_numpy(p).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.savez_compressed(path, params_bf16=bits, params_f32_bias=p * _bias_mask(net),
                        D=net.D, c=net.c)


def load_params(net, path):
    import torch
    z = np.load(path)
    w = torch.from_numpy(z["params_bf16"].view(np.int16)).view(torch.bfloat16).float().numpy()
    mask = _bias_mask(net)
    p = np.where(mask > 0, z["params_f32_bias"], w).astype(np.float32)
    net.set_params(torch.from_numpy(p).cuda())


def _bias_mask(net):
    """1 at the bias entries of the flat parameter vector (layout of lddmm.h), else 0."""
    c = net.c
    specs = [(2, c), (c, c), (c, 2 * c), (2 * c, 2 * c), (2 * c, 4 * c), (4 * c, 4 * c),
             (4 * c, 8 * c), (8 * c, 8 * c), (12 * c, 4 * c), (4 * c, 4 * c), (6 * c, 2 * c),
             (2 * c, 2 * c), (2 * c, 3)]
    m = np.zeros(net.num_params, dtype=np.float32)
    off = 0
    for cin, cout in specs:
        off += cout * cin * 27
        m[off:off + cout] = 1
        off += cout
    assert off == net.num_params
    return m


def low_band(v, kb):
    """The coefficient cube v [3, K, K, K] with every mode of |k_a| > kb on some axis set to
    zero (kb = None: v itself): the smooth part of a solution as a training target."""
    if kb is None:
        return v
    K = v.shape[-1]
    out = v.clone()
    k = (np.arange(K) - K // 2)
    drop = np.abs(k) > kb
    idx = np.nonzero(drop)[0].tolist()
    out[:, idx, :, :] = 0
    out[:, :, idx, :] = 0
    out[:, :, :, idx] = 0
    return out


def generate(seeds, net, max_vox=None, contexts=4, log=print, workload="blobs", target_band=None):
    """Registers every seed's pair from a cold start (``contexts`` pairs at a time through
    lddmm_register_batch, one stream each); returns (X, T, reports) with X the network
    inputs [N, 2, D^3] and T the targets [N, 3, (D/2)^3] on the device."""
    import torch
    nz, ny, nx = SHAPE
    D, d = net.D, net.D // 2
    X = torch.empty((len(seeds), 2, D, D, D), dtype=torch.float32, device="cuda")
    T = torch.empty((len(seeds), 3, d, d, d), dtype=torch.float32, device="cuda")
    streams = [torch.cuda.Stream() for _ in range(contexts)]
    ctxs = []
    for st in streams:
        with torch.cuda.stream(st):
            ctxs.append(L.Context(nx, ny, nz, K, **SOLVER))
    reps = []
    t0 = time.time()
    for a in range(0, len(seeds), contexts):
        chunk = seeds[a:a + contexts]
        pairs = [make_workload_pair(workload, s, max_vox=max_vox) for s in chunk]
        torch.cuda.synchronize()
        for c, (I0, I1) in zip(ctxs, pairs):
            c.set_images(I0, I1)
        vs = [c.zeros_cube() for c in ctxs[:len(chunk)]]
        torch.cuda.synchronize()
        reps += L.register_batch(ctxs[:len(chunk)], vs, max_threads=contexts)
        for j, ((I0, I1), v) in enumerate(zip(pairs, vs)):
            net.input(I0, I1, out=X[a + j])
            L.bl_include(low_band(v, target_band), (d, d, d), out=T[a + j])
        done = a + len(chunk)
        if done % 100 < contexts or done == len(seeds):
            log(f"  generated {done}/{len(seeds)} pairs, {time.time() - t0:.0f} s, "
                f"mean GN {np.mean([r['gn_iters'] for r in reps]):.2f}, reached gtol "
                f"{np.mean([r['grad_rel_l2'] <= SOLVER['gtol'] for r in reps]):.2f}")
    torch.cuda.synchronize()
    for c in ctxs:
        c.close()
    return X, T, reps


def reflect(X, T, axes):
    """The pairs and targets mirrored through the periodic domain's origin along the given
    axes (0 = x, 1 = y, 2 = z): f(x) -> f(-x mod n), and the mirrored velocity component
    changes sign. The registration problem is invariant under these reflections (isotropic
    regulariser, symmetric band, reflection-symmetric interpolation), so a mirrored pair's
    solution is the mirrored solution."""
    import torch
    for a in axes:
        dim = X.dim() - 1 - a
        X = torch.roll(torch.flip(X, [dim]), 1, dim)
        T = torch.roll(torch.flip(T, [dim]), 1, dim)
        T[:, a] = -T[:, a]
    return X.contiguous(), T.contiguous()


def train(net, X, T, epochs=30, batch=8, lr=1e-3, lr_min=1e-5, seed=0, augment=True, log=print):
    """Adam on contiguous mini-batches of (X, T) with a cosine learning-rate decay; the
    batch windows move by a random offset each epoch, and each batch is mirrored along a
    random subset of the axes (augment)."""
    N = X.shape[0]
    g = synth.rng(seed)
    nb = N // batch
    total = epochs * nb
    curve = []
    step = 0
    t0 = time.time()
    for ep in range(epochs):
        shift = int(g.integers(0, N - nb * batch + 1))
        order = g.permutation(nb)
        losses = []
        for j in order:
            a = shift + j * batch
            cur = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / max(total, 1)))
            xb, tb = X[a:a + batch], T[a:a + batch]
            if augment:
                r = int(g.integers(0, 8))
                xb, tb = reflect(xb, tb, [ax for ax in range(3) if r >> ax & 1])
            losses.append(net.train_step(xb, tb, cur))
            step += 1
        curve.append(float(np.mean(losses)))
        log(f"  epoch {ep + 1}/{epochs}: loss {curve[-1]:.4e} ({time.time() - t0:.0f} s)")
    return curve


def prediction_error(net, X, T, batch=8):
    """Relative L2 error of the network's output against the targets, per sample."""
    import torch
    errs = []
    for a in range(0, X.shape[0], batch):
        y = net.forward(X[a:a + batch])
        t = T[a:a + batch]
        errs += ((y - t).flatten(1).norm(dim=1) / t.flatten(1).norm(dim=1)).tolist()
    torch.cuda.synchronize()
    return errs


def evaluate(net, seeds, max_vox=None, max_gn=None, log=print, workload="blobs"):
    """Cold vs warm registrations of the seeds' pairs (wall time with device sync); both
    arms stop at the same relative residual gtol or after max_gn GN iterations."""
    import torch
    nz, ny, nx = SHAPE
    ctx = L.Context(nx, ny, nz, K, **dict(SOLVER, max_gn=max_gn or SOLVER["max_gn"]))
    # one untimed warm-up of both paths
    I0, I1 = make_workload_pair(workload, seeds[0], max_vox=max_vox)
    ctx.set_images(I0, I1)
    ctx.register()
    ctx.register(net.warm_start(I0, I1, K))
    rows = []
    for i, s in enumerate(seeds):
        I0, I1 = make_workload_pair(workload, s, max_vox=max_vox)
        ctx.set_images(I0, I1)
        torch.cuda.synchronize()
        t = time.perf_counter()
        v_cold, cold = ctx.register()
        torch.cuda.synchronize()
        cold["wall_s"] = time.perf_counter() - t
        t = time.perf_counter()
        v0 = net.warm_start(I0, I1, K)
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - t
        v_pred = v0.clone()
        v_warm, warm = ctx.register(v0)
        torch.cuda.synchronize()
        warm["wall_s"] = time.perf_counter() - t
        warm["predict_s"] = t_pred
        pred_err = float((v_pred - v_cold).abs().pow(2).sum().sqrt() / v_cold.abs().pow(2).sum().sqrt())
        sol_diff = float((v_warm - v_cold).abs().pow(2).sum().sqrt() / v_cold.abs().pow(2).sum().sqrt())
        rows.append({"seed": int(s), "cold": cold, "warm": warm, "pred_rel_l2": pred_err,
                     "solution_rel_diff": sol_diff})
        if (i + 1) % 25 == 0 or i + 1 == len(seeds):
            log(f"  evaluated {i + 1}/{len(seeds)}")
    ctx.close()
    return rows, summarize(rows)


def summarize(rows):
    def m(key, arm):
        return float(np.mean([r[arm][key] for r in rows]))

    gtol = SOLVER["gtol"]
    cold_ok = [r["cold"]["grad_rel_l2"] <= gtol for r in rows]
    warm_ok = [r["warm"]["grad_rel_l2"] <= gtol for r in rows]
    gap = [(r["warm"]["E"] - r["cold"]["E"]) / abs(r["cold"]["E"]) for r in rows]
    return {
        "pairs": len(rows),
        "gn_iters_cold": m("gn_iters", "cold"), "gn_iters_warm": m("gn_iters", "warm"),
        "gn_iters_saved": m("gn_iters", "cold") - m("gn_iters", "warm"),
        "pcg_iters_cold": m("pcg_iters_total", "cold"), "pcg_iters_warm": m("pcg_iters_total", "warm"),
        "seconds_cold": m("wall_s", "cold"), "seconds_warm": m("wall_s", "warm"),
        "seconds_saved": m("wall_s", "cold") - m("wall_s", "warm"),
        "speedup": m("wall_s", "cold") / m("wall_s", "warm"),
        "predict_seconds": m("predict_s", "warm"),
        "reached_gtol_cold": float(np.mean(cold_ok)), "reached_gtol_warm": float(np.mean(warm_ok)),
        "grad_rel_l2_cold": m("grad_rel_l2", "cold"), "grad_rel_l2_warm": m("grad_rel_l2", "warm"),
        "energy_gap_rel_mean": float(np.mean(gap)), "energy_gap_rel_max": float(np.max(np.abs(gap))),
        "pred_rel_l2_mean": float(np.mean([r["pred_rel_l2"] for r in rows])),
        "solution_rel_diff_mean": float(np.mean([r["solution_rel_diff"] for r in rows])),
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--train-pairs", type=int, default=1000)
    ap.add_argument("--eval-pairs", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=".")
    ap.add_argument("--init", default=None, help="start from saved weights")
    ap.add_argument("--max-vox", type=float, default=MAX_VOX,
                    help="maximum displacement of the generating velocity (voxels)")
    ap.add_argument("--eval-max-gn", type=int, default=EVAL_MAX_GN)
    ap.add_argument("--contexts", type=int, default=4)
    ap.add_argument("--target-band", type=int, default=None,
                    help="train on the solution's modes with |k_a| <= this only (its smooth part)")
    ap.add_argument("--weights-out", default=None, help="also save the weights here")
    ap.add_argument("--workload", default="blobs", choices=["blobs", "phantom"],
                    help="training and evaluation pairs: Gaussian blobs (no noise) or the "
                         "paper-scale ellipsoid-phantom recipe (noisy)")
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    os.makedirs(args.out, exist_ok=True)
    log = lambda msg: print(msg, flush=True)  # noqa: E731
    net = L.Net(NET_D, NET_C, batch_max=args.batch, seed=0)
    if args.init:
        load_params(net, args.init)
    log(f"network: {net.num_params} parameters")
    stride = 3 if args.workload == "phantom" else 2    # seeds consumed per pair
    train_seeds = [TRAIN_SEED0 + stride * i for i in range(args.train_pairs)]
    eval_seeds = [EVAL_SEED0 + stride * i for i in range(args.eval_pairs)]
    t = time.time()
    X, T, reps = generate(train_seeds, net, max_vox=args.max_vox, contexts=args.contexts, log=log,
                          workload=args.workload, target_band=args.target_band)
    t_gen = time.time() - t
    n_val = max(1, len(train_seeds) // 20)
    t = time.time()
    curve = train(net, X[n_val:], T[n_val:], epochs=args.epochs, batch=args.batch, lr=args.lr, log=log)
    t_train = time.time() - t
    val_err = prediction_error(net, X[:n_val], T[:n_val])
    save_params(net, os.path.join(args.out, "warmstart_params.npz"))
    if args.weights_out:
        save_params(net, args.weights_out)
    with open(os.path.join(args.out, "warmstart_train.json"), "w") as f:
        json.dump({"train_pairs": len(train_seeds) - n_val, "val_pairs": n_val,
                   "generate_s": t_gen, "train_s": t_train, "loss_per_epoch": curve,
                   "val_pred_rel_l2_mean": float(np.mean(val_err)),
                   "train_gn_iters_mean": float(np.mean([r["gn_iters"] for r in reps])),
                   "train_reached_gtol": float(np.mean([r["grad_rel_l2"] <= SOLVER["gtol"] for r in reps]))},
                  f, indent=1)
    del X, T
    rows, summary = evaluate(net, eval_seeds, max_vox=args.max_vox, max_gn=args.eval_max_gn, log=log,
                             workload=args.workload)
    summary.update({"max_vox": args.max_vox, "eval_max_gn": args.eval_max_gn, "workload": args.workload,
                    "train_pairs": len(train_seeds) - n_val, "epochs": args.epochs})
    with open(os.path.join(args.out, "warmstart_eval.json"), "w") as f:
        json.dump({"summary": summary, "pairs": rows}, f, indent=1)
    log(json.dumps(summary, indent=1))


if __name__ == "__main__":
    main()
