"""Learned warm start for skyrmion-tube relaxations.

The plain method relaxes an extruded skyrmion ansatz by the director-only
gradient flow (``nh_relax``: the predictor-corrector of Sec. II.B at u = 0)
until the director's largest rate of change, measured over ``check_every`` FD
steps, is below ``tol`` (``nh_director_change``).  A 3D U-Net with BF16 kernels
(``nh_unet_*``) is trained on such relaxations to predict the relaxed field
from the ansatz and (q0, Lz, W0); the plain relaxation then continues from the
prediction, and the prediction counts only if the result matches the relaxation from the ansatz
within ``max |dn| <= 1e-4`` (both continued to a stricter stop rate for that
comparison), and the saving to the ordinary stop rule is reported in FD steps
and wall time.

Usage:  python -m paper_2503_06610_gb300.warmstart --samples 2000 --held-out 200 --out ws.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs
from . import nh


class WarmStartNet:
    """FP32 master parameters + Adam state (torch CUDA tensors) and cached
    network instances per input shape."""

    def __init__(self, seed=0, device=0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        P = nh.UNet.param_count()
        flat = inputs.unet_init_params(seed)
        assert flat.size == P
        self.params = torch.tensor(flat, dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.steps = 0
        self.nets = {}

    def net(self, shape):
        if shape not in self.nets:
            self.nets[shape] = nh.UNet(*shape)
        return self.nets[shape]

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def predict(self, n_ansatz, scalars, dims):
        """n_ansatz [B][3][N] and scalars [B][3] (FP32 CUDA) -> predicted n [B][3][N]."""
        B = n_ansatz.shape[0]
        net = self.net((B,) + tuple(dims))
        out = self.torch.empty_like(n_ansatz)
        net.set_params(self.params, self._stream())
        net.forward(self.params, n_ansatz, scalars, out, self._stream())
        return out

    def loss_and_grad(self, n_ansatz, scalars, target, dims):
        B = n_ansatz.shape[0]
        net = self.net((B,) + tuple(dims))
        s = self._stream()
        net.set_params(self.params, s)
        net.forward(self.params, n_ansatz, scalars, None, s)
        net.backward(self.params, n_ansatz, target, self.grad, self.loss, s)
        return self.loss, self.grad

    def train_step(self, n_ansatz, scalars, target, dims, lr=1e-3):
        self.loss_and_grad(n_ansatz, scalars, target, dims)
        self.steps += 1
        nh.nh_unet_adam(self.params, self.grad, self.m, self.v, self.steps, lr, self._stream())
        return self.loss


# ------------------------------------------------------------------ plain relaxation

def relax(chans, tol=2e-10, check_every=100, max_steps=200000):
    """Relax every channel (batched) until the director's largest rate of change,
    max |n(t) - n(t - T)| / T over the last check interval T = check_every
    FD steps, is below tol; returns the FD steps each one needed (capped at
    max_steps) and the wall time."""
    import torch
    for c in chans:
        c.director_change()  # snapshot of the starting field
    active = list(range(len(chans)))
    steps = [0] * len(chans)
    t0 = time.perf_counter()
    while active:
        nh.batch_relax([chans[k] for k in active], check_every)
        still = []
        for k in active:
            steps[k] += check_every
            rate = chans[k].director_change() / (check_every * chans[k].params["dt_fd"])
            if rate >= tol and steps[k] < max_steps:
                still.append(k)
        active = still
    torch.cuda.synchronize()
    return steps, time.perf_counter() - t0


def make_channels(samples, fields=None, symmetrize=True):
    """One FP32 channel per sample, started from its ansatz or from fields[k];
    the start is projected onto the C4-symmetric fields about the tube axis
    (nh_symmetrize_c4), which pins the tube to the axis: its position is a
    zero mode of the relaxation."""
    chans = []
    for k, (params, n0) in enumerate(samples):
        ch = nh.Channel(dict(params, precision="fp32", storage="f32", shifted=True))
        ch.set_fields(n0 if fields is None else fields[k])
        if symmetrize and params["nx"] == params["ny"]:
            ch.symmetrize_c4()
        chans.append(ch)
    return chans


def scalars_of(params):
    return [params["q0"], float(params["nz"]), params["W0"]]


def generate(samples, batch=64, **relax_kw):
    """Relax each sample from its ansatz; returns targets, steps and wall time."""
    targets, steps, wall = [], [], 0.0
    for b0 in range(0, len(samples), batch):
        chans = make_channels(samples[b0:b0 + batch])
        st, w = relax(chans, **relax_kw)
        wall += w
        steps += st
        for c in chans:
            targets.append(c.get_fields()[0].astype(np.float32))
            c.close()
    return targets, steps, wall


def collapsed(target, nz, min_columns=5):
    """True when the relaxed tube has fewer than min_columns sites per layer
    with n_z < 0: the tube collapsed on the lattice.  Under the C4-symmetric
    dynamics the axis column with n = -z is then a fixed point (the symmetry
    forces n_x = n_y = 0 there), so such a target keeps a lone reversed column;
    these samples are left out of training and evaluation."""
    return float((np.asarray(target)[2] < 0).sum()) / nz < min_columns


def group_by_shape(indices, samples):
    groups = {}
    for i in indices:
        p = samples[i][0]
        groups.setdefault((p["nx"], p["ny"], p["nz"]), []).append(i)
    return groups


def train(net, samples, targets, train_idx, epochs=20, batch=8, lr=1e-3, lr_min=1e-4, seed=0, log=None):
    """Adam on mini-batches of one shape; the learning rate decays from lr to
    lr_min along a half cosine over the epochs."""
    torch = net.torch
    rng = np.random.Generator(np.random.PCG64(seed))
    groups = group_by_shape(train_idx, samples)
    dev = net.device
    cache = {}
    for shape, idx in groups.items():
        cache[shape] = (
            torch.tensor(np.stack([samples[i][1] for i in idx]).astype(np.float32), device=dev),
            torch.tensor(np.array([scalars_of(samples[i][0]) for i in idx], dtype=np.float32), device=dev),
            torch.tensor(np.stack([targets[i] for i in idx]), device=dev))
    history = []
    for ep in range(epochs):
        lr_ep = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * ep / max(1, epochs - 1)))
        losses = []
        order = [(shape, j) for shape, idx in groups.items() for j in range(0, len(idx) - batch + 1, batch)]
        rng.shuffle(order)
        perms = {shape: rng.permutation(len(idx)) for shape, idx in groups.items()}
        for shape, j in order:
            sel = torch.tensor(perms[shape][j:j + batch], device=dev)
            na, sc, tg = (t.index_select(0, sel) for t in cache[shape])
            losses.append(net.train_step(na.contiguous(), sc.contiguous(), tg.contiguous(), shape, lr_ep).clone())
        mean = float(torch.stack(losses).mean())
        history.append(mean)
        for unet in net.nets.values():  # a tensor-core convolution that gave up a wait raises here
            unet.status()
        if log:
            log(f"epoch {ep}: loss {mean:.3e}")
    return history


def evaluate(net, samples, targets, steps_ansatz, test_idx, batch=64, judge_tol=None, **relax_kw):
    """Relax the held-out samples from the network's prediction; compare with the
    relaxations from the ansatz (steps, wall time, final-field difference).

    Steps and wall time are counted to the stop rule of relax_kw on both sides.
    The judge then continues both relaxations, from the prediction and from the
    ansatz, to the stricter rate judge_tol (default: the same rule) and
    compares the final fields, so that the comparison does not depend on where
    two slowly converging runs happened to stop."""
    torch = net.torch
    dev = net.device
    t0 = time.perf_counter()
    preds = {}
    for shape, idx in group_by_shape(test_idx, samples).items():
        for j in range(0, len(idx), 8):
            sub = idx[j:j + 8]
            na = torch.tensor(np.stack([samples[i][1] for i in sub]).astype(np.float32), device=dev)
            sc = torch.tensor(np.array([scalars_of(samples[i][0]) for i in sub], dtype=np.float32), device=dev)
            out = net.predict(na, sc, shape).cpu().numpy().astype(np.float64)
            for k, i in enumerate(sub):
                preds[i] = out[k]
    torch.cuda.synchronize()
    t_pred = time.perf_counter() - t0
    judge_kw = dict(relax_kw, tol=judge_tol) if judge_tol is not None else None
    steps_p, wall_p, wall_a, dn, dn_pred, dn_ans, rms_pred, rms_ans, per = [], 0.0, 0.0, [], [], [], [], [], []
    for b0 in range(0, len(test_idx), batch):
        sub = test_idx[b0:b0 + batch]
        chans = make_channels([samples[i] for i in sub], [preds[i] for i in sub])
        st, w = relax(chans, **relax_kw)
        wall_p += w
        steps_p += st
        # the same held-out relaxations from the ansatz, timed the same way
        chans_a = make_channels([samples[i] for i in sub])
        _, w = relax(chans_a, **relax_kw)
        wall_a += w
        if judge_kw is not None:
            relax(chans, **judge_kw)
            relax(chans_a, **judge_kw)
        for c, ca, i in zip(chans, chans_a, sub):
            n = c.get_fields()[0]
            ref = ca.get_fields()[0] if judge_kw is not None else targets[i]
            d = np.abs(n - ref).max(axis=0)
            dn.append(float(d.max()))
            dn_pred.append(float(np.max(np.abs(preds[i] - targets[i]))))
            ans = np.asarray(samples[i][1]).reshape(3, -1)
            dn_ans.append(float(np.max(np.abs(ans - targets[i]))))
            rms_pred.append(float(np.sqrt(np.mean(np.sum((preds[i] - targets[i]) ** 2, axis=0)))))
            rms_ans.append(float(np.sqrt(np.mean(np.sum((ans - targets[i]) ** 2, axis=0)))))
            p = samples[i][0]
            z, y, x = np.unravel_index(int(np.argmax(d)), (p["nz"], p["ny"], p["nx"]))
            per.append({"index": i, "max_dn": dn[-1], "argmax_zyx": [int(z), int(y), int(x)],
                        "min_nz_target": float(targets[i][2].min()), "min_nz_prediction": float(preds[i][2].min()),
                        "min_nz_final": float(n[2].min()), "steps_ansatz": int(steps_ansatz[i]),
                        "steps_prediction": int(steps_p[len(per)])})
            c.close()
            ca.close()
    sa = np.array([steps_ansatz[i] for i in test_idx], dtype=float)
    sp = np.array(steps_p, dtype=float)
    return {"held_out": len(test_idx), "mean_steps_from_ansatz": float(sa.mean()),
            "mean_steps_from_prediction": float(sp.mean()), "step_ratio": float(sp.sum() / sa.sum()),
            "wall_s_prediction_inference": t_pred, "wall_s_relax_from_prediction": wall_p,
            "wall_s_relax_from_ansatz": wall_a, "wall_ratio": (t_pred + wall_p) / wall_a,
            "judge_tol": judge_tol if judge_tol is not None else relax_kw.get("tol"),
            "max_dn_final": float(np.max(dn)), "frac_final_within_1e-4": float(np.mean(np.array(dn) <= 1e-4)),
            "median_max_dn_prediction_vs_relaxed": float(np.median(dn_pred)),
            "median_max_dn_ansatz_vs_relaxed": float(np.median(dn_ans)),
            "median_rms_prediction_vs_relaxed": float(np.median(rms_pred)),
            "median_rms_ansatz_vs_relaxed": float(np.median(rms_ans)), "per_sample": per}


def conv_flops(dims):
    """Multiply-adds x 2 of the fourteen 3x3x3 convolutions of one forward pass
    of one sample of size dims = (nx, ny, nz)."""
    nx, ny, nz = dims
    level = {"enc1": 0, "enc2": 1, "enc3": 2, "bot": 3, "dec3": 2, "dec2": 1, "dec1": 0}
    total = 0
    for name, ci, co in inputs.UNET_CONV_LAYERS:
        vox = (nx * ny * nz) >> (3 * level[name[:-1]])
        total += 2 * vox * 27 * ci * co
    return total


def time_network(batch=8, dims=(64, 64, 32), reps=20):
    """CUDA-event times of the network's forward and forward + backward passes
    on a batch of extruded tube ansatzes; returns ms per pass and the
    convolution TFLOP/s (the backward's two products counted as 2x the
    forward's)."""
    import torch
    net = WarmStartNet(seed=0)
    samples = inputs.warmstart_samples(batch, seed=1, nx=dims[0], ny=dims[1], lz_choices=(dims[2],))
    dev = net.device
    na = torch.tensor(np.stack([s[1] for s in samples]).astype(np.float32), device=dev)
    sc = torch.tensor(np.array([scalars_of(s[0]) for s in samples], dtype=np.float32), device=dev)
    shape = (batch,) + tuple(dims)
    for _ in range(3):
        net.predict(na, sc, dims)
        net.loss_and_grad(na, sc, na, dims)
    net.net(shape).status()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    for _ in range(reps):
        net.predict(na, sc, dims)
    ev[1].record()
    for _ in range(reps):
        net.loss_and_grad(na, sc, na, dims)
    ev[2].record()
    torch.cuda.synchronize()
    net.net(shape).status()
    fwd = ev[0].elapsed_time(ev[1]) / reps
    both = ev[1].elapsed_time(ev[2]) / reps
    f = conv_flops(dims) * batch
    return {"batch": batch, "dims": list(dims), "forward_ms": fwd, "forward_backward_ms": both,
            "conv_gflop_forward": f / 1e9, "forward_tflops": f / (fwd * 1e-3) / 1e12,
            "forward_backward_tflops": 3 * f / (both * 1e-3) / 1e12}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--time-network", action="store_true",
                    help="only time the network's passes on a batch of 8 cells of 64x64x32")
    ap.add_argument("--samples", type=int, default=2000)
    ap.add_argument("--held-out", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--tol", type=float, default=2e-10, help="stop when max |dn/dt| < tol (per LB time unit)")
    ap.add_argument("--judge-tol", type=float, default=1e-11,
                    help="both relaxations continue to this rate before their final fields are compared")
    ap.add_argument("--max-steps", type=int, default=200000)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    if args.time_network:
        print(json.dumps(time_network()), flush=True)
        return
    samples = inputs.warmstart_samples(args.samples, seed=0)
    kw = dict(tol=args.tol, max_steps=args.max_steps)
    t0 = time.perf_counter()
    targets, steps, wall = generate(samples, **kw)
    print(f"generated {len(samples)} relaxations in {wall:.1f} s; mean FD steps {np.mean(steps):.0f}", flush=True)
    valid = [i for i in range(len(samples)) if not collapsed(targets[i], samples[i][0]["nz"])]
    n_test = args.held_out
    cut = len(samples) - n_test
    test_idx = [i for i in valid if i >= cut]
    train_idx = [i for i in valid if i < cut]
    net = WarmStartNet(seed=0)
    t1 = time.perf_counter()
    hist = train(net, samples, targets, train_idx, epochs=args.epochs, log=lambda s: print(s, flush=True))
    t_train = time.perf_counter() - t1
    res = evaluate(net, samples, targets, steps, test_idx, judge_tol=args.judge_tol, **kw)
    res.update({"samples": len(samples), "collapsed_excluded": len(samples) - len(valid),
                "train_epochs": args.epochs, "train_wall_s": t_train,
                "loss_history": hist, "generation_wall_s": wall, "mean_steps_generation": float(np.mean(steps)),
                "total_wall_s": time.perf_counter() - t0})
    print(json.dumps(res), flush=True)
    if args.out:
        json.dump(res, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
