"""Warm-start network kernels (BF16 activations, FP32 accumulation, tensor
cores) against the FP64 CPU oracle network, and the training / relaxation
driver.

The oracle runs with the same BF16-rounded weights and inputs; the remaining
differences come from rounding every activation to BF16 (2^-9 relative per
layer), so the tolerances are a few per cent.
"""
import math

import numpy as np
import pytest

from paper_2503_06610_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_06610_gb300 import nh, warmstart
    from oracle import unet as U
    nh.load_library()
    return torch, nh, warmstart, U


def _bf16(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _problem(B=2, nx=16, ny=16, nz=16, seed=0, smooth_target=False):
    """Network parameters, ansatz, target and scalars.  The random target makes
    every gradient a small residual of many random-sign terms; the smooth
    target (a tube of another radius, as in training) makes it a coherent sum."""
    rng = np.random.default_rng(seed)
    flat = I.unet_init_params(seed)
    hs = len(flat) - 51
    flat[hs:hs + 48] = rng.normal(0, 0.3, size=48)        # a head large enough to move n
    flat[:hs] += 0.02 * rng.normal(size=hs) * (rng.random(hs) < 0.01)
    n_ans = np.stack([I.skyrmion_tubes(nx, ny, nz, [(nx / 2 + k, ny / 2)], 5.0) for k in range(B)])
    if smooth_target:
        target = np.stack([I.skyrmion_tubes(nx, ny, nz, [(nx / 2 + k, ny / 2)], 3.5 + k) for k in range(B)])
    else:
        target = np.stack([I.random_director(nx, ny, nz, seed=10 + k) for k in range(B)])
    scal = np.array([[2 * math.pi / (12 + 4 * k), float(nz), 1e-5 * (k + 1)] for k in range(B)])
    return flat, n_ans, target, scal


def _oracle(U, flat, n_ans, target, scal, dims, bf16_storage=False):
    import torch
    B = n_ans.shape[0]
    nx, ny, nz = dims
    fr = flat.copy()
    # the GPU convolves with BF16 weights and adds FP32 biases; the head is FP32
    off = 0
    for _, ci, co in U.CONV_LAYERS:
        fr[off:off + 27 * ci * co] = _bf16(flat[off:off + 27 * ci * co])
        off += 27 * ci * co + co
    na5 = torch.tensor(n_ans.reshape(B, 3, nz, ny, nx))
    x = U.make_input(na5.numpy(), scal[:, 0], scal[:, 1], scal[:, 2])
    x = torch.tensor(_bf16(x.numpy()))
    tg = torch.tensor(target.reshape(B, 3, nz, ny, nx))
    loss, grad, n_pred = U.loss_and_grad(fr, x, na5, tg, bf16_storage)
    return loss, grad, n_pred.numpy().reshape(B, 3, -1)


def test_forward_and_gradients_match_oracle(env):
    torch, nh, ws, U = env
    dims = (16, 16, 16)
    flat, n_ans, target, scal = _problem(B=2)
    loss_o, grad_o, npred_o = _oracle(U, flat, n_ans, target, scal, dims)
    dev = torch.device("cuda")
    net = nh.UNet(2, *dims)
    params = torch.tensor(flat, dtype=torch.float32, device=dev)
    na = torch.tensor(n_ans, dtype=torch.float32, device=dev)
    sc = torch.tensor(scal, dtype=torch.float32, device=dev)
    tg = torch.tensor(target, dtype=torch.float32, device=dev)
    out = torch.empty_like(na)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    net.set_params(params)
    net.forward(params, na, sc, out)
    net.backward(params, na, tg, grad, loss)
    torch.cuda.synchronize()
    npred = out.cpu().numpy().astype(np.float64)
    delta_o = npred_o - n_ans
    delta_g = npred - n_ans
    assert np.linalg.norm(delta_g - delta_o) / np.linalg.norm(delta_o) < 3e-2
    assert abs(float(loss) - loss_o) / loss_o < 1e-2
    g = grad.cpu().numpy().astype(np.float64)
    rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
    cos = lambda a, b: float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))
    report = []
    off = 0
    for name, ci, co in U.CONV_LAYERS:
        n_w = 27 * ci * co
        for part, sl in (("W", slice(off, off + n_w)), ("b", slice(off + n_w, off + n_w + co))):
            report.append((name, part, rel(g[sl], grad_o[sl]), cos(g[sl], grad_o[sl])))
        off += n_w + co
    report.append(("head", "Wb", rel(g[off:], grad_o[off:]), cos(g[off:], grad_o[off:])))
    for r in report:
        print("grad %-6s %-2s rel %.3e cos %.6f" % r)
    # against the float64 network the BF16 activations and BF16 output
    # gradients cost several per cent per layer, but the direction must agree
    assert rel(g, grad_o) < 0.12
    assert all(r[2] < 0.25 and r[3] > 0.97 for r in report), report
    assert report[-1][2] < 2e-2


def _gpu_loss_grad(torch, nh, flat, n_ans, scal, target, dims):
    dev = torch.device("cuda")
    B = n_ans.shape[0]
    net = nh.UNet(B, *dims)
    params = torch.tensor(flat, dtype=torch.float32, device=dev)
    na = torch.tensor(n_ans, dtype=torch.float32, device=dev)
    out = torch.empty_like(na)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    net.set_params(params)
    net.forward(params, na, torch.tensor(scal, dtype=torch.float32, device=dev), out)
    net.backward(params, na, torch.tensor(target, dtype=torch.float32, device=dev), grad, loss)
    torch.cuda.synchronize()
    return float(loss), grad.cpu().numpy().astype(np.float64), out.cpu().numpy().astype(np.float64)


def _per_layer(U, g, ref):
    rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    rows = []
    off = 0
    for name, ci, co in U.CONV_LAYERS:
        n_w = 27 * ci * co
        rows.append((name, rel(g[off:off + n_w], ref[off:off + n_w]),
                     rel(g[off + n_w:off + n_w + co], ref[off + n_w:off + n_w + co])))
        off += n_w + co
    rows.append(("head", rel(g[off:], ref[off:]), 0.0))
    return rows


def test_gradients_match_bf16_storage_oracle(env):
    """Against the oracle that stores every activation in BF16 and rounds the
    gradient entering each convolution's products to BF16, with the bias
    gradient summed from the unrounded gradient as the kernels do (float64
    arithmetic otherwise), for a smooth target as in training: every layer's
    weight and bias gradient agrees to within 3 %.  What remains are the rare
    activations whose FP32 and float64 sums round to neighbouring BF16 values."""
    torch, nh, ws, U = env
    dims = (16, 16, 16)
    flat, n_ans, target, scal = _problem(B=2, smooth_target=True)
    loss_e, grad_e, npred_e = _oracle(U, flat, n_ans, target, scal, dims, bf16_storage=True)
    loss, g, npred = _gpu_loss_grad(torch, nh, flat, n_ans, scal, target, dims)
    rows = _per_layer(U, g, grad_e)
    for r in rows:
        print("vs BF16-storage oracle %-6s W %.3e b %.3e" % r)
    assert abs(loss - loss_e) / loss_e < 1e-3
    assert np.linalg.norm(npred - npred_e) / np.linalg.norm(npred_e - n_ans) < 1e-2
    assert all(w < 3e-2 and b < 3e-2 for _, w, b in rows), rows


def test_gradients_exact_representable_case(env):
    """Weights k/64, inputs m/16, biases k/64 and a smooth target: the FP32
    sums of the early layers are exact, so both sides round identical values
    to BF16 there and the GPU gradients follow the BF16-storage oracle's more
    closely still; differences start only in the deeper layers, whose sums
    round in FP32."""
    torch, nh, ws, U = env
    dims = (16, 16, 16)
    B = 2
    flat, n_ans, target, scal = _problem(B=B, smooth_target=True)
    hs = len(flat) - 51
    q = np.round(flat[:hs] * 64.0) / 64.0
    rng = np.random.default_rng(9)
    off = 0
    for _, ci, co in U.CONV_LAYERS:          # small non-zero biases, multiples of 1/64
        q[off + 27 * ci * co:off + 27 * ci * co + co] = rng.integers(-3, 4, size=co) / 64.0
        off += 27 * ci * co + co
    flat = np.concatenate([q, flat[hs:]])
    n_ans = np.round(n_ans * 16.0) / 16.0
    scal = np.array([[2 * math.pi / 16, 16.0, 0.0]] * B)   # q0 Lz / 2 pi = 1, Lz / 32 = 0.5, W0 = 0
    loss_e, grad_e, npred_e = _oracle(U, flat, n_ans, target, scal, dims, bf16_storage=True)
    loss, g, npred = _gpu_loss_grad(torch, nh, flat, n_ans, scal, target, dims)
    rows = _per_layer(U, g, grad_e)
    for r in rows:
        print("exact case %-6s W %.3e b %.3e" % r)
    assert abs(loss - loss_e) / loss_e < 1e-4
    assert all(w < 1e-2 and b < 1e-2 for _, w, b in rows), rows
    assert np.median([w for _, w, _ in rows]) < 2e-3


def test_forward_activations_match_bf16_oracle(env):
    """Every stored layer output of the GPU forward equals the BF16-storage
    oracle's (float64 arithmetic, BF16 storage) up to rare rounding flips."""
    torch, nh, ws, U = env
    dims = (16, 16, 16)
    B = 2
    flat, n_ans, target, scal = _problem(B=B)
    nx, ny, nz = dims
    fr = flat.copy()
    off = 0
    for _, ci, co in U.CONV_LAYERS:
        fr[off:off + 27 * ci * co] = _bf16(flat[off:off + 27 * ci * co])
        off += 27 * ci * co + co
    na5 = torch.tensor(n_ans.reshape(B, 3, nz, ny, nx))
    x = torch.tensor(_bf16(U.make_input(na5.numpy(), scal[:, 0], scal[:, 1], scal[:, 2]).numpy()))
    keep = {}
    with torch.no_grad():
        U.forward(U.unpack(fr), x, na5, bf16_storage=True, keep=keep)
    dev = torch.device("cuda")
    net = nh.UNet(B, *dims)
    params = torch.tensor(flat, dtype=torch.float32, device=dev)
    net.set_params(params)
    net.forward(params, torch.tensor(n_ans, dtype=torch.float32, device=dev),
                torch.tensor(scal, dtype=torch.float32, device=dev), None)
    net.status()  # no tensor-core wait expired
    levels = {"enc1": 1, "enc2": 2, "enc3": 4, "bot": 8, "dec3": 4, "dec2": 2, "dec1": 1}
    for l, (name, ci, co) in enumerate(U.CONV_LAYERS):
        s = levels[name[:-1]]
        shape = (B, nz // s, ny // s, nx // s, co)
        out = torch.empty(int(np.prod(shape)), dtype=torch.float32, device=dev)
        net.activation(l, out)
        torch.cuda.synchronize()
        g = out.cpu().numpy().reshape(shape).transpose(0, 4, 1, 2, 3)
        o = keep[name].numpy()
        err = np.linalg.norm(g - o) / max(np.linalg.norm(o), 1e-30)
        print("forward %-6s rel %.3e" % (name, err))
        assert err < 5e-3, (name, err)


def test_adam_matches_oracle(env):
    torch, nh, ws, U = env
    rng = np.random.default_rng(3)
    n = 1000
    p = rng.normal(size=n)
    g = rng.normal(size=n)
    m = np.zeros(n)
    v = np.zeros(n)
    dev = torch.device("cuda")
    tp, tg, tm, tv = (torch.tensor(a, dtype=torch.float32, device=dev) for a in (p, g, m, v))
    for step in (1, 2, 3):
        nh.nh_unet_adam(tp, tg, tm, tv, step, 1e-3)
        p, m, v = U.adam(p, g, m, v, step, 1e-3)
    torch.cuda.synchronize()
    assert np.allclose(tp.cpu().numpy(), p, rtol=1e-6, atol=1e-7)


def test_training_reduces_loss(env):
    torch, nh, ws, U = env
    dims = (16, 16, 8)
    flat, n_ans, target, scal = _problem(B=4, nz=8, seed=1)
    target = np.stack([I.skyrmion_tubes(16, 16, 8, [(8.0 + k, 8.0)], 6.5) for k in range(4)])
    net = ws.WarmStartNet(seed=2)
    dev = net.device
    na = torch.tensor(n_ans, dtype=torch.float32, device=dev)
    sc = torch.tensor(scal, dtype=torch.float32, device=dev)
    tg = torch.tensor(target, dtype=torch.float32, device=dev)
    first = float(net.train_step(na, sc, tg, dims, lr=2e-3))
    for _ in range(60):
        last = float(net.train_step(na, sc, tg, dims, lr=2e-3))
    assert last < 0.5 * first


def test_relaxation_driver_converges(env):
    torch, nh, ws, U = env
    samples = I.warmstart_samples(3, seed=5, nx=16, ny=16, lz_choices=(8,))
    chans = ws.make_channels(samples)
    steps, wall = ws.relax(chans, tol=1e-6, check_every=50, max_steps=5000)
    assert all(50 <= s <= 5000 for s in steps)
    for c in chans:
        d = c.diagnostics()
        assert abs(d["max_norm"] - 1) < 1e-6 and d["nonfinite"] == 0


def test_trained_network_saves_relaxation_steps(env):
    """The gain over the method without the network, on a small version of the
    warm-start experiment (48x48x16 cells, wide enough that a tube does not feel
    its periodic images): the plain relaxation continued from the trained
    network's prediction ends on the field of the relaxation from the ansatz
    (max |dn| <= 1e-4 once both are continued to a four times smaller stop
    rate) from a start several times closer to it, in fewer FD steps to the
    ordinary stop rate."""
    torch, nh, ws, U = env
    samples = I.warmstart_samples(176, seed=3, nx=48, ny=48, lz_choices=(16,))
    kw = dict(tol=2e-10, max_steps=160000)
    targets, steps, _ = ws.generate(samples, **kw)
    valid = [i for i in range(len(samples)) if not ws.collapsed(targets[i], samples[i][0]["nz"])]
    train_idx = [i for i in valid if i < 160]
    test_idx = [i for i in valid if i >= 160]
    assert len(train_idx) >= 150 and len(test_idx) >= 14
    net = ws.WarmStartNet(seed=0)
    hist = ws.train(net, samples, targets, train_idx, epochs=60)
    assert hist[-1] < 0.5 * hist[0]
    res = ws.evaluate(net, samples, targets, steps, test_idx, judge_tol=5e-11, **kw)
    print("warm start (48x48x16):", {k: v for k, v in res.items() if k != "per_sample"})
    for ps in sorted(res["per_sample"], key=lambda q: -q["max_dn"])[:3]:
        print("  worst held-out samples:", ps)
    assert res["max_dn_final"] <= 1e-4
    # the prediction starts several times closer (RMS over the cell) to the
    # relaxed field than the ansatz; relaxation to the stop tolerance is
    # exponential in time, so this buys a modest number of FD steps at this
    # training size
    # the median RMS distance to the relaxed field drops to 0.49-0.61 of the
    # ansatz's in repeated runs (the training trajectory varies with the
    # summation order of the FP32 gradient atomics and of the tensor-core
    # accumulation); 0.75 leaves room for that and still asks for a clear gain
    assert res["median_rms_prediction_vs_relaxed"] < 0.75 * res["median_rms_ansatz_vs_relaxed"]
    assert res["step_ratio"] < 0.98
