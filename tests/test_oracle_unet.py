"""Pins of the warm-start network oracle (plain PyTorch CPU float64).

* the 3x3x3 convolution equals a brute-force loop over taps with periodic x, y
  and zero z padding (the definition written out on a tiny grid);
* nearest upsampling is 8 x the adjoint of 2x2x2 mean pooling;
* parameter gradients equal central finite differences of the loss;
* the first Adam step moves every parameter by -lr sign(g) (bias-corrected
  moments reduce to g and g^2);
* the parameter table agrees with the input module's generator.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as U
from paper_2503_06610_gb300 import inputs as I


def test_conv3_is_the_periodic_cross_correlation():
    rng = np.random.default_rng(0)
    B, ci, co, Z, Y, X = 2, 3, 4, 3, 4, 5
    x = torch.tensor(rng.normal(size=(B, ci, Z, Y, X)))
    w = torch.tensor(rng.normal(size=(co, ci, 3, 3, 3)))
    b = torch.tensor(rng.normal(size=co))
    out = U.conv3(x, w, b).numpy()
    ref = np.zeros((B, co, Z, Y, X))
    xn, wn = x.numpy(), w.numpy()
    for bb in range(B):
        for o in range(co):
            for z in range(Z):
                for y in range(Y):
                    for xx in range(X):
                        acc = b[o].item()
                        for kz in range(3):
                            zs = z + kz - 1
                            if zs < 0 or zs >= Z:
                                continue
                            for ky in range(3):
                                for kx in range(3):
                                    acc += np.dot(wn[o, :, kz, ky, kx], xn[bb, :, zs, (y + ky - 1) % Y, (xx + kx - 1) % X])
                        ref[bb, o, z, y, xx] = acc
    assert np.allclose(out, ref, atol=1e-12)


def test_upsample_is_adjoint_of_pool():
    rng = np.random.default_rng(1)
    a = torch.tensor(rng.normal(size=(1, 2, 2, 3, 4)))
    bb = torch.tensor(rng.normal(size=(1, 2, 4, 6, 8)))
    assert abs(float((U.up(a) * bb).sum()) - 8 * float((a * U.pool(bb)).sum())) < 1e-12


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    flat = I.unet_init_params(seed=3)
    flat[: len(flat) - 51] += 0.01 * rng.normal(size=len(flat) - 51)  # non-zero biases
    n0 = I.skyrmion_tubes(8, 8, 8, [(4.0, 4.0)], 3.0).reshape(1, 3, 8, 8, 8)
    x = U.make_input(n0, [0.5], [8], [1e-5])
    target = torch.tensor(I.random_director(8, 8, 8, seed=4).reshape(1, 3, 8, 8, 8))
    n0t = torch.tensor(n0)
    loss, grad, _ = U.loss_and_grad(flat, x, n0t, target)
    idx = rng.choice(len(flat), size=24, replace=False)
    idx = np.concatenate([idx, [len(flat) - 1, len(flat) - 10, 5, 27 * 16 * 16 + 3]])
    for i in idx:
        h = 1e-6
        fp = flat.copy()
        fp[i] += h
        fm = flat.copy()
        fm[i] -= h
        lp = float(U.loss_fn(U.forward(U.unpack(fp), x, n0t)[0], target))
        lm = float(U.loss_fn(U.forward(U.unpack(fm), x, n0t)[0], target))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])), (i, fd, grad[i])


def test_first_adam_step_is_signed_lr():
    rng = np.random.default_rng(5)
    flat = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = U.adam(flat, g, np.zeros(50), np.zeros(50), step=1, lr=1e-3)
    assert np.allclose(new - flat, -1e-3 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-9, atol=0)
    assert np.allclose(new - flat, -1e-3 * np.sign(g), rtol=1e-5, atol=0)


def test_parameter_tables_agree():
    assert [(n, a, b) for n, a, b in U.CONV_LAYERS] == I.UNET_CONV_LAYERS
    assert (U.HEAD[1], U.HEAD[2]) == I.UNET_HEAD
    flat = I.unet_init_params(0)
    assert len(flat) == U.param_count()
    assert np.array_equal(U.pack(U.unpack(flat)), flat)
