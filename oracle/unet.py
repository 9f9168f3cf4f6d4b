"""FP64 CPU oracle of the warm-start network (plain PyTorch CPU ops, float64).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: used by tests only, to check the CUDA
kernels of the learned warm start (forward, backward, Adam).  It shares no code
with the CUDA library; only the parameter layout below (an interface) is the
same on both sides.

Network (a 3D U-Net with 4 levels):
  input  x: 16 channels = director ansatz (3), q0 * Lz / (2 pi), Lz / 32,
            W0 / 1e-3, then zeros
  enc1a 16->16, enc1b 16->16                (conv 3x3x3 + ReLU)   -> e1
  pool (2x2x2 mean), enc2a 16->16, enc2b 16->16                   -> e2
  pool, enc3a 16->32, enc3b 32->32                                -> e3
  pool, bota 32->64, botb 64->64                                  -> b
  up (nearest x2), concat [up | e3], dec3a 96->32, dec3b 32->32    -> d3
  up, concat [up | e2], dec2a 48->16, dec2b 16->16                 -> d2
  up, concat [up | e1], dec1a 32->16, dec1b 16->16                 -> d1
  head: 1x1x1 conv 16->3 (no ReLU) -> delta;  n = normalise(n_ansatz + delta)
Convolutions are cross-correlations with periodic padding in x and y and zero
padding in z.

Parameter layout (flat FP32 vector on the GPU, float64 here), layer by layer
in the order above: weights W[tap][cout][cin] with tap = 9*kz + 3*ky + kx
(kx, ky, kz in 0..2 for offsets -1, 0, +1), then bias[cout]; the head is
W[3][16] then bias[3].
Tensor layout here: torch NCDHW, i.e. [batch][channel][z][y][x].
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CONV_LAYERS = [
    ("enc1a", 16, 16), ("enc1b", 16, 16),
    ("enc2a", 16, 16), ("enc2b", 16, 16),
    ("enc3a", 16, 32), ("enc3b", 32, 32),
    ("bota", 32, 64), ("botb", 64, 64),
    ("dec3a", 96, 32), ("dec3b", 32, 32),
    ("dec2a", 48, 16), ("dec2b", 16, 16),
    ("dec1a", 32, 16), ("dec1b", 16, 16),
]
HEAD = ("head", 16, 3)
IN_CHANNELS = 16


def param_count() -> int:
    n = sum(27 * ci * co + co for _, ci, co in CONV_LAYERS)
    return n + HEAD[1] * HEAD[2] + HEAD[2]


def unpack(flat):
    """Flat parameter vector -> dict name -> (W torch [cout][cin][3][3][3], b)."""
    flat = torch.as_tensor(np.asarray(flat, dtype=np.float64))
    out = {}
    off = 0
    for name, ci, co in CONV_LAYERS:
        w = flat[off:off + 27 * co * ci].reshape(3, 3, 3, co, ci)       # [kz][ky][kx][co][ci]
        off += 27 * co * ci
        b = flat[off:off + co]
        off += co
        out[name] = (w.permute(3, 4, 0, 1, 2).contiguous(), b)          # -> [co][ci][kz][ky][kx]
    _, ci, co = HEAD
    w = flat[off:off + co * ci].reshape(co, ci)
    off += co * ci
    out["head"] = (w, flat[off:off + co])
    off += co
    assert off == flat.numel()
    return out


def pack(params) -> np.ndarray:
    parts = []
    for name, ci, co in CONV_LAYERS:
        w, b = params[name]
        parts.append(w.permute(2, 3, 4, 0, 1).reshape(-1))
        parts.append(b.reshape(-1))
    w, b = params["head"]
    parts += [w.reshape(-1), b.reshape(-1)]
    return torch.cat(parts).detach().numpy()


def conv3(x, w, b):
    """3x3x3 cross-correlation, periodic in x and y, zero-padded in z."""
    xp = F.pad(x, (1, 1, 1, 1, 0, 0), mode="circular")
    xp = F.pad(xp, (0, 0, 0, 0, 1, 1), mode="constant", value=0.0)
    return F.conv3d(xp, w, b)


def pool(x):
    return F.avg_pool3d(x, 2)


def up(x):
    return x.repeat_interleave(2, dim=2).repeat_interleave(2, dim=3).repeat_interleave(2, dim=4)


def _bf16(t):
    return t.to(torch.bfloat16).to(t.dtype)


class _RoundGrad(torch.autograd.Function):
    """Identity in the forward pass; rounds the gradient to BF16 (the operand of a BF16 matrix product)."""

    @staticmethod
    def forward(ctx, t):
        return t.clone()

    @staticmethod
    def backward(ctx, g):
        return _bf16(g)


class _RoundFwd(torch.autograd.Function):
    """Rounds to BF16 in the forward pass only (a BF16 copy whose gradient stays in FP32)."""

    @staticmethod
    def forward(ctx, t):
        return _bf16(t)

    @staticmethod
    def backward(ctx, g):
        return g


def forward(params, x, n_ansatz, bf16_storage=False, keep=None):
    """x [B][16][Z][Y][X], n_ansatz [B][3][Z][Y][X] -> (n_pred, delta).

    bf16_storage=True keeps every stored activation in BF16 and rounds the
    gradient entering each convolution's weight and data products to BF16, as a
    BF16-activation implementation does, while the bias gradient sums the
    unrounded gradient of the pre-activation (an FP32 reduction); the
    arithmetic itself stays float64."""
    rf = _RoundFwd.apply if bf16_storage else (lambda t: t)
    rg = _RoundGrad.apply if bf16_storage else (lambda t: t)

    def r(name, t):
        w, b = params[name]
        pre = rg(conv3(t, w, None)) + b.view(1, -1, 1, 1, 1)
        y = rf(F.relu(pre))
        if keep is not None:
            keep[name] = y.detach()
        return y

    e1 = r("enc1b", r("enc1a", x))
    e2 = r("enc2b", r("enc2a", rf(pool(e1))))
    e3 = r("enc3b", r("enc3a", rf(pool(e2))))
    bt = r("botb", r("bota", rf(pool(e3))))
    d3 = r("dec3b", r("dec3a", torch.cat([up(bt), e3], dim=1)))
    d2 = r("dec2b", r("dec2a", torch.cat([up(d3), e2], dim=1)))
    d1 = r("dec1b", r("dec1a", torch.cat([up(d2), e1], dim=1)))
    w, b = params["head"]
    delta = torch.einsum("oc,bczyx->bozyx", w, d1) + b.view(1, -1, 1, 1, 1)
    v = n_ansatz + delta
    return v / torch.linalg.vector_norm(v, dim=1, keepdim=True), delta


def loss_fn(n_pred, n_target):
    """Mean over sites of |n_pred - n_target|^2."""
    return ((n_pred - n_target) ** 2).sum(dim=1).mean()


def loss_and_grad(flat, x, n_ansatz, n_target, bf16_storage=False):
    """Loss and d loss / d params (flat layout) by autograd in float64."""
    flat_t = torch.tensor(np.asarray(flat, dtype=np.float64), requires_grad=True)
    params = unpack_tensor(flat_t)
    n_pred, _ = forward(params, x, n_ansatz, bf16_storage)
    loss = loss_fn(n_pred, n_target)
    loss.backward()
    return float(loss.detach()), flat_t.grad.numpy().copy(), n_pred.detach()


def unpack_tensor(flat_t):
    out = {}
    off = 0
    for name, ci, co in CONV_LAYERS:
        w = flat_t[off:off + 27 * co * ci].reshape(3, 3, 3, co, ci).permute(3, 4, 0, 1, 2)
        off += 27 * co * ci
        out[name] = (w, flat_t[off:off + co])
        off += co
    _, ci, co = HEAD
    out["head"] = (flat_t[off:off + co * ci].reshape(co, ci), flat_t[off + co * ci:off + co * ci + co])
    return out


def make_input(n_ansatz, q0, lz, w0):
    """Network input from the ansatz [B][3][Z][Y][X] and per-sample scalars."""
    n_ansatz = torch.as_tensor(n_ansatz, dtype=torch.float64)
    B = n_ansatz.shape[0]
    x = torch.zeros((B, IN_CHANNELS) + tuple(n_ansatz.shape[2:]), dtype=torch.float64)
    x[:, :3] = n_ansatz
    for k in range(B):
        x[k, 3] = q0[k] * lz[k] / (2 * np.pi)
        x[k, 4] = lz[k] / 32.0
        x[k, 5] = w0[k] / 1e-3
    return x


def adam(flat, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1), returns (flat, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return flat - lr * mhat / (np.sqrt(vhat) + eps), m, v
