"""CPU FP64 oracle of the learned warm start and diagonal correction.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import this module.  It shares no code with
the CUDA library and nothing on the product path calls it.

The paper has no learned component; this part of the method is defined here
(the written definition the GPU network follows):

  * Input planes, per pixel: [f, ln sigma, ln alpha] (f the noisy image).
  * A 4-level U-Net with base width C = 32: per level two 3x3 convolutions
    (zero padding, bias, ReLU) with C, 2C, 4C, 8C channels; 2x2 average
    pooling between encoder levels; nearest-neighbour 2x upsampling, then
    concatenation [upsampled, skip] on the way up; a final 1x1 convolution to
    2 channels (o0, o1) without activation.
  * Outputs: the initial guess u0 = mean(f) 1 + o0 (an untrained network,
    o0 = 0, gives the deflated solver's own start, (mean(b) / alpha) 1 with
    b = alpha f) and the log-correction c = clamp(o1, -4, 4) of the Jacobi
    preconditioner, P_c = P_a * exp(c), P_a = alpha + max(d - 1, 0) with
    d = Gamma_full 1.
  * Loss of one sample (u* the converged solution, r0 = b - A u0 and
    e0 = u* - u0 for a snapshot of u0, both treated as data, beta >= 0):
        l = ||P_a (u0 - u*)||^2 / ||b - mean(b) 1||^2
            + beta ||r0 / (P_a exp(c)) - e0||^2 / ||e0||^2,
    averaged over the batch.  The first term measures the initial error the
    way the residual b - A u0 = A (u* - u0) does for its rough part (A acts
    like P_a on components that Gamma averages away) and is normalised by
    the residual of the solver's own start, b - mean(b) 1.  The second term
    fits a diagonal that maps the initial residual to the initial error (the
    one-step ideal preconditioner).
  * Adam (Kingma & Ba 2015, Algorithm 1) on all parameters.

Canonical parameter layout (float, one flat vector): for every 3x3 layer in
the order of `layers()`, weights [cout][3][3][cin] then bias [cout]; then the
head, weights [2][C] and bias [2].

`forward(..., bf16=True)` rounds the values the GPU stores in bfloat16 (the
3x3 weights, the input planes, every convolution and pooling output) to
bfloat16, round-to-nearest-even: the difference to the exact network is the
size of the bfloat16 effect that bounds the GPU's parity.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np


@dataclass(frozen=True)
class Layer:
    name: str
    cin: int
    cout: int
    k: int  # 3 (3x3 convolution + ReLU) or 1 (the linear head)


def layers(base: int = 32, levels: int = 4, in_planes: int = 3) -> List[Layer]:
    """The layer list of the U-Net, in parameter order."""
    out: List[Layer] = []
    ch = [base << l for l in range(levels)]
    cin = in_planes
    for l in range(levels):
        out.append(Layer("enc%da" % l, cin, ch[l], 3))
        out.append(Layer("enc%db" % l, ch[l], ch[l], 3))
        cin = ch[l]
    for l in range(levels - 2, -1, -1):
        out.append(Layer("dec%da" % l, ch[l + 1] + ch[l], ch[l], 3))
        out.append(Layer("dec%db" % l, ch[l], ch[l], 3))
    out.append(Layer("head", base, 2, 1))
    return out


def param_count(base: int = 32, levels: int = 4) -> int:
    return sum(l.cout * l.k * l.k * l.cin + l.cout for l in layers(base, levels))


def unpack(theta: np.ndarray, base: int = 32, levels: int = 4) -> Dict[str, Tuple[np.ndarray, np.ndarray]]:
    """Split the flat parameter vector into {name: (W, b)} (W as [cout, k, k, cin])."""
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for l in layers(base, levels):
        nw = l.cout * l.k * l.k * l.cin
        W = theta[o:o + nw].reshape(l.cout, l.k, l.k, l.cin)
        o += nw
        b = theta[o:o + l.cout]
        o += l.cout
        out[l.name] = (W, b)
    assert o == theta.size, (o, theta.size)
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) through float32."""
    x32 = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = x32.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# ---- layers (NHWC arrays: batch, rows, columns, channels) -----------------

def conv3x3(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n, i, j, o] = b[o] + sum_{dy, dx, c} W[o, dy, dx, c] x[n, i+dy-1, j+dx-1, c],
    zero outside the image (cross-correlation, as in deep-learning convolution)."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, H, Wd, W.shape[0]))
    for dy in range(3):
        for dx in range(3):
            y += np.tensordot(xp[:, dy:dy + H, dx:dx + Wd, :], W[:, dy, dx, :], axes=([3], [1]))
    return y + b


def relu(x):
    return np.maximum(x, 0.0)


def avgpool2(x: np.ndarray) -> np.ndarray:
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def upsample2(x: np.ndarray) -> np.ndarray:
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def input_planes(f: np.ndarray, sigma, alpha) -> np.ndarray:
    """[f, ln sigma, ln alpha] per pixel; f of shape (B, H, W)."""
    B = f.shape[0]
    s = np.broadcast_to(np.log(np.asarray(sigma, dtype=np.float64)).reshape(-1), (B,))
    a = np.broadcast_to(np.log(np.asarray(alpha, dtype=np.float64)).reshape(-1), (B,))
    x = np.empty(f.shape + (3,))
    x[..., 0] = f
    x[..., 1] = s[:, None, None]
    x[..., 2] = a[:, None, None]
    return x


def forward(theta, f, sigma, alpha, base: int = 32, levels: int = 4, bf16: bool = False):
    """Return (o, u0, c): the raw head outputs o (B, H, W, 2), u0 and c.

    H and W must be multiples of 2^(levels-1)."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 2:
        f = f[None]
    P = unpack(theta, base, levels)
    rnd = bf16_round if bf16 else (lambda a: a)

    def conv(name, x):
        W, b = P[name]
        return rnd(relu(conv3x3(x, rnd(W), b)))

    x = rnd(input_planes(f, sigma, alpha))
    skips = []
    for l in range(levels):
        if l > 0:
            x = rnd(avgpool2(x))
        x = conv("enc%db" % l, conv("enc%da" % l, x))
        skips.append(x)
    for l in range(levels - 2, -1, -1):
        x = np.concatenate([upsample2(x), skips[l]], axis=3)
        x = conv("dec%db" % l, conv("dec%da" % l, x))
    Wh, bh = P["head"]
    o = np.tensordot(x, Wh[:, 0, 0, :], axes=([3], [1])) + bh
    u0 = f.mean(axis=(1, 2))[:, None, None] + o[..., 0]
    c = np.clip(o[..., 1], -4.0, 4.0)
    return o, u0, c


def loss(theta, f, sigma, alpha, ustar, r0, e0, pa, beta: float,
         base: int = 32, levels: int = 4, bf16: bool = False) -> float:
    """The batch-mean training loss defined in the module docstring."""
    f = np.asarray(f, dtype=np.float64)
    if f.ndim == 2:
        f, ustar, r0, e0, pa = (np.asarray(a, dtype=np.float64)[None]
                                for a in (f, ustar, r0, e0, pa))
    _, u0, c = forward(theta, f, sigma, alpha, base, levels, bf16)
    B = f.shape[0]
    tot = 0.0
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64).reshape(-1), (B,))
    for n in range(B):
        lu = (np.sum((pa[n] * (u0[n] - ustar[n])) ** 2)
              / np.sum((alpha[n] * (f[n] - f[n].mean())) ** 2))
        pr = r0[n] / (pa[n] * np.exp(c[n]))
        lc = np.sum((pr - e0[n]) ** 2) / np.sum(e0[n] ** 2) if beta > 0 else 0.0
        tot += lu + beta * lc
    return tot / B


def adam(theta, grad, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
         eps: float = 1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1); returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def directional_fd(fun, theta, direction, h: float = 1e-5) -> float:
    """Central finite difference of fun along a direction (exact for
    quadratics; O(h^2) error otherwise)."""
    return (fun(theta + h * direction) - fun(theta - h * direction)) / (2.0 * h)
