"""Pins of the network oracle (oracle/unet.py) against library routines,
closed forms and finite differences.

The oracle's layers are checked against PyTorch's CPU float64 operators
(conv2d, avg_pool2d, nearest interpolation, bfloat16 casts), the wiring of
the whole U-Net against an independent composition of those operators, its
finite-difference derivative against autograd, and the loss and the Adam step
against closed forms.
"""
import numpy as np
import pytest

from oracle import unet
from paper_2407_06834_gb300.inputs import net_init, synthetic_image

torch = pytest.importorskip("torch")
F = torch.nn.functional


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _theta(base, levels, seed=0):
    shapes = [(l.cout, l.k, l.cin) for l in unet.layers(base, levels)]
    return net_init(shapes, seed).astype(np.float64)


def test_layer_structure():
    ls = unet.layers(32, 4)
    assert [l.name for l in ls][:2] == ["enc0a", "enc0b"] and ls[-1].name == "head"
    assert len(ls) == 2 * 4 + 2 * 3 + 1
    widths = [l.cout for l in ls if l.name.endswith("b") and l.name.startswith("enc")]
    assert widths == [32, 64, 128, 256]
    # decoder inputs: upsampled coarser level + skip of this level
    dec = {l.name: l for l in ls}
    assert dec["dec2a"].cin == 256 + 128 and dec["dec0a"].cin == 64 + 32
    theta = _theta(32, 4)
    assert theta.size == unet.param_count(32, 4)
    P = unet.unpack(theta)
    assert P["enc0a"][0].shape == (32, 3, 3, 3) and P["head"][0].shape == (2, 1, 1, 32)


def test_conv3x3_equals_torch_conv2d():
    r = _rng(1)
    x = r.standard_normal((2, 9, 7, 5))
    W = r.standard_normal((4, 3, 3, 5))
    b = r.standard_normal(4)
    y = unet.conv3x3(x, W, b)
    ref = F.conv2d(torch.from_numpy(x).permute(0, 3, 1, 2), torch.from_numpy(W).permute(0, 3, 1, 2),
                   torch.from_numpy(b), padding=1).permute(0, 2, 3, 1).numpy()
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)
    # a single tap picks the shifted input: W[o, 0, 2, c] reads x[i-1, j+1]
    W1 = np.zeros((1, 3, 3, 1))
    W1[0, 0, 2, 0] = 1.0
    xs = r.standard_normal((1, 5, 6, 1))
    y1 = unet.conv3x3(xs, W1, np.zeros(1))[0, :, :, 0]
    assert y1[2, 3] == xs[0, 1, 4, 0] and y1[0, 0] == 0.0 and y1[3, 5] == 0.0


def test_pool_upsample_and_bf16_equal_torch():
    r = _rng(2)
    x = r.standard_normal((2, 8, 6, 3))
    t = torch.from_numpy(x).permute(0, 3, 1, 2)
    np.testing.assert_allclose(unet.avgpool2(x), F.avg_pool2d(t, 2).permute(0, 2, 3, 1).numpy(),
                               rtol=1e-14)
    np.testing.assert_array_equal(unet.upsample2(x),
                                  F.interpolate(t, scale_factor=2, mode="nearest")
                                  .permute(0, 2, 3, 1).numpy())
    v = np.concatenate([r.standard_normal(4000) * 10.0 ** r.integers(-6, 6, 4000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.005859375, 3.0e38]])
    ref = torch.from_numpy(v).float().to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(unet.bf16_round(v), ref)


def _torch_unet(theta, base, levels):
    """The oracle's parameters as PyTorch conv2d weights (NCHW)."""
    return {k: (torch.from_numpy(np.ascontiguousarray(W)).permute(0, 3, 1, 2), torch.from_numpy(b))
            for k, (W, b) in unet.unpack(theta, base, levels).items()}


def _torch_forward(Pt, f, sigma, alpha, levels):
    B = f.shape[0]
    planes = [f,
              torch.log(torch.as_tensor(sigma, dtype=torch.float64)).reshape(B, 1, 1).expand_as(f),
              torch.log(torch.as_tensor(alpha, dtype=torch.float64)).reshape(B, 1, 1).expand_as(f)]
    x = torch.stack(planes, 1)
    skips = []
    for l in range(levels):
        if l:
            x = F.avg_pool2d(x, 2)
        for s in "ab":
            W, b = Pt["enc%d%s" % (l, s)]
            x = F.relu(F.conv2d(x, W, b, padding=1))
        skips.append(x)
    for l in range(levels - 2, -1, -1):
        x = torch.cat([F.interpolate(x, scale_factor=2, mode="nearest"), skips[l]], 1)
        for s in "ab":
            W, b = Pt["dec%d%s" % (l, s)]
            x = F.relu(F.conv2d(x, W, b, padding=1))
    W, b = Pt["head"]
    return F.conv2d(x, W, b)


def test_forward_equals_torch_composition():
    base, levels = 32, 3
    theta = _theta(base, levels, 3)
    theta[-2:] = [0.05, -0.2]
    r = _rng(4)
    f = np.stack([synthetic_image(16, 24, s)[1] for s in (1, 2)])
    sig, alp = np.array([0.2, 0.07]), np.array([0.5, 3.0])
    o, u0, c = unet.forward(theta, f, sig, alp, base, levels)
    Pt = _torch_unet(theta, base, levels)
    ot = _torch_forward(Pt, torch.from_numpy(f), sig, alp, levels).permute(0, 2, 3, 1).numpy()
    np.testing.assert_allclose(o, ot, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(u0, f.mean(axis=(1, 2))[:, None, None] + ot[..., 0], rtol=1e-12)
    assert np.all(np.abs(c) <= 4.0)
    # the bf16 emulation stays within bfloat16 resolution of the exact network
    ob, _, _ = unet.forward(theta, f, sig, alp, base, levels, bf16=True)
    assert np.max(np.abs(ob - o)) < 0.05 * np.max(np.abs(o)) and np.any(ob != o)


def _loss_data(seed, B, H, W):
    r = _rng(seed)
    f = np.stack([synthetic_image(H, W, 50 + i)[1] for i in range(B)])
    ustar = f + 0.05 * r.standard_normal(f.shape)
    r0 = r.standard_normal(f.shape)
    e0 = r.standard_normal(f.shape)
    pa = 0.5 + r.uniform(0.0, 3.0, f.shape)
    return f, ustar, r0, e0, pa


def test_loss_closed_forms():
    """All 3x3 weights and biases zero: o = head bias everywhere."""
    base, levels = 32, 2
    theta = np.zeros(unet.param_count(base, levels))
    f, _, r0, e0, pa = _loss_data(5, 2, 8, 8)
    fbar = f.mean(axis=(1, 2))[:, None, None]
    ustar = fbar + 0.3 + 0.0 * f
    sig, alp = [0.2, 0.3], [0.5, 0.1]
    theta[-2:] = [0.3, 0.7]
    r0 = pa * np.exp(0.7) * e0
    assert unet.loss(theta, f, sig, alp, ustar, r0, e0, pa, 2.0, base, levels) == pytest.approx(0.0, abs=1e-24)
    # u0 - u* = 0.01 everywhere: sum (0.01 P_a)^2 / ||alpha (f - mean f)||^2
    theta[-2] = 0.3 + 0.01
    lu = np.mean([np.sum((0.01 * pa[n]) ** 2) / np.sum((alp[n] * (f[n] - f[n].mean())) ** 2)
                  for n in range(2)])
    assert unet.loss(theta, f, sig, alp, ustar, r0, e0, pa, 2.0, base, levels) == pytest.approx(lu, rel=1e-9)
    # beyond the clamp c stays at 4
    theta[-1] = 9.0
    _, _, c = unet.forward(theta, f, sig, alp, base, levels)
    assert np.all(c == 4.0)


def test_finite_difference_matches_autograd():
    """The oracle's loss differentiated by central differences equals the
    autograd gradient of the PyTorch composition (float64), along random
    directions."""
    base, levels = 32, 2
    theta = _theta(base, levels, 6)
    theta[-2:] = [0.02, 0.1]
    f, ustar, r0, e0, pa = _loss_data(7, 2, 8, 8)
    sig, alp = np.array([0.2, 0.4]), np.array([0.5, 2.0])
    beta = 0.5
    th = torch.tensor(theta, requires_grad=True)
    # PyTorch loss over the same flat layout
    o = 0
    Pt = {}
    for l in unet.layers(base, levels):
        nw = l.cout * l.k * l.k * l.cin
        W = th[o:o + nw].reshape(l.cout, l.k, l.k, l.cin).permute(0, 3, 1, 2)
        b = th[o + nw:o + nw + l.cout]
        o += nw + l.cout
        Pt[l.name] = (W, b)
    out = _torch_forward(Pt, torch.from_numpy(f), sig, alp, levels)
    ft, ut, rt, et, pt = (torch.from_numpy(a) for a in (f, ustar, r0, e0, pa))
    fbar = ft.mean((1, 2), keepdim=True)
    u0 = fbar + out[:, 0]
    c = torch.clamp(out[:, 1], -4.0, 4.0)
    at = torch.from_numpy(alp).reshape(-1, 1, 1)
    lu = ((pt * (u0 - ut)) ** 2).sum((1, 2)) / ((at * (ft - fbar)) ** 2).sum((1, 2))
    lc = ((rt / (pt * torch.exp(c)) - et) ** 2).sum((1, 2)) / (et ** 2).sum((1, 2))
    (lu + beta * lc).mean().backward()
    g = th.grad.numpy()
    fun = lambda t: unet.loss(t, f, sig, alp, ustar, r0, e0, pa, beta, base, levels)
    r = _rng(8)
    for _ in range(3):
        d = r.standard_normal(theta.size)
        fd = unet.directional_fd(fun, theta, d, h=1e-6)
        assert fd == pytest.approx(g @ d, rel=1e-6)
    # single parameters in the first layer and the head
    for idx in (5, theta.size - 3):
        e = np.zeros(theta.size)
        e[idx] = 1.0
        assert unet.directional_fd(fun, theta, e, h=1e-6) == pytest.approx(g[idx], rel=1e-5, abs=1e-10)


def test_adam_closed_form():
    """First Adam step: m_hat = g, v_hat = g^2, so theta moves by
    lr * g / (|g| + eps); with a constant gradient every step does."""
    r = _rng(9)
    theta = r.standard_normal(50)
    g = r.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    t1, m, v = unet.adam(theta, g, m, v, 1, 1e-2)
    np.testing.assert_allclose(t1, theta - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    t2, m, v = unet.adam(t1, g, m, v, 2, 1e-2)
    np.testing.assert_allclose(t2, t1 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)
