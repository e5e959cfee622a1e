"""Pins of the U-Net oracle against things other than itself: hand-checked
BF16 rounding, torch's BF16 conversion, a brute-force convolution, torch's
conv3d, adjoint identities of every linear operator, and the whole
network's hand-written gradient against torch autograd and finite
differences."""
import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_2303_04679_gb300 import inputs


def test_bf16_rounding_hand_values():
    one = 1.0
    assert U.bf16(one + 2.0 ** -8) == 1.0                       # tie, even mantissa kept
    assert U.bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6       # tie, rounds up to even
    assert U.bf16(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7
    assert U.bf16(-(one + 2.0 ** -7)) == -(one + 2.0 ** -7)     # representable


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(0).normal(0, 3, size=10000).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.bf16(x), ref)


def _brute_conv(X, W, b):
    B, S, _, _, C = X.shape
    O = W.shape[0]
    Y = np.zeros((B, S, S, S, O))
    taps = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    for n in range(B):
        for z in range(S):
            for y in range(S):
                for x in range(S):
                    for o in range(O):
                        s = b[o]
                        for t, (dz, dy, dx) in enumerate(taps):
                            zz, yy, xx = z + dz, y + dy, x + dx
                            if 0 <= zz < S and 0 <= yy < S and 0 <= xx < S:
                                s += float(np.dot(X[n, zz, yy, xx], W[o, t]))
                        Y[n, z, y, x, o] = s
    return Y


def test_conv3_brute_force():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(2, 3, 3, 3, 2))
    W = rng.normal(size=(3, 27, 2))
    b = rng.normal(size=3)
    assert np.allclose(U.conv3(X, W, b), _brute_conv(X, W, b), rtol=0, atol=1e-12)


def test_conv3_matches_torch_conv3d():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    X = rng.normal(size=(2, 5, 5, 5, 3))
    W = rng.normal(size=(4, 27, 3))
    Wt = torch.from_numpy(W.reshape(4, 3, 3, 3, 3).transpose(0, 4, 1, 2, 3).copy())  # O, C, kd, kh, kw
    Yt = torch.nn.functional.conv3d(torch.from_numpy(X.transpose(0, 4, 1, 2, 3).copy()), Wt, padding=1)
    assert np.allclose(U.conv3(X, W), Yt.numpy().transpose(0, 2, 3, 4, 1), atol=1e-12)


def test_adjoint_identities():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(2, 4, 4, 4, 3))
    W = rng.normal(size=(5, 27, 3))
    G = rng.normal(size=(2, 4, 4, 4, 5))
    lhs = np.sum(U.conv3(X, W) * G)
    assert np.isclose(lhs, np.sum(X * U.conv3_input_grad(G, W)), rtol=1e-12)
    assert np.isclose(lhs, np.sum(W * U.conv3_weight_grad(X, G)), rtol=1e-12)
    P = rng.normal(size=(2, 2, 2, 2, 3))
    assert np.isclose(np.sum(U.pool(X) * P), np.sum(X * U.pool_adjoint(P)), rtol=1e-12)
    assert np.isclose(np.sum(U.up(P) * X), np.sum(P * U.up_adjoint(X)), rtol=1e-12)


def _torch_net(spec, params, x):
    import torch
    F = torch.nn.functional
    L = spec.levels
    it = iter(params)

    def conv(a, W, b, taps=27):
        o, t, ci = W.shape
        if taps == 1:
            return torch.einsum("bzyxc,oc->bzyxo", a, W[:, 0, :]) + b
        Wt = W.reshape(o, 3, 3, 3, ci).permute(0, 4, 1, 2, 3)
        return F.conv3d(a.permute(0, 4, 1, 2, 3), Wt, b, padding=1).permute(0, 2, 3, 4, 1)

    xp = torch.zeros(x.shape[:4] + (spec.in_pad,), dtype=torch.float64)
    xp[..., :spec.in_ch] = x
    e = []
    inp = xp
    for l in range(L):
        if l > 0:
            inp = F.avg_pool3d(e[-1].permute(0, 4, 1, 2, 3), 2).permute(0, 2, 3, 4, 1)
        Wa, ba, Wb, bb = next(it), next(it), next(it), next(it)
        a = torch.relu(conv(inp, Wa, ba))
        e.append(torch.relu(conv(a, Wb, bb)))
    below = e[L - 1]
    for l in range(L - 2, -1, -1):
        Wc, bc, Wd, bd = next(it), next(it), next(it), next(it)
        u = torch.cat([below.repeat_interleave(2, 1).repeat_interleave(2, 2).repeat_interleave(2, 3), e[l]], -1)
        below = torch.relu(conv(torch.relu(conv(u, Wc, bc)), Wd, bd))
    Wh, bh = next(it), next(it)
    return conv(below, Wh, bh, taps=1)


def test_network_gradient_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    spec = U.Spec(levels=3, base=8, in_ch=4, out_ch=5)
    params = [p.astype(np.float64) for p in inputs.unet_params(spec.param_shapes(), 5, bias_scale=0.1)]
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2, 8, 8, 8, 4))
    y = rng.normal(size=(2, 8, 8, 8, 5))
    loss, grads = U.loss_and_grads(spec, params, x, y, emulate=False)
    tp = [torch.tensor(p, requires_grad=True) for p in params]
    out = _torch_net(spec, tp, torch.from_numpy(x))
    tl = ((out - torch.from_numpy(y)) ** 2).mean()
    tl.backward()
    assert np.isclose(loss, tl.item(), rtol=1e-12)
    for g, t in zip(grads, tp):
        ref = t.grad.numpy()
        assert np.allclose(g, ref, rtol=1e-9, atol=1e-12 * np.max(np.abs(ref))), np.max(np.abs(g - ref))


def test_network_gradient_finite_differences():
    spec = U.Spec(levels=2, base=8, in_ch=4, out_ch=5)
    params = [p.astype(np.float64) for p in inputs.unet_params(spec.param_shapes(), 7, bias_scale=0.1)]
    rng = np.random.default_rng(8)
    x = rng.normal(size=(1, 4, 4, 4, 4))
    y = rng.normal(size=(1, 4, 4, 4, 5))
    _, grads = U.loss_and_grads(spec, params, x, y, emulate=False)
    for k in (0, 3, 5, len(params) - 2):
        flat = params[k].reshape(-1)
        for j in rng.choice(flat.size, size=3, replace=False):
            h = 1e-6
            old = flat[j]
            flat[j] = old + h
            lp = U.loss_and_grads(spec, params, x, y, emulate=False)[0]
            flat[j] = old - h
            lm = U.loss_and_grads(spec, params, x, y, emulate=False)[0]
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[k].reshape(-1)[j]) <= 1e-6 * max(1.0, abs(fd)), (k, j, fd)
