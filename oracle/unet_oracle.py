"""CPU oracle of the learned warm start (test infrastructure only).

Plain numpy FP64 restatement of the 3-D U-Net that warm-starts the body
problem: 3x3x3 convolutions with zero padding, bias, ReLU, 2x2x2 average
pooling, nearest-neighbour upsampling, concatenation, a 1x1x1 output layer,
the mean-squared loss and its hand-written reverse pass.  The paper has no
network; the architecture is the one the library documents (encoder levels of
two convolutions, decoder levels of upsampling + concatenation + two
convolutions).

With ``emulate=True`` the oracle rounds to BF16 (round to nearest even) at
exactly the points where the device path stores BF16 -- the input, the
weights used in contractions, every activation after bias and ReLU, the
output gradient and every masked activation gradient -- and computes
everything else in FP64, so the device's FP32 accumulation is the only
difference.  With ``emulate=False`` it is the exact FP64 network.

Only tests, the package's smoke check and the benchmark's CPU baseline may
import this module.
"""
from __future__ import annotations

import numpy as np

__all__ = ["bf16", "conv3", "conv3_input_grad", "conv3_weight_grad", "pool", "pool_adjoint", "up",
           "up_adjoint", "Spec", "forward", "loss_and_grads"]


def bf16(x):
    """Round to the nearest BF16 value (ties to even); returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _taps():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shifted(Xp, S, dz, dy, dx):
    """X[v + (dz, dy, dx)] for every cell v of an S^3 grid, from the 1-padded Xp."""
    return Xp[:, 1 + dz:1 + dz + S, 1 + dy:1 + dy + S, 1 + dx:1 + dx + S, :]


def conv3(X, W, b=None):
    """Y[v, o] = sum_t sum_c X[v + off_t, c] W[o, t, c] (+ b[o]); zero outside.
    X: [B, S, S, S, C]; W: [O, 27, C]."""
    S = X.shape[1]
    Xp = np.pad(X, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    Y = np.zeros(X.shape[:4] + (W.shape[0],))
    for t, (dz, dy, dx) in enumerate(_taps()):
        Y += _shifted(Xp, S, dz, dy, dx) @ W[:, t, :].T
    if b is not None:
        Y += b
    return Y


def conv3_input_grad(G, W):
    """Adjoint of conv3 in X: dX[v, c] = sum_t sum_o G[v - off_t, o] W[o, t, c]."""
    S = G.shape[1]
    dXp = np.zeros(G.shape[:1] + (S + 2,) * 3 + (W.shape[2],))
    for t, (dz, dy, dx) in enumerate(_taps()):
        dXp[:, 1 + dz:1 + dz + S, 1 + dy:1 + dy + S, 1 + dx:1 + dx + S, :] += G @ W[:, t, :]
    return dXp[:, 1:-1, 1:-1, 1:-1, :]


def conv3_weight_grad(X, G):
    """Adjoint of conv3 in W: dW[o, t, c] = sum_v G[v, o] X[v + off_t, c]."""
    S = X.shape[1]
    Xp = np.pad(X, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    Gf = G.reshape(-1, G.shape[-1])
    dW = np.zeros((G.shape[-1], 27, X.shape[-1]))
    for t, (dz, dy, dx) in enumerate(_taps()):
        dW[:, t, :] = Gf.T @ _shifted(Xp, S, dz, dy, dx).reshape(-1, X.shape[-1])
    return dW


def pool(X):
    """2x2x2 average."""
    B, S, _, _, C = X.shape
    return X.reshape(B, S // 2, 2, S // 2, 2, S // 2, 2, C).mean(axis=(2, 4, 6))


def pool_adjoint(G):
    """Each fine cell receives 1/8 of its parent's value."""
    return up(G) / 8.0


def up(X):
    """Nearest-neighbour upsampling by 2 along each axis."""
    return X.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)


def up_adjoint(G):
    """Sum of the 8 children."""
    B, S, _, _, C = G.shape
    return G.reshape(B, S // 2, 2, S // 2, 2, S // 2, 2, C).sum(axis=(2, 4, 6))


class Spec:
    """levels, base channels, input channels (padded to in_pad), output channels."""

    def __init__(self, levels=4, base=32, in_ch=4, out_ch=5, in_pad=8):
        self.levels, self.base, self.in_ch, self.out_ch, self.in_pad = levels, base, in_ch, out_ch, in_pad

    def channels(self, l):
        return self.base << l

    def param_shapes(self):
        """Parameter order: encoder levels (conv a, conv b), decoder levels from
        the deepest (conv c, conv d), the output layer; each as (weight, bias)."""
        out = []
        L = self.levels

        def add(cin, cout, taps=27):
            out.append((cout, taps, cin))
            out.append((cout,))
        for l in range(L):
            add(self.in_pad if l == 0 else self.channels(l - 1), self.channels(l))
            add(self.channels(l), self.channels(l))
        for l in range(L - 2, -1, -1):
            add(self.channels(l + 1) + self.channels(l), self.channels(l))
            add(self.channels(l), self.channels(l))
        add(self.channels(0), self.out_ch, taps=1)
        return out


def _unpack(spec, params):
    L = spec.levels
    it = iter(params)
    enc = [((next(it), next(it)), (next(it), next(it))) for _ in range(L)]
    dec = {}
    for l in range(L - 2, -1, -1):
        dec[l] = ((next(it), next(it)), (next(it), next(it)))
    head = (next(it), next(it))
    return enc, dec, head


def forward(spec, params, x, emulate=True):
    """Output [B, S, S, S, out_ch] and the activations the reverse pass needs.
    x: [B, S, S, S, in_ch]."""
    R = bf16 if emulate else (lambda a: np.asarray(a, dtype=np.float64))
    relu = lambda a: np.maximum(a, 0.0)  # noqa: E731
    enc, dec, head = _unpack(spec, params)
    L = spec.levels
    xp = np.zeros(x.shape[:4] + (spec.in_pad,))
    xp[..., :spec.in_ch] = x
    c = {"x0": R(xp), "inp": [], "a": [], "e": [], "u": {}, "b": {}, "d": {}}
    Wq = lambda W: R(W)  # noqa: E731  the contractions use the rounded weights
    for l in range(L):
        inp = c["x0"] if l == 0 else R(pool(c["e"][l - 1]))
        (Wa, ba), (Wb, bb) = enc[l]
        a = R(relu(conv3(inp, Wq(Wa), np.asarray(ba, np.float64))))
        e = R(relu(conv3(a, Wq(Wb), np.asarray(bb, np.float64))))
        c["inp"].append(inp)
        c["a"].append(a)
        c["e"].append(e)
    for l in range(L - 2, -1, -1):
        below = c["e"][L - 1] if l == L - 2 else c["d"][l + 1]
        u = np.concatenate([up(below), c["e"][l]], axis=-1)
        (Wc, bc), (Wd, bd) = dec[l]
        b = R(relu(conv3(u, Wq(Wc), np.asarray(bc, np.float64))))
        d = R(relu(conv3(b, Wq(Wd), np.asarray(bd, np.float64))))
        c["u"][l], c["b"][l], c["d"][l] = u, b, d
    Wh, bh = head
    out = c["d"][0] @ Wq(Wh)[:, 0, :].T + np.asarray(bh, np.float64)
    return out, c


def loss_and_grads(spec, params, x, y, emulate=True):
    """Loss mean((out - y)^2) and its gradient for every parameter (same order)."""
    R = bf16 if emulate else (lambda a: np.asarray(a, dtype=np.float64))
    mask = lambda act, g: np.where(act > 0, g, 0.0)  # noqa: E731
    L = spec.levels
    enc, dec, head = _unpack(spec, params)
    out, c = forward(spec, params, x, emulate)
    n = out.size
    diff = out - y
    loss = float(np.sum(diff * diff)) / n
    dout = R(2.0 * diff / n)
    Wh, _ = head
    d0 = c["d"][0]
    dWh = (dout.reshape(-1, dout.shape[-1]).T @ d0.reshape(-1, d0.shape[-1]))[:, None, :]
    dbh = dout.reshape(-1, dout.shape[-1]).sum(axis=0)
    g = R(mask(d0, dout @ R(Wh)[:, 0, :]))
    gd = {}
    gU = {}
    for l in range(0, L - 1):
        (Wc, _), (Wd, _) = dec[l]
        b, u = c["b"][l], c["u"][l]
        dWd, dbd = conv3_weight_grad(b, g), g.reshape(-1, g.shape[-1]).sum(axis=0)
        g2 = R(mask(b, conv3_input_grad(g, R(Wd))))
        dWc, dbc = conv3_weight_grad(u, g2), g2.reshape(-1, g2.shape[-1]).sum(axis=0)
        gU[l] = conv3_input_grad(g2, R(Wc))
        gd[l] = ((dWc, dbc), (dWd, dbd))
        act = c["e"][L - 1] if l == L - 2 else c["d"][l + 1]
        C1 = act.shape[-1]
        g = R(mask(act, up_adjoint(gU[l][..., :C1])))
    ge = {}
    gin = None
    for l in range(L - 1, -1, -1):
        (Wa, _), (Wb, _) = enc[l]
        if l < L - 1:
            C1 = spec.channels(l + 1)
            g = R(mask(c["e"][l], gU[l][..., C1:] + pool_adjoint(gin)))
        a, inp = c["a"][l], c["inp"][l]
        dWb, dbb = conv3_weight_grad(a, g), g.reshape(-1, g.shape[-1]).sum(axis=0)
        g2 = R(mask(a, conv3_input_grad(g, R(Wb))))
        dWa, dba = conv3_weight_grad(inp, g2), g2.reshape(-1, g2.shape[-1]).sum(axis=0)
        gin = conv3_input_grad(g2, R(Wa)) if l > 0 else None
        ge[l] = ((dWa, dba), (dWb, dbb))
    grads = []
    for l in range(L):
        (dWa, dba), (dWb, dbb) = ge[l]
        grads += [dWa, dba, dWb, dbb]
    for l in range(L - 2, -1, -1):
        (dWc, dbc), (dWd, dbd) = gd[l]
        grads += [dWc, dbc, dWd, dbd]
    grads += [dWh, dbh]
    return loss, grads
