"""Learned warm start of the body-shape problem (3-D penalised Navier-Stokes).

Pipeline, all on the GPU through this library:
  1. forward solves: for seeded random ellipsoids, plain mODIL on the body
     problem with the body-fraction field pinned to the ellipsoid by dense
     data (velocity and pressure free, uniform inflow as the initial guess);
     many instances batched in one problem;
  2. training pairs: U-Net input = the wake slab's u, v, w samples of the
     forward solution plus a mask (zero elsewhere), target = the solution's
     five fields, normalised per channel;
  3. warm start: the trained network's prediction from the slab samples of a
     new case, written into one level of the inverse problem's multigrid
     decomposition (the other levels zero); zero-initialised mODIL (uniform
     inflow, chihat = 0) stays the fallback.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs, modil

FIELDS = 5  # u, v, w, p, chihat


def chihat_from_fraction(chi, clip=1e-3):
    """chihat with 1 / (1 + exp(-(chihat - 5))) = chi, chi clipped to [clip, 1 - clip]."""
    c = np.clip(chi, clip, 1.0 - clip)
    return np.log(c / (1.0 - c)) + 5.0


def fraction_from_chihat(ch):
    """Body fraction chi = 1 / (1 + exp(-(chihat - 5)))."""
    return 1.0 / (1.0 + np.exp(-(np.asarray(ch, np.float64) - 5.0)))


def zero_levels(shape, n_levels, inflow_level=0):
    """Uniform inflow u = 1 on one level, every other value zero (chihat = 0)."""
    lv = [[np.zeros(s, np.float32) for s in inputs.level_shapes(shape, n_levels)] for _ in range(FIELDS)]
    lv[0][inflow_level][:] = 1.0
    return lv


def forward_solves(cases, side, n_levels, steps, lr=1e-3, w_pin=10.0, batch=32, fractions=None,
                   lbfgs_iters=0, history=50, schedule=None):
    """Plain mODIL forward solutions of the body problem around each case's
    ellipsoid (cases: list of (centre, axes); fractions: their body fractions
    on the grid if already computed): `steps` Adam steps on batches of cases
    (or, with schedule = [(steps, lr), ...], Adam by learning-rate phases,
    each phase a new problem from the levels the last one reached), then,
    with lbfgs_iters > 0, that many L-BFGS iterations per case (the optimiser
    of Section 3.5).  Returns [n, 5, S, S, S] FP32 composed fields and the
    final loss terms."""
    import torch  # noqa: F401  (device memory and streams)
    shape = (side,) * 3
    ncell = side ** 3
    cf = inputs.NS3D_COEF
    out = np.zeros((len(cases), FIELDS) + shape, np.float32)
    terms = np.zeros((len(cases), 4))
    cells = np.arange(ncell, dtype=np.int32)
    field4 = np.full(ncell, 4, np.int32)
    if lbfgs_iters:
        batch = 1  # L-BFGS runs on single-instance problems
    for b0 in range(0, len(cases), batch):
        chunk = cases[b0:b0 + batch]
        chats = [chihat_from_fraction(fractions[b0 + k] if fractions is not None
                                      else inputs.ns3d_body_fraction(shape, c, a))
                 for k, (c, a) in enumerate(chunk)]
        def make(rate):
            return [modil.Desc("ns3d", shape, n_levels, "f32", coef=(cf["Re"], cf["D"], cf["lam"], cf["tau"]),
                               w_res=1.0, w_data=w_pin * ncell, meas_cell=cells, meas_field=field4,
                               meas_value=ch.reshape(-1), lr=rate) for ch in chats]
        starts = []
        for ch in chats:
            lv = zero_levels(shape, n_levels)
            lv[4][0][:] = ch
            starts.append(lv)
        phases = list(schedule) if schedule else []
        for steps_k, rate in phases[:-1]:  # all but the last phase
            with modil.Problem(make(rate)) as p:
                for i, lv in enumerate(starts):
                    p.write_fields(lv, instance=i)
                p.step(steps_k, read_loss=False)
                starts = [[p.read_levels(field=f, instance=i) for f in range(FIELDS)] for i in range(len(chats))]
        last_steps, last_rate = phases[-1] if phases else (steps, lr)
        with modil.Problem(make(last_rate)) as p:
            for i, lv in enumerate(starts):
                p.write_fields(lv, instance=i)
            if last_steps:
                p.step(last_steps, read_loss=False)
            if lbfgs_iters:
                with modil.LBFGS(p, history=history) as opt:
                    opt.run(lbfgs_iters)
            t = p.eval_loss()
            for i in range(len(chunk)):
                out[b0 + i] = np.stack([p.read_field(f, instance=i) for f in range(FIELDS)])
                terms[b0 + i] = t[i]
    return out, terms


def slab(shape, seed, centre, axes, fields):
    """Slab cells and field indices of a case, with values sampled from the
    given composed fields [5, *shape]."""
    cells, fidx, _ = inputs.ns3d_slab(shape, seed, centre, axes)
    vals = np.array([fields[f].reshape(-1)[c] for c, f in zip(cells, fidx)])
    return cells, fidx, vals


def unet_input(shape, cells, fidx, vals, side):
    """Input of the network on a side^3 grid: channels (u - 1, v, w) at the
    slab cells mapped to the network grid (several samples of one network
    cell averaged), and the mask of the cells that carry samples."""
    r = shape[0] // side
    ny, nx = shape[1], shape[2]
    z, y, xx = cells // (ny * nx), (cells // nx) % ny, cells % nx
    idx = ((z // r) * side + (y // r)) * side + (xx // r)
    sums = np.zeros((side ** 3, 3))
    cnt = np.zeros((side ** 3, 3))
    np.add.at(sums, (idx, fidx), vals - np.where(fidx == 0, 1.0, 0.0))
    np.add.at(cnt, (idx, fidx), 1.0)
    x = np.zeros((side ** 3, 4), np.float32)
    x[:, :3] = np.where(cnt > 0, sums / np.maximum(cnt, 1.0), 0.0)
    x[:, 3] = (cnt.sum(axis=1) > 0).astype(np.float32)
    return x.reshape(side, side, side, 4)


class Normaliser:
    """Per-channel affine normalisation of the targets."""

    def __init__(self, targets):
        axes = (0,) + tuple(range(2, targets.ndim))
        self.mean = targets.mean(axis=axes)
        self.std = targets.std(axis=axes) + 1e-6

    def to_net(self, t):          # [n, 5, S, S, S] -> [n, S, S, S, 5]
        z = (t - self.mean[:, None, None, None]) / self.std[:, None, None, None]
        return np.moveaxis(z, 1, -1).astype(np.float32)

    def from_net(self, y):        # [..., S, S, S, 5] -> [..., 5, S, S, S]
        return np.moveaxis(y, -1, -4) * self.std[:, None, None, None] + self.mean[:, None, None, None]


def param_shapes(levels, base, in_pad=8, out_ch=5):
    """Parameter shapes of the network in the library's order."""
    out = []

    def add(cin, cout, taps=27):
        out.append((cout, taps, cin))
        out.append((cout,))
    for l in range(levels):
        add(in_pad if l == 0 else base << (l - 1), base << l)
        add(base << l, base << l)
    for l in range(levels - 2, -1, -1):
        add((base << (l + 1)) + (base << l), base << l)
        add(base << l, base << l)
    add(base, out_ch, taps=1)
    return out


def train(xs, ys, epochs, batch=2, lr=1e-3, base_ch=32, levels=4, seed=0):
    """Train the U-Net on inputs xs [n, S, S, S, 4] and normalised targets
    ys [n, S, S, S, 5] (host FP32); returns (network, mean loss per epoch,
    seconds)."""
    import torch

    from . import unet
    n, side = xs.shape[0], xs.shape[1]
    net = unet.UNet(side, batch=batch, in_ch=4, out_ch=5, base_ch=base_ch, levels=levels, lr=lr)
    net.write_params(inputs.unet_params(param_shapes(levels, base_ch), seed))
    X = torch.from_numpy(np.ascontiguousarray(xs)).cuda()
    Y = torch.from_numpy(np.ascontiguousarray(ys)).cuda()
    rng = inputs.make_rng(seed + 1)
    hist = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(epochs):
        perm = rng.permutation(n)
        tot, k = 0.0, 0
        for b in range(0, n - batch + 1, batch):
            idx = torch.from_numpy(perm[b:b + batch]).cuda()
            tot += net.train_step(X[idx].contiguous(), Y[idx].contiguous())
            k += 1
        hist.append(tot / max(k, 1))
    torch.cuda.synchronize()
    return net, hist, time.perf_counter() - t0


def predict(net, norm, x):
    """Network prediction of the five fields [5, S, S, S] for one input [S, S, S, 4]
    (the network's batch must be 1)."""
    import torch
    y = net.forward(torch.from_numpy(np.ascontiguousarray(x[None])).cuda())
    return norm.from_net(y.cpu().numpy()[0])


def warm_levels(shape, n_levels, level, fields):
    """Multigrid levels with the predicted fields on `level` and zeros elsewhere."""
    lv = [[np.zeros(s, np.float32) for s in inputs.level_shapes(shape, n_levels)] for _ in range(FIELDS)]
    for f in range(FIELDS):
        lv[f][level][:] = fields[f]
    return lv


def inverse_problem(shape, n_levels, cells, fidx, vals, lr=1e-3):
    cf = inputs.NS3D_COEF
    return modil.Desc("ns3d", shape, n_levels, "f32", coef=(cf["Re"], cf["D"], cf["lam"], cf["tau"]),
                      w_res=1.0, w_data=1.0, meas_cell=cells, meas_field=fidx, meas_value=vals, lr=lr)


def steps_to_losses(desc, levels, thresholds, max_steps, chunk=100, chi_ref=None, run_all=False,
                    optimizer="adam", history=50, schedule=None):
    """Run mODIL from the given levels with Adam or L-BFGS (Section 3.5 uses
    L-BFGS); for every threshold the first step (iteration) count, a
    multiple of chunk, and the wall time at which the loss is at or below it
    (None if never).  schedule: Adam's learning rate by phases, [(steps, lr),
    ...] (each phase a new problem from the levels the last one reached, its
    moments restarted; the switch counts in the wall time; max_steps is then
    the schedule's total).  Returns (hits, loss history per chunk), and with
    chi_ref also the mean absolute body-fraction error per chunk (the
    composed chihat read back outside the timed steps).  Stops once every
    threshold is reached unless run_all, and when L-BFGS stops early."""
    import torch
    hits = {t: None for t in thresholds}
    hist, chi_err = [], []
    phases = [(max_steps, None)] if schedule is None else list(schedule)
    el = 0.0
    done = 0
    stalled = False
    for steps, lr in phases:
        if stalled or (not run_all and hits and all(v is not None for v in hits.values())):
            break
        t0 = time.perf_counter()
        d = desc if lr is None else modil.Desc(**{**desc.kwargs, "lr": lr})
        p = modil.Problem(d)
        p.write_fields(levels)
        opt = modil.LBFGS(p, history=history) if optimizer == "lbfgs" else None
        torch.cuda.synchronize()
        el += time.perf_counter() - t0
        end = done + steps
        while done < end and not stalled:
            t0 = time.perf_counter()
            if opt is None:
                loss = float(p.step(chunk)[0][0])
                done += chunk
            else:
                h = opt.run(chunk)
                loss = float(h[-1])
                done += len(h) - 1
                stalled = len(h) - 1 < chunk
            el += time.perf_counter() - t0
            hist.append(loss)
            if chi_ref is not None:
                chi_err.append(float(np.mean(np.abs(fraction_from_chihat(p.read_field(4)) - chi_ref))))
            for t in thresholds:
                if hits[t] is None and loss <= t:
                    hits[t] = (done, el)
            if not run_all and hits and all(v is not None for v in hits.values()):
                break
        if opt is not None:
            opt.close()
        t0 = time.perf_counter()
        levels = [p.read_levels(field=f) for f in range(desc.n_fields)]
        p.close()
        el += time.perf_counter() - t0
    if chi_ref is not None:
        return hits, hist, chi_err
    return hits, hist
