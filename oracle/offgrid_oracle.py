"""Off-grid measurements for the oracle (TEST INFRASTRUCTURE only: ``tests/``
may import it; the CUDA library never does).

The paper imposes known values u(x_i, t_i) = u_i at measurement points
(Section 3.2, the Burgers reconstruction; the data term 1/N sum_i
(u(x_i, t_i) - u_i)^2 of its loss) without saying how the discrete field is
evaluated between grid points.  Reading: the cell-centred field is
interpolated d-linearly (the tensor product of 1-D linear interpolation
between the two nearest cell centres along every axis); a point between a
wall and the outermost centre takes that centre's value along that axis
(clamped, no extrapolation); an axis of one cell is constant.  The data term
of M points is w_data / M * sum_m (sum_k w_mk u[c_mk] - v_m)^2; its gradient
scatters 2 w_data / M * (sample_m - v_m) * w_mk to the corner cells c_mk.
"""
from __future__ import annotations

import itertools

import numpy as np


def sample_weights(points, shape, lengths, origin=None):
    """Corner cells and weights of d-linear interpolation at physical points.

    points:  [M, d] coordinates, axes in the order of `shape` (slowest first).
    shape:   cells per axis.  lengths: domain length per axis.  origin: lower
             corner per axis (default 0).
    Returns (idx [M, 2^d] flat cell indices, w [M, 2^d] weights).
    """
    pts = np.atleast_2d(np.asarray(points, dtype=np.float64))
    d = len(shape)
    origin = np.zeros(d) if origin is None else np.asarray(origin, dtype=np.float64)
    lo, frac = [], []
    for a in range(d):
        n = shape[a]
        h = lengths[a] / n
        s = (pts[:, a] - origin[a]) / h - 0.5  # position in units of cell centres
        s = np.clip(s, 0.0, n - 1.0)
        if n == 1:
            i0 = np.zeros(len(pts), dtype=np.int64)
            t = np.zeros(len(pts))
        else:
            i0 = np.minimum(np.floor(s).astype(np.int64), n - 2)
            t = s - i0
        lo.append(i0)
        frac.append(t)
    strides = np.cumprod((list(shape[1:]) + [1])[::-1])[::-1]
    idx = np.zeros((len(pts), 2 ** d), dtype=np.int64)
    w = np.ones((len(pts), 2 ** d))
    for k, corner in enumerate(itertools.product((0, 1), repeat=d)):
        for a, c in enumerate(corner):
            i = np.minimum(lo[a] + c, shape[a] - 1)
            idx[:, k] += i * strides[a]
            w[:, k] *= frac[a] if c else (1.0 - frac[a])
    return idx, w


def sample(u, idx, w):
    """Values of the field u at the points (sum_k w_mk u[idx_mk])."""
    return np.sum(w * u.reshape(-1)[idx], axis=1)


def data_term(u, idx, w, values, w_data=1.0):
    """Off-grid data term and its gradient with respect to u."""
    m = len(values)
    if m == 0:
        return 0.0, np.zeros_like(u)
    diff = sample(u, idx, w) - np.asarray(values, dtype=np.float64)
    c = w_data / m
    g = np.zeros(u.size)
    np.add.at(g, idx.ravel(), (2.0 * c * diff[:, None] * w).ravel())
    return float(c * np.sum(diff * diff)), g.reshape(u.shape)
