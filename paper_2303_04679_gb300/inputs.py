"""Seeded synthetic inputs shared by the CUDA path's callers and the CPU oracle.

This module draws random numbers and evaluates closed-form data profiles
(initial conditions, analytic fields used as synthetic measurements).  It holds
none of the method's arithmetic: no prolongation, no residual stencil, no loss,
no gradient and no optimiser step.  Everything is a deterministic function of an
integer seed (numpy PCG64 through ``np.random.default_rng``).

Workload recipes follow the paper's problems (Section 3.2 Burgers
reconstruction, Section 3.3 lid-driven cavity, Section 3.4 conductivity
inference, Section 3.5 body shape) at the sizes of the configurations this
library is measured on.
"""
from __future__ import annotations

import math

import numpy as np


def make_rng(seed: int) -> np.random.Generator:
    """PCG64 generator for an integer seed."""
    return np.random.default_rng(int(seed))


def level_shapes(shape, n_levels):
    """Cells per axis on each level: N_i = N / 2^(i-1) (Section 2.2)."""
    out = []
    for i in range(n_levels):
        s = tuple(int(n) >> i for n in shape)
        if min(s) < 1 or any((int(n) >> i) << i != int(n) for n in shape):
            raise ValueError(f"shape {shape} cannot be halved {n_levels - 1} times")
        out.append(s)
    return out


def random_levels(shape, n_levels, n_fields, seed, fine_lo=-1.0, fine_hi=1.0,
                  coarse_scale=0.5, dtype=np.float64):
    """Random level values: list over fields of list over levels of arrays.

    The fine level is uniform in [fine_lo, fine_hi]; coarser levels are
    N(0, coarse_scale^2).  Values are rounded to ``dtype`` so that the FP32
    device path and the FP64 oracle start from identical numbers.
    """
    rng = make_rng(seed)
    shapes = level_shapes(shape, n_levels)
    out = []
    for _ in range(n_fields):
        lv = []
        for i, s in enumerate(shapes):
            if i == 0:
                a = rng.uniform(fine_lo, fine_hi, size=s)
            else:
                a = rng.normal(0.0, coarse_scale, size=s)
            lv.append(a.astype(dtype).astype(np.float64))
        out.append(lv)
    return out


def measurement_cells(n_cells, n_meas, seed):
    """Distinct random flat cell indices (sampling without replacement)."""
    rng = make_rng(seed)
    return np.sort(rng.choice(int(n_cells), size=int(n_meas), replace=False)).astype(np.int32)


# --------------------------------------------------------------------------
# Viscous Burgers (space-time, x in [-1, 1], t in [0, 1])
# --------------------------------------------------------------------------

BURGERS_X = (-1.0, 1.0)
BURGERS_T = (0.0, 1.0)


def burgers_ic_amplitudes(seed, n_modes=4, sigma=0.5):
    """Amplitudes a_k ~ N(0, sigma^2) of the initial condition."""
    return make_rng(seed).normal(0.0, sigma, size=n_modes)


def burgers_ic(x, amps):
    """u(x, 0) = sum_k a_k sin(k pi (x + 1) / 2); zero at x = -1 and x = 1."""
    x = np.asarray(x, dtype=np.float64)
    u = np.zeros_like(x)
    for k, a in enumerate(amps, start=1):
        u += a * np.sin(k * math.pi * (x + 1.0) / 2.0)
    return u


def burgers_batch_instance(i, base_seed=0):
    """Per-instance draw for the batched Burgers workload (512 instances).

    Returns (nx, nt, nu, seed): N_x, N_t uniform in {64, 128, 256, 512},
    nu log-uniform in [1e-3, 1e-1].
    """
    rng = make_rng(1_000_003 * (base_seed + 1) + i)
    sizes = np.array([64, 128, 256, 512])
    nx = int(rng.choice(sizes))
    nt = int(rng.choice(sizes))
    nu = float(10.0 ** rng.uniform(-3.0, -1.0))
    return nx, nt, nu, int(rng.integers(0, 2**31 - 1))


def burgers_smooth_field(nt, nx, amps, nu):
    """Closed-form smooth space-time field used as synthetic Burgers data.

    Each sine mode decays with its heat-equation rate, u = sum_k a_k
    exp(-nu (k pi / 2)^2 t) sin(k pi (x+1)/2), sampled at cell centres.  It
    is smooth, vanishes at the walls and starts at the Burgers initial
    condition; it is a data profile, not a solution of the discrete problem.
    """
    dx = 2.0 / nx
    dt = 1.0 / nt
    x = -1.0 + (np.arange(nx) + 0.5) * dx
    t = (np.arange(nt) + 0.5) * dt
    u = np.zeros((nt, nx))
    for k, a in enumerate(amps, start=1):
        lam = nu * (k * math.pi / 2.0) ** 2
        u += a * np.exp(-lam * t)[:, None] * np.sin(k * math.pi * (x + 1.0) / 2.0)[None, :]
    return u


# --------------------------------------------------------------------------
# Heat conduction with unknown conductivity (x, t in [0, 1])
# --------------------------------------------------------------------------

HEAT_KNODES = 32


def heat_g(x):
    """g(x) = exp(-50 (x - 1/2)^2) (Section 3.4)."""
    return np.exp(-50.0 * (np.asarray(x, dtype=np.float64) - 0.5) ** 2)


def heat_ic(nx):
    """Initial temperature u(x, 0) = g(x) - g(0) at the nx cell centres."""
    x = (np.arange(nx) + 0.5) / nx
    return heat_g(x) - heat_g(0.0)


def heat_k_true(u):
    """Reference conductivity k(u) = 0.02 exp(-20 (u - 1/2)^2) (Section 3.4)."""
    u = np.asarray(u, dtype=np.float64)
    return 0.02 * np.exp(-20.0 * (u - 0.5) ** 2)


def heat_linear_series(nt, nx, k0=0.02, n_modes=64):
    """Closed-form solution of u_t = k0 u_xx, u(0)=u(1)=0, u(x,0)=g(x)-g(0).

    Sine series with coefficients from a 4096-point midpoint quadrature, sampled
    at cell centres x_i = (i+1/2)/nx and rows t_n = (n+1/2)/nt.  Used as a
    smooth synthetic temperature record of the right shape and magnitude.
    """
    xq = (np.arange(4096) + 0.5) / 4096
    f = heat_g(xq) - heat_g(0.0)
    x = (np.arange(nx) + 0.5) / nx
    t = (np.arange(nt) + 0.5) / nt
    u = np.zeros((nt, nx))
    for n in range(1, n_modes + 1):
        b = 2.0 * np.mean(f * np.sin(n * math.pi * xq))
        u += b * np.exp(-k0 * (n * math.pi) ** 2 * t)[:, None] * np.sin(n * math.pi * x)[None, :]
    return u


def heat_measurements(nt, nx, frac=0.05, sigma=1e-3, seed=2, field=None):
    """5 % of cells with Gaussian noise of standard deviation sigma.

    ``field`` is the (nt, nx) temperature record to sample; by default the
    closed-form constant-conductivity series.  Returns (cells, values).
    """
    if field is None:
        field = heat_linear_series(nt, nx)
    n = nt * nx
    m = int(round(frac * n))
    cells = measurement_cells(n, m, seed)
    noise = make_rng(seed + 7919).normal(0.0, sigma, size=m)
    return cells, field.reshape(-1)[cells] + noise


def heat_k_init(value=0.02, n=HEAT_KNODES):
    """Initial conductivity nodes q_j (uniform value)."""
    return np.full(n, value, dtype=np.float64)


def heat_workload(nt=512, nx=512, n_levels=7, seed=2, field=None, frac=0.05, sigma=1e-3):
    """Conductivity inference on a 512 (x) by 512 (t) grid with 7 levels.

    A fraction ``frac`` of the cells (5 %) carry measurements with Gaussian
    noise (``sigma`` = 1e-3) of the temperature record ``field`` (nt x nx):
    a solution of the forward
    problem with the reference conductivity (records.heat_record), or by
    default the closed-form constant-conductivity series; the initial
    profile is g(x) - g(0); 32 conductivity nodes start at 0.02.
    """
    cells, vals = heat_measurements(nt, nx, frac, sigma, seed, field=field)
    return dict(shape=(nt, nx), n_levels=n_levels, meas_cell=cells, meas_value=vals,
                aux=heat_ic(nx), knodes=heat_k_init(), w_res=1.0, w_data=1.0, w_reg=1e-4,
                lr=1e-3, k_scale=0.02)


def burgers_workload(nt=64, nx=64, n_levels=4, seed=0, n_meas=200, nu=0.01):
    """Burgers reconstruction on 64 x 64 with 4 levels and 200 measurement cells.

    Returns the cells and the amplitudes of the initial condition; the
    measured values come from a reference solve done by the caller.
    """
    cells = measurement_cells(nt * nx, n_meas, seed)
    return dict(shape=(nt, nx), n_levels=n_levels, meas_cell=cells, nu=nu,
                amps=burgers_ic_amplitudes(seed), w_res=1.0, w_data=1.0, lr=5e-3)


# The paper's own Burgers reconstruction (Section 3.2): inviscid, (x, t) in
# [0, 1]^2 on 64 x 64 cells, six levels, the reference solution imposed at 84
# points on the edges of a rectangle.  The rectangle is not given in the
# paper; the reading here is the square [1/4, 3/4]^2 (21 points per edge,
# each corner counted once).
BURGERS_PAPER = dict(shape=(64, 64), n_levels=6, nu=0.0, domain=((0.0, 1.0), (0.0, 1.0)),
                     rect=((0.25, 0.75), (0.25, 0.75)), per_edge=21)


def burgers_paper_ic(x):
    """Initial condition u(x, 0) = (1 - cos 6 pi x) / 2 of Section 3.2."""
    return 0.5 * (1.0 - np.cos(6.0 * math.pi * np.asarray(x, dtype=np.float64)))


def rectangle_points(rect=BURGERS_PAPER["rect"], per_edge=BURGERS_PAPER["per_edge"]):
    """(t, x) points on the edges of the rectangle rect = ((t0, t1), (x0, x1)):
    per_edge equally spaced points on each edge, walked counter-clockwise from
    (t0, x0) so that every corner appears once (4 x per_edge points)."""
    (t0, t1), (x0, x1) = rect
    s = np.arange(per_edge) / per_edge
    edges = [np.stack([np.full(per_edge, t0), x0 + (x1 - x0) * s], axis=1),       # t = t0
             np.stack([t0 + (t1 - t0) * s, np.full(per_edge, x1)], axis=1),       # x = x1
             np.stack([np.full(per_edge, t1), x1 - (x1 - x0) * s], axis=1),       # t = t1
             np.stack([t1 - (t1 - t0) * s, np.full(per_edge, x0)], axis=1)]       # x = x0
    return np.concatenate(edges, axis=0)


def burgers_batch(n=512, base_seed=0, meas_frac=0.005):
    """The batched Burgers workload: n instances of uneven size.

    Per instance (seeded by its index): N_x, N_t in {64, 128, 256, 512}, nu
    log-uniform in [1e-3, 1e-1], 0.5 % of the cells measured (values of the
    closed-form decaying sine field of the instance's initial condition),
    L = log2(min(N_x, N_t) / 8) + 1 levels (coarsest grid at least 8 cells).
    Returns a list of dicts (shape = (N_t, N_x)).
    """
    out = []
    for i in range(n):
        nx, nt, nu, seed = burgers_batch_instance(i, base_seed)
        L = int(math.log2(min(nx, nt) // 8)) + 1
        m = max(1, int(round(meas_frac * nt * nx)))
        cells = measurement_cells(nt * nx, m, seed)
        amps = burgers_ic_amplitudes(seed)
        field = burgers_smooth_field(nt, nx, amps, nu)
        out.append(dict(shape=(nt, nx), n_levels=L, nu=nu, meas_cell=cells,
                        meas_value=field.reshape(-1)[cells], seed=seed))
    return out


# --------------------------------------------------------------------------
# Body shape in 3-D (Section 3.5): (z, y, x) cells of [0,1] x [0,1] x [0,2]
# --------------------------------------------------------------------------

NS3D_COEF = dict(Re=60.0, D=0.4, lam=1.0, tau=1.0)


def ns3d_ellipsoid(seed):
    """Seeded axis-aligned ellipsoid: centre (x, y, z) in [0.4, 0.6] x
    [0.35, 0.65]^2, semi-axes in [0.1, 0.25]."""
    rng = make_rng(seed)
    centre = np.array([rng.uniform(0.4, 0.6), rng.uniform(0.35, 0.65), rng.uniform(0.35, 0.65)])
    axes = rng.uniform(0.1, 0.25, size=3)
    return centre, axes


def ns3d_body_fraction(shape, centre, axes, sub=4):
    """Volume fraction of the ellipsoid in each cell from sub^3 point samples
    per cell (the reference body fraction chi_ref in [0, 1])."""
    nz, ny, nx = shape
    hz, hy, hx = 1.0 / nz, 1.0 / ny, 2.0 / nx
    off = (np.arange(sub) + 0.5) / sub
    z = ((np.arange(nz)[:, None] + off[None, :]) * hz).reshape(-1)
    y = ((np.arange(ny)[:, None] + off[None, :]) * hy).reshape(-1)
    x = ((np.arange(nx)[:, None] + off[None, :]) * hx).reshape(-1)
    cx, cy, cz = centre
    ax, ay, az = axes
    inside = (((z[:, None, None] - cz) / az) ** 2 + ((y[None, :, None] - cy) / ay) ** 2
              + ((x[None, None, :] - cx) / ax) ** 2) <= 1.0
    return inside.reshape(nz, sub, ny, sub, nx, sub).mean(axis=(1, 3, 5))


def ns3d_wake_velocity(z, y, x, centre, axes):
    """Closed-form synthetic wake behind the body: a Gaussian velocity
    deficit along x that widens downstream, small inward cross-flow."""
    cx, cy, cz = centre
    r0 = float(np.mean(axes[1:]))
    s = r0 * (1.0 + 0.5 * np.maximum(x - cx, 0.0))
    r2 = (y - cy) ** 2 + (z - cz) ** 2
    deficit = 0.6 * (r0 / s) ** 2 * np.exp(-r2 / (s * s))
    u = 1.0 - deficit
    v = -0.1 * deficit * (y - cy) / s
    w = -0.1 * deficit * (z - cz) / s
    return u, v, w


def ns3d_slab(shape, seed, centre, axes):
    """Wake measurements on a 32 x 32 x 4 slab: y and z every (n/32)-th cell,
    4 consecutive x planes from a seeded x in [1.2, 1.6]; u, v and w each.
    Returns (cells, fields, values) with fields 0, 1, 2 = u, v, w."""
    nz, ny, nx = shape
    rng = make_rng(seed + 104729)
    x0 = int(rng.uniform(1.2, 1.6) / (2.0 / nx))
    x0 = min(x0, nx - 4)
    sz, sy = max(1, nz // 32), max(1, ny // 32)
    kz = np.arange(0, nz, sz)[:32]
    ky = np.arange(0, ny, sy)[:32]
    kx = np.arange(x0, x0 + 4)
    K, J, I = np.meshgrid(kz, ky, kx, indexing="ij")
    cell = ((K * ny + J) * nx + I).reshape(-1).astype(np.int32)
    zc = (K.reshape(-1) + 0.5) / nz
    yc = (J.reshape(-1) + 0.5) / ny
    xc = (I.reshape(-1) + 0.5) * (2.0 / nx)
    u, v, w = ns3d_wake_velocity(zc, yc, xc, centre, axes)
    cells = np.concatenate([cell, cell, cell])
    fields = np.repeat(np.arange(3, dtype=np.int32), len(cell))
    return cells, fields, np.concatenate([u, v, w])


def ns3d_workload(n=128, n_levels=8, seed=5):
    """Body-shape inference on n^3 cells, 8 levels (128 -> 1), Re = 60,
    D = 0.4, lambda = 1: a seeded ellipsoid and its 32 x 32 x 4 wake slab
    (3 x 4096 velocity samples)."""
    shape = (n, n, n)
    centre, axes = ns3d_ellipsoid(seed)
    cells, fields, vals = ns3d_slab(shape, seed, centre, axes)
    return dict(shape=shape, n_levels=n_levels, meas_cell=cells, meas_field=fields,
                meas_value=vals, centre=centre, axes=axes, coef=dict(NS3D_COEF),
                w_res=1.0, w_data=1.0, lr=1e-3)


# --------------------------------------------------------------------------
# Learned warm start (3-D U-Net): parameter initialisation
# --------------------------------------------------------------------------

def unet_params(shapes, seed, bias_scale=0.0):
    """He-normal weights (std sqrt(2 / fan_in)) for the parameter shapes
    (weights (c_out, taps, c_in), biases (c_out,)); biases N(0, bias_scale^2).
    Values are FP32."""
    rng = make_rng(seed)
    out = []
    for s in shapes:
        if len(s) == 3:
            std = math.sqrt(2.0 / (s[1] * s[2]))
            out.append(rng.normal(0.0, std, size=s).astype(np.float32))
        else:
            out.append((rng.normal(0.0, bias_scale, size=s) if bias_scale else np.zeros(s)).astype(np.float32))
    return out


# --------------------------------------------------------------------------
# Lid-driven cavity (Section 3.3)
# --------------------------------------------------------------------------

def cavity_velocity(n):
    """Closed-form recirculating flow on the unit square (cell centres):
    stream function psi = sin(pi x)^2 sin(pi y)^2, u = dpsi/dy, v = -dpsi/dx
    (divergence free, zero on the walls).  A synthetic data profile, not a
    solution of the discrete cavity problem."""
    c = (np.arange(n) + 0.5) / n
    y, x = np.meshgrid(c, c, indexing="ij")
    u = 2.0 * np.pi * np.sin(np.pi * x) ** 2 * np.sin(np.pi * y) * np.cos(np.pi * y)
    v = -2.0 * np.pi * np.sin(np.pi * y) ** 2 * np.sin(np.pi * x) * np.cos(np.pi * x)
    return u, v


def cavity_workload(n=256, n_levels=8, n_samples=1000, seed=3, Re=100.0, field=None):
    """Cavity at Re = 100 on n^2 cells with 8 levels: 1000 velocity samples
    (u or v at seeded distinct cells) of ``field`` = (u, v), a forward
    solution (records.cavity_record), or by default of the closed-form
    recirculating flow."""
    rng = make_rng(seed)
    cells = measurement_cells(n * n, n_samples, seed)
    fields = rng.integers(0, 2, size=n_samples).astype(np.int32)
    u, v = cavity_velocity(n) if field is None else field
    vals = np.where(fields == 0, u.reshape(-1)[cells], v.reshape(-1)[cells])
    return dict(shape=(n, n), n_levels=n_levels, meas_cell=cells, meas_field=fields,
                meas_value=vals, coef=(Re, 1.0), lr=1e-3)


# --------------------------------------------------------------------------
# Poisson equation (Section 3.1): the paper's reference solution on [0,1]^2
# --------------------------------------------------------------------------

def poisson_workload(n=32, d=2, layout="cell"):
    """The reference solution u_ref = g(prod_i 5 (1 - x_i) x_i) with
    g(v) = (v^5 / (1 + v^5))^(1/5) of Section 3.1 on [0,1]^d, at the cell
    centres (cell layout, n per axis) or the nodes (node layout, n + 1 per
    axis), and the right-hand side f = lap(u_ref) from the closed-form
    derivatives (g' = (1 + v^5)^(-6/5), g'' = -6 v^4 (1 + v^5)^(-11/5)).  The
    paper takes f from the discrete Laplacian so that u_ref solves the
    discrete problem exactly; the closed form used here leaves the
    discretisation error (second order in 1/n) between the discrete solution
    and u_ref."""
    c = np.arange(n + 1) / n if layout == "node" else (np.arange(n) + 0.5) / n
    X = np.meshgrid(*([c] * d), indexing="ij")
    ph = [5.0 * (1.0 - x) * x for x in X]
    dph = [5.0 - 10.0 * x for x in X]
    v = np.prod(ph, axis=0)
    g = v / (1.0 + v ** 5) ** 0.2
    g1 = (1.0 + v ** 5) ** -1.2
    g2 = -6.0 * v ** 4 * (1.0 + v ** 5) ** -2.2
    grad2 = np.zeros_like(v)
    lapv = np.zeros_like(v)
    for i in range(d):
        others = np.prod([ph[j] for j in range(d) if j != i], axis=0) if d > 1 else np.ones_like(v)
        grad2 += (dph[i] * others) ** 2
        lapv += -10.0 * others
    return dict(shape=(n,) * d, u_ref=g, f=g2 * grad2 + g1 * lapv, layout=layout)


def uniform_noise(values, amplitude=0.05, seed=0):
    """Measured values with additive noise drawn from U[0, amplitude] (the
    noisy variant of the Burgers reconstruction in Section 3.2 uses
    U[0, 0.05])."""
    rng = make_rng(seed)
    v = np.asarray(values, dtype=np.float64)
    return v + rng.uniform(0.0, amplitude, size=v.shape)
