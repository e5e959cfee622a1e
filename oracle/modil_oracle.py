"""mODIL oracle: a plain, slow, FP64 restatement of the method on the CPU.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
this module.  It shares no code with the CUDA library (no kernels, headers,
tables or helpers); the only module both sides use is the seeded input
generator ``paper_2303_04679_gb300.inputs``, which holds none of the method's
arithmetic.

What is computed, and where the paper defines it:

* Levels N_i = N / 2^(i-1) and the multigrid decomposition
  u = M_L(u_1..u_L) = u_1 + T_1 u_2 + ... + T_1...T_{L-1} u_L, evaluated by
  Horner's scheme (Section 2.2, the two displayed forms of M_L).
* T_i: linear interpolation between consecutive grids, node-based (N+1
  values per axis) and cell-based (N values per axis), whose 1-D matrices for
  N = 8, 4, 2 are printed in Section 2.2.  Here each 1-D matrix is built
  explicitly from its definition and applied along every axis (tensor product).
  The transposed operator is the transposed matrix.
* The ODIL loss: weighted sum of squared discrete residuals over the grid
  plus squared mismatches at measurement points plus regularisers
  (Section 2.1, the displayed loss for the wave equation, and the loss
  formulas of Sections 3.1, 3.2, 3.4).
* Its gradient by a hand-written reverse pass through the stencils and then
  through the Horner chain (gw_{i+1} = T_i^T gw_i); the paper obtains it by
  automatic differentiation (Section 2.1, end of Section 2.2).
* Adam (Kingma and Ba, the optimiser named in Section 2.1).
* Reference generators used only to make test data: an explicit finite-volume
  Burgers solver and an implicit heat solver (Sections 3.2 and 3.4).

Discretisation readings where the paper gives no formula are stated next to
each function.  Nothing here is tuned for speed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "interp_matrix", "prolong", "restrict", "compose", "compose_explicit",
    "chain_grad", "level_shapes", "Problem", "burgers_residual",
    "heat_conductivity", "heat_residual", "poisson_residual", "loss_terms",
    "loss_grad_fine", "loss_grad_levels", "adam_step", "OracleState",
    "oracle_step", "burgers_explicit_solve", "heat_implicit_solve",
    "eo_flux", "ns2d_residuals", "ns2d_fields_residual_jacobian_grad", "ns3d_residuals",
    "ns3d_chi", "ns3d_residual_jacobian_grad", "ns3d_fine_grad_colours", "burgers_implicit_solve",
]


# ---------------------------------------------------------------------------
# Grids and the multigrid decomposition (Section 2.2)
# ---------------------------------------------------------------------------

def level_shapes(shape, n_levels, layout="cell"):
    """Cells per axis of each level: N_i = N / 2^(i-1), i = 1..L.

    For the node layout the arrays hold N_i + 1 values per axis.
    """
    shapes = []
    for i in range(n_levels):
        cells = []
        for n in shape:
            if n % (1 << i):
                raise ValueError("grid cannot be halved that many times")
            cells.append(n // (1 << i))
        if layout == "node":
            shapes.append(tuple(c + 1 for c in cells))
        else:
            shapes.append(tuple(cells))
    return shapes


def interp_matrix(n_coarse, layout="cell"):
    """1-D linear interpolation matrix T from a grid of n_coarse cells to 2*n_coarse.

    cell: values at cell centres.  A fine centre lies a quarter of a coarse
    cell from its parent centre, so it takes 3/4 of the parent and 1/4 of the
    nearer neighbour.  Beyond the first and last coarse centres the line
    through the two outermost centres is extended (linear extrapolation),
    which gives the printed boundary rows (5/4, -1/4).  A coarse grid of one
    cell has no line to extend; both fine cells copy it (constant).
    node: values at nodes; fine nodes on coarse nodes copy them and fine nodes
    between two coarse nodes take their mean.
    """
    if layout == "node":
        nc, nf = n_coarse + 1, 2 * n_coarse + 1
        T = np.zeros((nf, nc))
        for i in range(nf):
            if i % 2 == 0:
                T[i, i // 2] = 1.0
            else:
                T[i, i // 2] = 0.5
                T[i, i // 2 + 1] = 0.5
        return T
    nc, nf = n_coarse, 2 * n_coarse
    T = np.zeros((nf, nc))
    xc = np.arange(nc) + 0.5            # coarse centres in coarse-cell units
    for i in range(nf):
        x = (i + 0.5) / 2.0             # fine centre in coarse-cell units
        if nc == 1:
            T[i, 0] = 1.0
            continue
        # the two coarse centres bracketing x, clamped to the end pairs
        j = int(math.floor(x - 0.5))
        j = min(max(j, 0), nc - 2)
        t = (x - xc[j]) / (xc[j + 1] - xc[j])
        T[i, j] += 1.0 - t
        T[i, j + 1] += t
    return T


def _apply_axes(mats, a):
    """Apply one matrix along each axis of ``a`` (tensor-product operator)."""
    out = a
    for ax, M in enumerate(mats):
        out = np.moveaxis(np.tensordot(M, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


def _cells(shape, layout):
    return tuple(s - 1 for s in shape) if layout == "node" else tuple(shape)


def prolong(c, layout="cell"):
    """T_i c: interpolate a level to the next finer level (tensor product)."""
    cells = _cells(c.shape, layout)
    return _apply_axes([interp_matrix(n, layout) for n in cells], c)


def restrict(f, layout="cell"):
    """T_i^T f: the transposed interpolation applied to a fine-level array."""
    if layout == "node":
        cells = tuple((s - 1) // 2 for s in f.shape)
    else:
        cells = tuple(s // 2 for s in f.shape)
    return _apply_axes([interp_matrix(n, layout).T for n in cells], f)


def compose(levels, layout="cell"):
    """Horner form: w_L = u_L, w_i = u_i + T_i w_{i+1}, u = w_1."""
    w = np.array(levels[-1], dtype=np.float64)
    for u in reversed(levels[:-1]):
        w = np.asarray(u, dtype=np.float64) + prolong(w, layout)
    return w


def compose_explicit(levels, layout="cell"):
    """Explicit sum u_1 + T_1 u_2 + T_1 T_2 u_3 + ... (first displayed form of M_L)."""
    total = np.array(levels[0], dtype=np.float64)
    for i in range(1, len(levels)):
        term = np.array(levels[i], dtype=np.float64)
        for _ in range(i):
            term = prolong(term, layout)
        total = total + term
    return total


def chain_grad(g_fine, n_levels, layout="cell"):
    """Gradients of the loss with respect to every level from dL/du.

    Reverse of the Horner chain: dL/du_1 = g, dL/du_{i+1} = T_i^T dL/du_i.
    """
    grads = [np.array(g_fine, dtype=np.float64)]
    for _ in range(n_levels - 1):
        grads.append(restrict(grads[-1], layout))
    return grads


# ---------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------

@dataclass
class Problem:
    """One mODIL problem.

    pde:    "burgers" (space-time, axes (t, x)), "heat" (axes (t, x)) or
            "poisson" (d-dimensional, axes (..., y, x)).
    shape:  fine cells per axis, slowest axis first.
    coef:   burgers {"nu"}; heat {}; poisson {"f": right-hand side array}.
    meas_*: measurement cells (flat index into the fine field), field index
            and values; data term weight w_data / n_meas.
    aux:    heat initial temperature profile (one value per x cell).
    """
    pde: str
    shape: tuple
    n_levels: int
    layout: str = "cell"
    coef: dict = field(default_factory=dict)
    w_res: float = 1.0
    w_data: float = 1.0
    w_reg: float = 0.0
    meas_cell: np.ndarray = None
    meas_field: np.ndarray = None
    meas_value: np.ndarray = None
    aux: np.ndarray = None
    # off-grid measurements (single-field 2-D problems): physical (y, x) points
    # and values, sampled d-linearly (oracle/offgrid_oracle.py)
    meas_points: np.ndarray = None
    point_value: np.ndarray = None
    # physical extent ((lo, hi) per axis, same order as shape) of a 2-D
    # Burgers, heat or Poisson problem; None: the family's own domain
    domain_bounds: tuple = None
    # field sampled at each off-grid point (multi-field problems; None: 0)
    point_field: np.ndarray = None
    # heat: the conductivity is known (the forward problem that makes the
    # reference record of Section 3.4): q is a fixed input, dL/dq is zero and
    # the optimiser moves only the levels
    k_fixed: bool = False
    # heat: the unit of the optimiser's steps on the nodes (Adam's node step
    # is lr * k_scale; a diagonal preconditioner, not part of the loss)
    k_scale: float = 1.0

    @property
    def n_fields(self):
        return {"ns2d": 3, "ns3d": 5}.get(self.pde, 1)

    def domain(self):
        """Lower corner and length per axis (same order as shape)."""
        if self.domain_bounds is not None:
            return (tuple(float(lo) for lo, _ in self.domain_bounds),
                    tuple(float(hi) - float(lo) for lo, hi in self.domain_bounds))
        if self.pde == "burgers":       # t in [0,1], x in [-1,1]
            return (0.0, -1.0), (1.0, 2.0)
        if self.pde in ("heat", "poisson", "ns2d"):
            return tuple(0.0 for _ in self.shape), tuple(1.0 for _ in self.shape)
        if self.pde == "ns3d":              # [0,1] (z) x [0,1] (y) x [0,2] (x)
            return (0.0, 0.0, 0.0), (1.0, 1.0, 2.0)
        raise ValueError(self.pde)

    def spacing(self):
        """Grid spacings per axis (same order as shape)."""
        if self.domain_bounds is not None:
            return tuple(float(hi - lo) / n for (lo, hi), n in zip(self.domain_bounds, self.shape))
        if self.pde == "burgers":       # t in [0,1], x in [-1,1]
            return (1.0 / self.shape[0], 2.0 / self.shape[1])
        if self.pde == "heat":          # t in [0,1], x in [0,1]
            return (1.0 / self.shape[0], 1.0 / self.shape[1])
        if self.pde in ("poisson", "ns2d"):  # unit square / cube
            return tuple(1.0 / n for n in self.shape)
        if self.pde == "ns3d":              # [0,1] (z) x [0,1] (y) x [0,2] (x)
            return (1.0 / self.shape[0], 1.0 / self.shape[1], 2.0 / self.shape[2])
        raise ValueError(self.pde)


# ---------------------------------------------------------------------------
# Viscous Burgers, space-time finite volumes (Section 3.2)
# ---------------------------------------------------------------------------
# Reading.  Rows are time levels t_n = (n + 1/2) dt, columns are x cells.  The
# residual of row n >= 1 is the implicit (backward Euler) finite-volume step
#   r^n_i = (u^n_i - u^{n-1}_i)/dt + (F_{i+1/2} - F_{i-1/2})/dx
#           - nu (u^n_{i+1} - 2 u^n_i + u^n_{i-1})/dx^2,
# all spatial terms at row n.  Row 0 has no residual (only data constrain it).
# F is a first-order upwind flux for f(u) = u^2/2: the Engquist-Osher flux
# F(a, b) = max(a, 0)^2/2 + min(b, 0)^2/2, evaluated at interior faces from
# the two adjacent cells.  The walls carry zero Dirichlet data (Section 3.2):
# the upwind flux through a wall is the same flux between the wall value 0
# and the adjacent cell, F(0, u_0) = min(u_0, 0)^2/2 on the left and
# F(u_{N-1}, 0) = max(u_{N-1}, 0)^2/2 on the right, so a state flowing out of
# the domain leaves it and nothing enters from a wall; the viscous term uses
# the odd ghost u_{-1} = -u_0, u_{N} = -u_{N-1} (linear profile through zero
# at the wall).

def eo_flux(a, b):
    """Engquist-Osher flux for f(u) = u^2/2 and its two partial derivatives."""
    ap = np.maximum(a, 0.0)
    bm = np.minimum(b, 0.0)
    return 0.5 * ap * ap + 0.5 * bm * bm, ap, bm


def _ghost_odd(u):
    """Pad the last axis with odd ghosts (zero value at the wall)."""
    return np.concatenate([-u[..., :1], u, -u[..., -1:]], axis=-1)


def burgers_residual(u, nu, dt, dx):
    """Residuals r^n_i for rows n = 1..N_t-1, shape (N_t - 1, N_x)."""
    un, uo = u[1:], u[:-1]
    nx = u.shape[1]
    F = np.zeros((un.shape[0], nx + 1))
    F[:, 1:nx], _, _ = eo_flux(un[:, :-1], un[:, 1:])
    F[:, 0], _, _ = eo_flux(0.0 * un[:, 0], un[:, 0])      # left wall: value 0
    F[:, nx], _, _ = eo_flux(un[:, -1], 0.0 * un[:, -1])   # right wall
    ug = _ghost_odd(un)
    lap = (ug[:, 2:] - 2.0 * un + ug[:, :-2]) / dx**2
    return (un - uo) / dt + (F[:, 1:] - F[:, :-1]) / dx - nu * lap


def _burgers_adjoint(u, lam, nu, dt, dx):
    """dL/du given lam = dL/dr for the residual rows 1..N_t-1."""
    g = np.zeros_like(u)
    un = u[1:]
    nx = u.shape[1]
    # time difference
    g[1:] += lam / dt
    g[:-1] -= lam / dt
    # flux difference: face f (1..nx-1) is east of cell f-1 and west of cell f
    lamF = (lam[:, :-1] - lam[:, 1:]) / dx
    _, dFa, dFb = eo_flux(un[:, :-1], un[:, 1:])
    g[1:, :-1] += lamF * dFa
    g[1:, 1:] += lamF * dFb
    # wall faces: r_0 has -F(0, u_0)/dx, r_{N-1} has +F(u_{N-1}, 0)/dx
    _, _, dW = eo_flux(0.0 * un[:, 0], un[:, 0])
    _, dE, _ = eo_flux(un[:, -1], 0.0 * un[:, -1])
    g[1:, 0] -= lam[:, 0] * dW / dx
    g[1:, -1] += lam[:, -1] * dE / dx
    # viscous term, through the odd ghosts
    lamD = -nu * lam / dx**2
    gug = np.zeros((un.shape[0], nx + 2))
    gug[:, 2:] += lamD
    gug[:, :-2] += lamD
    gug[:, 1:-1] += -2.0 * lamD
    g[1:] += gug[:, 1:-1]
    g[1:, 0] -= gug[:, 0]
    g[1:, -1] -= gug[:, -1]
    return g


# ---------------------------------------------------------------------------
# Heat conduction with unknown conductivity k(u) (Section 3.4)
# ---------------------------------------------------------------------------
# Reading.  Rows are time levels, columns x cells on [0,1] with cell-based
# values.  Row m >= 1 carries the displayed implicit residual linking rows m-1
# and m, with k at the face taken at the mean of the two neighbouring values of
# row m.  Zero Dirichlet walls use the odd ghost, so the face value at a wall
# is exactly 0.  Row 0 carries the initial condition as a residual
# (u^0_i - u_init_i)/dt, i.e. a quadratic term on the initial values.
# k is represented by nodal values q_0..q_{K} at u_j = j/K (K = 31 for 32
# nodes), linear between nodes and constant outside [0, 1]:
#   ubar = clamp(u, 0, 1), s = min(floor(K ubar), K-1), theta = K ubar - s,
#   k = q_s + theta (q_{s+1} - q_s).
# The regulariser is w_reg * sum_j (q_{j+1} - 2 q_j + q_{j-1})^2.

def heat_conductivity(u, q):
    """k(u), dk/du, segment index s and local coordinate theta."""
    K = len(q) - 1
    ub = np.clip(u, 0.0, 1.0)
    s = np.minimum(np.floor(ub * K).astype(np.int64), K - 1)
    th = ub * K - s
    k = q[s] + th * (q[s + 1] - q[s])
    dk = np.where((u >= 0.0) & (u <= 1.0), K * (q[s + 1] - q[s]), 0.0)
    return k, dk, s, th


def _heat_faces(un):
    """Ghost-padded rows, face values (N_x + 1 faces) and face differences."""
    ug = _ghost_odd(un)
    uf = 0.5 * (ug[:, :-1] + ug[:, 1:])
    du = ug[:, 1:] - ug[:, :-1]
    return ug, uf, du


def heat_residual(u, q, dt, dx, u_init, kfun=None):
    """Residuals, shape (N_t, N_x): row 0 initial condition, rows >= 1 the PDE.

    k is the nodal representation q unless ``kfun`` (face value -> k) is given.
    """
    r = np.empty_like(u)
    r[0] = (u[0] - u_init) / dt
    un, uo = u[1:], u[:-1]
    _, uf, du = _heat_faces(un)
    kf = heat_conductivity(uf, q)[0] if kfun is None else kfun(uf)
    flux = kf * du / dx
    r[1:] = (un - uo) / dt - (flux[:, 1:] - flux[:, :-1]) / dx
    return r


def _heat_adjoint(u, q, lam, dt, dx):
    """dL/du and dL/dq given lam = dL/dr (shape of the residual array)."""
    g = np.zeros_like(u)
    gq = np.zeros_like(q)
    g[0] += lam[0] / dt
    li = lam[1:]
    g[1:] += li / dt
    g[:-1] -= li / dt
    un = u[1:]
    nx = u.shape[1]
    ug, uf, du = _heat_faces(un)
    kf, dkf, s, th = heat_conductivity(uf, q)
    # r = ... - (flux_E - flux_W)/dx, flux_f = kf * du_f / dx
    lamF = np.zeros((li.shape[0], nx + 1))
    lamF[:, 1:] -= li / dx
    lamF[:, :-1] += li / dx
    lam_du = lamF * kf / dx
    lam_k = lamF * du / dx
    gug = np.zeros_like(ug)
    gug[:, 1:] += lam_du
    gug[:, :-1] -= lam_du
    gug[:, 1:] += 0.5 * lam_k * dkf
    gug[:, :-1] += 0.5 * lam_k * dkf
    g[1:] += gug[:, 1:-1]
    g[1:, 0] -= gug[:, 0]
    g[1:, -1] -= gug[:, -1]
    np.add.at(gq, s, lam_k * (1.0 - th))
    np.add.at(gq, s + 1, lam_k * th)
    return g, gq


def _heat_reg(q):
    d2 = q[2:] - 2.0 * q[1:-1] + q[:-2]
    gq = np.zeros_like(q)
    gq[2:] += 2.0 * d2
    gq[1:-1] -= 4.0 * d2
    gq[:-2] += 2.0 * d2
    return float(np.sum(d2 * d2)), gq


# ---------------------------------------------------------------------------
# Poisson equation (Section 3.1)
# ---------------------------------------------------------------------------
# cell layout: finite volumes on [0,1]^d, value at cell centres; the Dirichlet
# value b = 0 is imposed by quadratic extrapolation from the wall and the two
# nearest centres: ghost = 8/3 b - 2 u_0 + 1/3 u_1.  Residual = discrete
# Laplacian - f in every cell; loss w_res * h^d * sum r^2.
# node layout: finite differences on the N+1 nodes per axis; the Dirichlet
# value is imposed directly on the boundary nodes (Section 3.1), so the
# stencil reads 0 there whatever the decomposition holds, the residual lives
# at the interior nodes, and the boundary nodes' unknowns do not enter the
# loss (their gradient is zero).

def _poisson_ghost_pad(u, axis):
    u0 = np.take(u, [0], axis=axis)
    u1 = np.take(u, [1], axis=axis)
    un = np.take(u, [-1], axis=axis)
    un1 = np.take(u, [-2], axis=axis)
    gl = -2.0 * u0 + u1 / 3.0
    gr = -2.0 * un + un1 / 3.0
    return np.concatenate([gl, u, gr], axis=axis)


def poisson_residual(u, f, h, layout="cell"):
    """Cell layout: Laplacian(u) - f in every cell.  Node: at interior nodes."""
    d = u.ndim
    if layout == "cell":
        lap = np.zeros_like(u)
        for ax in range(d):
            p = _poisson_ghost_pad(u, ax)
            n = u.shape[ax]
            lap += (np.take(p, range(2, n + 2), axis=ax) - 2.0 * u
                    + np.take(p, range(0, n), axis=ax)) / h[ax] ** 2
        return lap - f
    inner = tuple(slice(1, -1) for _ in range(d))
    u = np.where(_poisson_boundary_mask(u.shape), 0.0, u)   # the Dirichlet value on the nodes
    lap = np.zeros(tuple(s - 2 for s in u.shape))
    for ax in range(d):
        sp = [slice(1, -1)] * d
        sm = [slice(1, -1)] * d
        sp[ax] = slice(2, None)
        sm[ax] = slice(0, -2)
        lap += (u[tuple(sp)] - 2.0 * u[inner] + u[tuple(sm)]) / h[ax] ** 2
    return lap - f[inner]


def _poisson_boundary_mask(shape):
    m = np.zeros(shape, dtype=bool)
    for ax in range(len(shape)):
        idx = [slice(None)] * len(shape)
        idx[ax] = 0
        m[tuple(idx)] = True
        idx[ax] = -1
        m[tuple(idx)] = True
    return m


def _poisson_adjoint(u, lam, h, layout):
    d = u.ndim
    g = np.zeros_like(u)
    if layout == "cell":
        for ax in range(d):
            n = u.shape[ax]
            c = lam / h[ax] ** 2
            gp = np.zeros(tuple(s + 2 if a == ax else s for a, s in enumerate(u.shape)))
            sl = [slice(None)] * d
            sl[ax] = slice(2, n + 2)
            gp[tuple(sl)] += c
            sl[ax] = slice(0, n)
            gp[tuple(sl)] += c
            g += -2.0 * c
            sl[ax] = slice(1, n + 1)
            g += gp[tuple(sl)]
            # ghost_l = -2 u_0 + u_1/3, ghost_r = -2 u_{n-1} + u_{n-2}/3
            gl = np.take(gp, [0], axis=ax)
            gr = np.take(gp, [n + 1], axis=ax)
            for j, w in ((0, -2.0), (1, 1.0 / 3.0)):
                sl = [slice(None)] * d
                sl[ax] = slice(j, j + 1)
                g[tuple(sl)] += w * gl
                sl[ax] = slice(n - 1 - j, n - j)
                g[tuple(sl)] += w * gr
        return g
    inner = tuple(slice(1, -1) for _ in range(d))
    for ax in range(d):
        c = lam / h[ax] ** 2
        sp = [slice(1, -1)] * d
        sm = [slice(1, -1)] * d
        sp[ax] = slice(2, None)
        sm[ax] = slice(0, -2)
        g[tuple(sp)] += c
        g[tuple(sm)] += c
        g[inner] += -2.0 * c
    return np.where(_poisson_boundary_mask(u.shape), 0.0, g)  # boundary nodes are fixed


# ---------------------------------------------------------------------------
# Steady incompressible Navier-Stokes, lid-driven cavity (Section 3.3)
# ---------------------------------------------------------------------------
# Reading.  Collocated cell-centred finite volumes on [0,1]^2, N x N cells,
# fields u, v, p, axes (y, x).  No-slip walls by ghost cells: the wall value
# is the mean of the ghost and the adjacent cell (lid u = 1 at y = 1), zero
# normal pressure gradient (ghost p = adjacent p).  Momentum residuals use
# conservative central convection with face-averaged velocities (zero mass
# flux through walls), the central pressure gradient and the 5-point viscous
# term with 1/Re.  The continuity residual uses Rhie-Chow face velocities at
# interior faces,
#   U_e = (u_P + u_E)/2 - tau [ (p_E - p_P)/h - (g_P + g_E)/2 ],  g = (p_E - p_W)/(2h),
# tau = tau_factor * h, and zero flux through walls.  The pressure level is
# fixed by one extra residual p(0, 0).  Everything is polynomial in the
# unknowns (no branches), so the residual accepts complex input.

def _ns2d_pad(u, v, p, lid=1.0):
    n0, n1 = u.shape
    U = np.zeros((n0 + 2, n1 + 2), dtype=u.dtype)
    V = np.zeros_like(U)
    Pp = np.zeros_like(U)
    U[1:-1, 1:-1], V[1:-1, 1:-1], Pp[1:-1, 1:-1] = u, v, p
    U[1:-1, 0], U[1:-1, -1] = -u[:, 0], -u[:, -1]
    U[0, 1:-1], U[-1, 1:-1] = -u[0, :], 2.0 * lid - u[-1, :]
    V[1:-1, 0], V[1:-1, -1] = -v[:, 0], -v[:, -1]
    V[0, 1:-1], V[-1, 1:-1] = -v[0, :], -v[-1, :]
    Pp[1:-1, 0], Pp[1:-1, -1] = p[:, 0], p[:, -1]
    Pp[0, 1:-1], Pp[-1, 1:-1] = p[0, :], p[-1, :]
    return U, V, Pp


def ns2d_residuals(u, v, p, Re, h, tau_factor=1.0, lid=1.0):
    """Residuals (r_u, r_v, r_c) on every cell and the gauge residual p(0,0)."""
    n0, n1 = u.shape
    U, V, Pp = _ns2d_pad(u, v, p, lid)
    C = (slice(1, -1), slice(1, -1))
    E = (slice(1, -1), slice(2, None))
    W = (slice(1, -1), slice(0, -2))
    N = (slice(2, None), slice(1, -1))
    S = (slice(0, -2), slice(1, -1))
    jj, ii = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    me, mw, mn, ms = ii < n1 - 1, ii > 0, jj < n0 - 1, jj > 0   # interior faces
    nu = 1.0 / Re
    ue, uw, un, us = (U[C] + U[E]) / 2, (U[W] + U[C]) / 2, (U[C] + U[N]) / 2, (U[S] + U[C]) / 2
    ve, vw, vn, vs = (V[C] + V[E]) / 2, (V[W] + V[C]) / 2, (V[C] + V[N]) / 2, (V[S] + V[C]) / 2
    conv_u = (np.where(me, ue * ue, 0) - np.where(mw, uw * uw, 0)
              + np.where(mn, vn * un, 0) - np.where(ms, vs * us, 0)) / h
    conv_v = (np.where(me, ue * ve, 0) - np.where(mw, uw * vw, 0)
              + np.where(mn, vn * vn, 0) - np.where(ms, vs * vs, 0)) / h
    lap_u = (U[E] + U[W] + U[N] + U[S] - 4 * U[C]) / h**2
    lap_v = (V[E] + V[W] + V[N] + V[S] - 4 * V[C]) / h**2
    gx = (Pp[E] - Pp[W]) / (2 * h)
    gy = (Pp[N] - Pp[S]) / (2 * h)
    ru = conv_u + gx - nu * lap_u
    rv = conv_v + gy - nu * lap_v
    tau = tau_factor * h
    # Rhie-Chow face velocities at interior faces (index of the face's west/south cell)
    Ux = (u[:, :-1] + u[:, 1:]) / 2 - tau * ((p[:, 1:] - p[:, :-1]) / h - (gx[:, :-1] + gx[:, 1:]) / 2)
    Vy = (v[:-1, :] + v[1:, :]) / 2 - tau * ((p[1:, :] - p[:-1, :]) / h - (gy[:-1, :] + gy[1:, :]) / 2)
    Fx = np.zeros((n0, n1 + 1), dtype=Ux.dtype)
    Fy = np.zeros((n0 + 1, n1), dtype=Vy.dtype)
    Fx[:, 1:-1] = Ux
    Fy[1:-1, :] = Vy
    rc = (Fx[:, 1:] - Fx[:, :-1] + Fy[1:, :] - Fy[:-1, :]) / h
    return ru, rv, rc, p[0, 0]


def ns2d_fields_residual_jacobian_grad(u, v, p, lam_u, lam_v, lam_c, Re, h, tau_factor=1.0,
                                       lid=1.0, eps=1e-30):
    """J^T lambda for the three residual fields, J by complex-step differentiation.

    Every residual reads unknowns at most 2 cells away along each axis, so the
    unknowns of one field on cells (a, b) mod 5 never share a residual: one
    complex evaluation per (field, a, b) perturbs all of them at once and
    yields their Jacobian columns exactly (the imaginary part of r(w + i eps e)
    is eps dr/dw to rounding, with no subtraction).  75 evaluations in all.
    """
    n0, n1 = u.shape
    base = [np.asarray(u, complex), np.asarray(v, complex), np.asarray(p, complex)]
    grads = [np.zeros((n0, n1)) for _ in range(3)]
    jj, ii = np.meshgrid(np.arange(n0), np.arange(n1), indexing="ij")
    for f in range(3):
        for a in range(5):
            for b in range(5):
                w = [x.copy() for x in base]
                sel = ((jj % 5) == a) & ((ii % 5) == b)
                w[f] = w[f] + 1j * eps * sel
                ru, rv, rc, _ = ns2d_residuals(w[0], w[1], w[2], Re, h, tau_factor, lid)
                # the perturbed cell in each residual's 5 x 5 neighbourhood
                dj = ((a - jj + 2) % 5) - 2
                di = ((b - ii + 2) % 5) - 2
                tj, ti = jj + dj, ii + di
                ok = (tj >= 0) & (tj < n0) & (ti >= 0) & (ti < n1)
                contrib = (ru.imag * lam_u + rv.imag * lam_v + rc.imag * lam_c) / eps
                np.add.at(grads[f], (tj[ok], ti[ok]), contrib[ok])
    return grads


# ---------------------------------------------------------------------------
# Penalised steady Navier-Stokes in 3-D, body shape (Section 3.5, eq_nschi3)
# ---------------------------------------------------------------------------
# Reading.  Fields u, v, w, p, chihat on (z, y, x) cells of [0,1] x [0,1] x
# [0,2], flow along x.  chi = 1 / (1 + exp(-(chihat - 5))), so that the
# initial guess chihat = 0 is chi = 1 / (1 + e^5), almost no body.  Section
# 3.5 prints the transform with chihat + 5 but states in the same paragraph
# that chihat = 0 corresponds to chi = 1 / (1 + e^5); the two statements
# disagree, and only the shift by -5 makes the stated initial guess (uniform
# inflow, no pressure, no body) consistent, so that reading is taken.
# Residuals follow
# the cavity discretisation (Section 3.3 reading) in 3-D with the spacings of
# each axis:
#   momentum:  r = (1 - chi) (conv + grad p - (D/Re) lap) + lambda chi u_c
#   continuity: sum over axes of Rhie-Chow face fluxes.
# Boundaries by ghost cells: inlet x = 0 with u = (1, 0, 0) and zero normal
# pressure gradient; outlet x = 2 with p = 0 (odd ghost) and zero-gradient
# velocity; free-slip walls in y and z (odd ghost for the normal component,
# even ghosts for the tangential ones and p).  Convective and mass fluxes
# through x-boundary faces use the boundary values (inlet velocity, outlet
# cell value), through walls they vanish.  Polynomial in u, v, w, p and
# analytic in chihat, so complex input is accepted.

def ns3d_chi(ch):
    """Body fraction from its transform: chi = 1/(1 + exp(-(chihat - 5)))."""
    return 1.0 / (1.0 + np.exp(-(ch - 5.0)))


def _ns3d_pad(f, kind):
    """Pad one field with its ghost cells; kind in u, v, w, p."""
    nz, ny, nx = f.shape
    P = np.zeros((nz + 2, ny + 2, nx + 2), dtype=f.dtype)
    P[1:-1, 1:-1, 1:-1] = f
    c = P[1:-1, 1:-1, :]
    # x: inlet (low) / outlet (high)
    if kind == "u":
        c[:, :, 0] = 2.0 - f[:, :, 0]
    elif kind in ("v", "w"):
        c[:, :, 0] = -f[:, :, 0]
    else:
        c[:, :, 0] = f[:, :, 0]
    c[:, :, -1] = -f[:, :, -1] if kind == "p" else f[:, :, -1]
    # y walls: v normal, others even; z walls: w normal
    sy = -1.0 if kind == "v" else 1.0
    P[1:-1, 0, 1:-1] = sy * f[:, 0, :]
    P[1:-1, -1, 1:-1] = sy * f[:, -1, :]
    sz = -1.0 if kind == "w" else 1.0
    P[0, 1:-1, 1:-1] = sz * f[0, :, :]
    P[-1, 1:-1, 1:-1] = sz * f[-1, :, :]
    return P


def ns3d_residuals(u, v, w, p, ch, Re, D, lam, h, tau_factor=1.0):
    """(r_u, r_v, r_w, r_c) on every cell; h = (hz, hy, hx)."""
    hz, hy, hx = h
    nz, ny, nx = u.shape
    U, V, W, Pp = _ns3d_pad(u, "u"), _ns3d_pad(v, "v"), _ns3d_pad(w, "w"), _ns3d_pad(p, "p")
    C = (slice(1, -1),) * 3
    def sh(a, dz, dy, dx):
        return a[1 + dz:a.shape[0] - 1 + dz, 1 + dy:a.shape[1] - 1 + dy, 1 + dx:a.shape[2] - 1 + dx]
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mn, ms = jj < ny - 1, jj > 0
    mt, mb = kk < nz - 1, kk > 0
    nu = D / Re
    chi = ns3d_chi(ch)
    # face normal velocities (face averages; x-boundary faces get the boundary value)
    Ue, Uw = (U[C] + sh(U, 0, 0, 1)) / 2, (sh(U, 0, 0, -1) + U[C]) / 2
    Vn, Vs = np.where(mn, (V[C] + sh(V, 0, 1, 0)) / 2, 0), np.where(ms, (sh(V, 0, -1, 0) + V[C]) / 2, 0)
    Wt, Wb = np.where(mt, (W[C] + sh(W, 1, 0, 0)) / 2, 0), np.where(mb, (sh(W, -1, 0, 0) + W[C]) / 2, 0)
    res = []
    for F in (U, V, W):
        fe, fw = (F[C] + sh(F, 0, 0, 1)) / 2, (sh(F, 0, 0, -1) + F[C]) / 2
        fn, fs = (F[C] + sh(F, 0, 1, 0)) / 2, (sh(F, 0, -1, 0) + F[C]) / 2
        ft, fb = (F[C] + sh(F, 1, 0, 0)) / 2, (sh(F, -1, 0, 0) + F[C]) / 2
        conv = (Ue * fe - Uw * fw) / hx + (Vn * fn - Vs * fs) / hy + (Wt * ft - Wb * fb) / hz
        lap = ((sh(F, 0, 0, 1) - 2 * F[C] + sh(F, 0, 0, -1)) / hx**2
               + (sh(F, 0, 1, 0) - 2 * F[C] + sh(F, 0, -1, 0)) / hy**2
               + (sh(F, 1, 0, 0) - 2 * F[C] + sh(F, -1, 0, 0)) / hz**2)
        res.append((conv, lap, F[C]))
    gx = (sh(Pp, 0, 0, 1) - sh(Pp, 0, 0, -1)) / (2 * hx)
    gy = (sh(Pp, 0, 1, 0) - sh(Pp, 0, -1, 0)) / (2 * hy)
    gz = (sh(Pp, 1, 0, 0) - sh(Pp, -1, 0, 0)) / (2 * hz)
    out = []
    for (conv, lap, f), g in zip(res, (gx, gy, gz)):
        out.append((1.0 - chi) * (conv + g - nu * lap) + lam * chi * f)
    # continuity: Rhie-Chow at interior faces, boundary values at x ends, 0 at walls
    def rc_faces(vel, pres, gr, hh, axis):
        a0 = [slice(None)] * 3
        a1 = [slice(None)] * 3
        a0[axis] = slice(None, -1)
        a1[axis] = slice(1, None)
        a0, a1 = tuple(a0), tuple(a1)
        return (vel[a0] + vel[a1]) / 2 - tau_factor * hh * ((pres[a1] - pres[a0]) / hh - (gr[a0] + gr[a1]) / 2)
    Fx = np.zeros((nz, ny, nx + 1), dtype=np.result_type(u, p))
    Fx[:, :, 1:-1] = rc_faces(u, p, gx, hx, 2)
    Fx[:, :, 0] = 1.0
    Fx[:, :, -1] = u[:, :, -1]
    Fy = np.zeros((nz, ny + 1, nx), dtype=Fx.dtype)
    Fy[:, 1:-1, :] = rc_faces(v, p, gy, hy, 1)
    Fz = np.zeros((nz + 1, ny, nx), dtype=Fx.dtype)
    Fz[1:-1, :, :] = rc_faces(w, p, gz, hz, 0)
    rcont = ((Fx[:, :, 1:] - Fx[:, :, :-1]) / hx + (Fy[:, 1:, :] - Fy[:, :-1, :]) / hy
             + (Fz[1:, :, :] - Fz[:-1, :, :]) / hz)
    return out[0], out[1], out[2], rcont


def ns3d_residual_jacobian_grad(fields, lams, coef, h, eps=1e-30, colours=None):
    """J^T lambda for the four residual fields by complex-step differentiation;
    5 x 5 x 5 colouring (reach 2 along each axis), 5 fields: 625 evaluations.

    colours: optional list of (field, a, b, c); only those colour classes are
    evaluated, so the result is exact on the cells (k, j, i) = (a, b, c) mod 5
    of those fields and zero elsewhere (a sample of a grid too large for all
    625 evaluations)."""
    nz, ny, nx = fields[0].shape
    base = [np.asarray(f, complex) for f in fields]
    grads = [np.zeros((nz, ny, nx)) for _ in range(5)]
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    todo = None if colours is None else set(tuple(x) for x in colours)
    for f in range(5):
        for a in range(5):
            for b in range(5):
                for c in range(5):
                    if todo is not None and (f, a, b, c) not in todo:
                        continue
                    sel = ((kk % 5) == a) & ((jj % 5) == b) & ((ii % 5) == c)
                    if not sel.any():
                        continue
                    wv = list(base)
                    wv[f] = base[f] + 1j * eps * sel
                    rs = ns3d_residuals(*wv, coef["Re"], coef["D"], coef["lam"], h,
                                        coef.get("tau", 1.0))
                    contrib = sum(r.imag * l for r, l in zip(rs, lams)) / eps
                    dk = ((a - kk + 2) % 5) - 2
                    dj = ((b - jj + 2) % 5) - 2
                    di = ((c - ii + 2) % 5) - 2
                    tk, tj, ti = kk + dk, jj + dj, ii + di
                    ok = (tk >= 0) & (tk < nz) & (tj >= 0) & (tj < ny) & (ti >= 0) & (ti < nx)
                    np.add.at(grads[f], (tk[ok], tj[ok], ti[ok]), contrib[ok])
    return grads


def ns3d_fine_grad_colours(p, u, colours):
    """dL/du of the body problem on the cells of the given colour classes
    (field, a, b, c): exact there, zero elsewhere; for grids where the full
    625-evaluation Jacobian is too slow."""
    h = p.spacing()
    c = 2.0 * p.w_res * float(np.prod(h))
    rs = ns3d_residuals(*u, p.coef["Re"], p.coef["D"], p.coef["lam"], h, p.coef.get("tau", 1.0))
    g = ns3d_residual_jacobian_grad(u, [c * x for x in rs], p.coef, h, colours=colours)
    _, gd = _data_term(p, list(u))
    return [a + b for a, b in zip(g, gd)]


# ---------------------------------------------------------------------------
# Loss and gradient
# ---------------------------------------------------------------------------

def _data_term(p, u):
    """Data term of one field u, or of a list of fields (meas_field and
    point_field select the field of each cell and point).

    With off-grid points the misfits of the cells and of the points share one
    normalisation, w_data / (n_cells + n_points); a point's value is the
    d-linear sample of its field (oracle/offgrid_oracle.py)."""
    n_pts = 0 if p.meas_points is None else len(p.meas_points)
    if isinstance(u, (list, tuple)):
        n_cells = 0 if p.meas_cell is None else len(p.meas_cell)
        if n_cells + n_pts == 0:
            return 0.0, [np.zeros_like(x) for x in u]
        mf = np.zeros(n_cells, int) if p.meas_field is None else np.asarray(p.meas_field)
        pf = np.zeros(n_pts, int) if p.point_field is None else np.asarray(p.point_field)
        w = p.w_data / (n_cells + n_pts)
        total = 0.0
        gs = []
        if n_pts:
            from .offgrid_oracle import data_term, sample_weights
            origin, lengths = p.domain()
            idx, wt = sample_weights(p.meas_points, u[0].shape, lengths, origin)
        for f, x in enumerate(u):
            flat = x.reshape(-1)
            g = np.zeros_like(flat)
            if n_cells:
                sel = mf == f
                diff = flat[p.meas_cell[sel]] - p.meas_value[sel]
                np.add.at(g, p.meas_cell[sel], 2.0 * w * diff)
                total += float(w * np.sum(diff * diff))
            if n_pts and np.any(pf == f):
                sel = pf == f
                t, gp = data_term(x, idx[sel], wt[sel], np.asarray(p.point_value)[sel],
                                  w_data=w * int(sel.sum()))
                total += t
                g += gp.reshape(-1)
            gs.append(g.reshape(x.shape))
        return total, gs
    n_cells = 0 if p.meas_cell is None else len(p.meas_cell)
    if n_cells + n_pts == 0:
        return 0.0, np.zeros_like(u)
    w = p.w_data / (n_cells + n_pts)
    total = 0.0
    g = np.zeros(u.size)
    if n_cells:
        flat = u.reshape(-1)
        diff = flat[p.meas_cell] - p.meas_value
        np.add.at(g, p.meas_cell, 2.0 * w * diff)
        total += float(w * np.sum(diff * diff))
    if n_pts:
        from .offgrid_oracle import data_term, sample_weights
        origin, lengths = p.domain()
        idx, wt = sample_weights(p.meas_points, u.shape, lengths, origin)
        t, gp = data_term(u, idx, wt, p.point_value, w_data=w * n_pts)
        total += t
        g += gp.reshape(-1)
    return total, g.reshape(u.shape)


def loss_terms(p, u, q=None):
    """Loss components {"res", "data", "reg", "total"} of the composed field u."""
    h = p.spacing()
    dV = float(np.prod(h))
    reg = 0.0
    bnd = 0.0
    if p.pde == "burgers":
        r = burgers_residual(u, p.coef["nu"], h[0], h[1])
    elif p.pde == "heat":
        r = heat_residual(u, q, h[0], h[1], p.aux)
        reg = p.w_reg * _heat_reg(q)[0]
    elif p.pde == "poisson":
        r = poisson_residual(u, p.coef["f"], h, p.layout)
    elif p.pde == "ns2d":
        ru, rv, rc, rg = ns2d_residuals(u[0], u[1], u[2], p.coef["Re"], h[0],
                                        p.coef.get("tau", 1.0))
        r = np.concatenate([ru.ravel(), rv.ravel(), rc.ravel(), [rg]])
    elif p.pde == "ns3d":
        rs = ns3d_residuals(*u, p.coef["Re"], p.coef["D"], p.coef["lam"], h, p.coef.get("tau", 1.0))
        r = np.concatenate([x.ravel() for x in rs])
    else:
        raise ValueError(p.pde)
    res = p.w_res * dV * float(np.sum(r * r)) + bnd
    data, _ = _data_term(p, u)
    return {"res": res, "data": data, "reg": reg, "total": res + data + reg}


def loss_grad_fine(p, u, q=None):
    """Loss terms and dL/du (and dL/dq for heat) at the composed fine field."""
    h = p.spacing()
    dV = float(np.prod(h))
    terms = loss_terms(p, u, q)
    gq = None
    if p.pde == "burgers":
        r = burgers_residual(u, p.coef["nu"], h[0], h[1])
        g = _burgers_adjoint(u, 2.0 * p.w_res * dV * r, p.coef["nu"], h[0], h[1])
    elif p.pde == "heat":
        r = heat_residual(u, q, h[0], h[1], p.aux)
        g, gq = _heat_adjoint(u, q, 2.0 * p.w_res * dV * r, h[0], h[1])
        gq = np.zeros_like(q) if p.k_fixed else gq + p.w_reg * _heat_reg(q)[1]
    elif p.pde == "poisson":
        r = poisson_residual(u, p.coef["f"], h, p.layout)
        g = _poisson_adjoint(u, 2.0 * p.w_res * dV * r, h, p.layout)
    elif p.pde == "ns2d":
        Re, tf = p.coef["Re"], p.coef.get("tau", 1.0)
        ru, rv, rc, rg = ns2d_residuals(u[0], u[1], u[2], Re, h[0], tf)
        c = 2.0 * p.w_res * dV
        g = ns2d_fields_residual_jacobian_grad(u[0], u[1], u[2], c * ru, c * rv, c * rc, Re,
                                               h[0], tf)
        g[2][0, 0] += c * rg
        _, gd = _data_term(p, list(u))
        return terms, [a + b for a, b in zip(g, gd)], gq
    elif p.pde == "ns3d":
        rs = ns3d_residuals(*u, p.coef["Re"], p.coef["D"], p.coef["lam"], h, p.coef.get("tau", 1.0))
        c = 2.0 * p.w_res * dV
        g = ns3d_residual_jacobian_grad(u, [c * x for x in rs], p.coef, h)
        _, gd = _data_term(p, list(u))
        return terms, [a + b for a, b in zip(g, gd)], gq
    else:
        raise ValueError(p.pde)
    _, gd = _data_term(p, u)
    return terms, g + gd, gq


def loss_grad_levels(p, levels, q=None):
    """Loss terms and the gradient with respect to every level (and q).

    Multi-field problems take and return a list over fields of level lists.
    """
    if p.n_fields > 1:
        u = [compose(lv, p.layout) for lv in levels]
        terms, g, gq = loss_grad_fine(p, u, q)
        return terms, [chain_grad(gf, len(lv), p.layout) for gf, lv in zip(g, levels)], gq
    u = compose(levels, p.layout)
    terms, g, gq = loss_grad_fine(p, u, q)
    return terms, chain_grad(g, len(levels), p.layout), gq


# ---------------------------------------------------------------------------
# Adam (Kingma and Ba, Algorithm 1)
# ---------------------------------------------------------------------------

def adam_step(x, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns new (x, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1**t)
    vh = v / (1.0 - b2**t)
    return x - lr * mh / (np.sqrt(vh) + eps), m, v


@dataclass
class OracleState:
    levels: list
    m: list
    v: list
    q: np.ndarray = None
    mq: np.ndarray = None
    vq: np.ndarray = None
    t: int = 0

    @classmethod
    def zeros_like_levels(cls, levels, q=None):
        if levels and isinstance(levels[0], (list, tuple)):  # several fields
            return cls([[np.array(a, dtype=np.float64) for a in lv] for lv in levels],
                       [[np.zeros_like(a) for a in lv] for lv in levels],
                       [[np.zeros_like(a) for a in lv] for lv in levels], None, None, None, 0)
        z = [np.zeros_like(a) for a in levels]
        return cls([np.array(a, dtype=np.float64) for a in levels], z,
                   [np.zeros_like(a) for a in levels],
                   None if q is None else np.array(q, dtype=np.float64),
                   None if q is None else np.zeros_like(q),
                   None if q is None else np.zeros_like(q), 0)


def oracle_step(p, st, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One mODIL optimiser step: loss and gradient at the current levels, then
    Adam on every level and on q.  Returns the loss terms before the update."""
    terms, grads, gq = loss_grad_levels(p, st.levels, st.q)
    st.t += 1
    if p.n_fields > 1:
        for f, gf in enumerate(grads):
            for i, g in enumerate(gf):
                st.levels[f][i], st.m[f][i], st.v[f][i] = adam_step(
                    st.levels[f][i], st.m[f][i], st.v[f][i], g, st.t, lr, b1, b2, eps)
        return terms
    for i, g in enumerate(grads):
        st.levels[i], st.m[i], st.v[i] = adam_step(st.levels[i], st.m[i], st.v[i],
                                                   g, st.t, lr, b1, b2, eps)
    if st.q is not None:
        st.q, st.mq, st.vq = adam_step(st.q, st.mq, st.vq, gq, st.t, lr * p.k_scale, b1, b2, eps)
    return terms


# ---------------------------------------------------------------------------
# Reference generators (test data only)
# ---------------------------------------------------------------------------

def burgers_explicit_solve(u0, nu, dx, t_out, cfl=0.4, bc="dirichlet"):
    """March u_t + (u^2/2)_x = nu u_xx with forward Euler finite volumes.

    Same flux as the residual (Engquist-Osher, the upwind flux against the
    zero wall value at the walls, odd viscous ghosts) or a periodic variant.  Returns the cell
    averages at each time in ``t_out`` (linear interpolation between steps).
    """
    u = np.array(u0, dtype=np.float64)
    t = 0.0
    out = []
    k = 0
    t_out = list(t_out)
    prev_t, prev_u = t, u.copy()
    while k < len(t_out):
        if t >= t_out[k]:
            a = (t_out[k] - prev_t) / (t - prev_t) if t > prev_t else 1.0
            out.append((1.0 - a) * prev_u + a * u)
            k += 1
            continue
        umax = max(float(np.max(np.abs(u))), 1e-12)
        dt = cfl * min(dx / umax, dx * dx / (2.0 * nu) if nu > 0 else np.inf)
        if bc == "periodic":
            ul = np.roll(u, 1)
            ur = np.roll(u, -1)
            Fe, _, _ = eo_flux(u, ur)
            Fw = np.roll(Fe, 1)
            lap = (ur - 2.0 * u + ul) / dx**2
        else:
            F = np.zeros(len(u) + 1)
            F[1:-1], _, _ = eo_flux(u[:-1], u[1:])
            F[0], _, _ = eo_flux(0.0, u[0])        # zero Dirichlet walls, upwind
            F[-1], _, _ = eo_flux(u[-1], 0.0)
            Fe, Fw = F[1:], F[:-1]
            ug = np.concatenate([[-u[0]], u, [-u[-1]]])
            lap = (ug[2:] - 2.0 * u + ug[:-2]) / dx**2
        prev_t, prev_u = t, u.copy()
        u = u - dt * (Fe - Fw) / dx + dt * nu * lap
        t += dt
    return np.array(out)


def burgers_implicit_solve(u0, nt, dt, dx, nu=0.0, tol=1e-14, max_iter=100):
    """The discrete Burgers problem of the residual above, solved row by row:
    row 0 is the given initial condition, and each later row is the root of
    its residual given the previous row (backward Euler, Engquist-Osher flux,
    zero convective flux through the walls, odd viscous ghosts), found by
    Newton's method with the residual's tridiagonal Jacobian.  This is how the
    reference of the reconstruction problem of Section 3.2 is made ("solve the
    discrete problem with zero Dirichlet boundary conditions and the initial
    condition").  Returns the (nt, nx) field."""
    from scipy.linalg import solve_banded
    u0 = np.asarray(u0, dtype=np.float64)
    nx = len(u0)
    out = np.zeros((nt, nx))
    out[0] = u0
    for n in range(1, nt):
        prev = out[n - 1]
        w = prev.copy()
        for _ in range(max_iter):
            r = burgers_residual(np.stack([prev, w]), nu, dt, dx)[0]
            # Jacobian: dr_i/du_{i-1}, dr_i/du_i, dr_i/du_{i+1}
            _, dFa, dFb = eo_flux(w[:-1], w[1:])        # face i+1/2 of cells i, i+1
            lo = np.zeros(nx)
            di = np.full(nx, 1.0 / dt)
            up = np.zeros(nx)
            di[:-1] += dFa / dx                          # east face of cell i
            up[:-1] += dFb / dx
            di[1:] -= dFb / dx                           # west face of cell i+1
            lo[1:] -= dFa / dx
            di[0] -= min(w[0], 0.0) / dx                  # wall faces
            di[-1] += max(w[-1], 0.0) / dx
            c = nu / dx**2
            di += 2.0 * c
            di[0] += c                                   # odd ghosts
            di[-1] += c
            lo[1:] -= c
            up[:-1] -= c
            ab = np.zeros((3, nx))
            ab[0, 1:] = up[:-1]
            ab[1] = di
            ab[2, :-1] = lo[1:]
            dw = solve_banded((1, 1), ab, -r)
            w = w + dw
            if np.max(np.abs(dw)) < tol * max(1.0, np.max(np.abs(w))):
                break
        out[n] = w
    return out


def heat_implicit_solve(u_init, nt, dt, dx, kfun, tol=1e-13, max_iter=200):
    """Solve the heat residual rows to zero one time row after another.

    Picard iteration: freeze k at the current iterate, solve the tridiagonal
    linear system of the residual, repeat until the update is below tol.
    ``kfun(u)`` returns the conductivity at face values u.
    """
    from scipy.linalg import solve_banded
    nx = len(u_init)
    u = np.zeros((nt, nx))
    u[0] = u_init
    for m in range(1, nt):
        w = u[m - 1].copy()
        for _ in range(max_iter):
            wg = np.concatenate([[-w[0]], w, [-w[-1]]])
            kf = kfun(0.5 * (wg[:-1] + wg[1:]))
            kE, kW = kf[1:], kf[:-1]
            c = dt / dx**2
            ab = np.zeros((3, nx))
            diag = 1.0 + c * (kE + kW)
            diag[0] += c * kW[0]          # odd ghost on the left
            diag[-1] += c * kE[-1]        # odd ghost on the right
            ab[1] = diag
            ab[0, 1:] = -c * kE[:-1]
            ab[2, :-1] = -c * kW[1:]
            wn = solve_banded((1, 1), ab, u[m - 1])
            done = np.max(np.abs(wn - w)) < tol
            w = wn
            if done:
                break
        u[m] = w
    return u
