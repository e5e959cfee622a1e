"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each test checks a printed
value, a closed form, a convergence order, an invariant or a finite-difference
derivative, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as o
from paper_2303_04679_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden_matrices():
    mats = {}
    cur = None
    with open(os.path.join(GOLDEN, "interp_matrices.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith(("node", "cell")):
                parts = line.split()
                num, den = parts[-1].split("/")
                cur = (parts[0], parts[1])
                mats[cur] = [float(num) / float(den), []]
            else:
                mats[cur][1].append([float(x) for x in line.split()])
    return {k: v[0] * np.array(v[1]) for k, v in mats.items()}


# --------------------------------------------------------------------------
# Interpolation operators and the decomposition (Section 2.2)
# --------------------------------------------------------------------------

def test_interp_matrices_match_printed():
    """The node and cell matrices for grids 8 -> 4 -> 2 printed in Section 2.2."""
    g = _read_golden_matrices()
    np.testing.assert_array_equal(o.interp_matrix(4, "node"), g[("node", "T1")])
    np.testing.assert_array_equal(o.interp_matrix(2, "node"), g[("node", "T2")])
    np.testing.assert_array_equal(o.interp_matrix(4, "cell"), g[("cell", "T1")])
    np.testing.assert_array_equal(o.interp_matrix(2, "cell"), g[("cell", "T2")])


@pytest.mark.parametrize("n", [2, 3, 5, 16, 64])
def test_cell_interp_reproduces_linear_functions(n):
    """Linear interpolation/extrapolation is exact on linear data (closed form)."""
    xc = (np.arange(n) + 0.5) / n
    xf = (np.arange(2 * n) + 0.5) / (2 * n)
    a, b = 0.37, -1.9
    np.testing.assert_allclose(o.interp_matrix(n) @ (a * xc + b), a * xf + b, rtol=0, atol=1e-14)
    # rows sum to one: constants are preserved
    np.testing.assert_allclose(o.interp_matrix(n).sum(axis=1), 1.0, atol=1e-15)


def test_single_cell_level_is_injected():
    np.testing.assert_array_equal(o.interp_matrix(1), [[1.0], [1.0]])


def test_tensor_product_prolongation_bilinear_exact():
    """2-D and 3-D prolongation reproduce bilinear/trilinear data exactly."""
    for shape in [(4, 8), (2, 4, 8)]:
        grids_c = np.meshgrid(*[(np.arange(n) + 0.5) / n for n in shape], indexing="ij")
        grids_f = np.meshgrid(*[(np.arange(2 * n) + 0.5) / (2 * n) for n in shape], indexing="ij")
        fc = 1.0 + sum((k + 1) * g for k, g in enumerate(grids_c)) + 0.5 * grids_c[0] * grids_c[-1]
        ff = 1.0 + sum((k + 1) * g for k, g in enumerate(grids_f)) + 0.5 * grids_f[0] * grids_f[-1]
        np.testing.assert_allclose(o.prolong(fc), ff, atol=1e-13)


@pytest.mark.parametrize("layout,shape,L", [("cell", (16, 32), 4), ("cell", (8, 8, 16), 4),
                                            ("node", (16, 16), 3), ("cell", (64,), 7)])
def test_adjoint_identity_every_level_pair_and_chain(layout, shape, L):
    """<T x, y> = <x, T^T y> for every level pair and <M x, y> = <x, M^T y>."""
    rng = np.random.default_rng(1)
    shapes = o.level_shapes(shape, L, layout)
    for i in range(L - 1):
        x = rng.normal(size=shapes[i + 1])
        y = rng.normal(size=shapes[i])
        lhs = np.vdot(o.prolong(x, layout), y)
        rhs = np.vdot(x, o.restrict(y, layout))
        assert abs(lhs - rhs) <= 1e-14 * (abs(lhs) + np.linalg.norm(x) * np.linalg.norm(y))
    xs = [rng.normal(size=s) for s in shapes]
    y = rng.normal(size=shapes[0])
    lhs = np.vdot(o.compose(xs, layout), y)
    rhs = sum(np.vdot(a, b) for a, b in zip(xs, o.chain_grad(y, L, layout)))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


@pytest.mark.parametrize("layout", ["cell", "node"])
def test_horner_equals_explicit_sum(layout):
    """The Horner form of M_L equals its explicit sum (Section 2.2)."""
    rng = np.random.default_rng(2)
    shapes = o.level_shapes((32, 32), 5, layout)
    lv = [rng.normal(size=s) for s in shapes]
    np.testing.assert_allclose(o.compose(lv, layout), o.compose_explicit(lv, layout), atol=1e-12)


def test_one_level_is_plain_odil():
    """L = 1: the decomposition is the identity and the gradient is dL/du."""
    rng = np.random.default_rng(3)
    u = rng.normal(size=(16, 16))
    np.testing.assert_array_equal(o.compose([u]), u)
    p = _burgers_problem((16, 16), 1, seed=3)
    t1, g1, _ = o.loss_grad_levels(p, [u])
    t2, g2, _ = o.loss_grad_fine(p, u)
    assert t1["total"] == t2["total"]
    np.testing.assert_array_equal(g1[0], g2)


# --------------------------------------------------------------------------
# Burgers (Section 3.2; viscous variant)
# --------------------------------------------------------------------------

def _burgers_problem(shape, L, seed=0, nu=0.01, n_meas=20):
    nt, nx = shape
    cells = inputs.measurement_cells(nt * nx, n_meas, seed)
    vals = np.random.default_rng(seed + 1).normal(size=n_meas)
    return o.Problem("burgers", shape, L, coef={"nu": nu}, w_res=1.0, w_data=1.0,
                     meas_cell=cells, meas_value=vals)


def _burgers_exact(x, t, A=0.7):
    u = A * np.sin(math.pi * x) * np.exp(-t)
    ut = -u
    ux = A * math.pi * np.cos(math.pi * x) * np.exp(-t)
    uxx = -(math.pi**2) * u
    return u, ut, ux, uxx


def test_burgers_residual_consistent_with_pde_first_order():
    """Residual of a smooth field -> u_t + u u_x - nu u_xx at first order."""
    nu = 0.05
    errs = []
    for n in (32, 64, 128, 256):
        dt, dx = 1.0 / n, 2.0 / n
        x = -1.0 + (np.arange(n) + 0.5) * dx
        t = (np.arange(n) + 0.5) * dt
        X, Tm = np.meshgrid(x, t)
        u, ut, ux, uxx = _burgers_exact(X, Tm)
        r = o.burgers_residual(u, nu, dt, dx)
        R = (ut + u * ux - nu * uxx)[1:]
        errs.append(np.max(np.abs(r - R)))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.7 < q < 2.3 for q in rates), (errs, rates)


def test_burgers_constant_field_closed_form():
    """Constant c: interior residual 0.  The walls carry the value 0: with
    c > 0 the flow enters nothing at the left wall (upwind flux F(0, c) = 0)
    and leaves through the right one (F(c, 0) = c^2/2, the interior flux), so
    only the left cell sees a flux difference, c^2/(2 dx); with c < 0 the
    mirror image.  The odd viscous ghost adds 2 nu c / dx^2 at both walls."""
    n, nu = 16, 0.03
    dt, dx = 1.0 / n, 2.0 / n
    for c in (0.8, -0.6):
        r = o.burgers_residual(np.full((n, n), c), nu, dt, dx)
        np.testing.assert_allclose(r[:, 1:-1], 0.0, atol=1e-12)
        inflow = c * c / (2 * dx)
        left = (inflow if c > 0 else 0.0) + 2 * nu * c / dx**2
        right = (-inflow if c < 0 else 0.0) + 2 * nu * c / dx**2
        np.testing.assert_allclose(r[:, 0], left, rtol=1e-13)
        np.testing.assert_allclose(r[:, -1], right, rtol=1e-13)


def test_burgers_mass_balance_of_residual():
    """sum_i r^n_i dx = (M^n - M^{n-1})/dt + (outflow through the walls)
    + 2 nu (u_0 + u_{N-1})/dx (telescoping); the wall fluxes are the upwind
    fluxes against the wall value 0: max(u_{N-1}, 0)^2/2 and min(u_0, 0)^2/2."""
    rng = np.random.default_rng(5)
    n, nu = 24, 0.02
    dt, dx = 1.0 / n, 2.0 / n
    u = rng.normal(size=(n, n))
    r = o.burgers_residual(u, nu, dt, dx)
    M = u.sum(axis=1) * dx
    out = 0.5 * np.maximum(u[1:, -1], 0.0) ** 2 - 0.5 * np.minimum(u[1:, 0], 0.0) ** 2
    rhs = (M[1:] - M[:-1]) / dt + out + 2 * nu * (u[1:, 0] + u[1:, -1]) / dx
    np.testing.assert_allclose(r.sum(axis=1) * dx, rhs, rtol=1e-11, atol=1e-11)


def test_burgers_implicit_step_dissipates_energy():
    """A row solved to zero residual has no more energy than the row before."""
    from scipy.optimize import root
    rng = np.random.default_rng(6)
    n, nu = 32, 0.01
    dx, dt = 2.0 / n, 0.05
    x = -1.0 + (np.arange(n) + 0.5) * dx
    for trial in range(5):
        prev = inputs.burgers_ic(x, rng.normal(0, 0.5, 4))
        sol = root(lambda w: o.burgers_residual(np.vstack([prev, w]), nu, dt, dx)[0],
                   prev, method="hybr", tol=1e-13)
        assert sol.success
        assert np.sum(sol.x**2) <= np.sum(prev**2) + 1e-12


def test_burgers_explicit_solver_invariants():
    """Explicit solver: periodic mass conserved; Dirichlet energy non-increasing."""
    n = 64
    dx = 2.0 / n
    x = -1.0 + (np.arange(n) + 0.5) * dx
    u0 = inputs.burgers_ic(x, inputs.burgers_ic_amplitudes(11))
    ts = np.linspace(0.0, 1.0, 21)
    per = o.burgers_explicit_solve(u0 + 0.3, 0.01, dx, ts, bc="periodic")
    np.testing.assert_allclose(per.sum(axis=1), (u0 + 0.3).sum(), rtol=1e-12)
    dirich = o.burgers_explicit_solve(u0, 0.01, dx, ts)
    E = np.sum(dirich**2, axis=1)
    assert np.all(np.diff(E) <= 1e-12)


def test_burgers_implicit_solve_reference_of_the_paper_problem():
    """The discrete problem of Section 3.2 (inviscid, [0,1]^2, 64 x 64, zero
    Dirichlet walls, u(x, 0) = (1 - cos 6 pi x)/2) solved row by row: every
    row's residual vanishes; the scheme is conservative, so each row's mass
    changes only by the upwind outflow through the walls,
    (M^n - M^{n-1})/dt = -max(u^n_{N-1}, 0)^2/2 + min(u^n_0, 0)^2/2; the
    solution keeps within the initial range [0, 1] (monotone upwind scheme)
    and its energy never grows."""
    n = 64
    dt = dx = 1.0 / n
    x = (np.arange(n) + 0.5) * dx
    u0 = inputs.burgers_paper_ic(x)
    assert u0.min() >= 0.0 and u0.max() <= 1.0
    u = o.burgers_implicit_solve(u0, n, dt, dx, nu=0.0)
    np.testing.assert_array_equal(u[0], u0)
    assert np.max(np.abs(o.burgers_residual(u, 0.0, dt, dx))) < 1e-11
    M = u.sum(axis=1) * dx
    out = 0.5 * np.maximum(u[1:, -1], 0.0) ** 2 - 0.5 * np.minimum(u[1:, 0], 0.0) ** 2
    np.testing.assert_allclose((M[1:] - M[:-1]) / dt, -out, rtol=0, atol=1e-11)
    assert u.min() >= -1e-12 and u.max() <= 1.0 + 1e-12
    E = np.sum(u**2, axis=1)
    assert np.all(np.diff(E) <= 1e-12)


def test_burgers_paper_points_on_rectangle_edges():
    """84 points on the edges of the rectangle, 21 per edge, corners once."""
    p = inputs.rectangle_points()
    assert p.shape == (84, 2)
    assert len({(round(a, 12), round(b, 12)) for a, b in p}) == 84
    (t0, t1), (x0, x1) = inputs.BURGERS_PAPER["rect"]
    on_t = np.isclose(p[:, 0], t0) | np.isclose(p[:, 0], t1)
    on_x = np.isclose(p[:, 1], x0) | np.isclose(p[:, 1], x1)
    assert np.all(on_t | on_x)
    assert np.all((p[:, 0] >= t0) & (p[:, 0] <= t1) & (p[:, 1] >= x0) & (p[:, 1] <= x1))


# --------------------------------------------------------------------------
# Heat with unknown conductivity (Section 3.4)
# --------------------------------------------------------------------------

def test_conductivity_interpolation_closed_form():
    rng = np.random.default_rng(7)
    q = rng.uniform(0.01, 0.03, 32)
    nodes = np.arange(32) / 31.0
    k, dk, _, _ = o.heat_conductivity(nodes[:-1] + 1e-15, q)
    np.testing.assert_allclose(k, q[:-1], atol=1e-15)
    # linear between nodes: midpoint is the mean, slope is the difference quotient
    mid = (nodes[:-1] + nodes[1:]) / 2
    k, dk, _, _ = o.heat_conductivity(mid, q)
    np.testing.assert_allclose(k, (q[:-1] + q[1:]) / 2, atol=1e-15)
    np.testing.assert_allclose(dk, 31 * (q[1:] - q[:-1]), rtol=1e-12)
    # constant extrapolation outside [0, 1]
    k, dk, _, _ = o.heat_conductivity(np.array([-0.5, 1.5, 1.0]), q)
    np.testing.assert_allclose(k, [q[0], q[-1], q[-1]], atol=1e-15)
    assert dk[0] == 0.0 and dk[1] == 0.0


def test_heat_constant_k_is_textbook_implicit_euler():
    rng = np.random.default_rng(8)
    nt, nx, kap = 12, 16, 0.017
    dt, dx = 1.0 / nt, 1.0 / nx
    u = rng.uniform(-0.2, 1.2, size=(nt, nx))
    init = rng.normal(size=nx)
    r = o.heat_residual(u, np.full(32, kap), dt, dx, init)
    ug = np.concatenate([-u[:, :1], u, -u[:, -1:]], axis=1)
    lap = (ug[1:, 2:] - 2 * u[1:] + ug[1:, :-2]) / dx**2
    np.testing.assert_allclose(r[1:], (u[1:] - u[:-1]) / dt - kap * lap, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(r[0], (u[0] - init) / dt, rtol=1e-14)


def test_heat_residual_consistent_with_pde():
    """Smooth k and a smooth field: residual -> u_t - (k(u) u_x)_x.

    Backward Euler in t (first order) plus central faces in x (second order):
    the error ratio per halving lies between 2 and 4 and never stalls."""
    kf = inputs.heat_k_true

    def dk(v):
        return kf(v) * (-40.0) * (v - 0.5)

    errs = []
    for n in (32, 64, 128, 256):
        dt, dx = 1.0 / n, 1.0 / n
        x = (np.arange(n) + 0.5) * dx
        t = (np.arange(n) + 0.5) * dt
        X, Tm = np.meshgrid(x, t)
        u = 0.8 * np.sin(math.pi * X) * np.exp(-Tm / 2)
        ut = -u / 2
        ux = 0.8 * math.pi * np.cos(math.pi * X) * np.exp(-Tm / 2)
        uxx = -(math.pi**2) * u
        r = o.heat_residual(u, None, dt, dx, u[0], kfun=kf)
        R = ut - dk(u) * ux**2 - kf(u) * uxx
        errs.append(np.max(np.abs(r[1:] - R[1:])))
        assert np.max(np.abs(r[0])) == 0.0
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.8 < q < 4.2 for q in rates), (errs, rates)


def test_heat_implicit_solve_zeroes_residual():
    n = 32
    dt, dx = 1.0 / n, 1.0 / n
    init = inputs.heat_ic(n)
    u = o.heat_implicit_solve(init, n, dt, dx, inputs.heat_k_true)
    r = o.heat_residual(u, None, dt, dx, init, kfun=inputs.heat_k_true)
    assert np.max(np.abs(r)) < 1e-9
    # maximum principle of the implicit scheme: temperature stays within the initial range
    assert u.max() <= init.max() + 1e-12 and u.min() >= -1e-12


def test_heat_known_conductivity_forward_problem_is_the_implicit_solve():
    """With the conductivity known (k_fixed: the forward problem that makes the
    reference record of Section 3.4) dL/dq is zero, an Adam step leaves q
    alone, and minimising the loss over the levels alone (library L-BFGS, no
    data) reaches the row-by-row implicit solve of the same discrete problem
    with k the nodes' piecewise-linear interpolant.  A dropped k_fixed (q
    moves) or a residual that is not the implicit scheme fails."""
    from scipy.optimize import minimize
    n, L = 16, 2
    q = inputs.heat_k_true(np.arange(32) / 31)
    init = inputs.heat_ic(n)
    p = o.Problem("heat", (n, n), L, w_res=1.0, w_data=0.0, w_reg=1e-3, aux=init, k_fixed=True)
    shapes = o.level_shapes((n, n), L)
    sizes = [int(np.prod(s)) for s in shapes]

    def unpack(z):
        return [z[a:a + m].reshape(s) for a, m, s in zip(np.cumsum([0] + sizes[:-1]), sizes, shapes)]

    def fg(z):
        t, g, gq = o.loss_grad_levels(p, unpack(z), q)
        assert not np.any(gq)
        return t["total"], np.concatenate([a.ravel() for a in g])
    r = minimize(fg, np.zeros(sum(sizes)), jac=True, method="L-BFGS-B",
                 options=dict(maxiter=5000, maxcor=30, ftol=0.0, gtol=1e-14))
    u = o.compose(unpack(r.x))
    ref = o.heat_implicit_solve(init, n, 1.0 / n, 1.0 / n, lambda uf: o.heat_conductivity(uf, q)[0])
    assert np.max(np.abs(u - ref)) < 1e-7, np.max(np.abs(u - ref))
    st = o.OracleState.zeros_like_levels(unpack(r.x), q=q)
    o.oracle_step(p, st, 1e-2)
    assert np.array_equal(st.q, q)
    free = o.Problem("heat", (n, n), L, w_res=1.0, w_data=0.0, w_reg=1e-3, aux=init)
    assert np.any(o.loss_grad_levels(free, unpack(r.x), q)[2])


def test_heat_node_step_unit():
    """k_scale only rescales the optimiser's steps on the nodes: Adam's first
    step from zero moments moves every node by lr * k_scale * sign(dL/dq)
    (to within eps), and the levels move exactly as with k_scale = 1."""
    n, L = 16, 2
    rng = np.random.default_rng(5)
    lv = [rng.uniform(0.0, 1.0, s) for s in o.level_shapes((n, n), L)]
    q = inputs.heat_k_true(np.arange(32) / 31) + 0.005
    cells = inputs.measurement_cells(n * n, 20, 1)
    kw = dict(w_res=1.0, w_data=1.0, w_reg=1e-3, aux=inputs.heat_ic(n), meas_cell=cells,
              meas_value=rng.uniform(0.0, 1.0, 20))
    lr, ks = 1e-2, 0.05
    gq = o.loss_grad_levels(o.Problem("heat", (n, n), L, **kw), lv, q)[2]
    out = []
    for k_scale in (1.0, ks):
        st = o.OracleState.zeros_like_levels(lv, q=q)
        o.oracle_step(o.Problem("heat", (n, n), L, k_scale=k_scale, **kw), st, lr)
        out.append(st)
    big = np.abs(gq) > 1e-6  # nodes far from the data have gradients near eps
    assert big.sum() >= 16
    np.testing.assert_allclose((out[1].q - q)[big], -lr * ks * np.sign(gq[big]), rtol=1e-5)
    np.testing.assert_allclose((out[0].q - q)[big], -lr * np.sign(gq[big]), rtol=1e-5)
    np.testing.assert_allclose(out[1].q - q, ks * (out[0].q - q), rtol=1e-9, atol=1e-18)
    for a, b in zip(out[0].levels, out[1].levels):
        assert np.array_equal(a, b)


def test_heat_regulariser_closed_forms():
    """Second difference of the conductivity nodes (Section 3.4 reading R7):
    zero for nodes on a line; for q_j = j^2 every second difference is 2, so
    the regulariser is 4 per interior node, 4 (K - 1) for K + 1 = 32 nodes,
    and its gradient 2 sum_i d2_i d(d2_i)/dq_j is (4, -4, 0, ..., 0, -4, 4).
    A first difference, a q[2:] - q[:-2] stencil or a dropped factor fails."""
    n = 32
    p = o.Problem("heat", (4, 8), 1, w_res=0.0, w_data=0.0, w_reg=0.25,
                  aux=np.zeros(8))
    u = np.zeros((4, 8))
    lin = 0.013 + 0.002 * np.arange(n)
    assert o.loss_terms(p, u, lin)["reg"] == pytest.approx(0.0, abs=1e-30)
    q = np.arange(n, dtype=float) ** 2
    assert o.loss_terms(p, u, q)["reg"] == 0.25 * 4.0 * (n - 2)
    gq = o.loss_grad_fine(p, u, q)[2]
    want = np.zeros(n)
    want[[0, 1, -2, -1]] = [4.0, -4.0, -4.0, 4.0]
    np.testing.assert_array_equal(gq, 0.25 * want)


# --------------------------------------------------------------------------
# Poisson (Section 3.1): exact discrete solution and second-order convergence
# --------------------------------------------------------------------------

def _u_ref(x):
    v = np.prod([5 * (1 - xi) * xi for xi in x], axis=0)
    return (v**5 / (1 + v**5)) ** 0.2


@pytest.mark.parametrize("layout", ["cell", "node"])
def test_poisson_laplacian_exact_on_biquadratics(layout):
    """u = x(1-x) y(1-y) vanishes on the walls of [0,1]^2 and is quadratic in
    each axis, so the three-point difference is exact along each axis, and
    so (cell layout) is the quadratic extrapolation through the zero wall value
    (Section 3.1) that supplies the ghost: the residual against
    f = -2 y(1-y) - 2 x(1-x) is zero to rounding in every cell, the wall rows
    included.  A linear ghost (-u_0) or a wrong extrapolation weight leaves
    O(1) residuals in the wall rows."""
    n = 16
    h = (1.0 / n, 1.0 / n)
    c = (np.arange(n) + 0.5) / n if layout == "cell" else np.arange(n + 1) / n
    Y, X = np.meshgrid(c, c, indexing="ij")
    u = X * (1 - X) * Y * (1 - Y)
    f = -2.0 * Y * (1 - Y) - 2.0 * X * (1 - X)
    r = o.poisson_residual(u, f, h, layout)
    np.testing.assert_allclose(r, 0.0, atol=1e-11)
    p = o.Problem("poisson", (n, n), 1, layout=layout, coef={"f": f})
    assert o.loss_terms(p, u)["total"] < 1e-22
    # a field that does not vanish on the walls: u = 1 in every cell.  Its
    # quadratic-extrapolation ghost is -2 + 1/3 = -5/3, so a wall cell's
    # residual has (-5/3 - 2 + 1)/h^2 = -8/(3 h^2) per wall it touches.
    if layout == "cell":
        one = np.ones((n, n))
        r1 = o.poisson_residual(one, np.zeros((n, n)), h, layout)
        walls = (np.arange(n) == 0)[:, None].astype(int) + (np.arange(n) == n - 1)[:, None]
        walls = walls + walls.T
        np.testing.assert_allclose(r1, -8.0 / 3.0 * walls * n * n, rtol=1e-13, atol=1e-9)


def _quadratic_minimiser(p, shape):
    """Minimiser of a quadratic loss from its exact gradient: H u = -g(0)
    (least squares: in the node layout the boundary nodes hold the Dirichlet
    value and do not enter the loss, so their rows of H vanish and the
    minimum-norm minimiser keeps them at 0)."""
    n = int(np.prod(shape))
    g0 = o.loss_grad_fine(p, np.zeros(shape))[1].reshape(-1)
    H = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        H[:, j] = o.loss_grad_fine(p, e.reshape(shape))[1].reshape(-1) - g0
    return np.linalg.lstsq(H, -g0, rcond=None)[0].reshape(shape)


def test_poisson_node_boundary_holds_the_dirichlet_value():
    """Section 3.1: in the node layout the Dirichlet value is imposed on the
    boundary nodes themselves: whatever the field holds there, the stencil
    reads 0, the boundary values do not change the loss and get no gradient;
    the residual lives at the (N - 1)^d interior nodes."""
    rng = np.random.default_rng(14)
    n = 8
    u = rng.normal(size=(n + 1, n + 1))
    f = rng.normal(size=(n + 1, n + 1))
    p = o.Problem("poisson", (n, n), 1, layout="node", coef={"f": f})
    v = u.copy()
    v[0, :] += 3.0
    v[:, -1] -= 1.5
    assert o.poisson_residual(u, f, (1 / n, 1 / n), "node").shape == (n - 1, n - 1)
    assert o.loss_terms(p, u)["total"] == o.loss_terms(p, v)["total"]
    g = o.loss_grad_fine(p, u)[1]
    edge = np.ones_like(g, dtype=bool)
    edge[1:-1, 1:-1] = False
    assert np.all(g[edge] == 0.0) and np.any(g[~edge] != 0.0)


@pytest.mark.parametrize("layout", ["cell", "node"])
def test_poisson_minimiser_converges_second_order(layout):
    """Manufactured u = sin(pi x) sin(pi y): the loss minimiser is O(h^2) accurate."""
    errs = []
    for n in (8, 16, 32):
        h = (1.0 / n, 1.0 / n)
        c = (np.arange(n) + 0.5) / n if layout == "cell" else np.arange(n + 1) / n
        X, Y = np.meshgrid(c, c, indexing="ij")
        ue = np.sin(math.pi * X) * np.sin(math.pi * Y)
        f = -2 * math.pi**2 * ue
        p = o.Problem("poisson", (n, n), 1, layout=layout, coef={"f": f})
        u = _quadratic_minimiser(p, ue.shape)
        g = o.loss_grad_fine(p, u)[1]
        assert np.max(np.abs(g)) < 1e-8
        errs.append(np.max(np.abs(u - ue)))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.3 < q < 4.7 for q in rates), (errs, rates)


# --------------------------------------------------------------------------
# Gradients: central finite differences through levels, stencils and data
# --------------------------------------------------------------------------

def _fd_check(loss_fn, params, grads, h=1e-6, rtol=2e-6):
    worst = 0.0
    scale = max(np.max(np.abs(g)) for g in grads)
    for a, g in zip(params, grads):
        flat = a.reshape(-1)
        gf = g.reshape(-1)
        for j in range(flat.size):
            old = flat[j]
            step = h * max(1.0, abs(old))
            flat[j] = old + step
            lp = loss_fn()
            flat[j] = old - step
            lm = loss_fn()
            flat[j] = old
            fd = (lp - lm) / (2 * step)
            worst = max(worst, abs(fd - gf[j]) / scale)
    assert worst < rtol, worst


def test_burgers_gradient_finite_differences():
    p = _burgers_problem((8, 16), 3, seed=9, nu=0.04, n_meas=12)
    lv = inputs.random_levels((8, 16), 3, 1, seed=9)[0]
    _, grads, _ = o.loss_grad_levels(p, lv)
    _fd_check(lambda: o.loss_terms(p, o.compose(lv))["total"], lv, grads)


def test_heat_gradient_finite_differences():
    nt, nx = 8, 16
    rng = np.random.default_rng(10)
    cells = inputs.measurement_cells(nt * nx, 10, 10)
    p = o.Problem("heat", (nt, nx), 3, w_res=1.0, w_data=2.0, w_reg=0.3,
                  meas_cell=cells, meas_value=rng.uniform(0, 1, 10), aux=inputs.heat_ic(nx))
    lv = inputs.random_levels((nt, nx), 3, 1, seed=10, fine_lo=-0.1, fine_hi=1.1,
                              coarse_scale=0.1)[0]
    q = rng.uniform(0.01, 0.03, 32)
    _, grads, gq = o.loss_grad_levels(p, lv, q)
    _fd_check(lambda: o.loss_terms(p, o.compose(lv), q)["total"], lv + [q], grads + [gq])


def test_poisson_gradient_finite_differences():
    rng = np.random.default_rng(11)
    for layout in ("cell", "node"):
        n = 8
        sh = (n, n) if layout == "cell" else (n + 1, n + 1)
        f = rng.normal(size=sh)
        p = o.Problem("poisson", (n, n), 3, layout=layout, coef={"f": f})
        lv = [rng.normal(size=s) for s in o.level_shapes((n, n), 3, layout)]
        _, grads, _ = o.loss_grad_levels(p, lv)
        _fd_check(lambda: o.loss_terms(p, o.compose(lv, layout))["total"], lv, grads)


# --------------------------------------------------------------------------
# Adam
# --------------------------------------------------------------------------

def test_adam_constant_gradient_closed_form():
    """Constant g: bias correction gives m_hat = g, v_hat = g^2 at every step,
    so x_t = x_0 - t lr g / (|g| + eps)."""
    rng = np.random.default_rng(12)
    g = rng.normal(size=50) * np.logspace(-9, 2, 50)
    x0 = rng.normal(size=50)
    x, m, v = x0.copy(), np.zeros(50), np.zeros(50)
    lr, eps = 5e-3, 1e-8
    for t in range(1, 8):
        x, m, v = o.adam_step(x, m, v, g, t, lr, eps=eps)
        np.testing.assert_allclose(x, x0 - t * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)


def test_adam_two_steps_by_hand():
    """Two steps with g = 1 then g = -2 (b1 = 0.9, b2 = 0.999, eps = 0)."""
    x, m, v = np.array([0.0]), np.array([0.0]), np.array([0.0])
    x, m, v = o.adam_step(x, m, v, np.array([1.0]), 1, 0.1, eps=0.0)
    assert abs(x[0] + 0.1) < 1e-15
    x, m, v = o.adam_step(x, m, v, np.array([-2.0]), 2, 0.1, eps=0.0)
    # m = 0.9*0.1 + 0.1*(-2) = -0.11, mhat = -0.11/0.19; v = 0.999*0.001 + 0.001*4
    mh = -0.11 / 0.19
    vh = (0.000999 + 0.004) / (1 - 0.999**2)
    assert abs(x[0] - (-0.1 - 0.1 * mh / math.sqrt(vh))) < 1e-14


# --------------------------------------------------------------------------
# Lid-driven cavity, steady Navier-Stokes (Section 3.3)
# --------------------------------------------------------------------------

def test_ns2d_fluid_at_rest_closed_form():
    """u = v = 0, p = c: only the lid shears the top row, -2/(Re h^2) in r_u."""
    n, Re, c = 12, 100.0, 0.7
    h = 1.0 / n
    z = np.zeros((n, n))
    ru, rv, rc, rg = o.ns2d_residuals(z, z, np.full((n, n), c), Re, h)
    np.testing.assert_allclose(ru[:-1], 0.0, atol=1e-12)
    np.testing.assert_allclose(ru[-1], -2.0 / (Re * h * h), rtol=1e-13)
    np.testing.assert_allclose(rv, 0.0, atol=1e-12)
    np.testing.assert_allclose(rc, 0.0, atol=1e-12)
    assert rg == c


def test_ns2d_checkerboard_pressure_rhie_chow_closed_form():
    """Fluid at rest with a checkerboard pressure p = c (-1)^(i+j).  The
    central pressure gradient cannot see it (interior r_u = r_v = 0), which is
    why the continuity residual of Section 3.3 uses Rhie-Chow face velocities:
    at an interior face U = -tau (p_E - p_P)/h (the cell gradients vanish), so
    each axis contributes 4 tau p / h^2 and r_c = 8 tau_f p / h with
    tau = tau_f h.  A flipped sign or another coefficient of the correction
    fails here, though both are invisible to the consistency orders."""
    n, Re, c, tf = 10, 100.0, 0.3, 0.7
    h = 1.0 / n
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    p = c * (-1.0) ** (ii + jj)
    z = np.zeros((n, n))
    ru, rv, rc, _ = o.ns2d_residuals(z, z, p, Re, h, tau_factor=tf, lid=0.0)
    inner = (slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(ru[inner], 0.0, atol=1e-12)
    np.testing.assert_allclose(rv[inner], 0.0, atol=1e-12)
    np.testing.assert_allclose(rc[inner], (8.0 * tf * p / h)[inner], rtol=1e-12)


def test_ns2d_interior_consistency_second_order():
    """Smooth fields: interior residuals -> (u^2)_x + (uv)_y + p_x - nu lap u,
    (uv)_x + (v^2)_y + p_y - nu lap v and u_x + v_y at second order."""
    import sympy as sp
    X, Y = sp.symbols("x y")
    uu = sp.sin(2 * X) * sp.cos(3 * Y) + 0.3
    vv = sp.cos(X + 0.5) * sp.sin(2 * Y) - 0.2
    pp = sp.exp(X * Y) * sp.cos(X)
    Re = 50.0
    nu = 1.0 / Re
    ex_u = sp.diff(uu * uu, X) + sp.diff(uu * vv, Y) + sp.diff(pp, X) - nu * (sp.diff(uu, X, 2) + sp.diff(uu, Y, 2))
    ex_v = sp.diff(uu * vv, X) + sp.diff(vv * vv, Y) + sp.diff(pp, Y) - nu * (sp.diff(vv, X, 2) + sp.diff(vv, Y, 2))
    ex_c = sp.diff(uu, X) + sp.diff(vv, Y)
    fs = [sp.lambdify((X, Y), e, "numpy") for e in (uu, vv, pp, ex_u, ex_v, ex_c)]
    errs = []
    for n in (32, 64, 128, 256):
        h = 1.0 / n
        c = (np.arange(n) + 0.5) * h
        Yg, Xg = np.meshgrid(c, c, indexing="ij")
        u, v, p = fs[0](Xg, Yg), fs[1](Xg, Yg), fs[2](Xg, Yg)
        ru, rv, rc, _ = o.ns2d_residuals(u, v, p, Re, h)
        k = max(3, n // 8)
        sl = (slice(k, -k), slice(k, -k))
        e = max(np.max(np.abs(ru - fs[3](Xg, Yg))[sl]), np.max(np.abs(rv - fs[4](Xg, Yg))[sl]),
                np.max(np.abs(rc - fs[5](Xg, Yg))[sl]))
        errs.append(e)
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.3 < q < 4.7 for q in rates), (errs, rates)


def test_ns2d_gradient_finite_differences():
    n, L = 8, 3
    rng = np.random.default_rng(21)
    cells = inputs.measurement_cells(n * n, 14, 21)
    fields = (np.arange(14) % 2).astype(np.int32)
    p = o.Problem("ns2d", (n, n), L, coef={"Re": 100.0, "tau": 1.0}, w_res=1.0, w_data=3.0,
                  meas_cell=cells, meas_field=fields, meas_value=rng.normal(size=14))
    lv = inputs.random_levels((n, n), L, 3, seed=21, coarse_scale=0.3)
    _, grads, _ = o.loss_grad_levels(p, lv)
    flat_params = [a for f in lv for a in f]
    flat_grads = [g for f in grads for g in f]
    _fd_check(lambda: o.loss_terms(p, [o.compose(f) for f in lv])["total"], flat_params, flat_grads)


# --------------------------------------------------------------------------
# Penalised Navier-Stokes in 3-D, body shape (Section 3.5)
# --------------------------------------------------------------------------

def _ns3d_h(sh):
    return (1.0 / sh[0], 1.0 / sh[1], 2.0 / sh[2])


def test_ns3d_uniform_inflow_is_a_solution_away_from_the_body():
    """u = (1,0,0), p = 0, no body: only lambda chi u remains (chi ~ 1e-13)."""
    sh = (6, 5, 10)
    one, z = np.ones(sh), np.zeros(sh)
    ch = np.full(sh, -25.0)
    ru, rv, rw, rc = o.ns3d_residuals(one, z, z, z, ch, 60.0, 0.4, 1.0, _ns3d_h(sh))
    chi = o.ns3d_chi(ch)
    np.testing.assert_allclose(ru, chi, atol=1e-12)
    for r in (rv, rw, rc):
        np.testing.assert_allclose(r, 0.0, atol=1e-10)


def test_ns3d_inside_the_body_only_penalisation_remains():
    """chi = 1 (chihat large): momentum residual = lambda u exactly."""
    rng = np.random.default_rng(30)
    sh = (4, 5, 6)
    u, v, w, p = [rng.normal(size=sh) for _ in range(4)]
    ch = np.full(sh, 60.0)
    ru, rv, rw, _ = o.ns3d_residuals(u, v, w, p, ch, 60.0, 0.4, 0.7, _ns3d_h(sh))
    np.testing.assert_allclose(ru, 0.7 * u, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(rv, 0.7 * v, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(rw, 0.7 * w, rtol=1e-12, atol=1e-12)


def test_ns3d_chi_shift_of_the_initial_guess():
    """Section 3.5 states that the initial guess chihat = 0 is the body
    fraction chi = 1/(1 + e^5) (almost no body), which fixes the transform as
    chi = 1/(1 + exp(-(chihat - 5))); so chihat = 5 is chi = 1/2.  Uniform
    inflow u = (1, 0, 0), p = 0 solves the flow part exactly (inlet ghost
    2 - 1 = 1), so the x-momentum residual is the penalisation lambda chi u
    alone: lambda/(1 + e^5) at chihat = 0 and lambda/2 at chihat = 5.  A
    dropped or negated shift fails."""
    assert o.ns3d_chi(np.array(0.0)) == pytest.approx(1.0 / (1.0 + math.exp(5.0)), rel=1e-15)
    assert o.ns3d_chi(np.array(5.0)) == 0.5
    sh = (4, 5, 8)
    one, z = np.ones(sh), np.zeros(sh)
    lam = 0.7
    for chihat, chi in ((0.0, 1.0 / (1.0 + math.exp(5.0))), (5.0, 0.5)):
        ru, rv, rw, rc = o.ns3d_residuals(one, z, z, z, np.full(sh, chihat), 60.0, 0.4, lam,
                                          _ns3d_h(sh))
        np.testing.assert_allclose(ru, lam * chi, rtol=1e-12)
        for r in (rv, rw, rc):
            np.testing.assert_allclose(r, 0.0, atol=1e-10)


def test_ns3d_checkerboard_pressure_rhie_chow_closed_form():
    """Fluid at rest, checkerboard p = c (-1)^(i+j+k), no body: the central
    pressure gradient vanishes in the interior and the Rhie-Chow face
    velocity along axis a is -tau_f (p_+ - p_P), so r_c = 4 tau_f p sum_a 1/h_a
    (the 3-D form of the cavity's correction, Section 3.5 following 3.3)."""
    sh = (8, 8, 12)
    hz, hy, hx = _ns3d_h(sh)
    c, tf = 0.4, 0.6
    kk, jj, ii = np.meshgrid(*(np.arange(s) for s in sh), indexing="ij")
    p = c * (-1.0) ** (ii + jj + kk)
    z = np.zeros(sh)
    ru, rv, rw, rc = o.ns3d_residuals(z, z, z, p, np.full(sh, -40.0), 60.0, 0.4, 1.0,
                                      (hz, hy, hx), tau_factor=tf)
    inner = (slice(2, -2),) * 3
    for r in (ru, rv, rw):
        np.testing.assert_allclose(r[inner], 0.0, atol=1e-10)
    want = 4.0 * tf * p * (1.0 / hx + 1.0 / hy + 1.0 / hz)
    np.testing.assert_allclose(rc[inner], want[inner], rtol=1e-12)


def test_ns3d_mass_balance():
    """sum r_c dV = (outlet flux - inlet flux) over the x ends (walls carry none)."""
    rng = np.random.default_rng(31)
    sh = (5, 6, 8)
    hz, hy, hx = _ns3d_h(sh)
    f = [rng.normal(size=sh) for _ in range(5)]
    rc = o.ns3d_residuals(*f, 60.0, 0.4, 1.0, (hz, hy, hx))[3]
    lhs = rc.sum() * hx * hy * hz
    rhs = hy * hz * (f[0][:, :, -1].sum() - sh[0] * sh[1] * 1.0)
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(rhs))


def test_ns3d_interior_consistency_second_order():
    """Smooth fields, no body: interior residuals -> conservative NS with D/Re."""
    import sympy as sp
    X, Y, Z = sp.symbols("x y z")
    uu = 1 + 0.3 * sp.sin(X) * sp.cos(2 * Y) * sp.cos(Z)
    vv = 0.2 * sp.cos(X + Y) * sp.sin(Z + 0.3)
    ww = -0.1 * sp.sin(2 * Z) * sp.cos(X - Y)
    pp = sp.exp(0.3 * X) * sp.sin(Y + Z)
    nu = 0.4 / 60.0
    fields = (uu, vv, ww)
    lapl = lambda f: sp.diff(f, X, 2) + sp.diff(f, Y, 2) + sp.diff(f, Z, 2)  # noqa: E731
    ex = []
    for f, g in zip(fields, (sp.diff(pp, X), sp.diff(pp, Y), sp.diff(pp, Z))):
        ex.append(sp.diff(uu * f, X) + sp.diff(vv * f, Y) + sp.diff(ww * f, Z) + g - nu * lapl(f))
    ex.append(sp.diff(uu, X) + sp.diff(vv, Y) + sp.diff(ww, Z))
    fn = [sp.lambdify((X, Y, Z), e, "numpy") for e in (uu, vv, ww, pp)]
    en = [sp.lambdify((X, Y, Z), e, "numpy") for e in ex]
    errs = []
    for n in (16, 32, 64):
        sh = (n, n, 2 * n)  # equal spacing in all axes
        hz, hy, hx = 1.0 / n, 1.0 / n, 2.0 / (2 * n)
        zc = (np.arange(n) + 0.5) * hz
        yc = (np.arange(n) + 0.5) * hy
        xc = (np.arange(2 * n) + 0.5) * hx
        Zg, Yg, Xg = np.meshgrid(zc, yc, xc, indexing="ij")
        f = [g(Xg, Yg, Zg) * np.ones(sh) for g in fn] + [np.full(sh, -40.0)]
        rs = o.ns3d_residuals(*f, 60.0, 0.4, 1.0, (hz, hy, hx))
        k = 3
        sl = (slice(k, -k),) * 3
        errs.append(max(np.max(np.abs(r - e(Xg, Yg, Zg))[sl]) for r, e in zip(rs, en)))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.2 < q < 4.8 for q in rates), (errs, rates)


def test_ns3d_gradient_finite_differences():
    sh, L = (4, 4, 8), 2
    rng = np.random.default_rng(32)
    n = int(np.prod(sh))
    cells = inputs.measurement_cells(n, 12, 32)
    mf = (np.arange(12) % 3).astype(np.int32)
    p = o.Problem("ns3d", sh, L, coef={"Re": 60.0, "D": 0.4, "lam": 1.0, "tau": 1.0},
                  w_res=1.0, w_data=2.0, meas_cell=cells, meas_field=mf,
                  meas_value=rng.normal(size=12))
    lv = inputs.random_levels(sh, L, 5, seed=32, coarse_scale=0.3)
    _, grads, _ = o.loss_grad_levels(p, lv)
    flat_params = [a for f in lv for a in f]
    flat_grads = [g for f in grads for g in f]
    _fd_check(lambda: o.loss_terms(p, [o.compose(f) for f in lv])["total"], flat_params, flat_grads)
