"""Pins of the L-BFGS oracle (CPU): the two-loop recursion against the dense
BFGS inverse update it stands for, convergence to the closed-form minimiser of
a quadratic, the Rosenbrock valley, and monotone descent on a small mODIL
problem."""
import numpy as np

import oracle as o
from oracle import lbfgs_oracle as lb


def _pairs(n, k, rng):
    B = rng.standard_normal((n, n))
    B = B @ B.T + n * np.eye(n)  # SPD: every pair has s.y > 0
    out = []
    for _ in range(k):
        s = rng.standard_normal(n)
        y = B @ s
        out.append((s, y, 1.0 / float(s @ y)))
    return out


def test_two_loop_equals_dense_inverse_update():
    rng = np.random.default_rng(3)
    for n, k in ((7, 4), (5, 1), (9, 9)):
        pairs = _pairs(n, k, rng)
        g = rng.standard_normal(n)
        H = lb.explicit_inverse_hessian(pairs, n)
        d = lb.two_loop(g, pairs)
        assert np.allclose(d, -H @ g, rtol=1e-12, atol=1e-12), (n, k)


def test_no_pairs_is_steepest_descent():
    g = np.array([1.0, -2.0, 0.5])
    assert np.array_equal(lb.two_loop(g, []), -g)


def test_quadratic_reaches_closed_form_minimiser():
    rng = np.random.default_rng(4)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1.0, 100.0, n)) @ Q.T
    b = rng.standard_normal(n)
    xs = np.linalg.solve(A, b)
    f = lambda x: 0.5 * x @ A @ x - b @ x  # noqa: E731
    fg = lambda x: (f(x), A @ x - b)  # noqa: E731
    x, losses, done = lb.lbfgs(fg, f, np.zeros(n), 10, 300)
    assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs)
    assert all(b2 <= a2 for a2, b2 in zip(losses, losses[1:]))


def test_rosenbrock_valley():
    def f(x):
        return (1 - x[0]) ** 2 + 100 * (x[1] - x[0] ** 2) ** 2

    def fg(x):
        g = np.array([-2 * (1 - x[0]) - 400 * x[0] * (x[1] - x[0] ** 2), 200 * (x[1] - x[0] ** 2)])
        return f(x), g

    x, losses, done = lb.lbfgs(fg, f, np.array([-1.2, 1.0]), 5, 1000)
    assert np.max(np.abs(x - 1.0)) <= 1e-4, (x, done)


def test_monotone_descent_on_burgers_levels():
    from paper_2303_04679_gb300 import inputs
    shape, L = (16, 16), 3
    rng = np.random.default_rng(5)
    cells = inputs.measurement_cells(256, 30, 5)
    p = o.Problem("burgers", shape, L, coef={"nu": 0.05}, meas_cell=cells,
                  meas_value=rng.uniform(-0.5, 0.5, 30))
    shapes = o.level_shapes(shape, L)
    sizes = [int(np.prod(s)) for s in shapes]

    def unflat(x):
        out, k = [], 0
        for s, n in zip(shapes, sizes):
            out.append(x[k:k + n].reshape(s))
            k += n
        return out

    def f(x):
        return o.loss_terms(p, o.compose(unflat(x)))["total"]

    def fg(x):
        t, g, _ = o.loss_grad_levels(p, unflat(x))
        return t["total"], np.concatenate([a.ravel() for a in g])

    x0 = rng.uniform(-0.5, 0.5, sum(sizes))
    x, losses, done = lb.lbfgs(fg, f, x0, 5, 15)
    assert done == 15
    assert all(b2 < a2 for a2, b2 in zip(losses, losses[1:]))
