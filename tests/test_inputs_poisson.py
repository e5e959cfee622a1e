"""The Poisson reference recipe: the closed-form right-hand side equals a
fine finite-difference Laplacian of the reference solution (CPU)."""
import numpy as np

from paper_2303_04679_gb300 import inputs


def test_poisson_rhs_is_laplacian_of_reference():
    n = 32
    w = inputs.poisson_workload(n)

    def u(x, y):
        v = 25.0 * (1 - x) * x * (1 - y) * y
        return (v ** 5 / (1 + v ** 5)) ** 0.2

    c = (np.arange(n) + 0.5) / n
    y, x = np.meshgrid(c, c, indexing="ij")
    h = 1e-3
    lap = (u(x + h, y) + u(x - h, y) + u(x, y + h) + u(x, y - h) - 4 * u(x, y)) / h ** 2
    assert np.allclose(w["u_ref"], u(x, y), rtol=1e-13, atol=0)
    assert np.max(np.abs(lap - w["f"])) <= 1e-4 * np.max(np.abs(w["f"]))


def test_poisson_rhs_in_one_and_three_dimensions_and_at_nodes():
    """The same check for d = 1 and 3 and the node layout (values at j / n)."""
    h = 1e-3

    def u(*xs):
        v = np.prod([5.0 * (1 - x) * x for x in xs], axis=0)
        return (v ** 5 / (1 + v ** 5)) ** 0.2
    for d, layout in ((1, "cell"), (1, "node"), (3, "cell"), (3, "node"), (2, "node")):
        n = 16
        w = inputs.poisson_workload(n, d, layout)
        c = np.arange(n + 1) / n if layout == "node" else (np.arange(n) + 0.5) / n
        X = np.meshgrid(*([c] * d), indexing="ij")
        lap = -2 * d * u(*X)
        for i in range(d):
            for s in (-h, h):
                Y = list(X)
                Y[i] = X[i] + s
                lap = lap + u(*Y)
        lap /= h ** 2
        assert w["u_ref"].shape == X[0].shape
        assert np.allclose(w["u_ref"], u(*X), rtol=1e-13, atol=0)
        inner = tuple(slice(1, -1) for _ in range(d))  # away from the v = 0 kink of g at the walls
        assert np.max(np.abs(lap - w["f"])[inner]) <= 1e-4 * np.max(np.abs(w["f"])), (d, layout)
