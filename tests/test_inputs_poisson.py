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
