"""Pins of the off-grid measurement oracle (CPU): exact at cell centres,
exact for fields linear along every axis between the outermost centres,
clamped beyond them, weights forming a partition of unity, and a gradient
that matches finite differences of the data term."""
import numpy as np

from oracle import offgrid_oracle as og


def _centres(n, length):
    return (np.arange(n) + 0.5) * length / n


def test_cell_centres_return_cell_values():
    rng = np.random.default_rng(7)
    shape, lengths = (6, 9), (1.0, 2.0)
    u = rng.standard_normal(shape)
    yc, xc = _centres(6, 1.0), _centres(9, 2.0)
    pts = np.array([(y, x) for y in yc for x in xc])
    idx, w = og.sample_weights(pts, shape, lengths)
    assert np.allclose(og.sample(u, idx, w), u.reshape(-1), rtol=0, atol=1e-14)


def test_linear_fields_are_reproduced_inside_the_centres():
    rng = np.random.default_rng(8)
    for shape, lengths in (((7, 5), (1.0, 1.0)), ((4, 6, 8), (1.0, 1.0, 2.0))):
        d = len(shape)
        coef = rng.standard_normal(d + 1)
        grids = np.meshgrid(*[_centres(n, L) for n, L in zip(shape, lengths)], indexing="ij")
        u = coef[0] + sum(c * g for c, g in zip(coef[1:], grids))
        lo = np.array([L / n / 2 for n, L in zip(shape, lengths)])
        hi = np.array([L - L / n / 2 for n, L in zip(shape, lengths)])
        pts = lo + rng.uniform(0, 1, (200, d)) * (hi - lo)
        idx, w = og.sample_weights(pts, shape, lengths)
        exact = coef[0] + pts @ coef[1:]
        assert np.allclose(og.sample(u, idx, w), exact, rtol=0, atol=1e-12)
        assert np.all(w >= 0) and np.allclose(w.sum(axis=1), 1.0)


def test_points_beyond_the_outermost_centres_are_clamped():
    shape, lengths = (4, 4), (1.0, 1.0)
    u = np.arange(16.0).reshape(shape)
    idx, w = og.sample_weights([(0.0, 0.0), (1.0, 1.0), (0.05, 0.5)], shape, lengths)
    s = og.sample(u, idx, w)
    assert s[0] == u[0, 0] and s[1] == u[3, 3]
    assert np.isclose(s[2], 0.5 * (u[0, 1] + u[0, 2]))  # y clamped to row 0, x halfway


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(9)
    shape, lengths = (5, 7), (1.0, 2.0)
    u = rng.standard_normal(shape)
    pts = rng.uniform([0, 0], [1, 2], (30, 2))
    vals = rng.standard_normal(30)
    idx, w = og.sample_weights(pts, shape, lengths)
    _, g = og.data_term(u, idx, w, vals, w_data=1.7)
    d = rng.standard_normal(shape)
    eps = 1e-6
    fd = (og.data_term(u + eps * d, idx, w, vals, 1.7)[0] - og.data_term(u - eps * d, idx, w, vals, 1.7)[0]) / (2 * eps)
    assert abs(fd - float(np.sum(g * d))) <= 1e-8 * max(1.0, abs(fd))


def test_point_at_a_cell_centre_is_an_on_grid_measurement():
    """One data term over cells and points: a point at the centre of cell c
    contributes exactly what a measurement of cell c does."""
    import oracle as o
    from paper_2303_04679_gb300 import inputs
    shape, L = (16, 32), 3
    rng = np.random.default_rng(10)
    levels = inputs.random_levels(shape, L, 1, 10, -1.0, 1.0, 0.5)[0]
    cells = np.array([5, 77, 300, 511], dtype=np.int32)
    vals = rng.uniform(-0.5, 0.5, 4)
    y, x = cells // 32, cells % 32
    pts = np.stack([(y + 0.5) / 16, -1.0 + (x + 0.5) * 2.0 / 32], axis=1)  # Burgers: x in [-1, 1]
    on = o.Problem("burgers", shape, L, coef={"nu": 0.02}, meas_cell=cells, meas_value=vals)
    off = o.Problem("burgers", shape, L, coef={"nu": 0.02}, meas_points=pts, point_value=vals)
    t1, g1, _ = o.loss_grad_levels(on, levels)
    t2, g2, _ = o.loss_grad_levels(off, levels)
    assert np.isclose(t1["data"], t2["data"], rtol=1e-13)
    for a, b in zip(g1, g2):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def test_offgrid_level_gradient_matches_finite_differences():
    import oracle as o
    from paper_2303_04679_gb300 import inputs
    shape, L = (16, 16), 3
    rng = np.random.default_rng(11)
    levels = inputs.random_levels(shape, L, 1, 11, -1.0, 1.0, 0.5)[0]
    f = rng.standard_normal(shape)
    pts = rng.uniform(0, 1, (25, 2))
    p = o.Problem("poisson", shape, L, coef={"f": f}, meas_cell=np.array([3, 40], np.int32),
                  meas_value=np.array([0.1, -0.2]), meas_points=pts, point_value=rng.uniform(-1, 1, 25))
    _, grads, _ = o.loss_grad_levels(p, levels)
    d = [rng.standard_normal(a.shape) for a in levels]
    eps = 1e-6

    def loss(s):
        return o.loss_terms(p, o.compose([a + s * b for a, b in zip(levels, d)]))["total"]
    fd = (loss(eps) - loss(-eps)) / (2 * eps)
    an = sum(float(np.sum(g * b)) for g, b in zip(grads, d))
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


def test_multi_field_point_at_a_centre_is_a_cell_measurement_of_that_field():
    """Velocity samples at points (Sections 3.3, 3.5): a point at the centre
    of cell c measuring field f contributes exactly what a measurement of
    (c, f) does, in 2-D (cavity, bilinear) and 3-D (body, trilinear) -- the
    field routing and the corner weights at a centre."""
    import oracle as o
    from paper_2303_04679_gb300 import inputs
    rng = np.random.default_rng(12)
    for pde, shape, L, coef, nf in (("ns2d", (8, 8), 2, {"Re": 100.0, "tau": 1.0}, 3),
                                    ("ns3d", (4, 4, 8), 2, {"Re": 60.0, "D": 0.4, "lam": 1.0, "tau": 1.0}, 5)):
        levels = inputs.random_levels(shape, L, nf, 12, -0.5, 0.5, 0.2)
        n = int(np.prod(shape))
        cells = rng.choice(n, 6, replace=False).astype(np.int32)
        fields = np.array([0, 1, 2, 0, 1, 2], np.int32)
        vals = rng.normal(size=6)
        lengths = (1.0, 1.0) if pde == "ns2d" else (1.0, 1.0, 2.0)
        idx = np.array(np.unravel_index(cells, shape)).T
        pts = (idx + 0.5) * np.array(lengths) / np.array(shape)
        on = o.Problem(pde, shape, L, coef=coef, meas_cell=cells, meas_field=fields, meas_value=vals)
        off = o.Problem(pde, shape, L, coef=coef, meas_points=pts, point_value=vals, point_field=fields)
        t1, g1, _ = o.loss_grad_levels(on, levels)
        t2, g2, _ = o.loss_grad_levels(off, levels)
        assert np.isclose(t1["data"], t2["data"], rtol=1e-13)
        for f in range(nf):
            for a, b in zip(g1[f], g2[f]):
                assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def test_multi_field_points_gradient_matches_finite_differences():
    import oracle as o
    from paper_2303_04679_gb300 import inputs
    rng = np.random.default_rng(13)
    for pde, shape, L, coef, nf, lengths in (
            ("ns2d", (8, 8), 2, {"Re": 100.0, "tau": 1.0}, 3, (1.0, 1.0)),
            ("ns3d", (4, 4, 8), 2, {"Re": 60.0, "D": 0.4, "lam": 1.0, "tau": 1.0}, 5, (1.0, 1.0, 2.0))):
        levels = inputs.random_levels(shape, L, nf, 13, -0.5, 0.5, 0.2)
        pts = rng.uniform(0, 1, (9, len(shape))) * np.array(lengths)
        p = o.Problem(pde, shape, L, coef=coef, w_data=50.0, meas_points=pts,
                      point_value=rng.normal(size=9), point_field=rng.integers(0, nf, 9).astype(np.int32))
        _, grads, _ = o.loss_grad_levels(p, levels)
        d = [[rng.standard_normal(a.shape) for a in lv] for lv in levels]
        eps = 1e-6

        def loss(s):
            return o.loss_terms(p, [o.compose([a + s * b for a, b in zip(lv, dv)])
                                    for lv, dv in zip(levels, d)])["total"]
        fd = (loss(eps) - loss(-eps)) / (2 * eps)
        an = sum(float(np.sum(g * b)) for gf, df in zip(grads, d) for g, b in zip(gf, df))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (pde, fd, an)
