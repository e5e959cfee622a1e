"""The warp-streaming Burgers kernel (32-row x 60-column strips, one warp
each, two columns per lane; the default for Burgers problems and batches of at least 608 strips
without off-grid points, requested here with tile (32, 60)) against the
FP64 oracle on grids whose strips are ragged in both directions, on one-row
and one-column coarse levels and single-level problems; against the tile
kernel on the same problem; Adam trajectories in FP64; a batch of uneven
instances equal bit for bit to the same instances stepped alone."""
import numpy as np
import pytest

import oracle as o
from _cases import Case, check_loss_grad, rel

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-11


@pytest.fixture(scope="module")
def modil():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import modil as m
    return m


# odd widths (40 x 33, 45 x 61) take the element-by-element copies
SHAPES = [((72, 100), 3), ((96, 56), 4), ((2, 64), 2), ((64, 2), 2), ((16, 40), 1), ((40, 30), 2),
          ((256, 512), 6), ((40, 33), 1), ((45, 61), 1), ((70, 122), 2)]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape,L", SHAPES)
def test_stream_loss_grad(modil, shape, L, dtype):
    c = Case("burgers", shape, L, dtype, seed=70, n_meas=max(3, shape[0] * shape[1] // 40), nu=0.02,
             duplicate=2, tile=(32, 60))
    with modil.Problem(c.desc()) as p:
        labels = p.profile_labels()
        want = (["compose_L2"] if L >= 4 else []) + (["compose_L1"] if L >= 3 else []) + ["fine"]
        assert labels[:len(want)] == want
        c.load(p)
        check_loss_grad(c, p, TOL64 if dtype == "f64" else TOL32)
        u = p.read_field()
        np.testing.assert_allclose(u, o.compose(c.levels), rtol=0,
                                   atol=(1e-14 if dtype == "f64" else 2e-6) * np.max(np.abs(u)))


def test_stream_matches_tile_kernel(modil):
    c = Case("burgers", (96, 192), 4, "f32", seed=71, n_meas=400, nu=0.02)
    kw = dict(c.desc_kw)
    out = []
    for tile in ((32, 60), (16, 32)):
        kw["tile"] = tile
        with modil.Problem(modil.Desc(**kw)) as p:
            c.load(p)
            t = p.eval_grad()[0].copy()
            out.append((t, p.read_grads()))
    assert abs(out[0][0][0] - out[1][0][0]) <= 2e-6 * out[1][0][0]
    for a, b in zip(out[0][1], out[1][1]):
        assert rel(a, b) <= 2e-6


def test_stream_adam_f64_matches_oracle(modil):
    c = Case("burgers", (72, 100), 3, "f64", seed=72, n_meas=150, lr=5e-3, nu=0.01, tile=(32, 60))
    st = o.OracleState.zeros_like_levels(c.levels)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        for _ in range(4):
            ref = o.oracle_step(c.oracle, st, c.lr)
            t = p.step(1)[0]
            assert abs(t[0] - ref["total"]) <= 1e-11 * ref["total"]
        for lvl in range(c.L):
            a, r = p.read_level(lvl), st.levels[lvl]
            assert np.max(np.abs(a - r)) <= 1e-12 * max(1.0, np.max(np.abs(r))), lvl


def test_stream_batch_equals_single_bitwise(modil):
    # the odd-sized first instance puts the next ones at odd offsets (element-
    # by-element copies in the batch, paired accesses alone)
    specs = [((33, 33), 1, 0.05), ((64, 512), 4, 0.01), ((512, 64), 4, 0.002), ((128, 128), 5, 0.05),
             ((256, 64), 4, 0.02), ((64, 64), 4, 0.1), ((72, 100), 3, 0.03)]
    cases = [Case("burgers", s, L, "f32", seed=80 + i, n_meas=max(1, s[0] * s[1] // 200), nu=nu,
                  tile=(32, 60)) for i, (s, L, nu) in enumerate(specs)]
    with modil.Problem([c.desc() for c in cases]) as p:
        for i, c in enumerate(cases):
            c.load(p, instance=i)
        tb = p.step(4)
        lb = [[p.read_level(l, instance=i) for l in range(c.L)] for i, c in enumerate(cases)]
    for i, c in enumerate(cases):
        with modil.Problem(c.desc()) as q:
            c.load(q)
            ts = q.step(4)[0]
            np.testing.assert_array_equal(tb[i], ts)
            for lvl in range(c.L):
                np.testing.assert_array_equal(q.read_level(lvl), lb[i][lvl])
