"""Batched instances of uneven size, the persistent launch and the tile autotuner."""
import math
import os

import numpy as np
import pytest

from _cases import Case, check_loss_grad
from paper_2303_04679_gb300 import inputs


def test_batch_workload_recipe():
    b = inputs.burgers_batch(64, base_seed=3)
    sizes = {64, 128, 256, 512}
    for d in b:
        nt, nx = d["shape"]
        assert nt in sizes and nx in sizes
        assert d["n_levels"] == int(math.log2(min(nt, nx) // 8)) + 1
        assert min(nt, nx) >> (d["n_levels"] - 1) == 8
        assert 1e-3 <= d["nu"] <= 1e-1
        assert len(d["meas_cell"]) == max(1, round(0.005 * nt * nx))
        assert len(np.unique(d["meas_cell"])) == len(d["meas_cell"])
    # deterministic per instance index
    again = inputs.burgers_batch(64, base_seed=3)
    assert all(np.array_equal(a["meas_cell"], c["meas_cell"]) for a, c in zip(b, again))
    assert len({d["shape"] for d in b}) > 6


def test_autotune_picks_fastest_and_caches(tmp_path):
    from paper_2303_04679_gb300 import autotune, modil
    descs = [modil.Desc("burgers", (64, 128), 3, coef=(0.01,))]
    calls = []

    def fake(ds, tile, pers):
        calls.append((tuple(tile), pers))
        return 1.0 + 0.1 * tile[0] / tile[1] - (0.05 if pers else 0.0)

    cache = str(tmp_path / "tune.json")
    best = autotune.autotune(descs, measure=fake, cache_path=cache)
    assert best[0] == (8, 128) and best[1] is True
    assert len(calls) == 2 * len(autotune.ST_TILES) + 1   # the streaming strip: one variant
    calls.clear()
    again = autotune.autotune(descs, measure=fake, cache_path=cache)
    assert again[:2] == best[:2] and not calls           # served from the cache
    other = [modil.Desc("burgers", (64, 256), 3, coef=(0.01,))]
    assert autotune.signature(other) != autotune.signature(descs)


def _batch_cases():
    shapes = [((64, 512), 4, 0.01), ((512, 64), 4, 0.002), ((128, 128), 5, 0.05),
              ((256, 64), 4, 0.02), ((64, 64), 4, 0.1)]
    return [Case("burgers", s, L, "f32", seed=60 + i, n_meas=max(1, s[0] * s[1] // 200), nu=nu)
            for i, (s, L, nu) in enumerate(shapes)]


@pytest.fixture(scope="module")
def modil():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import modil as m
    return m


@pytest.mark.gpu
@pytest.mark.parametrize("persistent", [False, True])
def test_uneven_batch_matches_oracle(modil, persistent):
    cases = _batch_cases()
    with modil.Problem([c.desc() for c in cases]) as p:
        if persistent:
            p.set_persistent(True)
        for i, c in enumerate(cases):
            c.load(p, instance=i)
        for i, c in enumerate(cases):
            check_loss_grad(c, p, 1e-5, instance=i)


@pytest.mark.gpu
def test_persistent_launch_is_bit_identical(modil):
    cases = _batch_cases()
    out = []
    for pers in (False, True):
        with modil.Problem([c.desc() for c in cases]) as p:
            if pers:
                p.set_persistent(True)
            for i, c in enumerate(cases):
                c.load(p, instance=i)
            t = p.step(6)
            lv = [p.read_levels(instance=i) for i in range(len(cases))]
            out.append((t, lv))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


@pytest.mark.gpu
def test_batched_equals_single_instance_runs(modil):
    """A batch steps every instance exactly as a problem of its own does."""
    cases = _batch_cases()[:3]
    with modil.Problem([c.desc() for c in cases]) as p:
        for i, c in enumerate(cases):
            c.load(p, instance=i)
        tb = p.step(5)
        lb = [p.read_levels(instance=i) for i in range(len(cases))]
    for i, c in enumerate(cases):
        with modil.Problem(c.desc()) as q:
            c.load(q)
            ts = q.step(5)
            np.testing.assert_array_equal(ts[0], tb[i])
            for x, y in zip(q.read_levels(), lb[i]):
                np.testing.assert_array_equal(x, y)


@pytest.mark.gpu
def test_autotune_real_timing(modil, tmp_path):
    from paper_2303_04679_gb300 import autotune
    descs = [c.desc() for c in _batch_cases()[:2]]
    tile, pers, ms = autotune.autotune(descs, cache_path=str(tmp_path / "t.json"))
    assert tuple(tile) in autotune.ST_TILES and ms > 0


@pytest.mark.gpu
def test_small_problem_created_later_does_not_break_a_larger_one(modil):
    """Kernel shared-memory limits are process-wide: creating a smaller
    problem after a larger one must not lower the larger one's limit."""
    big = Case("heat", (512, 512), 7, "f32", seed=70, n_meas=500)
    small = Case("heat", (32, 32), 2, "f32", seed=71, n_meas=10)
    with modil.Problem(big.desc()) as p, modil.Problem(small.desc()) as q:
        big.load(p)
        small.load(q)
        q.step(2)
        p.step(2)
        assert np.isfinite(p.eval_grad()).all()
