"""Poisson equation (Section 3.1, cell layout, 2-D) on the GPU against the FP64
oracle: loss terms and every level gradient on grids spanning several tiles
with ragged edges and 2-cell coarse levels, Adam trajectories and L-BFGS
iterates in FP64, and the convergence of both optimisers on the paper's
reference solution with more levels."""
import numpy as np
import pytest

import oracle as o
from oracle import lbfgs_oracle as lb
from paper_2303_04679_gb300 import inputs

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


def _case(modil, shape, L, dtype, seed, n_meas=60, tile=(0, 0)):
    rng = np.random.default_rng(seed)
    npd = np.float64 if dtype == "f64" else np.float32
    rnd = lambda a: np.asarray(a, np.float64).astype(npd).astype(np.float64)  # noqa: E731
    f = rnd(rng.standard_normal(shape) * 20.0)
    levels = [rnd(a) for a in inputs.random_levels(shape, L, 1, seed, -1.0, 1.0, 0.5)[0]]
    n = int(np.prod(shape))
    cells = inputs.measurement_cells(n, min(n_meas, n), seed)
    vals = rnd(rng.uniform(-0.5, 0.5, len(cells)))
    orc = o.Problem("poisson", shape, L, coef={"f": f}, meas_cell=cells, meas_value=vals)
    desc = modil.Desc("poisson", shape, L, dtype, aux=f.ravel(), meas_cell=cells, meas_value=vals,
                      lr=5e-3, tile=tile)
    return orc, desc, levels


def _check(p, orc, levels, tol):
    terms, grads, _ = o.loss_grad_levels(orc, levels)
    t = p.eval_grad()[0]
    for j, name in enumerate(("total", "res", "data")):
        assert abs(t[j] - terms[name]) <= tol * abs(terms[name]), (name, t[j], terms[name])
    for lvl, gr in enumerate(grads):
        g = p.read_grad(lvl).astype(np.float64)
        assert np.linalg.norm(g - gr) <= tol * np.linalg.norm(gr), lvl
        assert np.max(np.abs(g - gr)) <= 10 * tol * np.max(np.abs(gr)), lvl


@pytest.mark.parametrize("shape,L,tile", [((48, 96), 3, (0, 0)), ((40, 72), 3, (16, 32)),
                                          ((32, 32), 5, (32, 32)), ((2, 8), 2, (8, 64))])
def test_poisson_f32_loss_grad(modil, shape, L, tile):
    orc, desc, levels = _case(modil, shape, L, "f32", seed=50, tile=tile)
    with modil.Problem(desc) as p:
        p.write_levels(levels)
        _check(p, orc, levels, TOL32)


def test_poisson_f64_loss_grad(modil):
    orc, desc, levels = _case(modil, (64, 64), 4, "f64", seed=51)
    with modil.Problem(desc) as p:
        p.write_levels(levels)
        _check(p, orc, levels, TOL64)


def test_poisson_adam_steps_f64(modil):
    orc, desc, levels = _case(modil, (32, 64), 3, "f64", seed=52)
    st = o.OracleState.zeros_like_levels(levels)
    hist = [o.oracle_step(orc, st, 5e-3) for _ in range(3)]
    with modil.Problem(desc) as p:
        p.write_levels(levels)
        for k in range(3):
            t = p.step(1)[0]
            assert abs(t[0] - hist[k]["total"]) <= 1e-11 * hist[k]["total"]
        for lvl in range(3):
            ref = st.levels[lvl]
            assert np.max(np.abs(p.read_level(lvl) - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_poisson_lbfgs_matches_oracle_f64(modil):
    orc, desc, levels = _case(modil, (32, 32), 3, "f64", seed=53, n_meas=0)
    shapes = [a.shape for a in levels]
    sizes = [a.size for a in levels]

    def unflat(x):
        out, k = [], 0
        for s, n in zip(shapes, sizes):
            out.append(x[k:k + n].reshape(s))
            k += n
        return out

    f = lambda x: o.loss_terms(orc, o.compose(unflat(x)))["total"]  # noqa: E731

    def fg(x):
        t, g, _ = o.loss_grad_levels(orc, unflat(x))
        return t["total"], np.concatenate([a.ravel() for a in g])

    x0 = np.concatenate([a.ravel() for a in levels])
    x, loss_ref, done = lb.lbfgs(fg, f, x0, 5, 12)
    with modil.Problem(desc) as p:
        p.write_levels(levels)
        with modil.LBFGS(p, history=5) as opt:
            loss = opt.run(12)
        assert len(loss) == done + 1
        assert np.all(np.abs(loss - np.array(loss_ref)) <= 1e-8 * np.abs(loss_ref))
        for lvl, ref in enumerate(unflat(x)):
            assert np.max(np.abs(p.read_level(lvl) - ref)) <= 1e-7 * max(1.0, np.max(np.abs(ref)))


def test_poisson_levels_accelerate_lbfgs(modil):
    """The paper's reference problem (2-D, 32 cells, zero initial guess): after
    60 L-BFGS iterations five levels are closer to the reference solution
    than one."""
    w = inputs.poisson_workload(32)
    err = {}
    for L in (1, 5):
        desc = modil.Desc("poisson", w["shape"], L, "f64", aux=w["f"].ravel())
        with modil.Problem(desc) as p, modil.LBFGS(p, history=50) as opt:
            opt.run(60)
            u = p.read_field()
        err[L] = np.sqrt(np.mean((u - w["u_ref"]) ** 2) / np.mean(w["u_ref"] ** 2))
    assert err[5] < 0.5 * err[1], err
