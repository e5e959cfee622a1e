"""The paper's Burgers reconstruction (Section 3.2) on the GPU: inviscid
Burgers on (x, t) in [0, 1]^2, 64 x 64 cells, six levels (64 .. 2 cells),
the reference solution of the discrete problem (zero Dirichlet walls, u(x, 0)
= (1 - cos 6 pi x)/2; oracle row-by-row solve) imposed at 84 points on the
edges of a rectangle.

* the loss terms and every level gradient match the FP64 oracle at random
  levels (FP64 and FP32), with the points sampled d-linearly;
* L-BFGS (history 50) on the device follows the oracle's L-BFGS on the same
  problem for its first iterations and, as Section 3.2 reports for mODIL with
  L-BFGS, drives the loss below 1e-4, recovers the solution inside the
  rectangle, and does not recover it everywhere (the rectangle's edges do
  not determine the solution outside the characteristics through them);
* with uniform noise U[0, 0.05] added to the imposed values the loss stays
  above the noise-free one but below 0.1 (Section 3.2), and the inside of the
  rectangle is still close to the reference."""
import numpy as np
import pytest

import oracle as o
from oracle import lbfgs_oracle as lb
from oracle import offgrid_oracle as og
from paper_2303_04679_gb300 import inputs

pytestmark = pytest.mark.gpu

P = inputs.BURGERS_PAPER


@pytest.fixture(scope="module")
def modil():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import modil as m
    return m


@pytest.fixture(scope="module")
def ref():
    nt, nx = P["shape"]
    x = (np.arange(nx) + 0.5) / nx
    u = o.burgers_implicit_solve(inputs.burgers_paper_ic(x), nt, 1.0 / nt, 1.0 / nx, nu=0.0)
    pts = inputs.rectangle_points()
    idx, wt = og.sample_weights(pts, (nt, nx), (1.0, 1.0), (0.0, 0.0))
    vals = (wt * u.reshape(-1)[idx]).sum(axis=1)
    return u, pts, vals


def _problems(modil, pts, vals, dtype):
    npd = np.float64 if dtype == "f64" else np.float32
    v = np.asarray(vals, np.float64).astype(npd).astype(np.float64)
    orc = o.Problem("burgers", P["shape"], P["n_levels"], coef={"nu": 0.0}, meas_points=pts,
                    point_value=v, domain_bounds=P["domain"])
    desc = modil.Desc("burgers", P["shape"], P["n_levels"], dtype, coef=(0.0,), points=pts,
                      point_value=v, domain=P["domain"], lr=5e-3)
    return orc, desc


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-5)])
def test_paper_problem_loss_grad(modil, ref, dtype, tol):
    _, pts, vals = ref
    orc, desc = _problems(modil, pts, vals, dtype)
    npd = np.float64 if dtype == "f64" else np.float32
    lv = [np.asarray(a, npd).astype(np.float64)
          for a in inputs.random_levels(P["shape"], P["n_levels"], 1, 12, 0.0, 1.0, 0.2)[0]]
    terms, grads, _ = o.loss_grad_levels(orc, lv)
    with modil.Problem(desc) as p:
        p.write_levels(lv)
        t = p.eval_grad()[0]
        for j, name in enumerate(("total", "res", "data")):
            assert abs(t[j] - terms[name]) <= tol * terms[name], (name, t[j], terms[name])
        for lvl, gr in enumerate(grads):
            g = p.read_grad(lvl).astype(np.float64)
            assert np.linalg.norm(g - gr) <= tol * np.linalg.norm(gr), lvl


def _flat_oracle(orc):
    shapes = o.level_shapes(P["shape"], P["n_levels"])
    sizes = [int(np.prod(s)) for s in shapes]

    def unpack(z):
        out, k = [], 0
        for s, n in zip(shapes, sizes):
            out.append(z[k:k + n].reshape(s))
            k += n
        return out

    def fg(z):
        t, g, _ = o.loss_grad_levels(orc, unpack(z))
        return t["total"], np.concatenate([a.reshape(-1) for a in g])

    def f(z):
        return o.loss_terms(orc, o.compose(unpack(z)))["total"]
    return fg, f, sum(sizes)


def _errors(u, u_ref):
    nt, nx = P["shape"]
    T, X = np.meshgrid((np.arange(nt) + 0.5) / nt, (np.arange(nx) + 0.5) / nx, indexing="ij")
    (t0, t1), (x0, x1) = P["rect"]
    inside = (T >= t0) & (T <= t1) & (X >= x0) & (X <= x1)
    d = u - u_ref
    return float(np.sqrt(np.mean(d[inside] ** 2))), float(np.sqrt(np.mean(d ** 2)))


def test_paper_reconstruction_lbfgs(modil, ref):
    u_ref, pts, vals = ref
    orc, desc = _problems(modil, pts, vals, "f64")
    fg, f, n = _flat_oracle(orc)
    _, want, _ = lb.lbfgs(fg, f, np.zeros(n), 50, 30)
    with modil.Problem(desc) as p, modil.LBFGS(p, history=50) as opt:
        hist = opt.run(400)
        u = p.read_field()
    # the device follows the oracle's iterations (same algorithm, FP64)
    np.testing.assert_allclose(hist[:31], want, rtol=1e-8)
    # Section 3.2: loss below 1e-4; the solution recovered inside the
    # rectangle, not everywhere (measured 2e-6, RMS 0.001 inside, 0.16 overall)
    assert hist[-1] < 1e-4, hist[-1]
    e_in, e_all = _errors(u, u_ref)
    assert e_in < 0.01, e_in
    assert 0.05 < e_all < 0.4, e_all


def test_paper_reconstruction_with_uniform_noise(modil, ref):
    u_ref, pts, vals = ref
    noisy = inputs.uniform_noise(vals, 0.05, seed=1)
    _, desc = _problems(modil, pts, noisy, "f64")
    with modil.Problem(desc) as p, modil.LBFGS(p, history=50) as opt:
        hist = opt.run(400)
        u = p.read_field()
    # measured: loss 2.2e-4, RMS 0.025 inside the rectangle
    assert 1e-5 < hist[-1] < 0.1, hist[-1]
    e_in, _ = _errors(u, u_ref)
    assert e_in < 0.06, e_in
