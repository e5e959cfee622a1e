"""L-BFGS on the device against the L-BFGS oracle (same algorithm in numpy
FP64 on the oracle's loss): loss history and final levels of FP64 problems,
with a history shorter than the run so that the pair ring wraps."""
import numpy as np
import pytest

import oracle as o
from oracle import lbfgs_oracle as lb
from _cases import Case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def modil():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import modil as m
    return m


def _oracle_run(c, m, iters):
    multi = c.nf > 1
    fields = c.levels if multi else [c.levels]
    shapes = [[np.asarray(a).shape for a in lv] for lv in fields]

    def unflat(x):
        out, k = [], 0
        for sh in shapes:
            lv = []
            for s in sh:
                n = int(np.prod(s))
                lv.append(x[k:k + n].reshape(s))
                k += n
            out.append(lv)
        return out if multi else out[0]

    def f(x):
        lv = unflat(x)
        u = [o.compose(a) for a in lv] if multi else o.compose(lv)
        return o.loss_terms(c.oracle, u)["total"]

    def fg(x):
        t, g, _ = o.loss_grad_levels(c.oracle, unflat(x))
        gs = g if multi else [g]
        return t["total"], np.concatenate([a.ravel() for gf in gs for a in gf])

    x0 = np.concatenate([np.asarray(a, np.float64).ravel() for lv in fields for a in lv])
    x, losses, done = lb.lbfgs(fg, f, x0, m, iters)
    return unflat(x), np.array(losses), done


@pytest.mark.parametrize("pde,shape,L,kw", [("burgers", (64, 64), 4, dict(n_meas=200, nu=0.01)),
                                            ("ns2d", (16, 16), 3, dict(n_meas=40, Re=100.0)),
                                            ("ns3d", (8, 8, 16), 3, dict(n_meas=50, Re=60.0))])
def test_lbfgs_matches_oracle_f64(modil, pde, shape, L, kw):
    c = Case(pde, shape, L, "f64", seed=40, **kw)
    m, iters = 4, 10
    lv_ref, loss_ref, done_ref = _oracle_run(c, m, iters)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        with modil.LBFGS(p, history=m) as opt:
            loss = opt.run(iters)
        assert len(loss) == done_ref + 1
        assert np.all(np.abs(loss - loss_ref) <= 1e-8 * np.abs(loss_ref)), (loss, loss_ref)
        fields = lv_ref if c.nf > 1 else [lv_ref]
        for f, lvf in enumerate(fields):
            for lvl, ref in enumerate(lvf):
                a = p.read_level(lvl, field=f)
                assert np.max(np.abs(a - ref)) <= 1e-7 * max(1.0, np.max(np.abs(ref))), (f, lvl)


@pytest.mark.parametrize("pde,shape,L,kw", [("burgers", (64, 64), 4, dict(n_meas=200, nu=0.01)),
                                            ("ns2d", (16, 16), 3, dict(n_meas=40, Re=100.0))])
def test_lbfgs_f32_tracks_oracle(modil, pde, shape, L, kw):
    """FP32 problems: the device's L-BFGS (FP32 vectors, FP64 dot products)
    follows the FP64 oracle's iterations to FP32 rounding for the first
    iterations and ends no higher."""
    c = Case(pde, shape, L, "f32", seed=44, **kw)
    m, iters = 4, 12
    _, loss_ref, _ = _oracle_run(c, m, iters)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        with modil.LBFGS(p, history=m) as opt:
            loss = opt.run(iters)
    k = min(5, len(loss), len(loss_ref))
    np.testing.assert_allclose(loss[:k], loss_ref[:k], rtol=1e-4)
    assert loss[-1] <= 1.05 * loss_ref[-1], (loss, loss_ref)


def test_lbfgs_descends_and_continues(modil):
    """FP32 Burgers: monotone loss, and a second run continues from the first."""
    c = Case("burgers", (64, 128), 4, "f32", seed=41, n_meas=300, nu=0.02)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        with modil.LBFGS(p, history=10) as opt:
            a = opt.run(15)
            b = opt.run(15)
        assert np.all(np.diff(a) < 0) and np.all(np.diff(b) <= 0)
        assert b[0] == pytest.approx(a[-1], rel=1e-6)
        t = p.eval_loss()[0]
        assert t[0] == pytest.approx(b[-1], rel=1e-6)


def test_lbfgs_rejects_batches(modil):
    cs = [Case("burgers", (32, 32), 2, "f32", seed=43 + i, n_meas=20) for i in range(2)]
    with modil.Problem([x.desc() for x in cs]) as p:
        with pytest.raises(modil.ModilError):
            modil.LBFGS(p)
