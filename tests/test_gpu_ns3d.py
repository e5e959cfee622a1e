"""Penalised 3-D Navier-Stokes (body shape, five fields) on the GPU against
the FP64 oracle: loss terms and every level gradient on grids that span
several tiles with ragged edges, the composed fields, Adam trajectories in
FP64, and the full 128^3, 8-level workload checked on sampled fine-grid
gradients and directional derivatives of the oracle loss."""
import numpy as np
import pytest

import oracle as o
from _cases import Case, check_loss_grad

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


@pytest.mark.parametrize("shape,L", [((8, 8, 16), 3),      # one tile in x and y, two in z
                                     ((12, 24, 48), 3),    # 3 x 3 x 3 tiles
                                     ((6, 12, 40), 2),     # ragged tiles on every axis
                                     ((16, 16, 32), 5),    # coarsest level 1 x 1 x 2
                                     ((4, 8, 8), 1)])      # single level (no multigrid)
def test_ns3d_f32_loss_grad(modil, shape, L):
    c = Case("ns3d", shape, L, "f32", seed=60, n_meas=80, Re=60.0)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL32)


def test_ns3d_f32_body_everywhere_and_nowhere(modil):
    """chi near 1 (all body: only penalisation survives) and near 0 (no body)."""
    for shift in (16.0, -6.0):
        c = Case("ns3d", (8, 16, 16), 3, "f32", seed=61, n_meas=40, chi_shift=shift)
        with modil.Problem(c.desc()) as p:
            c.load(p)
            check_loss_grad(c, p, TOL32)


def test_ns3d_f64_loss_grad(modil):
    c = Case("ns3d", (8, 8, 16), 4, "f64", seed=62, n_meas=50, Re=60.0, tau=0.5, lam=2.0)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL64)


def test_ns3d_composed_fields(modil):
    c = Case("ns3d", (16, 16, 32), 4, "f32", seed=63)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        for f in range(5):
            u = p.read_field(f)
            ref = o.compose(c.levels[f])
            assert u.shape == ref.shape
            assert np.max(np.abs(u - ref)) <= 2e-6 * np.max(np.abs(ref)), f


def test_ns3d_adam_steps_f64(modil):
    c = Case("ns3d", (8, 8, 16), 3, "f64", seed=64, n_meas=30, lr=1e-2)
    st = o.OracleState.zeros_like_levels(c.levels)
    hist = [o.oracle_step(c.oracle, st, c.lr) for _ in range(3)]
    with modil.Problem(c.desc()) as p:
        c.load(p)
        for k in range(3):
            t = p.step(1)[0]
            assert abs(t[0] - hist[k]["total"]) <= 1e-11 * hist[k]["total"]
        for f in range(5):
            for lvl in range(c.L):
                a = p.read_level(lvl, field=f)
                ref = st.levels[f][lvl]
                assert np.max(np.abs(a - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref))), (f, lvl)


def test_ns3d_steps_are_deterministic(modil):
    """The 3-D kernels use no atomics: every gradient is gathered per cell in a
    fixed order and the loss partials are summed in a fixed order, so two runs
    of the same steps agree bit for bit, loss and every field of every level."""
    c = Case("ns3d", (16, 16, 32), 4, "f32", seed=65, n_meas=40, lr=1e-3)
    out = []
    for _ in range(2):
        with modil.Problem(c.desc()) as p:
            c.load(p)
            t = p.step(5)[0]
            out.append((t.copy(), [[p.read_level(l, field=f) for l in range(c.L)] for f in range(5)]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for f in range(5):
        for lvl in range(c.L):
            np.testing.assert_array_equal(out[0][1][f][lvl], out[1][1][f][lvl])


def test_bounded_wait_timeout_is_reported(modil):
    """A bounded wait that runs out is reported as MODIL_ERR_TIMEOUT, once,
    without a hang or a fault: with the test hook's limit of zero polls every
    block of the 3-D kernel gives up its wait for the tile copies at once,
    flags the status, waits (bounded) for the copies still in flight and skips
    its tile; afterwards the same problem gives its earlier results bit for
    bit (the context and the problem stay usable)."""
    import ctypes
    c = Case("ns3d", (16, 16, 32), 3, "f32", seed=67, n_meas=40)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        ref = p.eval_grad()[0].copy()
        g_ref = p.read_grad(0, field=0)
        modil._check(modil.LIB.modil_test_set_spin_limit(ctypes.c_longlong(0)))
        try:
            with pytest.raises(modil.ModilError) as e:
                p.eval_grad()
            assert e.value.code == modil.ERR_TIMEOUT
        finally:
            modil._check(modil.LIB.modil_test_set_spin_limit(ctypes.c_longlong(-1)))
        t = p.eval_grad()[0]
        np.testing.assert_array_equal(t, ref)
        np.testing.assert_array_equal(p.read_grad(0, field=0), g_ref)


def test_ns3d_rejects_bad_descriptors(modil):
    c = Case("ns3d", (8, 8, 16), 3, "f32", seed=66)
    kw = dict(c.desc_kw)
    with pytest.raises(RuntimeError):
        modil.Problem(modil.Desc(**dict(kw, shape=(8, 16))))          # ndim 2
    with pytest.raises(RuntimeError):
        modil.Problem(modil.Desc(**dict(kw, tile=(8, 32))))           # tile is fixed
    with pytest.raises(RuntimeError):
        modil.Problem(modil.Desc(**dict(kw, coef=(0.0, 0.4, 1.0, 1.0))))  # Re = 0
    with pytest.raises(RuntimeError):
        modil.Problem(modil.Desc(**dict(kw, shape=(6, 8, 16))))       # 6 not divisible by 4


# ---------------------------------------------------------------------------
# Full size: 128^3 cells, 8 levels, 3 x 4096 wake samples
# ---------------------------------------------------------------------------
def _full_problem(modil):
    from paper_2303_04679_gb300 import inputs
    w = inputs.ns3d_workload()
    shape, L = w["shape"], w["n_levels"]
    levels = inputs.random_levels(shape, L, 5, 7, -0.5, 0.5, 0.2, dtype=np.float32)
    levels[4][0] = (levels[4][0] * 8.0 + 5.0).astype(np.float32).astype(np.float64)
    cf = w["coef"]
    coef = (cf["Re"], cf["D"], cf["lam"], cf["tau"])
    vals = w["meas_value"].astype(np.float32).astype(np.float64)
    desc = modil.Desc("ns3d", shape, L, "f32", coef=coef, meas_cell=w["meas_cell"],
                      meas_field=w["meas_field"], meas_value=vals, lr=w["lr"])
    orc = o.Problem("ns3d", shape, L, coef=dict(cf), meas_cell=w["meas_cell"],
                    meas_field=w["meas_field"], meas_value=vals)
    return desc, orc, levels


def test_ns3d_full_size_sampled(modil):
    desc, orc, levels = _full_problem(modil)
    u = [o.compose(lv) for lv in levels]
    ref = o.loss_terms(orc, u)
    with modil.Problem(desc) as p:
        p.write_fields(levels)
        t = p.eval_grad()[0]
        for j, name in enumerate(("total", "res", "data")):
            assert abs(t[j] - ref[name]) <= TOL32 * abs(ref[name]), (name, t[j], ref[name])
        # fine-grid gradient on one colour class (every 5th cell per axis) of every field
        colours = [(f, 1, 2, 3) for f in range(5)]
        g_ref = o.ns3d_fine_grad_colours(orc, u, colours)
        kk, jj, ii = np.meshgrid(*[np.arange(n) for n in desc.shape], indexing="ij")
        sel = (kk % 5 == 1) & (jj % 5 == 2) & (ii % 5 == 3)
        for f in range(5):
            g = p.read_grad(0, field=f)[sel].astype(np.float64)
            gr = g_ref[f][sel]
            assert np.linalg.norm(g - gr) <= TOL32 * np.linalg.norm(gr), f
            assert np.max(np.abs(g - gr)) <= 10 * TOL32 * np.max(np.abs(gr)), f
        # every level: directional derivative against the oracle loss
        # (central differences with Richardson extrapolation, truncation O(eps^4))
        rng = np.random.default_rng(11)
        for lvl in (0, 2, 5, 7):
            d = [rng.standard_normal(levels[f][lvl].shape) for f in range(5)]
            gl = [p.read_grad(lvl, field=f).astype(np.float64) for f in range(5)]
            gpu = sum(float(np.sum(a * b)) for a, b in zip(gl, d))

            def loss_at(eps):
                lv = [[a + (eps * d[f] if i == lvl else 0.0) for i, a in enumerate(levels[f])]
                      for f in range(5)]
                return o.loss_terms(orc, [o.compose(x) for x in lv])["total"]

            def cd(eps):
                return (loss_at(eps) - loss_at(-eps)) / (2 * eps)

            fd = (4 * cd(5e-4) - cd(1e-3)) / 3
            gnorm = np.sqrt(sum(float(np.sum(a * a)) for a in gl))
            assert abs(gpu - fd) <= TOL32 * gnorm, (lvl, gpu, fd, gnorm)


def test_ns3d_autograd_parameter_views(modil):
    """The flat torch parameter of a 3-D problem exposes every level as a
    (z, y, x) view at the library's offsets."""
    import torch
    from paper_2303_04679_gb300.autograd import ModilLoss, ModilParameters
    c = Case("ns3d", (8, 8, 16), 3, "f32", seed=67, n_meas=30)
    with modil.Problem(c.desc()) as p:
        params = ModilParameters(p)
        with torch.no_grad():
            for f in range(5):
                for lvl in range(c.L):
                    v = params.level(lvl, field=f)
                    assert tuple(v.shape) == tuple(np.asarray(c.levels[f][lvl]).shape)
                    v.copy_(torch.from_numpy(np.asarray(c.levels[f][lvl], np.float32)))
        terms, _, _ = c.oracle_eval()
        loss = ModilLoss.apply(params.flat, p)
        assert abs(loss.item() - terms["total"]) <= TOL32 * terms["total"]
