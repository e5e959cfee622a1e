"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP32 problems 1e-5 relative on every loss term, norm-wise on each
level gradient and on dL/dq (plus a max-abs check at 10x that, scaled by the
largest reference entry); FP64 problems 1e-12.  Inputs are seeded random
levels with O(1) residuals, zero levels, and states along an oracle Adam
trajectory loaded into the device.
"""
import numpy as np
import pytest

import oracle as o
from _cases import Case, check_loss_grad, rel

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


@pytest.fixture(scope="module")
def modil():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import modil as m
    return m


def _tol(case):
    return TOL64 if case.dtype == "f64" else TOL32


# ---------------------------------------------------------------------------
# composition (Horner on the device) against the oracle's matrices
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,L,dtype", [((48, 96), 4, "f32"), ((64, 64), 4, "f64"),
                                           ((8, 8), 4, "f32"), ((512, 512), 7, "f32"),
                                           ((40, 200), 3, "f64")])
def test_composed_field(modil, shape, L, dtype):
    c = Case("burgers", shape, L, dtype, seed=1)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        u = p.read_field()
        ref = o.compose(c.levels)
        tol = 1e-14 if dtype == "f64" else 2e-6
        assert np.max(np.abs(u - ref)) <= tol * np.max(np.abs(ref))
        for lvl in range(L):
            np.testing.assert_array_equal(p.read_level(lvl), c.levels[lvl].astype(c.npd))


# ---------------------------------------------------------------------------
# loss and gradient
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,L", [((64, 64), 4), ((40, 72), 3), ((16, 16), 1), ((8, 8), 4)])
def test_burgers_f64_loss_grad(modil, shape, L):
    c = Case("burgers", shape, L, "f64", seed=2, n_meas=200, nu=0.01)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL64)


@pytest.mark.parametrize("tile", [(16, 32), (16, 64), (8, 64), (32, 32), (8, 128)])
def test_burgers_f32_loss_grad_tiles(modil, tile):
    c = Case("burgers", (96, 192), 4, "f32", seed=3, n_meas=400, nu=0.02, tile=tile)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL32)


@pytest.mark.parametrize("tile", [(16, 32), (16, 64), (8, 64), (32, 32), (8, 128)])
def test_heat_f32_loss_grad_tiles(modil, tile):
    c = Case("heat", (96, 160), 4, "f32", seed=4, n_meas=700, w_reg=0.05, tile=tile)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL32)


def test_heat_f64_loss_grad(modil):
    c = Case("heat", (64, 128), 5, "f64", seed=5, n_meas=300, w_reg=0.1)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL64)


def test_heat_full_size_512(modil):
    """The measured workload: 512 x 512, 7 levels, 5 % measurements, FP32, in
    the bench's launch configuration (32 x 32 tiles: 256 tiles, 512-thread
    blocks)."""
    c = Case("heat", (512, 512), 7, "f32", seed=6, n_meas=13107, w_reg=1e-4, tile=(32, 32))
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL32)


def test_burgers_full_size_64_f64(modil):
    """64 x 64 space-time, 4 levels, FP64, 200 measurements."""
    c = Case("burgers", (64, 64), 4, "f64", seed=7, n_meas=200, nu=0.01)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL64)


# ---------------------------------------------------------------------------
# rows or level starts off 4-element boundaries: the fine kernel's element
# by element staging and stores instead of 16-byte vectors
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("pde,shape,L", [("burgers", (38, 46), 2), ("heat", (30, 70), 2),
                                         ("burgers", (37, 45), 1)])
def test_rows_off_vector_boundaries(modil, pde, shape, L):
    c = Case(pde, shape, L, "f32", seed=30, n_meas=90, w_reg=0.05 if pde == "heat" else 0.0)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL32)


def test_adam_steps_with_unaligned_level_start(modil):
    """Instance 1 starts at an element offset that is not a multiple of 4
    (instance 0 holds 38*46 + 19*23 elements), so its fine tiles take the
    element-by-element Adam path; both FP64 trajectories match the oracle."""
    cases = [Case("burgers", (38, 46), 2, "f64", seed=31, n_meas=60, lr=5e-3),
             Case("burgers", (64, 96), 3, "f64", seed=32, n_meas=80, lr=5e-3)]
    with modil.Problem([c.desc() for c in cases]) as p:
        for i, c in enumerate(cases):
            c.load(p, instance=i)
        assert p.level_offset(0, 0, 1) % 4 != 0
        refs = [_oracle_steps(c, 3) for c in cases]
        for k in range(3):
            t = p.step(1)
            for i, (_, hist) in enumerate(refs):
                assert abs(t[i][0] - hist[k]["total"]) <= 1e-11 * hist[k]["total"], (i, k)
        for i, (c, (st, _)) in enumerate(zip(cases, refs)):
            for lvl in range(c.L):
                a = p.read_level(lvl, instance=i)
                ref = st.levels[lvl]
                assert np.max(np.abs(a - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref))), (i, lvl)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_no_measurements(modil):
    c = Case("heat", (32, 64), 3, "f32", seed=8, n_meas=0)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        terms, _, _ = check_loss_grad(c, p, TOL32)
        assert terms["data"] == 0.0


def test_duplicate_measurement_cells(modil):
    c = Case("burgers", (32, 64), 3, "f64", seed=9, n_meas=40, duplicate=15)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL64)


def test_zero_levels(modil):
    """Zero initial guess: heat residual comes from the initial condition only."""
    c = Case("heat", (64, 64), 4, "f32", seed=10, n_meas=100)
    zero = [np.zeros_like(a) for a in c.levels]
    with modil.Problem(c.desc()) as p:
        c.load(p, levels=zero)
        check_loss_grad(c, p, TOL32, levels=zero, check_max=False)


def test_batch_of_uneven_instances(modil):
    cases = [Case("burgers", s, L, "f32", seed=20 + i, n_meas=60, nu=nu)
             for i, (s, L, nu) in enumerate([((64, 128), 4, 0.01), ((32, 32), 2, 0.1),
                                             ((128, 64), 5, 0.003)])]
    with modil.Problem([c.desc() for c in cases]) as p:
        for i, c in enumerate(cases):
            c.load(p, instance=i)
        for i, c in enumerate(cases):
            check_loss_grad(c, p, TOL32, instance=i)


@pytest.mark.parametrize("n,shape,L", [(200, (128, 128), 4), (700, (64, 64), 3)])
def test_large_batches_small_tail_clusters(modil, n, shape, L):
    """Batches large enough that the tail kernel runs with 2 (200 instances)
    or 1 (700 instances) blocks per instance and leaves a 64^2 or 32^2 level
    to the restriction kernel: sampled instances match the oracle, and Adam
    steps of the batch match the same instances stepped alone."""
    cases = [Case("burgers", shape, L, "f32", seed=100 + i, n_meas=20, nu=0.01 + 0.002 * (i % 7))
             for i in range(n)]
    with modil.Problem([c.desc() for c in cases]) as p:
        for i, c in enumerate(cases):
            c.load(p, instance=i)
        for i in (0, n // 2, n - 1):
            check_loss_grad(cases[i], p, TOL32, instance=i)
        p.step(3, read_loss=False)
        tb = p.eval_loss()
    for i in (1, n // 3):
        with modil.Problem(cases[i].desc()) as q:
            cases[i].load(q)
            q.step(3, read_loss=False)
            ts = q.eval_loss()[0]
        assert abs(tb[i][0] - ts[0]) <= 1e-6 * ts[0], (i, tb[i][0], ts[0])


def test_eval_loss_matches_eval_grad(modil):
    c = Case("heat", (64, 96), 3, "f32", seed=11, n_meas=100, w_reg=0.01)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        a = p.eval_loss()
        b = p.eval_grad()
        np.testing.assert_array_equal(a, b)


def test_deterministic(modil):
    c = Case("heat", (128, 128), 5, "f32", seed=12, n_meas=500, w_reg=0.01)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        t1 = p.eval_grad()
        g1 = p.read_grads()
        k1 = p.read_kgrad()
        t2 = p.eval_grad()
        g2 = p.read_grads()
        k2 = p.read_kgrad()
        np.testing.assert_array_equal(t1, t2)
        for a, b in zip(g1, g2):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(k1, k2)


def test_nonfinite_is_reported(modil):
    c = Case("burgers", (32, 32), 2, "f32", seed=13)
    with modil.Problem(c.desc()) as p:
        lv = [a.copy() for a in c.levels]
        lv[0][3, 4] = np.nan
        c.load(p, levels=lv)
        with pytest.raises(modil.ModilError) as e:
            p.eval_loss()
        assert e.value.code == -5


# ---------------------------------------------------------------------------
# Adam steps
# ---------------------------------------------------------------------------
def _oracle_steps(c, n):
    st = o.OracleState.zeros_like_levels(c.levels, c.q)
    hist = []
    for _ in range(n):
        hist.append(o.oracle_step(c.oracle, st, c.lr))
    return st, hist


def test_adam_steps_f64_match_oracle(modil):
    c = Case("burgers", (64, 64), 4, "f64", seed=14, n_meas=200, lr=5e-3)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        st, hist = _oracle_steps(c, 5)
        for k in range(5):
            t = p.step(1)[0]
            assert abs(t[0] - hist[k]["total"]) <= 1e-11 * hist[k]["total"]
        for lvl in range(c.L):
            a = p.read_level(lvl)
            assert np.max(np.abs(a - st.levels[lvl])) <= 1e-12 * max(1.0, np.max(np.abs(st.levels[lvl])))
        assert p.step_count() == 5


def test_adam_first_step_f32(modil):
    """One step from random levels.  Cells whose oracle gradient is below the
    FP32 resolution of the gradient (sign not determined) only need a valid
    Adam step, |dp| <= lr; all others match the oracle update."""
    c = Case("heat", (96, 128), 4, "f32", seed=15, n_meas=300, w_reg=0.01, lr=5e-3)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        st, _ = _oracle_steps(c, 1)
        _, grads_ref, _ = c.oracle_eval()
        p.step(1)
        for lvl in range(c.L):
            a = p.read_level(lvl).astype(np.float64)
            ref = st.levels[lvl]
            g = grads_ref[lvl]
            sure = np.abs(g) > 1e-4 * np.max(np.abs(g))
            err = np.abs(a - ref)
            assert np.all(err[sure] <= 1e-6 * np.maximum(1.0, np.abs(ref[sure]))), lvl
            dp = np.abs(a - c.levels[lvl])
            assert np.all(dp <= c.lr * (1 + 1e-5) + 1e-6 * np.abs(c.levels[lvl]))
        q = p.read_knodes()
        assert rel(q, st.q) <= 1e-6


def test_loss_grad_along_oracle_trajectory(modil):
    """States after k oracle Adam steps, loaded into the device, match too."""
    c = Case("heat", (64, 64), 4, "f32", seed=16, n_meas=200, w_reg=0.01, lr=1e-2)
    st = o.OracleState.zeros_like_levels(c.levels, c.q)
    with modil.Problem(c.desc()) as p:
        done = 0
        for k in (1, 10, 30):
            while done < k:
                o.oracle_step(c.oracle, st, c.lr)
                done += 1
            lv = [a.astype(np.float32).astype(np.float64) for a in st.levels]
            q = st.q.astype(np.float32).astype(np.float64)
            c.load(p, levels=lv, q=q)
            check_loss_grad(c, p, TOL32, levels=lv, q=q, check_max=False)


def test_graph_and_direct_launch_agree(modil, monkeypatch):
    import torch
    c = Case("burgers", (64, 128), 4, "f32", seed=17, n_meas=100)
    with modil.Problem(c.desc()) as p1:
        c.load(p1)
        p1.step(7, read_loss=False)
        a = p1.read_levels()
        t1 = p1.eval_loss()
    # the legacy default stream is never captured: direct launches
    with modil.Problem(c.desc(), stream=torch.cuda.default_stream()) as p2:
        c.load(p2)
        for _ in range(7):
            p2.step(1, read_loss=False)
        b = p2.read_levels()
        t2 = p2.eval_loss()
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(t1, t2)


def test_reset_optimizer_restarts_adam(modil):
    c = Case("burgers", (32, 64), 3, "f64", seed=18, n_meas=50)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        p.step(3, read_loss=False)
        lv = p.read_levels()
        p.reset_optimizer()
        assert p.step_count() == 0
        for a, b in zip(lv, p.read_levels()):
            np.testing.assert_array_equal(a, b)
        st = o.OracleState.zeros_like_levels(lv, None)
        o.oracle_step(c.oracle, st, c.lr)
        p.step(1, read_loss=False)
        for lvl in range(c.L):
            assert np.max(np.abs(p.read_level(lvl) - st.levels[lvl])) <= 1e-12


def test_library_arena(modil):
    c = Case("burgers", (32, 32), 3, "f64", seed=19)
    with modil.Problem(c.desc(), arena="library") as p:
        c.load(p)
        check_loss_grad(c, p, TOL64)
