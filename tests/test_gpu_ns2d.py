"""Lid-driven cavity (three fields) on the GPU against the FP64 oracle, and the
torch.autograd.Function path (forward, backward, finite differences, a torch
optimiser loop)."""
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


@pytest.mark.parametrize("shape,L,tile", [((48, 48), 4, (8, 32)), ((64, 64), 5, (16, 32)),
                                          ((16, 16), 1, (8, 32)), ((8, 8), 4, (8, 32))])
def test_ns2d_f32_loss_grad(modil, shape, L, tile):
    c = Case("ns2d", shape, L, "f32", seed=40, n_meas=60, tile=tile)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL32)


def test_ns2d_f64_loss_grad(modil):
    c = Case("ns2d", (32, 32), 4, "f64", seed=41, n_meas=40, Re=60.0, tau=0.5)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL64)


def test_ns2d_full_size_256(modil):
    """256^2 cells, 8 levels, 1000 velocity samples, FP32."""
    c = Case("ns2d", (256, 256), 8, "f32", seed=42, n_meas=1000)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        check_loss_grad(c, p, TOL32)


def test_ns2d_composed_fields(modil):
    c = Case("ns2d", (64, 64), 4, "f32", seed=43)
    with modil.Problem(c.desc()) as p:
        c.load(p)
        for f in range(3):
            u = p.read_field(f)
            ref = o.compose(c.levels[f])
            assert np.max(np.abs(u - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_ns2d_adam_steps_f64(modil):
    c = Case("ns2d", (32, 32), 3, "f64", seed=44, n_meas=30, lr=1e-2)
    st = o.OracleState.zeros_like_levels(c.levels)
    hist = [o.oracle_step(c.oracle, st, c.lr) for _ in range(4)]
    with modil.Problem(c.desc()) as p:
        c.load(p)
        for k in range(4):
            t = p.step(1)[0]
            assert abs(t[0] - hist[k]["total"]) <= 1e-11 * hist[k]["total"]
        for f in range(3):
            for lvl in range(c.L):
                a = p.read_level(lvl, field=f)
                ref = st.levels[f][lvl]
                assert np.max(np.abs(a - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


# ---------------------------------------------------------------------------
# torch.autograd.Function
# ---------------------------------------------------------------------------
def _flat_from_levels(p, levels_per_field, dtype):
    import torch
    flat = torch.zeros(p.param_count(), dtype=dtype)
    for f, lv in enumerate(levels_per_field):
        for lvl, a in enumerate(lv):
            off = p.level_offset(lvl, field=f)
            flat[off:off + a.size] = torch.from_numpy(np.ascontiguousarray(a).reshape(-1))
    return flat.cuda()


def test_autograd_matches_oracle(modil):
    import torch
    from paper_2303_04679_gb300.autograd import ModilLoss
    c = Case("ns2d", (64, 64), 5, "f32", seed=45, n_meas=100)
    terms, grads, _ = c.oracle_eval()
    with modil.Problem(c.desc()) as p:
        x = _flat_from_levels(p, c.levels, torch.float32).requires_grad_(True)
        loss = ModilLoss.apply(x, p)
        assert abs(loss.item() - terms["total"]) <= TOL32 * terms["total"]
        (2.5 * loss).backward()
        g = x.grad.cpu().numpy().astype(np.float64)
        for f in range(3):
            for lvl, gr in enumerate(grads[f]):
                off = p.level_offset(lvl, field=f)
                assert rel(g[off:off + gr.size], 2.5 * gr.reshape(-1)) <= TOL32, (f, lvl)


def test_autograd_finite_differences_16(modil):
    """The hand-written adjoint behind ModilLoss against central differences of
    its own forward pass, on a 16 x 16 copy in FP64."""
    import torch
    from paper_2303_04679_gb300.autograd import ModilLoss
    c = Case("ns2d", (16, 16), 3, "f64", seed=46, n_meas=20)
    with modil.Problem(c.desc()) as p:
        x = _flat_from_levels(p, c.levels, torch.float64).requires_grad_(True)
        ModilLoss.apply(x, p).backward()
        g = x.grad.cpu().numpy()
        rng = np.random.default_rng(0)
        idx = rng.choice(x.numel(), size=40, replace=False)
        base = x.detach().clone()
        for i in idx:
            h = 1e-6 * max(1.0, abs(float(base[i])))
            xp = base.clone(); xp[i] += h
            xm = base.clone(); xm[i] -= h
            fd = (ModilLoss.apply(xp, p).item() - ModilLoss.apply(xm, p).item()) / (2 * h)
            assert abs(fd - g[i]) <= 1e-6 * max(1.0, np.max(np.abs(g))), (i, fd, g[i])


def test_autograd_torch_adam_reduces_loss(modil):
    import torch
    from paper_2303_04679_gb300.autograd import ModilParameters
    c = Case("ns2d", (32, 32), 4, "f32", seed=47, n_meas=50)
    with modil.Problem(c.desc()) as p:
        params = ModilParameters(p)
        opt = torch.optim.Adam(params.parameters(), lr=1e-2)
        first = None
        for it in range(60):
            opt.zero_grad()
            loss = params()
            loss.backward()
            opt.step()
            first = loss.item() if first is None else first
        assert params().item() < 0.5 * first


def test_autograd_step_captured_in_cuda_graph(modil):
    """The autograd step (ModilLoss forward, backward, torch Adam) captured in
    a CUDA graph: the library's launches join torch's capture through the
    stream waits, and replays reproduce the eager steps."""
    import torch
    from paper_2303_04679_gb300.autograd import ModilParameters
    c = Case("ns2d", (32, 32), 4, "f32", seed=48, n_meas=50)

    def run(captured, n=5):
        with modil.Problem(c.desc()) as p:
            params = ModilParameters(p)
            # the same (capturable) Adam in both runs: only the launch mode differs
            opt = torch.optim.Adam(params.parameters(), lr=1e-2, capturable=True)

            def step():
                opt.zero_grad(set_to_none=False)
                params().backward()
                opt.step()
            # the first step also creates the gradient and optimiser buffers
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                step()
            torch.cuda.current_stream().wait_stream(side)
            if captured:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    step()
                for _ in range(n - 1):
                    g.replay()
            else:
                for _ in range(n - 1):
                    step()
            torch.cuda.synchronize()
            return params.flat.detach().cpu().numpy().copy()

    eager, graph = run(False), run(True)
    assert np.max(np.abs(eager - graph)) <= 1e-6 * max(1.0, np.max(np.abs(eager)))
