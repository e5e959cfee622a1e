"""The allocation-free entry point agrees with the regular one.

modil_eval_grad_noalloc serves callers that cannot allocate device memory
(a host application that owns all device allocations, or a loop that must not
allocate while running): it keeps its working memory in a fixed device array
inside the library instead of an arena.  Here it is called through the C ABI
twice in a row, on two different states, for every 2-D family it takes (one
field: Burgers, heat, Poisson; three fields, field-major: the cavity) in FP32
and FP64, and each result is compared with modil_eval_grad of a regular
problem at the test suite's tolerance.  The documented refusals (a problem
whose tables exceed the array, the 3-D body problem, off-grid points, pointers
off a 16-byte boundary) are checked to return their status codes; each
returns before any kernel is launched.  This file is collected last so that
a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from _cases import Case, rel

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-5, "f64": 1e-11}


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import modil
    return torch, modil


CASES = {
    "heat": lambda dt: Case("heat", (128, 192), 5, dt, seed=31, n_meas=1200, w_reg=0.02),
    "burgers": lambda dt: Case("burgers", (96, 160), 4, dt, seed=32, n_meas=300, nu=0.02),
    "poisson": lambda dt: Case("poisson", (64, 96), 4, dt, seed=33, n_meas=100),
    "ns2d": lambda dt: Case("ns2d", (48, 48), 4, dt, seed=34, n_meas=200),
}


def _poisson_aux(c):
    # the Poisson right-hand side travels in aux, one value per fine cell
    if c.pde == "poisson":
        rng = np.random.default_rng(7)
        c.desc_kw["aux"] = rng.normal(size=int(np.prod(c.shape)))
        c.oracle.coef["f"] = c.desc_kw["aux"].reshape(c.shape)
    return c


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("pde", ["heat", "burgers", "poisson", "ns2d"])
def test_noalloc_matches_regular_entry_point_twice(env, pde, dtype):
    torch, modil = env
    c = _poisson_aux(CASES[pde](dtype))
    tol = TOL[dtype]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if c.nf > 1:
        states = [c.levels, [[np.asarray(a) * 0.5 + 0.1 for a in f] for f in c.levels]]
    else:
        states = [c.levels, [np.asarray(a) * 0.5 + 0.1 for a in c.levels]]
    desc = c.desc()
    for lv in states:
        if c.nf > 1:
            lv = [[np.asarray(a, c.npd).astype(np.float64) for a in f] for f in lv]
            flat_host = np.concatenate([a.reshape(-1) for f in lv for a in f])
        else:
            lv = [np.asarray(a, c.npd).astype(np.float64) for a in lv]
            flat_host = np.concatenate([a.reshape(-1) for a in lv])
        with modil.Problem(desc) as p:
            c.load(p, levels=lv)
            ref_terms = p.eval_grad()[0]
            ref = [[p.read_grad(l, field=f) for l in range(c.L)] for f in range(c.nf)]
            ref_kg = p.read_kgrad() if pde == "heat" else None
        flat = torch.tensor(flat_host, dtype=tdt, device="cuda")
        grads = torch.full_like(flat, float("nan"))
        terms, kg = modil.eval_grad_noalloc(desc, flat, grads)
        for j in range(4):
            assert abs(terms[j] - ref_terms[j]) <= tol * max(abs(ref_terms[j]), 1e-300), j
        g = grads.cpu().numpy().astype(np.float64)
        off = 0
        for f in range(c.nf):
            for lvl, r in enumerate(ref[f]):
                n = r.size
                assert rel(g[off:off + n], r.reshape(-1)) <= tol, (f, lvl)
                off += n
        assert off == g.size
        if pde == "heat":
            assert rel(kg, ref_kg) <= tol


def _status(modil, desc, levels, grads):
    terms = np.zeros(modil.NTERMS)
    code = modil.LIB.modil_eval_grad_noalloc(
        modil.C.byref(desc.c), levels, grads,
        terms.ctypes.data_as(modil.C.POINTER(modil.C.c_double)), None, None)
    return code


def test_noalloc_refusals(env):
    torch, modil = env
    # tables beyond the 8 MiB array: one measurement per cell of a 2048^2 grid
    n = 2048
    big = modil.Desc("heat", (n, n), 3, aux=np.zeros(n), knodes=np.full(32, 0.02),
                     meas_cell=np.arange(n * n, dtype=np.int32), meas_value=np.zeros(n * n))
    buf = torch.zeros(big.param_count(), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(buf)
    assert _status(modil, big, buf.data_ptr(), out.data_ptr()) == modil.ERR_ARG
    # the 3-D body problem
    body = modil.Desc("ns3d", (8, 8, 16), 2, coef=(60.0, 0.4, 1.0, 1.0))
    b3 = torch.zeros(body.param_count(), dtype=torch.float32, device="cuda")
    assert _status(modil, body, b3.data_ptr(), b3.data_ptr()) == modil.ERR_UNSUPPORTED
    # off-grid points
    pts = modil.Desc("burgers", (32, 32), 2, coef=(0.01,), points=np.array([[0.3, 0.1]]),
                     point_value=np.array([0.2]))
    b2 = torch.zeros(pts.param_count(), dtype=torch.float32, device="cuda")
    assert _status(modil, pts, b2.data_ptr(), b2.data_ptr()) == modil.ERR_UNSUPPORTED
    # a view one element in: 4 bytes off the 16-byte boundary
    ok = modil.Desc("burgers", (32, 32), 2, coef=(0.01,))
    b4 = torch.zeros(ok.param_count() + 4, dtype=torch.float32, device="cuda")
    assert _status(modil, ok, b4[1:].data_ptr(), b4[4:].data_ptr()) == modil.ERR_ARG
    with pytest.raises(ValueError):
        modil.eval_grad_noalloc(ok, b4[1:1 + ok.param_count()], b4[:ok.param_count()])
