"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/modil.h declares, and validates descriptors."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(modil_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def mod():
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import modil
    return modil


def test_library_exports_every_declared_symbol(mod):
    names = _declared()
    assert len(names) >= 19
    missing = [n for n in sorted(names) if not hasattr(mod.LIB, n)]
    assert not missing, missing


def test_version_string(mod):
    assert "sm_103a" in mod.version()


def test_descriptor_struct_matches_the_header(mod):
    import ctypes as C
    assert mod.LIB.modil_desc_size() == C.sizeof(mod.modil_desc)


def test_k_fixed_only_for_the_heat_family(mod):
    assert mod.arena_bytes([_heat(mod, k_fixed=True)]) > 0
    with pytest.raises(mod.ModilError) as e:
        mod.arena_bytes([mod.Desc("burgers", (16, 16), 2, coef=(0.01,), k_fixed=True)])
    assert e.value.code == mod.ERR_ARG


def _heat(mod, shape=(64, 64), L=4, **kw):
    nt, nx = shape
    return mod.Desc("heat", shape, L, aux=np.zeros(nx), knodes=np.full(32, 0.02), **kw)


def test_arena_bytes_grows_with_problem(mod):
    a = mod.arena_bytes([_heat(mod, (64, 64), 4)])
    b = mod.arena_bytes([_heat(mod, (128, 128), 4)])
    c = mod.arena_bytes([_heat(mod, (64, 64), 4), _heat(mod, (64, 64), 4)])
    assert 0 < a < b and a < c
    # p0, p1, m, g (4 B) + v (8 B) per parameter at least
    P = sum((64 >> l) ** 2 for l in range(4))
    assert a >= 24 * P


@pytest.mark.parametrize("bad", [
    dict(shape=(60, 64), L=4),        # 60 not divisible by 8
    dict(shape=(64, 64), L=11),       # too many levels
    dict(shape=(64, 64), L=0),
])
def test_arena_bytes_rejects_bad_grids(mod, bad):
    with pytest.raises(mod.ModilError) as e:
        mod.arena_bytes([_heat(mod, bad["shape"], bad["L"])])
    assert e.value.code == -1


def test_rejects_bad_measurements_and_mixed_batches(mod):
    d = mod.Desc("burgers", (16, 16), 2, coef=(0.01,), meas_cell=[0, 300], meas_value=[1.0, 2.0])
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([d])
    d = mod.Desc("burgers", (16, 16), 2, coef=(0.01,), meas_cell=[3], meas_value=[np.nan])
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([d])
    a = mod.Desc("burgers", (16, 16), 2, coef=(0.01,))
    b = mod.Desc("burgers", (16, 16), 2, coef=(0.01,), dtype="f64")
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([a, b])
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([mod.Desc("heat", (16, 16), 2)])  # no initial profile / nodes
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([mod.Desc("burgers", (16, 16), 2, tile=(7, 7))])


def _body(mod, shape=(16, 16, 32), L=3, **kw):
    return mod.Desc("ns3d", shape, L, coef=(60.0, 0.4, 1.0, 1.0), **kw)


def test_ns3d_arena_bytes_and_validation(mod):
    a = mod.arena_bytes([_body(mod)])
    # five fields; p0, p1, m, g (4 B) + v (8 B) per parameter, plus the composed fields
    P = sum((16 >> l) * (16 >> l) * (32 >> l) for l in range(3))
    assert a >= 5 * (24 * P + 4 * 16 * 16 * 32)
    # measurement cells index the flat (z, y, x) grid and fields 0..4
    ok = _body(mod, meas_cell=[0, 16 * 16 * 32 - 1], meas_value=[1.0, 2.0], meas_field=[0, 4])
    assert mod.arena_bytes([ok]) > 0
    for bad in (dict(meas_cell=[16 * 16 * 32], meas_value=[1.0]),
                dict(meas_cell=[0], meas_value=[1.0], meas_field=[5])):
        with pytest.raises(mod.ModilError):
            mod.arena_bytes([_body(mod, **bad)])
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([_body(mod, shape=(16, 32))])            # 3-D family, ndim 2
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([mod.Desc("ns2d", (8, 8, 8), 2, coef=(100.0, 1.0))])  # 2-D family, ndim 3
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([_body(mod, tile=(8, 32))])
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([mod.Desc("ns3d", (16, 16, 32), 3, coef=(0.0, 0.4, 1.0, 1.0))])
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([_body(mod, shape=(12, 16, 32), L=4)])  # 12 not divisible by 8


def test_offgrid_points_in_the_plan(mod):
    """Off-grid points enlarge the arena (their per-tile records), non-finite
    coordinates and out-of-range fields are rejected (host only)."""
    import ctypes as C
    rng = np.random.default_rng(0)
    pts = np.column_stack([rng.uniform(0, 1, 300), rng.uniform(-1, 1, 300)])

    def nbytes(d):
        b = C.c_size_t()
        return mod.LIB.modil_arena_bytes(C.byref(d.c), 1, C.byref(b)), b.value

    base = mod.Desc("burgers", (48, 96), 3, "f32", coef=(0.02,), tile=(16, 32))
    with_pts = mod.Desc("burgers", (48, 96), 3, "f32", coef=(0.02,), points=pts,
                        point_value=np.zeros(300), tile=(16, 32))
    r0, b0 = nbytes(base)
    r1, b1 = nbytes(with_pts)
    assert r0 == 0 and r1 == 0 and b1 > b0
    bad = mod.Desc("burgers", (48, 96), 3, "f32", coef=(0.02,), points=[[np.nan, 0.0]],
                   point_value=np.zeros(1))
    assert nbytes(bad)[0] != 0
    # the multi-field families take points with a field index in range
    ns2d = mod.Desc("ns2d", (16, 16), 2, "f32", coef=(100.0, 1.0), points=[[0.5, 0.5]],
                    point_value=np.zeros(1), point_field=np.array([1], np.int32))
    assert nbytes(ns2d)[0] == 0
    ns2d_bad = mod.Desc("ns2d", (16, 16), 2, "f32", coef=(100.0, 1.0), points=[[0.5, 0.5]],
                        point_value=np.zeros(1), point_field=np.array([3], np.int32))
    assert nbytes(ns2d_bad)[0] != 0
    body = mod.Desc("ns3d", (8, 8, 16), 2, "f32", coef=(60.0, 0.4, 1.0, 1.0), points=[[0.5, 0.5, 1.0]],
                    point_value=np.zeros(1), point_field=np.array([2], np.int32))
    assert nbytes(body)[0] == 0


def test_streaming_strip_tile(mod):
    """The warp-streaming Burgers kernel's strip is 32 rows x 60 columns (two
    columns per lane of a warp): that tile is accepted for Burgers, also with
    odd widths and a single level, and refused for other families and with
    off-grid points; the former 32 x 28 strip is no tile shape any more
    (host only)."""
    from paper_2303_04679_gb300 import autotune
    assert autotune.STREAM_TILE == (32, 60)
    for shape, L in (((64, 512), 4), ((45, 61), 1), ((40, 33), 1)):
        assert mod.arena_bytes([mod.Desc("burgers", shape, L, "f32", coef=(0.01,), tile=(32, 60))]) > 0
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([mod.Desc("burgers", (64, 64), 3, "f32", coef=(0.01,), tile=(32, 28))])
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([_heat(mod, (64, 64), 3, tile=(32, 60))])
    with pytest.raises(mod.ModilError):
        mod.arena_bytes([mod.Desc("burgers", (64, 64), 3, "f32", coef=(0.01,), tile=(32, 60),
                                  points=[[0.5, 0.0]], point_value=np.zeros(1))])
