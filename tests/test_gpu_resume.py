"""Checkpoint and resume: a run that saves its state, and a fresh problem that
loads it and takes the same steps, agree bit for bit with the uninterrupted
run (levels of every field, Adam state through the next steps, loss terms,
step count); a checkpoint of another problem or a damaged file is refused."""
import os

import numpy as np
import pytest

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


def _state(p, case, n):
    return [[[p.read_level(l, field=f, instance=i) for l in range(case.L)] for f in range(case.nf)]
            for i in range(n)]


@pytest.mark.parametrize("pde,shape,L,dtype,n", [("heat", (64, 96), 4, "f32", 2),
                                                  ("burgers", (64, 64), 4, "f64", 1),
                                                  ("ns2d", (32, 32), 4, "f32", 1),
                                                  ("ns3d", (8, 16, 16), 3, "f32", 1)])
def test_resume_is_bit_identical(modil, tmp_path, pde, shape, L, dtype, n):
    c = Case(pde, shape, L, dtype, seed=90, n_meas=60, lr=2e-3,
             w_reg=0.01 if pde == "heat" else 0.0)
    path = os.path.join(tmp_path, "ckpt.bin")
    with modil.Problem([c.desc()] * n) as a:
        for i in range(n):
            c.load(a, instance=i)
        a.step(7, read_loss=False)           # odd: the levels live in the second buffer
        a.save(path)
        ta = a.step(6)
        want = _state(a, c, n)
        want_q = [a.read_knodes(i) for i in range(n)] if pde == "heat" else None
        steps = a.step_count()
    with modil.Problem([c.desc()] * n) as b:
        b.load(path)
        assert b.step_count() == 7
        tb = b.step(6)
        got = _state(b, c, n)
        np.testing.assert_array_equal(ta, tb)
        assert b.step_count() == steps
        for i in range(n):
            for f in range(c.nf):
                for lvl in range(c.L):
                    np.testing.assert_array_equal(got[i][f][lvl], want[i][f][lvl])
            if pde == "heat":
                np.testing.assert_array_equal(b.read_knodes(i), want_q[i])


def test_load_refuses_other_problems_and_damaged_files(modil, tmp_path):
    c = Case("burgers", (64, 64), 4, "f32", seed=91)
    d = Case("burgers", (64, 128), 4, "f32", seed=91)
    path = os.path.join(tmp_path, "ckpt.bin")
    with modil.Problem(c.desc()) as a:
        c.load(a)
        a.step(3, read_loss=False)
        a.save(path)
        lv = a.read_levels()
    with modil.Problem(d.desc()) as b:
        with pytest.raises(modil.ModilError) as e:
            b.load(path)
        assert e.value.code == modil.ERR_ARG
    bad = os.path.join(tmp_path, "bad.bin")
    with open(path, "rb") as f:
        raw = f.read()
    with open(bad, "wb") as f:
        f.write(raw[: len(raw) // 2])      # truncated
    with modil.Problem(c.desc()) as b:
        c.load(b)
        with pytest.raises(modil.ModilError) as e:
            b.load(bad)
        assert e.value.code == modil.ERR_ARG
        with open(bad, "wb") as f:
            f.write(b"not a checkpoint" * 8)
        with pytest.raises(modil.ModilError):
            b.load(bad)
        with pytest.raises(modil.ModilError):
            b.load(os.path.join(tmp_path, "missing.bin"))
        b.load(path)                       # the intact file still loads
        for lvl, ref in enumerate(lv):
            np.testing.assert_array_equal(b.read_level(lvl), ref)
