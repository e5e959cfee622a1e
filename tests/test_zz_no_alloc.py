"""The allocation-free entry point agrees with the regular one.

modil_eval_grad_noalloc serves callers that cannot allocate device memory
(a host application that owns all device allocations, or a loop that must not
allocate while running): it keeps its working memory in a fixed device array
inside the library instead of an arena.  Here it is called through the C ABI
twice in a row, on two different states, and each result is compared with
modil_eval_grad of a regular problem at the test suite's FP32 tolerance.
This file is collected last so that a failure here leaves every other test
already run.
"""
import numpy as np
import pytest

from _cases import Case, rel

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_04679_gb300 import build
    build.build()
    from paper_2303_04679_gb300 import modil

    c = Case("heat", (128, 192), 5, "f32", seed=31, n_meas=1200, w_reg=0.02)
    states = [c.levels, [np.asarray(a) * 0.5 + 0.1 for a in c.levels]]
    desc = c.desc()
    for lv in states:
        lv = [np.asarray(a, np.float32).astype(np.float64) for a in lv]
        with modil.Problem(desc) as p:
            c.load(p, levels=lv)
            ref_terms = p.eval_grad()[0]
            ref_grads = p.read_grads()
            ref_kg = p.read_kgrad()
        flat = torch.tensor(np.concatenate([a.reshape(-1) for a in lv]), dtype=torch.float32,
                            device="cuda")
        grads = torch.full_like(flat, float("nan"))
        terms, kg = modil.eval_grad_noalloc(desc, flat, grads)
        for j in range(4):
            assert abs(terms[j] - ref_terms[j]) <= TOL32 * max(abs(ref_terms[j]), 1e-300)
        g = grads.cpu().numpy()
        off = 0
        for lvl, r in enumerate(ref_grads):
            n = r.size
            assert rel(g[off:off + n], r.reshape(-1)) <= TOL32, lvl
            off += n
        assert off == g.size
        assert rel(kg, ref_kg) <= TOL32
