"""Matched problem builders: the same seeded inputs for the oracle and the CUDA path.

Inputs come from ``paper_2303_04679_gb300.inputs`` and are rounded to the
device dtype first, so both sides start from identical numbers.  Nothing here
computes any part of the method.
"""
import numpy as np

import oracle as o
from paper_2303_04679_gb300 import inputs


def rnd(a, dtype):
    return np.asarray(a, dtype=np.float64).astype(dtype).astype(np.float64)


class Case:
    def __init__(self, pde, shape, L, dtype="f32", seed=0, n_meas=50, nu=0.01, w_res=1.0,
                 w_data=1.0, w_reg=0.0, lr=5e-3, tile=(0, 0), duplicate=0, n_knodes=32,
                 fine_lo=None, fine_hi=None, coarse_scale=None, Re=100.0, tau=1.0):
        self.pde, self.shape, self.L, self.dtype = pde, tuple(shape), L, dtype
        self.npd = np.float64 if dtype == "f64" else np.float32
        nt, nx = shape
        rng = np.random.default_rng(seed + 17)
        n_meas = min(n_meas, nt * nx)
        cells = inputs.measurement_cells(nt * nx, n_meas, seed)
        if duplicate:
            cells = np.concatenate([cells, cells[:duplicate]]).astype(np.int32)
        vals = rnd(rng.uniform(-0.5, 1.2, size=len(cells)), self.npd)
        self.nf = 3 if pde == "ns2d" else 1
        mfield = None
        if pde == "ns2d":
            mfield = (rng.integers(0, 2, size=len(cells))).astype(np.int32)  # u or v samples
            vals = rnd(rng.normal(0.0, 0.3, size=len(cells)), self.npd)
        self.aux = None
        self.q = None
        if pde == "heat":
            self.aux = rnd(inputs.heat_ic(nx), self.npd)
            self.q = rnd(rng.uniform(0.005, 0.03, size=n_knodes), self.npd)
            lo, hi, cs = -0.15, 1.15, 0.1
        else:
            lo, hi, cs = -1.0, 1.0, 0.5
        lo = lo if fine_lo is None else fine_lo
        hi = hi if fine_hi is None else fine_hi
        cs = cs if coarse_scale is None else coarse_scale
        if pde == "ns2d":
            lo, hi, cs = -0.5, 0.5, 0.2
            lo = lo if fine_lo is None else fine_lo
            hi = hi if fine_hi is None else fine_hi
            cs = cs if coarse_scale is None else coarse_scale
            self.levels = inputs.random_levels(shape, L, 3, seed, lo, hi, cs, dtype=self.npd)
        else:
            self.levels = inputs.random_levels(shape, L, 1, seed, lo, hi, cs, dtype=self.npd)[0]
        coef = {"nu": nu} if pde == "burgers" else ({"Re": Re, "tau": tau} if pde == "ns2d" else {})
        self.oracle = o.Problem(pde, self.shape, L, coef=coef, w_res=w_res, w_data=w_data,
                                w_reg=w_reg, meas_cell=cells, meas_value=vals, aux=self.aux,
                                meas_field=mfield)
        dcoef = (nu,) if pde == "burgers" else ((Re, tau) if pde == "ns2d" else ())
        self.desc_kw = dict(pde=pde, shape=self.shape, n_levels=L, dtype=dtype,
                            coef=dcoef, w_res=w_res, w_data=w_data,
                            w_reg=w_reg, meas_cell=cells, meas_value=vals, meas_field=mfield,
                            aux=self.aux, knodes=self.q, lr=lr, tile=tile)
        self.lr = lr

    def desc(self):
        from paper_2303_04679_gb300 import modil
        return modil.Desc(**self.desc_kw)

    def load(self, prob, instance=0, levels=None, q=None):
        lv = self.levels if levels is None else levels
        if self.nf > 1:
            prob.write_fields(lv, instance=instance)
            return
        prob.write_levels(lv, instance=instance)
        if self.pde == "heat":
            prob.write_knodes(self.q if q is None else q, instance=instance)

    def oracle_eval(self, levels=None, q=None):
        lv = self.levels if levels is None else levels
        qq = self.q if q is None else q
        return o.loss_grad_levels(self.oracle, lv, qq)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def abs_chain(g_fine, n_levels):
    """|T_i|^T ... applied to |dL/du|: the sum of absolute terms each level
    gradient is formed from (the scale FP32 summation error is bounded by)."""
    out = [np.abs(np.asarray(g_fine, dtype=np.float64))]
    for _ in range(n_levels - 1):
        a = out[-1]
        for ax in range(a.ndim):
            M = np.abs(o.interp_matrix(a.shape[ax] // 2)).T
            a = np.moveaxis(np.tensordot(M, np.moveaxis(a, ax, 0), axes=(1, 0)), 0, ax)
        out.append(a)
    return out


def check_loss_grad(case, prob, tol, instance=0, levels=None, q=None, check_max=True):
    """Compare loss terms, every level gradient and dL/dq with the oracle.

    Gradient criterion per (field, level): ||g - g_ref|| <= tol * max(||g_ref||,
    0.1 ||A||), A = the absolute-value restriction of |dL/du_fine| to that
    level.  Where the terms of a coarse-level gradient cancel to much less than
    their size (the pressure levels of the cavity, whose constant mode only
    the gauge term sees), the error is measured against the terms."""
    terms_ref, grads_ref, gq_ref = case.oracle_eval(levels, q)
    t = prob.eval_grad()[instance]
    for j, name in enumerate(("total", "res", "data", "reg")):
        ref = terms_ref[name]
        assert abs(t[j] - ref) <= tol * max(abs(ref), 1e-300), (name, t[j], ref)
    per_field = grads_ref if case.nf > 1 else [grads_ref]
    for f, grads_f in enumerate(per_field):
        absl = abs_chain(grads_f[0], len(grads_f))
        for lvl, gr in enumerate(grads_f):
            g = prob.read_grad(lvl, field=f, instance=instance).astype(np.float64)
            scale = max(np.linalg.norm(gr), 0.1 * np.linalg.norm(absl[lvl]))
            r = np.linalg.norm(g - gr) / (scale if scale > 0 else 1.0)
            assert r <= tol, ("field", f, "level", lvl, r)
            if check_max:
                err = np.max(np.abs(g - gr))
                mscale = max(np.max(np.abs(gr)), 0.1 * np.max(absl[lvl]))
                assert err <= 10 * tol * mscale, ("level max", f, lvl, err, mscale)
    if case.pde == "heat":
        gq = prob.read_kgrad(instance)
        assert rel(gq, gq_ref) <= tol, ("kgrad", rel(gq, gq_ref))
    return terms_ref, grads_ref, gq_ref
