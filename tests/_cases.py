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
                 fine_lo=None, fine_hi=None, coarse_scale=None, Re=100.0, tau=1.0, D=0.4,
                 lam=1.0, chi_shift=5.0, k_fixed=False, k_scale=1.0):
        self.pde, self.shape, self.L, self.dtype = pde, tuple(shape), L, dtype
        self.npd = np.float64 if dtype == "f64" else np.float32
        nx = shape[-1]
        ncell = int(np.prod(shape))
        rng = np.random.default_rng(seed + 17)
        n_meas = min(n_meas, ncell)
        cells = inputs.measurement_cells(ncell, n_meas, seed)
        if duplicate:
            cells = np.concatenate([cells, cells[:duplicate]]).astype(np.int32)
        vals = rnd(rng.uniform(-0.5, 1.2, size=len(cells)), self.npd)
        self.nf = {"ns2d": 3, "ns3d": 5}.get(pde, 1)
        mfield = None
        if pde in ("ns2d", "ns3d"):
            # velocity samples: u or v (cavity), u, v or w (body)
            mfield = (rng.integers(0, 2 if pde == "ns2d" else 3, size=len(cells))).astype(np.int32)
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
        if pde in ("ns2d", "ns3d"):
            lo, hi, cs = -0.5, 0.5, 0.2
            lo = lo if fine_lo is None else fine_lo
            hi = hi if fine_hi is None else fine_hi
            cs = cs if coarse_scale is None else coarse_scale
            self.levels = inputs.random_levels(shape, L, self.nf, seed, lo, hi, cs, dtype=self.npd)
            if pde == "ns3d":
                # body-fraction logits around chihat = 5 (chi near 1/2) so that
                # both the flow and the penalisation terms are exercised
                self.levels[4][0] = rnd(self.levels[4][0] * 8.0 + chi_shift, self.npd)
        else:
            self.levels = inputs.random_levels(shape, L, 1, seed, lo, hi, cs, dtype=self.npd)[0]
        coef = {"burgers": {"nu": nu}, "ns2d": {"Re": Re, "tau": tau},
                "ns3d": {"Re": Re, "D": D, "lam": lam, "tau": tau}}.get(pde, {})
        self.oracle = o.Problem(pde, self.shape, L, coef=coef, w_res=w_res, w_data=w_data,
                                w_reg=w_reg, meas_cell=cells, meas_value=vals, aux=self.aux,
                                meas_field=mfield, k_fixed=k_fixed, k_scale=k_scale)
        dcoef = {"burgers": (nu,), "ns2d": (Re, tau), "ns3d": (Re, D, lam, tau)}.get(pde, ())
        self.desc_kw = dict(pde=pde, shape=self.shape, n_levels=L, dtype=dtype,
                            coef=dcoef, w_res=w_res, w_data=w_data,
                            w_reg=w_reg, meas_cell=cells, meas_value=vals, meas_field=mfield,
                            aux=self.aux, knodes=self.q, lr=lr, tile=tile, k_fixed=k_fixed,
                            k_scale=0.0 if k_scale == 1.0 else k_scale)
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


# (field, level) pairs of the criterion's floor, per PDE: the cavity's
# pressure on the coarse levels, whose constant mode only the single gauge
# residual sees, so their gradients are sums of terms that cancel to far
# below the terms' size (reading R14).  Everywhere else the error is measured
# against ||g_ref|| alone.
FLOOR_PAIRS = {"ns2d": lambda f, lvl: f == 2 and lvl >= 1}

# what the last check_loss_grad call compared: (field, level, branch, ratio),
# branch "ref" (against ||g_ref||) or "terms" (against 0.1 ||A||)
LAST_CRITERIA = []


def check_loss_grad(case, prob, tol, instance=0, levels=None, q=None, check_max=True):
    """Compare loss terms, every level gradient and dL/dq with the oracle.

    Gradient criterion per (field, level): ||g - g_ref|| <= tol ||g_ref||.
    Only for the pairs FLOOR_PAIRS names (the cavity's coarse pressure levels)
    is the scale max(||g_ref||, 0.1 ||A||), A = the absolute-value restriction
    of |dL/du_fine| to that level: there the terms of the gradient cancel to
    much less than their size, and FP32 cannot resolve the sum below the size
    of its terms.  LAST_CRITERIA records which scale each comparison used."""
    terms_ref, grads_ref, gq_ref = case.oracle_eval(levels, q)
    t = prob.eval_grad()[instance]
    for j, name in enumerate(("total", "res", "data", "reg")):
        ref = terms_ref[name]
        assert abs(t[j] - ref) <= tol * max(abs(ref), 1e-300), (name, t[j], ref)
    per_field = grads_ref if case.nf > 1 else [grads_ref]
    floor = FLOOR_PAIRS.get(case.pde, lambda f, lvl: False)
    LAST_CRITERIA.clear()
    for f, grads_f in enumerate(per_field):
        absl = abs_chain(grads_f[0], len(grads_f))
        for lvl, gr in enumerate(grads_f):
            g = prob.read_grad(lvl, field=f, instance=instance).astype(np.float64)
            nref = np.linalg.norm(gr)
            use_floor = floor(f, lvl) and 0.1 * np.linalg.norm(absl[lvl]) > nref
            scale = 0.1 * np.linalg.norm(absl[lvl]) if use_floor else nref
            r = np.linalg.norm(g - gr) / (scale if scale > 0 else 1.0)
            branch = "terms" if use_floor else "ref"
            LAST_CRITERIA.append((f, lvl, branch, r))
            assert r <= tol, ("field", f, "level", lvl, branch, r)
            if check_max:
                err = np.max(np.abs(g - gr))
                mscale = np.max(np.abs(gr))
                if floor(f, lvl):
                    mscale = max(mscale, 0.1 * np.max(absl[lvl]))
                assert err <= 10 * tol * mscale, ("level max", f, lvl, branch, err, mscale)
    if case.pde == "heat":
        gq = prob.read_kgrad(instance)
        assert rel(gq, gq_ref) <= tol, ("kgrad", rel(gq, gq_ref))
    return terms_ref, grads_ref, gq_ref
