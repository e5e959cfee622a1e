"""Reference records made by the library's own forward solves.

The reconstruction problems of Sections 3.2-3.4 take their measurements from
a solution of the forward problem.  Here that solution is this library's:
the same discrete problem with only its initial and boundary conditions
known (no measurements, the heat conductivity held fixed), the levels
minimised on the device with L-BFGS, coarse grids first (nested iteration:
each solution, prolonged, starts the next finer solve).  The
records are made once, before any timed work, and sampled by the callers
(inputs.heat_measurements and the like).

* heat: k(u) = 0.02 exp(-20 (u - 1/2)^2) (Section 3.4) on the conductivity
  nodes (32 nodes, piecewise linear in u), u(x, 0) = g(x) - g(0), zero walls;
* Burgers: the initial condition imposed on every cell of the first row (a
  measurement per cell, nothing else measured), zero walls;
* cavity: Re = 100, the lid and the no-slip walls in the residual, no data.
"""
from __future__ import annotations

import numpy as np

from . import inputs


def _nested(make_desc, shape, n_levels, iters, history, depth):
    """Forward solve by nested iteration: L-BFGS on the problem at
    shape / 2^depth (depth fewer levels) first; the levels of each solution
    become levels 2.. of the next finer problem, whose fine level starts at
    zero, so that it starts from the prolongation of the coarser solution.
    Returns the composed fields of the finest solve and its loss history."""
    from . import modil
    lv = None
    for d in range(depth, -1, -1):
        desc = make_desc(tuple(int(s) >> d for s in shape), n_levels - d)
        with modil.Problem(desc) as p, modil.LBFGS(p, history=history) as opt:
            if lv is not None:
                for f in range(desc.n_fields):
                    fine = [np.zeros(p.level_shape(0))] + lv[f]
                    p.write_levels(fine, field=f)
            hist = opt.run(iters)
            lv = [p.read_levels(field=f) for f in range(desc.n_fields)]
            fields = [p.read_field(field=f) for f in range(desc.n_fields)]
    return fields, hist


def heat_knodes_true(n=inputs.HEAT_KNODES):
    """The reference conductivity sampled on the n nodes u_j = j / (n - 1)."""
    return inputs.heat_k_true(np.arange(n) / (n - 1))


def heat_record(nt=512, nx=512, n_levels=7, knodes=None, iters=2000, history=50, dtype="f64", depth=3):
    """Temperature record u (nt x nx) of the forward heat problem with the
    conductivity nodes `knodes` (default: the reference k) held fixed, and the
    L-BFGS loss history of the finest solve."""
    from . import modil
    q = heat_knodes_true() if knodes is None else np.asarray(knodes, np.float64)

    def make(shape, L):
        return modil.Desc("heat", shape, L, dtype, w_res=1.0, w_data=0.0, w_reg=0.0,
                          aux=inputs.heat_ic(shape[1]), knodes=q, k_fixed=True)
    (u,), hist = _nested(make, (nt, nx), n_levels, iters, history, depth)
    return u, hist


def burgers_record(nt, nx, n_levels, nu, amps, iters=2000, history=50, dtype="f64", depth=0):
    """Space-time Burgers record (nt x nx, x in [-1, 1]) of the forward problem
    from the initial condition sum_k a_k sin(k pi (x + 1) / 2), and the L-BFGS
    loss history."""
    from . import modil

    def make(shape, L):
        n_x = shape[1]
        x = -1.0 + (np.arange(n_x) + 0.5) * (2.0 / n_x)
        return modil.Desc("burgers", shape, L, dtype, coef=(nu,), w_res=1.0, w_data=1.0,
                          meas_cell=np.arange(n_x, dtype=np.int32), meas_value=inputs.burgers_ic(x, amps))
    (u,), hist = _nested(make, (nt, nx), n_levels, iters, history, depth)
    return u, hist


def cavity_record(n=256, n_levels=8, Re=100.0, iters=3000, history=50, dtype="f64", depth=2):
    """Velocity (u, v) and pressure of the lid-driven cavity forward problem on
    n x n cells, and the L-BFGS loss history of the finest solve."""
    from . import modil

    def make(shape, L):
        return modil.Desc("ns2d", shape, L, dtype, coef=(Re, 1.0), w_res=1.0, w_data=0.0)
    (u, v, p), hist = _nested(make, (n, n), n_levels, iters, history, depth)
    return (u, v, p), hist
