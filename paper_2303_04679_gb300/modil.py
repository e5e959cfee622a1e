"""Thin Python binding of libmodil.so (argument marshalling only).

Every step of the method runs in the library's CUDA kernels; this module only
converts Python/numpy/torch arguments into the C ABI declared in
``include/modil.h``.  There is no CPU fallback: if the shared library is
missing, importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libmodil.so")

PDE_BURGERS = 1
PDE_HEAT = 2
PDE_NS2D = 3
PDE_NS3D = 4
PDE_POISSON = 5
F32 = 0
F64 = 1
NTERMS = 4
TERM_NAMES = ("total", "res", "data", "reg")
MAX_LEVELS = 10

STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_UNSUPPORTED",
          -5: "ERR_NONFINITE", -6: "ERR_STATE", -7: "ERR_TIMEOUT"}
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED, ERR_NONFINITE, ERR_STATE, ERR_TIMEOUT = -1, -2, -3, -4, -5, -6, -7


class ModilError(RuntimeError):
    def __init__(self, code, msg):
        self.code = code
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class modil_desc(C.Structure):
    _fields_ = [
        ("pde", C.c_int), ("dtype", C.c_int), ("ndim", C.c_int), ("shape", C.c_int * 3),
        ("n_levels", C.c_int), ("coef", C.c_double * 4), ("w_res", C.c_double),
        ("w_data", C.c_double), ("w_reg", C.c_double), ("n_meas", C.c_int),
        ("meas_cell", C.POINTER(C.c_int32)), ("meas_field", C.POINTER(C.c_int32)),
        ("meas_value", C.POINTER(C.c_double)), ("n_aux", C.c_int),
        ("aux", C.POINTER(C.c_double)), ("n_knodes", C.c_int),
        ("knodes", C.POINTER(C.c_double)), ("adam_lr", C.c_double),
        ("adam_beta1", C.c_double), ("adam_beta2", C.c_double), ("adam_eps", C.c_double),
        ("n_points", C.c_int), ("point_coord", C.POINTER(C.c_double)),
        ("point_value", C.POINTER(C.c_double)),
        ("tile", C.c_int * 2),
        ("domain_lo", C.c_double * 3), ("domain_hi", C.c_double * 3),
        ("point_field", C.POINTER(C.c_int32)), ("layout", C.c_int), ("k_fixed", C.c_int),
        ("k_scale", C.c_double),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmodil.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "modil_arena_bytes": ([C.POINTER(modil_desc), C.c_int, C.POINTER(C.c_size_t)], C.c_int),
        "modil_create": ([C.POINTER(modil_desc), C.c_int, P, C.c_size_t, P, C.POINTER(P)], C.c_int),
        "modil_destroy": ([P], None),
        "modil_set_stream": ([P, P], C.c_int),
        "modil_level_shape": ([P, C.c_int, C.c_int, C.POINTER(C.c_int)], C.c_int),
        "modil_write_level": ([P, C.c_int, C.c_int, C.c_int, P, C.c_size_t, C.c_int], C.c_int),
        "modil_read_level": ([P, C.c_int, C.c_int, C.c_int, P, C.c_size_t, C.c_int], C.c_int),
        "modil_read_grad": ([P, C.c_int, C.c_int, C.c_int, P, C.c_size_t, C.c_int], C.c_int),
        "modil_read_field": ([P, C.c_int, C.c_int, P, C.c_size_t, C.c_int], C.c_int),
        "modil_write_knodes": ([P, C.c_int, C.POINTER(C.c_double), C.c_int], C.c_int),
        "modil_read_knodes": ([P, C.c_int, C.POINTER(C.c_double), C.c_int], C.c_int),
        "modil_read_kgrad": ([P, C.c_int, C.POINTER(C.c_double), C.c_int], C.c_int),
        "modil_eval_loss": ([P, C.POINTER(C.c_double)], C.c_int),
        "modil_eval_grad": ([P, C.POINTER(C.c_double)], C.c_int),
        "modil_step": ([P, C.c_int, C.POINTER(C.c_double)], C.c_int),
        "modil_step_count": ([P, C.POINTER(C.c_longlong)], C.c_int),
        "modil_launches_per_step": ([P, C.POINTER(C.c_int)], C.c_int),
        "modil_profile_step": ([P, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)], C.c_int),
        "modil_reset_optimizer": ([P], C.c_int),
        "modil_set_persistent": ([P, C.c_int], C.c_int),
        "modil_param_count": ([P, C.POINTER(C.c_longlong)], C.c_int),
        "modil_level_offset": ([P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_longlong)], C.c_int),
        "modil_loss_fwd": ([P, P, C.POINTER(C.c_double)], C.c_int),
        "modil_loss_bwd": ([P, P, C.c_double, P], C.c_int),
        "modil_terms_device": ([P, C.POINTER(C.c_void_p), C.POINTER(C.c_int)], C.c_int),
        "modil_eval_grad_noalloc": ([C.POINTER(modil_desc), P, P, C.POINTER(C.c_double),
                                     C.POINTER(C.c_double), P], C.c_int),
        "modil_lbfgs_create": ([P, C.c_int, C.POINTER(P)], C.c_int),
        "modil_lbfgs_run": ([P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)], C.c_int),
        "modil_lbfgs_destroy": ([P], None),
        "modil_last_error": ([], C.c_char_p),
        "modil_version": ([], C.c_char_p),
        "modil_desc_size": ([], C.c_size_t),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if lib.modil_desc_size() != C.sizeof(modil_desc):
        raise ImportError(f"libmodil.so's modil_desc is {lib.modil_desc_size()} bytes, this binding's "
                          f"{C.sizeof(modil_desc)}: rebuild the library")
    return lib


LIB = _load()


def _check(code):
    if code != 0:
        raise ModilError(code, LIB.modil_last_error().decode())


def _dptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


class Desc:
    """One problem description; keeps its numpy buffers alive for the C struct."""

    def __init__(self, pde, shape, n_levels, dtype="f32", coef=(), w_res=1.0, w_data=1.0,
                 w_reg=0.0, meas_cell=None, meas_value=None, meas_field=None, aux=None,
                 knodes=None, lr=5e-3, beta1=0.9, beta2=0.999, eps=1e-8, tile=(0, 0),
                 points=None, point_value=None, domain=None, point_field=None, layout="cell",
                 k_fixed=False, k_scale=0.0):
        self.kwargs = dict(pde=pde, shape=shape, n_levels=n_levels, dtype=dtype, coef=coef,
                           w_res=w_res, w_data=w_data, w_reg=w_reg, meas_cell=meas_cell,
                           meas_value=meas_value, meas_field=meas_field, aux=aux, knodes=knodes,
                           lr=lr, beta1=beta1, beta2=beta2, eps=eps, tile=tile, points=points,
                           point_value=point_value, domain=domain, point_field=point_field,
                           layout=layout, k_fixed=k_fixed, k_scale=k_scale)
        self.pde = {"burgers": PDE_BURGERS, "heat": PDE_HEAT, "ns2d": PDE_NS2D,
                    "ns3d": PDE_NS3D, "poisson": PDE_POISSON}.get(pde, pde)
        self.dtype = {"f32": F32, "f64": F64}.get(dtype, dtype)
        self.shape = tuple(int(s) for s in shape)
        self.n_levels = int(n_levels)
        self._cell = None if meas_cell is None else np.ascontiguousarray(meas_cell, np.int32)
        self._val = None if meas_value is None else np.ascontiguousarray(meas_value, np.float64)
        self._field = None if meas_field is None else np.ascontiguousarray(meas_field, np.int32)
        self._aux = None if aux is None else np.ascontiguousarray(aux, np.float64)
        self._knodes = None if knodes is None else np.ascontiguousarray(knodes, np.float64)
        nd = 3 if self.pde == PDE_NS3D else 2
        self._pts = None if points is None else np.ascontiguousarray(np.reshape(points, (-1, nd)), np.float64)
        self._pfield = None if point_field is None else np.ascontiguousarray(point_field, np.int32)
        self._pval = None if point_value is None else np.ascontiguousarray(point_value, np.float64)
        # the C planner reads these arrays up to n_meas / n_points entries
        n_cells = 0 if self._cell is None else len(self._cell)
        if n_cells and (self._val is None or len(self._val) != n_cells):
            raise ValueError("meas_value needs one value per measurement cell")
        if self._field is not None and len(self._field) != n_cells:
            raise ValueError("meas_field needs one field index per measurement cell")
        n_pts = 0 if self._pts is None else len(self._pts)
        if n_pts and (self._pval is None or len(self._pval) != n_pts):
            raise ValueError("point_value needs one value per off-grid point")
        if self._pfield is not None and len(self._pfield) != n_pts:
            raise ValueError("point_field needs one field index per off-grid point")
        d = modil_desc()
        d.pde, d.dtype, d.ndim = self.pde, self.dtype, len(self.shape)
        for i, s in enumerate(self.shape):
            d.shape[i] = s
        d.n_levels = self.n_levels
        for i, c in enumerate(coef):
            d.coef[i] = float(c)
        d.w_res, d.w_data, d.w_reg = float(w_res), float(w_data), float(w_reg)
        d.n_meas = 0 if self._cell is None else len(self._cell)
        d.meas_cell = _dptr(self._cell, C.c_int32)
        d.meas_value = _dptr(self._val, C.c_double)
        d.meas_field = _dptr(self._field, C.c_int32)
        d.n_aux = 0 if self._aux is None else len(self._aux)
        d.aux = _dptr(self._aux, C.c_double)
        d.n_knodes = 0 if self._knodes is None else len(self._knodes)
        d.knodes = _dptr(self._knodes, C.c_double)
        d.adam_lr, d.adam_beta1, d.adam_beta2, d.adam_eps = lr, beta1, beta2, eps
        d.n_points = 0 if self._pts is None else len(self._pts)
        d.point_coord = _dptr(self._pts, C.c_double)
        d.point_value = _dptr(self._pval, C.c_double)
        d.point_field = _dptr(self._pfield, C.c_int32)
        self.layout = {"cell": 0, "node": 1}.get(layout, layout)
        d.layout = self.layout
        d.k_fixed = 1 if k_fixed else 0
        d.k_scale = float(k_scale)
        d.tile[0], d.tile[1] = int(tile[0]), int(tile[1])
        if domain is not None:  # ((lo, hi) per axis, slowest first)
            for a, (lo, hi) in enumerate(domain):
                d.domain_lo[a], d.domain_hi[a] = float(lo), float(hi)
        self.c = d

    @property
    def np_dtype(self):
        return np.float64 if self.dtype == F64 else np.float32

    @property
    def n_fields(self):
        return {PDE_NS2D: 3, PDE_NS3D: 5}.get(self.pde, 1)

    def param_count(self):
        """Unknowns of the levels: fields x sum over levels of the cells of each
        level (every axis halved per level)."""
        per_field = 0
        extra = 1 if getattr(self, "layout", 0) == 1 else 0
        for lvl in range(self.n_levels):
            n = 1
            for s in self.shape:
                n *= (s >> lvl) + extra
            per_field += n
        return self.n_fields * per_field


def _desc_array(descs):
    arr = (modil_desc * len(descs))()
    for i, d in enumerate(descs):
        arr[i] = d.c
    return arr


def arena_bytes(descs):
    out = C.c_size_t(0)
    _check(LIB.modil_arena_bytes(_desc_array(descs), len(descs), C.byref(out)))
    return out.value


class Problem:
    """A batch of mODIL problems living on the current CUDA device.

    arena="torch" lets PyTorch own the device memory (a uint8 tensor);
    arena="library" makes the library cudaMalloc it.  ``stream`` is a
    torch.cuda.Stream (default: a new one, so steps replay as a CUDA graph).
    """

    def __init__(self, descs, arena="torch", stream=None):
        import torch
        if isinstance(descs, Desc):
            descs = [descs]
        self.descs = list(descs)
        self._arr = _desc_array(self.descs)
        self.n = len(self.descs)
        self.np_dtype = self.descs[0].np_dtype
        self.stream = stream if stream is not None else torch.cuda.Stream()
        nbytes = arena_bytes(self.descs)
        self._arena = None
        aptr = None
        if arena == "torch":
            self._arena = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._arena.data_ptr()
            aptr = (base + 255) & ~255
        self._h = C.c_void_p()
        _check(LIB.modil_create(self._arr, self.n, aptr, nbytes, self.stream.cuda_stream,
                                C.byref(self._h)))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            LIB.modil_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- shapes ----------------------------------------------------------
    def level_shape(self, level, instance=0):
        s = (C.c_int * 3)()
        _check(LIB.modil_level_shape(self._h, instance, level, s))
        return tuple(v for v in (s[0], s[1], s[2]) if v)

    def n_levels(self, instance=0):
        return self.descs[instance].n_levels

    # -- level I/O (host numpy or device torch tensors) ---------------------
    def write_level(self, level, values, field=0, instance=0):
        if hasattr(values, "data_ptr"):
            _check(LIB.modil_write_level(self._h, instance, field, level, values.data_ptr(),
                                         values.numel() * values.element_size(), 1))
            return
        a = np.ascontiguousarray(values, dtype=self.np_dtype)
        _check(LIB.modil_write_level(self._h, instance, field, level, a.ctypes.data, a.nbytes, 0))

    def write_levels(self, levels, field=0, instance=0):
        for i, a in enumerate(levels):
            self.write_level(i, a, field, instance)

    def write_fields(self, levels_per_field, instance=0):
        for f, lv in enumerate(levels_per_field):
            self.write_levels(lv, f, instance)

    def _read(self, fn, level, field, instance, shape):
        out = np.empty(shape, dtype=self.np_dtype)
        _check(fn(self._h, instance, field, level, out.ctypes.data, out.nbytes, 0))
        return out

    def read_level(self, level, field=0, instance=0):
        return self._read(LIB.modil_read_level, level, field, instance, self.level_shape(level, instance))

    def read_levels(self, field=0, instance=0):
        return [self.read_level(l, field, instance) for l in range(self.n_levels(instance))]

    def read_grad(self, level, field=0, instance=0):
        return self._read(LIB.modil_read_grad, level, field, instance, self.level_shape(level, instance))

    def read_grads(self, field=0, instance=0):
        return [self.read_grad(l, field, instance) for l in range(self.n_levels(instance))]

    def read_field(self, field=0, instance=0):
        out = np.empty(self.level_shape(0, instance), dtype=self.np_dtype)
        _check(LIB.modil_read_field(self._h, instance, field, out.ctypes.data, out.nbytes, 0))
        return out

    def write_knodes(self, q, instance=0):
        q = np.ascontiguousarray(q, dtype=np.float64)
        _check(LIB.modil_write_knodes(self._h, instance, _dptr(q, C.c_double), len(q)))

    def _kio(self, fn, instance):
        q = np.empty(len(self.descs[instance]._knodes), dtype=np.float64)
        _check(fn(self._h, instance, _dptr(q, C.c_double), len(q)))
        return q

    def read_knodes(self, instance=0):
        return self._kio(LIB.modil_read_knodes, instance)

    def read_kgrad(self, instance=0):
        return self._kio(LIB.modil_read_kgrad, instance)

    # -- evaluation and steps ------------------------------------------------
    def _terms(self):
        return np.zeros(self.n * NTERMS, dtype=np.float64)

    def eval_loss(self):
        t = self._terms()
        _check(LIB.modil_eval_loss(self._h, _dptr(t, C.c_double)))
        return t.reshape(self.n, NTERMS)

    def eval_grad(self):
        t = self._terms()
        _check(LIB.modil_eval_grad(self._h, _dptr(t, C.c_double)))
        return t.reshape(self.n, NTERMS)

    def step(self, n=1, read_loss=True):
        if read_loss:
            t = self._terms()
            _check(LIB.modil_step(self._h, int(n), _dptr(t, C.c_double)))
            return t.reshape(self.n, NTERMS)
        _check(LIB.modil_step(self._h, int(n), None))
        return None

    def step_count(self):
        t = C.c_longlong()
        _check(LIB.modil_step_count(self._h, C.byref(t)))
        return t.value

    def launches_per_step(self):
        n = C.c_int()
        _check(LIB.modil_launches_per_step(self._h, C.byref(n)))
        return n.value

    def profile_labels(self):
        """Names of the launches profile_step times, in order ("compose_L2",
        "fine", "restrict_L1", ..., "tail")."""
        cap = 64
        kind, level = (C.c_int * cap)(), (C.c_int * cap)()
        n = C.c_int()
        _check(LIB.modil_profile_labels(self._h, kind, level, cap, C.byref(n)))
        names = {0: "compose_L{}", 1: "fine", 2: "restrict_L{}", 3: "tail"}
        return [names[kind[i]].format(level[i]) for i in range(n.value)]

    def profile_step(self):
        """One step launched kernel by kernel; returns the device ms of each launch."""
        cap = 64
        ms = (C.c_float * cap)()
        n = C.c_int()
        _check(LIB.modil_profile_step(self._h, ms, cap, C.byref(n)))
        return [ms[i] for i in range(n.value)]

    def param_count(self):
        n = C.c_longlong()
        _check(LIB.modil_param_count(self._h, C.byref(n)))
        return n.value

    def level_offset(self, level, field=0, instance=0):
        o = C.c_longlong()
        _check(LIB.modil_level_offset(self._h, instance, field, level, C.byref(o)))
        return o.value

    def loss_fwd(self, levels):
        """Loss terms of caller-owned levels (device tensor, parameter-vector layout)."""
        t = self._terms()
        _check(LIB.modil_loss_fwd(self._h, levels.data_ptr(), _dptr(t, C.c_double)))
        return t.reshape(self.n, NTERMS)

    def loss_fwd_async(self, levels):
        """Launch the loss pass of caller-owned levels without waiting; the terms
        are then read on the device (terms_device)."""
        _check(LIB.modil_loss_fwd(self._h, levels.data_ptr(), None))

    def terms_device(self):
        """[n_instances, 4] FP64 torch view of the loss terms in device memory
        (total, residual, data, regulariser), overwritten by every pass."""
        import torch
        ptr = C.c_void_p()
        stride = C.c_int()
        _check(LIB.modil_terms_device(self._h, C.byref(ptr), C.byref(stride)))
        n = (self.n - 1) * stride.value + NTERMS

        class _View:  # device memory owned by the problem
            __cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr.value, False),
                                        "version": 3, "strides": None}
        flat = torch.as_tensor(_View(), device="cuda")
        return flat.as_strided((self.n, NTERMS), (stride.value, 1))

    def loss_bwd(self, levels, grad_out, grads):
        """grads <- grad_out * dL/dlevels (device tensors, parameter-vector layout)."""
        _check(LIB.modil_loss_bwd(self._h, levels.data_ptr(), float(grad_out), grads.data_ptr()))

    def save(self, path):
        """Write the optimiser state (levels, Adam moments, step count) to a file."""
        _check(LIB.modil_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Continue from a file written by save() of a problem with the same descriptors."""
        _check(LIB.modil_load(self._h, os.fsencode(path)))

    def set_persistent(self, on=True):
        _check(LIB.modil_set_persistent(self._h, 1 if on else 0))

    def reset_optimizer(self):
        _check(LIB.modil_reset_optimizer(self._h))


class LBFGS:
    """Limited-memory BFGS on the levels of a single-instance problem (the
    library's two-loop recursion and Armijo backtracking on the device; see
    modil_lbfgs_create).  The problem must outlive the optimiser."""

    def __init__(self, problem, history=50):
        self.problem = problem
        h = C.c_void_p()
        _check(LIB.modil_lbfgs_create(problem._h, int(history), C.byref(h)))
        self._h = h

    def run(self, iterations):
        """Up to `iterations` iterations from the problem's current levels;
        returns the loss at the start and after each completed iteration."""
        loss = np.zeros(int(iterations) + 1, dtype=np.float64)
        done = C.c_int()
        _check(LIB.modil_lbfgs_run(self._h, int(iterations), _dptr(loss, C.c_double), C.byref(done)))
        return loss[:done.value + 1]

    def close(self):
        if getattr(self, "_h", None):
            LIB.modil_lbfgs_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def eval_grad_noalloc(desc, levels, grads, stream=None):
    """Loss and gradient of one problem with no device allocation.

    ``levels`` and ``grads`` are contiguous device tensors of the problem's
    dtype holding every field's levels back to back (field-major; within a
    field level 0 first, each row-major), 16-byte aligned; returns (terms,
    kgrad).  The library keeps its working memory in a fixed 8 MiB device
    array, for callers that cannot allocate.
    """
    import torch
    want = torch.float64 if desc.dtype == F64 else torch.float32
    n = desc.param_count()
    for name, t in (("levels", levels), ("grads", grads)):
        if not t.is_cuda or not t.is_contiguous() or t.dtype != want or t.numel() != n:
            raise ValueError(f"{name}: need a contiguous CUDA tensor of {want} with {n} elements, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")
        if t.data_ptr() % 16:
            raise ValueError(f"{name}: must start on a 16-byte boundary")
    s = stream if stream is not None else torch.cuda.current_stream()
    terms = np.zeros(NTERMS, dtype=np.float64)
    nk = 0 if desc._knodes is None else len(desc._knodes)
    kg = np.zeros(max(nk, 1), dtype=np.float64)
    _check(LIB.modil_eval_grad_noalloc(C.byref(desc.c), levels.data_ptr(), grads.data_ptr(),
                                       _dptr(terms, C.c_double),
                                       _dptr(kg, C.c_double) if nk else None, s.cuda_stream))
    return terms, kg[:nk]


def version():
    return LIB.modil_version().decode()
