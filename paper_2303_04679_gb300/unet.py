"""Python binding of the learned warm start (include/modil_unet.h).

Argument marshalling only: the network runs in libmodil.so's kernels (the
3-D convolutions as im2col GEMMs on the tcgen05 tensor cores).  Device
buffers are torch CUDA tensors; the library raises if it is not built.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import modil as _m

LIB = _m.LIB
_P = C.c_void_p


class unet_desc(C.Structure):
    _fields_ = [("side", C.c_int), ("batch", C.c_int), ("in_ch", C.c_int), ("out_ch", C.c_int),
                ("base_ch", C.c_int), ("levels", C.c_int), ("adam_lr", C.c_double),
                ("adam_beta1", C.c_double), ("adam_beta2", C.c_double), ("adam_eps", C.c_double)]


_SIG = {
    "modil_unet_create": ([C.POINTER(unet_desc), _P, C.POINTER(_P)], C.c_int),
    "modil_unet_destroy": ([_P], None),
    "modil_unet_set_implicit": ([_P, C.c_int], C.c_int),
    "modil_unet_set_graph": ([_P, C.c_int], C.c_int),
    "modil_unet_param_count": ([_P, C.POINTER(C.c_int)], C.c_int),
    "modil_unet_param_shape": ([_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "modil_unet_write_param": ([_P, C.c_int, C.POINTER(C.c_float), C.c_size_t], C.c_int),
    "modil_unet_read_param": ([_P, C.c_int, C.POINTER(C.c_float), C.c_size_t], C.c_int),
    "modil_unet_read_grad": ([_P, C.c_int, C.POINTER(C.c_float), C.c_size_t], C.c_int),
    "modil_unet_forward": ([_P, _P, _P], C.c_int),
    "modil_unet_eval_grad": ([_P, _P, _P, C.POINTER(C.c_double)], C.c_int),
    "modil_unet_train_step": ([_P, _P, _P, C.POINTER(C.c_double)], C.c_int),
    "modil_unet_profile_step": ([_P, _P, _P, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)],
                                C.c_int),
    "modil_gemm_bf16": ([_P, C.c_longlong, _P, C.c_longlong, _P, C.c_longlong, C.c_int, C.c_int,
                         C.c_int, C.c_int, C.c_int, _P, C.c_int, _P], C.c_int),
}
for _n, (_a, _r) in _SIG.items():
    _f = getattr(LIB, _n)
    _f.argtypes = _a
    _f.restype = _r

_check = _m._check


def _ptr(t):
    return None if t is None else t.data_ptr()


def gemm_bf16(A, B, D, mode=0, relu=False, bias=None, splits=1, stream=None):
    """D (+)= A @ B.T on the tensor cores; A [M, K], B [N, K] BF16 CUDA tensors
    (row pitch = their stride), D [M, N] BF16 (mode 0) or FP32 (modes 1, 2)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(LIB.modil_gemm_bf16(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), D.data_ptr(),
                               D.stride(0), M, N, K, mode, int(relu), _ptr(bias), splits,
                               s.cuda_stream))


class UNet:
    """The 3-D U-Net of the warm start; parameters live on the device."""

    def __init__(self, side, batch=1, in_ch=4, out_ch=5, base_ch=32, levels=4, lr=1e-3,
                 beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.side, self.batch, self.in_ch, self.out_ch = side, batch, in_ch, out_ch
        self.base_ch, self.levels = base_ch, levels
        d = unet_desc(side, batch, in_ch, out_ch, base_ch, levels, lr, beta1, beta2, eps)
        h = _P()
        _check(LIB.modil_unet_create(C.byref(d), self.stream.cuda_stream, C.byref(h)))
        self._h = h

    def set_implicit(self, on=True):
        """3x3x3 convolutions as implicit GEMMs (default) or through im2col."""
        _check(LIB.modil_unet_set_implicit(self._h, 1 if on else 0))

    def set_graph(self, on=True):
        """Training steps replayed from a captured CUDA graph (default) or launched directly."""
        _check(LIB.modil_unet_set_graph(self._h, 1 if on else 0))

    def close(self):
        if getattr(self, "_h", None):
            LIB.modil_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- parameters (host numpy FP32, host view) ---------------------------
    def param_shapes(self):
        n = C.c_int()
        _check(LIB.modil_unet_param_count(self._h, C.byref(n)))
        out = []
        for i in range(n.value):
            kind = C.c_int()
            dims = (C.c_int * 3)()
            _check(LIB.modil_unet_param_shape(self._h, i, C.byref(kind), dims))
            out.append((kind.value, tuple(dims)) if kind.value == 0 else (1, (dims[0],)))
        return out

    def write_params(self, params):
        for i, a in enumerate(params):
            a = np.ascontiguousarray(a, dtype=np.float32)
            _check(LIB.modil_unet_write_param(self._h, i, a.ctypes.data_as(C.POINTER(C.c_float)),
                                              a.size))

    def _read(self, fn):
        out = []
        for i, (kind, shape) in enumerate(self.param_shapes()):
            a = np.empty(shape, dtype=np.float32)
            _check(fn(self._h, i, a.ctypes.data_as(C.POINTER(C.c_float)), a.size))
            out.append(a)
        return out

    def read_params(self):
        return self._read(LIB.modil_unet_read_param)

    def read_grads(self):
        return self._read(LIB.modil_unet_read_grad)

    # -- compute (torch CUDA FP32 tensors, channels last) ------------------
    def forward(self, x, out=None):
        import torch
        if out is None:
            out = torch.empty(x.shape[:-1] + (self.out_ch,), dtype=torch.float32, device=x.device)
        self.stream.wait_stream(torch.cuda.current_stream())
        _check(LIB.modil_unet_forward(self._h, x.data_ptr(), out.data_ptr()))
        torch.cuda.current_stream().wait_stream(self.stream)
        return out

    def eval_grad(self, x, y):
        import torch
        loss = C.c_double()
        self.stream.wait_stream(torch.cuda.current_stream())
        _check(LIB.modil_unet_eval_grad(self._h, x.data_ptr(), y.data_ptr(), C.byref(loss)))
        return loss.value

    def train_step(self, x, y, read_loss=True):
        import torch
        loss = C.c_double()
        self.stream.wait_stream(torch.cuda.current_stream())
        _check(LIB.modil_unet_train_step(self._h, x.data_ptr(), y.data_ptr(),
                                         C.byref(loss) if read_loss else None))
        return loss.value if read_loss else None

    def profile_step(self, x, y, max_launches=512):
        ms = (C.c_float * max_launches)()
        n = C.c_int()
        _check(LIB.modil_unet_profile_step(self._h, x.data_ptr(), y.data_ptr(), ms, max_launches,
                                           C.byref(n)))
        return np.array(ms[:n.value])
