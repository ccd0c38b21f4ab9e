"""Thin ctypes binding of include/lsm_nn.h (U-Net warm start and its kernels).

Device tensors are passed as raw pointers (any CUDA buffer; tests and the
warm-start driver use torch tensors purely as storage)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import lsm as _lsm

_P, _I64, _I32, _D, _F, _U64 = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_float, C.c_uint64

SIGNATURES = [
    ("lsm_unet_create", C.c_int, [_I32, _I32, _I32, _U64, _P, C.POINTER(_P)]),
    ("lsm_unet_destroy", None, [_P]),
    ("lsm_unet_last_error", C.c_char_p, [_P]),
    ("lsm_unet_param_count", C.c_int, [_P, _P]),
    ("lsm_unet_get_params", C.c_int, [_P, _P, _I64]),
    ("lsm_unet_set_params", C.c_int, [_P, _P, _I64]),
    ("lsm_unet_forward", C.c_int, [_P, _P, _P, _I32]),
    ("lsm_unet_gradients", C.c_int, [_P, _P, _P, _I32, _P, _P]),
    ("lsm_unet_train_step", C.c_int, [_P, _P, _P, _I32, _F, _P]),
    ("lsm_unet_prepare_input", C.c_int, [_P, _P, _P, _F, _I32, _I32, _I32, _D, _P, _P]),
    ("lsm_unet_prepare_target", C.c_int, [_P, _P, _F, _I32, _I32, _I32, _D, _P, _P]),
    ("lsm_unet_prediction_to_displacement", C.c_int, [_P, _F, _I32, _I32, _I32, _D, _P, _P]),
    ("lsm_nn_conv_forward", C.c_int, [_P, _I32, _I32, _I32, _P, _P, _P, _I32, _I32, _I32, _I32, _I32, _I32,
                                      _I32, _I32, _P]),
    ("lsm_nn_conv_wgrad", C.c_int, [_P, _I32, _P, _I32, _I32, _I32, _I32, _I32, _I32, _I32, _P, _P, _P, _I64,
                                    _P]),
    ("lsm_nn_set_wait_limit", C.c_int, [_I32, _P]),
    ("lsm_batch_fields", C.c_int, [_P, _P, _P, _I32, _I32]),
    ("lsm_batch_add_displacements", C.c_int, [_P, _P, _I32, _I32]),
]

_bound = False


def lib():
    global _bound
    L = _lsm.load_library()
    if not _bound:
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _bound = True
    return L


def check(st, handle=None, batch=False):
    if st != _lsm.LSM_OK:
        if batch:
            from . import batch as _b
            msg = _b._lib().lsm_batch_last_error(handle)
        else:
            msg = lib().lsm_unet_last_error(handle)
        raise _lsm.LsmError(st, msg.decode() if msg else "")


def ptr(t):
    """Raw device pointer of a tensor-like object with data_ptr()."""
    return None if t is None else C.c_void_p(t.data_ptr())


class UNet:
    """stream: cudaStream_t handle to order the network's work on; by default
    torch's current stream, so that torch copies into the input buffers are
    ordered with the network's kernels."""

    def __init__(self, height, width, max_batch, seed=0, stream="torch"):
        if stream == "torch":
            stream = _lsm.torch_stream_handle()
        h = C.c_void_p()
        check(lib().lsm_unet_create(height, width, max_batch, seed, stream, C.byref(h)))
        self.h = h
        self.H, self.W, self.max_batch = height, width, max_batch
        n = C.c_int64()
        check(lib().lsm_unet_param_count(self.h, C.byref(n)), self.h)
        self.nparam = n.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().lsm_unet_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        p = np.empty(self.nparam, np.float32)
        check(lib().lsm_unet_get_params(self.h, p.ctypes.data_as(C.c_void_p), self.nparam), self.h)
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        check(lib().lsm_unet_set_params(self.h, p.ctypes.data_as(C.c_void_p), self.nparam), self.h)

    def forward(self, x, out, batch):
        check(lib().lsm_unet_forward(self.h, ptr(x), ptr(out), batch), self.h)

    def gradients(self, x, target, batch):
        loss = C.c_float()
        g = np.empty(self.nparam, np.float32)
        check(lib().lsm_unet_gradients(self.h, ptr(x), ptr(target), batch, C.byref(loss),
                                       g.ctypes.data_as(C.c_void_p)), self.h)
        return loss.value, g

    def train_step(self, x, target, batch, lr, want_loss=True):
        loss = C.c_float()
        check(lib().lsm_unet_train_step(self.h, ptr(x), ptr(target), batch, float(lr),
                                        C.byref(loss) if want_loss else None), self.h)
        return loss.value if want_loss else None
