"""Thin ctypes binding of the batched C ABI (include/lsm_batch.h)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import lsm as _lsm

_P, _I64, _I32, _D = C.c_void_p, C.c_int64, C.c_int32, C.c_double

SIGNATURES = [
    ("lsm_build_batch", C.c_int, [_P, _I32, C.POINTER(_P)]),
    ("lsm_batch_destroy", None, [_P]),
    ("lsm_batch_last_error", C.c_char_p, [_P]),
    ("lsm_batch_sizes", C.c_int, [_P, _I32, _P, _P, _P]),
    ("lsm_batch_autotune", C.c_int, [_P, _I32, _P, _P, _P, _P]),
    ("lsm_batch_set_schedule", C.c_int, [_P, _I32, _I32, _I32]),
    ("lsm_batch_apply_strain", C.c_int, [_P, _P]),
    ("lsm_batch_step", C.c_int, [_P, _I64]),
    ("lsm_batch_relax", C.c_int, [_P, _D, _I64, _I64, _P, _P]),
    ("lsm_batch_samples", C.c_int, [_P, _I32, _P, _I64, _P]),
    ("lsm_batch_get_state", C.c_int, [_P, _I32, _P, _P]),
    ("lsm_batch_set_state", C.c_int, [_P, _I32, _P, _P]),
    ("lsm_batch_broken_mask", C.c_int, [_P, _I32, _P, _I64, _P, _P]),
    ("lsm_batch_counters", C.c_int, [_P, _P, _P]),
    ("lsm_batch_synchronize", C.c_int, [_P]),
]

_bound = False


def _lib():
    global _bound
    lib = _lsm.load_library()
    if not _bound:
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _bound = True
    return lib


def _check(st, h=None):
    if st != _lsm.LSM_OK:
        msg = _lib().lsm_batch_last_error(h)
        raise _lsm.LsmError(st, msg.decode() if msg else "")


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Batch:
    """Many 2D specimens stepped together (include/lsm_batch.h)."""

    def __init__(self, images, k_tab, epsc_tab, mass_tab=None, k2_ratio=1.0, a=1.0, dt=0.01,
                 damping=0.1, grip_mode=0, load_mode=0, precision="df64", stream=None):
        lib = _lib()
        self._keep = []
        kt = np.ascontiguousarray(k_tab, dtype=np.float64)
        et = np.ascontiguousarray(epsc_tab, dtype=np.float64)
        nphase = int(round(np.sqrt(kt.size)))
        mt = None if mass_tab is None else np.ascontiguousarray(mass_tab, dtype=np.float64)
        self._keep += [kt, et, mt]
        descs = (_lsm.lsm_desc * len(images))()
        for q, img in enumerate(images):
            ph = np.ascontiguousarray(img, dtype=np.uint8)
            if ph.ndim != 2:
                raise ValueError("batch specimens are 2D images")
            self._keep.append(ph)
            ny, nx = ph.shape
            descs[q] = _lsm.lsm_desc(dim=2, nx=nx, ny=ny, nz=1, phase=_p(ph), nphase=nphase,
                                     k_tab=_p(kt), epsc_tab=_p(et), mass_tab=_p(mt), k2_ratio=k2_ratio,
                                     a=a, dt=dt, damping=damping, grip_mode=grip_mode,
                                     load_mode=load_mode,
                                     precision=_lsm.PRECISIONS.get(precision, precision), path=0,
                                     stream=stream)
        h = C.c_void_p()
        _check(lib.lsm_build_batch(descs, len(images), C.byref(h)))
        self._keep = []
        self.h = h
        self.count = len(images)
        self.sizes = [self._sizes(q) for q in range(self.count)]

    def _sizes(self, q):
        n, m = C.c_int64(), C.c_int64()
        _check(_lib().lsm_batch_sizes(self.h, q, None, C.byref(n), C.byref(m)), self.h)
        return n.value, m.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib().lsm_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, steps_per_trial=4):
        ty, gr, od, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        _check(_lib().lsm_batch_autotune(self.h, steps_per_trial, C.byref(ty), C.byref(gr), C.byref(od),
                                         C.byref(ms)), self.h)
        return dict(tile_y=ty.value, grid=gr.value, order=od.value, ms_per_step=ms.value)

    def set_schedule(self, tile_y=16, grid=0, order=1):
        _check(_lib().lsm_batch_set_schedule(self.h, tile_y, grid, order), self.h)

    def apply_strain(self, eps):
        e = np.broadcast_to(np.asarray(eps, dtype=np.float64), (self.count,)).copy()
        _check(_lib().lsm_batch_apply_strain(self.h, _p(e)), self.h)

    def step(self, n):
        _check(_lib().lsm_batch_step(self.h, int(n)), self.h)

    def relax(self, tol, max_steps, check_every=1):
        taken = np.zeros(self.count, np.int64)
        conv = np.zeros(self.count, np.int32)
        st = _lib().lsm_batch_relax(self.h, float(tol), int(max_steps), int(check_every), _p(taken), _p(conv))
        if st not in (_lsm.LSM_OK, _lsm.LSM_ENOTCONV):
            _check(st, self.h)
        return st, taken, conv.astype(bool)

    def samples(self, q):
        cnt = C.c_int64()
        _check(_lib().lsm_batch_samples(self.h, q, None, 0, C.byref(cnt)), self.h)
        buf = (_lsm.lsm_sample * max(cnt.value, 1))()
        _check(_lib().lsm_batch_samples(self.h, q, buf, cnt.value, C.byref(cnt)), self.h)
        return [buf[i].as_dict() for i in range(cnt.value)]

    def state(self, q):
        n, _ = self.sizes[q]
        x = np.empty((2, n))
        v = np.empty((2, n))
        _check(_lib().lsm_batch_get_state(self.h, q, _p(x), _p(v)), self.h)
        return x, v

    def set_state(self, q, x=None, v=None):
        xs = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        vs = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        _check(_lib().lsm_batch_set_state(self.h, q, _p(xs), _p(vs)), self.h)

    def broken(self, q):
        _, m = self.sizes[q]
        out = np.empty(max(m, 1), np.uint8)
        mm, fb = C.c_int64(), C.c_int64()
        _check(_lib().lsm_batch_broken_mask(self.h, q, _p(out), out.size, C.byref(mm), C.byref(fb)), self.h)
        return out[:m], fb.value

    def counters(self):
        su, kl = C.c_int64(), C.c_int64()
        _check(_lib().lsm_batch_counters(self.h, C.byref(su), C.byref(kl)), self.h)
        return su.value, kl.value

    def synchronize(self):
        _check(_lib().lsm_batch_synchronize(self.h), self.h)
