"""Thin ctypes binding of liblsm (include/lsm.h): same names, marshalling only.

Every compute step runs in the CUDA library; this module converts numpy
arrays to pointers and status codes to exceptions. If liblsm.so has not been
built (``python -m paper_2201_04565_gb300.build``) importing the library
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblsm.so")

LSM_OK, LSM_EINVAL, LSM_ENOMEM, LSM_ECUDA = 0, -1, -2, -3
LSM_ENOTCONV, LSM_ETIMEOUT, LSM_ENONFINITE, LSM_ESTATE = -4, -5, -6, -7
LSM_PREC_EXACT64, LSM_PREC_FAST64, LSM_PREC_F32, LSM_PREC_DF = 0, 1, 2, 3
PRECISIONS = {"exact64": LSM_PREC_EXACT64, "fast64": LSM_PREC_FAST64, "f32": LSM_PREC_F32,
              "df64": LSM_PREC_DF}
STATUS_NAMES = {0: "LSM_OK", -1: "LSM_EINVAL", -2: "LSM_ENOMEM", -3: "LSM_ECUDA",
                -4: "LSM_ENOTCONV", -5: "LSM_ETIMEOUT", -6: "LSM_ENONFINITE", -7: "LSM_ESTATE"}


class LsmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class lsm_desc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("phase", C.c_void_p), ("nphase", C.c_int32),
                ("k_tab", C.c_void_p), ("epsc_tab", C.c_void_p), ("mass_tab", C.c_void_p),
                ("k2_ratio", C.c_double), ("a", C.c_double), ("dt", C.c_double),
                ("damping", C.c_double), ("grip_mode", C.c_int32), ("load_mode", C.c_int32),
                ("precision", C.c_int32), ("path", C.c_int32), ("stream", C.c_void_p),
                ("lattice", C.c_int32)]


class lsm_net_desc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int64), ("m", C.c_int64),
                ("X", C.c_void_p), ("mass", C.c_void_p), ("fix", C.c_void_p), ("grip", C.c_void_p),
                ("si", C.c_void_p), ("sj", C.c_void_p), ("k", C.c_void_p), ("r0", C.c_void_p),
                ("rc2", C.c_void_p), ("dt", C.c_double), ("damping", C.c_double),
                ("xc", C.c_double), ("omega", C.c_double), ("grip_area", C.c_double),
                ("load_mode", C.c_int32), ("precision", C.c_int32), ("stream", C.c_void_p)]


class lsm_sample(C.Structure):
    _fields_ = [("eps", C.c_double), ("sigma_vir", C.c_double), ("sigma_grip", C.c_double),
                ("pe", C.c_double), ("ke", C.c_double), ("residual", C.c_double),
                ("n_broken", C.c_int64), ("step", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# (name, restype, argtypes) of every symbol include/lsm.h declares
_P, _I64, _I32, _D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
SIGNATURES = [
    ("lsm_build_from_image", C.c_int, [C.POINTER(lsm_desc), C.POINTER(_P)]),
    ("lsm_build_network", C.c_int, [C.POINTER(lsm_net_desc), C.POINTER(_P)]),
    ("lsm_destroy", None, [_P]),
    ("lsm_last_error", C.c_char_p, [_P]),
    ("lsm_sizes", C.c_int, [_P, _P, _P, _P]),
    ("lsm_apply_strain", C.c_int, [_P, _D]),
    ("lsm_step", C.c_int, [_P, _I64]),
    ("lsm_relax", C.c_int, [_P, _D, _I64, _I64, _P]),
    ("lsm_stress_strain", C.c_int, [_P, _P, _P, _I64, _P]),
    ("lsm_samples", C.c_int, [_P, _P, _I64, _P]),
    ("lsm_sample_last", C.c_int, [_P, C.POINTER(lsm_sample)]),
    ("lsm_broken_mask", C.c_int, [_P, _P, _I64, _P, _P]),
    ("lsm_readback_async", C.c_int, [_P, _P, _I64, _P]),
    ("lsm_readback_wait", C.c_int, [_P]),
    ("lsm_break_steps", C.c_int, [_P, _P, _I64]),
    ("lsm_get_state", C.c_int, [_P, _P, _P]),
    ("lsm_set_state", C.c_int, [_P, _P, _P]),
    ("lsm_topology", C.c_int, [_P, _P, _P, _P, _P, _P]),
    ("lsm_observe", C.c_int, [_P, C.POINTER(lsm_sample)]),
    ("lsm_synchronize", C.c_int, [_P]),
    ("lsm_fields", C.c_int, [_P, C.c_double, _P, _P]),
    ("lsm_set_strain_rate", C.c_int, [_P, C.c_double]),
    ("lsm_save", C.c_int, [_P, C.c_char_p]),
    ("lsm_load", C.c_int, [C.c_char_p, _P, C.POINTER(_P)]),
    ("lsm_counters", C.c_int, [_P, _P, _P, _P]),
    ("lsm_spring_energy_static", C.c_int, [_I32, _I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P]),
]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblsm.so. Raises if it is missing: there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblsm.so is not built (%s); run python -m paper_2201_04565_gb300.build"
                           % path)
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream, named explicitly


def torch_stream_handle():
    """cudaStream_t of torch's current stream, usable as a library stream
    argument. torch's default stream is the legacy default stream (handle 0),
    which the library would read as "create a stream of your own"; it is
    passed as the runtime's explicit cudaStreamLegacy handle instead."""
    import torch
    h = torch.cuda.current_stream().cuda_stream
    return h if h else CUDA_STREAM_LEGACY


def _check(status, ctx=None):
    if status != LSM_OK:
        msg = load_library().lsm_last_error(ctx)
        raise LsmError(status, msg.decode() if msg else "")
    return status


# ---------------------------------------------------------------- C ABI names

def lsm_build_from_image(phase, k_tab, epsc_tab, mass_tab=None, k2_ratio=1.0, a=1.0, dt=0.01,
                         damping=0.1, grip_mode=0, load_mode=0, precision="exact64", stream=None,
                         path=0, lattice=0):
    """Image -> context handle. phase: uint8 [ny, nx] or [nz, ny, nx];
    lattice 0 square/cubic, 1 triangular packing (2D)."""
    lib = load_library()
    ph = np.ascontiguousarray(phase, dtype=np.uint8)
    if ph.ndim == 2:
        dim, nz, (ny, nx) = 2, 1, ph.shape
    elif ph.ndim == 3:
        dim, (nz, ny, nx) = 3, ph.shape
    else:
        raise ValueError("phase must be 2D or 3D")
    kt = np.ascontiguousarray(k_tab, dtype=np.float64)
    et = np.ascontiguousarray(epsc_tab, dtype=np.float64)
    nphase = int(round(np.sqrt(kt.size)))
    if kt.size != nphase * nphase or et.size != kt.size:
        raise ValueError("k_tab and epsc_tab must be nphase x nphase")
    mt = None if mass_tab is None else np.ascontiguousarray(mass_tab, dtype=np.float64)
    d = lsm_desc(dim=dim, nx=nx, ny=ny, nz=nz, phase=_ptr(ph), nphase=nphase, k_tab=_ptr(kt),
                 epsc_tab=_ptr(et), mass_tab=_ptr(mt), k2_ratio=k2_ratio, a=a, dt=dt,
                 damping=damping, grip_mode=grip_mode, load_mode=load_mode,
                 precision=PRECISIONS.get(precision, precision), path=path, stream=stream,
                 lattice=lattice)
    h = C.c_void_p()
    _check(lib.lsm_build_from_image(C.byref(d), C.byref(h)))
    return h


def lsm_build_network(X, si, sj, k, r0, rc2, mass=None, fix=None, grip=None, dt=0.01, damping=0.0,
                      xc=0.0, omega=1.0, grip_area=1.0, load_mode=0, precision="exact64",
                      stream=None):
    lib = load_library()
    X = np.ascontiguousarray(X, dtype=np.float64)
    dim, n = X.shape
    arrs = dict(si=np.ascontiguousarray(si, dtype=np.int32), sj=np.ascontiguousarray(sj, dtype=np.int32),
                k=np.ascontiguousarray(k, dtype=np.float64), r0=np.ascontiguousarray(r0, dtype=np.float64),
                rc2=np.ascontiguousarray(rc2, dtype=np.float64))
    ms = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
    fx = None if fix is None else np.ascontiguousarray(fix, dtype=np.uint8)
    gr = None if grip is None else np.ascontiguousarray(grip, dtype=np.uint8)
    d = lsm_net_desc(dim=dim, n=n, m=arrs["si"].size, X=_ptr(X), mass=_ptr(ms), fix=_ptr(fx),
                     grip=_ptr(gr), si=_ptr(arrs["si"]), sj=_ptr(arrs["sj"]), k=_ptr(arrs["k"]),
                     r0=_ptr(arrs["r0"]), rc2=_ptr(arrs["rc2"]), dt=dt, damping=damping, xc=xc,
                     omega=omega, grip_area=grip_area, load_mode=load_mode,
                     precision=PRECISIONS.get(precision, precision), stream=stream)
    h = C.c_void_p()
    _check(lib.lsm_build_network(C.byref(d), C.byref(h)))
    return h


def lsm_destroy(h):
    load_library().lsm_destroy(h)


def lsm_sizes(h):
    n, m, d = C.c_int64(), C.c_int64(), C.c_int32()
    _check(load_library().lsm_sizes(h, C.byref(n), C.byref(m), C.byref(d)), h)
    return n.value, m.value, d.value


def lsm_apply_strain(h, eps):
    _check(load_library().lsm_apply_strain(h, float(eps)), h)


def lsm_step(h, nsteps):
    _check(load_library().lsm_step(h, int(nsteps)), h)


def lsm_relax(h, tol, max_steps, check_every=1, raise_on_notconv=False):
    taken = C.c_int64()
    st = load_library().lsm_relax(h, float(tol), int(max_steps), int(check_every), C.byref(taken))
    if st == LSM_ENOTCONV and not raise_on_notconv:
        return st, taken.value
    _check(st, h)
    return st, taken.value


def lsm_samples(h):
    cnt = C.c_int64()
    _check(load_library().lsm_samples(h, None, 0, C.byref(cnt)), h)
    buf = (lsm_sample * max(cnt.value, 1))()
    _check(load_library().lsm_samples(h, buf, cnt.value, C.byref(cnt)), h)
    return [buf[q].as_dict() for q in range(cnt.value)]


def lsm_sample_last(h):
    """The most recent sample only (one 64-byte copy)."""
    out = lsm_sample()
    _check(load_library().lsm_sample_last(h, C.byref(out)), h)
    return out.as_dict()


def lsm_stress_strain(h):
    cnt = C.c_int64()
    _check(load_library().lsm_stress_strain(h, None, None, 0, C.byref(cnt)), h)
    eps = np.empty(cnt.value)
    sig = np.empty(cnt.value)
    _check(load_library().lsm_stress_strain(h, _ptr(eps), _ptr(sig), cnt.value, C.byref(cnt)), h)
    return eps, sig


def lsm_broken_mask(h, out=None):
    """Broken flags in canonical spring order and the first break step.
    out: optional uint8 host array of at least m entries (e.g. page-locked
    memory reused across calls); a new array otherwise."""
    n, m, _ = lsm_sizes(h)
    if out is None:
        out = np.empty(max(m, 1), np.uint8)
    elif out.dtype != np.uint8 or out.ndim != 1 or not out.flags.c_contiguous or out.size < max(m, 1):
        raise ValueError("out must be a contiguous uint8 array of at least %d entries" % max(m, 1))
    mm, fb = C.c_int64(), C.c_int64()
    _check(load_library().lsm_broken_mask(h, _ptr(out), out.size, C.byref(mm), C.byref(fb)), h)
    return out[:m], fb.value


def lsm_readback_async(h, out_mask=None, out_sample=None):
    """Enqueue the canonical broken mask into out_mask (contiguous uint8 host
    array of at least m entries) and the latest sample into out_sample (a
    writable host buffer of 64 bytes, e.g. a uint8 array); both page-locked
    for the copies to overlap later steps. Returns at once; the buffers hold
    the results after lsm_readback_wait, and must be kept alive until then."""
    _, m, _ = lsm_sizes(h)
    if out_mask is not None and (out_mask.dtype != np.uint8 or out_mask.ndim != 1 or
                                 not out_mask.flags.c_contiguous or out_mask.size < max(m, 1)):
        raise ValueError("out_mask must be a contiguous uint8 array of at least %d entries" % max(m, 1))
    if out_sample is not None and (not out_sample.flags.c_contiguous or out_sample.nbytes < C.sizeof(lsm_sample)
                                   or not out_sample.flags.writeable):
        raise ValueError("out_sample must be a writable contiguous buffer of %d bytes" % C.sizeof(lsm_sample))
    cap = 0 if out_mask is None else out_mask.size
    _check(load_library().lsm_readback_async(h, _ptr(out_mask), cap, _ptr(out_sample)), h)


def lsm_readback_wait(h):
    _check(load_library().lsm_readback_wait(h), h)


def sample_from_buffer(buf):
    """The lsm_sample record in a host buffer filled by lsm_readback_async."""
    return lsm_sample.from_buffer_copy(bytes(memoryview(buf).cast("B")[:C.sizeof(lsm_sample)])).as_dict()


def lsm_break_steps(h):
    _, m, _ = lsm_sizes(h)
    out = np.empty(max(m, 1), np.int64)
    _check(load_library().lsm_break_steps(h, _ptr(out), out.size), h)
    return out[:m]


def lsm_get_state(h):
    n, _, d = lsm_sizes(h)
    x = np.empty((d, n))
    v = np.empty((d, n))
    _check(load_library().lsm_get_state(h, _ptr(x), _ptr(v)), h)
    return x, v


def lsm_set_state(h, x=None, v=None):
    xs = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
    vs = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    _check(load_library().lsm_set_state(h, _ptr(xs), _ptr(vs)), h)


def lsm_topology(h):
    _, m, _ = lsm_sizes(h)
    out = dict(si=np.empty(m, np.int32), sj=np.empty(m, np.int32), k=np.empty(m),
               r0=np.empty(m), rc2=np.empty(m))
    _check(load_library().lsm_topology(h, *[_ptr(out[q]) for q in ("si", "sj", "k", "r0", "rc2")]), h)
    return out


def lsm_observe(h):
    s = lsm_sample()
    _check(load_library().lsm_observe(h, C.byref(s)), h)
    return s.as_dict()


def lsm_set_strain_rate(h, rate):
    _check(load_library().lsm_set_strain_rate(h, float(rate)), h)


def lsm_fields(h, cell_volume=0.0, stress=True, strain=True):
    """Per-particle virial stress and Lagrangian strain, each [ncomp, n]
    (2D: xx, yy, xy; 3D: xx, yy, zz, xy, xz, yz); None for an output not asked for."""
    n, m, dim = lsm_sizes(h)
    nq = 6 if dim == 3 else 3
    st = np.empty((nq, n)) if stress else None
    sn = np.empty((nq, n)) if strain else None
    _check(load_library().lsm_fields(h, float(cell_volume), _ptr(st), _ptr(sn)), h)
    return st, sn


def lsm_synchronize(h):
    _check(load_library().lsm_synchronize(h), h)


def lsm_save(h, path):
    """Checkpoint the context to a file (network and complete state)."""
    _check(load_library().lsm_save(h, os.fsencode(path)), h)


def lsm_load(path, stream=None):
    """Context handle rebuilt from a checkpoint file, in the saved state."""
    h = C.c_void_p()
    _check(load_library().lsm_load(os.fsencode(path), stream, C.byref(h)))
    return h


def lsm_counters(h):
    st, su, kl = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load_library().lsm_counters(h, C.byref(st), C.byref(su), C.byref(kl)), h)
    return st.value, su.value, kl.value


def lsm_spring_energy_static(dim, n, m, x, si, sj, k, r0, broken, out, stream=None):
    """Device pointers in, device pointer out (see include/lsm.h); no
    allocation by the library."""
    st = load_library().lsm_spring_energy_static(int(dim), int(n), int(m), x, si, sj, k, r0, broken,
                                                  out, stream)
    _check(st)


class Specimen:
    """Owning wrapper of one context (destroyed with the object)."""

    def __init__(self, handle):
        self.h = handle
        self.n, self.m, self.dim = lsm_sizes(handle)

    @classmethod
    def from_image(cls, phase, k_tab, epsc_tab, mass_tab=None, **kw):
        return cls(lsm_build_from_image(phase, k_tab, epsc_tab, mass_tab, **kw))

    @classmethod
    def from_network(cls, X, si, sj, k, r0, rc2, **kw):
        return cls(lsm_build_network(X, si, sj, k, r0, rc2, **kw))

    @classmethod
    def load(cls, path, stream=None):
        return cls(lsm_load(path, stream))

    def save(self, path):
        lsm_save(self.h, path)

    def close(self):
        if self.h is not None and self.h.value:
            lsm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_strain(self, eps):
        lsm_apply_strain(self.h, eps)

    def step(self, n):
        lsm_step(self.h, n)

    def relax(self, tol, max_steps, check_every=1):
        return lsm_relax(self.h, tol, max_steps, check_every)

    def state(self):
        return lsm_get_state(self.h)

    def set_state(self, x=None, v=None):
        lsm_set_state(self.h, x, v)

    def samples(self):
        return lsm_samples(self.h)

    def last_sample(self):
        return lsm_sample_last(self.h)

    def stress_strain(self):
        return lsm_stress_strain(self.h)

    def broken(self, out=None):
        return lsm_broken_mask(self.h, out)

    def readback_async(self, out_mask=None, out_sample=None):
        lsm_readback_async(self.h, out_mask, out_sample)

    def readback_wait(self):
        lsm_readback_wait(self.h)

    def break_steps(self):
        return lsm_break_steps(self.h)

    def topology(self):
        return lsm_topology(self.h)

    def observe(self):
        return lsm_observe(self.h)

    def set_strain_rate(self, rate):
        lsm_set_strain_rate(self.h, rate)

    def fields(self, cell_volume=0.0):
        return lsm_fields(self.h, cell_volume)

    def synchronize(self):
        lsm_synchronize(self.h)

    def counters(self):
        return lsm_counters(self.h)
