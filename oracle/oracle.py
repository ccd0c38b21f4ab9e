"""ctypes wrapper of the plain-C FP64 oracle (lsm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests, the smoke check and the bench's
CPU-baseline leg, never by the CUDA product path.

Arrays cross the boundary component-major: component c of particle p sits at
[c * n + p]; the wrapper exposes them as numpy arrays of shape [dim, n].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SRC = os.path.join(_HERE, "lsm_oracle.c")
ORACLE_SO = os.path.join(_HERE, "liblsm_oracle.so")

OK, EINVAL, ENOMEM, ENOTCONV = 0, -1, -2, -4
OBS_KEYS = ("eps", "sigma_vir", "sigma_grip", "pe", "ke", "n_broken", "residual", "step")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with plain gcc: -O2, no fused multiply-add."""
    if (not force and os.path.exists(ORACLE_SO)
            and os.path.getmtime(ORACLE_SO) >= os.path.getmtime(ORACLE_SRC)):
        return ORACLE_SO
    tmp = ORACLE_SO + ".tmp.%d" % os.getpid()
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared", "-o", tmp,
            ORACLE_SRC, "-lm"]
    try:  # OpenMP only serves orc_set_threads; without it the oracle is single-threaded
        subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
    except (subprocess.CalledProcessError, OSError):
        subprocess.check_call(base)
    os.replace(tmp, ORACLE_SO)
    return ORACLE_SO


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build_oracle())
    P, D, I64, I = C.c_void_p, C.c_double, C.c_int64, C.c_int
    lib.orc_build_image.restype = P
    lib.orc_build_image.argtypes = [I, I, I, I, P, I, P, P, P, D, D, D, D, I, I, I]
    lib.orc_build_network.restype = P
    lib.orc_build_network.argtypes = [I, I64, I64, P, P, P, P, P, P, P, P, P, D, D, D, D, D, I]
    lib.orc_free.argtypes = [P]
    lib.orc_sizes.argtypes = [P, P, P, P]
    lib.orc_topology.argtypes = [P] + [P] * 9
    lib.orc_get_state.argtypes = [P, P, P, P]
    lib.orc_set_state.argtypes = [P, P, P, P]
    lib.orc_broken.argtypes = [P, P, P, P]
    lib.orc_forces.argtypes = [P, P, P, P, P]
    lib.orc_step.argtypes = [P, I64]
    lib.orc_apply_strain.argtypes = [P, D]
    lib.orc_observe.argtypes = [P, P]
    lib.orc_relax.restype = I
    lib.orc_relax.argtypes = [P, D, I64, I64, P]
    lib.orc_set_threads.restype = I
    lib.orc_set_threads.argtypes = [P, I]
    lib.orc_fields.argtypes = [P, D, P, P]
    lib.orc_set_strain_rate.argtypes = [P, D]
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One specimen held by the C oracle."""

    def __init__(self, handle):
        if not handle:
            raise ValueError("oracle build rejected its input")
        self._lib = _load()
        self._h = C.c_void_p(handle)
        n, m, d = C.c_int64(), C.c_int64(), C.c_int()
        self._lib.orc_sizes(self._h, C.byref(n), C.byref(m), C.byref(d))
        self.n, self.m, self.dim = n.value, m.value, d.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_free(h)
            self._h = None

    # ------------------------------------------------------------ builds
    @classmethod
    def from_image(cls, phase, k_tab, epsc_tab, mass=None, k2_ratio=1.0, a=1.0, dt=0.01,
                   damping=0.1, grip_mode=0, load_mode=0, lattice=0):
        lib = _load()
        ph = np.ascontiguousarray(phase, dtype=np.uint8)
        if ph.ndim == 2:
            dim, (ny, nx), nz = 2, ph.shape, 1
        elif ph.ndim == 3:
            dim, (nz, ny, nx) = 3, ph.shape
        else:
            raise ValueError("phase must be 2D or 3D")
        kt = np.ascontiguousarray(k_tab, dtype=np.float64)
        et = np.ascontiguousarray(epsc_tab, dtype=np.float64)
        nphase = int(round(np.sqrt(kt.size)))
        ms = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
        h = lib.orc_build_image(dim, nx, ny, nz, _ptr(ph), nphase, _ptr(kt), _ptr(et), _ptr(ms),
                                float(k2_ratio), float(a), float(dt), float(damping),
                                int(grip_mode), int(load_mode), int(lattice))
        return cls(h)

    @classmethod
    def from_network(cls, X, si, sj, k, r0, rc2, mass=None, fix=None, grip=None, dt=0.01,
                     damping=0.0, xc=0.0, omega=1.0, grip_area=1.0, load_mode=0):
        lib = _load()
        X = np.ascontiguousarray(X, dtype=np.float64)
        dim, n = X.shape
        si = np.ascontiguousarray(si, dtype=np.int32)
        sj = np.ascontiguousarray(sj, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.float64)
        r0 = np.ascontiguousarray(r0, dtype=np.float64)
        rc2 = np.ascontiguousarray(rc2, dtype=np.float64)
        ms = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
        fx = None if fix is None else np.ascontiguousarray(fix, dtype=np.uint8)
        gr = None if grip is None else np.ascontiguousarray(grip, dtype=np.uint8)
        h = lib.orc_build_network(dim, n, si.size, _ptr(X), _ptr(ms), _ptr(fx), _ptr(gr),
                                  _ptr(si), _ptr(sj), _ptr(k), _ptr(r0), _ptr(rc2),
                                  float(dt), float(damping), float(xc), float(omega),
                                  float(grip_area), int(load_mode))
        return cls(h)

    # ----------------------------------------------------------- queries
    def topology(self):
        n, m, d = self.n, self.m, self.dim
        out = dict(si=np.empty(m, np.int32), sj=np.empty(m, np.int32), k=np.empty(m),
                   r0=np.empty(m), rc2=np.empty(m), X=np.empty((d, n)), mass=np.empty(n),
                   fix=np.empty((d, n), np.uint8), grip=np.empty(n, np.uint8))
        self._lib.orc_topology(self._h, *[_ptr(out[q]) for q in
                                          ("si", "sj", "k", "r0", "rc2", "X", "mass", "fix", "grip")])
        return out

    def state(self):
        x, v, a = (np.empty((self.dim, self.n)) for _ in range(3))
        self._lib.orc_get_state(self._h, _ptr(x), _ptr(v), _ptr(a))
        return x, v, a

    def set_state(self, x=None, v=None, a=None):
        cv = [None if q is None else np.ascontiguousarray(q, dtype=np.float64) for q in (x, v, a)]
        self._lib.orc_set_state(self._h, *[_ptr(q) for q in cv])

    def broken(self):
        mask = np.empty(self.m, np.uint8)
        bs = np.empty(self.m, np.int64)
        fb = C.c_int64()
        self._lib.orc_broken(self._h, _ptr(mask), _ptr(bs), C.byref(fb))
        return mask, bs, fb.value

    # ----------------------------------------------------------- physics
    def forces(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        F = np.empty_like(x)
        U, W = C.c_double(), C.c_double()
        self._lib.orc_forces(self._h, _ptr(x), _ptr(F), C.byref(U), C.byref(W))
        return F, U.value, W.value

    def step(self, nsteps: int):
        self._lib.orc_step(self._h, int(nsteps))

    def fields(self, cell: float = 1.0):
        """Per-particle virial stress and Lagrangian strain, each [ncomp, n]
        (2D: xx, yy, xy; 3D: xx, yy, zz, xy, xz, yz)."""
        nq = 6 if self.dim == 3 else 3
        st = np.empty((nq, self.n))
        sn = np.empty((nq, self.n))
        self._lib.orc_fields(self._h, float(cell), _ptr(st), _ptr(sn))
        return st, sn

    def set_threads(self, nthreads: int) -> int:
        """Host threads of the spring pass (bit-identical results); returns
        the number in use (1 without OpenMP)."""
        got = self._lib.orc_set_threads(self._h, int(nthreads))
        if got < 0:
            raise MemoryError("oracle: incidence lists")
        return got

    def apply_strain(self, eps: float):
        self._lib.orc_apply_strain(self._h, float(eps))

    def set_strain_rate(self, rate: float):
        """Grips move every step at this engineering strain rate (0 stops)."""
        self._lib.orc_set_strain_rate(self._h, float(rate))

    def observe(self):
        out = np.empty(8)
        self._lib.orc_observe(self._h, _ptr(out))
        d = dict(zip(OBS_KEYS, out.tolist()))
        d["n_broken"] = int(d["n_broken"])
        d["step"] = int(d["step"])
        return d

    def relax(self, tol: float, max_steps: int, check_every: int = 1):
        taken = C.c_int64()
        st = self._lib.orc_relax(self._h, float(tol), int(max_steps), int(check_every),
                                 C.byref(taken))
        return st, taken.value
