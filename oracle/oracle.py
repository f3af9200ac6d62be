"""ctypes wrapper of the plain FP64 CPU oracle (fsl_oracle.c).

TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
CPU-baseline leg of the benchmark.  The product library never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fsl_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")

CFLAGS = ["-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction)."""
    return _build(LIB, [], force)


def build_openmp(force: bool = False):
    """The same source compiled with -fopenmp: per-cell loops in parallel over
    the host cores, bit-identical results (integer reductions only).  None if
    the compiler has no OpenMP support."""
    try:
        return _build(LIB_OMP, ["-fopenmp"], force)
    except (subprocess.CalledProcessError, OSError):
        return None


def _build(lib_path: str, extra, force: bool) -> str:
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "fsl_oracle.h"))):
        tmp = lib_path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, *extra, "-o", tmp, SRC, "-lm"])
        os.replace(tmp, lib_path)
    return lib_path


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("collision", ctypes.c_int32), ("tau", ctypes.c_double), ("magic", ctypes.c_double),
                ("sigma", ctypes.c_double), ("g", ctypes.c_double * 3), ("eps", ctypes.c_double),
                ("lid", ctypes.c_double * 3), ("normal_rule", ctypes.c_int32), ("lonely_rule", ctypes.c_int32)]


class Bubble(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("vfx", ctypes.c_int64), ("vxfx", ctypes.c_int64),
                ("vsfx", ctypes.c_int64), ("ncells", ctypes.c_int64), ("constp", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


_libs = {}


def lib(openmp: bool = False):
    """The serial oracle, or (openmp=True) its OpenMP build; raises if that
    build is unavailable."""
    if openmp in _libs:
        return _libs[openmp]
    path = build_openmp() if openmp else build()
    if path is None:
        raise RuntimeError("the OpenMP build of the oracle is unavailable (no -fopenmp support)")
    L = ctypes.CDLL(path)
    vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    L.ora_create.restype = vp
    L.ora_create.argtypes = [ctypes.POINTER(Params)]
    L.ora_destroy.argtypes = [vp]
    L.ora_init.restype = ctypes.c_int
    L.ora_init.argtypes = [vp, vp, vp, vp, vp]
    L.ora_set_source.restype = ctypes.c_int
    L.ora_set_source.argtypes = [vp, i64, dbl, dbl, i32]
    L.ora_step.restype = ctypes.c_int
    L.ora_step.argtypes = [vp, i64]
    L.ora_status.restype = ctypes.c_int
    L.ora_status.argtypes = [vp]
    for name in ("ora_get_f", "ora_get_flags", "ora_get_phi", "ora_get_mass", "ora_get_ids"):
        getattr(L, name).argtypes = [vp, vp]
    L.ora_get_bubbles.restype = i64
    L.ora_get_bubbles.argtypes = [vp, vp, i64]
    L.ora_bubble_pressure.restype = dbl
    L.ora_bubble_pressure.argtypes = [ctypes.POINTER(Bubble)]
    L.ora_pool_fx.restype = i64
    L.ora_pool_fx.argtypes = [vp]
    L.ora_last_conversions.restype = i64
    L.ora_last_conversions.argtypes = [vp]
    L.ora_lattice.argtypes = [vp, vp, vp]
    L.ora_feq.argtypes = [dbl, vp, vp]
    L.ora_collide.restype = dbl
    L.ora_collide.argtypes = [ctypes.POINTER(Params), vp, vp]
    L.ora_label.argtypes = [vp, i32, i32, i32, vp]
    L.ora_curvature.restype = dbl
    L.ora_curvature.argtypes = [vp, i64]
    L.ora_gradient.argtypes = [vp, i64, vp]
    _libs[openmp] = L
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(nx, ny, nz, collision=0, tau=0.8, magic=3.0 / 16.0, sigma=0.0, gravity=(0.0, 0.0, 0.0),
                eps=1e-3, lid=(0.0, 0.0, 0.0), normal_rule=1, lonely_rule=1) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.collision, p.tau, p.magic, p.sigma = collision, tau, magic, sigma
    for k in range(3):
        p.g[k] = gravity[k]
        p.lid[k] = lid[k]
    p.eps = eps
    p.normal_rule = normal_rule
    p.lonely_rule = lonely_rule
    return p


BUBBLE_DTYPE = np.dtype([("id", np.int64), ("volume", np.float64), ("init_volume", np.float64),
                         ("pressure", np.float64), ("n_cells", np.int64), ("const_pressure", np.int32),
                         ("extra_volume", np.float64), ("vfx", np.int64), ("vxfx", np.int64),
                         ("vsfx", np.int64)])


class Oracle:
    """One lattice advanced by the oracle (openmp=True: the OpenMP build)."""

    def __init__(self, openmp: bool = False, **params):
        self.L = lib(openmp)
        self.p = make_params(**params)
        self.n = self.p.nx * self.p.ny * self.p.nz
        self._s = self.L.ora_create(ctypes.byref(self.p))
        if not self._s:
            raise ValueError("bad oracle parameters")

    @classmethod
    def from_scenario(cls, sc, openmp: bool = False) -> "Oracle":
        o = cls(openmp=openmp, **sc.params())
        rc = o.init(sc.flags, sc.fill, sc.rho, sc.u)
        if rc != 0:
            raise ValueError(f"oracle rejected the geometry ({rc})")
        for seed, extra, rate, constp in sc.sources:
            o.set_source(seed, extra, rate, constp)
        return o

    def __del__(self):
        if getattr(self, "_s", None):
            self.L.ora_destroy(self._s)
            self._s = None

    def init(self, flags, fill, rho, u) -> int:
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        fi = np.ascontiguousarray(fill, dtype=np.float64).reshape(-1)
        rh = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        return self.L.ora_init(self._s, _ptr(fl), _ptr(fi), _ptr(rh), _ptr(uu))

    def set_source(self, seed_cell, extra0, rate, constp) -> int:
        return self.L.ora_set_source(self._s, int(seed_cell), float(extra0), float(rate), int(constp))

    def step(self, nsteps: int = 1) -> int:
        return self.L.ora_step(self._s, int(nsteps))

    @property
    def status(self) -> int:
        return self.L.ora_status(self._s)

    def f(self) -> np.ndarray:
        out = np.empty((19, self.n), dtype=np.float64)
        self.L.ora_get_f(self._s, _ptr(out))
        return out

    def flags(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.uint8)
        self.L.ora_get_flags(self._s, _ptr(out))
        return out

    def phi(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        self.L.ora_get_phi(self._s, _ptr(out))
        return out

    def mass(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float64)
        self.L.ora_get_mass(self._s, _ptr(out))
        return out

    def ids(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int64)
        self.L.ora_get_ids(self._s, _ptr(out))
        return out

    def pool_fx(self) -> int:
        return int(self.L.ora_pool_fx(self._s))

    def conversions(self) -> int:
        return int(self.L.ora_last_conversions(self._s))

    def curvature(self, i: int) -> float:
        return float(self.L.ora_curvature(self._s, int(i)))

    def gradient(self, i: int) -> np.ndarray:
        g = np.zeros(3)
        self.L.ora_gradient(self._s, int(i), _ptr(g))
        return g

    def bubbles(self) -> np.ndarray:
        L = self.L
        nb = L.ora_get_bubbles(self._s, None, 0)
        raw = (Bubble * max(nb, 1))()
        L.ora_get_bubbles(self._s, ctypes.cast(raw, ctypes.c_void_p), nb)
        out = np.zeros(nb, dtype=BUBBLE_DTYPE)
        scale = 2.0 ** -32
        for k in range(nb):
            b = raw[k]
            out[k] = (b.id, (b.vfx + b.vxfx) * scale, b.vsfx * scale, L.ora_bubble_pressure(ctypes.byref(b)),
                      b.ncells, b.constp, b.vxfx * scale, b.vfx, b.vxfx, b.vsfx)
        return out

    def total_mass(self) -> float:
        """Liquid mass: sum of rho over liquid cells plus m over interface cells plus the pool."""
        fl = self.flags()
        f = self.f()
        rho = f.sum(axis=0)
        m = self.mass()
        return float(rho[fl == 0].sum() + m[fl == 1].sum() + self.pool_fx() * 2.0 ** -40)


def lattice():
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, dtype=np.int32)
    lib().ora_lattice(_ptr(c), _ptr(w), _ptr(opp))
    return c, w, opp


def feq(rho: float, u) -> np.ndarray:
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(19)
    lib().ora_feq(float(rho), _ptr(uu), _ptr(out))
    return out


def collide(fin, **params):
    p = make_params(1, 1, 1, **params)
    fi = np.ascontiguousarray(fin, dtype=np.float64)
    fo = np.zeros(19)
    rho = lib().ora_collide(ctypes.byref(p), _ptr(fi), _ptr(fo))
    return fo, rho


def label(fg: np.ndarray) -> np.ndarray:
    """Connected components (18-neighbourhood, wrap); label = min linear index."""
    nz, ny, nx = fg.shape
    a = np.ascontiguousarray(fg, dtype=np.uint8).reshape(-1)
    out = np.empty(a.size, dtype=np.int64)
    lib().ora_label(_ptr(a), nx, ny, nz, _ptr(out))
    return out.reshape(fg.shape)
