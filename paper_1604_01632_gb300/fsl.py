"""Python binding of the C ABI in include/fsl.h (argument marshalling only).

Every step of the method runs in the CUDA library libfsl.so; this module only
converts arrays and calls it.  Importing works without a GPU; creating a
Simulation needs the built library and a CUDA device and fails loudly
otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsl.so")

FSL_OK = 0
STATUS_NAMES = {0: "FSL_OK", -1: "FSL_ERR_ARG", -2: "FSL_ERR_GEOMETRY", -3: "FSL_ERR_OOM", -4: "FSL_ERR_NAN",
                -5: "FSL_ERR_CCL_NOT_CONVERGED", -6: "FSL_ERR_TABLE_FULL", -7: "FSL_ERR_CUDA",
                -8: "FSL_ERR_SYNC"}
PRECISIONS = {"fp64": 0, "fp32": 1, "f16s": 2, "bf16s": 3}
FIELD_BITS = {"flags": 1, "fill": 2, "mass": 4, "id": 8, "rho": 16, "u": 32, "pdf": 64}
FIELD_DTYPES = {"flags": (np.uint8, 1), "fill": (np.float64, 1), "mass": (np.float64, 1), "id": (np.int64, 1),
                "rho": (np.float64, 1), "u": (np.float64, 3), "pdf": (np.float64, 19)}

# names the library must export (checked by the CPU test suite)
EXPORTS = ["fsl_create", "fsl_init_geometry", "fsl_set_bubble_source", "fsl_step", "fsl_sync", "fsl_bubbles",
           "fsl_fields", "fsl_destroy", "fsl_last_error", "fsl_kernel_launches", "fsl_set_timing",
           "fsl_stream_collide_ms", "fsl_cell_counts", "fsl_labelling_runs", "fsl_relabelled_bubbles", "fsl_set_graphs",
           "fsl_label_bubbles_static", "fsl_phase_ms", "fsl_set_limits",
           "fsl_total_mass", "fsl_set_stream_form", "fsl_stream_form",
           "fsl_set_interface_order", "fsl_interface_order", "fsl_tuning", "fsl_forget_tuning"]


class FslError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("collision", ctypes.c_int32), ("tau", ctypes.c_double), ("magic", ctypes.c_double),
                ("sigma", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("eps", ctypes.c_double),
                ("lid_velocity", ctypes.c_double * 3), ("normal_rule", ctypes.c_int32),
                ("bubble_capacity", ctypes.c_int32), ("lonely_rule", ctypes.c_int32),
                ("split_trigger", ctypes.c_int32)]


class BubbleRec(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("volume", ctypes.c_double), ("init_volume", ctypes.c_double),
                ("pressure", ctypes.c_double), ("n_cells", ctypes.c_int64), ("const_pressure", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("extra_volume", ctypes.c_double)]


BUBBLE_DTYPE = np.dtype([("id", np.int64), ("volume", np.float64), ("init_volume", np.float64),
                         ("pressure", np.float64), ("n_cells", np.int64), ("const_pressure", np.int32),
                         ("extra_volume", np.float64)])

_lib = None


def load_library():
    """Load libfsl.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1604_01632_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_double
    L.fsl_create.restype = i32
    L.fsl_create.argtypes = [ctypes.POINTER(Params), i32, i32, vp, ctypes.POINTER(vp)]
    L.fsl_init_geometry.restype = i32
    L.fsl_init_geometry.argtypes = [vp, i32, vp, vp, vp, vp, i32]
    L.fsl_set_bubble_source.restype = i32
    L.fsl_set_bubble_source.argtypes = [vp, i32, i64, dbl, dbl, i32]
    L.fsl_step.restype = i32
    L.fsl_step.argtypes = [vp, i64]
    L.fsl_sync.restype = i32
    L.fsl_sync.argtypes = [vp]
    L.fsl_bubbles.restype = i32
    L.fsl_bubbles.argtypes = [vp, i32, vp, i64, ctypes.POINTER(i64)]
    L.fsl_fields.restype = i32
    L.fsl_fields.argtypes = [vp, i32, u32, vp, i32]
    L.fsl_destroy.restype = i32
    L.fsl_destroy.argtypes = [vp]
    L.fsl_last_error.restype = ctypes.c_char_p
    L.fsl_last_error.argtypes = [vp]
    L.fsl_kernel_launches.restype = i64
    L.fsl_kernel_launches.argtypes = [vp]
    L.fsl_set_timing.restype = i32
    L.fsl_set_timing.argtypes = [vp, i32]
    L.fsl_stream_collide_ms.restype = dbl
    L.fsl_stream_collide_ms.argtypes = [vp]
    L.fsl_label_bubbles_static.restype = i32
    L.fsl_label_bubbles_static.argtypes = [vp, i32, i32, i32, vp, vp]
    L.fsl_phase_ms.restype = i32
    L.fsl_phase_ms.argtypes = [vp, vp]
    L.fsl_set_graphs.restype = i32
    L.fsl_set_graphs.argtypes = [vp, i32]
    L.fsl_tuning.restype = i32
    L.fsl_tuning.argtypes = [vp, vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.fsl_forget_tuning.restype = i32
    L.fsl_forget_tuning.argtypes = []
    L.fsl_set_interface_order.restype = i32
    L.fsl_set_interface_order.argtypes = [vp, i32]
    L.fsl_interface_order.restype = i32
    L.fsl_interface_order.argtypes = [vp]
    L.fsl_set_stream_form.restype = i32
    L.fsl_set_stream_form.argtypes = [vp, i32]
    L.fsl_stream_form.restype = i32
    L.fsl_stream_form.argtypes = [vp]
    L.fsl_total_mass.restype = i32
    L.fsl_total_mass.argtypes = [vp, i32, ctypes.POINTER(dbl)]
    L.fsl_set_limits.restype = i32
    L.fsl_set_limits.argtypes = [vp, i64, i64, i32]
    L.fsl_labelling_runs.restype = i64
    L.fsl_labelling_runs.argtypes = [vp]
    L.fsl_relabelled_bubbles.restype = i64
    L.fsl_relabelled_bubbles.argtypes = [vp]
    L.fsl_cell_counts.restype = i32
    L.fsl_cell_counts.argtypes = [vp, i32, ctypes.POINTER(i64)]
    _lib = L
    return L


def make_params(nx, ny, nz, collision=0, tau=0.8, magic=3.0 / 16.0, sigma=0.0, gravity=(0.0, 0.0, 0.0),
                eps=1e-3, lid=(0.0, 0.0, 0.0), normal_rule=1, lonely_rule=1, bubble_capacity=0,
                split_trigger=0) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.collision, p.tau, p.magic, p.sigma = collision, tau, magic, sigma
    for k in range(3):
        p.gravity[k] = gravity[k]
        p.lid_velocity[k] = lid[k]
    p.eps = eps
    p.normal_rule = normal_rule
    p.lonely_rule = lonely_rule
    p.bubble_capacity = bubble_capacity
    p.split_trigger = split_trigger
    return p


def _ptr(a) -> ctypes.c_void_p:
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(a.data_ptr())   # torch tensor


def _default_stream() -> int:
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


STATIC_MAX_CELLS = 1 << 21


def _check_device_tensor(t, name: str, dtype_name: str, n: int):
    """A CUDA tensor on the current device, of the given dtype, contiguous and
    holding at least n elements; ValueError otherwise (nothing is launched)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name} must be a torch CUDA tensor, not {type(t).__name__}")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} must live on the current CUDA device (got {t.device})")
    if t.dtype != getattr(torch, dtype_name):
        raise ValueError(f"{name} must be {dtype_name} (got {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{name} holds {t.numel()} elements, the lattice has {n} cells")


def label_bubbles_static(flags, nx: int, ny: int, nz: int, labels, stream: Optional[int] = None):
    """Allocation-free bubble labelling through fsl_label_bubbles_static.

    For callers that cannot allocate device memory.  `flags` (uint8) and
    `labels` (int64) are caller-owned contiguous CUDA tensors on the current
    device with at least nx*ny*nz elements (checked here before the call, so
    that a host array or a short buffer never reaches the kernels); the
    library uses only its fixed 2^21-cell scratch.  Labels are the minimum
    linear index of each 18-connected gas/interface component, -1 elsewhere.
    Calls that overlap on the GPU share the scratch and race."""
    if min(nx, ny, nz) <= 0:
        raise ValueError("lattice dimensions must be positive")
    n = int(nx) * int(ny) * int(nz)
    _check_device_tensor(flags, "flags", "uint8", n)
    _check_device_tensor(labels, "labels", "int64", n)
    L = load_library()
    st = L.fsl_label_bubbles_static(_ptr(flags), nx, ny, nz, _ptr(labels),
                                     ctypes.c_void_p(_default_stream() if stream is None else stream))
    if st != FSL_OK:
        raise FslError(st, "fsl_label_bubbles_static failed")


class Simulation:
    """One handle of the library: one or more independent lattices on one GPU."""

    def __init__(self, params: Sequence[dict], precision: str = "fp64", stream: Optional[int] = None,
                 bubble_capacity: int = 0, split_trigger: int = 0):
        self.L = load_library()
        plist = [make_params(**p, bubble_capacity=bubble_capacity, split_trigger=split_trigger) for p in params]
        self.dims = [(p.nx, p.ny, p.nz) for p in plist]
        arr = (Params * len(plist))(*plist)
        self.stream = _default_stream() if stream is None else stream
        h = ctypes.c_void_p()
        st = self.L.fsl_create(arr, len(plist), PRECISIONS[precision], ctypes.c_void_p(self.stream), ctypes.byref(h))
        if st != FSL_OK:
            raise FslError(st, "fsl_create failed")
        self._h = h
        self.precision = precision

    @classmethod
    def from_scenarios(cls, scenarios, precision="fp64", **kw) -> "Simulation":
        scs = list(scenarios) if isinstance(scenarios, (list, tuple)) else [scenarios]
        sim = cls([s.params() for s in scs], precision=precision, **kw)
        for d, s in enumerate(scs):
            sim.init_geometry(d, s.flags, s.fill, s.rho, s.u)
        for d, s in enumerate(scs):
            for seed, extra, rate, constp in s.sources:
                sim.set_source(d, seed, extra, rate, constp)
        return sim

    def _check(self, st: int):
        if st != FSL_OK:
            raise FslError(st, self.L.fsl_last_error(self._h).decode())

    def n(self, d: int = 0) -> int:
        nx, ny, nz = self.dims[d]
        return nx * ny * nz

    def init_geometry(self, d, flags, fill, rho, u, on_device: bool = False):
        if on_device:
            self._check(self.L.fsl_init_geometry(self._h, d, _ptr(flags), _ptr(fill), _ptr(rho), _ptr(u), 1))
            return
        fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        fi = np.ascontiguousarray(fill, dtype=np.float64).reshape(-1)
        rh = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        uu = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        n = self.n(d)
        if fl.size != n or fi.size != n or rh.size != n or uu.size != 3 * n:
            raise ValueError("field sizes do not match the domain")
        self._check(self.L.fsl_init_geometry(self._h, d, _ptr(fl), _ptr(fi), _ptr(rh), _ptr(uu), 0))

    def set_source(self, d, seed_cell, extra0, rate, const_pressure):
        self._check(self.L.fsl_set_bubble_source(self._h, d, int(seed_cell), float(extra0), float(rate),
                                                 int(const_pressure)))

    def step(self, nsteps: int = 1):
        self._check(self.L.fsl_step(self._h, int(nsteps)))

    def sync(self):
        self._check(self.L.fsl_sync(self._h))

    def bubbles(self, d: int = 0) -> np.ndarray:
        cnt = ctypes.c_int64(0)
        self._check(self.L.fsl_bubbles(self._h, d, None, 0, ctypes.byref(cnt)))
        nb = cnt.value
        raw = (BubbleRec * max(nb, 1))()
        self._check(self.L.fsl_bubbles(self._h, d, ctypes.cast(raw, ctypes.c_void_p), nb, ctypes.byref(cnt)))
        out = np.zeros(nb, dtype=BUBBLE_DTYPE)
        for k in range(nb):
            b = raw[k]
            out[k] = (b.id, b.volume, b.init_volume, b.pressure, b.n_cells, b.const_pressure, b.extra_volume)
        return out

    def fields(self, d: int = 0, names: Iterable[str] = ("flags", "fill", "mass", "id", "pdf"),
               out: Optional[Dict[str, np.ndarray]] = None) -> Dict[str, np.ndarray]:
        """Selected fields of domain d in host arrays; `out` may supply some of
        them (C-contiguous, of the field's dtype and size, e.g. views of pinned
        host memory), the others are allocated."""
        names = [k for k in FIELD_BITS if k in set(names)]
        n = self.n(d)
        res = {}
        mask = 0
        ptrs = []
        for k in names:
            dt, m = FIELD_DTYPES[k]
            if out is not None and k in out:
                a = out[k]
                if a.dtype != dt or a.size != m * n or not a.flags.c_contiguous:
                    raise ValueError(f"out[{k!r}] must be a C-contiguous {np.dtype(dt)} array of {m * n} elements")
                a = a.reshape(-1)
            else:
                a = np.empty(m * n, dtype=dt)
            res[k] = a if m == 1 else a.reshape(m, n)
            mask |= FIELD_BITS[k]
            ptrs.append(a.ctypes.data)
        arr = (ctypes.c_void_p * max(len(ptrs), 1))(*ptrs)
        self._check(self.L.fsl_fields(self._h, d, mask, ctypes.cast(arr, ctypes.c_void_p), 0))
        return res

    def fields_to(self, d: int, dst: Dict[str, "object"]):
        """Write selected fields into caller-owned device buffers (torch tensors)."""
        names = [k for k in FIELD_BITS if k in dst]
        mask = 0
        ptrs = []
        for k in names:
            mask |= FIELD_BITS[k]
            ptrs.append(dst[k].data_ptr())
        arr = (ctypes.c_void_p * max(len(ptrs), 1))(*ptrs)
        self._check(self.L.fsl_fields(self._h, d, mask, ctypes.cast(arr, ctypes.c_void_p), 1))

    def cell_counts(self, d: int = 0) -> np.ndarray:
        c = (ctypes.c_int64 * 5)()
        self._check(self.L.fsl_cell_counts(self._h, d, c))
        return np.array(list(c), dtype=np.int64)

    def total_mass(self, d: int = 0) -> float:
        """Liquid mass of domain d: rho over liquid cells + m over interface cells + pool."""
        v = ctypes.c_double(0.0)
        self._check(self.L.fsl_total_mass(self._h, d, ctypes.byref(v)))
        return float(v.value)

    @property
    def launches(self) -> int:
        return int(self.L.fsl_kernel_launches(self._h))

    @property
    def labelling_runs(self) -> int:
        return int(self.L.fsl_labelling_runs(self._h))

    @property
    def relabelled_bubbles(self) -> int:
        """Bubbles the labelling passes took, summed over the passes."""
        return int(self.L.fsl_relabelled_bubbles(self._h))

    def set_timing(self, on: bool):
        self._check(self.L.fsl_set_timing(self._h, 1 if on else 0))

    def set_limits(self, ccl_max_iter: int = 0, barrier_polls: int = 0, barrier_absent: bool = False):
        """Failure-path limits for tests (0 = default): labelling iteration cap,
        barrier polls, and a barrier that waits for a block that does not exist."""
        self._check(self.L.fsl_set_limits(self._h, int(ccl_max_iter), int(barrier_polls), 1 if barrier_absent else 0))

    def set_stream_form(self, form: int):
        """Stream-collide kernel form: 0 split, 1/2/3 persistent with 1/2/4 tiles per liquid
        item, 4 slab (interface list in cell order only), 5 two kernels (liquid, then one
        thread per interface cell), 6/7 tile-fused with 2/4 tiles per block (not FP64),
        8 the two kernels side by side on two streams, -1 autotune again."""
        self._check(self.L.fsl_set_stream_form(self._h, int(form)))

    def tuning(self) -> dict:
        """Autotuner record: per-form stream-collide ms, chosen form, source."""
        ms = (ctypes.c_double * 9)()
        form, src = ctypes.c_int32(0), ctypes.c_int32(0)
        self._check(self.L.fsl_tuning(self._h, ms, ctypes.byref(form), ctypes.byref(src)))
        names = ("split", "persistent_1tile", "persistent_2tiles", "persistent_4tiles", "slab", "two_kernel",
                 "tile_fused_2", "tile_fused_4", "two_kernel_concurrent")
        return {"ms_per_form": dict(zip(names, [round(v, 5) for v in ms])),
                "form": int(form.value), "form_name": names[form.value] if form.value >= 0 else None,
                "source": ("none", "measured", "cache", "caller")[src.value]}

    def set_interface_order(self, mode: int):
        """Interface list order: 1 rebuilt in cell order each step, 0 appended, -1 by lattice size."""
        self._check(self.L.fsl_set_interface_order(self._h, int(mode)))

    @property
    def interface_order(self) -> int:
        return int(self.L.fsl_interface_order(self._h))

    @property
    def stream_form(self) -> int:
        return int(self.L.fsl_stream_form(self._h))

    def set_graphs(self, on: bool):
        self._check(self.L.fsl_set_graphs(self._h, 1 if on else 0))

    def phase_ms(self) -> Dict[str, float]:
        out = (ctypes.c_double * 4)()
        self._check(self.L.fsl_phase_ms(self._h, out))
        return dict(zip(("stream_collide", "liquid_end", "interface_end", "conversion"), list(out)))

    def stream_collide_ms(self) -> float:
        return float(self.L.fsl_stream_collide_ms(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self.L.fsl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
