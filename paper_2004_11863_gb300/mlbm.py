"""Python binding of the C ABI in include/mlbm.h (argument marshalling only).

Every step of the method runs in the CUDA library libmlbm.so; this module
only converts arguments.  It raises if the library is missing or cannot be
loaded: there is no fallback.

PyTorch provides the CUDA stream (``torch.cuda.current_stream()``) and,
optionally, device memory through its caching allocator.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmlbm.so")

LBM_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EUNSTABLE", -5: "ESTATE",
          -6: "ETIMEOUT"}
STORAGE = {"fp32": 0, "fp16": 1}
MAX_LEVELS = 4


class LbmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({lib().lbm_strerror(code).decode()})")


class lbm_box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3)]


class lbm_config(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("collision", ctypes.c_int), ("storage", ctypes.c_int),
                ("tau0", ctypes.c_double), ("rho0", ctypes.c_double),
                ("dims", ctypes.c_int * 3), ("nlevels", ctypes.c_int),
                ("box", lbm_box * (MAX_LEVELS - 1)), ("batch", ctypes.c_int),
                ("u_ref", ctypes.c_double * 3), ("sigma", ctypes.c_double)]


class lbm_ic(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u0", ctypes.c_double * 3),
                ("center", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("amplitude", ctypes.c_double), ("eps", ctypes.c_double),
                ("drho", ctypes.c_double)]


IC_KINDS = {"uniform": 0, "vortex": 1, "pulse": 2}


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class lbm_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libmlbm.so (built by ``paper_2004_11863_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2004_11863_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    L.lbm_create.argtypes = [ctypes.POINTER(lbm_config), P, ctypes.POINTER(lbm_allocator),
                             ctypes.POINTER(P)]
    L.lbm_level_info.argtypes = [P, ctypes.c_int, ip, dp, ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_init.argtypes = [P, ctypes.c_int, ctypes.c_int, dp, dp]
    L.lbm_step.argtypes = [P, ctypes.c_int]
    L.lbm_set_graphs.argtypes = [P, ctypes.c_int]
    L.lbm_set_fused.argtypes = [P, ctypes.c_int]
    L.lbm_macros.argtypes = [P, ctypes.c_int, ctypes.c_int, dp, dp]
    L.lbm_macros_device.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
    L.lbm_populations.argtypes = [P, ctypes.c_int, ctypes.c_int, dp]
    L.lbm_sensors_enable.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.lbm_autotune.argtypes = [P, ctypes.c_int, ip]
    L.lbm_set_block_shape.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.lbm_sensors.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_ubyte), dp,
                              dp, dp]
    L.lbm_lattice.argtypes = [ctypes.c_int, ip, dp]
    L.lbm_probe_add.argtypes = [P, ctypes.c_int, ctypes.c_int, ip]
    L.lbm_probe.argtypes = [P, dp, ctypes.c_int, ip]
    L.lbm_probe_async.argtypes = [P, dp, ctypes.c_int, ip]
    L.lbm_diag.argtypes = [P, ctypes.c_int, dp, dp]
    L.lbm_diag_noalloc.argtypes = [P, ctypes.c_int, dp, dp]
    L.lbm_set_face_buffer.argtypes = [P, ctypes.c_int]
    L.lbm_bytes.argtypes = [ctypes.POINTER(lbm_config), ctypes.POINTER(ctypes.c_ulonglong)]
    L.lbm_init_analytic.argtypes = [P, ctypes.c_int, ctypes.POINTER(lbm_ic)]
    L.lbm_noise.argtypes = [P, P, ctypes.c_int, ctypes.c_int, dp, dp,
                            ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_sync.argtypes = [P]
    L.lbm_kernel_launches.argtypes = [P]
    L.lbm_kernel_launches.restype = ctypes.c_longlong
    L.lbm_profile.argtypes = [P, ctypes.c_int]
    L.lbm_profile_read.argtypes = [P, ctypes.c_int, ctypes.c_int, dp,
                                   ctypes.POINTER(ctypes.c_longlong)]
    L.lbm_destroy.argtypes = [P]
    L.lbm_destroy.restype = None
    L.lbm_strerror.argtypes = [ctypes.c_int]
    L.lbm_strerror.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != LBM_OK:
        raise LbmError(rc, what)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lbm_lattice(lattice: str):
    """The library's velocity set: (xi [q,3] int, w [q] float64)."""
    xi = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    q = lib().lbm_lattice(workloads.LATTICES[lattice],
                          xi.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w))
    if q <= 0:
        raise LbmError(q, "lbm_lattice")
    return xi[:q].copy(), w[:q].copy()


def make_config(lattice: str, collision: str, tau0: float, dims: Sequence[int], boxes,
                storage: str = "fp32", batch: int = 1, rho0: float = 1.0,
                u_ref=(0.0, 0.0, 0.0), sigma: float = 1.0) -> lbm_config:
    c = lbm_config()
    c.lattice = workloads.LATTICES[lattice]
    c.collision = workloads.COLLISIONS[collision]
    c.storage = STORAGE[storage]
    c.tau0 = float(tau0)
    c.rho0 = float(rho0)
    d = list(dims) + [1] * (3 - len(dims))
    for a in range(3):
        c.dims[a] = int(d[a])
    c.nlevels = 1 + len(boxes)
    for k, (lo, hi) in enumerate(boxes):
        for a in range(3):
            c.box[k].lo[a] = int(lo[a])
            c.box[k].hi[a] = int(hi[a])
    c.batch = int(batch)
    for a in range(3):
        c.u_ref[a] = float(u_ref[a])
    c.sigma = float(sigma)
    return c


def lbm_bytes(lattice, collision, tau0, dims, boxes, storage="fp32", batch=1, rho0=1.0,
              u_ref=(0.0, 0.0, 0.0), sigma=1.0) -> int:
    """Device bytes a run of this layout needs (no device work)."""
    cfg = make_config(lattice, collision, tau0, dims, boxes, storage, batch, rho0, u_ref, sigma)
    b = ctypes.c_ulonglong()
    _check(lib().lbm_bytes(ctypes.byref(cfg), ctypes.byref(b)), "lbm_bytes")
    return int(b.value)


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self):
        import torch
        self._torch = torch
        self._alloc = _ALLOC_FN(self._do_alloc)
        self._free = _FREE_FN(self._do_free)
        self.struct = lbm_allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, user):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:
            return None

    def _do_free(self, ptr, user):
        if ptr:
            self._torch.cuda.caching_allocator_delete(int(ptr))


class Lbm:
    """A multi-level run (or a batch of runs sharing one layout).

    Thin wrapper: lbm_create / lbm_init / lbm_step / lbm_macros / lbm_probe_add /
    lbm_probe / lbm_diag / lbm_destroy of the C ABI.
    """

    def __init__(self, lattice, collision, tau0, dims, boxes, storage="fp32", batch=1,
                 rho0=1.0, stream=None, torch_allocator=False, u_ref=(0.0, 0.0, 0.0),
                 sigma=1.0):
        L = lib()
        self.cfg = make_config(lattice, collision, tau0, dims, boxes, storage, batch, rho0, u_ref,
                               sigma)
        self.lattice = lattice
        self.q = workloads.Q_OF[lattice]
        self.nlevels = self.cfg.nlevels
        self.batch = batch
        self._allocator = _TorchAllocator() if torch_allocator else None
        h = ctypes.c_void_p()
        if stream is None:
            stream = 0
        rc = L.lbm_create(ctypes.byref(self.cfg), ctypes.c_void_p(int(stream)),
                          ctypes.byref(self._allocator.struct) if self._allocator else None,
                          ctypes.byref(h))
        _check(rc, "lbm_create")
        self._h = h
        self._steps = 0  # coarse steps since the last initial state

    @classmethod
    def from_case(cls, case, storage="fp32", batch=1, init=True, **kw):
        kw.setdefault("u_ref", case.u_ref)
        kw.setdefault("sigma", case.sigma)
        r = cls(case.lattice, case.collision, case.tau0, case.dims, case.boxes, storage, batch,
                case.rho0, **kw)
        if init:
            for l in range(r.nlevels):
                rho, u = workloads.initial_fields(case, l)
                for b in range(batch):
                    r.init(l, b, rho, u)
        return r

    # -- C ABI calls -------------------------------------------------------
    def level_info(self, level):
        n = (ctypes.c_int * 3)()
        tau = ctypes.c_double()
        na = ctypes.c_longlong()
        _check(lib().lbm_level_info(self._h, level, n, ctypes.byref(tau), ctypes.byref(na)),
               "lbm_level_info")
        return tuple(n), tau.value, na.value

    def nodes(self, level):
        n, _, _ = self.level_info(level)
        return n[0] * n[1] * n[2]

    def init(self, level, run, rho, u):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1)
        if rho.size != self.nodes(level) or u.shape[1] != rho.size:
            raise ValueError("field size does not match the level")
        _check(lib().lbm_init(self._h, level, run, _dp(rho), _dp(u)), "lbm_init")
        self._steps = 0

    def init_analytic(self, ic: dict, run=0):
        """Device-side initial state from a workload IC description
        (kind uniform / vortex / pulse, as in workloads.initial_fields)."""
        d = lbm_ic()
        d.kind = IC_KINDS[ic["kind"]]
        for a, v in enumerate(ic.get("u0", (0.0, 0.0, 0.0))):
            d.u0[a] = float(v)
        for a, v in enumerate(ic.get("center", (0.0, 0.0, 0.0))):
            d.center[a] = float(v)
        d.radius = float(ic.get("radius", 0.0))
        d.amplitude = float(ic.get("amplitude", 0.0))
        d.eps = float(ic.get("eps", 0.0))
        d.drho = float(ic.get("drho", 0.0))
        _check(lib().lbm_init_analytic(self._h, run, ctypes.byref(d)), "lbm_init_analytic")
        self._steps = 0

    def noise(self, single: "Lbm", run=0, margin=4):
        """(max, rms, nodes) of |rho - rho_single| outside the refined box."""
        mx = ctypes.c_double()
        rms = ctypes.c_double()
        n = ctypes.c_longlong()
        rc = lib().lbm_noise(self._h, single._h, run, margin, ctypes.byref(mx),
                             ctypes.byref(rms), ctypes.byref(n))
        if rc not in (LBM_OK, -4):
            _check(rc, "lbm_noise")
        return mx.value, rms.value, n.value

    def step(self, n=1):
        _check(lib().lbm_step(self._h, int(n)), "lbm_step")
        self._steps += int(n)

    def coarse_steps(self) -> int:
        """Coarse steps issued through this object since the last initial state."""
        return self._steps

    def set_graphs(self, enable: bool):
        _check(lib().lbm_set_graphs(self._h, int(bool(enable))), "lbm_set_graphs")

    def set_fused(self, mode=1):
        """lbm_set_fused: 1 runs every coarse step after the first as one
        persistent cooperative kernel; 0 (default) the per-operation
        kernels; 2 tests the bounded barrier wait (the next sync raises
        LbmError with code -6)."""
        _check(lib().lbm_set_fused(self._h, int(mode)), "lbm_set_fused")

    def macros(self, level, run=0, out=None):
        """lbm_macros: (rho [N], u [3, N]) float64.  out: optional
        caller-owned (rho, u) arrays of those shapes, C-contiguous float64
        (pinned host memory makes the copy faster), filled and returned."""
        N = self.nodes(level)
        if out is None:
            rho = np.empty(N)
            u = np.empty((3, N))
        else:
            rho, u = out
            for a, shp in ((rho, (N,)), (u, (3, N))):
                if a.dtype != np.float64 or a.shape != shp or not a.flags.c_contiguous:
                    raise ValueError(f"macros out arrays must be C-contiguous float64 {shp}")
        _check(lib().lbm_macros(self._h, level, run, _dp(rho), _dp(u)), "lbm_macros")
        return rho, u

    def autotune(self, reps=5):
        """lbm_autotune: choose each level's update block shape by timing;
        returns [(bx, by)] per level."""
        sh = (ctypes.c_int * (2 * self.nlevels))()
        _check(lib().lbm_autotune(self._h, int(reps), sh), "lbm_autotune")
        return [(sh[2 * l], sh[2 * l + 1]) for l in range(self.nlevels)]

    def set_block_shape(self, level, bx, by):
        _check(lib().lbm_set_block_shape(self._h, level, bx, by), "lbm_set_block_shape")

    def set_face_buffer(self, enable: bool):
        """lbm_set_face_buffer: route the rebuilt x-face nodes of 3D levels
        through the face buffer (default) or through the population planes."""
        _check(lib().lbm_set_face_buffer(self._h, int(bool(enable))), "lbm_set_face_buffer")

    def sensors_enable(self, level, eps=0.0, g_threshold=0.0):
        """lbm_sensors_enable: evaluate the non-hydrodynamic mode sensors of a
        level at every iteration from the next coarse step on."""
        _check(lib().lbm_sensors_enable(self._h, level, float(eps), float(g_threshold)),
               "lbm_sensors_enable")

    def sensors(self, level, run=0, with_gnorm=False):
        """lbm_sensors: (flags [N] uint8, div [N], curl [3, N]) of a level
        (and |f1G| [N])."""
        N = int(np.prod(self.level_info(level)[0]))
        fl = np.zeros(N, dtype=np.uint8)
        dv = np.zeros(N)
        cu = np.zeros((3, N))
        gn = np.zeros(N)
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(lib().lbm_sensors(self._h, level, run,
                                 fl.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                 dptr(dv), dptr(cu), dptr(gn)), "lbm_sensors")
        return (fl, dv, cu, gn) if with_gnorm else (fl, dv, cu)

    def macros_device(self, level, rho_ptr, u_ptr, run=0):
        _check(lib().lbm_macros_device(self._h, level, run, ctypes.c_void_p(rho_ptr),
                                       ctypes.c_void_p(u_ptr)), "lbm_macros_device")

    def populations(self, level, run=0):
        N = self.nodes(level)
        g = np.empty((self.q, N))
        _check(lib().lbm_populations(self._h, level, run, _dp(g)), "lbm_populations")
        return g

    def probe_add(self, level, ijk):
        ijk = np.ascontiguousarray(np.asarray(ijk, dtype=np.int32).reshape(-1, 3))
        _check(lib().lbm_probe_add(self._h, level, ijk.shape[0],
                                   ijk.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
               "lbm_probe_add")
        self._nprobe = ijk.shape[0]

    def probe(self, max_steps=65536):
        n = getattr(self, "_nprobe", 0)
        out = np.zeros((max_steps, self.batch, max(n, 1), 4))
        ns = ctypes.c_int()
        _check(lib().lbm_probe(self._h, _dp(out), max_steps, ctypes.byref(ns)), "lbm_probe")
        return out[: ns.value, :, :n]

    def probe_async(self, out):
        """Enqueue the read-out of the newest recorded probe steps into
        `out`, a C-contiguous float64 array [k, batch, n, 4] (pinned host
        memory for overlap); returns the number of steps that will land in
        out[:count] once the stream reaches them (after sync()).  `out` must
        stay alive and untouched until then."""
        n = getattr(self, "_nprobe", 0)
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.ndim != 4 \
                or out.shape[1:] != (self.batch, max(n, 1), 4):
            raise ValueError("probe_async needs a C-contiguous float64 [k, batch, n, 4] array")
        ns = ctypes.c_int()
        _check(lib().lbm_probe_async(self._h, _dp(out), out.shape[0], ctypes.byref(ns)),
               "lbm_probe_async")
        return ns.value

    def diag(self, run=0):
        mass = np.zeros(self.nlevels)
        mom = np.zeros((self.nlevels, 3))
        rc = lib().lbm_diag(self._h, run, _dp(mass), _dp(mom))
        if rc not in (LBM_OK, -4):
            _check(rc, "lbm_diag")
        return mass, mom, rc == LBM_OK

    NOALLOC_MAX_NODES = 1 << 24

    def diag_noalloc(self, run=0):
        """lbm_diag without any allocation, for callers that cannot let the
        library allocate device memory (fixed memory budget, device memory
        owned by another pool, no room for cudaFree's synchronisation).
        Uses one fixed 2 MiB device array shared by every call: serialise
        calls that could overlap on the GPU.  Levels are limited to 2^24
        nodes."""
        for l in range(self.nlevels):
            if self.nodes(l) > self.NOALLOC_MAX_NODES:
                raise ValueError(f"level {l} has {self.nodes(l)} nodes; lbm_diag_noalloc "
                                 f"handles at most {self.NOALLOC_MAX_NODES}")
        mass = np.zeros(self.nlevels)
        mom = np.zeros((self.nlevels, 3))
        rc = lib().lbm_diag_noalloc(self._h, run, _dp(mass), _dp(mom))
        if rc not in (LBM_OK, -4):
            _check(rc, "lbm_diag_noalloc")
        return mass, mom, rc == LBM_OK

    def sync(self):
        _check(lib().lbm_sync(self._h), "lbm_sync")

    def kernel_launches(self) -> int:
        return int(lib().lbm_kernel_launches(self._h))

    def profile(self, enable: bool):
        _check(lib().lbm_profile(self._h, int(bool(enable))), "lbm_profile")

    def profile_read(self, kind: int, level: int = -1):
        """(total ms, launches) of one kernel kind: 0 level update,
        1 capture, 2 inject, 3 restrict, 4 probe; hybrid collision: 5 velocity
        pass, 6 parent strain history, 7 outer-layer collision."""
        t = ctypes.c_double()
        n = ctypes.c_longlong()
        _check(lib().lbm_profile_read(self._h, kind, level, ctypes.byref(t), ctypes.byref(n)),
               "lbm_profile_read")
        return t.value, n.value

    def close(self):
        if getattr(self, "_h", None):
            lib().lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
