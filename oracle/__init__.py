"""ctypes wrapper of the FP64 CPU oracle (mlbm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg.  The product library never imports it.

The shared library is compiled from ``mlbm_oracle.c`` with gcc on first use
(or by ``__graft_entry__.build()``), in IEEE double precision without FMA
contraction.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mlbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LATTICE = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2}
COLLISION = {"BGK": 0, "REG": 1, "RR": 2, "HRR": 3}


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place; returns its path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mlbm_oracle.h"))):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.orc_lattice.argtypes = [ctypes.c_int, ip, dp]
            L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, dp, dp]
            L.orc_a1.argtypes = [ctypes.c_int, dp, dp]
            L.orc_collide.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
            L.orc_collide_hrr.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          dp, dp, dp]
            L.orc_interp_time.argtypes = [ctypes.c_double] * 3 + [ctypes.c_int]
            L.orc_interp_time.restype = ctypes.c_double
            L.orc_interp_space.argtypes = [ctypes.c_double] * 4
            L.orc_interp_space.restype = ctypes.c_double
            L.orc_filter_weight.argtypes = [ctypes.c_int] * 4
            L.orc_filter_weight.restype = ctypes.c_double
            L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, ip, ctypes.c_int, ip]
            L.orc_create.restype = ctypes.c_void_p
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_level_dims.argtypes = [ctypes.c_void_p, ctypes.c_int, ip]
            L.orc_level_tau.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_level_tau.restype = ctypes.c_double
            L.orc_level_classes.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_ubyte)]
            L.orc_init_level.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp]
            L.orc_init_done.argtypes = [ctypes.c_void_p]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_macros.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp]
            L.orc_populations.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
            L.orc_set_sigma.argtypes = [ctypes.c_void_p, ctypes.c_double]
            L.orc_sensors_enable.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double]
            L.orc_sensors.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_ubyte), dp, dp, dp]
            L.orc_set_populations.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
            L.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def lattice(name: str):
    xi = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27, dtype=np.float64)
    q = lib().orc_lattice(LATTICE[name], _ip(xi), _dp(w))
    return xi[:q].copy(), w[:q].copy()


def feq(name: str, rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3))
    out = np.zeros(27)
    lib().orc_feq(LATTICE[name], float(rho), _dp(u), _dp(out))
    return out[: lattice_q(name)].copy()


def lattice_q(name: str) -> int:
    return {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}[name]


def a1(name: str, f) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    out = np.zeros(9)
    lib().orc_a1(LATTICE[name], _dp(f), _dp(out))
    return out.reshape(3, 3)


def collide(name: str, collision: str, tau: float, f) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    out = np.zeros_like(f)
    lib().orc_collide(LATTICE[name], COLLISION[collision], float(tau), _dp(f), _dp(out))
    return out


def collide_hrr(name: str, tau: float, sigma: float, f, S6) -> np.ndarray:
    """H-RR collision with a given strain rate S6 = (xx, yy, zz, xy, xz, yz)."""
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
    S6 = np.ascontiguousarray(np.asarray(S6, dtype=np.float64).reshape(6))
    out = np.zeros_like(f)
    lib().orc_collide_hrr(LATTICE[name], float(tau), float(sigma), _dp(f), _dp(S6), _dp(out))
    return out


def interp_time(gm1, g0, gp1, first=False) -> float:
    return lib().orc_interp_time(gm1, g0, gp1, int(bool(first)))


def interp_space(gm3, gm1, gp1, gp3) -> float:
    return lib().orc_interp_space(gm3, gm1, gp1, gp3)


def filter_weight(d, dx, dy, dz) -> float:
    return lib().orc_filter_weight(d, dx, dy, dz)


class Run:
    """A multi-level FP64 run driven through the oracle's C API."""

    def __init__(self, lattice_name, collision, tau0, dims, boxes, rho0=1.0):
        self.lattice = lattice_name
        self.q = lattice_q(lattice_name)
        d = np.asarray(list(dims) + [1] * (3 - len(dims)), dtype=np.int32)[:3]
        nlev = 1 + len(boxes)
        b = np.zeros(max(1, 6 * len(boxes)), dtype=np.int32)
        for k, (lo, hi) in enumerate(boxes):
            b[6 * k: 6 * k + 3] = lo
            b[6 * k + 3: 6 * k + 6] = hi
        self._b = b
        self._h = lib().orc_create(LATTICE[lattice_name], COLLISION[collision],
                                   float(tau0), float(rho0), _ip(d), nlev, _ip(b))
        if not self._h:
            raise ValueError("oracle rejected the level layout")
        self.nlevels = nlev

    @classmethod
    def from_case(cls, case, init=True, sigma=None):
        r = cls(case.lattice, case.collision, case.tau0, case.dims, case.boxes, case.rho0)
        if sigma is None and case.collision == "HRR":
            sigma = case.sigma
        if sigma is not None:
            r.set_sigma(sigma)
        if init:
            from paper_2004_11863_gb300 import workloads
            for l in range(r.nlevels):
                rho, u = workloads.initial_fields(case, l)
                r.init_level(l, rho, u)
            r.init_done()
        return r

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dims(self, level):
        n = np.zeros(3, dtype=np.int32)
        N = lib().orc_level_dims(self._h, level, _ip(n))
        return tuple(int(v) for v in n), N

    def tau(self, level):
        return lib().orc_level_tau(self._h, level)

    def classes(self, level):
        _, N = self.dims(level)
        c = np.zeros(N, dtype=np.uint8)
        lib().orc_level_classes(self._h, level, c.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return c

    def init_level(self, level, rho, u):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, -1)
        _, N = self.dims(level)
        assert rho.size == N and u.shape[1] == N
        lib().orc_init_level(self._h, level, _dp(rho), _dp(u))

    def set_sigma(self, sigma):
        """Hybrid weight of the H-RR collision (call before init_done)."""
        if lib().orc_set_sigma(self._h, float(sigma)) != 0:
            raise ValueError("sigma must lie in [0, 1]")

    def sensors_enable(self, level, eps=0.0, g_threshold=0.0):
        """Evaluate the non-hydrodynamic mode sensors of a level from now on
        (eps: magnitude floor of the sign tests; g_threshold: of |f1G|)."""
        if lib().orc_sensors_enable(self._h, level, float(eps), float(g_threshold)) != 0:
            raise ValueError("bad sensor arguments")

    def sensors(self, level, with_gnorm=False):
        """Latest sensor flags [N] (bit 0 spuriousAc, 1 spuriousS, 2
        spuriousG), div u [N] and curl u [3, N] of a level (and |f1G| [N])."""
        _, N = self.dims(level)
        fl = np.zeros(N, dtype=np.uint8)
        dv = np.zeros(N)
        cu = np.zeros((3, N))
        gn = np.zeros(N)
        if lib().orc_sensors(self._h, level, fl.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                             _dp(dv), _dp(cu), _dp(gn)) != 0:
            raise ValueError("sensors not enabled on this level")
        return (fl, dv, cu, gn) if with_gnorm else (fl, dv, cu)

    def set_populations(self, level, f):
        """Set a level's (post-collision) populations, f [q, N]."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        _, N = self.dims(level)
        assert f.shape == (self.q, N)
        lib().orc_set_populations(self._h, level, _dp(f))

    def init_done(self):
        lib().orc_init_done(self._h)

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def macros(self, level):
        _, N = self.dims(level)
        rho = np.zeros(N)
        u = np.zeros((3, N))
        lib().orc_macros(self._h, level, _dp(rho), _dp(u))
        return rho, u

    def populations(self, level):
        _, N = self.dims(level)
        f = np.zeros((self.q, N))
        lib().orc_populations(self._h, level, _dp(f))
        return f
