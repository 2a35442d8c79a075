"""Seeded synthetic workloads: level layouts and initial macroscopic fields.

This module holds no part of the lattice Boltzmann arithmetic.  It only
describes *inputs*: the refinement layout of each workload (lattice, collision,
relaxation time, level boxes) and the initial density and velocity fields,
evaluated at every node of every level.  Both the CUDA library and the CPU
oracle consume these arrays, so the two sides always start from the same
numbers.

Initial conditions follow the paper's analytic setups:
  - convected vortex (Sec. 10.1, eq. init_COVO), with the density taken from
    the linearised relation rho0 [1 - eps^2/(2 cs^2) exp(-r^2/R^2)];
  - Gaussian acoustic pulse (Sec. 9.2, eq. init_Pulse), at rest unless a mean
    flow is given, half-width read as R in exp(-r^2/(2 R^2));
  - plane shear wave (Sec. 9.1 shape; a sine for decay-rate checks);
  - uniform flow.
Node positions are in level-0 (coarse) lattice units.  Level l has spacing
2^-l.  Nodes are numbered x fastest, then y, then z.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

CS = 1.0 / math.sqrt(3.0)

LATTICES = {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2}
COLLISIONS = {"BGK": 0, "REG": 1, "RR": 2, "HRR": 3}
Q_OF = {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}
DIM_OF = {"D2Q9": 2, "D3Q19": 3, "D3Q27": 3}


@dataclasses.dataclass
class Case:
    """One multi-level run: layout, physics parameters and initial state."""

    name: str
    lattice: str
    collision: str
    tau0: float
    dims: Tuple[int, int, int]
    boxes: List[Tuple[Tuple[int, int, int], Tuple[int, int, int]]]
    ic: dict
    steps: int
    rho0: float = 1.0
    sigma: float = 0.995  # hybrid weight, used when collision == "HRR"

    @property
    def u_ref(self):
        """Reference velocity for the shifted storage: the mean (free-stream)
        velocity of the initial condition."""
        return tuple(float(v) for v in self.ic.get("u0", (0.0, 0.0, 0.0)))

    @property
    def dim(self) -> int:
        return DIM_OF[self.lattice]

    @property
    def q(self) -> int:
        return Q_OF[self.lattice]

    @property
    def nlevels(self) -> int:
        return 1 + len(self.boxes)

    def with_(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


def level_layout(case: Case):
    """Per level: node counts n[3], periodic flags, origin (coarse units),
    spacing, and for l >= 1 the bounded-axis flags of its box."""
    D = case.dim
    out = []
    n = [case.dims[a] if a < D else 1 for a in range(3)]
    per = [True, True, True]
    origin = [0.0, 0.0, 0.0]
    h = 1.0
    out.append(dict(n=tuple(n), periodic=tuple(per), origin=tuple(origin),
                    h=h, boxed=(False, False, False)))
    for (lo, hi) in case.boxes:
        pn, pper, porg, ph = n, per, origin, h
        n, per, origin, boxed = [1, 1, 1], [True, True, True], [0.0] * 3, [False] * 3
        for a in range(3):
            if a >= D:
                continue
            E = hi[a] - lo[a]
            if pper[a] and lo[a] == 0 and E == pn[a]:
                n[a] = 2 * pn[a]
                origin[a] = porg[a]
            else:
                boxed[a] = True
                per[a] = False
                n[a] = 2 * E + 1
                origin[a] = porg[a] + lo[a] * ph
        h = ph / 2.0
        out.append(dict(n=tuple(n), periodic=tuple(per), origin=tuple(origin),
                        h=h, boxed=tuple(boxed)))
    return out


def level_coords(case: Case, level: int):
    """Node coordinates (X, Y, Z), each of shape [N], in coarse units,
    wrapped into the periodic level-0 domain."""
    lay = level_layout(case)[level]
    n, org, h = lay["n"], lay["origin"], lay["h"]
    axes = []
    for a in range(3):
        c = org[a] + h * np.arange(n[a], dtype=np.float64)
        if a < case.dim:
            c = np.mod(c, case.dims[a])
        axes.append(c)
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def _min_image(d, L):
    return d - L * np.round(d / L)


def initial_fields(case: Case, level: int):
    """rho [N] and u [3, N] (float64) at the nodes of one level."""
    X, Y, Z = level_coords(case, level)
    ic = case.ic
    kind = ic["kind"]
    rho0 = case.rho0
    N = X.size
    u = np.zeros((3, N), dtype=np.float64)
    U0 = np.asarray(ic.get("u0", (0.0, 0.0, 0.0)), dtype=np.float64)
    u += U0[:, None]
    if kind == "uniform":
        rho = np.full(N, rho0 + ic.get("drho", 0.0))
    elif kind == "vortex":
        xc, yc = ic["center"][0], ic["center"][1]
        R, eps = ic["radius"], ic["eps"]
        dx = _min_image(X - xc, case.dims[0])
        dy = _min_image(Y - yc, case.dims[1])
        r2 = dx * dx + dy * dy
        g = np.exp(-r2 / (2.0 * R * R))
        rho = rho0 * (1.0 - eps * eps / (2.0 * CS * CS) * g * g)
        u[0] += -eps * (dy / R) * g
        u[1] += eps * (dx / R) * g
    elif kind == "pulse":
        c = ic["center"]
        R, A = ic["radius"], ic["amplitude"]
        r2 = _min_image(X - c[0], case.dims[0]) ** 2 + _min_image(Y - c[1], case.dims[1]) ** 2
        if case.dim == 3:
            r2 = r2 + _min_image(Z - c[2], case.dims[2]) ** 2
        rho = rho0 * (1.0 + A * np.exp(-r2 / (2.0 * R * R)))
    elif kind == "shear":
        # u_t = U sin(2 pi x_n / L) with x_n along `axis`, u_t along `comp`
        ax, comp, U = ic["axis"], ic["comp"], ic["amplitude"]
        coord = (X, Y, Z)[ax]
        L = case.dims[ax]
        rho = np.full(N, rho0)
        u[comp] += U * np.sin(2.0 * np.pi * coord / L)
    elif kind == "vortex_exp":
        # barotropic vortex of eq. init_COVO: exponential density
        xc, yc = ic["center"][0], ic["center"][1]
        R, eps = ic["radius"], ic["eps"]
        dx = _min_image(X - xc, case.dims[0])
        dy = _min_image(Y - yc, case.dims[1])
        g = np.exp(-(dx * dx + dy * dy) / (2.0 * R * R))
        rho = rho0 * np.exp(-eps * eps / (2.0 * CS * CS) * g * g)
        u[0] += -eps * (dy / R) * g
        u[1] += eps * (dx / R) * g
    elif kind == "shear_gauss":
        # plane shear wave of eq. init_ShearW: u_y = U_y exp(-(x - xc)^2 / (2 R^2))
        g = np.exp(-_min_image(X - ic["xc"], case.dims[0]) ** 2 / (2.0 * ic["radius"] ** 2))
        rho = np.full(N, rho0)
        u[1] += ic["amplitude"] * g
    elif kind == "acoustic_gauss":
        # plane acoustic wave of eq. init_Pulse, travelling in -x relative to
        # the flow: rho' = rho0 A exp(-(x - xc)^2 / (2 R^2)), u_x = U_x - rho'/rho0 cs
        g = np.exp(-_min_image(X - ic["xc"], case.dims[0]) ** 2 / (2.0 * ic["radius"] ** 2))
        rp = rho0 * ic["amplitude"] * g
        rho = rho0 + rp
        u[0] -= rp / rho0 * CS
    elif kind == "random":
        rng = np.random.default_rng(ic["seed"])
        rho = rho0 + ic.get("drho", 1e-3) * rng.standard_normal(N)
        u += ic.get("du", 1e-2) * rng.standard_normal((3, N))
        if case.dim == 2:
            u[2] = 0.0
    else:
        raise ValueError(f"unknown initial condition {kind!r}")
    if case.dim == 2:
        u[2] = 0.0
    return rho, u


# --------------------------------------------------------------------------
# Validation setups of Sec. 9 and 10 (quasi-1D waves and the convected
# vortex), with periodic domains long enough that nothing that leaves the
# region of interest comes back within the measured window (the paper
# extends its domains with absorbing zones instead).  All in coarse units.
# --------------------------------------------------------------------------

def e4_shear_wave(collision: str = "RR", sigma: float = 0.995) -> Case:
    """Convected shear wave (Sec. 9.1, eqs. init_ShearW, init_ShearW2):
    U_x = U_y = 0.1 cs, R = 5, x_c = 150, nu = 1e-6; fine level on
    0 < x < 250, coarse elsewhere; 4 cells across (periodic), 1000 long."""
    return Case("e4_shear", "D2Q9", collision, 0.5 + 3e-6, (1000, 4, 1),
                [((0, 0, 0), (250, 4, 1))],
                dict(kind="shear_gauss", u0=(0.1 * CS, 0.0, 0.0), xc=150.0, radius=5.0,
                     amplitude=0.1 * CS), 2900, sigma=sigma)


def e5_acoustic_wave(collision: str = "RR", sigma: float = 0.995, length: int = 4000) -> Case:
    """Convected acoustic wave (Sec. 9.2, eqs. init_Pulse, init_Pulse2):
    A = 1e-4, R = 5, x_c = 750, U_x = 0.1 cs, nu = 1e-6; fine level on
    500 < x < 1000; 4 cells across (periodic), `length` long."""
    return Case("e5_acoustic", "D2Q9", collision, 0.5 + 3e-6, (length, 4, 1),
                [((500, 0, 0), (1000, 4, 1))],
                dict(kind="acoustic_gauss", u0=(0.1 * CS, 0.0, 0.0), xc=750.0, radius=5.0,
                     amplitude=1e-4), 2620, sigma=sigma)


def e6_vortex(collision: str = "RR", sigma: float = 0.995, nu: float = 1e-6,
              height: int = 1200, length: int = 1200) -> Case:
    """Convected barotropic vortex (Sec. 10, eqs. init_COVO, init_COVO2):
    U_x = 0.1 cs, eps = 0.15 U_x, R = 5, centre (100, 75) shifted to mid
    height, nu as given; fine level on 0 < x < 150 over the whole height;
    periodic `length` x `height` domain."""
    tau = 0.5 + nu / (CS * CS)
    return Case("e6_vortex", "D2Q9", collision, tau, (length, height, 1),
                [((0, 0, 0), (150, height, 1))],
                dict(kind="vortex_exp", u0=(0.1 * CS, 0.0, 0.0),
                     center=(100.0, height / 2.0), radius=5.0, eps=0.15 * 0.1 * CS), 1100,
                sigma=sigma)


def e6_probe(case: Case):
    """Probe P1 of Sec. 10 (x = 200, 50 cells off the vortex path)."""
    return (200, int(case.ic["center"][1]) + 50, 0)


# --------------------------------------------------------------------------
# Workload shapes.  The four single-run configurations of the build plan,
# plus reduced variants with the same structure that the CPU oracle finishes
# in seconds.
# --------------------------------------------------------------------------

def vortex_2level_d2q9(steps: int = 400) -> Case:
    """Coarse 128x64 D2Q9, fine patch x in [64,128] (y periodic), RR,
    tau_c = 0.51, vortex R=5, eps = 0.05 cs on U0 = 0.1 cs at (32,32)."""
    return Case("vortex2d", "D2Q9", "RR", 0.51, (128, 64, 1),
                [((64, 0, 0), (128, 64, 1))],
                dict(kind="vortex", u0=(0.1 * CS, 0.0, 0.0), center=(32.0, 32.0),
                     radius=5.0, eps=0.05 * CS), steps)


def pulse_2level_d2q9(collision: str = "RR", steps: int = 1500) -> Case:
    """Coarse 512^2 D2Q9, centred fine box [128,384]^2 (513^2 fine nodes),
    tau_c = 0.5 + 1e-4, pulse A = 1e-3, R = 6 at (88, 256), at rest."""
    return Case(f"pulse2d_{collision.lower()}", "D2Q9", collision, 0.5 + 1e-4,
                (512, 512, 1), [((128, 128, 0), (384, 384, 1))],
                dict(kind="pulse", center=(88.0, 256.0, 0.0), radius=6.0,
                     amplitude=1e-3), steps)


def vortex_slab_d3q19(steps: int = 500, side: int = 256, yz: int = 0) -> Case:
    """Coarse side^3 D3Q19 (256^3), fine slab x in [side/2, side] (y, z
    periodic), RR, tau_c = 0.5 + 5e-5, vortex column about z, R = 8, at
    (side/2 - 28, side/2): (100, 128) at full size, so that the vortex centre
    reaches the interface after 500 steps at 0.1 c_s.  Smaller sides keep the
    structure for bounded oracle runs; yz > 0 shrinks only the periodic y
    and z extents (same rows as the full size, for profiling captures)."""
    ny = yz or side
    name = ("vortex3d" if side == 256 else f"vortex3d_{side}") + (f"_yz{yz}" if yz else "")
    return Case(name, "D3Q19", "RR", 0.5 + 5e-5, (side, ny, ny),
                [((side // 2, 0, 0), (side, ny, ny))],
                dict(kind="vortex", u0=(0.1 * CS, 0.0, 0.0),
                     center=(side / 2.0 - 28.0, ny / 2.0),
                     radius=8.0, eps=0.05 * CS), steps)


def pulse_3level_d3q27(steps: int = 800, side: int = 192) -> Case:
    """Coarse side^3 D3Q27 (192^3), level 1 on the central half [side/4,
    3 side/4]^3 (193^3 nodes), level 2 on the central half of level 1, i.e.
    [side/4, 3 side/4]^3 in level-1 node units (193^3 nodes), RR, tau_c =
    0.5 + 1e-4, pulse A = 1e-3, R = 4 at (side/2 + 3 side/16, side/2,
    side/2): (132, 96, 96) at full size, inside level 1 and outside level 2.
    Smaller sides keep the structure for bounded oracle runs."""
    q = side // 4
    name = "pulse3d" if side == 192 else f"pulse3d_{side}"
    return Case(name, "D3Q27", "RR", 0.5 + 1e-4, (side, side, side),
                [((q, q, q), (3 * q, 3 * q, 3 * q)), ((q, q, q), (3 * q, 3 * q, 3 * q))],
                dict(kind="pulse", center=(side / 2.0 + 3.0 * side / 16.0, side / 2.0,
                                           side / 2.0), radius=4.0,
                     amplitude=1e-3), steps)


def small_2level_2d(collision="RR", ic=None, steps=40, tau0=0.52) -> Case:
    """96x64 coarse, fine box [24,72]x[16,48]: several tiles and a ragged
    tail on both levels, corners included."""
    ic = ic or dict(kind="vortex", u0=(0.1 * CS, 0.0, 0.0), center=(30.0, 32.0),
                    radius=4.0, eps=0.05 * CS)
    return Case("small2d", "D2Q9", collision, tau0, (96, 64, 1),
                [((24, 16, 0), (72, 48, 1))], ic, steps)


def small_3d(lattice="D3Q19", collision="RR", nlevels=2, ic=None, steps=6,
             tau0=0.52) -> Case:
    """Reduced 3D layouts with the structure of the slab and nested cases."""
    if nlevels == 1:
        boxes = []
        dims = (20, 12, 10)
    elif nlevels == 2:
        dims = (24, 20, 16)
        boxes = [((6, 5, 4), (18, 15, 12))]
    else:
        dims = (28, 24, 24)
        boxes = [((6, 6, 6), (22, 18, 18)), ((8, 6, 6), (24, 18, 18))]
    ic = ic or dict(kind="pulse", center=(12.0, 10.0, 8.0), radius=2.5,
                    amplitude=1e-3, u0=(0.05 * CS, 0.02 * CS, 0.01 * CS))
    return Case(f"small3d_{lattice}_{nlevels}", lattice, collision, tau0, dims,
                boxes, ic, steps)


def slab_small_3d(lattice="D3Q19", collision="RR", steps=10) -> Case:
    """64x32x16 coarse with a periodic fine slab x in [32,64]."""
    return Case("slab3d_small", lattice, collision, 0.5 + 5e-3, (64, 32, 16),
                [((32, 0, 0), (64, 32, 16))],
                dict(kind="vortex", u0=(0.1 * CS, 0.0, 0.0), center=(24.0, 16.0),
                     radius=4.0, eps=0.05 * CS), steps)


CONFIGS = {
    "vortex2d": vortex_2level_d2q9,
    "pulse2d": pulse_2level_d2q9,
    "vortex3d": vortex_slab_d3q19,
    "pulse3d": pulse_3level_d3q27,
}


def updates_per_coarse_step(case: Case, active_counts: Sequence[int]) -> int:
    """Node updates per coarse step, each level at its own rate: sum 2^l N_l."""
    return int(sum((2 ** l) * int(n) for l, n in enumerate(active_counts)))


# --------------------------------------------------------------------------
# Serving stream: mixed runs arriving as a Poisson process.
# --------------------------------------------------------------------------

def _central_half_boxes(dim: int, side: int, nlevels: int):
    """Each child box covers the central half of its parent on every axis."""
    boxes = []
    n = side  # parent node count per axis (level 0: periodic, side nodes)
    for l in range(1, nlevels):
        if l == 1:
            lo, hi = n // 4, n - n // 4
            nc = 2 * (hi - lo) + 1
        else:
            lo, hi = n // 4, n - 1 - n // 4
            nc = 2 * (hi - lo) + 1
        boxes.append((tuple([lo] * dim + [0] * (3 - dim)),
                      tuple([hi] * dim + [1] * (3 - dim))))
        n = nc
    return boxes


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float     # seconds after the stream starts
    case: Case


def serving_requests(n: int, rate: float, seed: int = 20041186, step_scale: float = 1.0,
                     size_scale: float = 1.0) -> List[Request]:
    """Seeded request stream shaped like the serving workload: lattice D2Q9
    (1/2), D3Q19 (1/4), D3Q27 (1/4); 2D coarse side in {64, 80, .., 1024},
    3D in {48, 64, .., 160}; 1-3 levels, each child box the central half of
    its parent; Mach 0.05-0.2 along x; tau_c - 1/2 log-uniform in
    [1e-5, 1e-2]; vortex or pulse (1/2 each); 100-1000 coarse steps; RR.
    Arrivals are a Poisson process of `rate` requests per second.
    step_scale / size_scale shrink steps and sides for bounded test runs."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        lat = rng.choice(["D2Q9", "D3Q19", "D3Q27"], p=[0.5, 0.25, 0.25])
        dim = DIM_OF[lat]
        if dim == 2:
            side = int(rng.choice(np.arange(64, 1025, 16)))
        else:
            side = int(rng.choice(np.arange(48, 161, 16)))
        side = max(48 if dim == 3 else 64, int(round(side * size_scale / 16)) * 16)
        nlev = int(rng.integers(1, 4))
        ma = rng.uniform(0.05, 0.2)
        tau0 = 0.5 + 10.0 ** rng.uniform(-5, -2)
        steps = max(4, int(round(rng.integers(100, 1001) * step_scale)))
        u0 = (ma * CS, 0.0, 0.0)
        c = side / 2.0
        if rng.random() < 0.5:
            ic = dict(kind="vortex", u0=u0, center=(c * 0.6, c, 0.0), radius=side / 24.0,
                      eps=0.05 * CS)
        else:
            ic = dict(kind="pulse", u0=u0, center=(c * 0.6, c, c if dim == 3 else 0.0),
                      radius=side / 32.0, amplitude=1e-3)
        dims = (side, side, side if dim == 3 else 1)
        case = Case(f"req{k}", lat, "RR", float(tau0), dims,
                    _central_half_boxes(dim, side, nlev), ic, steps)
        out.append(Request(k, t, case))
    return out
