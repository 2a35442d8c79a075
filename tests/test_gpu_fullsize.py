"""Parity at the full sizes of the four workloads, in the launch
configuration bench.py times, against the FP64 oracle element by element.

- vortex2d (coarse 128x64, fine 129x128, RR): the full 400 coarse steps;
- pulse2d (coarse 512^2, fine 513^2): RR and BGK for the full 1500 coarse
  steps, as a batch of 33 runs (the benchmark's batch) of which two are
  compared with the oracle, in binary32 (1e-6) and in binary16 shifted
  storage (run pairs, the stated bound); and the spurious-noise measure
  (max over t <= 450 coarse steps of the density difference to the
  single-level run outside the fine box) against the oracle's;
- vortex3d (coarse 256^3 + fine 257x512x512, D3Q19 RR) and pulse3d (coarse
  192^3 + two 193^3 levels, D3Q27 RR): 2 coarse steps at full size (the
  oracle needs 26 GB and 12 GB of host memory; skipped with a reason when the
  host has less), plus properties that hold at any length: a uniform flow
  stays uniform and two runs are bitwise identical.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2004_11863_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-6
BENCH_BATCH = 33


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2004_11863_gb300 import build
    build.build()
    from paper_2004_11863_gb300 import mlbm
    return mlbm


def host_mem_gb():
    with open("/proc/meminfo") as fh:
        for line in fh:
            if line.startswith("MemAvailable"):
                return int(line.split()[1]) / 1e6
    return 0.0


def max_err(g, o, nlev, run=0):
    dr = du = 0.0
    for l in range(nlev):
        rg, ug = g.macros(l, run)
        ro, uo = o.macros(l)
        m = ~np.isnan(ro)
        assert np.array_equal(np.isnan(rg), ~m)
        dr = max(dr, float(np.max(np.abs(rg[m] - ro[m]))))
        du = max(du, float(np.max(np.abs(ug[:, m] - uo[:, m]))))
    return dr, du


def test_vortex2d_full_400_steps(M):
    case = W.vortex_2level_d2q9(steps=400)
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(case.steps)
    o.step(case.steps)
    dr, du = max_err(g, o, 2)
    assert dr <= TOL32 and du <= TOL32, (dr, du)


_ORACLE = {}


def oracle_pulse2d(collision, steps=1500):
    """The oracle's pulse2d run after `steps` coarse steps (computed once per
    session, shared by the binary32 and binary16 checks)."""
    key = (collision, steps)
    if key not in _ORACLE:
        o = oracle.Run.from_case(W.pulse_2level_d2q9(collision, steps=steps))
        o.step(steps)
        _ORACLE[key] = o
    return _ORACLE[key]


def pulse2d_batch(M, case, storage):
    """The benchmark's 33-run batch: runs 0 and 32 carry the workload's
    pulse, the others a pulse at another place."""
    other = case.with_(ic=dict(kind="pulse", center=(300.0, 200.0, 0.0), radius=6.0,
                               amplitude=1e-3))
    g = M.Lbm(case.lattice, case.collision, case.tau0, case.dims, case.boxes,
              storage=storage, batch=BENCH_BATCH)
    for l in range(2):
        f0 = W.initial_fields(case, l)
        f1 = W.initial_fields(other, l)
        for b in range(BENCH_BATCH):
            g.init(l, b, *(f0 if b in (0, BENCH_BATCH - 1) else f1))
    g.autotune(reps=2)
    return g


def fp16_bound(case):
    """Stated error bound of binary16 shifted storage (derivation in
    test_gpu_parity.fp16_bound): 2 q^(1/2) 2^-11 gmax n^(1/2), gmax the
    largest stored deviation of the initial state, n the finest-level
    updates."""
    from tests.test_gpu_parity import fp16_bound as b
    o = oracle.Run.from_case(case)
    try:
        return b(case, o)
    finally:
        o.close()


@pytest.mark.parametrize("collision", ["RR", "BGK"])
@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_pulse2d_full_in_bench_batch(M, collision, storage):
    """Runs 0 and 32 of a 33-run batch (the benchmark launch) against the
    oracle after the full 1500 coarse steps; binary16 batches are stored as
    interleaved run pairs (run 32 is the first of the last, half-empty
    pair)."""
    case = W.pulse_2level_d2q9(collision, steps=1500)
    tol = TOL32 if storage == "fp32" else fp16_bound(case)
    g = pulse2d_batch(M, case, storage)
    g.step(case.steps)
    o = oracle_pulse2d(collision, case.steps)
    for run in (0, BENCH_BATCH - 1):
        dr, du = max_err(g, o, 2, run)
        print(f"pulse2d {collision} {storage} run {run}: max|drho| {dr:.3e} max|du| {du:.3e} "
              f"(bound {tol:.3e})")
        assert dr <= tol and du <= tol, (run, dr, du, tol)
    g.close()


def _noise_max(case, r2, r1, margin):
    """R23 noise measure on the host (the definition lbm_noise reduces on
    the device): max |rho_2lev - rho_1lev| over level-0 nodes outside the
    fine box grown by `margin` cells."""
    from tests.test_gpu_features import _noise_numpy
    return float(_noise_numpy(case, r2, r1, margin)[0])


def test_pulse2d_noise_measure_per_precision_and_collision(M):
    """Spurious-noise measure of the acoustic-pulse workload (the density
    difference between the two-level run and the same state on the uniform
    coarse grid, outside the fine box by >= 4 cells), sampled every 5
    coarse steps up to t = 450 (before the transmitted wave leaves the fine
    box), maximum over the samples: binary32 and binary16 storage, BGK and
    RR, against the FP64 oracle's value.  binary32 within 1e-6; binary16
    within the stated storage bound."""
    T, every, margin = 450, 5, 4
    rows = []
    for collision in ("BGK", "RR"):
        case = W.pulse_2level_d2q9(collision, steps=T)
        single = case.with_(boxes=[])
        o2 = oracle.Run.from_case(case)
        o1 = oracle.Run.from_case(single)
        onoise = 0.0
        for _ in range(T // every):
            o2.step(every)
            o1.step(every)
            onoise = max(onoise, _noise_max(case, o2.macros(0)[0], o1.macros(0)[0], margin))
        o2.close()
        o1.close()
        for storage in ("fp32", "fp16"):
            g2 = M.Lbm.from_case(case, storage=storage)
            g1 = M.Lbm.from_case(single, storage=storage)
            gnoise = 0.0
            for _ in range(T // every):
                g2.step(every)
                g1.step(every)
                gnoise = max(gnoise, g2.noise(g1, margin=margin)[0])
            g2.close()
            g1.close()
            tol = TOL32 if storage == "fp32" else 2 * fp16_bound(case)
            rows.append((collision, storage, gnoise, onoise, tol))
    for c, st, gn, on, tol in rows:
        print(f"noise R23 pulse2d {c} {st}: GPU {gn:.6e} oracle {on:.6e} "
              f"diff {abs(gn - on):.2e} (tolerance {tol:.2e})")
    for c, st, gn, on, tol in rows:
        assert gn > 0 and abs(gn - on) <= tol, (c, st, gn, on, tol)


def _full3d(M, case, need_gb, steps=2):
    if host_mem_gb() < need_gb:
        pytest.skip(f"the FP64 oracle of {case.name} needs ~{need_gb} GB of host memory; "
                    f"{host_mem_gb():.0f} GB available")
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(steps)
    o.step(steps)
    dr, du = max_err(g, o, case.nlevels)
    assert dr <= TOL32 and du <= TOL32, (dr, du)


def test_vortex3d_full_size_parity(M):
    _full3d(M, W.vortex_slab_d3q19(), need_gb=40)


def test_pulse3d_full_size_parity(M):
    _full3d(M, W.pulse_3level_d3q27(), need_gb=24)


@pytest.mark.parametrize("mk", [W.vortex_slab_d3q19, W.pulse_3level_d3q27],
                         ids=["vortex3d", "pulse3d"])
def test_full_size_uniform_flow_and_determinism(M, mk):
    """At full size: a uniform flow stays uniform to binary32 round-off after
    20 coarse steps on every level, and a second run gives the same bits."""
    case = mk().with_(ic=dict(kind="uniform", u0=(0.1 * W.CS, 0.0, 0.0)))
    g = M.Lbm.from_case(case)
    g.step(20)
    first = []
    for l in range(case.nlevels):
        r, u = g.macros(l)
        m = ~np.isnan(r)
        assert np.max(np.abs(r[m] - 1.0)) < 1e-6
        assert np.max(np.abs(u[0, m] - 0.1 * W.CS)) < 1e-6
        first.append((r, u))
    g.close()
    case2 = mk()
    a = M.Lbm.from_case(case2)
    b = M.Lbm.from_case(case2)
    a.step(3)
    b.step(3)
    for l in range(case2.nlevels):
        ra, ua = a.macros(l)
        rb, ub = b.macros(l)
        assert np.array_equal(ra, rb, equal_nan=True) and np.array_equal(ua, ub, equal_nan=True)
