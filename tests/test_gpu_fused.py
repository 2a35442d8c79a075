"""Persistent fused step (lbm_set_fused): every coarse step after the first
runs as one cooperative kernel with grid barriers between its phases.  The
results must match the FP64 oracle within the binary32 tolerance, agree
with the per-kernel path, keep the probe record, and a barrier wait that
runs out must come back as an error status with the GPU still usable."""
import numpy as np
import pytest

import oracle
from paper_2004_11863_gb300 import workloads as W
from tests.test_gpu_parity import FOUR_LEVELS

pytestmark = pytest.mark.gpu

TOL32 = 1e-6


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2004_11863_gb300 import build
    build.build()
    from paper_2004_11863_gb300 import mlbm
    return mlbm


def compare(g, o, nlev, run=0, tol=TOL32):
    for l in range(nlev):
        rg, ug = g.macros(l, run)
        ro, uo = o.macros(l)
        m = ~np.isnan(ro)
        assert np.array_equal(np.isnan(rg), ~m)
        dr = np.max(np.abs(rg[m] - ro[m]))
        du = np.max(np.abs(ug[:, m] - uo[:, m]))
        assert dr <= tol and du <= tol, (l, dr, du)


CASES = [
    ("small2d_rr", lambda: W.small_2level_2d("RR", steps=30)),
    ("small2d_bgk", lambda: W.small_2level_2d("BGK", steps=20)),
    ("small2d_reg", lambda: W.small_2level_2d("REG", steps=20)),
    ("vortex2d", lambda: W.vortex_2level_d2q9(steps=25)),
    ("band2d", lambda: W.Case("band2d", "D2Q9", "RR", 0.52, (70, 48, 1),
                              [((0, 12, 0), (70, 36, 1))],
                              dict(kind="vortex", u0=(0.0, 0.1 * W.CS, 0.0),
                                   center=(66.0, 16.0, 0.0), radius=4.0, eps=0.05 * W.CS), 20)),
    ("d3q19_2lev", lambda: W.small_3d("D3Q19", "RR", nlevels=2, steps=6)),
    ("d3q27_3lev", lambda: W.small_3d("D3Q27", "RR", nlevels=3, steps=4)),
    ("d3q19_slab", lambda: W.slab_small_3d("D3Q19", "RR", steps=6)),
    ("four_levels_2d", lambda: FOUR_LEVELS),
    ("d3q27_tube", lambda: W.Case("tube3d", "D3Q27", "RR", 0.52, (29, 16, 17),
                                  [((0, 4, 4), (29, 12, 13))],
                                  dict(kind="pulse", center=(27.0, 6.0, 8.0), radius=3.0,
                                       amplitude=1e-3, u0=(0.05, 0.0, 0.0)), 5)),
]


@pytest.mark.parametrize("name,mk", CASES, ids=[c[0] for c in CASES])
def test_fused_matches_oracle(M, name, mk):
    case = mk()
    g = M.Lbm.from_case(case)
    g.set_fused(1)
    o = oracle.Run.from_case(case)
    g.step(case.steps)
    o.step(case.steps)
    g.sync()
    compare(g, o, case.nlevels)


def test_fused_one_launch_per_call(M):
    """After the first coarse step, one lbm_step call is one kernel."""
    case = W.small_3d("D3Q19", "RR", nlevels=2, steps=6)
    g = M.Lbm.from_case(case)
    g.set_fused(1)
    g.step(1)
    n0 = g.kernel_launches()
    g.step(7)
    assert g.kernel_launches() - n0 == 1
    g.step(1)
    assert g.kernel_launches() - n0 == 2


def test_fused_agrees_with_per_kernel_path_batch_and_split_calls(M):
    """A batch of two runs, stepped in uneven calls (the six-step program
    cycle starts at different keys), with a moving reference and probes:
    fields and probe records agree with the per-kernel path."""
    c1 = W.small_3d("D3Q27", "RR", nlevels=2, steps=9)
    c2 = c1.with_(ic=dict(kind="pulse", center=(8.0, 9.0, 6.0), radius=3.0, amplitude=2e-3))
    runs = []
    for fused in (0, 1):
        g = M.Lbm(c1.lattice, c1.collision, c1.tau0, c1.dims, c1.boxes, batch=2,
                  u_ref=(0.03, -0.01, 0.02))
        for l in range(2):
            g.init(l, 0, *W.initial_fields(c1, l))
            g.init(l, 1, *W.initial_fields(c2, l))
        g.set_fused(fused)
        g.probe_add(1, [[4, 5, 6], [12, 10, 9]])
        for n in (1, 4, 2, 5, 1):
            g.step(n)
        runs.append((g, g.probe()))
    (a, pa), (b, pb) = runs
    assert pa.shape == pb.shape == (13, 2, 2, 4)
    assert np.max(np.abs(pa - pb)) <= TOL32
    for l in range(2):
        for run in range(2):
            ra, ua = a.macros(l, run)
            rb, ub = b.macros(l, run)
            m = ~np.isnan(ra)
            assert np.array_equal(m, ~np.isnan(rb))
            assert np.max(np.abs(ra[m] - rb[m])) <= TOL32
            assert np.max(np.abs(ua[:, m] - ub[:, m])) <= TOL32


def test_fused_fp16_pairs_within_bound(M):
    """binary16 storage with run pairs (es = 2) through the fused step."""
    from tests.test_gpu_parity import fp16_bound
    case = W.small_2level_2d("RR", steps=30)
    g = M.Lbm.from_case(case, storage="fp16", batch=2)
    g.set_fused(1)
    o = oracle.Run.from_case(case)
    tol = fp16_bound(case, o)
    g.step(case.steps)
    o.step(case.steps)
    for run in range(2):
        compare(g, o, case.nlevels, run=run, tol=tol)


def test_fused_barrier_timeout_is_reported(M):
    """Mode 2 makes every barrier wait for a block that does not exist: each
    wait gives up after its bound, the kernel returns, lbm_sync reports
    LBM_ETIMEOUT, and the GPU keeps working for a new run."""
    case = W.small_2level_2d("RR", steps=5)
    g = M.Lbm.from_case(case)
    g.set_fused(2)
    g.step(1)   # the first coarse step runs on the per-kernel path
    g.step(3)
    with pytest.raises(M.LbmError) as e:
        g.sync()
    assert e.value.code == -6
    with pytest.raises(M.LbmError):
        g.step(1)
    g.close()
    h = M.Lbm.from_case(case)
    h.set_fused(1)
    o = oracle.Run.from_case(case)
    h.step(case.steps)
    o.step(case.steps)
    compare(h, o, case.nlevels)


def test_fused_refuses_hybrid_collision(M):
    case = W.small_2level_2d("RR").with_(collision="HRR", sigma=0.5)
    g = M.Lbm.from_case(case)
    with pytest.raises(M.LbmError):
        g.set_fused(1)
