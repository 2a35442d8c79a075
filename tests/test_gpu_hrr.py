"""GPU parity of the hybrid recursive regularized collision (H-RR, eq.
a1ij_HRR) with its Sec. 4.4 strain-rate transfers, against the FP64 oracle,
through the C ABI.  sigma = 0.5 makes the finite-difference strain (and so
every transfer of it) weigh as much as the projected stress; sigma = 0.995
is the paper's setting."""
import numpy as np
import pytest

import oracle
from paper_2004_11863_gb300 import workloads as W

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


SEAM = W.Case("seam2d", "D2Q9", "HRR", 0.52, (64, 48, 1), [((40, 0, 0), (64, 48, 1))],
              dict(kind="vortex", u0=(0.1 * W.CS, 0.0, 0.0), center=(40.0, 24.0, 0.0),
                   radius=4.0, eps=0.05), 30)

CASES = {
    "2d": (lambda: W.small_2level_2d("RR"), 30),
    "2d_seam": (lambda: SEAM, 30),
    "3d_d3q19": (lambda: W.small_3d("D3Q19", nlevels=2), 6),
    "3d_d3q27_3lev": (lambda: W.small_3d("D3Q27", nlevels=3), 4),
    "3d_slab": (lambda: W.slab_small_3d("D3Q19"), 6),
}


@pytest.mark.parametrize("sigma", [0.5, 0.995])
@pytest.mark.parametrize("key", list(CASES))
def test_hrr_parity(M, key, sigma):
    mk, steps = CASES[key]
    case = mk().with_(collision="HRR", sigma=sigma)
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(steps)
    o.step(steps)
    dr, du = max_err(g, o, case.nlevels)
    assert dr <= TOL32 and du <= TOL32, (dr, du)


def test_hrr_pure_finite_difference(M):
    """sigma = 0: the stress comes from the finite differences alone."""
    case = W.small_2level_2d("RR").with_(collision="HRR", sigma=0.0)
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(20)
    o.step(20)
    dr, du = max_err(g, o, 2)
    assert dr <= TOL32 and du <= TOL32, (dr, du)


def test_hrr_vortex2d_full(M):
    """The convected-vortex workload at full size, H-RR sigma = 0.995, the
    first 200 coarse steps (the vortex reaches the interface)."""
    case = W.vortex_2level_d2q9(steps=200).with_(collision="HRR", sigma=0.995)
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(case.steps)
    o.step(case.steps)
    dr, du = max_err(g, o, 2)
    assert dr <= TOL32 and du <= TOL32, (dr, du)


def test_hrr_batch_graphs_and_eager_agree(M):
    """A batch of two runs stepped through the CUDA graphs equals the same
    runs stepped eagerly, bit for bit, and run 1 (another initial state)
    matches its own oracle run."""
    case = W.small_3d("D3Q19", nlevels=2).with_(collision="HRR", sigma=0.5)
    other = case.with_(ic=dict(kind="pulse", center=(10.0, 12.0, 8.0), radius=3.0,
                               amplitude=1e-3))
    runs = []
    for graphs in (True, False):
        g = M.Lbm.from_case(case, batch=2, init=False)
        for l in range(case.nlevels):
            g.init(l, 0, *W.initial_fields(case, l))
            g.init(l, 1, *W.initial_fields(other, l))
        g.set_graphs(graphs)
        g.step(8)
        runs.append(g)
    for l in range(case.nlevels):
        for run in (0, 1):
            ra, ua = runs[0].macros(l, run)
            rb, ub = runs[1].macros(l, run)
            assert np.array_equal(ra, rb, equal_nan=True) and np.array_equal(ua, ub, equal_nan=True)
    o = oracle.Run.from_case(other)
    o.step(8)
    dr, du = max_err(runs[0], o, case.nlevels, run=1)
    assert dr <= TOL32 and du <= TOL32, (dr, du)


def test_hrr_uniform_flow_stays_uniform(M):
    case = W.small_3d("D3Q27", nlevels=3).with_(
        collision="HRR", sigma=0.5, ic=dict(kind="uniform", u0=(0.1 * W.CS, 0.03, 0.0)))
    g = M.Lbm.from_case(case)
    g.step(10)
    for l in range(case.nlevels):
        r, u = g.macros(l)
        m = ~np.isnan(r)
        assert np.max(np.abs(r[m] - 1.0)) < 1e-6
        assert np.max(np.abs(u[0, m] - 0.1 * W.CS)) < 1e-6
        assert np.max(np.abs(u[1, m] - 0.03)) < 1e-6


def test_hrr_rejects_bad_sigma(M):
    with pytest.raises(M.LbmError):
        M.Lbm("D2Q9", "HRR", 0.6, (32, 32, 1), [], sigma=1.5)
