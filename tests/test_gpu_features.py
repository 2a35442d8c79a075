"""GPU tests of the device-side analytic initial state and of the FP64
spurious-noise diagnostic (through the C ABI)."""
import numpy as np
import pytest

import oracle
from paper_2004_11863_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2004_11863_gb300 import build
    build.build()
    from paper_2004_11863_gb300 import mlbm
    return mlbm


@pytest.mark.parametrize("mk", [lambda: W.small_2level_2d("RR"),
                                lambda: W.slab_small_3d("D3Q19"),
                                lambda: W.small_3d("D3Q27", nlevels=3),
                                lambda: W.vortex_2level_d2q9()],
                         ids=["2d_vortex", "3d_slab_vortex", "3d_nested_pulse", "vortex2d"])
def test_analytic_init_matches_host_fields(M, mk):
    """lbm_init_analytic evaluates the same initial fields as the host-side
    input generator (to FP64 round-off of exp), on every level."""
    case = mk()
    a = M.Lbm.from_case(case)
    b = M.Lbm.from_case(case, init=False)
    b.init_analytic(case.ic)
    for l in range(case.nlevels):
        ra, ua = a.macros(l)
        rb, ub = b.macros(l)
        m = ~np.isnan(ra)
        assert np.max(np.abs(ra[m] - rb[m])) < 1e-9
        assert np.max(np.abs(ua[:, m] - ub[:, m])) < 1e-9
    a.step(3)
    b.step(3)
    for l in range(case.nlevels):
        ra, _ = a.macros(l)
        rb, _ = b.macros(l)
        m = ~np.isnan(ra)
        assert np.max(np.abs(ra[m] - rb[m])) < 1e-9


def _noise_numpy(case, rho_ref, rho_single, margin):
    """max / rms of |rho_ref - rho_single| over level-0 nodes outside the
    level-1 box grown by `margin` (periodic distances)."""
    lay = W.level_layout(case)
    n0 = lay[0]["n"]
    (lo, hi) = case.boxes[0]
    X = np.indices((n0[2], n0[1], n0[0]))[::-1].reshape(3, -1)
    near = np.ones(X.shape[1], bool)
    for a in range(case.dim):
        if not lay[1]["boxed"][a]:
            continue
        rel = np.mod(X[a] - lo[a], n0[a])
        E = hi[a] - lo[a]
        near &= (rel <= E + margin) | (rel >= n0[a] - margin)
    d = np.abs(rho_ref - rho_single)[~near]
    return d.max(), np.sqrt(np.mean(d * d)), d.size


def test_noise_diagnostic_against_host_and_oracle(M):
    case = W.Case("pulse2dn", "D2Q9", "RR", 0.5 + 1e-3, (96, 80, 1), [((32, 24, 0), (64, 56, 1))],
                  dict(kind="pulse", center=(48.0, 40.0, 0.0), radius=4.0, amplitude=1e-3), 30)
    single = case.with_(boxes=[])
    g2 = M.Lbm.from_case(case)
    g1 = M.Lbm.from_case(single)
    g2.step(case.steps)
    g1.step(case.steps)
    mx, rms, n = g2.noise(g1, margin=4)
    r2, _ = g2.macros(0)
    r1, _ = g1.macros(0)
    hm, hr, hn = _noise_numpy(case, r2, r1, 4)
    assert n == hn and abs(mx - hm) < 1e-11 and abs(rms - hr) < 1e-11
    assert mx > 0 and np.isfinite(mx)
    # the same quantity from two FP64 oracle runs
    o2 = oracle.Run.from_case(case)
    o1 = oracle.Run.from_case(single)
    o2.step(case.steps)
    o1.step(case.steps)
    om, orr, _ = _noise_numpy(case, o2.macros(0)[0], o1.macros(0)[0], 4)
    assert abs(mx - om) < 2e-6 and abs(rms - orr) < 2e-6, (mx, om, rms, orr)


def test_noise_zero_for_uniform_flow(M):
    case = W.small_2level_2d("RR").with_(ic=dict(kind="uniform", u0=(0.05, 0.0, 0.0)))
    g2 = M.Lbm.from_case(case)
    g1 = M.Lbm.from_case(case.with_(boxes=[]))
    g2.step(10)
    g1.step(10)
    mx, rms, n = g2.noise(g1, margin=2)
    assert n > 0 and mx < 1e-6
