"""GPU non-hydrodynamic mode sensors (Sec. 7) against the FP64 oracle.

The sensors are decisions on continuous quantities (div u and curl u of two
consecutive iterations, |f1G|), which the GPU forms in binary32 and the
oracle in binary64.  The quantities are compared element by element; the
flags are compared exactly wherever no quantity lies within the value
tolerance of its threshold (elsewhere either flag is valid).  On level 0 the
previous iteration is the previous coarse step, so every decision is
checked; on a refined level the previous iteration is the first sub-step,
which the API does not expose, so its flags must agree at 99% of the nodes
and its values everywhere."""
import numpy as np
import pytest

import oracle
from paper_2004_11863_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TV = 1e-7    # div / curl tolerance (binary32 velocities agree to ~1e-8)
TG = 1e-7    # |f1G| tolerance
EPS = 5e-7   # magnitude floor of the sign tests
GTHR = 1e-6  # spuriousG threshold


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2004_11863_gb300 import build
    build.build()
    from paper_2004_11863_gb300 import mlbm
    return mlbm


CASES = {
    "2d_rr": lambda: W.small_2level_2d("RR"),
    "2d_bgk": lambda: W.small_2level_2d("BGK"),
    "2d_hrr": lambda: W.small_2level_2d("RR").with_(collision="HRR", sigma=0.5),
    "3d_rr": lambda: W.small_3d("D3Q19", nlevels=2),
}


def _curl_vec(cu, dim):
    return cu if dim == 3 else cu[2:3]


def _decisions_clear(prev, cur, gn, dim):
    """Nodes where no sensor decision depends on a quantity within tolerance
    of its threshold: a sign test is settled when either factor is clearly
    below the floor, or both clearly above it (and, for the vorticity dot
    product, clearly away from orthogonal)."""
    pd, pc = prev
    d, c = cur
    ac_clear = ((np.abs(pd) < EPS - TV) | (np.abs(d) < EPS - TV)
                | ((np.abs(pd) > EPS + TV) & (np.abs(d) > EPS + TV)))
    pn = np.linalg.norm(_curl_vec(pc, dim), axis=0)
    cn = np.linalg.norm(_curl_vec(c, dim), axis=0)
    dot = np.sum(_curl_vec(pc, dim) * _curl_vec(c, dim), axis=0)
    t = 2 * TV
    s_clear = ((pn < EPS - t) | (cn < EPS - t)
               | ((pn > EPS + t) & (cn > EPS + t) & (np.abs(dot) > t * (pn + cn))))
    return ac_clear & s_clear & (np.abs(gn - GTHR) > TG)


@pytest.mark.parametrize("key", list(CASES))
def test_sensor_parity(M, key):
    case = CASES[key]()
    steps = 12
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    for l in range(case.nlevels):
        g.sensors_enable(l, EPS, GTHR)
        o.sensors_enable(l, EPS, GTHR)
    g.step(steps - 1)
    o.step(steps - 1)
    prev0 = o.sensors(0)[1:3]
    g.step(1)
    o.step(1)
    fired = 0
    for l in range(case.nlevels):
        fg, dg, cg, ng = g.sensors(l, with_gnorm=True)
        fo, do, co, no = o.sensors(l, with_gnorm=True)
        mid = o.classes(l) == 1
        assert not fg[~mid].any()
        assert np.max(np.abs(dg - do)) <= TV, np.max(np.abs(dg - do))
        assert np.max(np.abs(cg - co)) <= TV, np.max(np.abs(cg - co))
        assert np.max(np.abs(ng - no)) <= TG, np.max(np.abs(ng - no))
        fired += int(np.count_nonzero(fo[mid]))
        if l == 0:
            clear = mid & _decisions_clear(prev0, (do, co), no, case.dim)
            assert clear.sum() > 0.7 * mid.sum()
            bad = np.nonzero(clear & (fg != fo))[0]
            assert bad.size == 0, (bad[:10], fg[bad[:10]], fo[bad[:10]])
        else:
            agree = np.mean(fg[mid] == fo[mid])
            assert agree >= 0.99, agree
    assert fired > 0  # the case exercises the sensors


def test_sensors_leave_the_solution_unchanged_and_graphs_match(M):
    """The sensor pass only reads populations: a run with sensors equals one
    without bit for bit; graph replay and eager launches give the same
    sensor output bit for bit."""
    case = W.small_2level_2d("RR")
    plain = M.Lbm.from_case(case)
    runs = []
    for graphs in (True, False):
        g = M.Lbm.from_case(case)
        g.set_graphs(graphs)
        for l in range(2):
            g.sensors_enable(l, EPS, GTHR)
        g.step(9)
        runs.append(g)
    plain.step(9)
    for l in range(2):
        rp, up = plain.macros(l)
        rs, us = runs[0].macros(l)
        assert np.array_equal(rp, rs, equal_nan=True) and np.array_equal(up, us, equal_nan=True)
        a = runs[0].sensors(l, with_gnorm=True)
        b = runs[1].sensors(l, with_gnorm=True)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_sensor_errors(M):
    g = M.Lbm.from_case(W.small_2level_2d("RR"))
    with pytest.raises(M.LbmError):
        g.sensors(0)  # not enabled
    with pytest.raises(M.LbmError):
        g.sensors_enable(0, -1.0, 0.0)
