"""GPU parity: the CUDA library against the FP64 oracle, element by element
on the same seeded inputs (through the C ABI).

Tolerance: max |drho| and max |du| <= 1e-6 in lattice units for binary32
storage; the binary16 (shifted) storage is held to the bound stated in the
test.  Sizes span several 32-wide tiles with ragged tails on every level.
"""
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


def compare(gpu, orc, nlev, run=0, tol=TOL32):
    worst = (0.0, 0.0)
    for l in range(nlev):
        rg, ug = gpu.macros(l, run)
        ro, uo = orc.macros(l)
        mo = np.isnan(ro)
        assert np.array_equal(np.isnan(rg), mo), f"inactive sets differ on level {l}"
        m = ~mo
        dr = np.max(np.abs(rg[m] - ro[m]))
        du = np.max(np.abs(ug[:, m] - uo[:, m]))
        assert dr <= tol and du <= tol, (l, dr, du)
        worst = (max(worst[0], dr), max(worst[1], du))
    return worst


CASES_2D = [
    ("small2d_rr", lambda: W.small_2level_2d("RR", steps=30)),
    ("small2d_bgk", lambda: W.small_2level_2d("BGK", steps=30)),
    ("small2d_reg", lambda: W.small_2level_2d("REG", steps=30)),
    ("vortex2d_40", lambda: W.vortex_2level_d2q9(steps=40)),
    ("pulse2d_small", lambda: W.Case("pulse2ds", "D2Q9", "BGK", 0.5 + 1e-3, (80, 72, 1),
                                     [((20, 18, 0), (60, 54, 1))],
                                     dict(kind="pulse", center=(12.0, 36.0, 0.0), radius=4.0,
                                          amplitude=1e-3), 40)),
    # a fine band spanning the periodic x axis: the interface faces are
    # normal to y and their tiles wrap around x
    ("band2d", lambda: W.Case("band2d", "D2Q9", "RR", 0.52, (70, 48, 1),
                              [((0, 12, 0), (70, 36, 1))],
                              dict(kind="vortex", u0=(0.0, 0.1 * W.CS, 0.0),
                                   center=(66.0, 16.0, 0.0), radius=4.0, eps=0.05 * W.CS), 30)),
]


@pytest.mark.parametrize("name,mk", CASES_2D, ids=[c[0] for c in CASES_2D])
def test_parity_2d(M, name, mk):
    case = mk()
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(case.steps)
    o.step(case.steps)
    compare(g, o, case.nlevels)


CASES_3D = [
    ("d3q19_single", lambda: W.small_3d("D3Q19", "RR", nlevels=1, steps=6)),
    ("d3q19_2lev_rr", lambda: W.small_3d("D3Q19", "RR", nlevels=2, steps=5)),
    ("d3q19_2lev_bgk", lambda: W.small_3d("D3Q19", "BGK", nlevels=2, steps=5)),
    ("d3q27_2lev_reg", lambda: W.small_3d("D3Q27", "REG", nlevels=2, steps=4)),
    ("d3q27_3lev_rr", lambda: W.small_3d("D3Q27", "RR", nlevels=3, steps=3)),
    ("d3q19_slab", lambda: W.slab_small_3d("D3Q19", "RR", steps=5)),
    # a fine tube along the periodic x axis: faces normal to y and z, tiles
    # wrapping around x, 29 TN nodes per face row (two ragged tiles)
    ("d3q27_tube", lambda: W.Case("tube3d", "D3Q27", "RR", 0.52, (29, 16, 17),
                                  [((0, 4, 4), (29, 12, 13))],
                                  dict(kind="pulse", center=(27.0, 6.0, 8.0), radius=3.0,
                                       amplitude=1e-3, u0=(0.05, 0.0, 0.0)), 4)),
]


@pytest.mark.parametrize("name,mk", CASES_3D, ids=[c[0] for c in CASES_3D])
def test_parity_3d(M, name, mk):
    case = mk()
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(case.steps)
    o.step(case.steps)
    compare(g, o, case.nlevels)


@pytest.mark.parametrize("u_ref", [(0.0, 0.0, 0.0), (0.1 * W.CS, 0.0, 0.0), (0.03, -0.02, 0.0)])
def test_reference_shift_does_not_change_results(M, u_ref):
    """The stored shift f - f0(rho0, U) is a storage choice: any reference
    velocity gives the oracle's result within the binary32 tolerance."""
    case = W.vortex_2level_d2q9(steps=60)
    g = M.Lbm.from_case(case, u_ref=u_ref)
    o = oracle.Run.from_case(case)
    g.step(case.steps)
    o.step(case.steps)
    compare(g, o, 2)


def test_populations_are_rest_shifted(M):
    """lbm_populations returns f - w rho0 whatever the reference velocity;
    matched to the oracle's populations direction by direction."""
    case = W.small_3d("D3Q19", "RR", nlevels=2, steps=3)
    g = M.Lbm.from_case(case, u_ref=(0.04, 0.01, -0.02))
    o = oracle.Run.from_case(case)
    g.step(3)
    o.step(3)
    xg, _ = M.lbm_lattice("D3Q19")
    xo, wo = oracle.lattice("D3Q19")
    order = [int(np.nonzero((xo == v).all(1))[0][0]) for v in xg]
    for l in range(2):
        pg = g.populations(l)
        po = o.populations(l) - wo[:, None] * case.rho0
        m = ~np.isnan(o.macros(l)[0])
        np.testing.assert_allclose(pg[:, m], po[order][:, m], rtol=0, atol=1e-6)


def test_three_level_2d(M):
    case = W.Case("nest2d", "D2Q9", "RR", 0.51, (64, 64, 1),
                  [((16, 16, 0), (48, 48, 1)), ((16, 16, 0), (48, 48, 1))],
                  dict(kind="pulse", center=(30.0, 34.0, 0.0), radius=3.0, amplitude=1e-3,
                       u0=(0.05 * W.CS, 0.0, 0.0)), 12)
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(case.steps)
    o.step(case.steps)
    compare(g, o, 3)


FOUR_LEVELS = W.Case("nest4", "D2Q9", "RR", 0.51, (40, 40, 1),
                     [((10, 10, 0), (30, 30, 1))] * 3,
                     dict(kind="pulse", center=(19.0, 21.0, 0.0), radius=3.0, amplitude=1e-3,
                          u0=(0.05 * W.CS, 0.0, 0.0)), 6)


def test_four_levels_2d(M):
    """The deepest nesting the library allows (four levels, 8 finest
    sub-steps per coarse step)."""
    case = FOUR_LEVELS
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(case.steps)
    o.step(case.steps)
    compare(g, o, 4)


def test_odd_and_even_step_counts(M):
    """AA parity: 1, 2 and 3 coarse steps all match (each level ends on
    either parity)."""
    case = W.small_2level_2d("RR")
    for n in (1, 2, 3):
        g = M.Lbm.from_case(case)
        o = oracle.Run.from_case(case)
        g.step(n)
        o.step(n)
        compare(g, o, 2)


def test_graphs_bitwise_equal_eager(M):
    case = W.small_3d("D3Q27", "RR", nlevels=3, steps=4)
    a = M.Lbm.from_case(case)
    b = M.Lbm.from_case(case)
    b.set_graphs(False)
    a.step(4)
    b.step(4)
    for l in range(3):
        ra, ua = a.macros(l)
        rb, ub = b.macros(l)
        assert np.array_equal(ra, rb, equal_nan=True) and np.array_equal(ua, ub, equal_nan=True)


def test_batch_runs_independent(M):
    """Runs of a batch evolve independently: each equals the same run alone,
    bit for bit."""
    c1 = W.small_2level_2d("RR")
    c2 = c1.with_(ic=dict(kind="pulse", center=(50.0, 20.0, 0.0), radius=3.0, amplitude=2e-3))
    g = M.Lbm(c1.lattice, c1.collision, c1.tau0, c1.dims, c1.boxes, batch=2, u_ref=c1.u_ref)
    for l in range(2):
        g.init(l, 0, *W.initial_fields(c1, l))
        g.init(l, 1, *W.initial_fields(c2, l))
    g.step(7)
    for run, c in ((0, c1), (1, c2)):
        s = M.Lbm.from_case(c, u_ref=c1.u_ref)
        s.step(7)
        for l in range(2):
            r1, u1 = g.macros(l, run)
            r2, u2 = s.macros(l)
            assert np.array_equal(r1, r2, equal_nan=True) and np.array_equal(u1, u2, equal_nan=True)


def fp16_bound(case, o_initial):
    """Stated error bound of binary16 shifted storage: every stored
    population is rounded to nearest, at most half an ulp of the largest
    stored magnitude gmax (2^-11 gmax relative spacing), once per update of
    the finest level; the roundings are unbiased, so they accumulate like a
    random walk over the n = 2^(L-1) * steps finest updates.  rho and u sum
    q such roundings (weights <= 1): bound = 2 * q^(1/2) * 2^-11 * gmax *
    n^(1/2), with a factor 2 of margin."""
    _, w = oracle.lattice(case.lattice)
    gmax = 0.0
    for l in range(case.nlevels):
        f = o_initial.populations(l)
        gmax = max(gmax, float(np.max(np.abs(f - w[:, None] * case.rho0))))
    n = case.steps * 2 ** (case.nlevels - 1)
    return 2.0 * np.sqrt(case.q) * 2.0 ** -11 * gmax * np.sqrt(n)


@pytest.mark.parametrize("mk", [lambda: W.small_2level_2d("RR", steps=30),
                                lambda: W.small_3d("D3Q19", "RR", nlevels=2, steps=5)])
def test_fp16_shifted_storage_bound(M, mk):
    """binary16 storage of g = f - w rho0 with binary32 arithmetic stays
    within the stated bound of the FP64 oracle."""
    case = mk()
    g = M.Lbm.from_case(case, storage="fp16")
    o = oracle.Run.from_case(case)
    tol = fp16_bound(case, o)
    g.step(case.steps)
    o.step(case.steps)
    compare(g, o, case.nlevels, tol=tol)


def test_rest_state_exact(M):
    """A uniform state stays uniform to binary32 round-off on every level."""
    case = W.small_3d("D3Q19", "RR", nlevels=2).with_(
        ic=dict(kind="uniform", u0=(0.05, 0.02, 0.01)))
    g = M.Lbm.from_case(case)
    g.step(10)
    for l in range(2):
        r, u = g.macros(l)
        m = ~np.isnan(r)
        assert np.max(np.abs(r[m] - 1)) < 1e-6
        assert np.max(np.abs(u[0, m] - 0.05)) < 1e-6


def test_diag_mass_conservation_single_level(M):
    """FP64 mass and momentum sums are conserved by a periodic single level
    (collision conserves both, streaming permutes)."""
    case = W.small_3d("D3Q27", "RR", nlevels=1)
    g = M.Lbm.from_case(case)
    m0, p0, ok0 = g.diag()
    g.step(20)
    m1, p1, ok1 = g.diag()
    assert ok0 and ok1
    assert abs(m1[0] - m0[0]) < 1e-5 * max(1.0, abs(m0[0]))
    assert np.max(np.abs(p1[0] - p0[0])) < 1e-4


def test_probe_records_every_coarse_step(M):
    case = W.small_2level_2d("RR", steps=9)
    g = M.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.probe_add(1, [[10, 12, 0], [40, 30, 0]])
    g.step(9)
    rec = g.probe()
    assert rec.shape == (9, 1, 2, 4)
    o.step(9)
    rho, u = o.macros(1)
    n = o.dims(1)[0]
    for k, (i, j) in enumerate([(10, 12), (40, 30)]):
        idx = j * n[0] + i
        assert abs(rec[-1, 0, k, 0] - rho[idx]) < TOL32
        assert abs(rec[-1, 0, k, 1] - u[0, idx]) < TOL32


def test_probe_async_matches_probe(M):
    """The asynchronous read-out, enqueued after every step into pinned
    memory and waited for once, returns the same samples, bit for bit, as
    the synchronous read-out after every step; a read-out of the newest few
    of several recorded steps agrees too."""
    import torch
    case = W.small_3d("D3Q19", "RR", nlevels=2, steps=12)
    a = M.Lbm.from_case(case, batch=2)
    b = M.Lbm.from_case(case, batch=2)
    nodes = [[3, 4, 5], [10, 9, 8], [20, 15, 11]]
    a.probe_add(1, nodes)
    b.probe_add(1, nodes)
    rec = torch.zeros((case.steps, 2, 3, 4), dtype=torch.float64).pin_memory().numpy()
    sync = []
    for k in range(case.steps):
        a.step(1)
        sync.append(a.probe(max_steps=1)[0])
        b.step(1)
        assert b.probe_async(rec[k:k + 1]) == 1
    b.sync()
    assert np.array_equal(np.stack(sync), rec)
    # several steps per read-out, fewer than recorded: the newest ones
    a.step(5)
    b.step(5)
    many = a.probe(max_steps=3)
    out = np.zeros((3, 2, 3, 4))
    assert b.probe_async(out) == 3
    b.sync()
    assert np.array_equal(many, out)
    assert b.probe_async(out) == 0


def test_macros_into_caller_buffers(M):
    """lbm_macros into caller-owned (pinned) arrays returns the same bits
    as into fresh arrays; wrong shapes are refused before any copy."""
    import torch
    case = W.small_3d("D3Q27", "RR", nlevels=2, steps=3)
    g = M.Lbm.from_case(case, batch=2)
    g.step(3)
    for l in range(2):
        N = g.nodes(l)
        out = (torch.empty(N, dtype=torch.float64).pin_memory().numpy(),
               torch.empty((3, N), dtype=torch.float64).pin_memory().numpy())
        for run in range(2):
            r0, u0 = g.macros(l, run)
            r1, u1 = g.macros(l, run, out=out)
            assert r1 is out[0] and u1 is out[1]
            assert np.array_equal(r0, r1, equal_nan=True) and np.array_equal(u0, u1, equal_nan=True)
    with pytest.raises(ValueError):
        g.macros(0, 0, out=(np.empty(3), np.empty((3, 3))))


def test_readout_moments_match_fp64_sums(M):
    """lbm_macros forms each node's moments from its binary32 populations by
    compensated binary32 summation (TwoSum errors carried alongside, added
    in FP64).  Against FP64 sums of the same stored values -- lbm_populations
    returns them exactly when the reference is at rest -- rho - rho0 and
    rho u agree within 1e-13 on every active node of every level (the
    summation's bound is below 1e-12 of sum |g_i|, here below 0.1), in 2D
    and 3D, binary32 and binary16 storage, after a few steps of flow."""
    for case, st in ((W.small_2level_2d(steps=7), "fp32"), (W.small_3d("D3Q27", steps=3), "fp32"),
                     (W.small_3d("D3Q19", steps=3), "fp16")):
        g = M.Lbm.from_case(case, storage=st, u_ref=(0.0, 0.0, 0.0))
        g.step(case.steps)
        xi, _ = M.lbm_lattice(case.lattice)
        for l in range(case.nlevels):
            rho, u = g.macros(l)
            f = g.populations(l)
            act = ~np.isnan(rho)
            drho = f.sum(axis=0)
            j = xi.T.astype(np.float64) @ f
            assert np.max(np.abs(f[:, act]).sum(axis=0)) < 0.1
            assert np.max(np.abs((rho[act] - case.rho0) - drho[act])) <= 1e-13, (case.name, l)
            assert np.max(np.abs(rho[act] * u[:, act] - j[:, act])) <= 1e-13, (case.name, l)
        g.close()


def test_reflected_acoustic_wave_matches_oracle(M):
    """The GPU reproduces the oracle's reflected-wave ratio of the convected
    1D acoustic wave (Sec. 9.2) and its fields within 1e-6."""
    from tests.test_oracle_pins import e5_case, e5_fields, e5_ratio
    case = e5_case("RR")
    g = M.Lbm(case.lattice, case.collision, case.tau0, case.dims, case.boxes, u_ref=case.u_ref)
    o = oracle.Run(case.lattice, case.collision, case.tau0, case.dims, case.boxes)
    for l in range(2):
        g.init(l, 0, *e5_fields(case, l))
        o.init_level(l, *e5_fields(case, l))
    o.init_done()
    g.step(case.steps)
    o.step(case.steps)
    compare(g, o, 2)
    gi, _, gr, _ = e5_ratio(g.macros(0)[0], g.macros(1)[0], case)
    oi, _, orf, _ = e5_ratio(o.macros(0)[0], o.macros(1)[0], case)
    assert abs(gr / gi - orf / oi) < 0.02 * (orf / oi)
