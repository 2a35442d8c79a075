"""Binary16 storage with the runs of a batch interleaved in pairs (one 4-byte
access moves a node's population of two runs): every run of a batch must
equal the same run stepped alone (single-run layout, one run per launch), on
every kernel of the step — level updates, interface transfers, read-outs —
for odd and even batches, rest and moving reference states, and H-RR."""
import numpy as np
import pytest

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


def _other(case):
    c = [0.5 * n for n in case.dims]
    return case.with_(ic=dict(kind="pulse", center=(c[0] + 3.0, c[1] - 2.0, c[2]), radius=3.0,
                              amplitude=1e-3))


CASES = {
    "2d_rr": lambda: W.small_2level_2d("RR"),
    "2d_bgk_moving": lambda: W.small_2level_2d("BGK"),   # vortex on a 0.1 cs flow
    "3d_d3q19": lambda: W.small_3d("D3Q19", nlevels=2),
    "3d_d3q27_3lev": lambda: W.small_3d("D3Q27", nlevels=3),
    "2d_hrr": lambda: W.small_2level_2d("RR").with_(collision="HRR", sigma=0.5),
}


@pytest.mark.parametrize("batch", [2, 3])
@pytest.mark.parametrize("key", list(CASES))
def test_paired_batch_equals_single_runs(M, key, batch):
    case = CASES[key]()
    ics = [case, _other(case), case][:batch]
    g = M.Lbm.from_case(case, storage="fp16", batch=batch, init=False)
    for b, c in enumerate(ics):
        for l in range(case.nlevels):
            g.init(l, b, *W.initial_fields(c, l))
    g.step(5)
    for b, c in enumerate(ics):
        s = M.Lbm.from_case(c, storage="fp16", u_ref=case.u_ref)
        s.step(5)
        for l in range(case.nlevels):
            ra, ua = g.macros(l, b)
            rb, ub = s.macros(l)
            assert np.array_equal(ra, rb, equal_nan=True), (b, l, np.nanmax(np.abs(ra - rb)))
            assert np.array_equal(ua, ub, equal_nan=True), (b, l, np.nanmax(np.abs(ua - ub)))
        s.close()
