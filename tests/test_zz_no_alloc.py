"""lbm_diag_noalloc against lbm_diag.

lbm_diag_noalloc is the conservation diagnostic for callers that cannot let
the library allocate device memory (a serving loop held to a fixed memory
budget, device memory owned by another framework's pool, or code that cannot
take the synchronisation cudaFree implies).  It keeps its partial sums in one
fixed array inside the library instead of a temporary buffer.  This file is
collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2004_11863_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-6  # the binary32 parity tolerance of the other GPU tests


def same_sums(got, ref):
    """Both entry points add the same FP64 block partials in the same order
    (additions only, nothing to contract into an FMA), so the sums must agree
    bit for bit; the tolerance check only sharpens the failure message."""
    if not np.array_equal(got, ref):
        np.testing.assert_allclose(got, ref, rtol=0,
                                   atol=TOL * max(1.0, float(np.abs(ref).max())))
        np.testing.assert_array_equal(got, ref)


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
                                lambda: W.small_3d("D3Q27", "RR", nlevels=3)],
                         ids=["2d_two_levels", "3d_three_levels"])
def test_noalloc_matches_diag_twice(M, mk):
    case = mk()
    g = M.Lbm.from_case(case)
    g.step(3)
    ref_m, ref_p, ok = g.diag()
    assert ok
    for _ in range(2):  # two calls in a row share the same fixed array
        m, p, ok2 = g.diag_noalloc()
        assert ok2
        same_sums(m, ref_m)
        same_sums(p, ref_p)
    # after more steps the array holds the previous call's sums; a new call
    # must still agree with lbm_diag
    g.step(2)
    ref_m, ref_p, _ = g.diag()
    m, p, _ = g.diag_noalloc()
    same_sums(m, ref_m)
    same_sums(p, ref_p)
    g.close()


def test_noalloc_rejects_levels_beyond_limit(M):
    """A level of 4097^2 > 2^24 nodes is refused before any device work."""
    g = M.Lbm("D2Q9", "BGK", 0.6, (4097, 4097, 1), [])
    with pytest.raises(ValueError, match="at most"):
        g.diag_noalloc()
    mass = np.zeros(1)
    mom = np.zeros(3)
    rc = M.lib().lbm_diag_noalloc(g._h, 0, mass.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  mom.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    assert rc == -1
    g.close()
