"""A level whose run exceeds 2^31 elements.

The two-node update addresses a run with 32-bit element offsets, so the
launcher gives larger runs to the one-node update.  This runs a periodic
D3Q19 level of 488^3 nodes (19 planes of 122 M elements: 9.3 GB in binary32)
whose initial field repeats with period 8 along every axis: a periodic
lattice is translation invariant, so after a few steps every node must
equal the node of a periodic 8^3 lattice (updated by the two-node update)
at its coordinates modulo 8, up to the last-bit differences between the
two updates' arithmetic.
"""
import math

import numpy as np
import pytest

from paper_2004_11863_gb300 import workloads as W

pytestmark = pytest.mark.gpu

P, N, STEPS = 8, 488, 3


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2004_11863_gb300 import build
    build.build()
    from paper_2004_11863_gb300 import mlbm
    return mlbm


def _pattern():
    z, y, x = np.meshgrid(*(np.arange(P),) * 3, indexing="ij")
    k = 2 * math.pi / P
    rho = 1.0 + 1e-3 * np.sin(k * x) * np.cos(k * y + 0.3) + 5e-4 * np.sin(k * z)
    u = np.stack([0.03 * W.CS + 0.01 * np.sin(k * y), 0.01 * np.cos(k * z + k * x),
                  0.005 * np.sin(k * x - k * y)])
    return rho, u


def test_large_run_matches_the_periodic_cell(M):
    import torch
    need = M.lbm_bytes("D3Q19", "RR", 0.52, (N, N, N), [])
    if torch.cuda.mem_get_info()[0] < need + (4 << 30):
        pytest.skip("not enough free device memory for the 488^3 level")
    rho, u = _pattern()
    small = M.Lbm("D3Q19", "RR", 0.52, (P, P, P), [])
    small.init(0, 0, rho.ravel(), u.reshape(3, -1))
    reps = (N // P,) * 3
    big = M.Lbm("D3Q19", "RR", 0.52, (N, N, N), [])
    big.init(0, 0, np.tile(rho, reps).ravel(), np.stack([np.tile(c, reps) for c in u]).reshape(3, -1))
    small.step(STEPS)
    big.step(STEPS)
    rs, us = small.macros(0)
    rb, ub = big.macros(0)
    big.close()
    small.close()
    rs, us = rs.reshape(P, P, P), us.reshape(3, P, P, P)
    rb, ub = rb.reshape(N, N, N), ub.reshape(3, N, N, N)
    idx = np.arange(N) % P
    want_r = rs[np.ix_(idx, idx, idx)]
    assert np.max(np.abs(rb - want_r)) <= 1e-6
    for a in range(3):
        assert np.max(np.abs(ub[a] - us[a][np.ix_(idx, idx, idx)])) <= 1e-6
    # the field moved (the check is not on a state at rest)
    assert np.max(np.abs(rs - rho)) > 1e-6
