"""Continuous-batching server: results are identical alone and in the mix
(and with either device allocator), the memory budget holds, and a served
run matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2004_11863_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2004_11863_gb300 import build
    build.build()
    from paper_2004_11863_gb300 import serve
    return serve


def _reqs(n=10, seed=7):
    return W.serving_requests(n, rate=200.0, seed=seed, step_scale=0.05, size_scale=0.35)


def test_results_same_alone_and_in_the_mix(S):
    reqs = _reqs()
    mixed = S.Server(hbm_budget=8e9, max_active=8, streams=4, chunk=7).run(reqs)
    assert mixed["max_concurrent"] > 1
    for r in reqs:
        # alone, and with device memory from cudaMalloc instead of the
        # caching allocator: the same bits
        alone = S.Server(max_active=1, streams=1, chunk=7, torch_allocator=False).run(
            [W.Request(r.rid, 0.0, r.case)])
        a = alone["results"][0]
        m = [x for x in mixed["results"] if x.rid == r.rid][0]
        assert np.array_equal(a.probes, m.probes), r.rid
        assert np.array_equal(a.mass, m.mass), r.rid


def test_memory_budget_respected(S):
    reqs = _reqs(12, seed=11)
    srv = S.Server(max_active=16, streams=4, chunk=5)
    biggest = max(srv.bytes_of(r.case) for r in reqs)
    srv.budget = 1.5 * biggest
    out = srv.run(reqs)
    assert len(out["results"]) == len(reqs)
    assert out["peak_bytes"] <= srv.budget
    assert out["p50_s"] <= out["p99_s"]


def test_served_fp32_run_matches_oracle(S):
    case = W.small_2level_2d("RR", steps=20)
    srv = S.Server(max_active=2, streams=2, chunk=6, storage="fp32")
    out = srv.run([W.Request(0, 0.0, case)])
    o = oracle.Run.from_case(case)
    o.step(case.steps)
    rho, u = o.macros(case.nlevels - 1)
    n = o.dims(case.nlevels - 1)[0]
    for k, (i, j, z) in enumerate(S.probe_nodes(case)):
        idx = (z * n[1] + j) * n[0] + i
        got = out["results"][0].probes[k]
        assert abs(got[0] - rho[idx]) < 1e-6 and abs(got[1] - u[0, idx]) < 1e-6
