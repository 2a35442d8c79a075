"""The paper's validation runs (Secs. 9, 10) on the GPU path: the outcomes the
paper reports, measured by paper_2004_11863_gb300.validation, and parity of
the full-length quasi-1D runs with the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2004_11863_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2004_11863_gb300 import build
    build.build()
    from paper_2004_11863_gb300 import validation
    return validation


def _at(run, t):
    return next(s for s in run["samples"] if s["t"] == t)


def test_e4_shear_wave(V):
    """Sec. 9.1 / 10.1: BGK and RR carry spuriousS modes (the S sensor fires
    on the fine level) and deform the wave at the fine-to-coarse crossing,
    BGK much more; H-RR (sigma = 0.995) has no spuriousS mode left from
    t = 840 on and crosses without deformation."""
    bgk, rr, hrr = V.e4("BGK"), V.e4("RR"), V.e4("HRR")
    assert _at(rr, 840)["sensors_per_level"][1][1] > 100
    assert 1e-4 < _at(rr, 2900)["deformation"] < 2e-3
    assert _at(bgk, 2900)["deformation"] > 5e-3
    for t in (840, 1280, 2900):
        assert all(c[1] == 0 for c in _at(hrr, t)["sensors_per_level"]), _at(hrr, t)
    assert _at(hrr, 2900)["deformation"] < 1e-6


def test_e5_acoustic_wave(V):
    """Sec. 9.2 / 10.2: a reflected wave of order 1/2000 of the incident one
    for both RR and H-RR; at t = 2620 the RR spuriousAc modes have become
    waves of 1/25 (upstream) and 1/100 (downstream, fine level) of the
    incident amplitude, and H-RR emits nothing."""
    rr, hrr = V.e5("RR"), V.e5("HRR")
    ratio = rr["t900"]["reflected_over_incident"]
    assert 1 / 6000 < ratio < 3 / 2000
    assert abs(hrr["t900"]["reflected_over_incident"] / ratio - 1) < 0.01
    assert 1 / 50 < rr["t2620"]["upstream_over_A"] < 1 / 12
    assert 1 / 200 < rr["t2620"]["downstream_fine_over_A"] < 1 / 50
    assert hrr["t2620"]["upstream_over_A"] < 1e-4
    assert hrr["t2620"]["downstream_fine_over_A"] < 1e-4


def test_e6_vortex_noise(V):
    """Sec. 10.3, Fig. psd_COVO: at nu = 1e-6 H-RR cuts the spurious noise at
    P1 by orders of magnitude; RR reaches the H-RR level only when its
    viscosity is raised to 4.18e-4 (eq. tauSpuriousAc, 418 nu); nu = 1e-4
    lies in between."""
    band = "0.01-0.1"
    rr = V.e6("RR")["band_power"][band]
    hrr = V.e6("HRR")["band_power"][band]
    rr4 = V.e6("RR", nu=1e-4)["band_power"][band]
    rr418 = V.e6("RR", nu=4.18e-4)["band_power"][band]
    assert hrr < rr / 1e3, (rr, hrr)
    assert hrr < rr4 < rr, (rr, rr4, hrr)
    assert abs(np.log10(rr418 / hrr)) < 0.5, (rr418, hrr)


@pytest.mark.parametrize("mk,steps", [(lambda: W.e4_shear_wave("RR"), 2900),
                                      (lambda: W.e4_shear_wave("HRR"), 2900),
                                      (lambda: W.e5_acoustic_wave("RR"), 2620)],
                         ids=["e4_rr", "e4_hrr", "e5_rr"])
def test_validation_runs_match_oracle(V, mk, steps):
    from paper_2004_11863_gb300 import mlbm
    case = mk()
    g = mlbm.Lbm.from_case(case)
    o = oracle.Run.from_case(case)
    g.step(steps)
    o.step(steps)
    for l in range(case.nlevels):
        rg, ug = g.macros(l)
        ro, uo = o.macros(l)
        m = ~np.isnan(ro)
        assert np.max(np.abs(rg[m] - ro[m])) <= 1e-6
        assert np.max(np.abs(ug[:, m] - uo[:, m])) <= 1e-6
