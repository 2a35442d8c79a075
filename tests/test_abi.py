"""CPU-side checks of the C ABI: the library loads, exports every function
include/mlbm.h declares, and its host-only logic (lattice tables, layout
validation, error strings) behaves.  No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2004_11863_gb300 import build as B
from paper_2004_11863_gb300 import mlbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mlbm.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "mlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
def test_lattice_tables_match_definition(lib, lat):
    """Same velocity set and weights as the lattice definitions (the
    library's own order; compared as sets)."""
    xi, w = mlbm.lbm_lattice(lat)
    oxi, ow = oracle.lattice(lat)
    assert len(w) == len(ow)
    a = sorted((tuple(v), round(x, 15)) for v, x in zip(xi.tolist(), w))
    b = sorted((tuple(v), round(x, 15)) for v, x in zip(oxi.tolist(), ow))
    assert a == b
    if lat == "D2Q9":  # order of eq. xi_i
        assert xi[:, 0].tolist() == [0, 1, 0, -1, 0, 1, -1, -1, 1]


@pytest.mark.parametrize("bad", [
    dict(tau0=0.5),
    dict(tau0=0.4),
    dict(dims=(2, 64, 1)),
    dict(boxes=[((24, 16, 0), (26, 48, 1))]),       # extent < 4
    dict(boxes=[((90, 16, 0), (100, 48, 1))]),      # crosses the periodic seam
    dict(boxes=[((0, 0, 0), (96, 64, 1))]),         # not bounded on any axis
    dict(boxes=[((24, 16, 0), (72, 48, 1)), ((2, 2, 0), (20, 20, 1))]),  # margin < 4
    dict(batch=0),
])
def test_layout_validation_rejects(lib, bad):
    kw = dict(lattice="D2Q9", collision="RR", tau0=0.52, dims=(96, 64, 1),
              boxes=[((24, 16, 0), (72, 48, 1))], batch=1)
    kw.update(bad)
    cfg = mlbm.make_config(kw["lattice"], kw["collision"], kw["tau0"], kw["dims"], kw["boxes"],
                           batch=kw["batch"])
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(cfg), None, None, ctypes.byref(h))
    assert rc == -1 and not h.value


def test_strerror(lib):
    for c in (0, -1, -2, -4, -5, 7):
        assert isinstance(lib.lbm_strerror(c), bytes)
    assert b"invalid" in lib.lbm_strerror(-1)


def test_null_arguments(lib):
    assert lib.lbm_create(None, None, None, None) == -1
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_kernel_launches(None) == -1
    assert lib.lbm_sensors_enable(None, 0, 0.0, 0.0) == -1
    assert lib.lbm_autotune(None, 1, None) == -1
    assert lib.lbm_set_block_shape(None, 0, 32, 4) == -1
    assert lib.lbm_sensors(None, 0, 0, None, None, None, None) == -1
    assert lib.lbm_probe_async(None, None, 0, None) == -1
    assert lib.lbm_set_fused(None, 1) == -1
    lib.lbm_destroy(None)
