"""The launch-shape autotuner: every candidate block shape gives bitwise the
same results (the shape only groups nodes into blocks), and the autotuner
leaves the run untouched and picks a valid shape."""
import numpy as np
import pytest

from paper_2004_11863_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(32, 4), (32, 2), (32, 1), (64, 2), (64, 1), (128, 1), (32, 3)]


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2004_11863_gb300 import build
    build.build()
    from paper_2004_11863_gb300 import mlbm
    return mlbm


def _fields(g, nlev):
    return [g.macros(l) for l in range(nlev)]


@pytest.mark.parametrize("mk", [lambda: W.small_2level_2d("RR"),
                                lambda: W.small_3d("D3Q27", nlevels=3),
                                lambda: W.pulse_2level_d2q9("BGK", steps=5)],
                         ids=["2d", "3d_3lev", "pulse2d_bgk"])
def test_every_shape_is_bitwise_identical(M, mk):
    case = mk()
    ref = M.Lbm.from_case(case)
    ref.step(6)
    want = _fields(ref, case.nlevels)
    for bx, by in SHAPES[1:]:
        g = M.Lbm.from_case(case)
        for l in range(case.nlevels):
            g.set_block_shape(l, bx, by)
        g.step(6)
        for (ra, ua), (rb, ub) in zip(want, _fields(g, case.nlevels)):
            assert np.array_equal(ra, rb, equal_nan=True) and np.array_equal(ua, ub, equal_nan=True)
        g.close()


def test_autotune_keeps_the_run_and_picks_a_candidate(M):
    case = W.small_2level_2d("RR")
    a = M.Lbm.from_case(case)
    b = M.Lbm.from_case(case)
    a.step(3)
    b.step(3)
    shapes = a.autotune(reps=3)
    assert all(tuple(s) in SHAPES for s in shapes)
    a.step(5)
    b.step(5)
    for (ra, ua), (rb, ub) in zip(_fields(a, 2), _fields(b, 2)):
        assert np.array_equal(ra, rb, equal_nan=True) and np.array_equal(ua, ub, equal_nan=True)


def test_bad_shapes_rejected(M):
    g = M.Lbm.from_case(W.small_2level_2d("RR"))
    for bx, by in ((16, 4), (32, 8), (48, 2), (32, 0)):
        with pytest.raises(M.LbmError):
            g.set_block_shape(0, bx, by)


LAYOUTS = [("slab3d_d3q19", lambda: W.slab_small_3d("D3Q19", "RR", steps=7)),
           ("box3d_d3q27_3lev", lambda: W.small_3d("D3Q27", "RR", nlevels=3, steps=7)),
           ("box3d_d3q19_bgk", lambda: W.small_3d("D3Q19", "BGK", nlevels=2, steps=7)),
           ("box2d", lambda: W.small_2level_2d("RR", steps=7))]


@pytest.mark.parametrize("storage,batch", [("fp32", 1), ("fp32", 3), ("fp16", 1), ("fp16", 3)])
@pytest.mark.parametrize("name,mk", LAYOUTS, ids=[n for n, _ in LAYOUTS])
def test_face_buffer_bitwise(M, name, mk, storage, batch):
    """The x-face buffer (on / off) changes where the rebuilt face nodes of
    3D levels are kept, never a node's arithmetic: the same bits on every
    level, for single runs, batches and binary16 run pairs."""
    case = mk()
    want = None
    for xf in (True, False):
        g = M.Lbm.from_case(case, storage=storage, batch=batch)
        g.set_face_buffer(xf)
        for l in range(case.nlevels):
            g.set_block_shape(l, 32, 2)
        g.step(case.steps)
        got = [g.macros(l, r) for l in range(case.nlevels) for r in range(batch)]
        g.close()
        if want is None:
            want = got
            continue
        for (ra, ua), (rb, ub) in zip(want, got):
            assert np.array_equal(ra, rb, equal_nan=True) and np.array_equal(ua, ub, equal_nan=True)
