"""CPU emulation of the tiled interface kernels' index arithmetic (no GPU).

k_restrict_tile (face tiles of TN nodes, three lanes per footprint column)
and k_inject_sep (3D rebuild, stencil applied one axis at a time) map
threads to nodes through tile arithmetic; here that arithmetic is replayed
on the host for every test and benchmark layout and checked against the
plain per-node enumeration: every TN node restricted exactly once, every
footprint column formed exactly once, every shared-memory index and child
or parent coordinate in range, and every rebuilt node reading exactly the
parent taps and weights of eq. spaceInt, all inside the history ring.

The layout rules (levels, TN faces, boundary faces) mirror the host
scheduler's; the tile constants are read from kernels.cuh, so a change of
tile shape there is checked here too.
"""
import itertools
import os
import re
from collections import defaultdict

import pytest

from paper_2004_11863_gb300 import workloads as W

KERNELS = os.path.join(os.path.dirname(__file__), "..", "paper_2004_11863_gb300", "csrc",
                       "kernels.cuh")


def _src():
    with open(KERNELS) as fh:
        return fh.read()


def tile_constants():
    """(restriction TI 3D, TI 2D, TJ 3D, warps 3D, warps 2D, rebuild TI, TJ 3D)."""
    s = _src()
    ti3, ti2 = map(int, re.search(r"int TI = \(L::D == 3\) \? (\d+) : (\d+);", s).groups())
    tj3 = int(re.search(r"#define RST_TJ_3D (\d+)", s).group(1))
    assert "#define RST_NW_3D (2 * RST_TJ_3D + 1)" in s
    nw2 = int(re.search(r"int NW = \(L::D == 3\) \? RST_NW_3D : (\d+);", s).group(1))
    iti = int(re.search(r"struct InjTile \{\s+static constexpr int TI = (\d+);", s).group(1))
    itj = int(re.search(r"#define INJ_TJ_3D (\d+)", s).group(1))
    return ti3, ti2, tj3, 2 * tj3 + 1, nw2, iti, itj


def levels(case):
    """Per level: node counts, periodic and boxed axes, box (parent units)."""
    D = 3 if case.lattice.startswith("D3") else 2
    out = [dict(n=[case.dims[a] if a < D else 1 for a in range(3)], per=[1, 1, 1],
                boxed=[0, 0, 0], lo=[0] * 3, hi=[0] * 3)]
    for lo, hi in case.boxes:
        p = out[-1]
        v = dict(n=[0] * 3, per=[0] * 3, boxed=[0] * 3, lo=list(lo), hi=list(hi))
        for a in range(3):
            if a >= D:
                v["n"][a], v["per"][a] = 1, 1
                continue
            E = hi[a] - lo[a]
            if p["per"][a] and lo[a] == 0 and E == p["n"][a]:
                v["per"][a], v["n"][a] = 1, 2 * p["n"][a]
            else:
                v["boxed"][a], v["n"][a] = 1, 2 * E + 1
        out.append(v)
    return D, out


def tn_faces(D, p, c):
    """TN faces of child c (each TN node on its first face only)."""
    faces = []
    for a in range(D):
        if not c["boxed"][a]:
            continue
        for side in range(2):
            rlo, rext = [0] * 3, [0] * 3
            for b in range(3):
                E = c["hi"][b] - c["lo"][b]
                if b == a:
                    rlo[b], rext[b] = (E - 1 if side else 1), 1
                elif b >= D:
                    rlo[b], rext[b] = 0, 1
                elif not c["boxed"][b]:
                    rlo[b], rext[b] = 0, p["n"][b]
                elif b < a:
                    rlo[b], rext[b] = 2, E - 3
                else:
                    rlo[b], rext[b] = 1, E - 1
            faces.append((a, rlo, rext))
    return faces


def parent_of(c, p, r):
    return tuple((c["lo"][b] + r[b]) % p["n"][b] if c["boxed"][b] else r[b] for b in range(3))


def tangents(D, a):
    if D == 2:
        return 1 - a, 2
    return (1 if a == 0 else 0), (1 if a == 2 else 2)


def check_restriction(case, TI, TJ, NW):
    """Replays k_restrict_tile's block/lane mapping for every tile."""
    D, L = levels(case)
    FI, FJ = 2 * TI + 1, (2 * TJ + 1 if D == 3 else 1)
    NCH = (FI + 9) // 10
    NT, NN = 32 * NW, TI * TJ
    G = NT // NN
    assert G >= 1
    for l in range(1, len(L)):
        p, c = L[l - 1], L[l]
        faces = tn_faces(D, p, c)
        want = set()
        for a, rlo, rext in faces:
            for r in itertools.product(*[range(rlo[b], rlo[b] + rext[b]) for b in range(3)]):
                P = parent_of(c, p, r)
                assert P not in want
                want.add(P)
        got = set()
        for a, rlo, rext in faces:
            t1, t2 = tangents(D, a)
            nt1, nt2 = -(-rext[t1] // TI), -(-rext[t2] // TJ)
            for tile in range(nt1 * nt2):
                ti, tj = tile % nt1, tile // nt1
                r1, r2 = rlo[t1] + ti * TI, rlo[t2] + tj * TJ
                n1 = min(TI, rlo[t1] + rext[t1] - r1)
                n2 = min(TJ, rlo[t2] + rext[t2] - r2)
                assert n1 >= 1 and n2 >= 1
                seen = defaultdict(int)
                for w in range(NW):                      # stage 1: warp w, its chunks
                    for ch in range(w, FJ * NCH, NW):
                        for lane in range(32):
                            col = lane // 3
                            d = lane - 3 * col - 1
                            v, u = ch // NCH, (ch % NCH) * 10 + col
                            if not (col < 10 and u <= 2 * n1 and v <= (2 * n2 if D == 3 else 0)):
                                continue
                            assert 0 <= u < FI and 0 <= v < FJ
                            seen[(u, v, d)] += 1
                            x1 = 2 * r1 - 1 + u
                            x2 = 2 * r2 - 1 + v if D == 3 else 0
                            if c["per"][t1]:
                                x1 %= c["n"][t1]
                            if D == 3 and c["per"][t2]:
                                x2 %= c["n"][t2]
                            xa = 2 * rlo[a] + d
                            assert 0 <= x1 < c["n"][t1] and 0 <= x2 < c["n"][t2]
                            assert 0 <= xa < c["n"][a]
                            if (u & 1) and (D == 2 or (v & 1)):
                                assert (u - 1) >> 1 < TI
                                assert D == 2 or (v - 1) >> 1 < TJ
                need = {(u, v, d) for u in range(2 * n1 + 1)
                        for v in range(2 * n2 + 1 if D == 3 else 1) for d in (-1, 0, 1)}
                assert set(seen) == need and set(seen.values()) == {1}
                for tid in range(NT):                    # stage 3: rebuild threads
                    node, grp = tid % NN, tid // NN
                    i, j = node % TI, node // TI
                    if grp >= G or i >= n1 or j >= n2 or grp:
                        continue
                    # stage 2 and the H-RR neighbour reads stay in the footprint
                    assert 2 * i + 2 <= 2 * n1 and (D == 2 or 2 * j + 2 <= 2 * n2)
                    r = [0] * 3
                    r[a], r[t1], r[t2] = rlo[a], r1 + i, (r2 + j if D == 3 else 0)
                    P = parent_of(c, p, r)
                    assert all(0 <= P[b] < p["n"][b] for b in range(3))
                    assert P not in got
                    got.add(P)
        assert got == want


def check_rebuild_3d(case, TI, TJ):
    """Replays k_inject_sep: its window taps against the eq. spaceInt taps."""
    D, L = levels(case)
    WI, WJ = TI // 2 + 3, TJ // 2 + 3

    def sw(k):
        return -1 / 16 if k in (0, 3) else 9 / 16

    odd_w = [-1 / 16, 9 / 16, 9 / 16, -1 / 16]
    for l in range(1, len(L)):
        p, c = L[l - 1], L[l]
        for a in range(3):
            if not c["boxed"][a]:
                continue
            t1, t2 = tangents(3, a)
            e1 = c["hi"][t1] - c["lo"][t1] + 3 if c["boxed"][t1] else p["n"][t1]
            e2 = c["hi"][t2] - c["lo"][t2] + 3 if c["boxed"][t2] else p["n"][t2]
            nt1, nt2 = -(-c["n"][t1] // TI), -(-c["n"][t2] // TJ)
            for side in range(2):
                for tile in range(nt1 * nt2):
                    X0, Y0 = (tile % nt1) * TI, (tile // nt1) * TJ
                    p0i, p0j = (X0 >> 1) - 1, (Y0 >> 1) - 1
                    for ty in range(TJ):
                        for tx in range(TI):
                            xi, xj = X0 + tx, Y0 + ty
                            if not (xi < c["n"][t1] and xj < c["n"][t2]):
                                continue
                            Xn = [0] * 3
                            Xn[a], Xn[t1], Xn[t2] = (c["n"][a] - 1 if side else 0), xi, xj
                            if any(c["boxed"][b] and Xn[b] in (0, c["n"][b] - 1)
                                   for b in range(a)):
                                continue
                            want = defaultdict(float)
                            for sj in range(4 if xj & 1 else 1):
                                for si in range(4 if xi & 1 else 1):
                                    pi = ((xi - 3) // 2 if xi & 1 else xi // 2) + si
                                    pj = ((xj - 3) // 2 if xj & 1 else xj // 2) + sj
                                    want[(pi, pj)] += ((sw(si) if xi & 1 else 1)
                                                       * (sw(sj) if xj & 1 else 1))
                            got = defaultdict(float)
                            b1 = (tx - 1) >> 1 if tx & 1 else tx >> 1
                            w1 = odd_w if tx & 1 else [0, 1, 0, 0]
                            b2, w2 = ((ty - 1) >> 1, odd_w) if ty & 1 else ((ty >> 1) + 1, [1])
                            for k2, ww2 in enumerate(w2):
                                pj = b2 + k2
                                assert 0 <= pj < WJ
                                for k1, ww1 in enumerate(w1):
                                    pi = b1 + k1
                                    assert 0 <= pi < WI
                                    if ww1 * ww2:
                                        ri, rj = p0i + pi, p0j + pj
                                        # staged entries that carry weight lie in the ring
                                        assert not c["boxed"][t1] or -1 <= ri <= e1 - 2
                                        assert not c["boxed"][t2] or -1 <= rj <= e2 - 2
                                        got[(ri, rj)] += ww1 * ww2
                            assert set(got) == set(want)
                            assert all(abs(got[k] - want[k]) < 1e-15 for k in want)


def _layouts():
    from tests.test_gpu_fused import CASES as FUSED
    from tests.test_gpu_parity import CASES_2D, CASES_3D
    seen, out = set(), []
    for name, mk in list(CASES_2D) + list(CASES_3D) + list(FUSED):
        case = mk()
        key = (case.lattice, tuple(case.dims), str(case.boxes))
        if key not in seen:
            seen.add(key)
            out.append((name, case))
    return out


LAYOUTS = _layouts()
BENCH = sorted(W.CONFIGS.items())


def _restriction(case):
    ti3, ti2, tj3, nw3, nw2, _, _ = tile_constants()
    if case.dim == 3:
        check_restriction(case, ti3, tj3, nw3)
    else:
        check_restriction(case, ti2, 1, nw2)


@pytest.mark.parametrize("name,case", LAYOUTS, ids=[n for n, _ in LAYOUTS])
def test_restriction_tiles_test_layouts(name, case):
    _restriction(case)


@pytest.mark.parametrize("name,mk", BENCH, ids=[k for k, _ in BENCH])
def test_restriction_tiles_benchmark_layouts(name, mk):
    _restriction(mk())


@pytest.mark.parametrize("name,case", [x for x in LAYOUTS if x[1].dim == 3],
                         ids=[n for n, c in LAYOUTS if c.dim == 3])
def test_rebuild_taps_test_layouts(name, case):
    *_, iti, itj = tile_constants()
    check_rebuild_3d(case, iti, itj)


def check_face_buffer(case, batch=1, es=1):
    """Replays the face buffer's index arithmetic: the rebuild writes every
    node of the two faces normal to a bounded x axis (and only those) once
    per direction and run, inside the buffer; the level update's warps that
    take the face path are exactly those holding x = 0 or x = n[0] - 1, for
    every block width the autotuner tries, and read back the same slots."""
    D, L = levels(case)
    q = case.q
    if D != 3:
        return  # 2D levels have no face buffer
    for l in range(1, len(L)):
        c = L[l]
        if not c["boxed"][0]:
            continue
        n = c["n"]
        F = n[1] * n[2]
        runs = -(-batch // es) * es
        size = runs * 2 * q * F
        written = {}
        # the rebuild: x-face tiles (t1 = y, t2 = z), every node of the face
        for side in range(2):
            x = n[0] - 1 if side else 0
            for z in range(n[2]):
                for y in range(n[1]):
                    for r in range(batch):
                        base = ((((r // es) * 2 + side) * q) * F + z * n[1] + y) * es + r % es
                        for i in range(q):
                            e = base + i * F * es
                            assert 0 <= e < size
                            assert e not in written
                            written[e] = (r, x, y, z, i)
        assert len(written) == batch * 2 * F * q
        # the update: face warps and the face lanes (x = 0 and x = n[0] - 1)
        for bx in (32, 64, 128):
            nbx = -(-n[0] // bx)
            face_lanes = set()
            for bxi in range(nbx):
                for w in range(bx // 32):
                    xw = bxi * bx + 32 * w
                    if xw >= n[0]:
                        continue
                    has = xw == 0 or (xw <= n[0] - 1 < xw + 32)
                    lanes = [x for x in range(xw, min(xw + 32, n[0])) if x in (0, n[0] - 1)]
                    assert has == bool(lanes)
                    face_lanes.update(lanes)
            assert face_lanes == {0, n[0] - 1}
        for r in range(batch):
            for x in (0, n[0] - 1):
                side = int(x != 0)
                for z in range(0, n[2], max(1, n[2] // 7)):
                    for y in range(0, n[1], max(1, n[1] // 7)):
                        for i in range(q):
                            e = ((((r // es) * 2 + side) * q + i) * F + z * n[1] + y) * es + r % es
                            assert written[e] == (r, x, y, z, i)


@pytest.mark.parametrize("name,case", LAYOUTS, ids=[n for n, _ in LAYOUTS])
def test_face_buffer_test_layouts(name, case):
    check_face_buffer(case, batch=3, es=1)
    check_face_buffer(case, batch=3, es=2)


@pytest.mark.parametrize("name,mk", [("vortex3d_64", lambda: W.vortex_slab_d3q19(side=64)),
                                     ("pulse3d_48", lambda: W.pulse_3level_d3q27(side=48))],
                         ids=["vortex3d_64", "pulse3d_48"])
def test_face_buffer_benchmark_layouts(name, mk):
    check_face_buffer(mk(), batch=1, es=1)



def pz_planes(storage):
    """z-planes each thread of the two-node update walks (K1X2_PFZ_F / _H)."""
    s = _src()
    f = int(re.search(r"#define K1X2_PFZ_F (\d+)", s).group(1))
    h = int(re.search(r"#define K1X2_PFZ_H (\d+)", s).group(1))
    return f if storage == "fp32" else h


def check_x2_walk(n, batch, bx, by, pz):
    """Replays k_stream_collide_x2's block / thread / z-walk mapping: every
    node of every run is updated exactly once, by a thread whose walk stays
    inside the level and whose prefetch targets the plane it walks to next."""
    nbx, nby, nzb = -(-n[0] // bx), -(-n[1] // (2 * by)), -(-n[2] // pz)
    seen = {}
    for bz in range(nzb * batch):
        run, zc = (bz // nzb, bz % nzb) if batch > 1 else (0, bz)
        for byi in range(nby):
            for ty in range(by):
                y0 = (byi * by + ty) * 2
                for k in range(pz):
                    z = zc * pz + k
                    if z >= n[2]:
                        break
                    if k + 1 < pz and z + 1 < n[2]:
                        assert zc * pz + k + 1 == z + 1 < n[2]
                    for yy in (y0, y0 + 1):
                        if yy >= n[1]:
                            continue
                        key = (run, z, yy)
                        seen[key] = seen.get(key, 0) + 1
    # x: every node of a row by exactly one lane of the row's x blocks
    lanes = [b * bx + t for b in range(nbx) for t in range(bx) if b * bx + t < n[0]]
    assert lanes == list(range(n[0]))
    assert len(seen) == batch * n[1] * n[2] and set(seen.values()) == {1}


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_x2_walk_covers_every_node_once(storage):
    """For the test and benchmark 3D layouts' levels, every block shape the
    autotuner tries, one and three runs."""
    pz = pz_planes(storage)
    cases = [c for _, c in LAYOUTS] + [mk() for _, mk in BENCH]
    shapes = [(32, 4), (32, 2), (32, 1), (64, 2), (64, 1), (128, 1), (32, 3)]
    done = 0
    for case in cases:
        D, L = levels(case)
        if D != 3:
            continue
        for lev in L:
            n = lev["n"]
            if n[0] * n[1] * n[2] > 3_000_000:
                n = [n[0], min(n[1], 70), min(n[2], 37)]  # (the mapping does not depend on size)
            for bx, by in shapes:
                for batch in (1, 3):
                    check_x2_walk(n, batch, bx, by, pz)
                    done += 1
    assert done > 0
