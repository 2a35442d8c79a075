"""Write the stored oracle results of the long 3D runs.

The FP64 oracle needs tens of minutes for the reduced-size 3D workloads at
their full step counts, too long to recompute in every GPU test session, so
this script runs it once and stores sampled outputs that the GPU tests
compare against.  It calls only the oracle (``oracle/``) and the seeded input
generators (``workloads.py``); nothing here comes from the CUDA path.

Cases (the structure of the two 3D workloads at reduced size, full step
counts):

- ``vortex3d_64``: D3Q19 RR, coarse 64^3, fine slab x in [32, 64]
  (65 x 128 x 128), vortex column, 500 coarse steps;
- ``pulse3d_96``: D3Q27 RR, coarse 96^3, level 1 on [24, 72]^3 (97^3),
  level 2 on [24, 72]^3 in level-1 units (97^3), pulse, 800 coarse steps.

Stored per level (float32 deviations rho - rho0 and u, which keep ~1e-10
absolute accuracy at these magnitudes):

- every node of one plane through the flow feature (z = the vortex plane, or
  the pulse centre's z), which crosses every interface of the level;
- 2048 seeded random active nodes of the level (all faces, edges, corners);
- the FP64 sums over the level's active nodes of (rho - rho0) and rho u.

    python tests/golden/make_oracle_golden.py [name ...]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2004_11863_gb300 import workloads as W  # noqa: E402

CASES = {
    "vortex3d_64": lambda: W.vortex_slab_d3q19(steps=500, side=64),
    "pulse3d_96": lambda: W.pulse_3level_d3q27(steps=800, side=96),
}
N_RANDOM = 2048


def plane_z(case, level):
    """z index of the stored plane on `level`: the node nearest the feature's
    z (the middle of the domain for the z-uniform vortex column)."""
    lay = W.level_layout(case)[level]
    zc = case.ic["center"][2] if len(case.ic["center"]) > 2 else case.dims[2] / 2.0
    z = (zc - lay["origin"][2]) / lay["h"]
    return int(np.clip(round(z), 0, lay["n"][2] - 1))


def sample(case, r):
    out = {}
    rng = np.random.default_rng(20041186)
    for l in range(case.nlevels):
        rho, u = r.macros(l)
        n = W.level_layout(case)[l]["n"]
        act = ~np.isnan(rho)
        z = plane_z(case, l)
        plane = np.arange(z * n[0] * n[1], (z + 1) * n[0] * n[1])
        idx = np.nonzero(act)[0]
        rnd = np.sort(rng.choice(idx, size=min(N_RANDOM, idx.size), replace=False))
        for tag, ids in (("plane", plane), ("rand", rnd)):
            out[f"L{l}_{tag}_idx"] = ids.astype(np.int64)
            out[f"L{l}_{tag}_drho"] = (rho[ids] - case.rho0).astype(np.float32)
            out[f"L{l}_{tag}_u"] = u[:, ids].astype(np.float32)
        out[f"L{l}_mass"] = np.float64(np.sum(rho[act] - case.rho0))
        out[f"L{l}_mom"] = np.sum(rho[act][None, :] * u[:, act], axis=1).astype(np.float64)
        out[f"L{l}_active"] = np.int64(act.sum())
    return out


def main(names):
    cores = oracle.set_threads(0)
    for name in names:
        case = CASES[name]()
        t0 = time.time()
        r = oracle.Run.from_case(case)
        r.step(case.steps)
        data = sample(case, r)
        r.close()
        data["steps"] = np.int64(case.steps)
        path = os.path.join(HERE, f"oracle_{name}_{case.steps}.npz")
        np.savez_compressed(path, **data)
        print(f"{name}: {case.steps} coarse steps in {time.time() - t0:.0f} s on {cores} "
              f"threads -> {os.path.basename(path)} ({os.path.getsize(path) / 1e3:.0f} kB)",
              flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
