"""Benchmark of the multi-level lattice Boltzmann step on GB300.

Workload (default, the largest single-GPU configuration): the D3Q19
convected vortex column across a refinement slab -- coarse 256^3 (y, z
periodic), fine slab x in [128, 256] coarse units (257 x 512 x 512 fine
nodes, 2 sub-steps per coarse step), recursive-regularized collision,
tau_c = 0.5 + 5e-5, binary32 shifted storage: 143.3 M node updates per
coarse step, 6.4 GB of resident populations (far above the 129 MB L2).

A step is one coarse step of the whole hot path: history capture, two fine
sub-steps with their coarse-to-fine rebuilds, the fine-to-coarse
restriction and the coarse update.

Metric: MLUPS, node updates per second counted at each level's own rate
(sum_l 2^l N_l^active per coarse step), and the fraction of the measured HBM
bandwidth reached by the dominant kernel (the fine-level update).  The
timed region (K coarse steps) is repeated and the median reported.  Other
workloads (the 2D acoustic pulse as a batch in binary32 and binary16, the
three-level D3Q27 pulse), storage and collision variants, the serving
stream and the oracle on the host cores are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2004_11863_gb300 import workloads as W  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes per launch of the dominant kernel from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), per active node of the
# level and run, with the hash of the kernel sources it was taken on;
# ignored once the sources change.
NCU_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on the fine-
    # level update of the same slab with full-width rows (257 fine nodes per
    # row) and y, z cut to 128 fine nodes (vortex3d_yz64, a 2-run batch,
    # 8,421,376 node updates per launch): odd launches 722.5 + 604.9 and
    # 722.6 + 601.7 MB, even 727.4 + 599.9 and 727.3 + 599.7 MB; per node
    # update 157.6, 157.3, 157.6 and 157.6 B, mean 157.5 B (152 B
    # algorithmic).  The rows, and so the per-node traffic, are those of the
    # full size.
    ("vortex3d", "fp32", "update_L1"): {"bytes_per_node": 157.5, "src": "c278bde650f8157f"},
}


def kernel_source_hash() -> str:
    """Hash of the level update's source: lattice.cuh and lattice_x2.cuh
    (the collisions) and the part of kernels.cuh from the addressing helpers
    to the end of the paired binary16 update.  Edits elsewhere do not void a
    traffic capture."""
    csrc = os.path.join(ROOT, "paper_2004_11863_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("lattice.cuh", "lattice_x2.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "kernels.cuh"), "r") as fh:
        k = fh.read()
    start = k.index("__device__ __forceinline__ int wrapi")
    end = k.index("k_stream_collide_pair(LevelView v")
    end = k.index("\n}\n", end) + 3  # the end of k_stream_collide_pair
    h.update(k[start:end].encode())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.05)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, n in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def workload_case(name: str):
    """A workload by name: pulse2d[_bgk], vortex2d, vortex3d, pulse3d; a
    suffix _<side> gives a 3D workload's structure at a smaller coarse side
    (e.g. vortex3d_64); vortex3d_yz<n> keeps the full-size rows (x) with n
    coarse nodes along y and z (profiling captures of the same kernels)."""
    if name == "pulse2d":
        return W.pulse_2level_d2q9("RR")
    if name == "pulse2d_bgk":
        return W.pulse_2level_d2q9("BGK")
    if name == "vortex2d":
        return W.vortex_2level_d2q9()
    base, _, side = name.partition("_")
    if base == "vortex3d" and side.startswith("yz"):  # full-width rows, shorter y, z
        return W.vortex_slab_d3q19(side=256, yz=int(side[2:]))
    if base == "vortex3d":
        return W.vortex_slab_d3q19(side=int(side) if side else 256)
    if base == "pulse3d":
        return W.pulse_3level_d3q27(side=int(side) if side else 192)
    raise SystemExit(f"unknown workload {name}")


def oracle_sample_case(case):
    """The case the host oracle is timed on: the workload itself, except for
    the full-size 3D workloads, whose FP64 oracle holds 12-26 GB and needs
    tens of seconds per coarse step; those are sampled at the same structure
    with a 64^3 (vortex) or 96^3 (pulse) coarse level.  The oracle's cost
    per node update does not depend on the size."""
    if case.name == "vortex3d":
        return W.vortex_slab_d3q19(side=64)
    if case.name == "pulse3d":
        return W.pulse_3level_d3q27(side=96)
    return case


def active_counts_oracle_free(case):
    """Active nodes per level from the layout rules (no library call)."""
    lay = W.level_layout(case)
    counts = []
    for l, lv in enumerate(lay):
        N = int(np.prod(lv["n"]))
        if l + 1 < len(lay):
            lo, hi = case.boxes[l]
            ch = lay[l + 1]
            ina = 1
            for a in range(3):
                ina *= (hi[a] - lo[a] - 3) if ch["boxed"][a] else lv["n"][a]
            N -= ina
        counts.append(N)
    return counts


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(vals, ws):
    """Element-wise maximum of a list of floats over all ranks (the list
    itself at one rank): every rank's timings reduce to the slowest."""
    if ws <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def run_reference(args, case, ws, rank):
    """The oracle as it stands on the host cores: same metric and config,
    each step a bounded sample (one coarse step of one run of the workload,
    or of its reduced-size sample for the full-size 3D workloads)."""
    if rank != 0:
        return
    import oracle
    cores = oracle.set_threads(0)
    sc = oracle_sample_case(case)
    r = oracle.Run.from_case(sc)
    U = W.updates_per_coarse_step(sc, active_counts_oracle_free(sc))
    for _ in range(args.warmup):
        r.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.step(1)
    dt = time.perf_counter() - t0
    r.close()
    mlups = U * args.steps / dt / 1e6
    sample = (f"{args.steps} coarse steps of one {sc.name} run (after {args.warmup} warm-up)"
              + ("" if sc is case else f"; {sc.name} has the structure of {case.name} at "
                 f"coarse {sc.dims[0]}^3"))
    line = {"impl": "reference", "metric": "MLUPS", "value": round(mlups, 3), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": case.name, "lattice": case.lattice,
                       "collision": case.collision, "batch": 1},
            "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(case, budget_s=15.0):
    """Time the oracle (as it stands) on a bounded sample of the workload."""
    import oracle
    cores = oracle.set_threads(0)
    sc = oracle_sample_case(case)
    r = oracle.Run.from_case(sc)
    U = W.updates_per_coarse_step(sc, active_counts_oracle_free(sc))
    t0 = time.perf_counter()
    r.step(1)
    one = time.perf_counter() - t0
    k = max(1, min(200, int(budget_s / max(one, 1e-6))))
    t0 = time.perf_counter()
    r.step(k)
    dt = time.perf_counter() - t0
    r.close()
    sample = f"{k} coarse steps of one {sc.name} run (FP64, OpenMP on {cores} threads)"
    if sc is not case:
        sample += (f"; {sc.name} is {case.name}'s structure at coarse {sc.dims[0]}^3 "
                   f"({U} node updates per coarse step)")
    return {"value": round(U * k / dt / 1e6, 3), "unit": "MLUPS", "cores": cores,
            "kind": "oracle", "sample": sample}


# kinds of the library's per-kernel timing records (lbm_profile_read)
KERNEL_KINDS = ((0, "update"), (1, "capture"), (2, "inject"), (3, "restrict"), (5, "velocity"),
                (6, "parent_strain"), (7, "outer_layer_collide"))


def timed_region(g, stream, steps, repeats):
    """`repeats` regions of K coarse steps, each between its own CUDA events
    on the launching stream with a synchronize on both sides; ms per region."""
    import torch
    out = []
    for _ in range(repeats):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def kernel_times(g, nlevels, steps):
    """Per-kernel CUDA-event durations over `steps` coarse steps (the
    library's profiling mode launches the kernels directly, one after
    another): {name_L<level>: (total ms, launches)}."""
    g.profile(True)
    g.step(steps)
    kt = {}
    for kind, name in KERNEL_KINDS:
        for l in range(nlevels):
            t_ms, n = g.profile_read(kind, l)
            if n:
                kt[f"{name}_L{l}"] = (t_ms, n)
    g.profile(False)
    return kt


def dominant_update(kt):
    return max((k for k in kt if k.startswith("update")), key=lambda k: kt[k][0])


def new_handle(mlbm, case, storage, batch, stream, collision=None):
    return mlbm.Lbm(case.lattice, collision or case.collision, case.tau0, case.dims, case.boxes,
                    storage=storage, batch=batch, rho0=case.rho0, stream=stream.cuda_stream,
                    u_ref=case.u_ref, sigma=case.sigma)


def max_field_diff(a, b, level, run=0):
    ra, ua = a.macros(level, run)
    rb, ub = b.macros(level, run)
    m = ~np.isnan(ra)
    return (float(np.max(np.abs(ra[m] - rb[m]))), float(np.max(np.abs(ua[:, m] - ub[:, m]))))


def workload_block(mlbm, case, storage, batch, stream, args, peak, collision=None,
                   fp32_error=False):
    """MLUPS (median of the repeated timed regions) of one workload, the
    dominant level update's bandwidth and fraction of the HBM peak, and each
    kernel's share of the step.  The initial state is set on the device
    (lbm_init_analytic).  fp32_error: also step a binary32 run of the same
    state as far and report the largest difference of rho and u on the
    finest level (binary32 itself is within 1e-6 of the FP64 oracle)."""
    coll = collision or case.collision
    counts = active_counts_oracle_free(case)
    U = W.updates_per_coarse_step(case, counts)
    g = new_handle(mlbm, case, storage, batch, stream, coll)
    for b in range(batch):
        g.init_analytic(case.ic, b)
    g.autotune(reps=5)
    g.step(args.warmup)
    ms = timed_region(g, stream, args.steps, args.repeats)
    kt = kernel_times(g, case.nlevels, args.steps)
    dom = dominant_update(kt)
    lev = int(dom.split("_L")[1])
    t_ms, n = kt[dom]
    sb = 4 if storage == "fp32" else 2
    # algorithmic bytes of the level update: q populations read and written;
    # the hybrid update also reads the D velocity planes once
    ab = counts[lev] * batch * (2 * case.q * sb + (4 * case.dim if coll == "HRR" else 0))
    gbs = ab / (t_ms / n * 1e-3) / 1e9
    tot = sum(v[0] for v in kt.values())
    med = float(np.median(ms))
    out = {"value": round(U * batch * args.steps / (med * 1e-3) / 1e6, 1), "unit": "MLUPS",
           "batch": batch, "ms_per_step": round(med / args.steps, 4),
           "dominant_kernel": f"update level {lev}",
           "dominant_kernel_gbs": round(gbs, 1), "dominant_kernel_frac": round(gbs / peak, 4),
           "interface_share": round(sum(v[0] for k, v in kt.items()
                                        if not k.startswith("update")) / tot, 4),
           "kernel_time_share": {k: round(v[0] / tot, 4) for k, v in kt.items()}}
    if coll == "HRR":
        pt, pn = kt[f"velocity_L{lev}"]
        pb = counts[lev] * batch * (case.q * sb + 4 * case.dim)
        out.update({"sigma": case.sigma,
                    "velocity_pass_gbs": round(pb / (pt / pn * 1e-3) / 1e9, 1),
                    "velocity_pass_frac": round(pb / (pt / pn * 1e-3) / 1e9 / peak, 4)})
    if fp32_error:
        total = g.coarse_steps()
        r = new_handle(mlbm, case, "fp32", 1, stream, coll)
        r.init_analytic(case.ic, 0)
        r.step(total)
        dr, du = max_field_diff(g, r, case.nlevels - 1)
        out["max_abs_diff_vs_fp32_after"] = {"coarse_steps": total, "drho": dr, "du": du,
                                             "level": case.nlevels - 1}
        r.close()
    g.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--repeats", type=int, default=5, help="timed regions of K steps (median)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="vortex3d")
    ap.add_argument("--batch", type=int, default=0, help="runs per GPU (0: enough to exceed L2 4x)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-others", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-variants", action="store_true", help="skip the storage/collision variants")
    ap.add_argument("--serve", type=int, default=32, help="requests of the serving run (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.repeats = max(args.repeats, 1)

    ws, rank, local = dist_setup(args)
    case = workload_case(args.workload)
    if args.impl == "reference":
        run_reference(args, case, ws, rank)
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2004_11863_gb300 import build as B
    B.build()
    from paper_2004_11863_gb300 import mlbm

    counts = active_counts_oracle_free(case)
    U = W.updates_per_coarse_step(case, counts)
    s_bytes = 4 if args.storage == "fp32" else 2
    bytes_per_run = sum(2 * case.q * s_bytes * n for n in counts)  # one update of every level
    batch = args.batch or max(1, math.ceil(4 * L2_BYTES / (bytes_per_run / 2)))
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peaks()

    # initial fields (pinned host buffers, reused by the end-to-end pass)
    fields = []
    for l in range(case.nlevels):
        rho, u = W.initial_fields(case, l)
        rp = torch.from_numpy(rho).pin_memory()
        up = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
        fields.append((rp, up))
        del rho, u

    g = mlbm.Lbm(case.lattice, case.collision, case.tau0, case.dims, case.boxes,
                 storage=args.storage, batch=batch, rho0=case.rho0, stream=stream.cuda_stream,
                 u_ref=case.u_ref)
    for l in range(case.nlevels):
        for b in range(batch):
            g.init(l, b, fields[l][0].numpy(), fields[l][1].numpy())
    # launch shapes of the level updates, chosen by the library's autotuner
    shapes = g.autotune(reps=5)
    g.step(args.warmup)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()

    # ------------- timed region: K graph-replayed coarse steps, repeated ---
    l0 = g.kernel_launches()
    with ClockSampler(local) as clk:
        regions = timed_region(g, stream, args.steps, args.repeats)
    launches = (g.kernel_launches() - l0) // args.repeats
    ms = max_over_ranks([float(np.median(regions))], ws)[0]
    mlups = U * batch * ws * args.steps / (ms * 1e-3) / 1e6
    mass, mom, stable = g.diag(0)

    # ------------- per-kernel durations (CUDA events, same workload) -------
    kt = kernel_times(g, case.nlevels, args.steps)
    dom = dominant_update(kt)
    dom_level = int(dom.split("_L")[1])
    t_ms, n = kt[dom]
    avg_s = t_ms / n * 1e-3
    alg_bytes = counts[dom_level] * batch * 2 * case.q * s_bytes
    achieved = alg_bytes / avg_s / 1e9
    src_hash = kernel_source_hash()
    tr = NCU_TRAFFIC.get((case.name, args.storage, dom))
    traffic = (round(tr["bytes_per_node"] * counts[dom_level] * batch)
               if tr and tr["src"] == src_hash else None)
    step_total = sum(v[0] for v in kt.values()) / args.steps
    shares = {k: round(v[0] / args.steps / step_total, 4) for k, v in kt.items()}

    # ------------- end to end through the C ABI with host buffers ----------
    # Initial fields uploaded from pinned host memory, then every coarse step
    # followed by a device-to-host read of that step's result: the probe
    # samples (rho, u at 16 probe nodes of the finest level, every run), the
    # time series the paper's noise analysis is built on; finally the
    # macroscopic fields of every level and run are read back.
    torch.cuda.synchronize()
    n1 = W.level_layout(case)[-1]["n"]
    probes = [[int(n1[0] * (k + 1) / 17), int(n1[1] / 2), int(n1[2] / 2)] for k in range(16)]
    g.probe_add(case.nlevels - 1, probes)
    rec = torch.empty((args.steps, batch, len(probes), 4), dtype=torch.float64).pin_memory()
    recn = rec.numpy()
    outs = []
    for l in range(case.nlevels):
        N = fields[l][0].numel()
        outs.append((torch.empty(N, dtype=torch.float64).pin_memory().numpy(),
                     torch.empty((3, N), dtype=torch.float64).pin_memory().numpy()))
    # three passes, each from a fresh set-up of the same fields (host-to-
    # device copy rates on this host vary from pass to pass); the median
    # pass is reported, the others beside it
    passes = []
    for rep in range(3):
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for l in range(case.nlevels):
            for b in range(batch):
                g.init(l, b, fields[l][0].numpy(), fields[l][1].numpy())
        t_init = time.perf_counter()
        d2h_probe = 0
        for k in range(args.steps):
            g.step(1)
            got = g.probe_async(recn[k:k + 1])
            d2h_probe += got * recn[k].nbytes
        g.sync()
        t_steps = time.perf_counter()
        for l in range(case.nlevels):
            for b in range(batch):
                g.macros(l, b, out=outs[l])
        t_end = time.perf_counter()
        passes.append(max_over_ranks([t_end - t0, t_init - t0, t_steps - t_init,
                                      t_end - t_steps], ws))
    order = sorted(range(3), key=lambda r: passes[r][0])
    e2e_s, ti, ts_, tr = passes[order[1]]
    phases = {"init_s": round(ti, 4), "steps_s": round(ts_, 4), "readout_s": round(tr, 4)}
    if not np.all(np.isfinite(recn)):
        raise RuntimeError("probe record not finite after the end-to-end run")
    h2d = sum(4 * fields[l][0].numel() * 8 for l in range(case.nlevels)) * batch
    d2h = h2d + d2h_probe
    e2e = {"value": round(U * batch * ws * args.steps / e2e_s / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
           "note": f"lbm_init of every level and run from pinned host fields, then {args.steps} x "
                   f"(lbm_step 1 + lbm_probe_async read-back of that step's 16 probes x {batch} "
                   f"runs into pinned host memory, enqueued behind the step), then lbm_macros of "
                   f"every level and run into pinned host memory (synchronising); bytes amortised "
                   f"per step; median of three such passes",
           "phases": phases,
           "passes_mlups": [round(U * batch * ws * args.steps / p[0] / 1e6, 1) for p in passes]}
    g.close()
    del outs, rec, recn, fields

    # ------------- variants of the same workload (storage, collision) ------
    variants = {}
    if not args.no_variants:
        for vname, st, coll in (("fp16_shifted_rr", "fp16", case.collision),
                                ("fp32_shifted_bgk", "fp32", "BGK"),
                                ("fp32_shifted_hrr", "fp32", "HRR")):
            if vname.startswith(args.storage) and coll == case.collision:
                continue
            variants[vname] = workload_block(mlbm, case, st, batch, stream, args, peak, coll,
                                             fp32_error=(st == "fp16"))

    # ------------- the other workloads ------------------------------------
    others = {}
    if not args.no_others:
        for oname, wl, st in (("pulse2d_fp32", "pulse2d", "fp32"),
                              ("pulse2d_fp16", "pulse2d", "fp16"),
                              ("pulse3d_fp32", "pulse3d", "fp32"),
                              ("vortex3d_fp32", "vortex3d", "fp32")):
            oc = workload_case(wl)
            if oc.name == case.name and st == args.storage:
                continue
            oc_counts = active_counts_oracle_free(oc)
            ob = max(1, math.ceil(4 * L2_BYTES / (sum(2 * oc.q * 4 * n for n in oc_counts) / 2)))
            blk = workload_block(mlbm, oc, st, ob, stream, args, peak)
            blk["workload"] = (f"{oc.name}: {oc.lattice} {oc.collision} {oc.nlevels}-level, "
                               f"coarse {'x'.join(str(d) for d in oc.dims[:oc.dim])}, "
                               f"{st}-shifted, {ob} run(s)")
            others[oname] = blk

    # ------------- serving: continuous batching vs one run at a time -------
    # Capacities (every request there at the start) of plain one-run-at-a-
    # time stepping in FP32 and FP16 and of the FP16 server; then the server
    # under Poisson arrivals at 0.5x and 2x the sequential FP32 capacity
    # (the same seeded runs, arrival times rescaled).  The requests are the
    # first ones of the seeded serving stream, sizes and step counts as drawn.
    serving = None
    if args.serve > 0:
        from paper_2004_11863_gb300 import serve as SV
        mk = lambda rate: W.serving_requests(args.serve, rate=rate)
        new_server = lambda: SV.Server(hbm_budget=64e9, max_active=32, streams=16, chunk=25,
                                       storage="fp16")
        base = mk(1.0)
        # untimed warm-up: one short request of every (lattice, level count)
        # in the mix, through both arms, so that no timed run pays the
        # first-use load of a kernel module
        kinds = {}
        for r in base:
            kinds.setdefault((r.case.lattice, r.case.nlevels), r)
        warm = [W.Request(r.rid, 0.0, r.case.with_(steps=4)) for r in kinds.values()]
        SV.serve_sequential(warm, storage="fp16", realtime=False)
        SV.serve_sequential(warm, storage="fp32", realtime=False)
        new_server().run(warm, realtime=False)

        def fig(r):
            return {"runs_per_s": round(r["runs_per_s"], 2), "p50_s": round(r["p50_s"], 4),
                    "p99_s": round(r["p99_s"], 4), "unstable": r["unstable"]}

        seq32 = SV.serve_sequential(base, storage="fp32", realtime=False)
        seq16 = SV.serve_sequential(base, storage="fp16", realtime=False)
        cap = new_server().run(base, realtime=False)
        C = seq32["runs_per_s"]
        loads = {}
        for f in (0.5, 2.0):
            r = new_server().run(mk(f * C), realtime=True)
            loads[f"{f}x"] = {**fig(r), "arrival_rate_per_s": round(f * C, 2),
                              "max_concurrent": r["max_concurrent"]}
        same16 = all(np.array_equal(a.probes, b.probes) and np.array_equal(a.mass, b.mass)
                     for a, b in zip(cap["results"], seq16["results"]))
        d16 = max(float(np.max(np.abs(a.probes - b.probes)))
                  for a, b in zip(cap["results"], seq32["results"]))
        upd = sum(W.updates_per_coarse_step(r.case, active_counts_oracle_free(r.case))
                  * r.case.steps for r in base)
        serving = {
            "requests": args.serve,
            "stream": f"the first {args.serve} requests of the seeded serving stream "
                      "(D2Q9 1/2, D3Q19 1/4, D3Q27 1/4; 2D coarse sides 64-1024, 3D 48-160; "
                      "1-3 levels; Ma 0.05-0.2; tau-1/2 log-uniform in [1e-5,1e-2]; vortex or "
                      "pulse; 100-1000 coarse steps), sizes and step counts unscaled",
            "node_updates_total": int(upd),
            "capacity": {"sequential_fp32": fig(seq32), "sequential_fp16": fig(seq16),
                         "served_fp16": {**fig(cap), "max_concurrent": cap["max_concurrent"]}},
            "served_fp16_mlups": round(upd / cap["wall_s"] / 1e6, 1),
            "sequential_fp32_mlups": round(upd / seq32["wall_s"] / 1e6, 1),
            "served_fp16_under_load": loads,
            "accuracy": {"served_fp16_equals_sequential_fp16_bitwise": bool(same16),
                         "max_abs_probe_diff_fp16_vs_fp32": d16},
            "note": "server: continuous batching, up to 32 resident runs on 16 streams, "
                    "device memory from the caching allocator; sequential: one run at a time "
                    "with the library's defaults",
        }

    # ------------- persistent fused step vs graph replay on small runs -----
    # (lbm_set_fused: one cooperative kernel per lbm_step call; the default
    # path replays one CUDA graph per coarse step)
    fused_cmp = None
    if args.serve > 0:
        fused_cmp = {}
        small = {
            "d2q9_64": W.Case("s2d", "D2Q9", "RR", 0.52, (64, 64, 1), [((16, 16, 0), (48, 48, 1))],
                              dict(kind="pulse", center=(21.0, 32.0, 0.0), radius=3.0,
                                   amplitude=1e-3), 200),
            "d3q19_32": W.Case("s3d", "D3Q19", "RR", 0.52, (32, 32, 32),
                               [((8, 8, 8), (24, 24, 24))],
                               dict(kind="pulse", center=(11.0, 16.0, 16.0), radius=3.0,
                                    amplitude=1e-3), 200),
        }
        for key, sc in small.items():
            row = {}
            for mode, label in ((0, "graphs_us_per_coarse_step"), (1, "fused_us_per_coarse_step")):
                gs = mlbm.Lbm.from_case(sc)
                gs.set_fused(mode)
                gs.step(8)
                gs.sync()
                t0 = time.perf_counter()
                gs.step(sc.steps)
                gs.sync()
                row[label] = round((time.perf_counter() - t0) / sc.steps * 1e6, 1)
                gs.close()
            fused_cmp[key] = row

    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline or ws > 1 else cpu_baseline(case)
    dims = "x".join(str(d) for d in case.dims[:case.dim])
    line = {
        "metric": "MLUPS", "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.storage == "fp32" else "f16 storage, f32 compute",
        "data": "synthetic",
        "config": {"workload": f"{case.name}: {case.lattice} {case.collision} "
                               f"{case.nlevels}-level, coarse {dims}, boxes {case.boxes}, "
                               f"tau_c={case.tau0}, {args.storage}-shifted storage",
                   "batch_per_gpu": batch, "updates_per_coarse_step_per_run": U,
                   "update_block_shapes": [f"{bx}x{by}" for bx, by in shapes],
                   "active_nodes_per_level": counts,
                   "l2": f"inputs larger than L2: {batch} run(s) x {bytes_per_run / 2 / 1e6:.1f} MB "
                         f"resident populations",
                   "timed_regions_ms": [round(x, 4) for x in regions],
                   "timing": f"median of {args.repeats} timed regions of {args.steps} coarse steps, "
                             f"each between CUDA events on the launching stream",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": f"level update, level {dom_level}",
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, a copy; burst "
                                    f"figure: the kernel is timed alone)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "avg_launch_ms": round(t_ms / n, 5), "src_hash": src_hash},
        "kernel_time_share": shares,
        "interface_share": round(sum(v for k, v in shares.items() if not k.startswith("update")), 4),
        "clocks": clk.summary(),
        "gpu_launches": int(launches),
        "e2e": e2e,
        "variants": variants,
        "other_workloads": others,
        "serving": serving,
        "fused_step_small_runs": fused_cmp,
        "cpu_baseline": cpu,
        "stable": bool(stable),
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
