"""The paper's validation runs (Secs. 9 and 10) on the GPU path, with the
quantities its claims are about.  Everything runs through the C ABI
(lbm_create / lbm_init / lbm_step / lbm_macros / lbm_sensors / lbm_probe).

  E4, convected shear wave (Sec. 9.1; H-RR: Sec. 10.1): spuriousS modes
      detected on the fine level and a shear wave deformed by the fine-to-
      coarse crossing with BGK and RR; none detected and no deformation with
      H-RR (sigma = 0.995).
  E5, convected acoustic wave (Sec. 9.2; H-RR: Sec. 10.2): a reflected wave
      of about 1/2000 of the incident one where it leaves the fine level
      (alike for every collision); at t = 2620 the spuriousAc modes excited
      at start have turned into acoustic waves of about 1/25 (upstream,
      coarse side) and 1/100 (downstream, fine side) of the incident
      amplitude with RR, and nothing with H-RR.
  E6, convected vortex (Sec. 10.3): power spectral density of the density
      at probe P1; H-RR lowers the spurious noise by orders of magnitude at
      nu = 1e-6, and RR needs nu = 4.18e-4 (eq. tauSpuriousAc) to match it.

`python -m paper_2004_11863_gb300.validation [e4|e5|e6|all]` prints one
JSON object per run.
"""
from __future__ import annotations

import json
import math
import sys

import numpy as np

from . import workloads as W

E4_TIMES = (90, 170, 380, 840, 1280, 2900)
E5_TIMES = (900, 2050, 2620)


def _lbm():
    from . import mlbm
    return mlbm


def _union(case, g, comp):
    """(x, value) of every active node of every level, x in coarse units."""
    xs, vs = [], []
    for l in range(case.nlevels):
        rho, u = g.macros(l)
        X, _, _ = W.level_coords(case, l)
        m = ~np.isnan(rho)
        xs.append(X[m])
        vs.append((rho - case.rho0)[m] if comp == "rho" else u[comp][m])
    return np.concatenate(xs), np.concatenate(vs)


def e4(collision="RR", sigma=0.995, eps=1e-10, g_threshold=1e-8):
    """Convected shear wave.  Per sampled time: sensor counts per level
    (Ac, S, G) and the deformation -min(u_y) / max(u_y) over all levels."""
    case = W.e4_shear_wave(collision, sigma)
    g = _lbm().Lbm.from_case(case)
    for l in range(case.nlevels):
        g.sensors_enable(l, eps, g_threshold)
    out, t = [], 0
    for T in E4_TIMES:
        g.step(T - t)
        t = T
        counts = []
        for l in range(case.nlevels):
            fl = g.sensors(l)[0]
            counts.append([int(((fl >> b) & 1).sum()) for b in range(3)])
        _, uy = _union(case, g, 1)
        out.append({"t": T, "sensors_per_level": counts,
                    "uy_max": float(uy.max()), "uy_min": float(uy.min()),
                    "deformation": float(-uy.min() / uy.max())})
    g.close()
    return {"case": "E4 convected shear wave", "collision": collision,
            "sigma": sigma if collision == "HRR" else None, "samples": out}


def e5(collision="RR", sigma=0.995, length=4000):
    """Convected acoustic wave.  t = 900: incident peak and the reflected
    wave on the fine level (ratio); t = 2620: the largest |rho'| on the
    coarse side upstream of the fine level (x < 500) and on the fine level,
    where neither the incident nor the reflected wave is any more, relative
    to the amplitude A."""
    case = W.e5_acoustic_wave(collision, sigma, length)
    A = case.ic["amplitude"]
    g = _lbm().Lbm.from_case(case)
    res, t = {}, 0
    for T in E5_TIMES:
        g.step(T - t)
        t = T
        X, rp = _union(case, g, "rho")
        if T == 900:
            inc = float(rp.max())
            xi = float(X[np.argmax(rp)])
            sel = (X > 520) & (X < 990)
            refl = float(np.abs(rp[sel]).max())
            res["t900"] = {"incident": inc, "incident_x": xi, "reflected": refl,
                           "reflected_x": float(X[sel][np.argmax(np.abs(rp[sel]))]),
                           "reflected_over_incident": refl / inc}
        if T == 2620:
            coarse = X < 500  # upstream of the fine level (both waves are far away)
            fine = (X >= 500) & (X <= 1000)
            res["t2620"] = {"upstream_over_A": float(np.abs(rp[coarse]).max()) / A,
                            "downstream_fine_over_A": float(np.abs(rp[fine]).max()) / A}
    g.close()
    return {"case": "E5 convected acoustic wave", "collision": collision,
            "sigma": sigma if collision == "HRR" else None, "periodic_length": length, **res}


def psd(series, dt=1.0):
    """One-sided power spectral density of a mean-removed, Hann-windowed
    series: (frequencies in cycles per coarse step, PSD)."""
    x = np.asarray(series, dtype=np.float64)
    x = x - x.mean()
    w = np.hanning(x.size)
    X = np.fft.rfft(x * w)
    p = (np.abs(X) ** 2) / (np.sum(w * w) / dt)
    p[1:-1] *= 2.0
    return np.fft.rfftfreq(x.size, dt), p


def e6(collision="RR", sigma=0.995, nu=1e-6, steps=1800, start=300,
       bands=((0.01, 0.1), (0.1, 0.5))):
    """Convected vortex.  Density at probe P1 every coarse step; from step
    `start` on (after the acoustic transient of the initial state has passed
    the probe; its periodic images arrive after about 2000 steps) its PSD
    normalised by drho_max^2 = (rho0 - rho(centre, 0))^2 (Fig. psd_COVO),
    and the PSD integrated over frequency bands."""
    case = W.e6_vortex(collision, sigma, nu)
    g = _lbm().Lbm.from_case(case)
    g.probe_add(0, [list(W.e6_probe(case))])
    rho_c = case.rho0 * math.exp(-case.ic["eps"] ** 2 / (2 * W.CS * W.CS))
    drho_max = case.rho0 - rho_c
    series = []
    for _ in range(steps):
        g.step(1)
        rec = g.probe(max_steps=1)
        series.append(float(rec.reshape(-1)[0]))
    g.close()
    series = series[start:]
    f, p = psd(np.asarray(series))
    p = p / (drho_max ** 2)
    df = f[1] - f[0]
    band = {f"{lo}-{hi}": float(np.sum(p[(f >= lo) & (f < hi)]) * df) for lo, hi in bands}
    return {"case": "E6 convected vortex", "collision": collision,
            "sigma": sigma if collision == "HRR" else None, "nu": nu, "steps": steps,
            "window": [start, steps],
            "probe": W.e6_probe(case), "rms_rho_prime": float(np.std(series)),
            "band_power": band}


def main(argv):
    which = argv[1] if len(argv) > 1 else "all"
    runs = []
    if which in ("e4", "all"):
        runs += [e4("BGK"), e4("RR"), e4("HRR")]
    if which in ("e5", "all"):
        runs += [e5("RR"), e5("HRR")]
    if which in ("e6", "all"):
        runs += [e6("RR"), e6("HRR"), e6("RR", nu=1e-4), e6("RR", nu=4.18e-4)]
    for r in runs:
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main(sys.argv)
