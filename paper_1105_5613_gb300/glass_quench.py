"""Liquid-glass quench of the soft-sphere mixture (Sec. 4): the caloric curve U(T) and the
radial distribution function of the glass, run through the library's public calls.

Protocol (Sec. 4, Fig. 5): 80:20 soft-sphere mixture (Eq. sc0, the benchmark parameters of
Sec. 3) at number density 1.2, cutoff r_c = 1.2 with the shifted-force truncation
(Eq. mod0), time step 1e-3; the system is brought to T = 3, held there, then cooled along a
linear ramp to T = 1e-3.  Temperatures are imposed by the Nose-Hoover thermostat.  Every
`every` steps the target temperature, the kinetic temperature and the potential energy per
particle are recorded; at the end the partial and total g(r) of the glass.

    python -m paper_1105_5613_gb300.glass_quench --ncell 40 --out glass.json

analyse() fits the liquid branch with U = a + b T^(3/5) (the form of Sec. 4) and the glass
branch with a straight line, and reports T_g where the two fits cross.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def soft_sphere_params(rc=1.2, skin=0.3, block_z=0):
    from . import bbmd

    p = bbmd.ka_params(potential=bbmd.POT_SOFT, shift=bbmd.SHIFT_FORCE, skin=skin,
                       block_z=block_z)
    for a in range(2):
        for b in range(2):
            p.rcut[a][b] = rc
    return p


def run(ncell=40, heat_steps=200_000, cool_steps=3_000_000, dt=1e-3, T_high=3.0, T_low=1e-3,
        tau=0.5, every=1000, rc=1.2, seed=0, gr_bins=500, gr_rmax=5.0, frac_b=0.8, log=None):
    """Run the quench; returns a dict with the recorded curve and the final g(r).  frac_b:
    fraction of species B (label 1, sigma_BB = 0.88): 0.8 is the paper's "20:80" read literally
    (species 1 first), the reading that reproduces its T_g."""
    from inputs import generate as gen

    from . import bbmd

    n = 4 * ncell ** 3
    L = gen.box_for(n, 1.2)
    nb = int(round(frac_b * n))
    sp = gen.assign_species(n, nb, seed)
    sim = bbmd.Sim(soft_sphere_params(rc), n, L, sp, None, None, T0=T_high, seed=seed)
    rows = []
    t0 = time.perf_counter()
    done = 0

    def record(T_target):
        o = sim.observe(bbmd.OBS_ENERGY)
        rows.append((done, T_target, o["temperature"], o["pe"] / n, o["n_rebuilds"]))

    while done < heat_steps:
        k = min(every, heat_steps - done)
        sim.step(k, dt, (bbmd.THERMO_NH, T_high, T_high, tau))
        done += k
        record(T_high)
    if heat_steps > 0:
        sim.tune()  # block shape for the liquid
    c = 0
    while c < cool_steps:
        k = min(every, cool_steps - c)
        Ta = T_high + (T_low - T_high) * c / cool_steps
        Tb = T_high + (T_low - T_high) * (c + k) / cool_steps
        sim.step(k, dt, (bbmd.THERMO_NH, Ta, Tb, tau))
        c += k
        done += k
        record(Tb)
        if log and len(rows) % 200 == 0:
            log(f"step {done}: T {rows[-1][2]:.4f} U/N {rows[-1][3]:.5f}")
    o = sim.observe(bbmd.OBS_GR | bbmd.OBS_ENERGY, nbins=gr_bins, rmax=gr_rmax)
    na = n - nb
    gab = o["gr"]
    w = np.array([[na * (na - 1), na * nb], [nb * na, nb * (nb - 1)]], dtype=np.float64)
    g_total = (gab * w[:, :, None]).sum(axis=(0, 1)) / w.sum()
    info = sim.info()
    sim.close()
    return {"n": n, "frac_b": frac_b, "box": L, "dt": dt, "rc": rc, "heat_steps": heat_steps,
            "cool_steps": cool_steps, "every": every, "block_z": info["block_z"],
            "seconds": time.perf_counter() - t0,
            "curve": {"step": [r[0] for r in rows], "T_target": [r[1] for r in rows],
                      "T": [r[2] for r in rows], "U": [r[3] for r in rows],
                      "rebuilds": [r[4] for r in rows]},
            "gr": {"r": list(((np.arange(gr_bins) + 0.5) * gr_rmax / gr_bins)),
                   "total": g_total.tolist(), "AA": gab[0, 0].tolist(),
                   "AB": gab[0, 1].tolist(), "BB": gab[1, 1].tolist()}}


def analyse(T, U, liquid_min=0.6, glass_max=0.1):
    """Caloric-curve analysis of Sec. 4: U = a + b T^(3/5) fitted on T >= liquid_min, a
    straight line on T <= glass_max (least squares); T_g = the temperature in between where
    the two fits meet (the liquid fit minus the glass fit changes sign)."""
    T = np.asarray(T, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64)
    liq = T >= liquid_min
    gla = T <= glass_max
    A = np.stack([np.ones(liq.sum()), T[liq] ** 0.6], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, U[liq], rcond=None)
    B = np.stack([np.ones(gla.sum()), T[gla]], axis=1)
    (c, d), *_ = np.linalg.lstsq(B, U[gla], rcond=None)
    grid = np.linspace(glass_max, liquid_min, 4001)
    diff = (a + b * grid ** 0.6) - (c + d * grid)
    sgn = np.flatnonzero(np.diff(np.sign(diff)) != 0)
    Tg = float(grid[sgn[0]]) if sgn.size else float("nan")
    res_liq = U[liq] - (a + b * T[liq] ** 0.6)
    return {"liquid_fit": {"a": float(a), "b": float(b), "rms": float(np.sqrt(np.mean(res_liq ** 2)))},
            "glass_fit": {"c": float(c), "d": float(d)}, "T_g": Tg}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--ncell", type=int, default=40)
    ap.add_argument("--heat-steps", type=int, default=200_000)
    ap.add_argument("--cool-steps", type=int, default=3_000_000)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--rc", type=float, default=1.2)
    ap.add_argument("--frac-b", type=float, default=0.8,
                    help="fraction of species B (sigma_BB = 0.88): 0.8 reads the paper's 20:80 "
                         "literally, species 1 first")
    ap.add_argument("--liquid-min", type=float, default=0.6)
    ap.add_argument("--glass-max", type=float, default=0.1)
    ap.add_argument("--out", default="glass.json")
    args = ap.parse_args()
    res = run(args.ncell, args.heat_steps, args.cool_steps, args.dt, every=args.every, rc=args.rc,
              frac_b=args.frac_b, log=print)
    c = res["curve"]
    k = args.heat_steps // args.every  # the cooling part of the curve
    res["analysis"] = analyse(c["T"][k:], c["U"][k:], args.liquid_min, args.glass_max)
    with open(args.out, "w") as f:
        json.dump(res, f)
    print(json.dumps({"n": res["n"], "seconds": res["seconds"], "block_z": res["block_z"],
                      "analysis": res["analysis"]}))


if __name__ == "__main__":
    main()
