"""Algorithmic operation count per cell update (roofline numerator).

Test/measurement infrastructure: runs only the oracle's operation-counting
instantiation (oracle/real.hpp, Counted) and writes
paper_1103_3373_gb300/data/flops_per_cell.json, which bench.py reads as data.

Definition.  One group step of the oracle is counted on groups of the
benchmark workload (periodic lognormal box, rms Mach 1.5, k^-3 fields).  Each
program section (state conversions, reconstruction, tracing, prediction,
Riemann solves, transverse correction, update; nested operations belong to
the outermost section) gives an average cost per call.  The count per cell
update is the sum over sections of that cost times the number of calls ONE
cell needs on an unbounded grid with nothing recomputed:
  CTU: 7 conversions (1 U->W, 6 face W->U), 15 reconstructions (3 directions
       x 5 variables), 3 tracings, 6 Riemann solves (3 faces x 2 stages),
       3 transverse corrections (one per direction, both sides);
  MHM: 13 conversions (1 U->W, 6 W->U, 6 physical fluxes), 15
       reconstructions, 1 prediction, 3 Riemann solves;
  VL : 7 conversions (1 U->W of the half step, 6 face W->U), 15
       reconstructions, 1 prediction, 6 Riemann solves (3 first-order + 3);
plus the update, counted per cell.  The directionally split schemes sweep
each cell once per direction; per cell and sweep:
  RTVD: 2 flux splittings (U^n and the half step), 1 first-order flux
       difference, 1 half step, 1 limited flux, 1 update;
  WAF : 1 side state, 1 HLLC wave fan, 1 weighted-average flux, 1 update.
CTU with characteristic reconstruction: as CTU, but one reconstruction per
direction (all 5 waves, with the projections) instead of one per variable.  Flops = additions + multiplications +
divisions + square roots + powers; comparisons / min / max / abs are reported
apart ("cmp").  The halo recomputation a patch group actually does on top is
therefore not credited.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1103_3373_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(ROOT, "paper_1103_3373_gb300", "data", "flops_per_cell.json")
FLOP = ("add", "mul", "div", "sqrt", "pow")
MIN_CALLS = {
    O.CTU: {"eos": 7, "recon": 15, "trace": 3, "riemann": 6, "correct": 3},
    O.MHM: {"eos": 13, "recon": 15, "predict": 1, "riemann": 3},
    O.VL: {"eos": 7, "recon": 15, "predict": 1, "riemann": 6},
    O.RTVD: {"eos": 6, "riemann": 3, "predict": 3, "recon": 3, "update": 3},
    O.WAF: {"eos": 3, "riemann": 3, "recon": 3, "update": 3},
}
SCHEME_NAMES = {O.MHM: "mhm", O.VL: "vl", O.CTU: "ctu", O.RTVD: "rtvd", O.WAF: "waf"}
RECON_NAMES = {O.PLM: "plm", O.PPM: "ppm"}
SOLVER_NAMES = {O.EXACT: "exact", O.HLLE: "hlle", O.HLLC: "hllc", O.ROE: "roe"}


def count(scheme, recon, rs, groups, characteristic=0):
    N = 16
    tot = {s: {c: 0 for c in O.OPCLASSES} for s in O.SECTIONS}
    calls = {s: 0 for s in O.SECTIONS}
    for Ug, dt, dx in groups:
        P = O.Params(scheme=scheme, recon=recon, riemann=rs, limiter=O.MINMOD, dt=dt, dx=dx,
                     characteristic=characteristic)
        ops, cl = O.count_ops(P, Ug, N)
        for s in O.SECTIONS:
            calls[s] += cl[s]
            for c in O.OPCLASSES:
                tot[s][c] += ops[s][c]
    per_cell = {}
    cmp_cell = 0.0
    ng = len(groups)
    need = dict(MIN_CALLS[scheme])
    if characteristic:
        need["recon"] = 3
    for s, k in need.items():
        f = sum(tot[s][c] for c in FLOP) / calls[s]
        per_cell[s] = k * f
        cmp_cell += k * tot[s]["cmp"] / calls[s]
    if "update" not in need:
        per_cell["update"] = sum(tot["update"][c] for c in FLOP) / (ng * N ** 3)
        cmp_cell += tot["update"]["cmp"] / (ng * N ** 3)
    executed = sum(sum(tot[s][c] for c in FLOP) for s in O.SECTIONS) / (ng * N ** 3)
    div_sqrt = {c: sum(tot[s][c] for s in O.SECTIONS) / (ng * N ** 3) for c in ("div", "sqrt", "pow")}
    return {"flops": sum(per_cell.values()), "by_section": per_cell, "cmp": cmp_cell,
            "executed_in_group_per_cell": executed, "executed_div_sqrt_pow_per_cell": div_sqrt}


def main():
    n, N = 32, 16
    U = W.lognormal(n, seed=1, mach=1.5)
    dx = (1.0 / n,) * 3
    dt = O.cfl_dt(U, dx, 0.4)
    table = {"definition": __doc__.strip().splitlines()[0], "workload": "periodic lognormal 32^3, rms Mach 1.5",
             "entries": {}}
    for scheme in (O.MHM, O.VL, O.CTU):
        for recon in (O.PLM, O.PPM):
            g = O.required_ghost(scheme, recon)
            Ug = O.gather(U, W.group_origins(n, n, n, N), N, g, bc=0)
            groups = [(Ug[i], dt, dx) for i in range(0, Ug.shape[0], 3)]
            for rs in (O.EXACT, O.HLLE, O.HLLC, O.ROE):
                key = "%s-%s-%s" % (SCHEME_NAMES[scheme], RECON_NAMES[recon], SOLVER_NAMES[rs])
                table["entries"][key] = count(scheme, recon, rs, groups)
                print(key, round(table["entries"][key]["flops"], 1))
    g = O.required_ghost(O.CTU, O.PPM)
    Ug = O.gather(U, W.group_origins(n, n, n, N), N, g, bc=0)
    groups = [(Ug[i], dt, dx) for i in range(0, Ug.shape[0], 3)]
    table["entries"]["ctu-ppm-roe-char"] = count(O.CTU, O.PPM, O.ROE, groups, characteristic=1)
    print("ctu-ppm-roe-char", round(table["entries"]["ctu-ppm-roe-char"]["flops"], 1))
    for scheme in (O.RTVD, O.WAF):
        g = O.required_ghost(scheme, 0)
        Ug = O.gather(U, W.group_origins(n, n, n, N), N, g, bc=0)
        groups = [(Ug[i], dt, dx) for i in range(0, Ug.shape[0], 3)]
        key = SCHEME_NAMES[scheme]
        table["entries"][key] = count(scheme, O.PLM, O.HLLC, groups)
        print(key, round(table["entries"][key]["flops"], 1))
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    with open(OUT, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
