"""Long precision study (run as a script on a GPU; not collected by pytest):
the Sedov-Taylor blast of the precision test carried to a blast radius of
0.25 box lengths, the FP32-mixed form on the whole 512^3 box against the FP64
path, which equals the oracle bit for bit in every parity test.

The FP64 reference runs on the central 288^3 sub-box with outflow edges.
While the blast stays inside it this is the same problem: outside the blast
the state is uniform, a uniform state is exactly steady in every scheme, and
an outflow edge of a uniform state is uniform.  The script checks both
sides of that claim at every report: the mixed run's field outside the
sub-box and the FP64 run's outermost layer equal the background exactly.

Both forms take the FP64 run's dt (CFL 0.4 on its state).  Reported at
Sedov-Taylor radii R = 0.05 ... 0.25 (t from R = xi0 (E t^2/rho)^(1/5),
xi0 = 1.15): relative L1 per variable (max over variables) of mixed vs FP64
on the 64^3 cut around the centre and on the whole sub-box, the blast radius
from the density maximum along the six axis rays, and the largest difference
between those six profiles (symmetry).

    python -m tests.study_sedov_long [--n 512] [--sub 288]
"""
import argparse
import json
import time

import numpy as np

from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import workloads as W

GAMMA = 5.0 / 3.0
FLOORS = dict(dens_floor=1e-12, pres_floor=1e-12)
XI0 = 1.15


def _params(prec, dx, dt_dev=None):
    return H.Params(scheme=H.CTU, recon=H.PPM, riemann=H.RS_HLLC, limiter=H.LIM_MINMOD, precision=prec,
                    gamma=GAMMA, dx=dx, dt_dev=dt_dev, **FLOORS)


def _rel_l1(a, b):
    a = a.reshape(5, -1)
    b = b.reshape(5, -1)
    out = []
    for v in range(5):
        den = np.abs(b[v]).sum()
        if den < 1e-9 * np.abs(b[0]).sum():
            den = np.abs(b[0]).sum()
        out.append(float(np.abs(a[v] - b[v]).sum() / den))
    return max(out)


def run(n=512, sub=288, radii=(0.05, 0.10, 0.15, 0.20, 0.25), cfl=0.4):
    import torch
    dev = torch.device("cuda:0")
    dx = (1.0 / n,) * 3
    a = n // 2 - sub // 2
    Usub = W.sedov(n, gamma=GAMMA, window=sub)
    bg = Usub[:, 0, 0, 0].copy()
    # mixed form: the whole box
    fm = torch.empty((5, n, n, n), dtype=torch.float32, device=dev)
    for v in range(5):
        fm[v].fill_(float(bg[v]))
    fm[:, a:a + sub, a:a + sub, a:a + sub] = torch.tensor(Usub, dtype=torch.float32, device=dev)
    gm = torch.empty_like(fm)
    # FP64 reference: the sub-box
    f64 = torch.tensor(Usub, dtype=torch.float64, device=dev)
    g64 = torch.empty_like(f64)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    red_ws = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=dev)
    p64 = _params(H.FP64, dx, dt)
    ws = H.hydro_workspace_bytes(p64)
    p64.workspace = torch.empty(max(ws, 16), dtype=torch.uint8, device=dev)
    pm = _params(H.FP32_MIXED, dx, dt)
    t_targets = [(R / XI0) ** 2.5 for R in radii]  # rho = E = 1
    t, step, k = 0.0, 0, 0
    rows = []
    t0 = time.perf_counter()
    bg64 = torch.tensor(bg, dtype=torch.float64, device=dev)
    bg32 = torch.tensor(bg, dtype=torch.float32, device=dev)
    while k < len(t_targets):
        H.hydro_cfl_dt(f64, dx, cfl, dt, red_ws, gamma=GAMMA, precision=H.FP64, **FLOORS)
        dtv = float(dt.item())
        if t + dtv > t_targets[k]:
            dtv = t_targets[k] - t
            dt.fill_(dtv)
        H.hydro_advance_uniform(p64, f64, g64, bc=H.BC_OUTFLOW)
        H.hydro_advance_uniform(pm, fm, gm, bc=H.BC_OUTFLOW)
        f64, g64 = g64, f64
        fm, gm = gm, fm
        t += dtv
        step += 1
        if t >= t_targets[k] * (1 - 1e-12):
            torch.cuda.synchronize()
            ref = f64.cpu().numpy()
            got = fm[:, a:a + sub, a:a + sub, a:a + sub].double().cpu().numpy()
            c = sub // 2
            cut = (slice(None), slice(c - 32, c + 32), slice(c - 32, c + 32), slice(c - 32, c + 32))
            # outside the sub-box the mixed run is still the background
            out_dev = float((fm[:, :a].reshape(5, -1) - bg32[:, None]).abs().max())
            edge = torch.cat([f64[:, 0].reshape(5, -1), f64[:, -1].reshape(5, -1), f64[:, :, 0].reshape(5, -1),
                              f64[:, :, -1].reshape(5, -1), f64[:, :, :, 0].reshape(5, -1),
                              f64[:, :, :, -1].reshape(5, -1)], dim=1)
            edge_dev = float((edge - bg64[:, None]).abs().max())
            rho = ref[0]
            rays = [rho[c, c, c:], rho[c, c, :c][::-1], rho[c, c:, c], rho[c, :c, c][::-1], rho[c:, c, c],
                    rho[:c, c, c][::-1]]
            rays = [r[:min(len(x) for x in rays)] for r in rays]
            R_num = (np.mean([np.argmax(r) for r in rays]) + 0.5) / n
            sym = float(max(np.abs(r - rays[0]).max() for r in rays[1:]))
            row = {"R_target": radii[k], "t": t, "steps": step, "R_numeric": R_num,
                   "R_sedov_taylor": XI0 * t ** 0.4,
                   "rel_l1_cut64": _rel_l1(got[cut], ref[cut]), "rel_l1_subbox": _rel_l1(got, ref),
                   "max_rel_dev_density_cut": float(np.abs(got[0][cut[1:]] - ref[0][cut[1:]]).max() /
                                                   np.abs(ref[0][cut[1:]]).max()),
                   "mixed_outside_subbox_max_dev": out_dev, "fp64_subbox_edge_max_dev": edge_dev,
                   "ray_symmetry_max_diff_fp64": sym, "wall_s": time.perf_counter() - t0}
            rows.append(row)
            print(json.dumps(row), flush=True)
            k += 1
    return rows


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--sub", type=int, default=288)
    args = ap.parse_args()
    run(args.n, args.sub)
