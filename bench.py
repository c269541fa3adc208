#!/usr/bin/env python
"""Benchmark of the unsplit patch-group fluid update on GB300.

Workload (the paper's uniform-mesh benchmark shape, Sec. 5.1, with synthetic
data): a 256^3 periodic box of 4096 patch groups (16^3 cells + 3 ghost
layers), lognormal density (sigma 0.5, k^-3 Gaussian field, seed 1), p = 1,
k^-3 random velocities at rms Mach 1.5, gamma 1.4, CTU + PPM (minmod) + Roe
with HLLE fallback, CFL 0.4, FP32.

One step = the whole hot path: ghost gather fused into the CTU group update
(reconstruct + trace, Riemann, transverse correction, Riemann, update, store
the group-boundary fluxes), then the FP64 CFL reduction that gives the next
step's dt on the device.  Metric: cell-updates/s (interior cells x steps /
device time), p50/p99 step latency, the roofline fraction of the dominant
kernel, the oracle on the host cores as cpu_baseline, and an end-to-end
number through host buffers.  FP64 and the mixed form are measured on the same
box as extra lines of detail.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (torchrun, one rank per GPU) every rank advances its own box
(independent replicas: weak scaling, no collective on the data path).
"""
import argparse
import dataclasses
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s (CTU+PPM+Roe, FP32 vs FP64) and % roofline; p50/p99 step latency"
UNIT = "cell-updates/s"
N_BOX = 256
CFL = 0.4
FLOORS = dict(dens_floor=1e-6, pres_floor=1e-6)
CONFIG = {"workload": "uniform 256^3 periodic box as 4096 16^3-cell patch groups (3 ghost layers); lognormal "
                      "density sigma 0.5 (k^-3 Gaussian field, seed 1), rms Mach 1.5 k^-3 velocities; CTU+PPM+Roe",
          "scheme": "ctu", "recon": "ppm", "limiter": "minmod", "riemann": "roe", "roe_fallback": "hlle",
          "box": [256, 256, 256], "patch_group": 16, "ghost": 3, "groups": 4096, "cfl": CFL, "gamma": 1.4,
          "step": "fused gather + CTU group update + boundary-flux store, then FP64 CFL reduction (device dt)",
          "l2": "no flush: the 335 MB FP32 state (671 MB FP64) exceeds the 129 MB L2 and is streamed every step"}


def mach_distribution(U, gamma=1.4):
    """Per-cell Mach number |v| / c of a conserved state [5][Z][Y][X] (host,
    FP64): the input's distribution, reported beside the workload."""
    rho = U[0].astype(np.float64)
    v2 = (U[1].astype(np.float64) ** 2 + U[2].astype(np.float64) ** 2 + U[3].astype(np.float64) ** 2) / rho ** 2
    p = (gamma - 1.0) * (U[4].astype(np.float64) - 0.5 * rho * v2)
    m = np.sqrt(v2 / (gamma * p / rho))
    q = np.percentile(m, [5, 50, 95])
    return {"rms": float(np.sqrt((m ** 2).mean())), "p05": float(q[0]), "p50": float(q[1]), "p95": float(q[2]),
            "max": float(m.max()), "supersonic_fraction": float((m > 1.0).mean())}


def sm_peak_fp32_tflops(nsm, sm_mhz):
    """Nominal FP32 ALU peak (context only): SMs x 128 FP32 lanes x 2 flop per
    FMA x clock."""
    return nsm * 128 * 2 * sm_mhz * 1e6 / 1e12


def alu_peaks(H, torch, dev, local, seconds=0.8):
    """Measured FMA rates of this GPU (include/hydro_peaks.h): FP32 scalar,
    FP32 packed pairs and FP64, each a loop of independent FMA chains on 4
    CTAs x 256 threads per SM, timed with CUDA events over about `seconds`
    of launches after one warm-up launch, SM clock sampled meanwhile."""
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    ctas, threads = 4 * nsm, 256
    out = {"ctas": ctas, "threads": threads, "chains_per_thread": 8}
    s = torch.cuda.Stream(device=dev)
    for name, kind, dt in (("fp32", H.PEAK_FP32, torch.float32), ("fp32x2", H.PEAK_FP32X2, torch.float32),
                           ("fp64", H.PEAK_FP64, torch.float64)):
        buf = torch.empty(ctas * threads, dtype=dt, device=dev)
        iters = 4096
        with torch.cuda.stream(s):
            H.hydro_fma_peak(kind, ctas, threads, iters, buf, stream=s)  # warm-up
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            H.hydro_fma_peak(kind, ctas, threads, iters, buf, stream=s)
            b.record(s)
        torch.cuda.synchronize()
        one = a.elapsed_time(b) / 1e3
        # about 20 ms per launch, `seconds` in all
        iters = max(64, int(iters * 0.02 / max(one, 1e-6)))
        reps = max(3, int(seconds / 0.02))
        sampler = ClockSampler(local)
        sampler.start()
        flops = 0.0
        with torch.cuda.stream(s):
            H.hydro_fma_peak(kind, ctas, threads, iters, buf, stream=s)
            a.record(s)
            for _ in range(reps):
                flops += H.hydro_fma_peak(kind, ctas, threads, iters, buf, stream=s)
            b.record(s)
        torch.cuda.synchronize()
        clk = sampler.stop()
        sec = a.elapsed_time(b) / 1e3
        out[name] = {"tflops": flops / sec / 1e12, "seconds": sec, "launches": reps, "iters": iters,
                     "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons")}
        del buf
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# Sources the headline kernel (CTU, primitive reconstruction, FP32) is built
# from; the stored DRAM-traffic figure is used only while they are unchanged.
HEADLINE_SOURCES = ("phys.cuh", "group.cuh", "stages.cuh", "ctu.cuh", "mhm.cuh", "vl.cuh", "split.cuh", "kernels.cuh",
                    "k_ctu_fp32.cu")


def source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1103_3373_gb300", "csrc")
    for f in HEADLINE_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.idx = vis.split(",")[local_rank] if vis else str(local_rank)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", self.idx], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": float(max(power))}


def make_params(H, precision, dx):
    return H.Params(scheme=H.CTU, recon=H.PPM, limiter=H.LIM_MINMOD, riemann=H.RS_ROE, roe_fallback=H.RS_HLLE,
                    precision=precision, gamma=1.4, dx=dx, **FLOORS)


def time_box(box, steps, warmup, torch, sampler=None):
    """Time `steps` steps (after `warmup`) with CUDA events on the box's stream.
    Returns per-step ms, mean advance-kernel ms and total ms."""
    s = box.stream
    for _ in range(warmup):
        box.step(s)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    if sampler:
        sampler.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    t0.record(s)
    for k in range(steps):
        ev[k][0].record(s)
        box.advance(s)
        ev[k][1].record(s)
        box.swap()
        box.compute_dt(s)
        box.end_step()
        ev[k][2].record(s)
    t1.record(s)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    adv_ms = [e[0].elapsed_time(e[1]) for e in ev]
    return step_ms, float(np.mean(adv_ms)), t0.elapsed_time(t1), clocks


def amr_leg(H, RT, W, torch, dev, steps=20, block_threads=0):
    """AMR-shaped batch: 4 levels of 4096/2500/1500/800 halo-prepared groups
    (refined where |grad rho|/rho > 0.3 on a seeded 128^3 lognormal root), per-
    level dx and device dt.  FP32 batched persistent launch replayed from a
    CUDA graph and autotuned (block_threads > 0: that fixed shape with whole
    runs as chains, no tuning launches, for profiling), against the same FP32
    step as one launch per level, the same batched launch with every group
    advanced alone, and the plain FP64 per-level launch (groups alone)."""
    t = time.perf_counter()
    levels = W.amr_levels()
    gen_s = time.perf_counter() - t
    out = {"groups_per_level": [int(l["U"].shape[0]) for l in levels], "generate_s": gen_s,
           "flagged_fraction": [l["flagged_fraction"] for l in levels]}
    p = make_params(H, H.FP32, (1.0, 1.0, 1.0))
    lb = RT.LevelBatch(levels, p, cfl=CFL, device=dev)
    if block_threads:
        lb.p.block_threads = min(block_threads, H.hydro_max_block_threads(lb.p))
        lb.p.chain = 0
        lb._alloc_ws()
        tb = {"block_threads": lb.p.block_threads, "chain": 0}
    else:
        tb = lb.tune()
    lb.capture()
    cells = lb.cells
    for _ in range(3):
        lb.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        lb.replay()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    out["fp32_batched_graph"] = {"value": cells / (ms / 1e3), "ms_per_step": ms,
                                 "block_threads": tb["block_threads"], "chain": tb["chain"],
                                 "runs": "z-continuations streamed as chains (zrun)"}
    # the same launch shape with every group advanced alone
    lb1 = RT.LevelBatch(levels, dataclasses.replace(lb.p, chain=1), cfl=CFL, device=dev, chains=False)
    lb1.capture()
    for _ in range(3):
        lb1.replay()
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        lb1.replay()
    b.record()
    torch.cuda.synchronize()
    ms1 = a.elapsed_time(b) / steps
    out["fp32_batched_graph_groups_alone"] = {"value": cells / (ms1 / 1e3), "ms_per_step": ms1}
    del lb1
    for _ in range(2):
        lb.step_per_level()
    torch.cuda.synchronize()
    a.record()
    for _ in range(5):
        lb.step_per_level()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 5
    out["fp32_per_level"] = {"value": cells / (ms / 1e3), "ms_per_step": ms}
    del lb
    torch.cuda.empty_cache()
    lb = RT.LevelBatch(levels, make_params(H, H.FP64, (1.0, 1.0, 1.0)), cfl=CFL, device=dev, chains=False)
    lb.step_per_level()
    torch.cuda.synchronize()
    a.record()
    for _ in range(2):
        lb.step_per_level()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / 2
    out["fp64_per_level"] = {"value": cells / (ms / 1e3), "ms_per_step": ms}
    out["unit"] = UNIT
    out["cells_per_step"] = cells
    del lb
    return out


def amr_hierarchy_leg(H, RT, W, torch, dev, replays=10):
    """Device AMR hierarchy (ghost zones interpolated in space and time,
    coarse-grid correction by the stored fluxes, restriction): a 256^3
    periodic base of 4096 groups and refined levels of 2504 / 1504 / 800
    groups (octets nearest the box centre; smooth seeded field), adaptive
    time steps (level l takes 2^l steps of dt0 / 2^l).  FP32 CTU+PPM+Roe,
    two hierarchy steps per CUDA-graph replay; cell-updates count every
    level's substeps.  Also the device time per kind of launch of one eager
    step."""
    t = time.perf_counter()
    levels = W.amr_hierarchy(256, counts=(2500, 1500, 800), seed=5)
    gen_s = time.perf_counter() - t
    p = make_params(H, H.FP32, (1.0, 1.0, 1.0))
    hier = RT.AmrHierarchy(levels, p, device=dev)
    dt0 = hier.compute_dt(CFL)
    out = {"groups_per_level": [len(lv["origin"]) for lv in levels], "generate_s": gen_s, "dt0": dt0,
           "cells_per_step": hier.cells_per_step, "launches_per_step": hier.launches_per_step()}
    split = hier.step_timed(dt0)
    hier.capture(dt0)
    hier.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(replays):
        hier.replay()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / (2 * replays)
    out["fp32_graph"] = {"value": hier.cells_per_step / (ms / 1e3), "ms_per_step": ms, "steps": 2 * replays,
                         "runs": "each level's columns streamed as chains (zrun)"}
    tot = sum(split.values())
    out["eager_split_ms"] = {k: round(v, 3) for k, v in split.items()}
    out["eager_split_share"] = {k: round(v / tot, 4) for k, v in split.items()}
    out["errors"] = hier.errors()
    out["state_finite"] = bool(all(torch.isfinite(u).all().item() for u in hier.cur))
    out["unit"] = UNIT
    del hier
    torch.cuda.empty_cache()
    # the same hierarchy with every group advanced alone
    hier = RT.AmrHierarchy(levels, make_params(H, H.FP32, (1.0, 1.0, 1.0)), device=dev, chains=False)
    hier.capture(dt0)
    hier.replay()
    torch.cuda.synchronize()
    a.record()
    for _ in range(replays):
        hier.replay()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / (2 * replays)
    out["fp32_graph_groups_alone"] = {"value": hier.cells_per_step / (ms / 1e3), "ms_per_step": ms}
    del hier
    torch.cuda.empty_cache()
    return out


def serving_leg(H, torch, dev, n_requests=2000):
    """Serving: the n_requests of the seeded Poisson stream (200/s;
    boxes 32/64/128/256^3 with weights .4/.3/.2/.1; Mach 0.5-3; 5-50 steps;
    FP32 CTU+PPM+Roe), admitted by an HBM budget of half the free memory."""
    from paper_1103_3373_gb300 import serving as SV
    from paper_1103_3373_gb300 import workloads as W
    reqs = SV.requests_from_arrivals(W.poisson_arrivals(rate=200.0, n=n_requests, seed=6))
    eng = SV.ServingEngine(make_params(H, H.FP32, (1.0, 1.0, 1.0)), device=dev)
    summ = eng.run(reqs, realtime=True)
    summ["unit"] = UNIT
    summ["requests_offered"] = n_requests
    return summ


def cpu_baseline(U, dx, budget_s=12.0):
    """The FP64 oracle as it stands, OpenMP over patch groups on all host cores,
    on a bounded sample of the workload's groups (one step each)."""
    import oracle as O
    from paper_1103_3373_gb300 import workloads as W
    Uq = U.astype(np.float32).astype(np.float64)
    dt = O.cfl_dt(Uq, dx, CFL, 1.4, **FLOORS)
    P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, limiter=O.MINMOD, fallback=O.HLLE, gamma=1.4, dt=dt,
                 dx=dx, **FLOORS)
    orig = W.group_origins(N_BOX, N_BOX, N_BOX, 16)
    cores = O.max_threads()
    probe = min(len(orig), max(8, cores))
    Ug = O.gather(Uq, orig[:probe], 16, 3, bc=0)
    t = time.perf_counter()
    O.advance(P, Ug, 16)
    per_group = (time.perf_counter() - t) / probe
    S = int(min(len(orig), max(probe, budget_s / max(per_group, 1e-6))))
    S = max(cores, (S // cores) * cores)
    Ug = O.gather(Uq, orig[:S], 16, 3, bc=0)
    t = time.perf_counter()
    O.advance(P, Ug, 16)
    el = time.perf_counter() - t
    # one core, small sample
    S1 = max(1, min(4, S))
    t = time.perf_counter()
    O.advance(P, Ug[:S1], 16, nthreads=1)
    el1 = time.perf_counter() - t
    return {"value": S * 4096 / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one CTU+PPM+Roe FP64 step of the first %d of the 4096 patch groups of the same box "
                      "(%.1f s on %d threads)" % (S, el, cores),
            "single_core": {"value": S1 * 4096 / el1, "groups": S1, "seconds": el1}}


def oracle_configs(H, RT, W, torch, dev, cpu_c2=None, gpu_c2=None):
    """The oracle (one core and all host cores) beside the GPU on the other
    stated workloads, and the paper's "speed-up over one CPU core" as GPU /
    oracle-1-core (a different CPU and a different code than the paper's):
      c1      32^3 Sod along x, FP64, MHM + PLM minmod + Roe, outflow, CFL 0.5,
              10 steps (GPU: FP64);
      c4_cut  the central 64^3 cells of the 512^3 Sedov start, one
              CTU + PPM + HLLC step, outflow (GPU: FP64 and the FP32 mixed form);
      c2      the headline box (from the main line and the cpu_baseline leg)."""
    import oracle as O
    out = {}
    N = 16

    def gpu_rate(U, p, bc, steps, cfl):
        box = RT.UniformBox(U, p, cfl=cfl, bc=bc, device=dev)
        box.compute_dt()
        for _ in range(2):
            box.step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(box.stream)
        for _ in range(steps):
            box.step()
        b.record(box.stream)
        torch.cuda.synchronize()
        cells = U[0].size
        return cells * steps / (a.elapsed_time(b) / 1e3)

    def oracle_rate(U, P, ghost, bc, steps, cfl, nthreads=None):
        n = U.shape[1]
        orig = W.group_origins(n, n, n, N)
        dx = P.dx
        t = time.perf_counter()
        for _ in range(steps):
            P.dt = O.cfl_dt(U, dx, cfl, P.gamma, P.dens_floor, P.pres_floor)
            kw = {} if nthreads is None else {"nthreads": nthreads}
            U = W.scatter_groups(O.advance(P, O.gather(U, orig, N, ghost, bc=bc), N, **kw)[0], n, n, n)
        return U[0].size * steps / (time.perf_counter() - t)

    # C1
    U = W.sod(32, 0)
    dx = (1.0 / 32,) * 3
    P = O.Params(scheme=O.MHM, recon=O.PLM, riemann=O.ROE, limiter=O.MINMOD, dx=dx)
    p = H.Params(scheme=H.MHM, recon=H.PLM, riemann=H.RS_ROE, limiter=H.LIM_MINMOD, precision=H.FP64, dx=dx)
    c1 = {"oracle_all_cores": oracle_rate(U, P, 2, 1, 10, 0.5), "oracle_1_core": oracle_rate(U, P, 2, 1, 10, 0.5, 1),
          "gpu_fp64": gpu_rate(U, p, H.BC_OUTFLOW, 10, 0.5)}
    c1["gpu_fp64_over_1_core"] = c1["gpu_fp64"] / c1["oracle_1_core"]
    out["c1"] = c1
    # C4 cut
    U = W.sedov(512, gamma=SEDOV_GAMMA, window=64)
    dx = (1.0 / 512,) * 3
    P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.HLLC, limiter=O.MINMOD, gamma=SEDOV_GAMMA, dx=dx,
                 **SEDOV_FLOORS)
    c4 = {"oracle_all_cores": oracle_rate(U, P, 3, 1, 1, 0.4), "oracle_1_core": oracle_rate(U, P, 3, 1, 1, 0.4, 1),
          "gpu_fp64": gpu_rate(U, _sedov_params(H, H.FP64, dx), H.BC_OUTFLOW, 10, 0.4),
          "gpu_fp32_mixed": gpu_rate(U, _sedov_params(H, H.FP32_MIXED, dx), H.BC_OUTFLOW, 10, 0.4)}
    c4["gpu_fp32_mixed_over_1_core"] = c4["gpu_fp32_mixed"] / c4["oracle_1_core"]
    out["c4_cut"] = c4
    if cpu_c2 and gpu_c2:
        out["c2"] = {"oracle_all_cores": cpu_c2["value"], "oracle_1_core": cpu_c2["single_core"]["value"],
                     "gpu_fp32": gpu_c2, "gpu_fp32_over_1_core": gpu_c2 / cpu_c2["single_core"]["value"]}
    out["cores"] = O.max_threads()
    out["unit"] = UNIT
    return out


SEDOV_GAMMA = 5.0 / 3.0
SEDOV_FLOORS = dict(dens_floor=1e-12, pres_floor=1e-12)
XI0 = 1.15


def _sedov_params(H, prec, dx, dt_dev=None):
    return H.Params(scheme=H.CTU, recon=H.PPM, riemann=H.RS_HLLC, limiter=H.LIM_MINMOD, precision=prec,
                    gamma=SEDOV_GAMMA, dx=dx, dt_dev=dt_dev, **SEDOV_FLOORS)


def _box_rel_l1(a, b):
    a = a.reshape(5, -1)
    b = b.reshape(5, -1)
    out = []
    for v in range(5):
        den = np.abs(b[v]).sum()
        if den < 1e-9 * np.abs(b[0]).sum():
            den = np.abs(b[0]).sum()
        out.append(float(np.abs(a[v] - b[v]).sum() / den))
    return max(out)


def sedov_long_study(n=512, sub=288, radii=(0.05, 0.10, 0.15, 0.20, 0.25), cfl=0.4):
    """Precision study (--study sedov_long; about half an hour on one GB300,
    not part of the default run): the Sedov-Taylor blast of the precision
    test carried to a blast radius of 0.25 box lengths, the FP32-mixed form
    on the whole n^3 box against the FP64 path (which equals the oracle bit
    for bit in every parity test).

    The FP64 reference runs on the central sub^3 sub-box with outflow edges.
    While the blast stays inside it this is the same problem: outside the
    blast the state is uniform, a uniform state is exactly steady in every
    scheme, and an outflow edge of a uniform state is uniform.  Both sides of
    that claim are checked at every report: the mixed run's field outside the
    sub-box and the FP64 run's outermost layer equal the background exactly.
    Both forms take the FP64 run's dt (CFL 0.4 on its state).  Reported at
    Sedov-Taylor radii R = 0.05 ... 0.25 (t from R = xi0 (E t^2/rho)^(1/5),
    xi0 = 1.15): relative L1 per variable (max over variables) of mixed vs
    FP64 on the 64^3 cut around the centre and on the whole sub-box, the blast
    radius from the density maximum along the six axis rays, and the largest
    difference between those six profiles (symmetry).  One JSON line per
    report."""
    import torch
    from paper_1103_3373_gb300 import hydro as H
    from paper_1103_3373_gb300 import workloads as W
    dev = torch.device("cuda:0")
    dx = (1.0 / n,) * 3
    a = n // 2 - sub // 2
    Usub = W.sedov(n, gamma=SEDOV_GAMMA, window=sub)
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
    p64 = _sedov_params(H, H.FP64, dx, dt)
    ws = H.hydro_workspace_bytes(p64)
    p64.workspace = torch.empty(max(ws, 16), dtype=torch.uint8, device=dev)
    pm = _sedov_params(H, H.FP32_MIXED, dx, dt)
    t_targets = [(R / XI0) ** 2.5 for R in radii]  # rho = E = 1
    t, step, k = 0.0, 0, 0
    rows = []
    t0 = time.perf_counter()
    bg64 = torch.tensor(bg, dtype=torch.float64, device=dev)
    bg32 = torch.tensor(bg, dtype=torch.float32, device=dev)
    while k < len(t_targets):
        H.hydro_cfl_dt(f64, dx, cfl, dt, red_ws, gamma=SEDOV_GAMMA, precision=H.FP64, **SEDOV_FLOORS)
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
                   "rel_l1_cut64": _box_rel_l1(got[cut], ref[cut]), "rel_l1_subbox": _box_rel_l1(got, ref),
                   "max_rel_dev_density_cut": float(np.abs(got[0][cut[1:]] - ref[0][cut[1:]]).max() /
                                                   np.abs(ref[0][cut[1:]]).max()),
                   "mixed_outside_subbox_max_dev": out_dev, "fp64_subbox_edge_max_dev": edge_dev,
                   "ray_symmetry_max_diff_fp64": sym, "wall_s": time.perf_counter() - t0}
            rows.append(row)
            print(json.dumps(row), flush=True)
            k += 1
    return rows


def record_traffic(csv_path, command=""):
    """data/ncu_traffic.json from an ncu --csv launch list of advance_kernel
    launches of the benchmark box (DRAM read + write bytes per launch)."""
    import csv
    import io
    txt = open(csv_path).read()
    rows = list(csv.DictReader(io.StringIO(txt[txt.index('"ID"'):])))
    per = {}
    for r in rows:
        if "advance_kernel" not in r.get("Kernel Name", ""):
            continue
        if r["Metric Name"] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            v = float(r["Metric Value"].replace(",", ""))
            unit = r.get("Metric Unit", "byte")
            scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(unit, 1.0)
            per[r["ID"]] = per.get(r["ID"], 0.0) + v * scale
    if not per:
        raise SystemExit("no advance_kernel DRAM metrics in " + csv_path)
    launches = [per[k] for k in sorted(per, key=int)]
    out = {"source_sha": source_hash(),
           "kernel": "advance_kernel<CTU,PPM,ROE,FP32,16>, 256^3 periodic box, fused gather, chained columns",
           "bytes_per_launch": launches, "bytes_per_cell": float(np.mean(launches)) / N_BOX ** 3,
           "command": "python bench.py --steps 20 --warmup 3 --quick --block-threads 512 > plain.log && "
                      "ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum "
                      "--clock-control none -k regex:\"advance_kernel|cfl_\" --csv --log-file launches.csv "
                      "python bench.py --steps 20 --warmup 3 --quick --block-threads 512 && "
                      "python bench.py --record-traffic launches.csv",
           "note": "dram__bytes_read.sum + dram__bytes_write.sum per launch; valid only while source_sha matches "
                   "the headline kernel's sources"}
    with open(os.path.join(ROOT, "paper_1103_3373_gb300", "data", "ncu_traffic.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))
    return 0


def reference_arm(args, rank, world):
    """--impl reference: the oracle (FP64 CPU), as it stands, on the host cores."""
    if rank != 0:
        return 0
    import oracle as O
    from paper_1103_3373_gb300 import workloads as W
    U = W.lognormal(N_BOX, seed=1, mach=1.5)
    dx = (1.0 / N_BOX,) * 3
    Uq = U.astype(np.float32).astype(np.float64)
    dt = O.cfl_dt(Uq, dx, CFL, 1.4, **FLOORS)
    P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, limiter=O.MINMOD, fallback=O.HLLE, gamma=1.4, dt=dt,
                 dx=dx, **FLOORS)
    orig = W.group_origins(N_BOX, N_BOX, N_BOX, 16)
    cores = O.max_threads()
    probe = O.gather(Uq, orig[:cores], 16, 3, bc=0)
    t = time.perf_counter()
    O.advance(P, probe, 16)
    per_group = (time.perf_counter() - t) / cores
    budget = min(10.0, 150.0 / max(1, args.steps + args.warmup))  # whole run within a few minutes
    S = int(max(cores, min(len(orig), budget / max(per_group, 1e-6))))
    S = max(cores, (S // cores) * cores)
    Ug = O.gather(Uq, orig[:S], 16, 3, bc=0)
    for _ in range(args.warmup):
        O.advance(P, Ug, 16)
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        O.advance(P, Ug, 16)
        ts.append(time.perf_counter() - t)
    el = sum(ts)
    value = S * 4096 * args.steps / el
    sample = "each step: one CTU+PPM+Roe FP64 oracle step of the first %d of the 4096 patch groups" % S
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(CONFIG, mach=mach_distribution(U)), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# slab partitions (group layers) the e2e leg chooses from on each box
E2E_PARTITIONS = ("1,2,3,4,3,2,1", "1,1,2,2,2,2,2,2,1,1", "1,1,2,3,4,3,1,1", "2,4,4,4,2")


def slab_arg(s):
    """'8' -> 8 equal slabs; '1,2,2,1' -> group layers per slab."""
    parts = [int(x) for x in str(s).split(",") if x.strip()]
    return parts[0] if len(parts) == 1 else parts


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="skip the FP64 / mixed / VL detail lines")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--e2e-slabs", default="auto",
                    help="z-slabs of the end-to-end pipeline: auto (the fastest of E2E_PARTITIONS on this box), "
                         "a count (1: copy in, step, copy out in series) or group layers per slab, e.g. 1,2,3,4,3,2,1")
    ap.add_argument("--e2e-sweep", default="",
                    help="also time the end-to-end step at these ';'-separated slab settings (e.g. '1;4;8;1,2,2,1')")
    ap.add_argument("--quick", action="store_true", help="main line only (no extra, cpu_baseline or e2e legs)")
    ap.add_argument("--legs", default="all",
                    help="comma list of extra legs to run: precisions, schemes, amr_levels, amr_hierarchy, "
                         "serving (default all)")
    ap.add_argument("--record-traffic", default="",
                    help="write the headline kernel's DRAM bytes per launch from this ncu CSV (the launch-list "
                         "capture with dram__bytes_read.sum and dram__bytes_write.sum) to data/ncu_traffic.json, "
                         "stamped with the hash of the kernel's sources, and exit")
    ap.add_argument("--study", default="", choices=["", "sedov_long"],
                    help="run only this long study instead of the benchmark (sedov_long: the Sedov blast to "
                         "R = 0.25, mixed vs FP64, about half an hour)")
    ap.add_argument("--block-threads", type=int, default=0,
                    help="use this many threads per CTA (capped per kernel) instead of autotuning")
    ap.add_argument("--chain", type=int, default=-1,
                    help="with --block-threads: chain length / z-segment of the work order (0 = whole columns)")
    args = ap.parse_args()
    if args.quick:
        args.no_extra = args.no_cpu = True
    from paper_1103_3373_gb300 import replicas
    rank, world, local = replicas.rank_info()
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.record_traffic:
        return record_traffic(args.record_traffic)
    if args.study == "sedov_long":
        from paper_1103_3373_gb300 import build as hb
        hb.build()
        sedov_long_study()
        return 0

    import torch
    from paper_1103_3373_gb300 import build as hb
    if rank == 0 and world == 1:
        hb.build()
    from paper_1103_3373_gb300 import hydro as H
    from paper_1103_3373_gb300 import runtime as RT
    from paper_1103_3373_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.warmup < 3:
        args.warmup = 3

    U = W.lognormal(N_BOX, seed=1, mach=1.5)
    dx = (1.0 / N_BOX,) * 3
    cells = N_BOX ** 3
    stream = torch.cuda.Stream(device=dev)
    box = RT.UniformBox(U, make_params(H, H.FP32, dx), cfl=CFL, device=dev, stream=stream)
    if args.block_threads:
        box.p.block_threads = args.block_threads
        box.p.chain = max(0, args.chain)
        tuned = {"block_threads": args.block_threads, "grid_ctas": 0, "chain": box.p.chain, "fixed": True}
    else:
        tuned = box.tune()
    box.compute_dt()
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms, adv_ms, total_ms, clocks = time_box(box, args.steps, args.warmup, torch, sampler)
    # every rank advanced its own box (replicas): whole-job rate over the
    # slowest rank's time
    value, total_ms, _ = replicas.job_rate(total_ms, cells * args.steps, dist, device=dev)
    st = box.status.cpu().numpy()
    finite = bool(torch.isfinite(box.state()).all().item())

    # roofline of the dominant kernel (the fused CTU group update), against
    # the FP32 FMA rate measured on this GPU (include/hydro_peaks.h): the
    # larger of the scalar and packed-pair forms
    with open(os.path.join(ROOT, "paper_1103_3373_gb300", "data", "flops_per_cell.json")) as fh:
        flops_cell = json.load(fh)["entries"]["ctu-ppm-roe"]["flops"]
    props = torch.cuda.get_device_properties(dev)
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    alu = alu_peaks(H, torch, dev, local)
    fp32_form = "fp32x2" if alu["fp32x2"]["tflops"] > alu["fp32"]["tflops"] else "fp32"
    peak = alu[fp32_form]["tflops"]
    peak_fp64 = alu["fp64"]["tflops"]
    achieved = flops_cell * cells / (adv_ms / 1e3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "paper_1103_3373_gb300", "data", "ncu_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as fh:
            tj = json.load(fh)
        if tj.get("source_sha") == source_hash():
            traffic = tj["bytes_per_cell"] * cells
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "advance_kernel<CTU,PPM,ROE,FP32,16> (fused gather)",
                "flops_per_cell": flops_cell, "kernel_ms": adv_ms,
                "peak_note": "measured on this GPU: FP32 FMA loop (%s form, %.0f MHz median SM clock), "
                             "include/hydro_peaks.h; nominal %d SMs x 128 lanes x 2 x %.0f MHz = %.1f"
                             % (fp32_form, alu[fp32_form]["sm_mhz"] or 0, props.multi_processor_count, sm_max,
                                sm_peak_fp32_tflops(props.multi_processor_count, sm_max)),
                "alu_peaks": alu,
                "hbm_frac_of_measured": (40.0 * cells + 30.0 * 4 * 256 * 4096) / (adv_ms / 1e3) / 1e9 /
                                        peaks.get("hbm_gbs", 6775.3)}

    # end to end through host buffers (pinned), same metric: the slab
    # pipeline (copies overlapped with the solver, Sec. 4.1), and the serial
    # form (copy in, step, copy out) for context
    e2e = None
    if not args.quick:
        def e2e_run(slabs):
            hs = RT.HostBoxStepper(U, make_params(H, H.FP32, dx), cfl=CFL, device=dev, slabs=slabs)
            ke = max(5, min(args.steps, 50))
            for _ in range(3):
                hs.step()
            torch.cuda.synchronize()
            # events on the stream the steps are issued on (each step's last
            # operation makes it wait for the pipeline's streams)
            st = hs.box.stream
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(ke + 1)]
            evs[0].record(st)
            for k in range(ke):
                hs.step()
                evs[k + 1].record(st)
            torch.cuda.synchronize()
            e_ms = evs[0].elapsed_time(evs[ke])
            per = [evs[k].elapsed_time(evs[k + 1]) for k in range(ke)]
            out = {"value": world * cells * ke / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": hs.h2d_bytes,
                   "d2h_bytes_per_step": hs.d2h_bytes, "steps": ke, "ms_per_step": e_ms / ke,
                   "p50_step_ms": RT.percentile(per, 50), "p99_step_ms": RT.percentile(per, 99),
                   "slabs": hs.slabs, "layers": hs.layers}
            del hs
            return out
        if args.e2e_slabs == "auto":
            # the slab partition that suits this machine's host link: a few
            # candidates timed over a few steps each, the fastest kept
            trials = []
            for S in E2E_PARTITIONS:
                hs = RT.HostBoxStepper(U, make_params(H, H.FP32, dx), cfl=CFL, device=dev, slabs=slab_arg(S))
                for _ in range(2):
                    hs.step()
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(hs.box.stream)
                for _ in range(5):
                    hs.step()
                b.record(hs.box.stream)
                torch.cuda.synchronize()
                trials.append((a.elapsed_time(b) / 5, S))
                del hs
            best = min(trials)[1]
            e2e = e2e_run(slab_arg(best))
            e2e["partition_trials_ms"] = {S: round(t, 3) for t, S in trials}
        else:
            e2e = e2e_run(slab_arg(args.e2e_slabs))
        if e2e["slabs"] > 1:
            s = e2e_run(1)
            e2e["serial"] = {"value": s["value"], "ms_per_step": s["ms_per_step"]}
        if args.e2e_sweep:
            e2e["sweep"] = []
            for S in args.e2e_sweep.split(";"):
                s = e2e_run(slab_arg(S))
                e2e["sweep"].append({"slabs": s["slabs"], "layers": s["layers"], "value": s["value"],
                                     "ms_per_step": s["ms_per_step"]})

    extra = {}
    legs = set(args.legs.split(",")) if args.legs != "all" else {"precisions", "schemes", "amr_levels",
                                                                  "amr_hierarchy", "serving"}
    if not args.no_extra and rank == 0:
        del box
        torch.cuda.empty_cache()
        with open(os.path.join(ROOT, "paper_1103_3373_gb300", "data", "flops_per_cell.json")) as fh:
            flops_tab = json.load(fh)["entries"]

        def leg_roofline(key, kernel_ms, pk, note):
            a = flops_tab[key]["flops"] * cells / (kernel_ms / 1e3) / 1e12
            return {"flops_per_cell": flops_tab[key]["flops"], "achieved_tflops": a, "peak_tflops": pk,
                    "frac": a / pk, "peak_note": note}

        fp32_note = "measured FP32 FMA rate (as the main line)"
        for name, prec, k in (("fp64", H.FP64, 16), ("mixed", H.FP32_MIXED, 50)) if "precisions" in legs else ():
            bx = RT.UniformBox(U, make_params(H, prec, dx), cfl=CFL, device=dev, stream=stream)
            tb = bx.tune() if prec != H.FP64 else None
            bx.compute_dt()
            sm, am, tm, _ = time_box(bx, k, 3, torch)
            extra[name] = {"value": cells * k / (tm / 1e3), "unit": UNIT, "ms_per_step": tm / k,
                           "kernel_ms": am, "steps": k,
                           "block_threads": tb["block_threads"] if tb else bx.p.block_threads,
                           "roofline": leg_roofline("ctu-ppm-roe", am, peak_fp64 if prec == H.FP64 else peak,
                                                    "measured FP64 FMA rate of this GPU" if prec == H.FP64
                                                    else fp32_note)}
            del bx
            torch.cuda.empty_cache()
        for tag, sch, rec, rs, ch, fkey in (("vl_plm_hllc_fp32", H.VL, H.PLM, H.RS_HLLC, 0, "vl-plm-hllc"),
                                            ("mhm_ppm_roe_fp32", H.MHM, H.PPM, H.RS_ROE, 0, "mhm-ppm-roe"),
                                            ("ctu_ppm_roe_characteristic_fp32", H.CTU, H.PPM, H.RS_ROE, 1,
                                             "ctu-ppm-roe-char"),
                                            ("rtvd_fp32", H.RTVD, H.PLM, H.RS_HLLC, 0, "rtvd"),
                                            ("waf_hllc_fp32", H.WAF, H.PLM, H.RS_HLLC, 0, "waf")) \
                if "schemes" in legs else ():
            p = make_params(H, H.FP32, dx)
            p.scheme, p.recon, p.riemann, p.characteristic = sch, rec, rs, ch
            bx = RT.UniformBox(U, p, cfl=CFL, device=dev, stream=stream)
            if args.block_threads:
                # a fixed launch shape (profiling): no tuning launches
                bx.p.block_threads = min(args.block_threads, H.hydro_max_block_threads(bx.p))
                bx.p.chain = max(0, args.chain)
                tb = {"block_threads": bx.p.block_threads, "chain": bx.p.chain}
            else:
                tb = bx.tune()
            bx.compute_dt()
            sm, am, tm, _ = time_box(bx, 50, 3, torch)
            extra[tag] = {"value": cells * 50 / (tm / 1e3), "unit": UNIT, "ms_per_step": tm / 50,
                          "kernel_ms": am, "block_threads": tb["block_threads"], "chain": tb.get("chain", 0),
                          "roofline": leg_roofline(fkey, am, peak, fp32_note)}
            del bx
        torch.cuda.empty_cache()
        if "amr_levels" in legs:
            extra["amr_levels"] = amr_leg(H, RT, W, torch, dev, block_threads=args.block_threads)
        if "amr_hierarchy" in legs:
            extra["amr_hierarchy"] = amr_hierarchy_leg(H, RT, W, torch, dev)
        torch.cuda.empty_cache()
        if "serving" in legs:
            extra["serving"] = serving_leg(H, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(U, dx)
        if not args.no_extra:
            extra["oracle_configs"] = oracle_configs(H, RT, W, torch, dev, cpu, value)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(CONFIG, mach=mach_distribution(U)),
                "parallelism": "replicas%d" % world if world > 1 else "single GPU",
                "p50_step_ms": RT.percentile(step_ms, 50), "p99_step_ms": RT.percentile(step_ms, 99),
                "step_latency_samples": len(step_ms),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": 3 * args.steps,
                "autotuned": {"block_threads": tuned["block_threads"], "grid_ctas": tuned["grid_ctas"],
                              "chain": tuned.get("chain", 0)},
                "status_error_groups": int(np.count_nonzero(st & H.ST_ERROR_MASK)),
                "state_finite": finite, "extra": extra,
                "paper_context": "3.0e7 cell-updates/s, CTU+PPM+Roe FP32 on one Tesla C2050 incl. transfers "
                                 "(Sec. 3.2); other hardware, not a target"}
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
