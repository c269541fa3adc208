"""Serving form: continuous batching of independent simulations.

Requests (independent periodic boxes of different sizes, each with its own
step count) arrive over time.  The engine keeps every admitted box's state
resident on the device and, at every tick, advances ALL active boxes by one
step with one persistent launch (hydro_advance_levels, one entry per box with
its own dx and device dt; chunks of HYDRO_MAX_LEVELS boxes), then reduces
every box's next dt in one pass (hydro_cfl_dt_boxes, chunks of
HYDRO_CFL_MAX_BOXES boxes).  Requests that arrive while others are running
are admitted at the next tick (FIFO) as soon as two budgets allow: device
memory (HBM) and the cells advanced per tick.  The second bounds the length
of a tick, so the step latency of every request in the batch stays bounded
under overload while the GPU still gets tens of millions of cell updates per
launch; new work joins the batch in flight instead of waiting for it to
drain, and finished boxes leave the batch and return their memory.

A box's result does not depend on what else is in the batch: every group is
computed by one CTA from its own box's data only, with its own dt.

Initial states: seeded periodic lognormal boxes (workloads.lognormal) made
once per size at rms Mach 1 and, per request, rolled by a seeded periodic
shift with velocities scaled to the request's Mach number.
"""
import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import hydro as H
from . import workloads as W


@dataclass
class Request:
    rid: int
    t_arrive: float
    n: int
    mach: float
    steps: int
    seed: int
    # filled by the engine
    t_admit: float = float("nan")
    t_done: float = float("nan")
    tick_admit: int = -1
    tick_done: int = -1
    steps_done: int = 0
    result: object = None


@dataclass
class _Active:
    req: Request
    a: object
    b: object
    dt: object
    status: object
    bytes: int
    dx: tuple


class BaseStates:
    """Per box size, the Mach-1 lognormal base state split into the pieces a
    request rescales (density, momentum, internal and kinetic energy)."""

    def __init__(self, sizes, device, dtype, gamma=1.4, seed=101):
        import torch
        self.torch = torch
        self.gamma = gamma
        self.base = {}
        for k, n in enumerate(sorted(set(sizes))):
            U = W.lognormal(n, seed=seed + k, mach=1.0, gamma=gamma)
            kin = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
            t = lambda a: torch.as_tensor(a, dtype=torch.float64).to(device)
            self.base[n] = (t(U[0]), t(U[1:4]), t(U[4] - kin), t(kin))
        self.dtype = dtype

    def make(self, n, mach, seed):
        torch = self.torch
        rho, m, eint, kin = self.base[n]
        rng = np.random.default_rng(seed)
        sh = tuple(int(s) for s in rng.integers(0, n, 3))
        U = torch.empty((5, n, n, n), dtype=torch.float64, device=rho.device)
        U[0] = rho
        U[1:4] = mach * m
        U[4] = eint + (mach * mach) * kin
        return torch.roll(U, shifts=sh, dims=(1, 2, 3)).to(self.dtype).contiguous()


class ServingEngine:
    def __init__(self, params: H.Params, sizes=(32, 64, 128, 256), budget_bytes=None, cfl=0.4, device="cuda:0",
                 keep_results=False, max_inflight=2, max_cells_per_tick=1 << 26):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.p = params
        self.cfl = cfl
        self.dtype = torch.float64 if params.precision == H.FP64 else torch.float32
        self.esize = 8 if params.precision == H.FP64 else 4
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            budget_bytes = int(0.5 * free)
        self.budget = budget_bytes
        self.used = 0
        # cells advanced per tick (a box larger than this still runs, alone)
        self.max_cells = int(max_cells_per_tick)
        self.active_cells = 0
        self.queue = collections.deque()
        self.active = []
        self.done = []
        self.keep_results = keep_results
        self.states = BaseStates(sizes, self.dev, self.dtype, gamma=params.gamma)
        self.red_ws = torch.empty(max(H.hydro_cfl_workspace_bytes(), H.hydro_cfl_boxes_workspace_bytes()),
                                  dtype=torch.uint8, device=self.dev)
        nws = H.hydro_workspace_bytes(params)
        self.p.workspace = torch.empty(nws, dtype=torch.uint8, device=self.dev) if nws else None
        self.stream = torch.cuda.Stream(device=self.dev)
        self.tick_events = []   # (start, end, cells) per tick
        self.max_inflight = max_inflight
        self.ticks = 0
        self.cell_updates = 0

    def footprint(self, n):
        return 2 * 5 * n ** 3 * self.esize + (n // 16) ** 3 * 4 + 8

    def submit(self, req: Request):
        self.queue.append(req)

    def _admit(self, now):
        torch = self.torch
        while self.queue and self.queue[0].t_arrive <= now:
            req = self.queue[0]
            need = self.footprint(req.n)
            if self.active and (self.used + need > self.budget or self.active_cells + req.n ** 3 > self.max_cells):
                break  # FIFO: wait until memory and tick capacity free up
            self.queue.popleft()
            with torch.cuda.stream(self.stream):
                a = self.states.make(req.n, req.mach, req.seed)
                b = torch.empty_like(a)
                dt = torch.zeros(1, dtype=torch.float64, device=self.dev)
                st = torch.zeros((req.n // 16) ** 3, dtype=torch.int32, device=self.dev)
            box = _Active(req, a, b, dt, st, need, (1.0 / req.n,) * 3)
            H.hydro_cfl_dt(a, box.dx, self.cfl, dt, self.red_ws, gamma=self.p.gamma, dens_floor=self.p.dens_floor,
                           pres_floor=self.p.pres_floor, precision=self.p.precision, stream=self.stream)
            req.t_admit = now
            req.tick_admit = self.ticks
            self.used += need
            self.active_cells += req.n ** 3
            self.active.append(box)

    def _tick(self):
        torch = self.torch
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        cells = 0
        for k in range(0, len(self.active), H.MAX_LEVELS):
            chunk = self.active[k:k + H.MAX_LEVELS]
            levels = [H.Level(U_in=bx.a, U_out=bx.b, status=bx.status, dt_dev=bx.dt, dx=bx.dx, mode=1,
                              bc=H.BC_PERIODIC) for bx in chunk]
            H.hydro_advance_levels(self.p, levels, stream=self.stream)
            cells += sum(bx.req.n ** 3 for bx in chunk)
        for bx in self.active:
            bx.a, bx.b = bx.b, bx.a
            bx.req.steps_done += 1
        for k in range(0, len(self.active), H.CFL_MAX_BOXES):
            chunk = self.active[k:k + H.CFL_MAX_BOXES]
            H.hydro_cfl_dt_boxes([(bx.a, bx.dx, bx.dt) for bx in chunk], self.cfl, self.red_ws, gamma=self.p.gamma,
                                 dens_floor=self.p.dens_floor, pres_floor=self.p.pres_floor,
                                 precision=self.p.precision, stream=self.stream)
        e1.record(self.stream)
        self.tick_events.append((e0, e1, cells, len(self.active)))
        self.cell_updates += cells
        self.ticks += 1
        # bound the ticks in flight, then retire finished requests
        if len(self.tick_events) > self.max_inflight:
            self.tick_events[-1 - self.max_inflight][1].synchronize()
        still = []
        for bx in self.active:
            if bx.req.steps_done >= bx.req.steps:
                e1.synchronize()
                bx.req.t_done = time.perf_counter()
                if self.keep_results:
                    bx.req.result = bx.a.detach().to("cpu")
                self.used -= bx.bytes
                self.active_cells -= bx.req.n ** 3
                bx.req.tick_done = self.ticks
                self.done.append(bx.req)
            else:
                still.append(bx)
        self.active = still

    def run(self, requests, realtime=True, t0=None, clock="wall"):
        """Serve `requests` (sorted by arrival).  clock="wall": with realtime
        the arrival times are wall-clock offsets from the start, otherwise
        all requests are present at t = 0.  clock="ticks": t_arrive is the
        tick at whose start the request becomes admissible (deterministic:
        the batch a request joins does not depend on timing).  Returns the
        summary dict."""
        ticks = clock == "ticks"
        for r in sorted(requests, key=lambda r: r.t_arrive):
            if not realtime and not ticks:
                r.t_arrive = 0.0
            self.submit(r)
        start = time.perf_counter() if t0 is None else t0
        if not ticks:
            for r in self.queue:
                r.t_arrive += start
        while self.queue or self.active:
            now = float(self.ticks) if ticks else time.perf_counter()
            self._admit(now)
            if self.active:
                self._tick()
            elif ticks:
                self.ticks += 1  # idle tick: nothing admissible yet
            else:
                nxt = self.queue[0].t_arrive
                time.sleep(max(0.0, min(0.01, nxt - time.perf_counter())))
        self.torch.cuda.synchronize()
        wall = time.perf_counter() - start
        tick_ms = [a.elapsed_time(b) for a, b, _, _ in self.tick_events]
        turn = [r.t_done - r.t_arrive for r in self.done] if not ticks else []
        wait = [r.t_admit - r.t_arrive for r in self.done] if not ticks else []
        gpu_s = sum(tick_ms) / 1e3
        return {"requests": len(self.done), "ticks": self.ticks, "cell_updates": self.cell_updates,
                "wall_s": wall, "cell_updates_per_s_wall": self.cell_updates / wall,
                "cell_updates_per_s_gpu": self.cell_updates / gpu_s if gpu_s else float("nan"),
                "p50_step_ms": float(np.percentile(tick_ms, 50)) if tick_ms else None,
                "p99_step_ms": float(np.percentile(tick_ms, 99)) if tick_ms else None,
                "p50_turnaround_s": float(np.percentile(turn, 50)) if turn else None,
                "p99_turnaround_s": float(np.percentile(turn, 99)) if turn else None,
                "p99_queue_wait_s": float(np.percentile(wait, 99)) if wait else None,
                "max_active": max((n for _, _, _, n in self.tick_events), default=0),
                "max_cells_in_a_tick": max((c for _, _, c, _ in self.tick_events), default=0),
                "budget_bytes": self.budget, "max_cells_per_tick": self.max_cells}


def requests_from_arrivals(arrivals):
    return [Request(rid=i, t_arrive=a["t"], n=a["n"], mach=a["mach"], steps=a["steps"], seed=a["seed"])
            for i, a in enumerate(arrivals)]
