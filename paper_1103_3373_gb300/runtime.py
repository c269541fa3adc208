"""Drivers on top of the C ABI: a device-resident uniform-box simulation (the
benchmarked step), its end-to-end form with host buffers, CUDA-graph capture
of a step, and helpers shared by the batched / serving forms.

Every numerical step runs in libhydro's kernels; this module only owns device
buffers (through PyTorch) and orders the calls on a stream.
"""
import numpy as np

from . import hydro as H


def _torch():
    import torch
    return torch


class UniformBox:
    """A periodic / outflow box [5,Z,Y,X] advanced by hydro_advance_uniform
    (ghost gather fused, Sec. 4.2), with the boundary fluxes of every group
    stored (Sec. 2 step (5)) and the next dt reduced on the device (Sec. 4.3).

    One step = advance (reads dt from the device) + CFL reduction of the new
    state into that same device dt.  No host synchronisation inside a step.
    """

    def __init__(self, U0, params: H.Params, cfl=0.4, bc=H.BC_PERIODIC, N=16, store_flux=True, device="cuda:0",
                 stream=None):
        torch = _torch()
        self.torch = torch
        self.dev = torch.device(device)
        self.p = params
        self.cfl = cfl
        self.bc = bc
        self.N = N
        self.dtype = torch.float64 if params.precision == H.FP64 else torch.float32
        _, Z, Y, X = U0.shape
        self.shape = (5, Z, Y, X)
        self.cells = X * Y * Z
        self.G = (X // N) * (Y // N) * (Z // N)
        self.a = torch.as_tensor(U0, dtype=self.dtype).to(self.dev).contiguous()
        self.b = torch.empty_like(self.a)
        self.flux = torch.empty((self.G, 6, 5, N, N), dtype=self.dtype, device=self.dev) if store_flux else None
        self.status = torch.zeros(self.G, dtype=torch.int32, device=self.dev)
        self.dt = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.red_ws = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=self.dev)
        self.p.dt_dev = self.dt
        nws = H.hydro_workspace_bytes(self.p, N)
        self.p.workspace = torch.empty(nws, dtype=torch.uint8, device=self.dev) if nws else None
        self.stream = stream
        self.compute_dt()

    def compute_dt(self, stream=None):
        H.hydro_cfl_dt(self.a, self.p.dx, self.cfl, self.dt, self.red_ws, gamma=self.p.gamma,
                       dens_floor=self.p.dens_floor, pres_floor=self.p.pres_floor, precision=self.p.precision,
                       stream=stream if stream is not None else self.stream)

    def advance(self, stream=None):
        """The fused patch-group update only (one kernel)."""
        H.hydro_advance_uniform(self.p, self.a, self.b, bc=self.bc, flux=self.flux, status=self.status, N=self.N,
                                stream=stream if stream is not None else self.stream)

    def swap(self):
        self.a, self.b = self.b, self.a

    def end_step(self):
        """Host-side bookkeeping after a step: the split schemes alternate
        their sweep order (Strang)."""
        if self.p.scheme >= H.RTVD:
            self.p.split_order ^= 1

    def step(self, stream=None):
        self.advance(stream)
        self.swap()
        self.compute_dt(stream)
        self.end_step()

    def state(self):
        return self.a

    def tune(self, verbose=False):
        """Autotune the launch shape of this box's step on its own data."""
        from . import autotune
        torch = self.torch
        torch.cuda.synchronize()
        best = autotune.tune(self.p, lambda p: H.hydro_advance_uniform(p, self.a, self.b, bc=self.bc, flux=self.flux,
                                                                       status=self.status, N=self.N, stream=None),
                             tag="uniform", verbose=verbose)
        nws = H.hydro_workspace_bytes(self.p, self.N)
        self.p.workspace = torch.empty(nws, dtype=torch.uint8, device=self.dev) if nws else None
        return best


def rotation(n):
    """Device fields (indices into three) of end-to-end step n: input
    D[2n % 3], output D[(2n+1) % 3].  Step n+1's input is then neither of
    step n's fields and its output is not step n's output, the condition for
    chaining the two steps (include/hydro_pipeline.h)."""
    return (2 * n) % 3, (2 * n + 1) % 3


class HostBoxStepper:
    """End-to-end form of UniformBox.step for a caller that keeps its data on
    the host: each step copies the state in from pinned host memory, runs the
    step on the device and copies the new state and dt back (the paper times
    its GPU solver the same way, Sec. 3.2).  The step is one native call
    (hydro_pipeline_step).

    slabs = 1: copy in, advance, copy out, one after the other.
    slabs = S > 1 (S equal slabs) or a list of group-layer counts per slab:
    the asynchronous-copy scheme of Sec. 4.1 on z-slabs of group layers (a
    copy-in stream, two compute streams alternating slabs, a copy-out stream;
    see include/hydro_pipeline.h); consecutive steps overlap (the copy-in of
    one starts while the last finishes) on three device fields in rotation.
    The result equals UniformBox.step bit for bit.
    """

    def __init__(self, U0, params: H.Params, cfl=0.4, bc=H.BC_PERIODIC, N=16, device="cuda:0", slabs=1):
        torch = _torch()
        self.torch = torch
        self.box = UniformBox(U0, params, cfl=cfl, bc=bc, N=N, device=device)
        b = self.box
        self.host_in = torch.empty(b.shape, dtype=b.dtype).pin_memory()
        self.host_in.copy_(torch.as_tensor(U0, dtype=b.dtype))
        self.host_out = torch.empty_like(self.host_in).pin_memory()
        self.host_dt = torch.zeros(1, dtype=torch.float64).pin_memory()
        self.h2d_bytes = self.host_in.numel() * self.host_in.element_size()
        self.d2h_bytes = self.h2d_bytes + 8
        _, Z, Y, X = b.shape
        GZ = Z // N
        if not isinstance(slabs, (list, tuple)):
            slabs = max(1, min(int(slabs), GZ))
        ghost = H.hydro_required_ghost(params.scheme, params.recon)
        with torch.cuda.device(b.dev):
            self.pipe = H.Pipeline(X, Y, Z, ghost, bc=bc, slabs=slabs, N=N)
        self.slabs = self.pipe.nslab
        self.layers = list(slabs) if isinstance(slabs, (list, tuple)) else \
            [(s + 1) * GZ // slabs - s * GZ // slabs for s in range(slabs)]
        nws = H.hydro_workspace_bytes(b.p, N)
        self.ws2 = torch.empty(nws, dtype=torch.uint8, device=b.dev) if nws else None
        self.red_ws = torch.empty(self.pipe.workspace_bytes, dtype=torch.uint8, device=b.dev)
        # three device fields in rotation (in = D[2n % 3], out = D[(2n+1) % 3]):
        # consecutive steps then chain, the copy-in of one overlapping the
        # end of the last (include/hydro_pipeline.h)
        self.dev_fields = [b.a, b.b, torch.empty_like(b.a)]
        self.n = 0

    def step(self):
        b = self.box
        i, o = rotation(self.n)
        din, dout = self.dev_fields[i], self.dev_fields[o]
        self.pipe.step(b.p, self.host_in, self.host_out, din, dout, b.cfl, self.red_ws, host_dt=self.host_dt,
                       flux=b.flux, status=b.status, ws2=self.ws2, stream=b.stream)
        b.a, b.b = dout, din
        self.n += 1
        b.end_step()
        # the next step starts from the state just returned
        self.host_in, self.host_out = self.host_out, self.host_in


def capture_graph(fn, stream=None, warmup=1):
    """Capture fn() (a sequence of C-ABI launches) into a CUDA graph."""
    torch = _torch()
    s = stream or torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(warmup):
            fn()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn()
    return g


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")


class LevelBatch:
    """Uneven per-AMR-level lists of halo-prepared groups advanced by ONE
    persistent launch (hydro_advance_levels), each level with its own dx and
    its own device dt from its own CFL reduction over the interior cells of
    its groups (Sec. 4.3 per level).

    step() = one CFL reduction per level + the batched launch; it takes no
    host synchronisation and can be captured once into a CUDA graph
    (capture()) and replayed.  step_per_level() is the plain form: one
    hydro_advance launch per level.  A level dict may carry `zrun` (runs of
    groups that continue one another along z, hydro_params.zrun): both forms
    then stream through those runs (chains=False ignores them).
    """

    def __init__(self, levels, params: H.Params, cfl=0.4, N=16, ghost=3, device="cuda:0", stream=None,
                 store_flux=True, chains=True):
        torch = _torch()
        self.torch = torch
        self.dev = torch.device(device)
        self.p = params
        self.cfl = cfl
        self.N, self.ghost = N, ghost
        dt = torch.float64 if params.precision == H.FP64 else torch.float32
        self.U_in, self.U_out, self.flux, self.status, self.dts, self.dx = [], [], [], [], [], []
        self.zrun = []
        for lv in levels:
            zr = lv.get("zrun") if chains else None
            self.zrun.append(torch.as_tensor(np.asarray(zr, dtype=np.int32)).to(self.dev) if zr is not None else None)
            U = torch.as_tensor(lv["U"], dtype=dt).to(self.dev).contiguous()
            G = U.shape[0]
            self.U_in.append(U)
            self.U_out.append(torch.empty((G, 5, N, N, N), dtype=dt, device=self.dev))
            self.flux.append(torch.empty((G, 6, 5, N, N), dtype=dt, device=self.dev) if store_flux else None)
            self.status.append(torch.zeros(G, dtype=torch.int32, device=self.dev))
            self.dts.append(torch.zeros(1, dtype=torch.float64, device=self.dev))
            self.dx.append((lv["dx"],) * 3)
        self.cells = sum(u.shape[0] for u in self.U_in) * N ** 3
        # autotuner cache tag: chain lengths are candidates only with runs
        self.tune_tag = "levels_runs" if any(z is not None for z in self.zrun) else "levels"
        self.red_ws = torch.empty(H.hydro_cfl_boxes_workspace_bytes(), dtype=torch.uint8, device=self.dev)
        # each level's dt from its groups' interior cells (the ghosts belong
        # to other groups or are interpolated from the coarser level)
        self.cfl_boxes = H.make_cfl_boxes([(self.U_in[l], self.dx[l], self.dts[l], 1.0, None, ghost)
                                           for l in range(len(self.U_in))], params.precision)
        self.stream = stream
        self._alloc_ws()
        self.graph = None

    def _alloc_ws(self):
        nws = H.hydro_workspace_bytes(self.p, self.N)
        self.p.workspace = self.torch.empty(nws, dtype=self.torch.uint8, device=self.dev) if nws else None
        self.entries = [H.Level(U_in=self.U_in[l], U_out=self.U_out[l], flux=self.flux[l], status=self.status[l],
                                dx=self.dx[l], dt_dev=self.dts[l], mode=0, zrun=self.zrun[l])
                        for l in range(len(self.U_in))]
        self.carray = H.make_levels(self.entries, self.p.precision)

    def reduce_dt(self, stream=None):
        """Every level's dt in one device pass (hydro_cfl_dt_boxes)."""
        s = stream if stream is not None else self.stream
        H.hydro_cfl_dt_boxes(None, self.cfl, self.red_ws, gamma=self.p.gamma, dens_floor=self.p.dens_floor,
                             pres_floor=self.p.pres_floor, precision=self.p.precision, stream=s, _carray=self.cfl_boxes)

    def advance_batched(self, stream=None):
        s = stream if stream is not None else self.stream
        H.hydro_advance_levels(self.p, self.entries, N=self.N, ghost=self.ghost, stream=s, _carray=self.carray)

    def step(self, stream=None):
        self.reduce_dt(stream)
        self.advance_batched(stream)

    def step_per_level(self, stream=None):
        s = stream if stream is not None else self.stream
        self.reduce_dt(s)
        for l in range(len(self.U_in)):
            self.p.dx, self.p.dt_dev, self.p.zrun = self.dx[l], self.dts[l], self.zrun[l]
            H.hydro_advance(self.p, self.U_in[l], self.U_out[l], self.flux[l], self.status[l], N=self.N,
                            ghost=self.ghost, stream=s)
        self.p.dt_dev, self.p.zrun = None, None

    def tune(self, verbose=False):
        from . import autotune
        self.torch.cuda.synchronize()
        best = autotune.tune(self.p, lambda p: H.hydro_advance_levels(
            p, self.entries, N=self.N, ghost=self.ghost, stream=None,
            _carray=H.make_levels(self.entries, p.precision)), tag=self.tune_tag, verbose=verbose)
        self._alloc_ws()
        return best

    def capture(self):
        """Capture step() into a CUDA graph (replay with replay())."""
        self.graph = capture_graph(lambda: self.step(self.torch.cuda.current_stream()))
        return self.graph

    def replay(self):
        self.graph.replay()


class _NoTimer:
    def __enter__(self):
        return None

    def __exit__(self, *exc):
        return False


def _no_timer(kind):
    return _NoTimer()


def zrun_of(origin, N=16):
    """Runs of z-continuations of a list of group origins (host int [G][3]):
    zrun[g] = 1 + zrun[g+1] when group g+1 lies directly above group g, else
    1 (hydro_params.zrun).  Groups of one level whose ghost zones are filled
    from that level hold each other's interiors, as the runs require."""
    o = np.asarray(origin, dtype=np.int64).reshape(-1, 3)
    z = np.ones(len(o), dtype=np.int32)
    for g in range(len(o) - 2, -1, -1):
        if o[g + 1, 0] == o[g, 0] and o[g + 1, 1] == o[g, 1] and o[g + 1, 2] == o[g, 2] + N:
            z[g] = z[g + 1] + 1
    return z


class AmrHierarchy:
    """A static AMR hierarchy resident on the GPU (level 0 covers the box,
    level l+1 refines whole level-l groups as octets; dx_l = dx_0 / 2^l),
    stepped with adaptive time steps dt_l = dt_0 / 2^l entirely by library
    kernels (include/hydro_amr.h and hydro_advance), recursively per level:

      prepare  ghost zones of every group of level l: copies from level l,
               else interpolation from level l-1 in space and in time
               (theta = 0 for the first substep, 1/2 for the second; Sec. 4.2)
      advance  hydro_advance of the level's groups, boundary fluxes stored
               (Sec. 2 steps (1)-(5))
      finer    level l+1 twice with dt_l / 2
      reflux   coarse cells next to level l+1 take its fluxes (Sec. 4.3)
      restrict coarse cells under level l+1 take the mean of its cells

    No host synchronisation inside step(), so a step can be captured into a
    CUDA graph (capture()/replay()).  `levels` is a list of dicts {U
    [G][5][N][N][N], origin [G][3], box, dx} (workloads.amr_hierarchy).
    Groups of a level listed in runs of z-neighbours (zrun_of) are advanced
    as chains (chains=False: every group alone).
    """

    def __init__(self, levels, params: H.Params, bc=H.BC_PERIODIC, N=16, device="cuda:0", stream=None,
                 chains=True):
        import dataclasses
        torch = _torch()
        self.torch = torch
        self.dev = torch.device(device)
        self.bc, self.N, self.stream = bc, N, stream
        self.prec = params.precision
        dt = torch.float64 if self.prec == H.FP64 else torch.float32
        self.ghost = H.hydro_required_ghost(params.scheme, params.recon)
        M = N + 2 * self.ghost
        self.L = len(levels)
        self.err = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.origin, self.map, self.box, self.cur, self.new, self.Ug, self.flux, self.status = ([] for _ in range(8))
        self.params = []
        for l, lv in enumerate(levels):
            G = len(lv["origin"])
            X, Y, Z = lv["box"]
            self.box.append((X, Y, Z))
            self.origin.append(torch.as_tensor(np.asarray(lv["origin"], dtype=np.int32)).to(self.dev).contiguous())
            m = torch.empty((Z // N, Y // N, X // N), dtype=torch.int32, device=self.dev)
            H.hydro_amr_map(self.origin[l], (X, Y, Z), m, N=N, error=self.err, stream=stream)
            self.map.append(m)
            self.cur.append(torch.as_tensor(lv["U"], dtype=dt).to(self.dev).contiguous())
            self.new.append(torch.empty_like(self.cur[l]))
            self.Ug.append(torch.empty((G, 5, M, M, M), dtype=dt, device=self.dev))
            nsub = 1 if l == 0 else 2
            self.flux.append([torch.empty((G, 6, 5, N, N), dtype=dt, device=self.dev) for _ in range(nsub)])
            self.status.append(torch.zeros(G, dtype=torch.int32, device=self.dev))
            p = dataclasses.replace(params)
            p.dx = tuple(float(a) for a in lv["dx"])
            p.dt_dev = None
            zr = zrun_of(lv["origin"], N)
            p.zrun = torch.as_tensor(zr).to(self.dev) if chains and zr.max() > 1 else None
            self.params.append(p)
        nws = H.hydro_workspace_bytes(self.params[0], N)
        ws = torch.empty(nws, dtype=torch.uint8, device=self.dev) if nws else None
        for p in self.params:
            p.workspace = ws
        self.cells_per_step = sum(len(lv["origin"]) * N ** 3 * 2 ** l for l, lv in enumerate(levels))
        self.graph = None

    def level(self, l, U):
        return H.AmrLevel(U=U, origin=self.origin[l], map=self.map[l], box=self.box[l])

    def _step(self, l, dt, s, st, tm):
        coarse = self.level(l - 1, self.cur[l - 1]) if l > 0 else None
        coarse_new = self.new[l - 1] if (l > 0 and s == 1) else None
        with tm("prepare"):
            H.hydro_amr_prepare(self.level(l, self.cur[l]), coarse, coarse_new, 0.5 * s, self.Ug[l], bc=self.bc,
                                N=self.N, ghost=self.ghost, precision=self.prec, error=self.err, stream=st)
        p = self.params[l]
        p.dt = dt
        with tm("advance"):
            H.hydro_advance(p, self.Ug[l], self.new[l], self.flux[l][s], self.status[l], N=self.N,
                            ghost=self.ghost, stream=st)
        if l + 1 < self.L:
            self._step(l + 1, 0.5 * dt, 0, st, tm)
            self._step(l + 1, 0.5 * dt, 1, st, tm)
            with tm("reflux"):
                H.hydro_amr_reflux(self.level(l, self.new[l]), self.flux[l][s], self.level(l + 1, self.cur[l + 1]),
                                   self.flux[l + 1][0], self.flux[l + 1][1], dt, p.dx, bc=self.bc, N=self.N,
                                   precision=self.prec, error=self.err, stream=st)
            with tm("restrict"):
                H.hydro_amr_restrict(self.level(l + 1, self.cur[l + 1]), self.level(l, self.new[l]), N=self.N,
                                     precision=self.prec, error=self.err, stream=st)
        self.cur[l], self.new[l] = self.new[l], self.cur[l]

    def step(self, dt0, stream=None):
        """One step of the whole hierarchy with base time step dt0."""
        self._step(0, float(dt0), 0, stream if stream is not None else self.stream, _no_timer)

    def step_timed(self, dt0):
        """step() on the current stream with CUDA events around every launch;
        returns the device milliseconds per kind of launch (prepare, advance,
        reflux, restrict)."""
        torch = self.torch
        marks = []

        class _T:
            def __init__(self, kind):
                self.kind = kind

            def __enter__(self):
                self.a = torch.cuda.Event(enable_timing=True)
                self.a.record()

            def __exit__(self, *exc):
                b = torch.cuda.Event(enable_timing=True)
                b.record()
                marks.append((self.kind, self.a, b))

        self._step(0, float(dt0), 0, None, _T)
        torch.cuda.synchronize()
        out = {}
        for kind, a, b in marks:
            out[kind] = out.get(kind, 0.0) + a.elapsed_time(b)
        return out

    def launches_per_step(self):
        """Kernels one step enqueues: prepare + advance per level step, reflux +
        restrict per refined level step."""
        n = 0
        for l in range(self.L):
            n += 2 ** l * (2 + (2 if l + 1 < self.L else 0))
        return n

    def compute_dt(self, cfl=0.4):
        """dt_0 = min over levels of 2^l x the CFL dt of level l, reduced on
        the device in one pass (hydro_cfl_dt_boxes with dt_scale = 2^l);
        returns the host value."""
        torch = self.torch
        ws = torch.empty(H.hydro_cfl_boxes_workspace_bytes(), dtype=torch.uint8, device=self.dev)
        dts = torch.zeros(self.L + 1, dtype=torch.float64, device=self.dev)
        p = self.params[0]
        boxes = [(self.cur[l], self.params[l].dx, dts[l:l + 1], 2.0 ** l) for l in range(self.L)]
        H.hydro_cfl_dt_boxes(boxes, cfl, ws, dt_min_out=dts[self.L:], gamma=p.gamma, dens_floor=p.dens_floor,
                             pres_floor=p.pres_floor, precision=self.prec, stream=self.stream)
        return float(dts[self.L].item())

    def errors(self):
        return int(self.err.item())

    def capture(self, dt0):
        """Capture two steps of dt0 into a CUDA graph (a graph replays fixed
        buffers; level 0 swaps its double buffer once per step, the finer
        levels an even number of times, so two steps bring every level back
        to the buffers it started from).  capture_graph's warm-up runs the
        two steps once eagerly; replay() then advances two steps each."""
        st = self.torch.cuda.current_stream

        def two():
            self.step(dt0, st())
            self.step(dt0, st())

        self.graph = capture_graph(two)
        return self.graph

    def replay(self):
        """Two steps (see capture)."""
        self.graph.replay()
