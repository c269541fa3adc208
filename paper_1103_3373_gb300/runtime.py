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

    def step(self, stream=None):
        self.advance(stream)
        self.swap()
        self.compute_dt(stream)

    def state(self):
        return self.a


class HostBoxStepper:
    """End-to-end form of UniformBox.step for a caller that keeps its data on
    the host: each step copies the state in from pinned host memory, runs the
    step on the device and copies the new state and dt back (the paper times
    its GPU solver the same way, Sec. 3.2)."""

    def __init__(self, U0, params: H.Params, cfl=0.4, bc=H.BC_PERIODIC, N=16, device="cuda:0"):
        torch = _torch()
        self.box = UniformBox(U0, params, cfl=cfl, bc=bc, N=N, device=device)
        self.host_in = torch.empty(self.box.shape, dtype=self.box.dtype).pin_memory()
        self.host_in.copy_(torch.as_tensor(U0, dtype=self.box.dtype))
        self.host_out = torch.empty_like(self.host_in).pin_memory()
        self.host_dt = torch.zeros(1, dtype=torch.float64).pin_memory()
        self.h2d_bytes = self.host_in.numel() * self.host_in.element_size()
        self.d2h_bytes = self.h2d_bytes + 8

    def step(self):
        b = self.box
        b.a.copy_(self.host_in, non_blocking=True)
        b.step()
        self.host_out.copy_(b.a, non_blocking=True)
        self.host_dt.copy_(b.dt, non_blocking=True)
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
