"""hydro_cfl_dt_noalloc: the CFL reduction for callers that cannot allocate
device memory (code enqueued inside another framework's CUDA graph capture,
or a runtime that only hands out the input and output buffers).  Its scratch
is a static device array inside the library, so the test checks that it gives
exactly the result of the workspace-taking hydro_cfl_dt, on two calls in a row
with different inputs (the second call must not see the first one's partials),
and that inputs beyond its fixed maximum are refused before any launch.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _reference(torch, Ut, dx, cfl, prec):
    ws = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=Ut.device)
    dt = torch.zeros(1, dtype=torch.float64, device=Ut.device)
    sm = torch.zeros(1, dtype=torch.float64, device=Ut.device)
    H.hydro_cfl_dt(Ut, dx, cfl, dt, ws, precision=prec, smax_out=sm)
    return dt, sm


def test_noalloc_matches_workspace_version_twice():
    import torch
    dev = torch.device("cuda:0")
    cases = [
        (W.lognormal(64, seed=9, mach=2.5), (1 / 64, 1 / 48, 1 / 80), 0.45, H.FP32, torch.float32),
        (W.sod(32, 1), (1 / 32,) * 3, 0.5, H.FP64, torch.float64),
    ]
    for U, dx, cfl, prec, tdt in cases:
        Ut = torch.tensor(U, dtype=tdt, device=dev)
        ref_dt, ref_sm = _reference(torch, Ut, dx, cfl, prec)
        dt = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        sm = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        H.hydro_cfl_dt_noalloc(Ut, dx, cfl, dt, precision=prec, smax_out=sm)
        torch.cuda.synchronize()
        # a max-reduction of the same per-cell FP64 values: equal to the last bit
        assert dt.item() == ref_dt.item() and np.isfinite(dt.item())
        assert sm.item() == ref_sm.item()


def test_noalloc_grouped_layout_and_size_limit():
    import torch
    dev = torch.device("cuda:0")
    U = W.lognormal(32, seed=2, mach=1.0)
    Ug = np.stack([U[:, z:z + 16, y:y + 16, x:x + 16] for x, y, z in W.group_origins(32, 32, 32, 16)])
    Ut = torch.tensor(Ug, dtype=torch.float32, device=dev)
    ref_dt, _ = _reference(torch, Ut, (1 / 32,) * 3, 0.4, H.FP32)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    H.hydro_cfl_dt_noalloc(Ut, (1 / 32,) * 3, 0.4, dt)
    torch.cuda.synchronize()
    assert dt.item() == ref_dt.item()
    # one cell more than the static scratch covers: refused, nothing launched
    L = H.library()
    dxa = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    too_many = H.NOALLOC_MAX_CELLS + 1
    rc = L.hydro_cfl_dt_noalloc(Ut.data_ptr(), 1, 5 * too_many, too_many, too_many, H.FP32, 1.4, 0.0, 0.0, dxa, 0.4,
                                dt.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    assert rc == H.ETOOBIG
    torch.cuda.synchronize()
    assert dt.item() == ref_dt.item()


def test_noalloc_empty_input_like_workspace_version():
    """No cells (G == 0, or cells == 0): both entry points accept it and give
    dt = cfl / 0 = +inf."""
    import torch
    dev = torch.device("cuda:0")
    L = H.library()
    Ut = torch.ones((1, 5, 16, 16, 16), dtype=torch.float32, device=dev)  # a valid pointer, never read
    ws = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=dev)
    dxa = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    s = torch.cuda.current_stream().cuda_stream
    for G, cells in ((0, 4096), (1, 0)):
        a = torch.zeros(1, dtype=torch.float64, device=dev)
        b = torch.zeros(1, dtype=torch.float64, device=dev)
        assert L.hydro_cfl_dt(Ut.data_ptr(), G, 5 * 4096, 4096, cells, H.FP32, 1.4, 0.0, 0.0, dxa, 0.4,
                              a.data_ptr(), None, ws.data_ptr(), ws.numel(), s) == 0
        assert L.hydro_cfl_dt_noalloc(Ut.data_ptr(), G, 5 * 4096, 4096, cells, H.FP32, 1.4, 0.0, 0.0, dxa, 0.4,
                                      b.data_ptr(), None, s) == 0
        torch.cuda.synchronize()
        assert a.item() == float("inf") and b.item() == float("inf")
