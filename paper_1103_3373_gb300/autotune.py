"""Project-written autotuner for the patch-group kernels.

For one configuration (scheme, reconstruction, solver, precision, limiter
class) it times the real launch on the caller's data for every candidate
launch shape and keeps the fastest:
  * threads per CTA: multiples of 32 between 128 and the kernel's maximum
    (hydro_max_block_threads);
  * CTAs per SM of the persistent grid: 1, and 2 where a second CTA fits
    (the FP64 kernels keep their rings in global memory, so their occupancy is
    set by registers only).
The tile shape itself (a 16^3 group streamed along z, one CTA per group at a
time) and the ghost width (the minimum the scheme needs, hydro_required_ghost:
more only adds gather traffic) are fixed by the kernel design.

Results are cached in memory per device and configuration, and optionally in
a JSON file (HYDRO_AUTOTUNE_CACHE).
"""
import json
import os

from . import hydro as H

_CACHE = {}


def _key(p: H.Params, tag):
    import torch
    dev = torch.cuda.current_device()
    name = torch.cuda.get_device_name(dev)
    lim = "minmod" if p.limiter == H.LIM_MINMOD else "other"
    return "%s|%d|%d|%d|%d|%d|%d|%s|%s" % (name, p.scheme, p.recon if p.scheme <= H.CTU else 0,
                                          p.characteristic, p.riemann, p.precision, p.roe_fallback, lim, tag)


def _load_file():
    path = os.environ.get("HYDRO_AUTOTUNE_CACHE")
    if path and os.path.exists(path):
        try:
            with open(path) as fh:
                for k, v in json.load(fh).items():
                    _CACHE.setdefault(k, v)
        except (OSError, ValueError):
            pass


def _save_file():
    path = os.environ.get("HYDRO_AUTOTUNE_CACHE")
    if path:
        try:
            with open(path, "w") as fh:
                json.dump(_CACHE, fh, indent=1, sort_keys=True)
        except OSError:
            pass


def candidates(p: H.Params, nsm):
    maxt = H.hydro_max_block_threads(p)
    out = []
    for t in range(128, maxt + 1, 32):
        out.append((t, 0))
        if p.precision == H.FP64:
            out.append((t, 2 * nsm))
    return out


def tune(p: H.Params, launch, tag="uniform", reps=6, warmup=2, verbose=False):
    """Pick (block_threads, grid_ctas) for `launch(params)`, a callable that
    enqueues one step on the CURRENT stream (the timing events are recorded
    there).  Sets them on p and returns {"block_threads", "grid_ctas", "ms",
    "tried"}."""
    import torch
    _load_file()
    k = _key(p, tag)
    if k in _CACHE:
        best = _CACHE[k]
        p.block_threads, p.grid_ctas = best["block_threads"], best["grid_ctas"]
        return best
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    saved = (p.block_threads, p.grid_ctas, p.workspace)
    tried = []
    best = None
    for bt, gc in candidates(p, nsm):
        p.block_threads, p.grid_ctas = bt, gc
        nws = H.hydro_workspace_bytes(p)
        ws = None
        if nws:
            ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
            p.workspace = ws
        try:
            for _ in range(warmup):
                launch(p)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                launch(p)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
        except H.HydroError:
            continue
        finally:
            del ws
        tried.append([bt, gc, ms])
        if verbose:
            print("autotune %s threads=%d grid=%d %.3f ms" % (tag, bt, gc, ms))
        if best is None or ms < best["ms"]:
            best = {"block_threads": bt, "grid_ctas": gc, "ms": ms}
    p.block_threads, p.grid_ctas, p.workspace = saved
    if best is None:
        raise RuntimeError("autotune: no launch shape ran")
    best["tried"] = tried
    _CACHE[k] = best
    _save_file()
    p.block_threads, p.grid_ctas = best["block_threads"], best["grid_ctas"]
    return best
