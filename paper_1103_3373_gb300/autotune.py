"""Project-written autotuner for the patch-group kernels.

For one configuration (scheme, reconstruction, solver, precision, limiter
class) it times the real launch on the caller's data for every candidate
and keeps the fastest:
  * threads per CTA: multiples of 32 between 128 and the kernel's maximum
    (hydro_max_block_threads);
  * CTAs per SM of the persistent grid: 1, and 2 where a second CTA fits
    (the FP64 kernels keep their rings in global memory, so their occupancy is
    set by registers only);
  * for uniform fields of the unsplit schemes, the chain length (the tile's
    extent along z: how many z-consecutive 16^3 groups a CTA streams through
    without restarting, 1 .. CHAIN_MAX; the work list then runs in
    z-segments of that many layers), so the tile shape is tuned between one
    group (16^3) and a whole column (16^2 x 16 K); for prepared groups given
    with runs of z-continuations (an AMR level's columns, a refined group's
    z-pairs), the longest chain through those runs.
The tile's lateral extent (16^2, one patch group) and the ghost width are
not candidates: the lateral extent is set by the shared-memory rings of a
group's planes (the CTU rings take 220 KB of the 227 KB a CTA may hold, so a
wider tile does not fit), and the ghost width is the minimum the scheme needs
(hydro_required_ghost): a wider one only adds gather traffic and traced
halo cells, and changes no result.

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


def chain_candidates(p: H.Params, tag):
    """Chain lengths worth timing: uniform fields of the unsplit schemes
    (0 = whole columns, up to CHAIN_MAX), and prepared groups given with
    runs of z-continuations (tag "levels_runs"; 0 = whole runs, 1 = every
    group alone).  Other work does not chain."""
    if p.scheme > H.CTU:
        return [p.chain]
    if tag == "uniform":
        return [0, 8, 4, 2]
    if tag == "levels_runs":
        return [0, 4, 2, 1]
    return [p.chain]


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


def candidates(p: H.Params, nsm, tag="uniform"):
    maxt = H.hydro_max_block_threads(p)
    out = []
    for ch in chain_candidates(p, tag):
        for t in range(128, maxt + 1, 32):
            if ch != chain_candidates(p, tag)[0] and t < maxt - 128:
                continue  # other chain lengths: only the largest CTAs
            out.append((t, 0, ch))
            if p.precision == H.FP64 or t in (192, 256):
                # two CTAs per SM: FP64 (rings in global memory), and the
                # FP32 kernels whose shared-memory rings fit twice (MHM + PLM)
                out.append((t, 2 * nsm, ch))
    return out


def tune(p: H.Params, launch, tag="uniform", reps=6, warmup=2, verbose=False):
    """Pick (block_threads, grid_ctas, chain) for `launch(params)`, a
    callable that enqueues one step on the CURRENT stream (the timing events
    are recorded there).  Sets them on p and returns {"block_threads",
    "grid_ctas", "chain", "ms", "tried"}."""
    import torch
    _load_file()
    k = _key(p, tag)
    if k in _CACHE:
        best = _CACHE[k]
        p.block_threads, p.grid_ctas, p.chain = best["block_threads"], best["grid_ctas"], best.get("chain", 0)
        return best
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    saved = (p.block_threads, p.grid_ctas, p.chain, p.workspace)
    tried = []
    best = None
    for bt, gc, ch in candidates(p, nsm, tag):
        p.block_threads, p.grid_ctas, p.chain = bt, gc, ch
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
        tried.append([bt, gc, ch, ms])
        if verbose:
            print("autotune %s threads=%d grid=%d chain=%d %.3f ms" % (tag, bt, gc, ch, ms))
        if best is None or ms < best["ms"]:
            best = {"block_threads": bt, "grid_ctas": gc, "chain": ch, "ms": ms}
    p.block_threads, p.grid_ctas, p.chain, p.workspace = saved
    if best is None:
        raise RuntimeError("autotune: no launch shape ran")
    best["tried"] = tried
    _CACHE[k] = best
    _save_file()
    p.block_threads, p.grid_ctas, p.chain = best["block_threads"], best["grid_ctas"], best["chain"]
    return best
