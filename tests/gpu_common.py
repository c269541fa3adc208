"""Shared helpers of the GPU tests (all comparisons go through the C ABI)."""
import json
import os

import numpy as np

import oracle as O
from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import workloads as W

# Tolerances against the FP64 oracle, per variable and step.
# Relative L1 (sum |a-b| / sum |b|):
TOL_FP64 = 1e-12   # same formulas in the same operation order, no FMA contraction
TOL_FP32 = 1e-5    # single-precision bulk arithmetic (both FP32 forms)
# Per element: |a-b| <= ELEM * (|b| + s_v), s_v the mean magnitude of variable v
# over the compared values (so a momentum component near zero is measured on
# its own scale, not on its tiny local value):
ELEM_FP64 = 1e-12
ELEM_FP32 = 3e-5        # unsplit schemes: 10x the largest value observed (2.9e-6)
ELEM_FP32_SPLIT = 5e-4  # split RTVD / WAF: 6x the largest observed (8.6e-5); WAF's
                        # limiter takes the ratio of two density jumps, which
                        # amplifies rounding where the upwind jump is tiny

PREC_NAME = {H.FP64: "fp64", H.FP32: "fp32", H.FP32_MIXED: "mixed"}


def tdtype(prec):
    import torch
    return torch.float64 if prec == H.FP64 else torch.float32


def ndtype(prec):
    return np.float64 if prec == H.FP64 else np.float32


def quantise(U, prec):
    """The values the GPU actually receives, back in float64 for the oracle."""
    return U.astype(ndtype(prec)).astype(np.float64)


def rel_l1(a, b, axis_var=1):
    """max over variables of sum|a-b| / sum|b|; variables whose reference is
    identically ~0 are compared by their absolute error relative to the
    density scale instead."""
    a = np.moveaxis(np.asarray(a, dtype=np.float64), axis_var, 0).reshape(5, -1)
    b = np.moveaxis(np.asarray(b, dtype=np.float64), axis_var, 0).reshape(5, -1)
    scale = np.abs(b[0]).sum()
    out = []
    for v in range(5):
        den = np.abs(b[v]).sum()
        if den < 1e-9 * scale:
            den = scale
        out.append(np.abs(a[v] - b[v]).sum() / den)
    return max(out)


def _by_var(a, axis_var):
    return np.moveaxis(np.asarray(a, dtype=np.float64), axis_var, 0).reshape(5, -1)


def max_rel(a, b, axis_var=1):
    """Max-norm companion of rel_l1: max over variables and elements of
    |a-b| / (|b| + s_v), s_v = mean |b_v| (the density's mean where the
    variable is identically ~0)."""
    a = _by_var(a, axis_var)
    b = _by_var(b, axis_var)
    dens = np.abs(b[0]).mean()
    out = 0.0
    for v in range(5):
        s = np.abs(b[v]).mean()
        if s < 1e-9 * dens:
            s = dens
        out = max(out, float((np.abs(a[v] - b[v]) / (np.abs(b[v]) + s)).max(initial=0.0)))
    return out


def tols(prec):
    """(relative L1 bound, per-element bound) of a precision form."""
    from paper_1103_3373_gb300 import hydro as H
    return (TOL_FP64, ELEM_FP64) if prec == H.FP64 else (TOL_FP32, ELEM_FP32)


def report(what, prec, l1, mx):
    """Append one comparison to the JSON-lines file named by
    HYDRO_PARITY_REPORT (if set): the test, what was compared, the precision
    form, the relative L1 and the max-norm."""
    path = os.environ.get("HYDRO_PARITY_REPORT")
    if not path:
        return
    rec = {"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0], "what": what,
           "prec": PREC_NAME.get(prec, str(prec)), "rel_l1": l1, "max_rel": mx}
    with open(path, "a") as fh:
        fh.write(json.dumps(rec) + "\n")


def assert_close(got, ref, prec, what="state", axis_var=1, tol=None, elem=None):
    """Element-by-element parity: every value finite, the relative L1 per
    variable within `tol` AND every element within `elem` of the reference
    (bounds of the precision form unless given).  Returns (l1, max-norm)."""
    t, e = tols(prec)
    tol = t if tol is None else tol
    elem = e if elem is None else elem
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    assert np.all(np.isfinite(got)), (what, "non-finite values", int((~np.isfinite(got)).sum()))
    l1 = rel_l1(got, ref, axis_var)
    mx = max_rel(got, ref, axis_var)
    report(what, prec, l1, mx)
    assert l1 <= tol, (what, "relative L1", l1, tol)
    assert mx <= elem, (what, "max-norm", mx, elem, worst_element(got, ref, axis_var))
    return l1, mx


def worst_element(a, b, axis_var=1):
    """(variable, flat index, got, ref) of the largest scaled difference."""
    A = _by_var(a, axis_var)
    B = _by_var(b, axis_var)
    dens = np.abs(B[0]).mean()
    best = (-1.0, None)
    for v in range(5):
        s = np.abs(B[v]).mean()
        if s < 1e-9 * dens:
            s = dens
        r = np.abs(A[v] - B[v]) / (np.abs(B[v]) + s)
        if r.size and r.max() > best[0]:
            i = int(r.argmax())
            best = (float(r.max()), (v, i, float(A[v, i]), float(B[v, i])))
    return best[1]


def params_pair(scheme, recon, riemann, prec, dt, dx, limiter=O.MINMOD, theta=1.0, fallback=O.HLLE, gamma=1.4,
                dens_floor=0.0, pres_floor=0.0, characteristic=0):
    po = O.Params(scheme=scheme, recon=recon, riemann=riemann, limiter=limiter, theta=theta, fallback=fallback,
                  gamma=gamma, dens_floor=dens_floor, pres_floor=pres_floor, dt=dt, dx=dx,
                  characteristic=characteristic)
    ph = H.Params(scheme=scheme, recon=recon, riemann=riemann, limiter=limiter, theta=theta, roe_fallback=fallback,
                  precision=prec, gamma=gamma, dens_floor=dens_floor, pres_floor=pres_floor, dt=dt, dx=dx,
                  characteristic=characteristic)
    return po, ph


def with_workspace(ph, device):
    import torch
    n = H.hydro_workspace_bytes(ph)
    ph.workspace = torch.empty(max(n, 16), dtype=torch.uint8, device=device) if n else None
    return ph


def gpu_advance(ph, Ug, N=16, device="cuda:0", want_flux=True):
    """Run hydro_advance on float64 numpy groups (cast to the storage type)."""
    import torch
    dt = tdtype(ph.precision)
    G = Ug.shape[0]
    U_in = torch.tensor(Ug, dtype=dt, device=device)
    U_out = torch.full((G, 5, N, N, N), float("nan"), dtype=dt, device=device)
    flux = torch.full((G, 6, 5, N, N), float("nan"), dtype=dt, device=device) if want_flux else None
    st = torch.full((G,), -1, dtype=torch.int32, device=device)
    with_workspace(ph, device)
    H.hydro_advance(ph, U_in, U_out, flux, st, N=N)
    torch.cuda.synchronize()
    return (U_out.double().cpu().numpy(), flux.double().cpu().numpy() if want_flux else None,
            st.cpu().numpy().astype(np.uint32))


def lognormal_groups(n=32, N=16, g=3, seed=1, mach=1.5, prec=H.FP64, p_index=0.0):
    U = W.lognormal(n, seed=seed, mach=mach, p_index=p_index)
    Uq = quantise(U, prec)
    return Uq, O.gather(Uq, W.group_origins(n, n, n, N), N, g, bc=0)
