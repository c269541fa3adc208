"""Shared helpers of the GPU tests (all comparisons go through the C ABI)."""
import numpy as np

import oracle as O
from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import workloads as W

# Tolerances (relative L1 per variable and step against the FP64 oracle):
TOL_FP64 = 1e-12   # same formulas in the same operation order, no FMA contraction
TOL_FP32 = 1e-5    # single-precision bulk arithmetic (both FP32 forms)

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
