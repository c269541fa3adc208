"""FP64 CPU oracle of the unsplit patch-group fluid update — TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and the ``--impl reference`` arm) may import this module.
The product package never imports it and has no CPU fallback.

Thin ctypes wrapper over ``liboracle.so`` (built from the C++ sources in this
folder by ``oracle/build.py``).  All arrays are float64 numpy arrays, C order.
Enumerations follow the paper's names (Sec. 2):
  scheme  MHM=0, VL=1, CTU=2 (unsplit), RTVD=3, WAF=4 (split);  recon PLM=0, PPM=1;
  limiter MINMOD=0 (generalized, theta), VANLEER=1, VANALBADA=2, HYBRID=3;
  riemann EXACT=0, HLLE=1, HLLC=2, ROE=3 (fallback: EXACT/HLLE/HLLC).
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

MHM, VL, CTU, RTVD, WAF = 0, 1, 2, 3, 4
PLM, PPM = 0, 1
MINMOD, VANLEER, VANALBADA, HYBRID = 0, 1, 2, 3
EXACT, HLLE, HLLC, ROE = 0, 1, 2, 3

ST_ROE_FALLBACK, ST_NEG_DENS, ST_NEG_PRES, ST_NAN, ST_EXACT_FAIL = 1, 2, 4, 8, 16
ST_ERROR_MASK = ST_NEG_DENS | ST_NEG_PRES | ST_NAN | ST_EXACT_FAIL

SECTIONS = ["eos", "recon", "trace", "predict", "riemann", "correct", "update", "other"]
OPCLASSES = ["add", "mul", "div", "sqrt", "pow", "cmp"]

_dp = ctypes.POINTER(ctypes.c_double)


class _OrcParams(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("recon", ctypes.c_int), ("limiter", ctypes.c_int),
                ("riemann", ctypes.c_int), ("fallback", ctypes.c_int), ("theta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("dens_floor", ctypes.c_double),
                ("pres_floor", ctypes.c_double), ("dt", ctypes.c_double), ("dx", ctypes.c_double * 3),
                ("characteristic", ctypes.c_int), ("split_order", ctypes.c_int)]


@dataclass
class Params:
    scheme: int = CTU
    recon: int = PPM
    limiter: int = MINMOD
    riemann: int = ROE
    fallback: int = HLLE
    theta: float = 1.0
    gamma: float = 1.4
    dens_floor: float = 0.0
    pres_floor: float = 0.0
    dt: float = 0.0
    dx: tuple = field(default_factory=lambda: (1.0, 1.0, 1.0))
    characteristic: int = 0  # 1: reconstruct characteristic variables (Sec. 2)
    split_order: int = 0     # RTVD / WAF: sweeps x, y, z (0) or z, y, x (1)

    def c(self):
        p = _OrcParams()
        for k in ("scheme", "recon", "limiter", "riemann", "fallback", "characteristic", "split_order"):
            setattr(p, k, int(getattr(self, k)))
        for k in ("theta", "gamma", "dens_floor", "pres_floor", "dt"):
            setattr(p, k, float(getattr(self, k)))
        for d in range(3):
            p.dx[d] = float(self.dx[d])
        return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_required_ghost.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_advance.argtypes = [ctypes.POINTER(_OrcParams), _dp, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_uint), ctypes.c_int]
        L.orc_gather.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.orc_cfl_dt.restype = ctypes.c_double
        L.orc_cfl_dt.argtypes = [_dp, ctypes.c_int, ctypes.c_long, ctypes.c_long, ctypes.c_long, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, _dp, ctypes.c_double]
        L.orc_limiter.restype = ctypes.c_double
        L.orc_limiter.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_recon1d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, ctypes.c_int, _dp, _dp]
        L.orc_recon_line.argtypes = [ctypes.POINTER(_OrcParams), ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp]
        L.orc_trace.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, ctypes.c_double, _dp, _dp]
        L.orc_split_row.argtypes = [ctypes.POINTER(_OrcParams), _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, _dp, _dp]
        L.orc_riemann.restype = ctypes.c_uint
        L.orc_riemann.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, _dp, _dp, _dp]
        L.orc_roe_only.argtypes = [ctypes.c_double, _dp, _dp, _dp]
        L.orc_exact_star.argtypes = [ctypes.c_double, _dp, _dp, _dp, _dp, _dp, ctypes.c_int, _dp]
        L.orc_count_ops.argtypes = [ctypes.POINTER(_OrcParams), _dp, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_longlong)]
        L.orc_count_riemann.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                        ctypes.POINTER(ctypes.c_longlong)]
        _lib = L
    return _lib


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def required_ghost(scheme, recon):
    return lib().orc_required_ghost(scheme, recon)


def advance(params: Params, U_in, N=16, ghost=None, want_flux=True, nthreads=0):
    """One step of G patch groups.  U_in: [G,5,M,M,M] float64 (M = N + 2 ghost).

    Returns (U_out [G,5,N,N,N], flux [G,6,5,N,N] or None, status [G] uint32).
    """
    U_in = _f64(U_in)
    G = U_in.shape[0]
    M = U_in.shape[-1]
    g = (M - N) // 2 if ghost is None else ghost
    assert U_in.shape == (G, 5, M, M, M) and M == N + 2 * g
    U_out = np.zeros((G, 5, N, N, N))
    flux = np.zeros((G, 6, 5, N, N)) if want_flux else None
    status = np.zeros(G, dtype=np.uint32)
    rc = lib().orc_advance(ctypes.byref(params.c()), _ptr(U_in), _ptr(U_out),
                           _ptr(flux) if want_flux else None, G, N, g,
                           status.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)), int(nthreads))
    if rc != 0:
        raise ValueError("ghost width %d below the %d the scheme needs" % (g, required_ghost(params.scheme,
                                                                                               params.recon)))
    return U_out, flux, status


def max_threads():
    return lib().orc_max_threads()


def gather(field, origins, N=16, ghost=3, bc=0):
    """Halo-padded groups [G,5,M,M,M] from a field [5,Z,Y,X]; bc 0 periodic, 1 outflow."""
    field = _f64(field)
    _, Z, Y, X = field.shape
    origins = np.ascontiguousarray(origins, dtype=np.int32)
    G = origins.shape[0]
    M = N + 2 * ghost
    out = np.zeros((G, 5, M, M, M))
    lib().orc_gather(_ptr(field), X, Y, Z, bc, origins.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), G, N,
                     ghost, _ptr(out))
    return out


def cfl_dt(U, dx, cfl, gamma=1.4, dens_floor=0.0, pres_floor=0.0):
    """dt = cfl / max (|v_d|+c)/dx_d over U shaped [G,5,...] (or [5,...])."""
    U = _f64(U)
    if U.ndim in (2, 4) and U.shape[0] == 5:
        U = U[None]
    G = U.shape[0]
    cells = int(np.prod(U.shape[2:]))
    dxa = _f64(np.asarray(dx, dtype=np.float64))
    return lib().orc_cfl_dt(_ptr(U), G, 5 * cells, cells, cells, gamma, dens_floor, pres_floor, _ptr(dxa), cfl)


def limiter(kind, dL, dR, theta=1.0):
    return lib().orc_limiter(kind, theta, dL, dR)


def recon_line(params: Params, d, W):
    """Face values of a line of primitive states W [5][n] (global frame) laid
    along direction d, as the schemes reconstruct them (primitive or
    characteristic form per params).  Returns (WL, WR, slope) [5][n] for the
    cells S..n-1-S (NaN elsewhere)."""
    W = _f64(W)
    n = W.shape[1]
    WL, WR, sl = (np.full((5, n), np.nan) for _ in range(3))
    lib().orc_recon_line(ctypes.byref(params.c()), int(d), _ptr(W), n, _ptr(WL), _ptr(WR), _ptr(sl))
    return WL, WR, sl


def recon1d(recon, limiter_kind, w, theta=1.0):
    w = _f64(w)
    n = w.shape[0]
    wL = np.full(n, np.nan)
    wR = np.full(n, np.nan)
    lib().orc_recon1d(recon, limiter_kind, theta, _ptr(w), n, _ptr(wL), _ptr(wR))
    return wL, wR


def split_row(params: Params, u, lo, hi, dx):
    """One RTVD / WAF sweep (params.scheme) of a row of conserved states
    u [n][5] in the sweep's local frame (normal momentum second) with the
    full params.dt: returns (the row updated on [lo, hi), flux through face
    lo - 1/2, flux through face hi - 1/2)."""
    u = np.array(u, dtype=np.float64, order="C")
    n = u.shape[0]
    assert u.shape == (n, 5)
    Flo, Fhi = np.zeros(5), np.zeros(5)
    lib().orc_split_row(ctypes.byref(params.c()), _ptr(u), n, int(lo), int(hi), float(dx), _ptr(Flo), _ptr(Fhi))
    return u, Flo, Fhi


def trace(recon, W0, a, b, dtdx, gamma=1.4):
    W0, a = _f64(W0), _f64(a)
    b = _f64(b if b is not None else np.zeros(5))
    Wl = np.zeros(5)
    Wr = np.zeros(5)
    lib().orc_trace(recon, gamma, _ptr(W0), _ptr(a), _ptr(b), dtdx, _ptr(Wl), _ptr(Wr))
    return Wl, Wr


def riemann(solver, UL, UR, d=0, gamma=1.4, fallback=HLLE, dens_floor=0.0, pres_floor=0.0):
    UL, UR = _f64(UL), _f64(UR)
    F = np.zeros(5)
    st = lib().orc_riemann(solver, fallback, d, gamma, dens_floor, pres_floor, _ptr(UL), _ptr(UR), _ptr(F))
    return F, st


def roe_only(UL, UR, gamma=1.4):
    UL, UR = _f64(UL), _f64(UR)
    F = np.zeros(5)
    ok = lib().orc_roe_only(gamma, _ptr(UL), _ptr(UR), _ptr(F))
    return F, bool(ok)


def exact_star(WL, WR, gamma=1.4, xi=(0.0,)):
    """(p*, u*, iterations (<0 on failure), primitive states [len(xi),5] sampled
    at x/t = xi), local frame (normal velocity second)."""
    WL, WR = _f64(WL), _f64(WR)
    xi = _f64(np.atleast_1d(np.asarray(xi, dtype=np.float64)))
    ps, us = ctypes.c_double(), ctypes.c_double()
    Ws = np.zeros((xi.shape[0], 5))
    it = lib().orc_exact_star(gamma, _ptr(WL), _ptr(WR), ctypes.byref(ps), ctypes.byref(us), _ptr(xi),
                              xi.shape[0], _ptr(Ws))
    return ps.value, us.value, it, Ws


def _tally(arr):
    n = len(SECTIONS) * len(OPCLASSES)
    ops = {s: {c: int(arr[i * len(OPCLASSES) + j]) for j, c in enumerate(OPCLASSES)}
           for i, s in enumerate(SECTIONS)}
    calls = {s: int(arr[n + i]) for i, s in enumerate(SECTIONS)}
    return ops, calls


def count_ops(params: Params, U_in_group, N=16):
    """Operation tally of one group step: ({section: {class: n}}, {section: calls})."""
    U = _f64(U_in_group)
    M = U.shape[-1]
    g = (M - N) // 2
    out = (ctypes.c_longlong * (len(SECTIONS) * (len(OPCLASSES) + 1)))()
    rc = lib().orc_count_ops(ctypes.byref(params.c()), _ptr(U), N, g, out)
    if rc != 0:
        raise ValueError("ghost too small")
    return _tally(out)


def count_riemann(solver, UL, UR, d=0, gamma=1.4, fallback=HLLE):
    UL, UR = _f64(UL), _f64(UR)
    out = (ctypes.c_longlong * (len(SECTIONS) * (len(OPCLASSES) + 1)))()
    lib().orc_count_riemann(solver, fallback, d, gamma, _ptr(UL), _ptr(UR), out)
    return _tally(out)
