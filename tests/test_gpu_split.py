"""GPU parity of the directionally split schemes (RTVD, WAF; Sec. 3.2's
comparison schemes) against the oracle, through the C ABI: every precision,
both sweep orders and several limiters on a periodic lognormal box of 2x2x2
groups (state, boundary fluxes, status); the fused uniform path equal to
gather + hydro_advance byte for byte; ten steps of Sod along y with
alternating sweep orders in FP64 (each step within 1e-12 of the oracle's)."""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import workloads as W
from tests.gpu_common import (ELEM_FP32_SPLIT, PREC_NAME, assert_close, gpu_advance, lognormal_groups, params_pair, quantise, tdtype,
                              with_workspace)

pytestmark = pytest.mark.gpu
N = 16


def _pair(scheme, prec, dt, dx, limiter, theta, order):
    po, ph = params_pair(scheme, O.PLM, O.HLLC, prec, dt, dx, limiter=limiter, theta=theta)
    po.split_order = order
    ph.split_order = order
    return po, ph


@pytest.mark.parametrize("prec", [H.FP64, H.FP32, H.FP32_MIXED], ids=lambda p: PREC_NAME[p])
@pytest.mark.parametrize("scheme", [O.RTVD, O.WAF])
@pytest.mark.parametrize("order,limiter,theta", [(0, O.MINMOD, 1.0), (1, O.VANLEER, 1.0), (0, O.HYBRID, 1.5),
                                                 (1, O.VANALBADA, 1.0)])
def test_split_matches_oracle(prec, scheme, order, limiter, theta):
    g = O.required_ghost(scheme, 0)
    Uq, Ug = lognormal_groups(n=32, g=g, seed=5, prec=prec, p_index=1.4, mach=1.0)
    dx = (1.0 / 32,) * 3
    dt = O.cfl_dt(Uq, dx, 0.4)
    po, ph = _pair(scheme, prec, dt, dx, limiter, theta, order)
    ref, ref_flux, ref_st = O.advance(po, Ug, N)
    got, flux, st = gpu_advance(ph, Ug)
    elem = ELEM_FP32_SPLIT if prec != H.FP64 else None
    assert_close(got, ref, prec, "state", elem=elem)
    assert_close(flux, ref_flux, prec, "flux", axis_var=2, elem=elem)
    assert np.array_equal(st & H.ST_ERROR_MASK, ref_st & H.ST_ERROR_MASK)
    if prec == H.FP64:
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("scheme", [O.RTVD, O.WAF])
@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
def test_split_fused_uniform_equals_gather_then_advance(scheme, prec):
    import torch
    dev = torch.device("cuda:0")
    n = 32
    g = O.required_ghost(scheme, 0)
    U = quantise(W.lognormal(n, seed=3, mach=1.0, p_index=1.4), prec)
    dx = (1.0 / n,) * 3
    _, ph = _pair(scheme, prec, O.cfl_dt(U, dx, 0.4), dx, O.MINMOD, 1.0, 1)
    with_workspace(ph, dev)
    dtp = tdtype(prec)
    ft = torch.tensor(U, dtype=dtp, device=dev)
    orig = torch.tensor(W.group_origins(n, n, n, N), dtype=torch.int32, device=dev)
    G = orig.shape[0]
    M = N + 2 * g
    Ug = torch.empty((G, 5, M, M, M), dtype=dtp, device=dev)
    H.hydro_gather_uniform(ft, orig, Ug, N=N, ghost=g, bc=0, precision=prec)
    Uo = torch.empty((G, 5, N, N, N), dtype=dtp, device=dev)
    fl = torch.empty((G, 6, 5, N, N), dtype=dtp, device=dev)
    st = torch.empty(G, dtype=torch.int32, device=dev)
    H.hydro_advance(ph, Ug, Uo, fl, st, ghost=g)
    out = torch.empty_like(ft)
    fl2 = torch.empty_like(fl)
    st2 = torch.empty_like(st)
    H.hydro_advance_uniform(ph, ft, out, bc=0, flux=fl2, status=st2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.double().cpu().numpy(), W.scatter_groups(Uo.double().cpu().numpy(), n, n, n))
    np.testing.assert_array_equal(fl2.cpu().numpy(), fl.cpu().numpy())
    np.testing.assert_array_equal(st2.cpu().numpy(), st.cpu().numpy())


@pytest.mark.parametrize("scheme", [O.RTVD, O.WAF])
def test_split_sod_ten_steps_fp64(scheme):
    import torch
    from paper_1103_3373_gb300 import runtime as RT
    n = 64
    U = W.sod(n, 1, ny=n, nz=16)  # along y
    U = U[:, :, :, :16].copy()     # 16 x 64 x 16 (x, y, z) -> [5][16][64][16]
    dx = (1.0 / 16, 1.0 / n, 1.0 / 16)
    _, ph = _pair(scheme, H.FP64, 0.0, dx, O.VANLEER, 1.0, 0)
    box = RT.UniformBox(U, ph, cfl=0.4, bc=H.BC_OUTFLOW)
    Uo = U.copy()
    org = W.group_origins(16, n, 16, N)
    g = O.required_ghost(scheme, 0)
    for k in range(10):
        # the oracle takes its own dt; the device's agrees
        dt = O.cfl_dt(Uo, dx, 0.4)
        assert box.dt.item() == pytest.approx(dt, rel=1e-14)
        P = O.Params(scheme=scheme, limiter=O.VANLEER, dt=dt, dx=dx, split_order=k % 2)
        Uo = W.scatter_groups(O.advance(P, O.gather(Uo, org, N, g, bc=1), N)[0], 16, n, 16)
        box.step()
        torch.cuda.synchronize()
        assert_close(box.state().cpu().numpy()[None], Uo[None], H.FP64, "state step %d" % k)
