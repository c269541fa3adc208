"""Pins of the oracle's characteristic-variable reconstruction (Sec. 2: the
reconstruction acts on primitive or on characteristic variables), each
against something other than the oracle's own eigenvector formulas:

* two acoustic waves superposed on a state: the face values are the state
  plus each wave's limited profile along its eigenvector, the eigenvectors
  taken from numpy.linalg.eig of the primitive Jacobian of the Euler
  equations (scale-free: every limiter is homogeneous of degree one), along
  each axis; the primitive form gives other values there;
* data linear along the line: nothing is limited, so the characteristic form
  equals the primitive one (to rounding), for every limiter and axis;
* a whole scheme: Sod along x with characteristic reconstruction stays close
  to the exact solution and does not overshoot more than the primitive form.
"""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import workloads as W

GAMMA = 1.4


def _jacobian(Wc, d):
    """Primitive-variable Jacobian along axis d of the Euler equations,
    W = (rho, vx, vy, vz, p): W_t + A W_d = 0."""
    rho, p = Wc[0], Wc[4]
    u = Wc[1 + d]
    A = u * np.eye(5)
    A[0, 1 + d] = rho
    A[1 + d, 4] = 1.0 / rho
    A[4, 1 + d] = GAMMA * p
    return A


def _acoustic(Wc, d):
    lam, V = np.linalg.eig(_jacobian(Wc, d))
    lam, V = lam.real, V.real
    c = np.sqrt(GAMMA * Wc[4] / Wc[0])
    u = Wc[1 + d]
    rm = V[:, np.argmin(np.abs(lam - (u - c)))]
    rp = V[:, np.argmin(np.abs(lam - (u + c)))]
    return rm, rp


def _minmod(a, b):
    return 0.0 if a * b <= 0 else np.sign(a) * min(abs(a), abs(b))


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("recon", [O.PLM, O.PPM])
def test_two_acoustic_waves_limit_separately(d, recon):
    Wc = np.array([1.0, 0.3, -0.2, 0.1, 0.8])
    rm, rp = _acoustic(Wc, d)
    eps = 0.01
    if recon == O.PLM:
        s = eps * np.array([-1.0, 0.0, 2.0])   # monotone: slope min(1, 2) = 1
        t = eps * np.array([0.5, 0.0, 0.25])   # extremum: slope 0
    else:
        s = eps * np.array([-2.0, -1.5, 0.0, 2.0, 2.5])
        t = eps * np.array([0.3, 0.5, 0.0, 0.25, -0.1])
    Wl = Wc[:, None] + np.outer(rp, s) + np.outer(rm, t)
    P = O.Params(recon=recon, characteristic=1, gamma=GAMMA)
    WL, WR, _ = O.recon_line(P, d, Wl)
    i = len(s) // 2
    if recon == O.PLM:
        ms, mt = _minmod(s[1] - s[0], s[2] - s[1]), _minmod(t[1] - t[0], t[2] - t[1])
        wantL = Wc - 0.5 * (ms * rp + mt * rm)
        wantR = Wc + 0.5 * (ms * rp + mt * rm)
    else:
        sL, sR = O.recon1d(O.PPM, O.MINMOD, s)
        tL, tR = O.recon1d(O.PPM, O.MINMOD, t)
        wantL = Wc + sL[i] * rp + tL[i] * rm
        wantR = Wc + sR[i] * rp + tR[i] * rm
    np.testing.assert_allclose(WL[:, i], wantL, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(WR[:, i], wantR, rtol=1e-12, atol=1e-14)
    # the primitive form limits the components instead and differs here
    Pp = O.Params(recon=recon, characteristic=0, gamma=GAMMA)
    WLp, WRp, _ = O.recon_line(Pp, d, Wl)
    assert np.abs(WLp[:, i] - WL[:, i]).max() > 1e-5


@pytest.mark.parametrize("limiter", [O.MINMOD, O.VANLEER, O.VANALBADA, O.HYBRID])
@pytest.mark.parametrize("recon", [O.PLM, O.PPM])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_linear_data_equals_primitive_reconstruction(limiter, recon, d):
    n = 9
    x = np.arange(n, dtype=np.float64)
    Wl = np.stack([1.0 + 0.05 * x, 0.2 - 0.03 * x, 0.1 + 0.02 * x, -0.3 + 0.01 * x, 0.9 + 0.04 * x])
    theta = 1.5
    Pc = O.Params(recon=recon, limiter=limiter, theta=theta, characteristic=1, gamma=GAMMA)
    Pp = O.Params(recon=recon, limiter=limiter, theta=theta, characteristic=0, gamma=GAMMA)
    a, b = O.recon_line(Pc, d, Wl), O.recon_line(Pp, d, Wl)
    for u, w in zip(a, b):
        ok = ~np.isnan(w)
        np.testing.assert_allclose(u[ok], w[ok], rtol=1e-13, atol=1e-14)


def test_sod_with_characteristic_reconstruction():
    """CTU + PPM + Roe on Sod along x (64 cells, outflow), 40 steps at CFL
    0.4: the characteristic form is as close to the exact solution as the
    primitive one and overshoots the post-shock plateau no more."""
    n, N = 64, 16
    U = W.sod(n, 0, ny=16, nz=16)
    dx = (1.0 / n,) * 3
    org = W.group_origins(n, 16, 16, N)
    res = {}
    for ch in (0, 1):
        Uc = U.copy()
        t = 0.0
        for _ in range(40):
            dt = O.cfl_dt(Uc, dx, 0.4)
            P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, dt=dt, dx=dx, characteristic=ch)
            Uc = W.scatter_groups(O.advance(P, O.gather(Uc, org, N, 3, bc=1), N)[0], n, 16, 16)
            t += dt
        res[ch] = (Uc[0, 8, 8, :], t)
    x = (np.arange(n) + 0.5) / n
    WL, WR = np.array([1.0, 0.0, 0.0, 0.0, 1.0]), np.array([0.125, 0.0, 0.0, 0.0, 0.1])
    xi = (x - 0.5) / res[0][1]
    rho_ex = O.exact_star(WL, WR, GAMMA, xi=xi)[3][:, 0]
    err = {ch: np.abs(res[ch][0] - rho_ex).mean() for ch in (0, 1)}
    assert err[1] < 0.02 and err[0] < 0.02
    assert err[1] <= 1.2 * err[0]
    assert res[1][0].max() <= res[0][0].max() + 1e-12
