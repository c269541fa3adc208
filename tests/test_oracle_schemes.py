"""Whole-step pins of the oracle's MHM / VL / CTU group update (Sec. 2 and 3.1).

What fixes each expectation, independently of the oracle's own code:
  * a uniform state is a steady solution: every flux difference vanishes;
  * on a periodic box the flux-difference update telescopes (Sec. 2 step (4)):
    totals of mass, momentum and energy are conserved to roundoff;
  * an unsplit scheme treats the axes alike (Sec. 1): a problem posed along
    y or z, or with the axes permuted, gives the permuted answer;
  * a density profile carried by a uniform flow at uniform pressure reduces
    every scheme to a textbook 1D linear-advection scheme (written here in
    numpy from its definition: MUSCL with minmod slopes, the VL predictor /
    corrector, and Colella & Woodward's PPM advection);
  * Sod's shock tube converges to the exact Riemann solution (itself pinned
    by the jump conditions in test_oracle_local.py);
  * a linear sound wave converges at second order;
  * the ghost-zone gather equals numpy's periodic / edge padding.
"""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import workloads as W
from tests.oracle_runs import oracle_box_step, oracle_run

SCHEMES = [O.MHM, O.VL, O.CTU]
RECONS = [O.PLM, O.PPM]
SOLVERS = [O.EXACT, O.HLLE, O.HLLC, O.ROE]


def ghost_for(scheme, recon):
    return O.required_ghost(scheme, recon)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("recon", RECONS)
@pytest.mark.parametrize("solver", SOLVERS)
def test_uniform_state_is_steady(scheme, recon, solver):
    N = 8
    U = W.uniform((8, 8, 8), rho=1.3, v=(0.4, -0.3, 0.2), p=0.9)
    P = O.Params(scheme=scheme, recon=recon, riemann=solver, limiter=O.VANLEER, dt=0.01, dx=(1 / 8,) * 3)
    g = ghost_for(scheme, recon)
    Ug = O.gather(U, W.group_origins(8, 8, 8, N), N, g, bc=0)
    Uo, fl, st = O.advance(P, Ug, N)
    np.testing.assert_array_equal(Uo[0], U)
    assert st[0] == 0


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("recon,solver,lim", [(O.PPM, O.ROE, O.MINMOD), (O.PLM, O.HLLC, O.VANLEER),
                                               (O.PLM, O.HLLE, O.HYBRID), (O.PPM, O.EXACT, O.VANALBADA)])
def test_conservation_periodic(scheme, recon, solver, lim):
    n, N = 16, 8
    U = W.lognormal(n, seed=11, mach=1.0)
    P = O.Params(scheme=scheme, recon=recon, riemann=solver, limiter=lim, theta=1.5, dx=(1 / n,) * 3)
    P.dt = O.cfl_dt(U, P.dx, 0.4)
    U1, fl, st = oracle_box_step(U, P, N, ghost_for(scheme, recon), bc=0)
    assert np.all(st & O.ST_ERROR_MASK == 0)
    tot0 = U.reshape(5, -1).sum(axis=1)
    tot1 = U1.reshape(5, -1).sum(axis=1)
    scale = np.abs(U).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale)
    # the update changed the state (the test is not vacuous)
    assert np.abs(U1 - U).max() > 1e-3


@pytest.mark.parametrize("scheme,recon,solver", [(O.MHM, O.PLM, O.ROE), (O.CTU, O.PPM, O.ROE),
                                                 (O.VL, O.PLM, O.HLLC), (O.CTU, O.PLM, O.EXACT)])
def test_sod_identical_along_each_axis(scheme, recon, solver):
    n, N = 16, 8
    g = ghost_for(scheme, recon)
    P = O.Params(scheme=scheme, recon=recon, riemann=solver, limiter=O.MINMOD, dx=(1 / n,) * 3, dt=0.2 / n)
    res = []
    for axis in range(3):
        U = W.sod(n, axis)
        U1, _, _ = oracle_run(U, P, N, g, bc=1, steps=3, dt=0.2 / n)
        # bring the result back to an x-directed tube
        if axis == 1:
            U1 = U1[[0, 2, 3, 1, 4]].transpose(0, 1, 3, 2)
        elif axis == 2:
            U1 = U1[[0, 3, 1, 2, 4]].transpose(0, 3, 2, 1)
        res.append(U1)
    np.testing.assert_array_equal(res[1], res[0])
    np.testing.assert_array_equal(res[2], res[0])


@pytest.mark.parametrize("scheme,recon,solver", [(O.MHM, O.PPM, O.ROE), (O.CTU, O.PPM, O.ROE),
                                                 (O.VL, O.PLM, O.HLLC)])
def test_axis_permutation_symmetry_diagonal_sod(scheme, recon, solver):
    n, N = 16, 8
    g = ghost_for(scheme, recon)
    P = O.Params(scheme=scheme, recon=recon, riemann=solver, limiter=O.VANLEER, dx=(1 / n,) * 3)
    U = W.sod(n, diagonal=True)
    U1, _, _ = oracle_run(U, P, N, g, bc=1, steps=3, dt=0.15 / n)
    # the diagonal problem is invariant under any permutation of the axes
    for perm in ([1, 0, 2], [2, 1, 0], [0, 2, 1]):  # (x,y,z) -> permuted
        Up = U1[[0, 1 + perm[0], 1 + perm[1], 1 + perm[2], 4]]
        Up = Up.transpose([0] + [3 - perm[2 - a] for a in range(3)])
        np.testing.assert_allclose(Up, U1, rtol=1e-12, atol=1e-13)


# ---------------------------------------------- 1D linear advection reduction
def minmod(a, b):
    return np.where(a * b > 0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def adv_muscl(r, nu):
    d = minmod(r - np.roll(r, 1), np.roll(r, -1) - r)
    face = r + 0.5 * (1 - nu) * d  # value at i+1/2 carried by the upwind cell
    return r - nu * (face - np.roll(face, 1))


def adv_vl(r, nu):
    rh = r - 0.5 * nu * (r - np.roll(r, 1))
    d = minmod(rh - np.roll(rh, 1), np.roll(rh, -1) - rh)
    face = rh + 0.5 * d
    return r - nu * (face - np.roll(face, 1))


def adv_ppm(r, nu):
    d = minmod(r - np.roll(r, 1), np.roll(r, -1) - r)
    edge = 0.5 * (r + np.roll(r, -1)) - (np.roll(d, -1) - d) / 6.0  # value at i+1/2
    aL, aR = np.roll(edge, 1).copy(), edge.copy()
    for i in range(r.size):
        a = r[i]
        if (aR[i] - a) * (a - aL[i]) <= 0:
            aL[i] = aR[i] = a
        else:
            dA = aR[i] - aL[i]
            a6 = 6 * (a - 0.5 * (aL[i] + aR[i]))
            if dA * a6 > dA * dA:
                aL[i] = 3 * a - 2 * aR[i]
            elif -dA * dA > dA * a6:
                aR[i] = 3 * a - 2 * aL[i]
    dA = aR - aL
    a6 = 6 * (r - 0.5 * (aL + aR))
    face = aR - 0.5 * nu * (dA - (1 - 2.0 / 3.0 * nu) * a6)
    return r - nu * (face - np.roll(face, 1))


@pytest.mark.parametrize("scheme,recon,ref", [(O.MHM, O.PLM, adv_muscl), (O.CTU, O.PLM, adv_muscl),
                                              (O.VL, O.PLM, adv_vl), (O.CTU, O.PPM, adv_ppm)])
@pytest.mark.parametrize("solver", [O.ROE, O.HLLC, O.EXACT])
@pytest.mark.parametrize("axis", [0, 2])
def test_reduces_to_linear_advection(scheme, recon, ref, solver, axis):
    nx, N = 32, 8
    shape = [8, 8, 8]
    shape[2 - axis] = nx
    vel = [0.0, 0.0, 0.0]
    vel[axis] = 0.8
    U = W.advection(tuple(shape), velocity=tuple(vel), kind="square", axis=axis)
    dx = 1.0 / nx
    dt = 0.45 * dx / 0.8
    nu = 0.8 * dt / dx
    P = O.Params(scheme=scheme, recon=recon, riemann=solver, limiter=O.MINMOD, dx=(dx,) * 3)
    U1, _, _ = oracle_run(U, P, N, ghost_for(scheme, recon), bc=0, steps=6, dt=dt)
    r = np.moveaxis(U[0], 2 - axis, 0)[:, 0, 0].copy()
    for _ in range(6):
        r = ref(r, nu)
    got = np.moveaxis(U1[0], 2 - axis, 0)
    np.testing.assert_allclose(got, np.broadcast_to(r[:, None, None], got.shape), rtol=0, atol=2e-13)


# ------------------------------------------------------------ convergence
def sod_exact_rho(x, t, x0=0.5):
    _, _, _, Ws = O.exact_star([1.0, 0, 0, 0, 1.0], [0.125, 0, 0, 0, 0.1], xi=(x - x0) / t)
    return Ws[:, 0]


@pytest.mark.parametrize("scheme,recon,solver", [(O.MHM, O.PLM, O.ROE), (O.CTU, O.PPM, O.ROE),
                                                 (O.VL, O.PLM, O.HLLC), (O.CTU, O.PLM, O.HLLE)])
def test_sod_converges_to_exact(scheme, recon, solver):
    N = 8
    errs = []
    for nx in (32, 64):
        U = W.sod(nx, 0, ny=8, nz=8)
        dx = 1.0 / nx
        P = O.Params(scheme=scheme, recon=recon, riemann=solver, limiter=O.MINMOD, dx=(dx,) * 3)
        U1, t, st = oracle_run(U, P, N, ghost_for(scheme, recon), bc=1, steps=10 ** 6, cfl=0.5, t_end=0.1)
        assert st & O.ST_ERROR_MASK == 0
        x = (np.arange(nx) + 0.5) * dx
        errs.append(np.abs(U1[0, 4, 4, :] - sod_exact_rho(x, t)).mean())
    assert errs[0] < 0.02
    assert errs[1] < 0.75 * errs[0]


@pytest.mark.slow
@pytest.mark.parametrize("scheme,recon,solver", [(O.MHM, O.PLM, O.ROE), (O.CTU, O.PPM, O.ROE),
                                                 (O.VL, O.PLM, O.HLLC)])
def test_sound_wave_second_order(scheme, recon, solver):
    N = 8
    errs = []
    for nx in (16, 32, 64):
        U0 = W.sound_wave(nx, amp=1e-6, shape=(8, 8, nx))
        dx = 1.0 / nx
        P = O.Params(scheme=scheme, recon=recon, riemann=solver, limiter=O.VANLEER, dx=(dx,) * 3)
        U1, t, st = oracle_run(U0, P, N, ghost_for(scheme, recon), bc=0, steps=10 ** 6, cfl=0.4, t_end=1.0)
        errs.append(np.abs(U1[0] - U0[0]).mean())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r2 > 3.0, errs
    assert r1 > 2.5, errs


@pytest.mark.slow
def test_diagonal_sound_wave_converges():
    N = 8
    errs = []
    for n in (16, 32):
        U0 = W.sound_wave(n, amp=1e-6, direction=(1, 1, 1))
        dx = 1.0 / n
        P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, limiter=O.VANLEER, dx=(dx,) * 3)
        U1, t, st = oracle_run(U0, P, N, 3, bc=0, steps=10 ** 6, cfl=0.4, t_end=1.0 / 3 ** 0.5)
        errs.append(np.abs(U1[0] - U0[0]).mean())
    assert errs[0] / errs[1] > 3.0, errs


# --------------------------------------------------------------- gather, dt
@pytest.mark.parametrize("bc,mode", [(0, "wrap"), (1, "edge")])
def test_gather_matches_numpy_pad(bc, mode):
    rng = np.random.default_rng(5)
    f = rng.normal(size=(5, 16, 24, 32))
    N, g = 8, 3
    orig = W.group_origins(32, 24, 16, N)
    got = O.gather(f, orig, N, g, bc=bc)
    pad = np.pad(f, ((0, 0), (g, g), (g, g), (g, g)), mode=mode)
    for gi, (x0, y0, z0) in enumerate(orig):
        np.testing.assert_array_equal(got[gi], pad[:, z0:z0 + N + 2 * g, y0:y0 + N + 2 * g, x0:x0 + N + 2 * g])


def test_cfl_dt_closed_form():
    g = 1.4
    U = W.uniform((4, 4, 4), rho=2.0, v=(0.5, -1.5, 0.25), p=3.0, gamma=g)
    c = np.sqrt(g * 3.0 / 2.0)
    dx = (0.1, 0.2, 0.05)
    expect = 0.5 / max((0.5 + c) / 0.1, (1.5 + c) / 0.2, (0.25 + c) / 0.05)
    assert O.cfl_dt(U, dx, 0.5, gamma=g) == pytest.approx(expect, rel=1e-15)


def test_ghost_too_small_rejected():
    U = np.zeros((1, 5, 14, 14, 14))
    with pytest.raises(ValueError):
        O.advance(O.Params(scheme=O.VL, recon=O.PPM), U, N=8)  # needs 4


def test_op_count_is_positive_and_deterministic():
    n, N = 8, 8
    U = W.lognormal(n, seed=3, mach=1.0)
    Ug = O.gather(U, W.group_origins(n, n, n, N), N, 3, bc=0)
    P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, dx=(1 / n,) * 3, dt=0.01)
    a, ca = O.count_ops(P, Ug[0], N)
    b, cb = O.count_ops(P, Ug[0], N)
    assert a == b and ca == cb
    assert a["riemann"]["add"] > 0 and a["trace"]["mul"] > 0 and a["correct"]["add"] > 0


@pytest.mark.slow
def test_sedov_taylor_radius_and_spherical_symmetry():
    """Sedov-Taylor blast (E = 1 in r < 2 cells, rho = 1, p = 1e-5, gamma = 5/3;
    CTU + PPM + HLLC, outflow, 48^3): the shock radius, taken from the density
    maximum along the six axis rays, follows the self-similar closed form
    R(t) = xi0 (E t^2 / rho)^(1/5), xi0 = 1.15 for gamma = 5/3, within one cell
    width at R = 0.2 and 0.3; the six rays are the same profile (the blast
    sits on the cube's centre, so every axis is equivalent) to roundoff."""
    from tests.oracle_runs import oracle_run
    n, xi0 = 48, 1.15
    U = W.sedov(n)
    P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.HLLC, limiter=O.MINMOD, theta=1.0, fallback=O.HLLE,
                 gamma=5.0 / 3.0, dens_floor=1e-12, pres_floor=1e-12, dt=0.0, dx=(1.0 / n,) * 3)
    t = 0.0
    for R in (0.2, 0.3):
        t_end = (R / xi0) ** 2.5  # E = rho = 1
        U, dt_t, st = oracle_run(U, P, 16, 3, 1, 100000, cfl=0.4, t_end=t_end - t)
        t += dt_t
        assert st & O.ST_ERROR_MASK == 0
        assert t == pytest.approx(t_end, rel=1e-12)
        rho, c = U[0], n // 2
        rays = [rho[c, c, c:], rho[c, c, :c][::-1], rho[c, c:, c], rho[c, :c, c][::-1], rho[c:, c, c],
                rho[:c, c, c][::-1]]
        for r in rays[1:]:
            np.testing.assert_allclose(r, rays[0], rtol=0, atol=1e-12)
        R_num = (np.argmax(rays[0]) + 0.5) / n
        assert abs(R_num - xi0 * t ** 0.4) <= 1.0 / n, (R, R_num)


def test_stored_flop_counts_are_the_oracles():
    """The roofline numerator bench.py reads (data/flops_per_cell.json) is what
    oracle/count_ops.py computes now: the headline and VL entries recounted
    on the same workload equal the stored values."""
    import json
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    import importlib.util
    # loaded under a name of its own: as the submodule oracle.count_ops it would
    # shadow the package's count_ops function, which it calls
    spec = importlib.util.spec_from_file_location("oracle_count_script", os.path.join(root, "oracle", "count_ops.py"))
    C = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(C)
    stored = json.load(open(os.path.join(root, "paper_1103_3373_gb300", "data", "flops_per_cell.json")))["entries"]
    n, N = 32, 16
    U = W.lognormal(n, seed=1, mach=1.5)
    dx = (1.0 / n,) * 3
    dt = O.cfl_dt(U, dx, 0.4)
    for scheme, recon, rs, key in ((O.CTU, O.PPM, O.ROE, "ctu-ppm-roe"), (O.VL, O.PLM, O.HLLC, "vl-plm-hllc")):
        g = O.required_ghost(scheme, recon)
        Ug = O.gather(U, W.group_origins(n, n, n, N), N, g, bc=0)
        groups = [(Ug[i], dt, dx) for i in range(0, Ug.shape[0], 3)]
        got = C.count(scheme, recon, rs, groups)
        assert got["flops"] == pytest.approx(stored[key]["flops"], rel=1e-12), key
