"""Pins of the oracle's AMR operations (oracle/amr.py: ghost-zone preparation
by spatial and temporal interpolation, Sec. 4.2; coarse-grid correction by the
stored boundary fluxes, Sec. 2 step (5) and Sec. 4.3; restriction), each
against something other than the oracle itself:

* prolongation reproduces a linear field exactly (closed form), and linear
  time interpolation gives the midpoint at theta = 1/2;
* restriction of a prolongation is the identity (dyadic data: exact), and
  restriction equals the block mean computed by reshaping;
* refluxing equals the closed form built from analytic face fluxes;
* the layout of the stored face fluxes ([z][y] on x faces, [z][x] on y
  faces, [y][x] on z faces) against a planar flow that varies along one
  transverse axis only;
* a whole hierarchy step conserves the composite totals to roundoff in a
  periodic box (and measurably does not without refluxing);
* a level refining the whole box evolves exactly like a uniform box of twice
  the resolution stepped twice with dt/2;
* a uniform state stays exactly uniform.
"""
import numpy as np
import pytest

import oracle as O
from oracle import amr as A
from paper_1103_3373_gb300 import workloads as W

N = 16


def _level_from_field(F, N=16):
    """Split a [5][Z][Y][X] field into a level dict (x-fastest groups)."""
    Z, Y, X = F.shape[1:]
    org = W.group_origins(X, Y, Z, N)
    U = np.stack([F[:, z:z + N, y:y + N, x:x + N] for (x, y, z) in org])
    return {"U": U, "origin": org, "box": (X, Y, Z)}


def _octet(slot, N=16):
    sx, sy, sz = slot
    return np.asarray([(2 * sx * N + dx * N, 2 * sy * N + dy * N, 2 * sz * N + dz * N)
                       for dz in range(2) for dy in range(2) for dx in range(2)], dtype=np.int32)


def _linear(n, alpha, beta):
    """[5][n][n][n]: alpha_v + beta_v . (cell centre in cell units)."""
    c = np.arange(n) + 0.5
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([alpha[v] + beta[v][0] * xx + beta[v][1] * yy + beta[v][2] * zz for v in range(5)])


ALPHA = [1.0, 2.0, -1.0, 0.5, 4.0]
BETA = [(2.0 ** -2 * (v + 1), -(2.0 ** -3) * (v + 1), 2.0 ** -4 * (v + 2)) for v in range(5)]


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_prolongation_of_a_linear_field_is_exact(theta):
    n = 48
    coarse = _level_from_field(_linear(n, ALPHA, BETA))
    shift = np.array([0.25, -0.5, 0.125, 1.0, -2.0])  # dyadic, per variable
    cnew = coarse["U"] + shift[None, :, None, None, None]
    org = _octet((1, 1, 1))
    fine = {"U": np.full((8, 5, N, N, N), np.nan), "origin": org, "box": (2 * n,) * 3}
    g = 3
    Ug = A.prepare(fine, coarse, cnew if theta else None, theta, ghost=g)
    M = N + 2 * g
    r = np.arange(M) - g
    for k, (x0, y0, z0) in enumerate(org):
        zz, yy, xx = np.meshgrid(z0 + r, y0 + r, x0 + r, indexing="ij")
        outside = ~((xx >= 32) & (xx < 64) & (yy >= 32) & (yy < 64) & (zz >= 32) & (zz < 64))
        for v in range(5):
            # fine cell centre in coarse cell units: (f + 0.5) / 2
            want = ALPHA[v] + BETA[v][0] * (xx + 0.5) / 2 + BETA[v][1] * (yy + 0.5) / 2 + \
                BETA[v][2] * (zz + 0.5) / 2 + theta * shift[v]
            np.testing.assert_array_equal(Ug[k, v][outside], want[outside])
        assert np.all(np.isnan(Ug[k][:, ~outside]))  # covered cells are copies of the fine data


def test_restriction_inverts_prolongation_and_is_the_block_mean():
    rng = np.random.default_rng(3)
    n = 48
    coarse = _level_from_field(rng.integers(-64, 64, size=(5, n, n, n)) / 64.0)
    org = _octet((1, 1, 1))
    fine = {"U": np.zeros((8, 5, N, N, N)), "origin": org, "box": (2 * n,) * 3}
    r = np.arange(N)
    for k, (x0, y0, z0) in enumerate(org):
        zz, yy, xx = np.meshgrid(z0 + r, y0 + r, x0 + r, indexing="ij")
        fine["U"][k] = A.prolong(coarse, None, 0.0, xx.ravel(), yy.ravel(), zz.ravel()).T.reshape(5, N, N, N)
    back = A.restrict(fine, coarse, coarse["U"])
    np.testing.assert_array_equal(back, coarse["U"])
    # arbitrary data: the block mean by reshaping
    fine["U"] = rng.normal(size=fine["U"].shape)
    got = A.restrict(fine, coarse, coarse["U"])
    q = 13  # the group at slot (1, 1, 1) of the 3x3x3 level
    assert tuple(coarse["origin"][q]) == (16, 16, 16)
    for k, o in enumerate(org):
        off = o // 2 - 16
        blk = fine["U"][k].reshape(5, 8, 2, 8, 2, 8, 2).mean(axis=(2, 4, 6))
        np.testing.assert_allclose(got[q][:, off[2]:off[2] + 8, off[1]:off[1] + 8, off[0]:off[0] + 8], blk,
                                   rtol=1e-15, atol=1e-15)
    others = [i for i in range(27) if i != q]
    np.testing.assert_array_equal(got[others], coarse["U"][others])


def _face_pos(d, side, o, a, b, N=16):
    """Global face-centre position (in cell units of its level) of face
    (2d + side) at transverse indices (a, b) of a group with origin o."""
    p = np.zeros(3)
    t1, t2 = [e for e in range(3) if e != d]
    p[d] = o[d] + (N if side else 0)
    p[t2] = o[t2] + a + 0.5
    p[t1] = o[t1] + b + 0.5
    return p


def _analytic_flux(p, v, s, scale):
    x = p / scale
    return np.sin(1.3 * x[0] + 0.7 * x[1] - 0.4 * x[2] + v + 0.3 * s) + 0.1 * v


def test_reflux_equals_the_closed_form():
    n = 48
    rng = np.random.default_rng(4)
    coarse = _level_from_field(rng.normal(size=(5, n, n, n)))
    Gc = 27
    org = _octet((1, 1, 1))
    fine = {"U": np.zeros((8, 5, N, N, N)), "origin": org, "box": (2 * n,) * 3}
    # flux arrays from analytic functions of the face position (coarse units)
    cf = np.empty((Gc, 6, 5, N, N))
    ff = [np.empty((8, 6, 5, N, N)) for _ in range(2)]
    for q in range(Gc):
        for f in range(6):
            for a in range(N):
                for b in range(N):
                    p = _face_pos(f // 2, f % 2, coarse["origin"][q], a, b)
                    for v in range(5):
                        cf[q, f, v, a, b] = _analytic_flux(p, v, 9, 1.0)
    for s in range(2):
        for k in range(8):
            for f in range(6):
                for a in range(N):
                    for b in range(N):
                        p = _face_pos(f // 2, f % 2, org[k], a, b) / 2.0
                        for v in range(5):
                            ff[s][k, f, v, a, b] = _analytic_flux(p, v, s, 1.0)
    dt, dx = 0.01, (1 / 48, 1 / 40, 1 / 56)
    got = A.reflux(coarse, coarse["U"], cf, fine, ff[0], ff[1], dt, dx)
    # closed form: every coarse cell face-adjacent to the refined cube [16, 32)^3
    want = coarse["U"].copy()
    m = A.group_map(coarse["origin"], coarse["box"])
    for d in range(3):
        t1, t2 = [e for e in range(3) if e != d]
        for side_q in range(2):  # the coarse cell's face: 0 -> its -d face (cell at 32), 1 -> its +d face (cell at 15)
            cd = 32 if side_q == 0 else 15
            face = 32 if side_q == 0 else 16
            for u in range(16, 32):
                for w in range(16, 32):
                    c = [0, 0, 0]
                    c[d], c[t2], c[t1] = cd, u, w
                    pc = np.zeros(3)
                    pc[d], pc[t2], pc[t1] = face, u + 0.5, w + 0.5
                    q = m[c[2] // N, c[1] // N, c[0] // N]
                    for v in range(5):
                        Fc = _analytic_flux(pc, v, 9, 1.0)
                        tot = 0.0
                        for s in range(2):
                            for da in (0.25, 0.75):
                                for db in (0.25, 0.75):
                                    pf = np.zeros(3)
                                    pf[d], pf[t2], pf[t1] = face, u + da, w + db
                                    tot += _analytic_flux(pf, v, s, 1.0)
                        sgn = 1.0 if side_q == 0 else -1.0
                        want[q, v, c[2] % N, c[1] % N, c[0] % N] += sgn * dt / dx[d] * (tot / 8.0 - Fc)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    assert not np.array_equal(got, coarse["U"])


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_stored_face_flux_layout(axis):
    """Planar flow along `axis` whose state varies along one transverse axis
    only: the face fluxes of the faces normal to `axis` vary along exactly the
    array index that the layout assigns to that transverse axis."""
    n = 16
    c = (np.arange(n) + 0.5) / n
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    coords = (xx, yy, zz)
    t1, t2 = [e for e in range(3) if e != axis]
    for vary in (t1, t2):
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * coords[vary])
        v = [np.zeros_like(rho)] * 3
        v = list(v)
        v[axis] = np.full_like(rho, 0.7)
        U = W.conserved(rho, v[0], v[1], v[2], 1.0, 1.4)
        Ug = O.gather(U, W.group_origins(n, n, n, N), N, 3, bc=0)
        P = O.Params(scheme=O.MHM, recon=O.PLM, riemann=O.HLLE, dt=0.2 / n, dx=(1 / n,) * 3)
        _, fl, _ = O.advance(P, Ug, N)
        F = fl[0, 2 * axis, 0]  # mass flux through the -axis face, [a][b]
        # a = the larger transverse axis (t2), b = the smaller (t1)
        along_a = np.ptp(F, axis=0).max()
        along_b = np.ptp(F, axis=1).max()
        if vary == t2:
            assert along_a > 0.1 and along_b == 0.0
        else:
            assert along_b > 0.1 and along_a == 0.0


def _composite_totals(levels, Us):
    """Sum of U dV over the cells of each level not covered by the next."""
    tot = np.zeros(5)
    for l, lv in enumerate(levels):
        dV = np.prod(lv["dx"])
        cover = np.zeros(len(lv["origin"]), dtype=bool)
        if l + 1 < len(levels):
            mf = A.group_map(levels[l + 1]["origin"], levels[l + 1]["box"])
            for k, o in enumerate(lv["origin"]):
                s = o // N
                cover[k] = mf[2 * s[2], 2 * s[1], 2 * s[0]] >= 0
        tot += Us[l][~cover].sum(axis=(0, 2, 3, 4)) * dV
    return tot


@pytest.mark.parametrize("case", ["two_levels_ctu", "three_levels_mhm"])
def test_hierarchy_step_conserves_composite_totals(case):
    if case == "two_levels_ctu":
        levels = W.amr_hierarchy(48, (0.2,), mach=1.0)
        P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE)
    else:
        levels = W.amr_hierarchy(64, (0.3, 0.12), mach=1.0)
        P = O.Params(scheme=O.MHM, recon=O.PLM, riemann=O.HLLE)
    assert len(levels) == (2 if case == "two_levels_ctu" else 3)
    dt0 = 0.3 * levels[0]["dx"][0] / 3.0
    before = _composite_totals(levels, [lv["U"] for lv in levels])
    after = A.amr_step(levels, P, dt0)
    got = _composite_totals(levels, after)
    scale = np.abs(before).max()
    assert np.abs(got - before).max() <= 1e-13 * scale
    # level 0 alone now holds the composite totals (restriction)
    lvl0 = after[0].sum(axis=(0, 2, 3, 4)) * np.prod(levels[0]["dx"])
    assert np.abs(lvl0 - before).max() <= 1e-13 * scale
    # without the flux correction the coarse-fine faces leak
    leak = _composite_totals(levels, A.amr_step(levels, P, dt0, reflux_on=False))
    assert np.abs(leak - before).max() > 1e-9 * scale


def test_full_refinement_equals_uniform_double_resolution():
    levels = W.amr_hierarchy(32, (0.0,), full=0, mach=1.0)
    assert len(levels[1]["origin"]) == 64
    P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE)
    dt0 = 0.3 / 32 / 3.0
    after = A.amr_step(levels, P, dt0)
    # the fine level alone, as a uniform 64^3 box stepped twice with dt0 / 2
    fine = levels[1]
    order = np.lexsort((fine["origin"][:, 0], fine["origin"][:, 1], fine["origin"][:, 2]))
    U = W.scatter_groups(fine["U"][order], 64, 64, 64)
    P2 = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, dt=dt0 / 2, dx=(1 / 64,) * 3)
    org = W.group_origins(64, 64, 64, N)
    for _ in range(2):
        U = W.scatter_groups(O.advance(P2, O.gather(U, org, N, 3, bc=0), N)[0], 64, 64, 64)
    np.testing.assert_array_equal(W.scatter_groups(after[1][order], 64, 64, 64), U)


def test_uniform_state_stays_uniform():
    levels = W.amr_hierarchy(48, (0.2,))
    state = W.conserved(1.0, 0.25, -0.5, 0.125, 0.5, 1.4)  # dyadic values
    for lv in levels:
        lv["U"][:] = state[None, :, None, None, None] if np.ndim(state) == 1 else state
    P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.HLLC)
    after = A.amr_step(levels, P, 0.002)
    for l in range(len(levels)):
        np.testing.assert_array_equal(after[l], levels[l]["U"])
