"""Brute-force pin of the oracle's CTU group step (Sec. 2, the corner
transport upwind scheme): the fluxes of one cell of a tiny group, composed
here face by face from the oracle's single-cell pieces (line reconstruction,
characteristic tracing, one Riemann problem), must give the whole-group
step's stored boundary flux and its updated cell.

The composition follows the scheme's definition, not the group code's loop
order: for the face between cells c - e_d and c along d,
  1. each cell's face states along each direction are the reconstructed
     values traced to t + dt/2 (Sec. 2 step (1)), as conserved variables;
  2. stage-1 fluxes F1_e solve the Riemann problem between the traced
     states of neighbours along e (step (2));
  3. the states facing the face along d are corrected by the transverse
     flux gradients of the two other directions, each with dt/(2 dx_e)
     (step (3));
  4. the face flux is the Riemann problem between the corrected states, and
     the cell moves by the flux differences times dt/dx_d (steps (4), (5)).
Conversions between primitive and conserved variables and the rotation into
a direction's frame are written out in numpy.  The cell spacings differ per
axis, so a pairing of a correction with the wrong axis's dt/dx, a dropped
transverse term or a swapped side changes the answer, which the second test
shows by planting each of them here.
"""
import numpy as np
import pytest

import oracle as O

GAMMA = 1.4
# local frame of direction d: normal momentum second, then the two others
# in cyclic order (d+1, d+2)
MOM = [(1, 2, 3), (2, 3, 1), (3, 1, 2)]
# status bit that only reports a Roe problem handed to the fallback solver
ROE_FALLBACK = 1


def prim(U):
    rho = U[0]
    kin = 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / rho
    return np.array([rho, U[1] / rho, U[2] / rho, U[3] / rho, (GAMMA - 1.0) * (U[4] - kin)])


def cons(W):
    return np.array([W[0], W[0] * W[1], W[0] * W[2], W[0] * W[3],
                     W[4] / (GAMMA - 1.0) + 0.5 * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3])])


def to_local(a, d):
    n, t1, t2 = MOM[d]
    return np.array([a[0], a[n], a[t1], a[t2], a[4]])


def to_global(b, d):
    n, t1, t2 = MOM[d]
    a = np.empty(5)
    a[0], a[n], a[t1], a[t2], a[4] = b[0], b[1], b[2], b[3], b[4]
    return a


class Composer:
    """Face fluxes of one group, built up from single-cell oracle calls.
    Cells are addressed by interior coordinates (x, y, z); ghosts are
    negative or >= N.  `plant` names a deliberate mistake (for the second
    test only)."""

    def __init__(self, P, Upad, N, g, plant=None):
        self.P, self.N, self.g, self.plant = P, N, g, plant
        M = Upad.shape[-1]
        self.W = np.empty((5, M, M, M))  # [v, z, y, x], padded
        for z in range(M):
            for y in range(M):
                for x in range(M):
                    self.W[:, z, y, x] = prim(Upad[:, z, y, x])
        self.S = 2 if P.recon == O.PPM else 1
        self.dtdx = [P.dt / P.dx[d] for d in range(3)]
        self.hdtdx = [0.5 * P.dt / P.dx[d] for d in range(3)]
        self._fs, self._f1 = {}, {}

    def line(self, c, d):
        """Primitive states of the cells c - S e_d .. c + S e_d, [5][2S+1]."""
        g, S = self.g, self.S
        out = np.empty((5, 2 * S + 1))
        for k in range(-S, S + 1):
            q = list(c)
            q[d] += k
            x, y, z = (q[0] + g, q[1] + g, q[2] + g)
            out[:, k + S] = self.W[:, z, y, x]
        return out

    def traced(self, c, d):
        """Step (1): the conserved face states (left, right) of cell c along d."""
        key = (c, d)
        if key not in self._fs:
            S = self.S
            WL, WR, sl = O.recon_line(self.P, d, self.line(c, d))
            w0 = to_local(self.line(c, d)[:, S], d)
            if self.P.recon == O.PPM:
                tl, tr = O.trace(O.PPM, w0, to_local(WL[:, S], d), to_local(WR[:, S], d), self.dtdx[d], GAMMA)
            else:
                tl, tr = O.trace(O.PLM, w0, to_local(sl[:, S], d), None, self.dtdx[d], GAMMA)
            self._fs[key] = (cons(to_global(tl, d)), cons(to_global(tr, d)))
        return self._fs[key]

    def solve(self, d, UL, UR):
        F, st = O.riemann(self.P.riemann, UL, UR, d, GAMMA, self.P.fallback)
        assert int(st) & ~ROE_FALLBACK == 0
        return F

    def stage1(self, c, e):
        """Step (2): F1_e on the face between c - e_e and c."""
        key = (c, e)
        if key not in self._f1:
            cm = list(c)
            cm[e] -= 1
            self._f1[key] = self.solve(e, self.traced(tuple(cm), e)[1], self.traced(c, e)[0])
        return self._f1[key]

    def corrected(self, c, d, side):
        """Step (3): the traced state of cell c on side `side` along d, moved
        by the transverse flux differences of the two other directions."""
        u = self.traced(c, d)[side].copy()
        others = [e for e in range(3) if e != d]
        if self.plant == "drop_second":
            others = others[:1]
        for e in others:
            cp = list(c)
            cp[e] += 1
            h = self.hdtdx[e]
            if self.plant == "wrong_spacing":
                h = self.hdtdx[3 - d - e]
            dF = self.stage1(tuple(cp), e) - self.stage1(c, e)
            u = u - h * dF
        return u

    def face(self, c, d):
        """Step (4): the flux on the face between c - e_d and c."""
        cm = list(c)
        cm[d] -= 1
        UL = self.corrected(tuple(cm), d, 1)
        UR = self.corrected(c, d, 0)
        if self.plant == "swap_sides":
            UL, UR = UR, UL
        return self.solve(d, UL, UR)

    def update(self, Upad, c):
        """Step (5): the new conserved state of cell c."""
        g = self.g
        x, y, z = c
        dU = np.zeros(5)
        for d in range(3):
            cp = list(c)
            cp[d] += 1
            dU = dU + self.dtdx[d] * (self.face(tuple(cp), d) - self.face(c, d))
        return Upad[:, z + g, y + g, x + g] - dU


def tiny_group(N, g, seed):
    """A smooth, compressible, lognormal state on one padded group."""
    M = N + 2 * g
    r = np.random.default_rng(seed)
    rho = np.exp(0.3 * r.standard_normal((M, M, M)))
    v = 0.6 * r.standard_normal((3, M, M, M))
    p = np.exp(0.3 * r.standard_normal((M, M, M)))
    W = np.stack([rho, v[0], v[1], v[2], p])
    U = np.empty_like(W)
    for z in range(M):
        for y in range(M):
            for x in range(M):
                U[:, z, y, x] = cons(W[:, z, y, x])
    return U


CASES = [(O.PPM, O.ROE, O.MINMOD), (O.PLM, O.HLLC, O.VANLEER), (O.PPM, O.EXACT, O.VANALBADA)]


def setup(recon, solver, lim, N=2, g=3, seed=11):
    Upad = tiny_group(N, g, seed)
    dx = (1.0, 0.7, 1.3)
    dt = O.cfl_dt(Upad[None], dx, 0.4, GAMMA)
    P = O.Params(scheme=O.CTU, recon=recon, riemann=solver, limiter=lim, fallback=O.HLLE, dt=dt, dx=dx,
                 gamma=GAMMA)
    Uo, flux, st = O.advance(P, Upad[None], N=N, ghost=g)
    assert int(st[0]) & ~ROE_FALLBACK == 0
    return P, Upad, Uo[0], flux[0]


@pytest.mark.parametrize("recon,solver,lim", CASES)
def test_ctu_cell_composed_face_by_face(recon, solver, lim):
    """N = 2, three ghost layers: every boundary-face flux the group step
    stores, and every updated cell, equal the face-by-face composition bit
    for bit (the oracle is built without floating-point contraction, and the
    numpy conversions here take its operations in the same order)."""
    N, g = 2, 3
    P, Upad, Uo, flux = setup(recon, solver, lim, N, g)
    C = Composer(P, Upad, N, g)
    # stored fluxes: flux[2d + side, v, a, b] on the face -1/2 (side 0) or
    # N-1/2 (side 1) along d; (a, b) = (z, y) for x, (z, x) for y, (y, x) for z
    for d in range(3):
        for side in range(2):
            cn = 0 if side == 0 else N
            for a in range(N):
                for b in range(N):
                    c = [(cn, b, a), (b, cn, a), (b, a, cn)][d]
                    F = C.face(c, d)
                    assert np.array_equal(flux[2 * d + side, :, a, b], F), (d, side, a, b)
    for z in range(N):
        for y in range(N):
            for x in range(N):
                assert np.array_equal(Uo[:, z, y, x], C.update(Upad, (x, y, z))), (x, y, z)


@pytest.mark.parametrize("plant", ["drop_second", "wrong_spacing", "swap_sides"])
def test_composition_detects_planted_mistakes(plant):
    """The comparison above is sharp: each planted wiring mistake in the
    composition moves the cell's update far beyond the tolerance."""
    N, g = 2, 3
    P, Upad, Uo, _ = setup(O.PPM, O.ROE, O.MINMOD, N, g)
    bad = Composer(P, Upad, N, g, plant=plant).update(Upad, (0, 1, 1))
    err = np.abs(bad - Uo[:, 1, 1, 0]).max() / np.abs(Uo).max()
    assert err > 1e-6
