"""Brute-force pins of the oracle's group step for the three unsplit schemes
(Sec. 2): the fluxes and updated cells of a tiny group, composed here face
by face from the oracle's single-cell pieces (line reconstruction,
characteristic tracing, one Riemann problem), must equal the whole-group
step's stored boundary fluxes and updated cells bit for bit.

The compositions follow each scheme's definition, not the group code's loop
order.  For the face between cells c - e_d and c along d the Riemann problem
takes the right-side state of c - e_d and the left-side state of c, where:
  * CTU: the face states along each direction are the reconstructed values
    traced to t + dt/2 (step (1)); stage-1 fluxes F1_e solve the Riemann
    problem between neighbours' traced states along e (step (2)); a state is
    corrected by the flux differences of the two other directions, each with
    dt/(2 dx_e) (step (3));
  * MHM: the six reconstructed face states of a cell, in conserved form, all
    move by the same half step -sum_e dt/(2 dx_e) (F_e(U_e+) - F_e(U_e-)) of
    their physical fluxes;
  * VL: first-order fluxes between cell averages give the half-step state
    U^{n+1/2} = U^n - sum_e dt/(2 dx_e) (F_e(c + e_e) - F_e(c)), which is
    reconstructed without tracing.
Then every cell moves by the flux differences times dt/dx_d (steps (4),
(5)).  Conversions between primitive and conserved variables, rotations
into a direction's frame and physical fluxes are written out in numpy.  The
spacings differ per axis, so a correction paired with the wrong axis's
dt/dx, a dropped term or swapped sides changes the answer, which the second
test shows by planting each of them here.
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


def phys_flux(W, U, d):
    """Physical flux along d of a global-frame state (W primitive, U conserved)."""
    w = to_local(W, d)
    mn = w[0] * w[1]
    f = np.array([mn, mn * w[1] + w[4], mn * w[2], mn * w[3], (U[4] + w[4]) * w[1]])
    return to_global(f, d)


def shifted(c, d, k):
    q = list(c)
    q[d] += k
    return tuple(q)


class Group:
    """One padded group and the pieces every scheme shares.  Cells are
    addressed by interior coordinates (x, y, z); ghosts are negative or
    >= N.  `plant` names a deliberate mistake (second test only)."""

    def __init__(self, P, Upad, N, g, plant=None):
        self.P, self.U, self.N, self.g, self.plant = P, Upad, N, g, plant
        self.S = 2 if P.recon == O.PPM else 1
        self.dtdx = [P.dt / P.dx[d] for d in range(3)]
        self.hdtdx = [0.5 * P.dt / P.dx[d] for d in range(3)]
        self._memo = {}

    def memo(self, key, make):
        if key not in self._memo:
            self._memo[key] = make()
        return self._memo[key]

    def Uc(self, c):
        g = self.g
        return self.U[:, c[2] + g, c[1] + g, c[0] + g]

    def Wc(self, c):
        return self.memo(("W", c), lambda: prim(self.Uc(c)))

    def line(self, Wof, c, d):
        """Primitive states Wof(cell) of the cells c - S e_d .. c + S e_d, [5][2S+1]."""
        S = self.S
        return np.stack([Wof(shifted(c, d, k)) for k in range(-S, S + 1)], axis=1)

    def recon(self, Wof, c, d):
        """Reconstructed face values (left, right) and slope of cell c along d."""
        WL, WR, sl = O.recon_line(self.P, d, self.line(Wof, c, d))
        S = self.S
        return WL[:, S], WR[:, S], sl[:, S]

    def solve(self, d, UL, UR):
        F, st = O.riemann(self.P.riemann, UL, UR, d, GAMMA, self.P.fallback)
        assert int(st) & ~ROE_FALLBACK == 0
        return F

    def face(self, c, d):
        """The flux on the face between c - e_d and c."""
        UL = self.state(shifted(c, d, -1), d, 1)
        UR = self.state(c, d, 0)
        if self.plant == "swap_sides":
            UL, UR = UR, UL
        return self.solve(d, UL, UR)

    def update(self, c):
        """Steps (4), (5): the new conserved state of cell c."""
        dU = np.zeros(5)
        for d in range(3):
            dU = dU + self.dtdx[d] * (self.face(shifted(c, d, 1), d) - self.face(c, d))
        return self.Uc(c) - dU


class CTU(Group):
    def traced(self, c, d):
        """Step (1): the conserved face states (left, right) of cell c along d."""
        def make():
            WL, WR, sl = self.recon(self.Wc, c, d)
            w0 = to_local(self.Wc(c), d)
            if self.P.recon == O.PPM:
                tl, tr = O.trace(O.PPM, w0, to_local(WL, d), to_local(WR, d), self.dtdx[d], GAMMA)
            else:
                tl, tr = O.trace(O.PLM, w0, to_local(sl, d), None, self.dtdx[d], GAMMA)
            return cons(to_global(tl, d)), cons(to_global(tr, d))
        return self.memo(("tr", c, d), make)

    def stage1(self, c, e):
        """Step (2): F1_e on the face between c - e_e and c."""
        return self.memo(("F1", c, e),
                         lambda: self.solve(e, self.traced(shifted(c, e, -1), e)[1], self.traced(c, e)[0]))

    def state(self, c, d, side):
        """Step (3): the traced state moved by the transverse flux differences."""
        u = self.traced(c, d)[side].copy()
        others = [e for e in range(3) if e != d]
        if self.plant == "drop_second":
            others = others[:1]
        for e in others:
            h = self.hdtdx[3 - d - e] if self.plant == "wrong_spacing" else self.hdtdx[e]
            u = u - h * (self.stage1(shifted(c, e, 1), e) - self.stage1(c, e))
        return u


class MHM(Group):
    def predicted(self, c):
        """The six face states of cell c, conserved, after the half step."""
        def make():
            Uf, Ff = [], []
            for e in range(3):
                WL, WR, _ = self.recon(self.Wc, c, e)
                pair = [cons(WL), cons(WR)]
                Uf.append(pair)
                Ff.append([phys_flux(WL, pair[0], e), phys_flux(WR, pair[1], e)])
            h = self.dtdx if self.plant == "full_step" else self.hdtdx
            S = h[0] * (Ff[0][1] - Ff[0][0]) + h[1] * (Ff[1][1] - Ff[1][0]) + h[2] * (Ff[2][1] - Ff[2][0])
            out = []
            for d in range(3):
                Sd = h[d] * (Ff[d][1] - Ff[d][0]) if self.plant == "own_direction_only" else S
                out.append([Uf[d][0] - Sd, Uf[d][1] - Sd])
            return out
        return self.memo(("pred", c), make)

    def state(self, c, d, side):
        return self.predicted(c)[d][side]


class VL(Group):
    def first_order(self, c, e):
        """Flux between the cell averages of c - e_e and c."""
        return self.memo(("F1", c, e), lambda: self.solve(e, self.Uc(shifted(c, e, -1)), self.Uc(c)))

    def Wh(self, c):
        """Primitive form of the half-step state U^{n+1/2} of cell c."""
        def make():
            h = [self.hdtdx[(e + 1) % 3] for e in range(3)] if self.plant == "wrong_spacing" else self.hdtdx
            dF = [self.first_order(shifted(c, e, 1), e) - self.first_order(c, e) for e in range(3)]
            return prim(self.Uc(c) - (h[0] * dF[0] + h[1] * dF[1] + h[2] * dF[2]))
        return self.memo(("Wh", c), make)

    def state(self, c, d, side):
        Wof = self.Wc if self.plant == "no_half_step" else self.Wh
        return cons(self.recon(Wof, c, d)[side])


def tiny_group(N, g, seed):
    """A rough, compressible, lognormal state on one padded group."""
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


COMPOSERS = {O.CTU: CTU, O.MHM: MHM, O.VL: VL}
CASES = [
    (O.CTU, O.PPM, O.ROE, O.MINMOD),
    (O.CTU, O.PLM, O.HLLC, O.VANLEER),
    (O.CTU, O.PPM, O.EXACT, O.VANALBADA),
    (O.MHM, O.PPM, O.ROE, O.MINMOD),
    (O.MHM, O.PLM, O.HLLE, O.HYBRID),
    (O.VL, O.PLM, O.HLLC, O.MINMOD),
    (O.VL, O.PPM, O.ROE, O.VANLEER),
    # characteristic-variable reconstruction (Sec. 2)
    (O.CTU, O.PPM, O.ROE, O.MINMOD, 1),
    (O.MHM, O.PLM, O.HLLC, O.VANALBADA, 1),
    (O.VL, O.PLM, O.ROE, O.VANLEER, 1),
]


def setup(scheme, recon, solver, lim, characteristic=0, N=2, seed=11):
    g = O.required_ghost(scheme, recon)
    Upad = tiny_group(N, g, seed)
    dx = (1.0, 0.7, 1.3)
    dt = O.cfl_dt(Upad[None], dx, 0.3, GAMMA)
    P = O.Params(scheme=scheme, recon=recon, riemann=solver, limiter=lim, fallback=O.HLLE, dt=dt, dx=dx,
                 gamma=GAMMA, characteristic=characteristic)
    Uo, flux, st = O.advance(P, Upad[None], N=N, ghost=g)
    assert int(st[0]) & ~ROE_FALLBACK == 0
    return P, Upad, g, Uo[0], flux[0]


def case_id(case):
    names = ({O.CTU: "ctu", O.MHM: "mhm", O.VL: "vl"}, {O.PLM: "plm", O.PPM: "ppm"},
             {O.EXACT: "exact", O.HLLE: "hlle", O.HLLC: "hllc", O.ROE: "roe"},
             {O.MINMOD: "minmod", O.VANLEER: "vanleer", O.VANALBADA: "vanalbada", O.HYBRID: "hybrid"})
    parts = [n[v] for n, v in zip(names, case)]
    return "-".join(parts + (["char"] if len(case) > 4 and case[4] else []))


@pytest.mark.parametrize("case", CASES, ids=case_id)
def test_cell_composed_face_by_face(case):
    """N = 2 with the scheme's ghost width: every boundary-face flux the
    group step stores, and every updated cell, equal the face-by-face
    composition bit for bit (the oracle is built without floating-point
    contraction, and the numpy arithmetic here takes its operations in the
    same order)."""
    N = 2
    P, Upad, g, Uo, flux = setup(*case, N=N)
    C = COMPOSERS[case[0]](P, Upad, N, g)
    # stored fluxes: flux[2d + side, v, a, b] on the face -1/2 (side 0) or
    # N-1/2 (side 1) along d; (a, b) = (z, y) for x, (z, x) for y, (y, x) for z
    for d in range(3):
        for side in range(2):
            cn = 0 if side == 0 else N
            for a in range(N):
                for b in range(N):
                    c = [(cn, b, a), (b, cn, a), (b, a, cn)][d]
                    assert np.array_equal(flux[2 * d + side, :, a, b], C.face(c, d)), (d, side, a, b)
    for z in range(N):
        for y in range(N):
            for x in range(N):
                assert np.array_equal(Uo[:, z, y, x], C.update((x, y, z))), (x, y, z)


PLANTS = [
    (O.CTU, "drop_second"), (O.CTU, "wrong_spacing"), (O.CTU, "swap_sides"),
    (O.MHM, "full_step"), (O.MHM, "own_direction_only"), (O.MHM, "swap_sides"),
    (O.VL, "no_half_step"), (O.VL, "wrong_spacing"), (O.VL, "swap_sides"),
]


@pytest.mark.parametrize("scheme,plant", PLANTS)
def test_composition_detects_planted_mistakes(scheme, plant):
    """The comparison above is sharp: each planted wiring mistake in a
    composition moves the cell's update far beyond rounding."""
    case = next(c for c in CASES if c[0] == scheme)
    N = 2
    P, Upad, g, Uo, _ = setup(*case, N=N)
    bad = COMPOSERS[scheme](P, Upad, N, g, plant=plant).update((0, 1, 1))
    err = np.abs(bad - Uo[:, 1, 1, 0]).max() / np.abs(Uo).max()
    assert err > 1e-6
