"""AMR level operations of the FP64 oracle — TEST INFRASTRUCTURE.

Same import rule as the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and the
``--impl reference`` arm) may use it; the product package never does.

The paper names three operations around the patch-group solver without
giving their formulas:
  * the preparation step fills the ghost zones of patch groups next to a
    coarse-fine boundary by spatial and temporal interpolation of the coarser
    level (Sec. 4.2);
  * the fluxes stored across the patch-group boundaries (Sec. 2 step (5))
    correct the coarse-grid data (Sec. 4.3 lists "correcting the coarse-grid
    data" among the CPU tasks);
  * the coarse cells covered by finer ones take the finer data.
This module writes each of them out cell by cell in numpy (FP64), with these
readings:
  * refinement ratio 2 in space and time: dx_l = dx_0 / 2^l, the finer level
    takes two substeps of dt/2 per step of its parent;
  * refinement unit: one whole coarse patch group, refined into the 8 fine
    groups covering it (an "octet"), so every coarse-fine face lies on a
    coarse group face, where step (5) stored the coarse flux;
  * proper nesting: every cell a fine ghost zone or its interpolation stencil
    needs exists at the fine or the parent level (checked, NestingError);
  * spatial interpolation (prolongation): per conserved component, the parent
    value plus a quarter of the minmod-limited central difference per axis,
    with the sign of the child's offset; the 8 children average to the
    parent:  u = ((Uc + qx) + qy) + qz,  q_d = (s_d / 4) minmod(Uc[+1] - Uc,
    Uc - Uc[-1]),  s_d = -1 for the lower child, +1 for the upper;
  * temporal interpolation: linear in time between the parent's state before
    and after its step, Uc(theta) = U^n + theta (U^{n+1} - U^n), theta = 0 for
    the first substep and 1/2 for the second;
  * flux correction (refluxing, Berger & Colella 1989): the unrefined coarse
    cell next to a coarse-fine face replaces the coarse flux of that face by
    the mean of the 2 x 2 fine face fluxes over the 2 substeps:
      Fbar = 0.125 (S0 + S1),
      Sk = ((Fk[a0,b0] + Fk[a0,b1]) + Fk[a1,b0]) + Fk[a1,b1]   (substep k),
      U += -h (Fbar - Fc)  if the face is the cell's +d face,
      U += +h (Fbar - Fc)  if it is the cell's -d face,   h = dt / dx_d,
    faces taken in the order -x, +x, -y, +y, -z, +z;
  * restriction: coarse cell = 0.125 x the sum of its 8 fine cells, summed in
    the order (dz, dy, dx) = 000, 001, 010, 011, 100, 101, 110, 111.

Boundary-flux arrays are [G][6][5][N][N], faces -x,+x,-y,+y,-z,+z, indexed
[a][b] = [z][y] on x faces, [z][x] on y faces, [y][x] on z faces (the layout
of step (5) in both the oracle and the library).

A level is a dict: U [G][5][N][N][N] (interior data), origin [G][3] (x, y, z
interior corner in the level's cells, multiples of N), box (X, Y, Z) (the
level's extent in cells: 2^l times the base box).
"""
import numpy as np


class NestingError(ValueError):
    pass


def group_map(origin, box, N=16):
    """[GZ][GY][GX] group index at each slot of the level box, -1 if empty."""
    X, Y, Z = box
    m = -np.ones((Z // N, Y // N, X // N), dtype=np.int64)
    for k, (x, y, z) in enumerate(np.asarray(origin)):
        assert x % N == 0 and y % N == 0 and z % N == 0
        assert m[z // N, y // N, x // N] < 0, "two groups on one slot"
        m[z // N, y // N, x // N] = k
    return m


def _cell(f, n, bc):
    """Box-edge map of integer cell coordinates: periodic wrap or outflow clamp."""
    return np.mod(f, n) if bc == 0 else np.clip(f, 0, n - 1)


def _minmod(a, b):
    return np.where(a * b > 0.0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)


def _values(level, U, x, y, z, N):
    """Values [n][5] of the level at in-box cell coordinates (arrays)."""
    m = group_map(level["origin"], level["box"], N)
    g = m[z // N, y // N, x // N]
    if np.any(g < 0):
        raise NestingError("cell not covered by the level")
    return U[g, :, z % N, y % N, x % N]


def prolong(coarse, coarse_new, theta, fx, fy, fz, bc=0, N=16):
    """Interpolated values [n][5] at fine cells (fx, fy, fz), which must lie in
    the fine box (2x the coarse box), from the coarse level at time theta of
    its step (coarse_new = its data after the step, or None for theta = 0)."""
    Xc, Yc, Zc = coarse["box"]
    U0 = coarse["U"]

    def at(x, y, z):
        u0 = _values(coarse, U0, x, y, z, N)
        if coarse_new is None:
            return u0
        u1 = _values(coarse, coarse_new, x, y, z, N)
        return u0 + theta * (u1 - u0)

    fx, fy, fz = (np.asarray(a, dtype=np.int64) for a in (fx, fy, fz))
    cx, cy, cz = fx // 2, fy // 2, fz // 2
    uc = at(cx, cy, cz)
    out = uc.copy()
    for d, (f, n) in enumerate(((fx, Xc), (fy, Yc), (fz, Zc))):
        step = [cx, cy, cz]
        up = list(step)
        dn = list(step)
        up[d] = _cell(step[d] + 1, n, bc)
        dn[d] = _cell(step[d] - 1, n, bc)
        delta = _minmod(at(*up) - uc, uc - at(*dn))
        s = np.where(f % 2 == 1, 1.0, -1.0)
        out = out + (0.25 * s)[:, None] * delta
    return out


def prepare(fine, coarse=None, coarse_new=None, theta=0.0, ghost=3, bc=0, N=16):
    """Halo-padded input [G][5][M][M][M] (M = N + 2 ghost) of every group of
    the fine level: cells inside a group of the same level are copied from it,
    all others are interpolated from the parent level at time theta."""
    Uf, of = fine["U"], np.asarray(fine["origin"])
    X, Y, Z = fine["box"]
    mf = group_map(of, fine["box"], N)
    M = N + 2 * ghost
    G = len(of)
    out = np.empty((G, 5, M, M, M))
    r = np.arange(M) - ghost
    for k in range(G):
        fx = _cell(of[k, 0] + r, X, bc)
        fy = _cell(of[k, 1] + r, Y, bc)
        fz = _cell(of[k, 2] + r, Z, bc)
        FZ, FY, FX = np.meshgrid(fz, fy, fx, indexing="ij")
        gk = mf[FZ // N, FY // N, FX // N]
        have = gk >= 0
        block = np.empty((5, M, M, M))
        block[:, have] = Uf[gk[have], :, FZ[have] % N, FY[have] % N, FX[have] % N].T
        if np.any(~have):
            if coarse is None:
                raise NestingError("ghost cell outside the base level")
            block[:, ~have] = prolong(coarse, coarse_new, theta, FX[~have], FY[~have], FZ[~have], bc, N).T
        out[k] = block
    return out


def _face_ab(d, x, y, z):
    """Transverse indices (a, b) of the face arrays along direction d."""
    if d == 0:
        return z, y
    if d == 1:
        return z, x
    return y, x


def reflux(coarse, coarse_new, coarse_flux, fine, fine_flux0, fine_flux1, dt, dx, bc=0, N=16):
    """Coarse data after its step (coarse_new [Gc][5][N^3]) with every
    unrefined cell next to a coarse-fine face corrected by the fine fluxes of
    the two substeps (returns a corrected copy)."""
    oc = np.asarray(coarse["origin"])
    Xc, Yc, Zc = coarse["box"]
    nc = (Xc, Yc, Zc)
    of = np.asarray(fine["origin"])
    mf = group_map(of, fine["box"], N)
    out = np.array(coarse_new, dtype=np.float64, copy=True)
    idx = np.arange(N)

    def refined(slot):
        sx, sy, sz = slot
        return mf[2 * sz, 2 * sy, 2 * sx] >= 0

    for q in range(len(oc)):
        slot = oc[q] // N
        if refined(slot):
            continue
        for d in range(3):
            h = dt / dx[d]
            for side in range(2):  # 0: the group's -d face, 1: its +d face
                nb = list(slot)
                nb[d] = slot[d] + (1 if side else -1)
                ng = nc[d] // N
                if bc == 0:
                    nb[d] %= ng
                elif nb[d] < 0 or nb[d] >= ng:
                    continue  # domain boundary: no coarse-fine face
                if not refined(nb):
                    continue
                # coarse cells of q on this face, as (a, b) grids
                A, B = np.meshgrid(idx, idx, indexing="ij")
                cl = [None, None, None]
                cl[d] = np.full_like(A, N - 1 if side else 0)
                t1, t2 = [e for e in range(3) if e != d]
                # (a, b) = [z][y] for x faces, [z][x] for y faces, [y][x] for z
                # faces: a is the larger transverse axis index
                cl[t2] = A
                cl[t1] = B
                Fc = coarse_flux[q, 2 * d + side][:, A, B]  # [5][N][N]
                # fine cells across the face (inside the refined neighbour)
                gc = [oc[q][e] + cl[e] for e in range(3)]  # global coarse coordinates
                fd = 2 * nb[d] * N + (2 * N - 1 if side == 0 else 0)
                fsum = None
                for F in (fine_flux0, fine_flux1):
                    acc = None
                    for da in range(2):
                        for db in range(2):
                            fc = [None, None, None]
                            fc[d] = np.full_like(A, fd)
                            fc[t2] = 2 * gc[t2] + da
                            fc[t1] = 2 * gc[t1] + db
                            k = mf[fc[2] // N, fc[1] // N, fc[0] // N]
                            if np.any(k < 0):
                                raise NestingError("refined neighbour without its octet")
                            a, b = _face_ab(d, fc[0] % N, fc[1] % N, fc[2] % N)
                            # the fine cell's face toward the coarse cell
                            ff = 2 * d + (1 if side == 0 else 0)
                            val = F[k, ff, :, a, b].transpose(2, 0, 1)  # [5][N][N]
                            acc = val if acc is None else acc + val
                    fsum = acc if fsum is None else fsum + acc
                Fbar = 0.125 * fsum
                corr = h * (Fbar - Fc)
                sgn = -1.0 if side else 1.0
                cz, cy, cx = cl[2], cl[1], cl[0]
                out[q][:, cz, cy, cx] = out[q][:, cz, cy, cx] + sgn * corr
    return out


def restrict(fine, coarse, coarse_new, N=16):
    """Coarse data with the cells covered by fine groups replaced by the mean of
    their 8 fine cells (returns a corrected copy of coarse_new)."""
    oc = np.asarray(coarse["origin"])
    mc = group_map(oc, coarse["box"], N)
    out = np.array(coarse_new, dtype=np.float64, copy=True)
    H = N // 2
    for k, o in enumerate(np.asarray(fine["origin"])):
        c0 = o // 2
        q = mc[c0[2] // N, c0[1] // N, c0[0] // N]
        if q < 0:
            raise NestingError("fine group without a parent group")
        off = c0 - oc[q]
        f = fine["U"][k]
        acc = None
        for dz in range(2):
            for dy in range(2):
                for dx_ in range(2):
                    t = f[:, dz::2, dy::2, dx_::2]
                    acc = t.copy() if acc is None else acc + t
        out[q][:, off[2]:off[2] + H, off[1]:off[1] + H, off[0]:off[0] + H] = 0.125 * acc
    return out


def check_octets(fine, N=16):
    """Every fine group belongs to a complete octet (the 8 groups refining one
    coarse group)."""
    mf = group_map(fine["origin"], fine["box"], N)
    for o in np.asarray(fine["origin"]):
        base = (o // N) // 2 * 2
        for dz in range(2):
            for dy in range(2):
                for dx_ in range(2):
                    if mf[base[2] + dz, base[1] + dy, base[0] + dx_] < 0:
                        raise NestingError("incomplete octet")


def amr_step(levels, params, dt0, bc=0, N=16, ghost=None, reflux_on=True, advance=None):
    """One step of the whole hierarchy (levels[0] the base level covering the
    box), recursively: advance level l by dt_l, then its finer level twice by
    dt_l / 2 (ghost zones at theta = 0 and 1/2 of level l's step), then
    correct level l with the fine fluxes and restrict the fine data onto it.
    `params` is an oracle.Params (dt and dx are set per level); `advance`
    defaults to oracle.advance.  Returns the new data of every level."""
    from . import advance as _advance
    from . import required_ghost
    adv = advance or _advance
    g = ghost if ghost is not None else required_ghost(params.scheme, params.recon)
    L = len(levels)
    for l in range(1, L):
        check_octets(levels[l], N)
    cur = [np.array(lv["U"], dtype=np.float64, copy=True) for lv in levels]

    def lev(l, U):
        return dict(U=U, origin=levels[l]["origin"], box=levels[l]["box"])

    def step(l, dt, parent_old, parent_new, theta):
        dx = levels[l]["dx"]
        Ug = prepare(lev(l, cur[l]), None if l == 0 else lev(l - 1, parent_old), parent_new, theta, g, bc, N)
        params.dt = dt
        params.dx = tuple(dx)
        U_new, flux, _ = adv(params, Ug, N)
        if l + 1 < L:
            U_old = cur[l]
            ff = [step(l + 1, 0.5 * dt, U_old, U_new, 0.0), step(l + 1, 0.5 * dt, U_old, U_new, 0.5)]
            if reflux_on:
                U_new = reflux(lev(l, U_old), U_new, flux, lev(l + 1, cur[l + 1]), ff[0], ff[1], dt, dx, bc, N)
            U_new = restrict(lev(l + 1, cur[l + 1]), lev(l, U_old), U_new, N)
        cur[l] = U_new
        return flux

    step(0, dt0, None, None, 0.0)
    return cur
