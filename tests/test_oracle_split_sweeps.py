"""Brute-force pin of the oracle's split-scheme group step (RTVD and WAF, the
directionally split schemes Sec. 3.2 compares with): on a periodic box that is
one group, the group step with its ghost-limited sweeps must equal three
sweeps of the whole periodic box, each sweep every row of the box along its
direction with the full dt, in the order x, y, z (or z, y, x for the other
half of a Strang pair).

The group step sweeps only the rows that later sweeps read (the transverse
ranges widen by the ghost width along the axes still to come); the whole-box
composition sweeps every row, so a range too narrow, a sweep out of order or
a spacing paired with the wrong axis shows up as a difference.  Both sides
run the oracle's own single-row sweep; what is pinned is the group step's
orchestration and its stored boundary fluxes, bit for bit.
"""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import workloads as W

MOM = [(1, 2, 3), (2, 3, 1), (3, 1, 2)]  # local frame: normal momentum second


def to_local(a, d):
    n, t1, t2 = MOM[d]
    return a[[0, n, t1, t2, 4]]


def to_global(b, d):
    n, t1, t2 = MOM[d]
    a = np.empty_like(b)
    a[[0, n, t1, t2, 4]] = b
    return a


def sweep_box(P, U, d, g, dx):
    """Every row of the periodic box U [5, Z, Y, X] along d, padded with g
    periodic cells on each side, advanced by one sweep.  Returns the new box
    and the fluxes through the faces -1/2 and N-1/2 of each row, [2, 5, ...]
    indexed by the two transverse coordinates (larger axis first)."""
    axis = 3 - d  # numpy axis of direction d in [v, z, y, x]
    Ul = np.moveaxis(U, axis, -1)  # [5, a, b, n] with (a, b) the transverse axes, larger first
    N = Ul.shape[-1]
    out = np.empty_like(Ul)
    flux = np.empty((2, 5) + Ul.shape[1:3])
    for a in range(Ul.shape[1]):
        for b in range(Ul.shape[2]):
            row = np.take(Ul[:, a, b, :], np.arange(-g, N + g), axis=-1, mode="wrap")
            loc = np.stack([to_local(row[:, j], d) for j in range(N + 2 * g)])
            new, flo, fhi = O.split_row(P, loc, g, g + N, dx)
            for j in range(N):
                out[:, a, b, j] = to_global(new[g + j], d)
            flux[0, :, a, b] = to_global(flo, d)
            flux[1, :, a, b] = to_global(fhi, d)
    return np.moveaxis(out, -1, axis), flux


def compose(P, U, g, order, dx):
    fluxes = {}
    for d in order:
        U, fluxes[d] = sweep_box(P, U, d, g, dx[d])
    return U, fluxes


def setup(scheme, split_order, N=4, seed=21):
    U = W.lognormal(N, seed=seed, mach=1.2, sigma=0.4)
    dx = (1.0, 0.8, 1.25)
    dt = O.cfl_dt(U, dx, 0.3)
    g = O.required_ghost(scheme, O.PLM)
    P = O.Params(scheme=scheme, limiter=O.VANLEER, riemann=O.HLLC, dt=dt, dx=dx, split_order=split_order)
    return U, dx, g, P


@pytest.mark.parametrize("scheme", [O.RTVD, O.WAF])
@pytest.mark.parametrize("split_order", [0, 1])
def test_group_step_equals_whole_box_sweeps(scheme, split_order):
    N = 4
    U, dx, g, P = setup(scheme, split_order, N)
    Ug = O.gather(U, np.zeros((1, 3), dtype=np.int32), N, g, bc=0)
    Uo, flux, st = O.advance(P, Ug, N, ghost=g)
    assert st[0] == 0
    order = (0, 1, 2) if split_order == 0 else (2, 1, 0)
    Uc, fl = compose(P, U, g, order, dx)
    assert np.array_equal(Uo[0], Uc)
    for d in range(3):
        # stored as flux[2d + side, v, a, b], a the larger transverse axis
        assert np.array_equal(flux[0, 2 * d], fl[d][0]), d
        assert np.array_equal(flux[0, 2 * d + 1], fl[d][1]), d


@pytest.mark.parametrize("plant", ["order", "spacing"])
def test_composition_detects_planted_mistakes(plant):
    """A sweep order other than the stated one, or a sweep using another
    axis's spacing, moves the result far beyond rounding."""
    N = 4
    U, dx, g, P = setup(O.RTVD, 0, N)
    Ug = O.gather(U, np.zeros((1, 3), dtype=np.int32), N, g, bc=0)
    Uo = O.advance(P, Ug, N, ghost=g)[0][0]
    if plant == "order":
        Uc, _ = compose(P, U, g, (0, 2, 1), dx)
    else:
        Uc, _ = compose(P, U, g, (0, 1, 2), (dx[0], dx[2], dx[1]))
    assert np.abs(Uc - Uo).max() / np.abs(Uo).max() > 1e-6
