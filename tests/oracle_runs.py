"""Helpers that drive the oracle over whole boxes (test support only)."""
import numpy as np

import oracle as O
from paper_1103_3373_gb300 import workloads as W


def oracle_box_step(U, P, N, g, bc):
    """One oracle step of a whole field [5,Z,Y,X] tiled by N^3 groups."""
    _, Z, Y, X = U.shape
    orig = W.group_origins(X, Y, Z, N)
    Ug = O.gather(U, orig, N, g, bc=bc)
    Uo, fl, st = O.advance(P, Ug, N)
    return W.scatter_groups(Uo, X, Y, Z), fl, st


def oracle_run(U, P, N, g, bc, steps, cfl=None, dt=None, t_end=None):
    """Several steps; dt from the CFL condition unless given.  Returns (U, t, status_or)."""
    t = 0.0
    st_all = 0
    for _ in range(steps):
        if dt is None:
            step_dt = O.cfl_dt(U, P.dx, cfl, P.gamma, P.dens_floor, P.pres_floor)
        else:
            step_dt = dt
        if t_end is not None:
            if t >= t_end * (1 - 1e-14):
                break
            step_dt = min(step_dt, t_end - t)
        P.dt = step_dt
        U, _, st = oracle_box_step(U, P, N, g, bc)
        st_all |= int(np.bitwise_or.reduce(st))
        t += step_dt
    return U, t, st_all
