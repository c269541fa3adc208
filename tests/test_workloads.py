"""Host logic of the seeded input generators that the chained prepared-group
path relies on (no device): the column order of a tiling, the runs of
z-continuations, and the AMR-shaped batch's runs, whose linked groups must
hold each other's interiors in their ghost planes (the property under which
a chain of prepared groups reproduces the groups advanced alone)."""
import numpy as np

from paper_1103_3373_gb300 import runtime as RT
from paper_1103_3373_gb300 import workloads as W


def test_column_origins_is_the_tiling_z_fastest():
    a = W.group_origins(48, 32, 64, 16)
    b = W.column_origins(48, 32, 64, 16)
    assert sorted(map(tuple, a)) == sorted(map(tuple, b))
    # z fastest: consecutive entries of a column differ by one group along z
    GZ = 64 // 16
    for c in range(len(b) // GZ):
        col = b[c * GZ:(c + 1) * GZ]
        assert (col[:, 0] == col[0, 0]).all() and (col[:, 1] == col[0, 1]).all()
        assert list(col[:, 2]) == [16 * k for k in range(GZ)]


def test_runs_from_links():
    assert list(W.runs_from_links([])) == []
    assert list(W.runs_from_links([False])) == [1]
    assert list(W.runs_from_links([True, True, False, True, False])) == [3, 2, 1, 2, 1]
    assert list(W.runs_from_links([True, False, True, True, False, False])) == [2, 1, 3, 2, 1, 1]


def test_amr_batch_runs_link_matching_ghost_planes():
    N, g = 16, 3
    for counts, n0 in (((40, 24, 16, 8), 32), ((70, 20, 13, 5), 32)):
        levels = W.amr_levels(counts=counts, n0=n0, seed=5)
        for lv, G in zip(levels, counts):
            U, z = lv["U"], lv["zrun"]
            assert len(z) == G and (z >= 1).all()
            assert z[-1] == 1 and z.max() >= 2
            for k in range(G - 1):
                # a run counts down by one group at a time
                assert z[k] == 1 or z[k + 1] == z[k] - 1
                if z[k] >= 2:
                    a, b = U[k], U[k + 1]
                    assert np.array_equal(a[:, N + g:N + 2 * g], b[:, g:2 * g])  # top ghosts = interior above
                    assert np.array_equal(a[:, N:N + g], b[:, 0:g])              # bottom ghosts of the upper one


def test_hierarchy_levels_run_by_column():
    """Every level of the hierarchy workload lists its groups column by column,
    so runtime.zrun_of finds runs of z-neighbours; zrun_of itself follows the
    definition on a hand-made list."""
    o = np.asarray([(0, 0, 0), (0, 0, 16), (0, 0, 32), (16, 0, 0), (16, 0, 32), (16, 0, 48)], dtype=np.int32)
    assert list(RT.zrun_of(o)) == [3, 2, 1, 1, 2, 1]
    assert list(RT.zrun_of(o[:0])) == []
    for lv in W.amr_hierarchy(64, (0.3, 0.12)):
        o = lv["origin"]
        key = [(y, x, z) for x, y, z in o]
        assert key == sorted(key)
        z = RT.zrun_of(o)
        assert z.max() >= 2 and z[-1] == 1
