"""Host logic of the end-to-end pipeline (Sec. 4.1: copies of chunks of
patch groups overlapped with the solver): the copy plan that
hydro_pipeline_create makes, checked on the CPU for every slab partition of
small boxes.

* the slab boundaries are whole group layers covering the box;
* every plane is copied exactly once;
* when slab s is advanced, the chunks copied so far hold every plane it
  reads: its own planes and `ghost` planes on each side, wrapped (periodic)
  or clamped (outflow) at the box edge.
"""
import itertools
import os
import shutil

import pytest

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="no nvcc")


def _partitions(gz, max_parts=5):
    for k in range(1, min(gz, max_parts) + 1):
        for cut in itertools.combinations(range(1, gz), k - 1):
            b = (0,) + cut + (gz,)
            yield [b[i + 1] - b[i] for i in range(k)]


def _needed(zb, s, g, Z, bc):
    lo, hi = zb[s] - g, zb[s + 1] + g
    if bc == 0:
        return {z % Z for z in range(lo, hi)}
    return {min(max(z, 0), Z - 1) for z in range(lo, hi)}


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("gz,g", [(1, 3), (2, 2), (4, 3), (5, 4), (7, 3)])
def test_every_partition_completes_each_slab_halo(bc, gz, g):
    from paper_1103_3373_gb300 import hydro as H
    N = 16
    Z = gz * N
    for layers in _partitions(gz):
        zb, chunks = H.pipeline_plan(Z, g, bc=bc, slabs=layers, N=N)
        assert zb[0] == 0 and zb[-1] == Z
        assert [zb[i + 1] - zb[i] for i in range(len(layers))] == [N * a for a in layers]
        copied = []
        have = set()
        for s in range(len(layers)):
            for lo, hi in chunks[s]:
                assert 0 <= lo < hi <= Z
                copied.extend(range(lo, hi))
                have.update(range(lo, hi))
            assert _needed(zb, s, g, Z, bc) <= have, (layers, s)
        assert sorted(copied) == list(range(Z)), layers


def test_even_split_and_errors():
    from paper_1103_3373_gb300 import hydro as H
    zb, chunks = H.pipeline_plan(256, 3, slabs=8)
    assert zb == [32 * s for s in range(9)]
    assert chunks[0] == [(253, 256), (0, 35)] and chunks[-1] == [(227, 253)]
    zb, chunks = H.pipeline_plan(256, 3, bc=H.BC_OUTFLOW, slabs=2)
    assert chunks == [[(0, 131)], [(131, 256)]]
    for bad in (dict(slabs=0), dict(slabs=17), dict(slabs=(2, 2)), dict(slabs=(16, 0))):
        with pytest.raises(H.HydroError):
            H.pipeline_plan(256, 3, **bad)
    with pytest.raises(H.HydroError):
        H.pipeline_plan(256, 16, slabs=2)  # ghost >= N


def test_device_field_rotation_chains_every_step():
    """The three-field rotation of HostBoxStepper meets the chaining
    condition of hydro_pipeline_step at every step: the next input is
    neither of the last step's fields, and the next output differs from the
    last output (so the last output can still be copied out)."""
    from paper_1103_3373_gb300 import runtime as RT
    for n in range(12):
        i0, o0 = RT.rotation(n)
        i1, o1 = RT.rotation(n + 1)
        assert len({i0, o0}) == 2 and len({i1, o1}) == 2
        assert i1 not in (i0, o0) and o1 != o0
