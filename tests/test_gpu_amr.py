"""GPU parity of the AMR level operations (include/hydro_amr.h) and of whole
hierarchy steps (runtime.AmrHierarchy) against the oracle (oracle/amr.py),
through the C ABI:

* group maps equal the oracle's; duplicate slots and misaligned origins set
  their error bits;
* ghost-zone preparation (copy, spatial and temporal interpolation),
  refluxing and restriction element by element (FP64 bit-exact: same
  expressions in the same order, -fmad=false; FP32 within 1e-6 relative);
* a 2-level CTU+PPM+Roe and a 3-level MHM+PLM+HLLE hierarchy step against
  oracle.amr.amr_step (FP64 <= 1e-12, FP32 <= 1e-5 relative L1 per level),
  two steps in a row, and the CUDA-graph replay equal to the eager steps;
* a fine level whose ghost zone needs a cell the parent level lacks sets
  HYDRO_AMR_ENESTING and writes NaN there (no fault, no trap).
"""
import numpy as np
import pytest

import oracle as O
from oracle import amr as A
from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import runtime as RT
from paper_1103_3373_gb300 import workloads as W
from tests.gpu_common import assert_close, params_pair, quantise, tdtype

pytestmark = pytest.mark.gpu
N = 16


def _torch():
    import torch
    return torch


def _dev_level(lv, prec, U=None, err=None):
    torch = _torch()
    dev = torch.device("cuda:0")
    origin = torch.tensor(np.asarray(lv["origin"], dtype=np.int32), device=dev)
    X, Y, Z = lv["box"]
    m = torch.empty((Z // N, Y // N, X // N), dtype=torch.int32, device=dev)
    H.hydro_amr_map(origin, lv["box"], m, error=err)
    Ut = torch.tensor(lv["U"] if U is None else U, dtype=tdtype(prec), device=dev)
    return H.AmrLevel(U=Ut, origin=origin, map=m, box=lv["box"])


def _close(got, ref, prec):
    if prec == H.FP64:
        np.testing.assert_array_equal(got, ref)
    else:
        np.testing.assert_allclose(got, ref, rtol=2e-6, atol=2e-6 * np.abs(ref).max())


def test_group_maps_and_error_bits():
    torch = _torch()
    for lv in W.amr_hierarchy(64, (0.3, 0.12)):
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        dl = _dev_level(lv, H.FP64, err=err)
        np.testing.assert_array_equal(dl.map.cpu().numpy(), A.group_map(lv["origin"], lv["box"]))
        assert err.item() == 0
    m = torch.empty((2, 2, 2), dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    org = torch.tensor([[0, 0, 0], [16, 0, 0], [0, 0, 0]], dtype=torch.int32, device="cuda")
    H.hydro_amr_map(org, (32, 32, 32), m, error=err)
    assert err.item() & H.AMR_EDUPLICATE
    err.zero_()
    org = torch.tensor([[8, 0, 0], [16, 16, 16]], dtype=torch.int32, device="cuda")
    H.hydro_amr_map(org, (32, 32, 32), m, error=err)
    assert err.item() & H.AMR_ENESTING
    assert m[1, 1, 1].item() == 1 and (m >= 0).sum().item() == 1


@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
@pytest.mark.parametrize("bc", [H.BC_PERIODIC, H.BC_OUTFLOW])
def test_prepare_matches_oracle(prec, bc):
    torch = _torch()
    levels = W.amr_hierarchy(48, (0.25,), center=(0.2, 0.5, 0.6))
    rng = np.random.default_rng(1)
    Uc = quantise(levels[0]["U"], prec)
    Uc_new = quantise(Uc * (1.0 + 0.02 * rng.standard_normal(Uc.shape)), prec)
    Uf = quantise(levels[1]["U"], prec)
    g = 3
    M = N + 2 * g
    dl0 = _dev_level(levels[0], prec, Uc)
    dl1 = _dev_level(levels[1], prec, Uf)
    cnew = torch.tensor(Uc_new, dtype=tdtype(prec), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    cases = [(0, None, None, 0.0), (1, 0, None, 0.0), (1, 0, Uc_new, 0.5)]
    for (l, c, cn, theta) in cases:
        fine = dict(U=Uc if l == 0 else Uf, origin=levels[l]["origin"], box=levels[l]["box"])
        coarse = None if c is None else dict(U=Uc, origin=levels[0]["origin"], box=levels[0]["box"])
        ref = A.prepare(fine, coarse, cn, theta, ghost=g, bc=bc)
        out = torch.full((len(levels[l]["origin"]), 5, M, M, M), float("nan"), dtype=tdtype(prec), device="cuda")
        H.hydro_amr_prepare(dl0 if l == 0 else dl1, None if c is None else dl0, None if cn is None else cnew, theta,
                            out, bc=bc, ghost=g, precision=prec, error=err)
        torch.cuda.synchronize()
        _close(out.double().cpu().numpy(), ref, prec)
    assert err.item() == 0


@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
@pytest.mark.parametrize("bc", [H.BC_PERIODIC, H.BC_OUTFLOW])
def test_reflux_and_restrict_match_oracle(prec, bc):
    torch = _torch()
    # the refined block sits at the low-x box edge: with periodic edges the
    # groups at the high-x edge are its neighbours, with outflow they are not
    levels = W.amr_hierarchy(64, (0.2,), center=(0.125, 0.5, 0.5))
    assert len(levels) == 2
    rng = np.random.default_rng(2)
    Gc, Gf = len(levels[0]["origin"]), len(levels[1]["origin"])
    Uc = quantise(levels[0]["U"], prec)
    cflux = quantise(rng.standard_normal((Gc, 6, 5, N, N)), prec)
    ff = [quantise(rng.standard_normal((Gf, 6, 5, N, N)), prec) for _ in range(2)]
    Uf = quantise(rng.standard_normal((Gf, 5, N, N, N)) + 3.0, prec)
    dt, dx = 0.003, (1 / 64, 1 / 60, 1 / 70)
    coarse = dict(U=Uc, origin=levels[0]["origin"], box=levels[0]["box"])
    fine = dict(U=Uf, origin=levels[1]["origin"], box=levels[1]["box"])
    ref = A.reflux(coarse, Uc, cflux, fine, ff[0], ff[1], dt, dx, bc=bc)
    assert not np.array_equal(ref, Uc)
    dc = _dev_level(levels[0], prec, Uc)
    df = _dev_level(levels[1], prec, Uf)
    tt = lambda a: torch.tensor(a, dtype=tdtype(prec), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.hydro_amr_reflux(dc, tt(cflux), df, tt(ff[0]), tt(ff[1]), dt, dx, bc=bc, precision=prec, error=err)
    torch.cuda.synchronize()
    _close(dc.U.double().cpu().numpy(), ref, prec)
    ref2 = A.restrict(fine, coarse, ref)
    H.hydro_amr_restrict(df, dc, precision=prec, error=err)
    torch.cuda.synchronize()
    _close(dc.U.double().cpu().numpy(), ref2, prec)
    assert err.item() == 0


def _quantised_levels(levels, prec):
    return [dict(lv, U=quantise(lv["U"], prec)) for lv in levels]


@pytest.mark.parametrize("case", ["ctu_2_levels", "mhm_3_levels"])
@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
def test_hierarchy_steps_match_oracle(case, prec):
    torch = _torch()
    if case == "ctu_2_levels":
        levels = _quantised_levels(W.amr_hierarchy(48, (0.2,)), prec)
        po, ph = params_pair(O.CTU, O.PPM, O.ROE, prec, 0.0, (1, 1, 1))
    else:
        levels = _quantised_levels(W.amr_hierarchy(64, (0.3, 0.12)), prec)
        po, ph = params_pair(O.MHM, O.PLM, O.HLLE, prec, 0.0, (1, 1, 1))
    dt0 = 0.3 * levels[0]["dx"][0] / 3.0
    hier = RT.AmrHierarchy(levels, ph)
    ref_levels = [dict(lv) for lv in levels]
    for step in range(2):
        ref = A.amr_step(ref_levels, po, dt0)
        hier.step(dt0)
        torch.cuda.synchronize()
        for l in range(len(levels)):
            got = hier.cur[l].double().cpu().numpy()
            assert_close(got, ref[l], prec, "level %d step %d" % (l, step))
            if prec == H.FP64:
                np.testing.assert_array_equal(got, ref[l])
        # the next oracle step starts from the GPU's state (FP32: the stored values)
        ref_levels = [dict(lv, U=hier.cur[l].double().cpu().numpy()) for l, lv in enumerate(levels)]
    assert hier.errors() == 0


def test_hierarchy_graph_replay_equals_eager_steps():
    torch = _torch()
    levels = _quantised_levels(W.amr_hierarchy(64, (0.3, 0.12)), H.FP32)
    _, ph = params_pair(O.CTU, O.PPM, O.ROE, H.FP32, 0.0, (1, 1, 1))
    dt0 = 0.3 / 64 / 3.0
    eager = RT.AmrHierarchy(levels, ph)
    for _ in range(4):
        eager.step(dt0)
    _, ph2 = params_pair(O.CTU, O.PPM, O.ROE, H.FP32, 0.0, (1, 1, 1))
    g = RT.AmrHierarchy(levels, ph2)
    g.capture(dt0)  # its warm-up runs two steps
    g.replay()      # two more
    torch.cuda.synchronize()
    for l in range(len(levels)):
        assert torch.equal(g.cur[l], eager.cur[l])
    assert eager.launches_per_step() == 1 * 4 + 2 * 4 + 4 * 2


def test_missing_parent_cell_sets_the_nesting_bit():
    torch = _torch()
    # level 1: one octet over the centre group of a 48^3 base; level 2: an
    # octet over the corner group (32, 32, 32) of that octet, whose ghost
    # zone reaches level-1 cells outside the octet
    base = W.amr_hierarchy(48, (0.2,))
    l1 = base[1]
    assert tuple(l1["origin"][0]) == (32, 32, 32)
    org2 = np.asarray([(64 + dx * N, 64 + dy * N, 64 + dz * N) for dz in range(2) for dy in range(2)
                       for dx in range(2)], dtype=np.int32)
    l2 = dict(U=np.ones((8, 5, N, N, N)), origin=org2, box=(192, 192, 192))
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    d1 = _dev_level(l1, H.FP64)
    d2 = _dev_level(l2, H.FP64)
    M = N + 6
    out = torch.zeros((8, 5, M, M, M), dtype=torch.float64, device="cuda")
    H.hydro_amr_prepare(d2, d1, None, 0.0, out, ghost=3, precision=H.FP64, error=err)
    torch.cuda.synchronize()
    assert err.item() & H.AMR_ENESTING
    o = out.cpu().numpy()
    assert np.isnan(o[0, :, 0, 0, 0]).all()          # below the level-1 octet
    assert np.isfinite(o[0, :, 3:3 + N, 3:3 + N, 3:3 + N]).all()  # the interior is copied
    with pytest.raises(A.NestingError):
        A.prepare(dict(l2), dict(l1), None, 0.0, ghost=3)


@pytest.mark.parametrize("scheme,prec", [(O.WAF, H.FP64), (O.RTVD, H.FP32)])
def test_hierarchy_step_split_scheme_outflow(scheme, prec):
    """A directionally split scheme inside a 2-level hierarchy with outflow
    box edges (the refined octet next to the low-x edge): one step against
    oracle.amr.amr_step."""
    torch = _torch()
    levels = _quantised_levels(W.amr_hierarchy(48, (0.25,), center=(0.2, 0.5, 0.6)), prec)
    assert len(levels) == 2
    po, ph = params_pair(scheme, O.PLM, O.HLLC, prec, 0.0, (1, 1, 1))
    dt0 = 0.3 * levels[0]["dx"][0] / 3.0
    ref = A.amr_step(levels, po, dt0, bc=1)
    hier = RT.AmrHierarchy(levels, ph, bc=H.BC_OUTFLOW)
    hier.step(dt0)
    torch.cuda.synchronize()
    for l in range(2):
        got = hier.cur[l].double().cpu().numpy()
        if prec == H.FP64:
            np.testing.assert_array_equal(got, ref[l])
        else:
            assert_close(got, ref[l], prec, "level %d" % l)
    assert hier.errors() == 0
