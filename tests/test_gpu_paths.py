"""GPU tests of the other entry points and of the edge cases, through the C ABI.

* gather (Sec. 4.2 preparation step) is bit-exact against the oracle's gather;
* the fused uniform path and the multi-level batch give exactly the bytes of
  gather + hydro_advance on the same groups;
* the CFL reduction (Sec. 4.3) and the FP64 totals match the oracle / numpy;
* edge cases: no groups, one group, a ragged count, tuning shapes, argument
  errors;
* the plain-method workload (Sod along x, 32^3 FP64, MHM + PLM minmod + Roe,
  10 steps at CFL 0.5) stays on the oracle step after step.
(The full-size workloads are in test_gpu_fullsize.py.)
"""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import workloads as W
from tests.gpu_common import (assert_close, gpu_advance, lognormal_groups, ndtype, params_pair, quantise, tdtype,
                              with_workspace)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    assert torch.cuda.is_available()
    return torch, torch.device("cuda:0")


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
def test_gather_bit_exact(torch_dev, bc, prec):
    torch, dev = torch_dev
    rng = np.random.default_rng(2)
    f = rng.normal(size=(5, 32, 48, 64)).astype(ndtype(prec)).astype(np.float64)
    N, g = 16, 4
    orig = W.group_origins(64, 48, 32, N)
    ref = O.gather(f, orig, N, g, bc=bc)
    ft = torch.tensor(f, dtype=tdtype(prec), device=dev)
    ot = torch.tensor(orig, dtype=torch.int32, device=dev)
    out = torch.empty(ref.shape, dtype=tdtype(prec), device=dev)
    H.hydro_gather_uniform(ft, ot, out, N=N, ghost=g, bc=bc, precision=prec)
    np.testing.assert_array_equal(out.double().cpu().numpy(), ref)


@pytest.mark.parametrize("prec", [H.FP64, H.FP32, H.FP32_MIXED])
@pytest.mark.parametrize("scheme,recon,rs", [(O.CTU, O.PPM, O.ROE), (O.VL, O.PLM, O.HLLC), (O.MHM, O.PPM, O.HLLE)])
@pytest.mark.parametrize("bc", [0, 1])
def test_fused_uniform_equals_gather_then_advance(torch_dev, prec, scheme, recon, rs, bc):
    torch, dev = torch_dev
    n, N = 32, 16
    g = O.required_ghost(scheme, recon)
    U = quantise(W.lognormal(n, seed=3, mach=1.2), prec)
    dx = (1.0 / n,) * 3
    dt = O.cfl_dt(U, dx, 0.4)
    _, ph = params_pair(scheme, recon, rs, prec, dt, dx)
    with_workspace(ph, dev)
    dtp = tdtype(prec)
    ft = torch.tensor(U, dtype=dtp, device=dev)
    orig = torch.tensor(W.group_origins(n, n, n, N), dtype=torch.int32, device=dev)
    G = orig.shape[0]
    M = N + 2 * g
    Ug = torch.empty((G, 5, M, M, M), dtype=dtp, device=dev)
    H.hydro_gather_uniform(ft, orig, Ug, N=N, ghost=g, bc=bc, precision=prec)
    Uo = torch.empty((G, 5, N, N, N), dtype=dtp, device=dev)
    fl = torch.empty((G, 6, 5, N, N), dtype=dtp, device=dev)
    st = torch.empty(G, dtype=torch.int32, device=dev)
    H.hydro_advance(ph, Ug, Uo, fl, st)
    out = torch.empty_like(ft)
    fl2 = torch.empty_like(fl)
    st2 = torch.empty_like(st)
    H.hydro_advance_uniform(ph, ft, out, bc=bc, flux=fl2, status=st2)
    torch.cuda.synchronize()
    a = W.scatter_groups(Uo.double().cpu().numpy(), n, n, n)
    np.testing.assert_array_equal(out.double().cpu().numpy(), a)
    np.testing.assert_array_equal(fl2.cpu().numpy(), fl.cpu().numpy())
    np.testing.assert_array_equal(st2.cpu().numpy(), st.cpu().numpy())


@pytest.mark.parametrize("prec,bc", [(H.FP64, 0), (H.FP32, 1), (H.FP32_MIXED, 0)])
@pytest.mark.parametrize("scheme,recon,rs", [(O.CTU, O.PPM, O.ROE), (O.VL, O.PLM, O.ROE), (O.MHM, O.PPM, O.ROE)])
def test_chained_columns_equal_single_groups(torch_dev, prec, bc, scheme, recon, rs):
    """In a uniform field a CTA streams through runs of z-consecutive groups
    (chains of at most 32) without restarting.  Field, boundary fluxes and the
    status of every group equal those of the same groups advanced one by one
    (gather + hydro_advance), whatever the grid and the chain length (the
    z-segments of the work order; chains cut at other places) and for columns
    longer than the longest chain.  A double rarefaction
    along z centred on a group boundary (and one along x) makes Roe's
    linearisation fail near the boundaries, so the fallback bit is set in
    some groups and must land in the same groups."""
    torch, dev = torch_dev
    N = 16
    X, Y, Z = 32, 16, 576  # 2 columns of 36 groups
    g = O.required_ghost(scheme, recon)
    z = (np.arange(Z) + 0.5) / Z
    x = (np.arange(X) + 0.5) / X
    y = (np.arange(Y) + 0.5) / Y
    zz, yy, xx = np.meshgrid(z, y, x, indexing="ij")
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * (xx + 2 * yy)) * np.cos(6 * np.pi * zz)
    vz = np.where(zz < 288.0 / Z, -2.0, 2.0) + 0.1 * np.sin(2 * np.pi * yy)
    vx = np.where(xx < 0.5, -1.5, 1.5) * (np.abs(zz - 0.25) < 0.05)
    vy = 0.2 * np.cos(2 * np.pi * xx)
    U = quantise(W.conserved(rho, vx, vy, vz, 0.4 + 0.1 * rho, 1.4), prec)
    dx = (1.0 / X, 1.0 / Y, 1.0 / Z)
    dt = 0.2 / Z
    _, ph = params_pair(scheme, recon, rs, prec, dt, dx, fallback=O.HLLE, pres_floor=1e-10, dens_floor=1e-10)
    with_workspace(ph, dev)
    dtp = tdtype(prec)
    ft = torch.tensor(U, dtype=dtp, device=dev)
    orig = torch.tensor(W.group_origins(X, Y, Z, N), dtype=torch.int32, device=dev)
    G = orig.shape[0]
    M = N + 2 * g
    Ug = torch.empty((G, 5, M, M, M), dtype=dtp, device=dev)
    H.hydro_gather_uniform(ft, orig, Ug, N=N, ghost=g, bc=bc, precision=prec)
    Uo = torch.empty((G, 5, N, N, N), dtype=dtp, device=dev)
    fl = torch.empty((G, 6, 5, N, N), dtype=dtp, device=dev)
    st = torch.empty(G, dtype=torch.int32, device=dev)
    H.hydro_advance(ph, Ug, Uo, fl, st)
    torch.cuda.synchronize()
    ref = W.scatter_groups(Uo.double().cpu().numpy(), X, Y, Z)
    ref_fl, ref_st = fl.cpu().numpy(), st.cpu().numpy()
    fb = (ref_st & H.ST_ROE_FALLBACK) != 0
    assert fb.any() and not fb.all()
    # grid sizes and chain lengths (z-segments of the work order) cut the
    # chains at other places
    for grid, chain in ((1, 0), (5, 3), (7, 8), (0, 0), (0, 1), (0, 5), (11, 32)):
        ph.grid_ctas, ph.chain = grid, chain
        with_workspace(ph, dev)
        out = torch.full_like(ft, float("nan"))
        fl2 = torch.full_like(fl, float("nan"))
        st2 = torch.full_like(st, -1)
        H.hydro_advance_uniform(ph, ft, out, bc=bc, flux=fl2, status=st2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.double().cpu().numpy(), ref)
        np.testing.assert_array_equal(fl2.cpu().numpy(), ref_fl)
        np.testing.assert_array_equal(st2.cpu().numpy(), ref_st)


@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
def test_levels_batch_equals_separate_launches(torch_dev, prec):
    """Uneven per-level group lists with per-level dx and dt in one persistent
    launch give the same bytes as one launch per level."""
    torch, dev = torch_dev
    N, g = 16, 3
    dtp = tdtype(prec)
    sizes = [7, 3, 12, 1]
    levels, sep = [], []
    _, ph = params_pair(O.CTU, O.PPM, O.ROE, prec, 0.0, (1, 1, 1))
    with_workspace(ph, dev)
    for l, G in enumerate(sizes):
        _, Ug = lognormal_groups(n=32, N=N, g=g, seed=10 + l, prec=prec)
        Ug = np.concatenate([Ug] * 2)[:G]
        dxl = (1.0 / (32 * 2 ** l),) * 3
        dtl = O.cfl_dt(Ug[:, :, g:-g, g:-g, g:-g], dxl, 0.4)
        U_in = torch.tensor(Ug, dtype=dtp, device=dev)
        outs = [torch.empty((G, 5, N, N, N), dtype=dtp, device=dev) for _ in range(2)]
        fls = [torch.empty((G, 6, 5, N, N), dtype=dtp, device=dev) for _ in range(2)]
        sts = [torch.empty(G, dtype=torch.int32, device=dev) for _ in range(2)]
        levels.append(H.Level(U_in=U_in, U_out=outs[0], flux=fls[0], status=sts[0], dx=dxl, dt=dtl))
        sep.append((U_in, outs[1], fls[1], sts[1], dxl, dtl))
    H.hydro_advance_levels(ph, levels, N=N, ghost=g)
    for U_in, out, fl, st, dxl, dtl in sep:
        ph.dx, ph.dt = dxl, dtl
        H.hydro_advance(ph, U_in, out, fl, st)
    torch.cuda.synchronize()
    for lv, s in zip(levels, sep):
        np.testing.assert_array_equal(lv.U_out.cpu().numpy(), s[1].cpu().numpy())
        np.testing.assert_array_equal(lv.flux.cpu().numpy(), s[2].cpu().numpy())
        np.testing.assert_array_equal(lv.status.cpu().numpy(), s[3].cpu().numpy())


@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
def test_cfl_dt_and_totals(torch_dev, prec):
    torch, dev = torch_dev
    U = quantise(W.lognormal(32, seed=5, mach=2.0), prec)
    dx = (1 / 32, 1 / 24, 1 / 40)
    ref = O.cfl_dt(U, dx, 0.45)
    ft = torch.tensor(U, dtype=tdtype(prec), device=dev)
    ws = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=dev)
    dt = torch.zeros(1, dtype=torch.float64, device=dev)
    H.hydro_cfl_dt(ft, dx, 0.45, dt, ws, precision=prec)
    # FP64: the same formula, exactly; FP32 data: per-cell speeds in FP32
    if prec == H.FP64:
        assert dt.item() == ref
    else:
        assert dt.item() == pytest.approx(ref, rel=1e-6)
    tot = torch.zeros(5, dtype=torch.float64, device=dev)
    H.hydro_conserved_totals(ft, tot, ws, precision=prec)
    np.testing.assert_allclose(tot.cpu().numpy(), U.reshape(5, -1).sum(axis=1), rtol=1e-13)
    # grouped layout [G,5,N,N,N]
    Ug = W.group_origins(32, 32, 32, 16)
    Ugr = np.stack([U[:, z:z + 16, y:y + 16, x:x + 16] for x, y, z in Ug])
    gt = torch.tensor(Ugr, dtype=tdtype(prec), device=dev)
    dt2 = torch.zeros(1, dtype=torch.float64, device=dev)
    H.hydro_cfl_dt(gt, dx, 0.45, dt2, ws, precision=prec)
    assert dt2.item() == dt.item()


def test_edge_cases_and_errors(torch_dev):
    torch, dev = torch_dev
    N = 16
    po, ph = params_pair(O.CTU, O.PPM, O.ROE, H.FP32, 1e-3, (1 / 32,) * 3)
    # no groups: a no-op that still validates its arguments
    empty = torch.empty((0, 5, 22, 22, 22), dtype=torch.float32, device=dev)
    out0 = torch.empty((0, 5, N, N, N), dtype=torch.float32, device=dev)
    H.hydro_advance(ph, empty, out0)
    # one group and a ragged count
    for G in (1, 7):
        Uq, Ug = lognormal_groups(n=32, g=3, seed=6, prec=H.FP32)
        Ug = np.concatenate([Ug] * 2)[:G]
        ref, ref_flux, _ = O.advance(po, Ug, N)
        got, flux, _ = gpu_advance(ph, Ug)
        assert_close(got, ref, H.FP32, "state")
        assert_close(flux, ref_flux, H.FP32, "flux", axis_var=2)
    # launch shapes: fewer threads, small grids (more groups per CTA)
    Uq, Ug = lognormal_groups(n=32, g=3, seed=7, prec=H.FP32)
    ref, _, _ = O.advance(po, Ug, N)
    base, _, _ = gpu_advance(ph, Ug)
    for threads, grid in ((128, 1), (256, 3), (352, 0), (96, 8)):
        ph.block_threads, ph.grid_ctas = threads, grid
        got, _, _ = gpu_advance(ph, Ug)
        np.testing.assert_array_equal(got, base)
    ph.block_threads, ph.grid_ctas = 0, 0
    # errors are returned, never trapped
    U_in = torch.zeros((1, 5, 22, 22, 22), dtype=torch.float32, device=dev)
    U_out = torch.zeros((1, 5, N, N, N), dtype=torch.float32, device=dev)
    bad = [dict(scheme=7), dict(riemann=9), dict(gamma=1.0), dict(theta=3.0), dict(block_threads=100),
           dict(block_threads=1024), dict(dx=(0.0, 1.0, 1.0)), dict(chain=-1), dict(chain=H.CHAIN_MAX + 1)]
    for kw in bad:
        _, p = params_pair(O.CTU, O.PPM, O.ROE, H.FP32, 1e-3, (1 / 32,) * 3)
        for k, v in kw.items():
            setattr(p, k, v)
        with pytest.raises(H.HydroError) as e:
            H.hydro_advance(p, U_in, U_out)
        assert e.value.code == H.EINVAL
    # output overlapping the input (not only the same base address): refused
    big = torch.zeros(2 * 5 * 22 ** 3, dtype=torch.float32, device=dev)
    with pytest.raises(H.HydroError) as e:
        H.hydro_advance(ph, big[:5 * 22 ** 3].view(1, 5, 22, 22, 22), big[1000:1000 + 5 * N ** 3].view(1, 5, N, N, N))
    assert e.value.code == H.EINVAL
    fld = torch.zeros(2 * 5 * 32 ** 3, dtype=torch.float32, device=dev)
    with pytest.raises(H.HydroError) as e:
        H.hydro_advance_uniform(ph, fld[:5 * 32 ** 3].view(5, 32, 32, 32), fld[64:64 + 5 * 32 ** 3].view(5, 32, 32, 32))
    assert e.value.code == H.EINVAL
    _, p = params_pair(O.VL, O.PPM, O.ROE, H.FP32, 1e-3, (1 / 32,) * 3)  # needs 4 ghost layers
    with pytest.raises(H.HydroError) as e:
        H.hydro_advance(p, U_in, U_out, ghost=3)
    assert e.value.code == H.EGHOST
    _, p = params_pair(O.CTU, O.PPM, O.ROE, H.FP64, 1e-3, (1 / 32,) * 3)  # FP64 needs its workspace
    with pytest.raises(H.HydroError) as e:
        H.hydro_advance(p, U_in.double(), U_out.double())
    assert e.value.code == H.EWORKSPACE
    with pytest.raises(H.HydroError) as e:
        H.hydro_advance(ph, U_in, U_out, N=8, ghost=7)
    assert e.value.code == H.EUNSUPPORTED
    torch.cuda.synchronize()


def test_plain_method_sod_10_steps_fp64(torch_dev):
    """Plain-method workload: uniform 32^3 FP64, Sod along x, outflow, MHM +
    PLM minmod + Roe, 10 steps at CFL 0.5; every step within 1e-12."""
    torch, dev = torch_dev
    n, N, g = 32, 16, 2
    U = W.sod(n, 0)
    dx = (1.0 / n,) * 3
    po, ph = params_pair(O.MHM, O.PLM, O.ROE, H.FP64, 0.0, dx)
    with_workspace(ph, dev)
    ft = torch.tensor(U, dtype=torch.float64, device=dev)
    out = torch.empty_like(ft)
    ws = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=dev)
    dtt = torch.zeros(1, dtype=torch.float64, device=dev)
    ph.dt_dev = dtt
    orig = W.group_origins(n, n, n, N)
    for step in range(10):
        dt = O.cfl_dt(U, dx, 0.5)
        H.hydro_cfl_dt(ft, dx, 0.5, dtt, ws, precision=H.FP64)
        po.dt = dt
        U = W.scatter_groups(O.advance(po, O.gather(U, orig, N, g, bc=1), N)[0], n, n, n)
        H.hydro_advance_uniform(ph, ft, out, bc=H.BC_OUTFLOW)
        torch.cuda.synchronize()
        assert dtt.item() == dt
        assert_close(out.cpu().numpy()[None], U[None], H.FP64, "state step %d" % step)
        ft, out = out, ft
        ft.copy_(torch.tensor(U, device=dev))  # both sides continue from the oracle state


def test_fma_peak_kernels(torch_dev):
    """The FMA-loop kernels behind the measured roofline peak: exact flop
    count, bounded chain values (fixed point 1), and rates within a broad
    window around the part's nominal FP32 / FP64 rates."""
    torch, dev = torch_dev
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    ctas, threads = 4 * nsm, 256
    rates = {}
    for kind, dt, per in ((H.PEAK_FP32, torch.float32, 2), (H.PEAK_FP32X2, torch.float32, 4),
                          (H.PEAK_FP64, torch.float64, 2)):
        buf = torch.full((ctas * threads,), float("nan"), dtype=dt, device=dev)
        iters = 2048 if kind != H.PEAK_FP64 else 256
        H.hydro_fma_peak(kind, ctas, threads, iters, buf)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fl = H.hydro_fma_peak(kind, ctas, threads, iters, buf)
        b.record()
        torch.cuda.synchronize()
        assert fl == per * 8 * iters * ctas * threads
        v = buf.double().cpu().numpy()
        assert np.all(np.isfinite(v)) and np.all((v > 0) & (v < 40))
        rates[kind] = fl / (a.elapsed_time(b) / 1e3) / 1e12
    assert 10.0 < rates[H.PEAK_FP32] < 200.0, rates
    assert 10.0 < rates[H.PEAK_FP32X2] < 400.0, rates
    assert 0.1 < rates[H.PEAK_FP64] < 10.0, rates
    with pytest.raises(H.HydroError) as e:
        H.hydro_fma_peak(7, 1, 32, 1, torch.empty(32, device=dev))
    assert e.value.code == H.EINVAL


@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
def test_cfl_dt_boxes_equals_per_box(torch_dev, prec):
    """The many-box CFL reduction (one pass for a list of boxes, Sec. 4.3 per
    box) gives every box exactly hydro_cfl_dt's dt and max speed, and the
    scaled minimum over boxes; a NaN box makes its dt and the minimum NaN."""
    torch, dev = torch_dev
    dtp = tdtype(prec)
    fields = [torch.tensor(quantise(W.lognormal(n, seed=30 + n, mach=0.5 + n / 64), prec), dtype=dtp, device=dev)
              for n in (32, 64, 16, 48)]
    grouped = torch.tensor(lognormal_groups(n=32, g=3, seed=7, prec=prec)[1], dtype=dtp, device=dev)
    Us = fields + [grouped]
    dxs = [(1 / 32, 1 / 30, 1 / 34), (1 / 64,) * 3, (0.1, 0.2, 0.3), (1 / 48,) * 3, (1 / 40,) * 3]
    scales = [1.0, 2.0, 4.0, 0.5, 8.0]
    ws1 = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=dev)
    ref_dt = torch.zeros(len(Us), dtype=torch.float64, device=dev)
    ref_sm = torch.zeros(len(Us), dtype=torch.float64, device=dev)
    for k, U in enumerate(Us):
        H.hydro_cfl_dt(U, dxs[k], 0.45, ref_dt[k:k + 1], ws1, precision=prec, smax_out=ref_sm[k:k + 1])
    ws = torch.empty(H.hydro_cfl_boxes_workspace_bytes(), dtype=torch.uint8, device=dev)
    dt = torch.full((len(Us) + 1,), float("nan"), dtype=torch.float64, device=dev)
    sm = torch.full((len(Us),), float("nan"), dtype=torch.float64, device=dev)
    boxes = [(U, dxs[k], dt[k:k + 1], scales[k], sm[k:k + 1]) for k, U in enumerate(Us)]
    H.hydro_cfl_dt_boxes(boxes, 0.45, ws, dt_min_out=dt[len(Us):], precision=prec)
    torch.cuda.synchronize()
    a, b = dt.cpu().numpy(), ref_dt.cpu().numpy()
    np.testing.assert_array_equal(a[:-1], b)
    np.testing.assert_array_equal(sm.cpu().numpy(), ref_sm.cpu().numpy())
    assert a[-1] == min(s * x for s, x in zip(scales, b))
    # a NaN cell in one box: that box's dt and the minimum are NaN, the others unchanged
    Us[1].view(-1)[12345] = float("nan")
    H.hydro_cfl_dt_boxes(boxes, 0.45, ws, dt_min_out=dt[len(Us):], precision=prec)
    torch.cuda.synchronize()
    a = dt.cpu().numpy()
    assert np.isnan(a[1]) and np.isnan(a[-1])
    np.testing.assert_array_equal(np.delete(a[:-1], 1), np.delete(b, 1))
    # the largest table: CFL_MAX_BOXES boxes in one call, each its own dt
    many = [(Us[k % len(Us)], dxs[k % len(Us)]) for k in range(H.CFL_MAX_BOXES)]
    dtm = torch.full((H.CFL_MAX_BOXES,), float("nan"), dtype=torch.float64, device=dev)
    H.hydro_cfl_dt_boxes([(U, dx_, dtm[k:k + 1]) for k, (U, dx_) in enumerate(many)], 0.45, ws, precision=prec)
    torch.cuda.synchronize()
    a = dt.cpu().numpy()[:-1]
    np.testing.assert_array_equal(dtm.cpu().numpy(), np.array([a[k % len(Us)] for k in range(H.CFL_MAX_BOXES)]))
    # argument errors
    with pytest.raises(H.HydroError) as e:
        H.hydro_cfl_dt_boxes([], 0.45, ws)
    assert e.value.code == H.EINVAL
    with pytest.raises(H.HydroError) as e:
        H.hydro_cfl_dt_boxes([(Us[0], dxs[0], dtm[:1])] * (H.CFL_MAX_BOXES + 1), 0.45, ws, precision=prec)
    assert e.value.code == H.EINVAL
    with pytest.raises(H.HydroError) as e:
        H.hydro_cfl_dt_boxes(boxes[:1], 0.45, ws1[:64], precision=prec)
    assert e.value.code == H.EWORKSPACE


@pytest.mark.parametrize("prec", [H.FP64, H.FP32])
def test_cfl_dt_boxes_interior_of_padded_groups(torch_dev, prec):
    """A box of halo-padded groups with ghost > 0 reduces only the groups'
    interior cells: its dt and max speed equal hydro_cfl_dt's on the copied-out
    interiors bit for bit, and the oracle's dt over the same cells; a NaN in a
    ghost cell is not seen, one in an interior cell is.  Malformed interior
    descriptions are refused."""
    torch, dev = torch_dev
    dtp = tdtype(prec)
    g = 3
    grouped = torch.tensor(lognormal_groups(n=32, g=g, seed=8, prec=prec)[1], dtype=dtp, device=dev)
    inner = grouped[:, :, g:-g, g:-g, g:-g].contiguous()
    dx = (1 / 32, 1 / 30, 1 / 34)
    ws1 = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=dev)
    ref = torch.zeros(2, dtype=torch.float64, device=dev)
    H.hydro_cfl_dt(inner, dx, 0.45, ref[0:1], ws1, precision=prec, smax_out=ref[1:2])
    ws = torch.empty(H.hydro_cfl_boxes_workspace_bytes(), dtype=torch.uint8, device=dev)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    boxes = [(grouped, dx, out[0:1], 1.0, out[1:2], g)]
    H.hydro_cfl_dt_boxes(boxes, 0.45, ws, precision=prec)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    dt_o = O.cfl_dt(inner.double().cpu().numpy(), dx, 0.45)
    assert out[0].item() == (dt_o if prec == H.FP64 else pytest.approx(dt_o, rel=1e-6))
    # a ghost cell is not part of the reduction; an interior cell is
    grouped[1, 0, 0, 0, 0] = float("nan")
    H.hydro_cfl_dt_boxes(boxes, 0.45, ws, precision=prec)
    torch.cuda.synchronize()
    assert out[0].item() == ref[0].item()
    grouped[1, 0, g + 2, g + 5, g + 7] = float("nan")
    H.hydro_cfl_dt_boxes(boxes, 0.45, ws, precision=prec)
    torch.cuda.synchronize()
    assert np.isnan(out[0].item())
    for field, value in (("ghost", -1), ("cells", 5), ("interior_n", 0), ("var_stride", 10)):
        arr = H.make_cfl_boxes(boxes, prec)
        setattr(arr[0], field, value)
        with pytest.raises(H.HydroError) as e:
            H.hydro_cfl_dt_boxes(None, 0.45, ws, precision=prec, _carray=arr)
        assert e.value.code == H.EINVAL
