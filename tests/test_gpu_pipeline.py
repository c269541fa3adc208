"""GPU tests of the z-slab advance and of the end-to-end stepper that overlaps
the host transfers with the solver on slabs of patch groups (Sec. 4.1,
asynchronous memory copy over chunks of patch groups), through the C ABI.

* hydro_advance_uniform_zrange on each slab of a partition of the box: the
  slab's cells, boundary fluxes and status equal the oracle step of those
  groups (within the precision's tolerance) and the whole-box advance bit for
  bit; nothing outside the slab is written; an empty slab is a no-op;
* the end-to-end HostBoxStepper (hydro_pipeline_step: 1 slab, or S slabs on
  a copy-in, two compute and a copy-out stream) returns the state, dt,
  boundary fluxes and status of the same number of device-resident steps,
  for periodic and outflow boxes, unsplit and split schemes; bad plans and
  a scheme needing more halo than planned are rejected.
"""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import runtime as RT
from paper_1103_3373_gb300 import workloads as W
from tests.gpu_common import assert_close, params_pair, quantise, tdtype, with_workspace

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    import torch
    assert torch.cuda.is_available()
    return torch, torch.device("cuda:0")


def _field(X, Y, Z, seed):
    c = [W.cell_centres(n)[0] for n in (X, Y, Z)]
    return W.smooth_field(c[0], c[1], c[2], seed=seed, mach=1.2, modes=8, kmax=4)


CASES = [(H.FP64, 0, O.CTU, O.PPM, O.ROE), (H.FP32, 1, O.CTU, O.PPM, O.ROE), (H.FP32_MIXED, 0, O.MHM, O.PPM, O.HLLC),
         (H.FP32, 0, O.VL, O.PLM, O.HLLE), (H.FP64, 1, O.WAF, O.PLM, O.HLLC), (H.FP32, 0, O.RTVD, O.PLM, O.HLLC)]


@pytest.mark.parametrize("prec,bc,scheme,recon,rs", CASES)
def test_zrange_slabs_equal_whole_box_and_oracle(torch_dev, prec, bc, scheme, recon, rs):
    torch, dev = torch_dev
    N = 16
    X, Y, Z = 32, 32, 80  # 5 group layers: slabs of 1, 3 and 1 layers
    U = quantise(_field(X, Y, Z, 11), prec)
    dx = (1.0 / X,) * 3
    dt = O.cfl_dt(U, dx, 0.4)
    po, ph = params_pair(scheme, recon, rs, prec, dt, dx, pres_floor=1e-10, dens_floor=1e-10)
    with_workspace(ph, dev)
    dtp = tdtype(prec)
    ft = torch.tensor(U, dtype=dtp, device=dev)
    G = (X // N) * (Y // N) * (Z // N)
    whole = torch.empty_like(ft)
    fl = torch.empty((G, 6, 5, N, N), dtype=dtp, device=dev)
    st = torch.empty(G, dtype=torch.int32, device=dev)
    H.hydro_advance_uniform(ph, ft, whole, bc=bc, flux=fl, status=st, N=N)
    sent = -12345.0
    part = torch.full_like(ft, sent)
    fl2 = torch.full_like(fl, sent)
    st2 = torch.full_like(st, -1)
    # an empty slab writes nothing
    H.hydro_advance_uniform_zrange(ph, ft, part, 32, 32, bc=bc, flux=fl2, status=st2, N=N)
    torch.cuda.synchronize()
    assert bool((part == sent).all()) and bool((st2 == -1).all())
    bounds = [0, 16, 64, 80]
    per_layer = (X // N) * (Y // N)
    for z0, z1 in zip(bounds[:-1], bounds[1:]):
        H.hydro_advance_uniform_zrange(ph, ft, part, z0, z1, bc=bc, flux=fl2, status=st2, N=N)
        torch.cuda.synchronize()
        got = part.cpu().numpy()
        # only this slab and the slabs before it are written
        assert np.all(got[:, z1:] == sent)
        g1 = z1 // N * per_layer
        assert bool((st2[g1:] == -1).all()) and bool((fl2[g1:] == sent).all())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(part.cpu().numpy(), whole.cpu().numpy())
    np.testing.assert_array_equal(fl2.cpu().numpy(), fl.cpu().numpy())
    np.testing.assert_array_equal(st2.cpu().numpy(), st.cpu().numpy())
    # and the oracle on the middle slab
    g = O.required_ghost(scheme, recon)
    org = W.group_origins(X, Y, Z, N)
    sel = (org[:, 2] >= 16) & (org[:, 2] < 64)
    Uo, Fo, So = O.advance(po, O.gather(U, org[sel], N, g, bc=bc), N)
    got = part.double().cpu().numpy()
    mine = np.stack([got[:, o[2]:o[2] + N, o[1]:o[1] + N, o[0]:o[0] + N] for o in org[sel]])
    assert_close(mine, Uo, prec, "state")
    if prec == H.FP64:
        np.testing.assert_array_equal(st2.cpu().numpy()[sel], So)


@pytest.mark.parametrize("prec,bc,scheme,recon,rs", CASES[:5])
@pytest.mark.parametrize("slabs", [1, 2, 5, (1, 3, 1)])
def test_host_stepper_equals_device_steps(torch_dev, prec, bc, scheme, recon, rs, slabs):
    """Four end-to-end steps through hydro_pipeline_step (host buffers in and
    out) give the bytes of four device-resident UniformBox steps: state, dt,
    boundary fluxes and status."""
    torch, dev = torch_dev
    X, Y, Z = 32, 32, 80
    U = _field(X, Y, Z, 12)
    dx = (1.0 / X,) * 3

    def params():
        return params_pair(scheme, recon, rs, prec, 0.0, dx, pres_floor=1e-10, dens_floor=1e-10)[1]

    box = RT.UniformBox(U, params(), cfl=0.4, bc=bc, device=dev)
    hs = RT.HostBoxStepper(U, params(), cfl=0.4, bc=bc, device=dev, slabs=slabs)
    assert hs.slabs == (len(slabs) if isinstance(slabs, tuple) else slabs)
    for _ in range(4):
        box.step()
        hs.step()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hs.host_in.numpy(), box.state().cpu().numpy())
    np.testing.assert_array_equal(hs.host_dt.numpy(), box.dt.cpu().numpy())
    np.testing.assert_array_equal(hs.box.status.cpu().numpy(), box.status.cpu().numpy())
    np.testing.assert_array_equal(hs.box.flux.cpu().numpy(), box.flux.cpu().numpy())
    assert not np.array_equal(hs.host_in.numpy(), quantise(U, prec).astype(hs.host_in.numpy().dtype))


@pytest.mark.parametrize("slabs", [1, 3])
def test_unchained_steps_equal_device_steps(torch_dev, slabs):
    """Two device buffers in ping-pong (the next step's input is the last
    step's output buffer): every step then waits for the work on the stream
    instead of chaining, and the result is the same."""
    torch, dev = torch_dev
    X, Y, Z = 32, 32, 48
    U = _field(X, Y, Z, 13)
    dx = (1.0 / X,) * 3
    _, p1 = params_pair(O.CTU, O.PPM, O.ROE, H.FP32, 0.0, dx)
    _, p2 = params_pair(O.CTU, O.PPM, O.ROE, H.FP32, 0.0, dx)
    box = RT.UniformBox(U, p1, cfl=0.4, device=dev)
    ref = RT.UniformBox(U, p2, cfl=0.4, device=dev)
    pipe = H.Pipeline(X, Y, Z, 3, slabs=slabs)
    hin = torch.tensor(U, dtype=torch.float32).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    for _ in range(3):
        pipe.step(box.p, hin, hout, box.a, box.b, 0.4, box.red_ws, flux=box.flux, status=box.status)
        box.swap()
        hin, hout = hout, hin
        ref.step()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hin.numpy(), ref.state().cpu().numpy())
    np.testing.assert_array_equal(box.dt.cpu().numpy(), ref.dt.cpu().numpy())
    pipe.close()


def test_pipeline_argument_errors(torch_dev):
    torch, dev = torch_dev
    with pytest.raises(H.HydroError):
        H.Pipeline(32, 32, 80, 3, slabs=(2, 2))          # layers do not sum to Z/N
    with pytest.raises(H.HydroError):
        H.Pipeline(32, 32, 80, 3, slabs=6)               # more slabs than group layers
    pipe = H.Pipeline(32, 32, 64, 2, slabs=2)
    p = H.Params(scheme=H.CTU, recon=H.PPM, riemann=H.RS_ROE, precision=H.FP32, dx=(0.1,) * 3,
                 dt_dev=torch.zeros(1, dtype=torch.float64, device=dev))
    a = torch.zeros((5, 64, 32, 32), dtype=torch.float32).pin_memory()
    b = torch.zeros_like(a).pin_memory()
    da = torch.zeros((5, 64, 32, 32), dtype=torch.float32, device=dev)
    db = torch.zeros_like(da)
    ws = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device=dev)
    with pytest.raises(H.HydroError):                    # PPM + CTU needs 3 ghost layers, planned for 2
        pipe.step(p, a, b, da, db, 0.4, ws)
    pipe.close()
    # the per-slab CFL maxima need hydro_pipeline_workspace_bytes() of scratch
    pipe = H.Pipeline(32, 32, 64, 3, slabs=4)
    assert pipe.workspace_bytes >= H.hydro_cfl_workspace_bytes()
    with pytest.raises(H.HydroError) as ei:
        pipe.step(p, a, b, da, db, 0.4, ws[:1024])
    assert ei.value.code == H.EWORKSPACE
    pipe.close()
    # FP64 kernels keep their rings in scratch: the second compute stream's
    # is required, checked before any work is enqueued
    pipe = H.Pipeline(32, 32, 64, 3, slabs=2)
    p64 = H.Params(scheme=H.CTU, recon=H.PPM, riemann=H.RS_ROE, precision=H.FP64, dx=(0.1,) * 3,
                   dt_dev=torch.zeros(1, dtype=torch.float64, device=dev))
    n = H.hydro_workspace_bytes(p64)
    assert n > 0
    p64.workspace = torch.empty(n, dtype=torch.uint8, device=dev)
    a64 = torch.zeros((5, 64, 32, 32), dtype=torch.float64).pin_memory()
    b64 = torch.zeros_like(a64).pin_memory()
    da64 = torch.zeros((5, 64, 32, 32), dtype=torch.float64, device=dev)
    with pytest.raises(H.HydroError) as ei:
        pipe.step(p64, a64, b64, da64, torch.zeros_like(da64), 0.4, ws)
    assert ei.value.code == H.EWORKSPACE
    pipe.close()
