"""Parity at the full sizes of the paper-shaped workloads, in the launch
configuration the benchmark times (through the C ABI).

* Uniform 256^3 periodic lognormal box as 4096 patch groups of 16^3 (3 ghost
  layers; stands in for the paper's uniform-mesh runs, Sec. 5.1), for both
  solvers the benchmark reports (CTU+PPM+Roe and VL+PLM+HLLC): one step of the
  fused path; sampled groups element by element against the oracle, the whole
  box by its conserved totals.
* The same box carried 20 steps in FP32 and in the mixed form against the FP64
  GPU path (which equals the oracle bit for bit): the relative L1 after N
  steps, within a stated bound.
* AMR-shaped batch at its stated sizes (4096 / 2500 / 1500 / 800 prepared
  groups on 4 levels; stands in for the paper's AMR runs, Sec. 5.2): one
  persistent launch; sampled groups of every level against the oracle with
  that level's dx and dt.
"""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import runtime as RT
from paper_1103_3373_gb300 import workloads as W
from tests.gpu_common import PREC_NAME, assert_close, max_rel, params_pair, quantise, rel_l1, report, tdtype, \
    with_workspace

pytestmark = pytest.mark.gpu

C2_SCHEMES = [(O.CTU, O.PPM, O.ROE), (O.VL, O.PLM, O.HLLC)]
C2_IDS = ["ctu_ppm_roe", "vl_plm_hllc"]

# Relative L1 per variable after N steps of the 256^3 box, FP32 / mixed
# against FP64 (both from the same FP32-rounded initial state, each with its
# own CFL dt).  Set from the first measurement (CTU+PPM+Roe 3.2e-8, 6.5e-8,
# 9.5e-8, 1.4e-7; VL+PLM+HLLC 3.1e-8, 6.0e-8, 8.0e-8, 1.05e-7) with a margin
# of about 3, then frozen.
L1_AFTER_STEPS = {1: 1e-7, 5: 2e-7, 10: 3e-7, 20: 4.5e-7}


@pytest.fixture(scope="module")
def box256():
    return W.lognormal(256, seed=1, mach=1.5)


@pytest.mark.parametrize("prec", [H.FP64, H.FP32, H.FP32_MIXED], ids=lambda p: PREC_NAME[p])
@pytest.mark.parametrize("scheme,recon,rs", C2_SCHEMES, ids=C2_IDS)
def test_c2_one_step_sampled_groups(box256, scheme, recon, rs, prec):
    import torch
    dev = torch.device("cuda:0")
    n, N = 256, 16
    g = O.required_ghost(scheme, recon)
    U = quantise(box256, prec)
    dx = (1.0 / n,) * 3
    dt = O.cfl_dt(U, dx, 0.4)
    po, ph = params_pair(scheme, recon, rs, prec, dt, dx)
    with_workspace(ph, dev)
    ft = torch.tensor(U, dtype=tdtype(prec), device=dev)
    out = torch.full_like(ft, float("nan"))
    fl = torch.full((4096, 6, 5, N, N), float("nan"), dtype=tdtype(prec), device=dev)
    st = torch.full((4096,), -1, dtype=torch.int32, device=dev)
    H.hydro_advance_uniform(ph, ft, out, bc=H.BC_PERIODIC, flux=fl, status=st)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    sts = st.cpu().numpy().astype(np.uint32)
    # groups at the box corners (periodic wrap on every face), at chain ends
    # (first / last layer of a column) and a random draw
    rng = np.random.default_rng(0)
    pick = np.unique(np.concatenate([[0, 15, 240, 255, 3840, 4095], rng.choice(4096, 6, replace=False)]))
    orig = W.group_origins(n, n, n, N)[pick]
    ref, ref_flux, ref_st = O.advance(po, O.gather(U, orig, N, g, bc=0), N)
    sub = np.stack([got[:, z0:z0 + N, y0:y0 + N, x0:x0 + N] for x0, y0, z0 in orig])
    assert_close(sub, ref, prec, "state")
    assert_close(fl[torch.as_tensor(pick, device=dev)].double().cpu().numpy(), ref_flux, prec, "flux", axis_var=2)
    assert np.array_equal(sts[pick] & H.ST_ERROR_MASK, ref_st & H.ST_ERROR_MASK)
    if prec == H.FP64:
        assert np.array_equal(sts[pick], ref_st)
        np.testing.assert_array_equal(sub, ref)  # same formulas, same order: bit for bit
    assert not np.any(sts & H.ST_ERROR_MASK)
    tot0 = U.reshape(5, -1).sum(axis=1)
    tot1 = got.reshape(5, -1).sum(axis=1)
    scale = np.abs(U).reshape(5, -1).sum(axis=1)
    assert np.all(np.abs(tot1 - tot0) <= (1e-12 if prec == H.FP64 else 1e-5) * scale)


@pytest.mark.parametrize("scheme,recon,rs", C2_SCHEMES, ids=C2_IDS)
def test_c2_fp32_l1_after_20_steps(box256, scheme, recon, rs):
    import torch
    n = 256
    U0 = quantise(box256, H.FP32)  # the same initial values for every form
    dx = (1.0 / n,) * 3
    boxes = {}
    for prec in (H.FP64, H.FP32, H.FP32_MIXED):
        _, ph = params_pair(scheme, recon, rs, prec, 0.0, dx)
        boxes[prec] = RT.UniformBox(U0, ph, cfl=0.4)
    for step in range(1, 21):
        for b in boxes.values():
            b.step()
        if step in L1_AFTER_STEPS:
            torch.cuda.synchronize()
            ref = boxes[H.FP64].state().cpu().numpy()
            for prec in (H.FP32, H.FP32_MIXED):
                got = boxes[prec].state().double().cpu().numpy()
                assert np.all(np.isfinite(got))
                l1 = rel_l1(got[None], ref[None])
                report("state after %d steps vs FP64" % step, prec, l1, max_rel(got[None], ref[None]))
                assert l1 <= L1_AFTER_STEPS[step], (PREC_NAME[prec], step, l1)
    for b in boxes.values():
        assert not np.any(b.status.cpu().numpy() & H.ST_ERROR_MASK)


@pytest.fixture(scope="module")
def amr_levels_full():
    return W.amr_levels()  # 4096 / 2500 / 1500 / 800 groups, seeded


def test_c3_stated_sizes_sampled_levels(amr_levels_full):
    import torch
    assert [lv["U"].shape[0] for lv in amr_levels_full] == [4096, 2500, 1500, 800]
    p = H.Params(scheme=H.CTU, recon=H.PPM, riemann=H.RS_ROE, precision=H.FP32, dens_floor=1e-6,
                 pres_floor=1e-6)
    lb = RT.LevelBatch(amr_levels_full, p)
    lb.capture()
    lb.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    for l, lv in enumerate(amr_levels_full):
        G = lv["U"].shape[0]
        dt = lb.dts[l].item()
        dx = (lv["dx"],) * 3
        # the level's dt is its own CFL reduction over its groups' interior
        # cells (FP32 per-cell speeds); the oracle takes its own
        dt_o = O.cfl_dt(lv["U"][:, :, 3:-3, 3:-3, 3:-3], dx, 0.4, 1.4, 1e-6, 1e-6)
        assert dt == pytest.approx(dt_o, rel=1e-6)
        pick = np.unique(np.concatenate([[0, G - 1], rng.choice(G, 4, replace=False)]))
        Ul = lv["U"][pick].astype(np.float64)
        P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, dt=dt_o, dx=dx, dens_floor=1e-6, pres_floor=1e-6)
        ref, ref_flux, ref_st = O.advance(P, Ul, 16)
        idx = torch.as_tensor(pick, device=lb.U_out[l].device)
        assert_close(lb.U_out[l][idx].double().cpu().numpy(), ref, H.FP32, "level %d state" % l)
        assert_close(lb.flux[l][idx].double().cpu().numpy(), ref_flux, H.FP32, "level %d flux" % l, axis_var=2)
        st = lb.status[l].cpu().numpy().astype(np.uint32)
        assert np.array_equal(st[pick] & H.ST_ERROR_MASK, ref_st & H.ST_ERROR_MASK)
