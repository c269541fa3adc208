"""GPU tests of the batched and serving forms (through the C ABI).

* AMR-shaped batch: uneven per-level group lists advanced by one persistent
  launch equal one launch per level byte for byte; the CUDA-graph replay of a
  step equals the eager step; sampled groups of every level match the oracle
  with that level's dx and dt.
* Prepared groups in runs of z-continuations stream as chains with the
  bytes of every group advanced alone.
* Autotuner: picks a launch shape that runs and gives the same bytes.
* Serving: every request's result is the same alone and in the mix (and
  equal to stepping its box on its own with UniformBox).
"""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import hydro as H
from paper_1103_3373_gb300 import runtime as RT
from paper_1103_3373_gb300 import serving as SV
from paper_1103_3373_gb300 import workloads as W
from tests.gpu_common import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_levels():
    return W.amr_levels(counts=(40, 24, 16, 8), n0=32, seed=5)


def _params(prec=H.FP32):
    return H.Params(scheme=H.CTU, recon=H.PPM, riemann=H.RS_ROE, precision=prec, dens_floor=1e-6, pres_floor=1e-6)


def test_levels_batched_graph_and_oracle(small_levels):
    import torch
    lb = RT.LevelBatch(small_levels, _params())
    lb.step()
    torch.cuda.synchronize()
    batched = [u.clone() for u in lb.U_out]
    fl = [f.clone() for f in lb.flux]
    dts = [d.item() for d in lb.dts]
    for u in lb.U_out:
        u.fill_(float("nan"))
    lb.step_per_level()
    torch.cuda.synchronize()
    for a, b in zip(batched, lb.U_out):
        assert torch.equal(a, b)
    for u in lb.U_out:
        u.fill_(float("nan"))
    lb.capture()
    lb.replay()
    torch.cuda.synchronize()
    for a, b in zip(batched, lb.U_out):
        assert torch.equal(a, b)
    for a, b in zip(fl, lb.flux):
        assert torch.equal(a, b)
    # sampled groups of every level against the oracle (same dt, dx)
    for l, lv in enumerate(small_levels):
        U = lv["U"].astype(np.float64)
        dx = (lv["dx"],) * 3
        # the oracle takes its own dt, over the groups' interior cells; the
        # device's (FP32 per-cell speeds) agrees
        dt_o = O.cfl_dt(U[:, :, 3:-3, 3:-3, 3:-3], dx, 0.4, 1.4, 1e-6, 1e-6)
        assert dts[l] == pytest.approx(dt_o, rel=1e-6)
        P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, dt=dt_o, dx=dx, dens_floor=1e-6, pres_floor=1e-6)
        pick = [0, U.shape[0] - 1]
        ref, ref_flux, _ = O.advance(P, U[pick], 16)
        got = batched[l][pick].double().cpu().numpy()
        assert_close(got, ref, H.FP32, "level %d state" % l)
        assert_close(fl[l][pick].double().cpu().numpy(), ref_flux, H.FP32, "level %d flux" % l, axis_var=2)


@pytest.mark.parametrize("prec", [H.FP64, H.FP32, H.FP32_MIXED])
@pytest.mark.parametrize("scheme,recon,rs", [(H.CTU, H.PPM, H.RS_ROE), (H.CTU, H.PLM, H.RS_HLLC),
                                             (H.VL, H.PLM, H.RS_HLLC), (H.MHM, H.PPM, H.RS_HLLE)])
def test_levels_runs_equal_groups_alone(small_levels, prec, scheme, recon, rs):
    """Prepared groups given with runs of z-continuations (zrun: a level's
    columns, a refined group's z-pairs) stream through each run as one chain
    in the unsplit schemes' kernels.  State, boundary fluxes and
    status equal, byte for byte, those of every group advanced alone (runs
    of one: the same kernel, which launches with runs use), for every chain
    limit and grid (grids of 7 and 3 CTAs give each CTA several groups, so
    runs become chains, cut at other places) and per level as in the batched
    launch.  Without runs the groups go through the plain kernel; that
    equals the runs of one to the tolerance of the parity tests, and in FP64
    byte for byte."""
    import torch
    assert max(int(lv["zrun"].max()) for lv in small_levels) >= 2
    ones = [dict(lv, zrun=np.ones_like(lv["zrun"])) for lv in small_levels]

    def batch(levels, chains=True):
        p = H.Params(scheme=scheme, recon=recon, riemann=rs, precision=prec, dens_floor=1e-6, pres_floor=1e-6)
        assert H.hydro_required_ghost(scheme, recon) <= 3  # the workload's groups carry 3 ghost layers
        return RT.LevelBatch(levels, p, ghost=3, chains=chains)

    def snap(lb):
        torch.cuda.synchronize()
        return ([u.clone() for u in lb.U_out], [f.clone() for f in lb.flux], [s.clone() for s in lb.status])

    def reset(lb):
        for u, f, s in zip(lb.U_out, lb.flux, lb.status):
            u.fill_(float("nan"))
            f.fill_(float("nan"))
            s.fill_(-1)

    alone = batch(ones)
    alone.step()
    ref = snap(alone)
    plain = batch(small_levels, chains=False)
    plain.step()
    for a, b in zip(snap(plain)[0], ref[0]):
        assert_close(a.double().cpu().numpy(), b.double().cpu().numpy(), prec, "plain kernel vs runs of one")
        if prec == H.FP64:
            # built without contraction, the two kernel variants round alike
            assert torch.equal(a, b)
    lb = batch(small_levels)
    for grid, chain in ((0, 0), (0, 1), (0, 2), (7, 0), (3, 3)):
        lb.p.grid_ctas, lb.p.chain = grid, chain
        lb._alloc_ws()
        reset(lb)
        lb.step()
        got = snap(lb)
        for a, b in zip(ref, got):
            for x, y in zip(a, b):
                assert torch.equal(x, y), (grid, chain)
    reset(lb)
    lb.step_per_level()
    got = snap(lb)
    for a, b in zip(ref, got):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    # run values are clamped to [1, groups left in the entry]: zeros and
    # negatives mean every group alone, and a run that reaches the end of its
    # level may overstate its length
    for fill in ("nonpositive", "overstated"):
        odd = []
        for lv in small_levels:
            z = lv["zrun"].copy()
            if fill == "nonpositive":
                z[:] = np.where(np.arange(len(z)) % 2 == 0, 0, -3)
                want_alone = True
            else:
                tail = len(z) - 1
                while tail > 0 and z[tail - 1] == z[tail] + 1:
                    tail -= 1
                z[tail:] += 1000
                want_alone = False
            odd.append(dict(lv, zrun=z))
        lbo = batch(odd)
        lbo.p.grid_ctas = 7
        lbo._alloc_ws()
        lbo.step()
        got = snap(lbo)
        for a, b in zip(ref, got):
            for x, y in zip(a, b):
                assert torch.equal(x, y), (fill, want_alone)


def test_autotune_picks_a_working_shape(small_levels):
    import torch
    from paper_1103_3373_gb300 import autotune
    lb = RT.LevelBatch(small_levels, _params())
    lb.step()
    torch.cuda.synchronize()
    ref = [u.clone() for u in lb.U_out]
    best = lb.tune()
    assert 128 <= best["block_threads"] <= H.hydro_max_block_threads(lb.p)
    lb.step()
    torch.cuda.synchronize()
    for a, b in zip(ref, lb.U_out):
        assert torch.equal(a, b)
    # cached: a second call returns the same choice without re-timing
    again = autotune.tune(lb.p, lambda p: None, tag=lb.tune_tag)
    assert (again["block_threads"], again["grid_ctas"]) == (best["block_threads"], best["grid_ctas"])


def test_autotune_uniform_picks_chain_length():
    """On a uniform box the tuner also searches the chain length (the tile's
    extent along z) and returns it; the step's bytes do not depend on it."""
    import torch
    from paper_1103_3373_gb300 import autotune
    U = W.lognormal(64, seed=3, mach=1.2)
    box = RT.UniformBox(U, _params(), cfl=0.4)
    box.advance()
    torch.cuda.synchronize()
    ref = box.b.clone()
    autotune._CACHE.clear()
    best = box.tune()
    assert best["chain"] in (0, 8, 4, 2)
    assert {t[2] for t in best["tried"]} == {0, 8, 4, 2}
    assert box.p.chain == best["chain"]
    box.b.fill_(float("nan"))
    box.advance()
    torch.cuda.synchronize()
    assert torch.equal(box.b, ref)


def test_serving_results_same_alone_and_in_the_mix():
    import torch
    reqs = [SV.Request(rid=i, t_arrive=0.0, n=n, mach=m, steps=s, seed=sd)
            for i, (n, m, s, sd) in enumerate([(32, 0.7, 3, 11), (64, 2.0, 5, 12), (32, 2.8, 7, 13),
                                                (64, 1.1, 2, 14), (32, 1.5, 4, 15)])]
    mixed = SV.ServingEngine(_params(), sizes=(32, 64), keep_results=True)
    summ = mixed.run([SV.Request(**{k: getattr(r, k) for k in ("rid", "t_arrive", "n", "mach", "steps", "seed")})
                      for r in reqs], realtime=False)
    assert summ["requests"] == len(reqs) and summ["max_active"] == len(reqs)
    res_mix = {r.rid: r.result for r in mixed.done}
    for r in reqs:
        alone = SV.ServingEngine(_params(), sizes=(32, 64), keep_results=True)
        alone.run([SV.Request(**{k: getattr(r, k) for k in ("rid", "t_arrive", "n", "mach", "steps", "seed")})],
                  realtime=False)
        assert torch.equal(alone.done[0].result, res_mix[r.rid])
        # and the same as stepping the box by itself
        U0 = alone.states.make(r.n, r.mach, r.seed).double().cpu().numpy()
        box = RT.UniformBox(U0, _params(), cfl=0.4)
        for _ in range(r.steps):
            box.step()
        torch.cuda.synchronize()
        assert torch.equal(box.state().cpu(), res_mix[r.rid])


def test_serving_admission_respects_budget():
    reqs = [SV.Request(rid=i, t_arrive=0.0, n=64, mach=1.0, steps=2, seed=i) for i in range(6)]
    eng = SV.ServingEngine(_params(), sizes=(64,), budget_bytes=3 * (2 * 5 * 64 ** 3 * 4 + 64 * 4 + 8))
    summ = eng.run(reqs, realtime=False)
    assert summ["requests"] == 6
    assert summ["max_active"] == 3


def _req(rid, t, n, mach, steps, seed):
    return SV.Request(rid=rid, t_arrive=t, n=n, mach=mach, steps=steps, seed=seed)


def test_serving_join_in_flight_same_as_alone():
    """Deterministic tick clock: request 1 becomes admissible at tick 2 while
    request 0 (admitted at tick 0) is still being stepped, and request 2 at
    tick 3; each joins the batch in flight, and each result is the same, bit
    for bit, as the same request run alone."""
    import torch
    spec = [(0, 0, 64, 1.2, 6, 21), (1, 2, 32, 2.5, 5, 22), (2, 3, 32, 0.8, 3, 23)]
    mixed = SV.ServingEngine(_params(), sizes=(32, 64), keep_results=True)
    mixed.run([_req(*x) for x in spec], clock="ticks")
    by = {r.rid: r for r in mixed.done}
    assert by[0].tick_admit == 0 and by[1].tick_admit == 2 and by[2].tick_admit == 3
    # 1 and 2 joined while 0 was in flight (0 finishes after 6 ticks)
    assert by[1].tick_admit < by[0].tick_done and by[2].tick_admit < by[0].tick_done
    for x in spec:
        alone = SV.ServingEngine(_params(), sizes=(32, 64), keep_results=True)
        alone.run([_req(*x)], clock="ticks")
        assert alone.done[0].steps_done == x[4]
        assert torch.equal(alone.done[0].result, by[x[0]].result)


def test_serving_admission_bounds_cells_per_tick():
    """The work bound: with room for two 64^3 boxes per tick, four requests
    never run more than two at a time, every tick advances at most 2 x 64^3
    cells, and every request still completes its steps."""
    reqs = [_req(i, 0, 64, 1.0, 3, 40 + i) for i in range(4)]
    eng = SV.ServingEngine(_params(), sizes=(64,), max_cells_per_tick=2 * 64 ** 3)
    summ = eng.run(reqs, clock="ticks")
    assert summ["requests"] == 4
    assert summ["max_active"] == 2
    assert summ["max_cells_in_a_tick"] <= 2 * 64 ** 3
    assert all(r.steps_done == 3 for r in eng.done)


def test_amr_hierarchy_dt_is_min_over_levels():
    """dt_0 of an AMR hierarchy (one device pass over the levels) equals the
    minimum over levels of 2^l times each level's own CFL dt."""
    import torch
    levels = W.amr_hierarchy(48, (0.2,))
    hier = RT.AmrHierarchy(levels, _params())
    ws = torch.empty(H.hydro_cfl_workspace_bytes(), dtype=torch.uint8, device="cuda:0")
    per = []
    for l in range(hier.L):
        d = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        p = hier.params[l]
        H.hydro_cfl_dt(hier.cur[l], p.dx, 0.4, d, ws, gamma=p.gamma, dens_floor=p.dens_floor,
                       pres_floor=p.pres_floor, precision=hier.prec)
        per.append((2.0 ** l) * d.item())
    assert hier.compute_dt(0.4) == min(per)
