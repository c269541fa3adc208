"""Host logic of the launch-shape autotuner (no device): which launch shapes
and chain lengths it times for each kind of work."""
from paper_1103_3373_gb300 import autotune as A
from paper_1103_3373_gb300 import hydro as H


def _p(**kw):
    base = dict(scheme=H.CTU, recon=H.PPM, riemann=H.RS_ROE, precision=H.FP32)
    base.update(kw)
    return H.Params(**base)


def test_chain_candidates_per_kind_of_work():
    assert A.chain_candidates(_p(), "uniform") == [0, 8, 4, 2]       # whole columns first
    assert A.chain_candidates(_p(), "levels_runs") == [0, 4, 2, 1]   # whole runs .. every group alone
    assert A.chain_candidates(_p(chain=3), "levels") == [3]          # prepared groups without runs
    assert A.chain_candidates(_p(scheme=H.RTVD, chain=5), "uniform") == [5]  # split schemes do not chain


def test_candidates_are_valid_launch_shapes():
    nsm = 152
    for prec in (H.FP32, H.FP32_MIXED, H.FP64):
        for scheme, recon, rs in ((H.CTU, H.PPM, H.RS_ROE), (H.MHM, H.PLM, H.RS_HLLE), (H.VL, H.PLM, H.RS_HLLC),
                                  (H.CTU, H.PPM, H.RS_EXACT), (H.RTVD, H.PLM, H.RS_HLLC)):
            p = _p(scheme=scheme, recon=recon, riemann=rs, precision=prec)
            maxt = H.hydro_max_block_threads(p)
            assert maxt in (256, 384, 512)
            for tag in ("uniform", "levels_runs"):
                cand = A.candidates(p, nsm, tag)
                assert cand and len(set(cand)) == len(cand)
                for t, grid, ch in cand:
                    assert t % 32 == 0 and 128 <= t <= maxt
                    assert grid in (0, 2 * nsm)
                    assert ch in A.chain_candidates(p, tag)
                # every thread count is timed with the first chain length
                first = A.chain_candidates(p, tag)[0]
                assert {t for t, _, ch in cand if ch == first} == set(range(128, maxt + 1, 32))


def test_fp32_ctu_candidates():
    nsm = 152
    p = _p()
    cand = A.candidates(p, nsm, "uniform")
    # whole columns at every thread count, two CTAs per SM only where the
    # rings could fit twice, the other chain lengths only with the largest CTAs
    assert (512, 0, 0) in cand and (192, 2 * nsm, 0) in cand and (256, 2 * nsm, 0) in cand
    assert not any(grid for t, grid, ch in cand if t not in (192, 256))
    assert {t for t, _, ch in cand if ch == 8} == {384, 416, 448, 480, 512}
    # FP64 rings live in global memory: two CTAs per SM at every thread count
    p64 = _p(precision=H.FP64)
    c64 = A.candidates(p64, nsm, "uniform")
    assert {t for t, g, ch in c64 if g == 2 * nsm and ch == 0} == set(range(128, 257, 32))
