"""The GPU parity comparison itself, on the CPU: a localised error that the
relative L1 alone lets through is caught by the per-element bound.

The "GPU result" here is the oracle's own output with FP32-sized rounding
noise; the planted mistakes are single values changed in it (one cell on a
group face, one boundary-flux value), the places where the plane-streaming
kernels differ most from a plain loop (group and chain seams).
"""
import numpy as np
import pytest

import oracle as O
from paper_1103_3373_gb300 import hydro as H
from tests.gpu_common import ELEM_FP32, TOL_FP32, assert_close, lognormal_groups, max_rel, rel_l1


@pytest.fixture(scope="module")
def oracle_case():
    Uq, Ug = lognormal_groups(n=32, g=3, seed=1, prec=H.FP32)
    dx = (1.0 / 32,) * 3
    dt = O.cfl_dt(Uq, dx, 0.4)
    P = O.Params(scheme=O.CTU, recon=O.PPM, riemann=O.ROE, limiter=O.MINMOD, theta=1.0, fallback=O.HLLE,
                 gamma=1.4, dens_floor=0.0, pres_floor=0.0, dt=dt, dx=dx, characteristic=0)
    ref, flux, _ = O.advance(P, Ug, 16)
    return ref, flux


def _fp32_like(a, seed):
    """a with relative noise of a few FP32 units in the last place."""
    rng = np.random.default_rng(seed)
    return a * (1.0 + 4.0 * 2.0 ** -24 * rng.standard_normal(a.shape))


def test_rounding_noise_passes(oracle_case):
    ref, flux = oracle_case
    assert_close(_fp32_like(ref, 1), ref, H.FP32)
    assert_close(_fp32_like(flux, 2), flux, H.FP32, "flux", axis_var=2)


@pytest.mark.parametrize("var", [0, 2, 4])
def test_one_cell_on_a_group_face_fails(oracle_case, var):
    ref, _ = oracle_case
    got = _fp32_like(ref, 3)
    # group 5, cell (x = 0, y = 7, z = 15): on its -x and +z faces
    got[5, var, 15, 7, 0] *= 1.0 + 1e-3
    # the aggregate L1 cannot see it ...
    assert rel_l1(got, ref) <= TOL_FP32
    # ... the per-element bound does
    assert max_rel(got, ref) > ELEM_FP32
    with pytest.raises(AssertionError, match="max-norm"):
        assert_close(got, ref, H.FP32)


def test_one_boundary_flux_value_fails(oracle_case):
    _, flux = oracle_case
    got = _fp32_like(flux, 4)
    got[3, 5, 1, 0, 9] += 1e-3 * np.abs(flux[:, :, 1]).mean()  # +z face, x-momentum flux
    assert rel_l1(got.reshape(-1, 5, 256), flux.reshape(-1, 5, 256)) <= TOL_FP32
    with pytest.raises(AssertionError, match="max-norm"):
        assert_close(got, flux, H.FP32, "flux", axis_var=2)


def test_non_finite_value_fails(oracle_case):
    ref, _ = oracle_case
    got = ref.copy()
    got[0, 0, 0, 0, 0] = np.nan
    with pytest.raises(AssertionError, match="non-finite"):
        assert_close(got, ref, H.FP64)
