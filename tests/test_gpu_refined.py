"""Refined near-real reference set omega_C U omega_V (Sec. 3.3) through the C ABI against the oracle.

The points are compared element by element with the oracle's refined set (the same roundings on both sides); the
CD-WAC(N_core, N_val, N_Im) self-energy and QP energies are compared with the oracle's CD-WAC along the GPU's
greedy node orders, under the Sigma and QP criteria of the generic-set parity tests.
"""
import numpy as np
import pytest

from oracle import cdwac_oracle as o
from paper_2305_15955_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_15955_gb300 import cdwac  # noqa: E402
from test_gpu_parity import HA_TOL, _assert_sigma, _wac_case, make  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = cdwac.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n_core,n_val,delta_c,delta_v", [(5, 7, 0.3, 0.8), (1, 1, 0.2, 0.5), (0, 6, 0.2, 40.0),
                                                          (4, 0, 0.0, 1.0)])
def test_refined_points_match_oracle(ctx, n_core, n_val, delta_c, delta_v):
    # three states (two core levels and a valence level): the core centres span eps_4 - eps_0, the valence
    # centres |eps_F - eps_n| span [r_4, r_0]; a radius of 40 Ha is cut at Re z = 0
    spec = inputs.custom_system(45, 6, 150, seed=21, n_core=2, states=(0, 1, 4))
    eps, B, On, st, sysd = make(spec)
    p = cdwac.Params.refined(n_core, n_val, delta_c, delta_v, n_imag=16, pade_M=12)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    zr = pade.z_real.cpu().numpy()
    zo = o.refined_reference_points(eps, spec.n_occ, eps[list(st)], n_core, n_val, delta_c, delta_v, p.eta_ref)
    assert zr.shape == (len(st), n_core + n_val)
    for s in range(len(st)):
        np.testing.assert_allclose(zr[s], zo, rtol=1e-15, atol=1e-15)
    assert np.all(zr.real >= 0.0)


def test_refined_cdwac_sigma_and_qp_small(ctx):
    # CD-WAC(20, 20, 100), the paper's recommended split of 40 near-real points
    spec = inputs.small_system()
    p = cdwac.Params.refined(20, 20, delta_c=0.5, delta_v=1.0, n_imag=100, pade_M=64)
    omega = inputs.omega_grid(128)
    r = _wac_case(ctx, spec, p, omega)
    sig_rep, q, sens = r["rep"][0]
    _assert_sigma(r["sig"][0], sig_rep, sens)
    assert r["qs"][0] == q.status == 0
    assert abs(r["e"][0] - q.e_qp) < HA_TOL
    assert abs(r["Z"][0] - q.Z) < 1e-6
    assert abs(r["e"][0] - r["ref"]["states"][0]["qp"].e_qp) < 1e-6


def test_refined_two_states_ragged(ctx):
    spec = inputs.custom_system(70, 9, 200, seed=8, n_core=2, states=(0, 1), core_scale=0.3)
    # CD-WAC(12, 12, 40) with M = 40: a setting whose continuation is well conditioned on much of the grid (with
    # M = 48 nearly every omega is ill conditioned, which leaves only the loose sensitivity-scaled bound)
    p = cdwac.Params.refined(12, 12, delta_c=0.5, delta_v=1.0, n_imag=40, pade_M=40)
    omega = inputs.omega_grid(48)
    r = _wac_case(ctx, spec, p, omega)
    for s in range(2):
        sig_rep, q, sens = r["rep"][s]
        _assert_sigma(r["sig"][s], sig_rep, sens)
        assert r["qs"][s] == q.status
        if q.status < 2:
            # the fixed point stops once |e_k+1 - e_k| < 1e-7 Ha, which fixes e_QP only to 1e-7 |s| / (1 - |s|)
            # with s = dSigma/domega = 1 - 1/Z on each side (here Z ~ 0.5: a slow, oscillating iteration)
            slope = abs(1.0 - 1.0 / q.Z)
            assert abs(r["e"][s] - q.e_qp) < max(HA_TOL, 2e-7 * slope / (1.0 - slope))


@pytest.mark.parametrize("bad", [dict(n_real=39), dict(delta_c=-0.1), dict(delta_v=float("nan")), dict(n_core=-1,
                                 n_real=19), dict(real_set=2)])
def test_refined_argument_errors(ctx, bad):
    spec = inputs.small_system()
    _, _, _, _, sysd = make(spec)
    p = cdwac.Params.refined(20, 20, n_imag=16, pade_M=12)
    for k, v in bad.items():
        setattr(p, k, v)
    with pytest.raises(cdwac.CdwacError) as ei:
        ctx.build_W_imag(sysd, p)
    assert ei.value.status == cdwac.ERR_ARG
