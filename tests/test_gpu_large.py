"""The W build at a size whose polarizability spans several groups of tiles and more than one wave of CTAs on the
GPU (N_aux = 2200: 18 row tiles of 128, 171 lower-triangle 128 x 128 tiles or 90 tiles of 128 x 256 for 152 SMs, a
ragged last row tile of 24, N_ov = 32 400 with a ragged K tail), against the oracle on a few frequencies.

FP64 path: W(i xi) and W(z) to FP64 rounding.  Mixed path: the tolerance of every table row is derived from the
split-BF16 error of Pi and the conditioning of I - Pi at that frequency (mixed_bound.py): near-real points among
the excitations (kappa ~ 1e4 and more) get a correspondingly loose tolerance; the imaginary axis (kappa of order
||Pi||) is held to a fraction of W's size.
"""
import numpy as np
import pytest

from oracle import cdwac_oracle as o
from paper_2305_15955_gb300 import inputs

from mixed_bound import w_bound

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_15955_gb300 import cdwac  # noqa: E402



@pytest.fixture(scope="module")
def ctx():
    c = cdwac.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def system():
    # 600 orbitals (6 core levels, 54 valence, 540 virtual), N_aux = 2200, two core states
    spec = inputs.custom_system(600, 60, 2200, seed=7, n_core=6, states=(0, 3))
    eps = inputs.eigenvalues(spec)
    B32 = inputs.build_B(spec, dtype=np.float32)
    On32 = inputs.build_On(spec, dtype=np.float32)
    return spec, eps, B32, On32


def _oracle_tables(spec, eps, B, On, xi, zr):
    D = o.transition_energies(eps, spec.n_occ)
    Wim = o.w_imag_table(B, D, On, xi)
    Wre = o.w_complex_table(B, D, On, zr, np.arange(spec.n_occ))
    return D, Wim, Wre


def test_fp64_path_at_multi_wave_size(ctx, system):
    spec, eps, B32, On32 = system
    B, On = B32.astype(np.float64), On32.astype(np.float64)
    sysd = cdwac.System(eps, B, On, spec.states, spec.n_occ)
    p = cdwac.Params(n_imag=3, n_real=2, pade_M=4, precision=cdwac.PREC_FP64)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    zr = pade.z_real.cpu().numpy()[0]
    D, Wim, Wre = _oracle_tables(spec, eps, B, On, xi.cpu().numpy(), zr)
    err = np.abs(W.cpu().numpy() - Wim) / np.abs(Wim).max(axis=2, keepdims=True)
    assert err.max() < 1e-11, err.max()
    err_r = np.abs(pade.W_real.cpu().numpy() - Wre) / np.abs(Wre).max(axis=2, keepdims=True)
    assert err_r.max() < 1e-10, err_r.max()


def test_mixed_path_at_multi_wave_size_within_derived_bound(ctx, system):
    spec, eps, B32, On32 = system
    B, On = B32.astype(np.float64), On32.astype(np.float64)      # the FP32 inputs, exactly, in FP64
    sysd = cdwac.System(eps, B32, On32, spec.states, spec.n_occ)
    p = cdwac.Params(n_imag=3, n_real=2, pade_M=4, precision=cdwac.PREC_MIXED)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    xi_h = xi.cpu().numpy()
    zr = pade.z_real.cpu().numpy()[0]
    D, Wim, Wre = _oracle_tables(spec, eps, B, On, xi_h, zr)
    Wg, Wrg = W.cpu().numpy(), pade.W_real.cpu().numpy()
    m_all = np.arange(spec.n_basis)
    for k, x in enumerate(xi_h):
        bound, kappa = w_bound(B, D, On, 1j * x, m_all)
        err = np.abs(Wg[:, k, :] - Wim[:, k, :])
        assert np.all(err <= bound), (k, kappa, float((err / bound).max()))
        # the bound is not vacuous: on the imaginary axis it holds W to a fraction of its size
        assert np.all(bound.max(axis=1) < 0.05 * np.abs(Wim[:, k, :]).max(axis=1)), (k, kappa)
    m_occ = np.arange(spec.n_occ)
    for j, z in enumerate(zr):
        bound, kappa = w_bound(B, D, On, z, m_occ)
        err = np.abs(Wrg[:, j, :] - Wre[:, j, :])
        assert np.all(err <= bound), (j, z, kappa, float((err / bound).max()))
