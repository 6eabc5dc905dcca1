"""Diagonal spectral function (Sec. 5.5) through cdwac_spectral against the oracle.

A_nn(omega) = |Im[(omega - eps_n - shift_n - Sigma^c_n(omega))^-1]| / pi on the paper's window: 50 eV at 0.01 eV
spacing (5000 points) from 15 eV below to 35 eV above the core level of the small system.  The CD-WAC self-energy is compared with the
oracle's along the GPU's greedy node order (as in the Sigma parity tests); A inherits its tolerance through
|dA / dSigma| <= 1 / (pi |d|^2), d = omega - eps_n - shift_n - Sigma^c_n(omega).
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
from test_gpu_parity import HA_TOL, _replayed_state, make, oracle_params  # noqa: E402

EV = 1.0 / 27.211386


@pytest.fixture(scope="module")
def ctx():
    c = cdwac.Context(0)
    yield c
    c.close()


def _window(eps_n, n=5000):
    """50 eV at 0.01 eV from 15 eV below the core level: every residue argument eps_m - omega (occupied m above
    omega) then stays inside the near-real reference grid [0, |eps_F - eps_n| + 0.5 Ha], where the continuation
    interpolates; further below it extrapolates and its conditioning bound no longer holds."""
    return eps_n - 15.0 * EV + np.arange(n) * (0.01 * EV)


def test_spectral_cdwac_5000_points(ctx):
    spec = inputs.small_system()
    eps, B, On, st, sysd = make(spec)
    p = cdwac.Params(n_imag=100, n_real=40, pade_M=64)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    omega = _window(eps[0])
    sig, A = ctx.spectral(sysd, p, xi, wxi, W, pade, omega)
    sig, A = sig.cpu().numpy()[0], A.cpu().numpy()[0]
    # the kernel applies the definition to its own Sigma
    A_own = o.spectral_function(sig, eps[0], omega)
    assert np.max(np.abs(A - A_own)) <= 1e-12 * np.max(A_own)
    # against the oracle's Sigma along the GPU's node orders
    D = o.transition_energies(eps, spec.n_occ)
    ref = o.run_cdwac(B, D, On, eps, spec.n_occ, list(st), oracle_params(p), omega[:2], with_sigma=False)
    sig_ref, _, sens = _replayed_state(ref, 0, pade, p, spec.n_occ, eps, omega)
    tol_sig = np.maximum(HA_TOL, 30.0 * sens)     # the Sigma parity criterion, point by point
    assert np.all(np.abs(sig - sig_ref) <= tol_sig), np.max(np.abs(sig - sig_ref) / tol_sig)
    A_ref = o.spectral_function(sig_ref, eps[0], omega)
    d2 = np.abs(omega - eps[0] - sig_ref) ** 2
    tol = 3.0 * tol_sig / (np.pi * d2) + 1e-12 * np.max(A_ref)
    assert np.all(np.abs(A - A_ref) <= tol), np.max(np.abs(A - A_ref) / tol)
    # the window holds the quasiparticle peak and satellite weight; A is a density: positive and finite
    assert np.all(np.isfinite(A)) and np.all(A >= 0.0)


def test_spectral_plain_cd_and_shift(ctx):
    spec = inputs.small_system()
    eps, B, On, st, sysd = make(spec)
    p = cdwac.Params(n_imag=100, n_real=0, pade_M=8)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    omega = np.array([-11.0, -10.8, -10.45, -10.1])
    shift = np.array([0.25])
    sig, A = ctx.spectral(sysd, p, xi, wxi, W, None, omega, shift=shift)
    sig, A = sig.cpu().numpy()[0], A.cpu().numpy()[0]
    D = o.transition_energies(eps, spec.n_occ)
    xo, wo = o.imaginary_grid(100)
    Wo = o.w_imag_table(B, D, On, xo)
    sig_ref = np.array([o.sigma_c_cd(B, D, On[0], Wo[0], eps, spec.n_occ, xo, wo, w, p.eta) for w in omega])
    assert np.abs(sig - sig_ref).max() < HA_TOL
    A_ref = o.spectral_function(sig_ref, eps[0], omega, shift[0])
    d2 = np.abs(omega - eps[0] - shift[0] - sig_ref) ** 2
    assert np.all(np.abs(A - A_ref) <= 3.0 * HA_TOL / (np.pi * d2) + 1e-12 * A_ref.max())


def test_spectral_rejects_null_outputs(ctx):
    spec = inputs.small_system()
    eps, B, On, st, sysd = make(spec)
    p = cdwac.Params(n_imag=16, n_real=0, pade_M=8)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    om = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = ctx.lib.cdwac_spectral(ctx.h, cdwac.ctypes.byref(sysd.c), cdwac.ctypes.byref(p.c()), cdwac._ptr(xi),
                                cdwac._ptr(wxi), cdwac._ptr(W), None, None, cdwac._ptr(om), 4, None, None, None)
    assert rc == cdwac.ERR_ARG
