"""The W build at a size whose polarizability spans several 12 x 12 groups of 128 x 128 tiles and more than one wave
of CTAs on the GPU (N_aux = 2200: 18 row tiles, 171 lower-triangle tiles for 152 SMs, a ragged last row tile of 24,
N_ov = 32 400 with a ragged K tail), against the oracle on a few frequencies.

FP64 path: W(i xi) and W(z) to FP64 rounding.  Mixed path: the tolerance of every table row is derived from the
split-BF16 error of Pi and the conditioning of I - Pi at that frequency.  With hi = bf16(x) and lo = bf16(x - hi)
an FP32 operand keeps x - hi - lo <= 2^-17 |x|, the dropped lo*lo product is <= 2^-18 |x y|, and the weighted
operand S = fp32(w) * x adds two FP32 roundings: every term S_Pk B_Qk of Pi carries a relative error below
2^-16, with signs that vary from term to term (the tensor-core accumulation runs in chunks of 128 columns summed
with round-to-nearest, so it adds no bias), and the normwise error of Pi is taken as 2^-16 ||Pi||_2.  The W solves'
split-BF16 products and FP32 block solves act as a backward error of the same size on the factor.  Together
u = 2^-15 of ||I - Pi||_2, and first-order perturbation of W_nm = o_m^T [(I - Pi)^-1 - I] o_m bounds
|dW_nm| <= u kappa(I - Pi) ||(I - Pi)^-1||_2 ||o_m||^2 with kappa the 2-norm condition number, which the test
evaluates from the oracle's matrices (FP64) with a safety factor of 4.  Near-real points
among the excitations (kappa ~ 1e4 and more) get a correspondingly loose tolerance; the imaginary axis (kappa of
order ||Pi||) is held to a fraction of W's size.
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

U_BF16X3 = 2.0 ** -15
SAFETY = 4.0


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


def _w_bound(B, D, On, z, m_idx):
    """Per-state bound on |dW_nm| over m_idx from a BF16x3 Pi and its condition number (module docstring)."""
    A = np.eye(B.shape[0]) - o.polarizability(B, D, complex(z))
    sv = np.linalg.svd(A, compute_uv=False)
    kappa, inv_norm = sv[0] / sv[-1], 1.0 / sv[-1]
    on2 = np.sum(On[:, :, m_idx] ** 2, axis=1)                      # [n_states, len(m_idx)]
    return SAFETY * U_BF16X3 * kappa * inv_norm * on2, kappa


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
        bound, kappa = _w_bound(B, D, On, 1j * x, m_all)
        err = np.abs(Wg[:, k, :] - Wim[:, k, :])
        assert np.all(err <= bound), (k, kappa, float((err / bound).max()))
        # the bound is not vacuous: on the imaginary axis it holds W to a fraction of its size
        assert np.all(bound.max(axis=1) < 0.05 * np.abs(Wim[:, k, :]).max(axis=1)), (k, kappa)
    m_occ = np.arange(spec.n_occ)
    for j, z in enumerate(zr):
        bound, kappa = _w_bound(B, D, On, z, m_occ)
        err = np.abs(Wrg[:, j, :] - Wre[:, j, :])
        assert np.all(err <= bound), (j, z, kappa, float((err / bound).max()))
