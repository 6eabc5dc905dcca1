"""The W build at a size whose polarizability spans several 12 x 12 groups of 128 x 128 tiles and more than one wave
of CTAs on the GPU (N_aux = 2200: 18 row tiles, 171 lower-triangle tiles for 152 SMs, a ragged last row tile of 24,
N_ov = 32 400 with a ragged K tail), against the oracle on a few frequencies.

FP64 path: W(i xi) and W(z) to FP64 rounding.  Mixed path: the tolerance of every table row is derived from the
split-BF16 error of Pi and the conditioning of I - Pi at that frequency.  With hi = bf16(x) and lo = bf16(x - hi) an
FP32 operand keeps x - hi - lo <= 2^-17 |x|; the dropped lo*lo product is <= 2^-18 |x y|; the weighted operand
S = fp32(w) * x adds two FP32 roundings (2^-24 each) and the FP32 accumulation of the tensor cores adds at most
about log2(K) * 2^-24 per term for a tree-blocked sum.  So every term of Pi_PQ = sum_k S_Pk B_Qk carries at most
u = 2^-15 of |S_Pk B_Qk| and |dPi| <= u |S| |B|^T elementwise.  A first-order perturbation bound for
W = o^T (I - Pi)^-1 Pi o then gives |dW| <= ||(I - Pi)^-1||_2^2 ||u |S| |B|^T||_2 ||o||^2, which the test evaluates
with the oracle's own matrices (FP64) and multiplies by a safety factor of 4.
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
    """Per-state first-order bound on |dW_nm| over m_idx from a BF16x3 Pi (see the module docstring)."""
    z = complex(z)
    if z.real == 0.0:
        w = -4.0 * D / (z.imag ** 2 + D ** 2)
    else:
        w = 4.0 * D / (z * z - D * D)
    absB = np.abs(B)
    E = U_BF16X3 * ((absB * np.abs(w)[None, :]) @ absB.T)
    A = np.eye(B.shape[0]) - o.polarizability(B, D, z)
    inv_norm = 1.0 / np.linalg.svd(A, compute_uv=False)[-1]
    e_norm = np.linalg.norm(E, 2)
    on2 = np.sum(On[:, :, m_idx] ** 2, axis=1)                      # [n_states, len(m_idx)]
    return SAFETY * inv_norm ** 2 * e_norm * on2, inv_norm * np.linalg.norm(A, 2)


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
        bound, cond = _w_bound(B, D, On, 1j * x, m_all)
        err = np.abs(Wg[:, k, :] - Wim[:, k, :])
        assert np.all(err <= bound), (k, cond, float((err / bound).max()))
        # the bound is not vacuous: W is resolved to well under its size on the imaginary axis
        assert np.all(bound < 1e-2 * np.abs(Wim[:, k, :]).max(axis=1, keepdims=True))
    m_occ = np.arange(spec.n_occ)
    for j, z in enumerate(zr):
        bound, cond = _w_bound(B, D, On, z, m_occ)
        err = np.abs(Wrg[:, j, :] - Wre[:, j, :])
        assert np.all(err <= bound), (j, z, cond, float((err / bound).max()))
