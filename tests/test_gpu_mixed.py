"""Mixed-precision path (split-BF16 tcgen05 polarizability, FP64 LDL^T, Thiele, Sigma, QP) against the FP64 oracle.

The tensor-core products carry ~2^-16 relative error per term, so W(i xi) is compared at 2e-4 of its scale, W at
near-real points at 5e-3 (amplified by the conditioning of I - Pi(z) near poles) and the quasiparticle energies at 1 meV (the
accuracy target of the mixed form).
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

MEV = 1.0 / 27211.386


@pytest.fixture(scope="module")
def ctx():
    c = cdwac.Context(0)
    yield c
    c.close()


def make(spec, dtype=np.float64):
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec, dtype=dtype)
    On = inputs.build_On(spec, dtype=dtype)
    return eps, B.astype(np.float64), On.astype(np.float64), cdwac.System(eps, B, On, spec.states, spec.n_occ)


@pytest.mark.parametrize("case", ["small", "ragged_f32", "two_tiles"])
def test_mixed_w_tables(ctx, case):
    if case == "small":
        spec, dt = inputs.small_system(), np.float64
    elif case == "ragged_f32":
        spec, dt = inputs.custom_system(45, 6, 150, seed=21, n_core=2, states=(0, 1, 4)), np.float32
    else:
        spec, dt = inputs.custom_system(90, 10, 300, seed=31, n_core=2, states=(0, 3)), np.float64
    eps, B, On, sysd = make(spec, dt)
    p = cdwac.Params(n_imag=12, n_real=5, pade_M=8, precision=cdwac.PREC_MIXED)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    D = o.transition_energies(eps, spec.n_occ)
    xi_h = xi.cpu().numpy()
    Wo = o.w_imag_table(B, D, On, xi_h)
    Wg = W.cpu().numpy()
    # every entry within the error bound derived from the split-BF16 Pi and cond(I - Pi) at its frequency
    # (mixed_bound.py); at the smallest xi, where W is largest, the bound holds W to a fraction of its size (W
    # decays like 1/xi^2 at large xi, the backward-error part of the bound does not)
    for k, x in enumerate(xi_h):
        bound, kappa = w_bound(B, D, On, 1j * x, np.arange(spec.n_basis))
        err = np.abs(Wg[:, k, :] - Wo[:, k, :])
        assert np.all(err <= bound), (k, kappa, float((err / bound).max()))
        if k == int(np.argmin(xi_h)):
            assert np.all(bound.max(axis=1) < 0.05 * np.abs(Wo[:, k, :]).max(axis=1)), (k, kappa)
    pade = ctx.fit_pade(sysd, p, xi, W)
    zo = o.near_real_points(eps, spec.n_occ, eps[list(spec.states)], p.n_real, p.eta_ref, p.real_margin)
    Wro = o.w_complex_table(B, D, On, zo, np.arange(spec.n_occ))
    Wrg = pade.W_real.cpu().numpy()
    # near a pole of W the error is amplified by the conditioning of I - Pi(z) (Im z = 1e-3 Ha): the same bound
    for j, z in enumerate(zo):
        bound, kappa = w_bound(B, D, On, z, np.arange(spec.n_occ))
        err = np.abs(Wrg[:, j, :] - Wro[:, j, :])
        assert np.all(err <= bound), (j, z, kappa, float((err / bound).max()))


@pytest.mark.parametrize("n_real,M", [(40, 64), (40, 48)])
def test_mixed_cdwac_qp_within_1mev(ctx, n_real, M):
    spec = inputs.small_system()
    eps, B, On, sysd = make(spec)
    omega = inputs.omega_grid(128)
    p = cdwac.Params(n_imag=100, n_real=n_real, pade_M=M, precision=cdwac.PREC_MIXED)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    e, Z, it, qs = ctx.qp_solve(sysd, p, xi, wxi, W, pade, omega)
    D = o.transition_energies(eps, spec.n_occ)
    ref = o.run_cdwac(B, D, On, eps, spec.n_occ, [0], o.Params(n_imag=100, n_real=n_real, pade_M=M), omega,
                      with_sigma=False)
    q = ref["states"][0]["qp"]
    assert int(qs.cpu()[0]) == 0 and q.status == 0
    assert abs(float(e.cpu()[0]) - q.e_qp) < 1.0 * MEV, (float(e.cpu()[0]) - q.e_qp) / MEV


def test_mixed_plain_cd_sigma(ctx):
    spec = inputs.small_system()
    eps, B, On, sysd = make(spec)
    p = cdwac.Params(n_imag=60, n_real=0, precision=cdwac.PREC_MIXED)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    omega = np.array([-11.0, -10.7, -10.2])
    sig = ctx.sigma(sysd, p, xi, wxi, W, None, omega).cpu().numpy()[0]
    D = o.transition_energies(eps, spec.n_occ)
    xo, wo = o.imaginary_grid(60)
    Wo = o.w_imag_table(B, D, On, xo)
    ref = np.array([o.sigma_c_cd(B, D, On[0], Wo[0], eps, spec.n_occ, xo, wo, w, p.eta) for w in omega])
    assert np.abs(sig - ref).max() < 0.1 * MEV


def test_pi_tile_widths_agree(monkeypatch):
    """The 128 x 256 and 128 x 128 tensor-core Pi kernels sum the same split-BF16 products and differ only in how
    the FP32 accumulation is chunked (128 x 256: corrections and hi*hi products of 64 columns per chain; 128 x 128:
    hi*hi per 64 columns, corrections per 2048), i.e. in FP32 rounding: W(i xi) and W(z) from the two agree far
    inside the mixed path's 2^-15 error model (N_aux = 300: two 128 x 256 column pairs, a ragged last row block
    of 44 rows)."""
    spec = inputs.custom_system(96, 9, 300, seed=23, n_core=2, states=(0, 1))
    eps = inputs.eigenvalues(spec)
    sysd = cdwac.System(eps, inputs.build_B(spec, dtype=np.float32), inputs.build_On(spec, dtype=np.float32),
                        spec.states, spec.n_occ)
    p = cdwac.Params(n_imag=24, n_real=8, pade_M=24, precision=cdwac.PREC_MIXED)
    out = {}
    for width in (128, 256):
        monkeypatch.setenv("CDWAC_PI_TILE", str(width))
        c = cdwac.Context(0)
        try:
            xi, wxi, W = c.build_W_imag(sysd, p)
            pade = c.fit_pade(sysd, p, xi, W)
            out[width] = (W.cpu().numpy(), pade.W_real.cpu().numpy())
        finally:
            c.close()
    # FP32 rounding of Pi (relative ~1e-7) reaches W through cond(I - Pi): about 10 on the imaginary axis, up to
    # ~1e4 at the near-real points (Im z = 1e-3 Ha)
    for (a, b), tol in zip(zip(out[128], out[256]), (1e-5, 1e-3)):
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(a)), np.max(np.abs(a - b)) / np.max(np.abs(a))
