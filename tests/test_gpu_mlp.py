"""Learned continuation on the GPU against its CPU oracle: features, loss and gradient of the training kernels,
BF16 inference, the residue term with the pole model, and a short training run."""
import numpy as np
import pytest

from oracle import cdwac_oracle as o
from oracle import mlp_oracle as mo
from paper_2305_15955_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_15955_gb300 import cdwac, learned  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = cdwac.Context(0)
    yield c
    c.close()


def _batch(seed=3, B=300, J=40):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, mo.N_IN)) * 0.5 - 0.3
    scale = rng.uniform(0.05, 0.5, size=B)
    z = np.concatenate([1j * rng.uniform(0.01, 50, size=(B, 12)), rng.uniform(0, 11, size=(B, J - 12)) + 1e-3j],
                       axis=1)
    W_ref = scale[:, None] * (-rng.uniform(0.1, 1.0, size=(B, J)) + 0.05j * rng.normal(size=(B, J)))
    return x, scale, z, W_ref


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_loss_and_gradient_match_oracle(ctx):
    theta = mo.init_params(2)
    x, scale, z, W_ref = _batch()
    L, g = mo.loss_and_grad(theta, x, scale, z, W_ref)
    grad, loss = ctx.mlp_loss_grad(_dev(theta, torch.float32), _dev(x, torch.float32), _dev(scale, torch.float32),
                                   _dev(z, torch.complex128), _dev(W_ref, torch.complex128))
    gg = grad.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - L) < 1e-4 * L
    assert np.linalg.norm(gg - g) < 2e-3 * np.linalg.norm(g)
    for lo, hi in [(0, 32 * 256), (32 * 256 + 256, 32 * 256 + 256 + 256 * 256), (mo.N_PARAMS - 16, mo.N_PARAMS)]:
        assert np.linalg.norm(gg[lo:hi] - g[lo:hi]) < 5e-3 * np.linalg.norm(g[lo:hi])


def test_bf16_inference_matches_oracle(ctx):
    theta = mo.init_params(4)
    x, scale, _, _ = _batch(5, B=64)
    poles = ctx.mlp_poles(_dev(theta, torch.float32), _dev(x, torch.float32), _dev(scale, torch.float32)).cpu().numpy()
    out, _ = mo.forward(theta, x)
    Om, r = mo.poles(out)
    assert np.max(np.abs(poles[:, :, 0] - Om) / Om) < 2e-2
    assert np.max(np.abs(poles[:, :, 1] - r * scale[:, None])) < 2e-2 * np.max(r * scale[:, None])


def test_features_match_oracle(ctx):
    spec = learned.training_systems([101])[0]
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec)
    On = inputs.build_On(spec)
    sysd = cdwac.System(eps, B, On, spec.states, spec.n_occ)
    p = cdwac.Params(n_imag=100, n_real=6, pade_M=32)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    x, scale, z_ref, w_ref = ctx.mlp_features(xi, W, spec.n_occ, pade, p.n_real)
    D = o.transition_energies(eps, spec.n_occ)
    xo, _ = o.imaginary_grid(100)
    Wo = o.w_imag_table(B, D, On, xo)                          # [n_states, 100, N_b]
    rows = np.stack([Wo[s][:, m] for s in range(spec.n_occ) for m in range(spec.n_occ)])
    xf, sf, idx = mo.features(rows)
    np.testing.assert_allclose(x.cpu().numpy(), xf, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(scale.cpu().numpy(), sf, rtol=1e-6)
    np.testing.assert_allclose(z_ref.cpu().numpy()[:, :32].imag, np.tile(xo[idx], (rows.shape[0], 1)), rtol=0)
    zr = o.near_real_points(eps, spec.n_occ, eps[list(spec.states)], p.n_real)
    Wr = o.w_complex_table(B, D, On, zr, np.arange(spec.n_occ))
    wr_rows = np.stack([Wr[s][:, m] for s in range(spec.n_occ) for m in range(spec.n_occ)])
    np.testing.assert_allclose(w_ref.cpu().numpy()[:, 32:], wr_rows, rtol=1e-9, atol=1e-12)


def test_sigma_and_qp_with_pole_model_match_oracle(ctx):
    spec = inputs.small_system()
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec)
    On = inputs.build_On(spec)
    sysd = cdwac.System(eps, B, On, spec.states, spec.n_occ)
    p = cdwac.Params(n_imag=100, n_real=0)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    rng = np.random.default_rng(9)
    poles = np.stack([rng.uniform(0.3, 12.0, size=(spec.n_occ, 8)), rng.uniform(0.0, 0.02, size=(spec.n_occ, 8))],
                     axis=-1)[None]
    omega = inputs.omega_grid(24)
    sig = ctx.sigma_poles(sysd, p, xi, wxi, W, _dev(poles, torch.float64), omega).cpu().numpy()[0]
    D = o.transition_energies(eps, spec.n_occ)
    xo, wo = o.imaginary_grid(100)
    Wo = o.w_imag_table(B, D, On, xo)[0]
    ref = np.array([o.sigma_R_poles(poles[0], eps, spec.n_occ, w, p.eta) - o.sigma_I(Wo, eps, spec.n_occ, xo, wo, w,
                                                                                    p.eta) for w in omega])
    assert np.abs(sig - ref).max() < 1e-8
    e, Z, it, qs = ctx.qp_solve_poles(sysd, p, xi, wxi, W, _dev(poles, torch.float64), omega)
    sfn = lambda w: o.sigma_R_poles(poles[0], eps, spec.n_occ, w, p.eta) - o.sigma_I(Wo, eps, spec.n_occ, xo, wo, w,
                                                                                     p.eta)
    q = o.qp_solve(sfn, eps[0], 0.0, omega, upper=eps[spec.n_occ])
    assert int(qs.cpu()[0]) == q.status
    if q.status == 0:
        assert abs(float(e.cpu()[0]) - q.e_qp) < 1e-8


def test_training_lowers_the_loss(ctx):
    p = cdwac.Params(n_imag=100, n_real=20, pade_M=32)
    data = learned.generate(ctx, learned.training_systems(range(100, 112)), p)
    params0 = learned.init_params(data.x.device, 0)
    l0 = learned.mean_loss(ctx, params0, data)
    params, _ = learned.train(ctx, data, steps=300, batch=256, lr=1e-3)
    l1 = learned.mean_loss(ctx, params, data)
    assert np.isfinite(l1) and l1 < 0.5 * l0, (l0, l1)


def test_learned_continuation_skips_the_near_real_builds(ctx):
    """What the network buys: the residue term from imaginary-axis data alone, so the near-real W builds (complex
    Pi and complex LDL^T at every reference point) drop out of the QP solve.  The time saved is asserted; the
    accuracy against plain CD is reported (it is the price: see the evaluation recorded with the design)."""
    import time
    p = cdwac.Params(n_imag=100, n_real=40, pade_M=64)
    data = learned.generate(ctx, learned.training_systems(range(100, 112)), p)
    params, _ = learned.train(ctx, data, steps=200, batch=256, lr=2e-3)
    spec = learned.training_systems([2000])[0]
    eps = inputs.eigenvalues(spec)
    sysd = cdwac.System(eps, inputs.build_B(spec), inputs.build_On(spec, states=(0,)), (0,), spec.n_occ)
    grid = inputs.omega_grid(64)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            out = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / reps, out

    def with_pade():
        xi, wxi, W = ctx.build_W_imag(sysd, p, sync=False)
        pade = ctx.fit_pade(sysd, p, xi, W, sync=False)
        return ctx.qp_solve(sysd, p, xi, wxi, W, pade, grid, sync=False)[0]

    def with_mlp():
        xi, wxi, W = ctx.build_W_imag(sysd, p, sync=False)
        x, sc, _, _ = ctx.mlp_features(xi, W, spec.n_occ)
        poles = ctx.mlp_poles(params, x, sc)
        return ctx.qp_solve_poles(sysd, p, xi, wxi, W, poles, grid, sync=False)[0]

    t_pade, e_pade = timed(with_pade)
    t_mlp, e_mlp = timed(with_mlp)
    ctx.sync_status(allow=(cdwac.ERR_PADE_BREAKDOWN, cdwac.ERR_QP_NOT_CONVERGED))
    print(f"QP solve: Pade with 40 near-real points {t_pade * 1e3:.1f} ms, learned {t_mlp * 1e3:.1f} ms; "
          f"e_qp {float(e_pade.cpu()[0]):.6f} vs {float(e_mlp.cpu()[0]):.6f} Ha")
    assert t_mlp < 0.75 * t_pade
