"""GPU path (libcdwac.so through its C ABI) against the CPU oracle on the same seeded inputs.

FP64 path: W, Sigma and QP energies within 1e-8 Ha (W within 1e-11).  Sizes span several 64-wide tiles and a
ragged tail; edge cases cover a single transition, one auxiliary function, M = 1 and imaginary-only fits.
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

HA_TOL = 1e-8


@pytest.fixture(scope="module")
def ctx():
    c = cdwac.Context(0)
    yield c
    c.close()


def make(spec, dtype=np.float64, states=None):
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec, dtype=dtype)
    On = inputs.build_On(spec, states=states, dtype=dtype)
    st = spec.states if states is None else tuple(states)
    sysd = cdwac.System(eps, B, On, st, spec.n_occ)
    return eps, B.astype(np.float64), On.astype(np.float64), st, sysd


def oracle_params(p: cdwac.Params):
    return o.Params(n_imag=p.n_imag, omega0=p.omega0, n_real=p.n_real, eta_ref=p.eta_ref, eta=p.eta,
                    pade_M=p.pade_M, greedy_first=["absmax", "max", "first"][p.greedy_first],
                    greedy_criterion=["max", "min"][p.greedy_crit], real_margin=p.real_margin, pade_tol=p.pade_tol,
                    real_set=["generic", "refined"][p.real_set], n_core=p.n_core, n_val=p.n_val, delta_c=p.delta_c,
                    delta_v=p.delta_v)


def test_gauss_legendre_grid(ctx):
    spec = inputs.small_system()
    _, _, _, _, sysd = make(spec)
    for n in (1, 7, 100, 200):
        p = cdwac.Params(n_imag=n)
        xi, wxi, _ = ctx.build_W_imag(sysd, p)
        xo, wo = o.imaginary_grid(n)
        # both sides round the exact rule once: the grids agree bit for bit
        assert np.array_equal(xi.cpu().numpy(), xo)
        assert np.array_equal(wxi.cpu().numpy(), wo)


@pytest.mark.parametrize("case", ["small", "ragged", "ragged_f32"])
def test_w_imag_fp64(ctx, case):
    if case == "small":
        spec, dt = inputs.small_system(), np.float64
    else:
        spec = inputs.custom_system(45, 6, 150, seed=21, n_core=2, states=(0, 1, 4))
        dt = np.float32 if case == "ragged_f32" else np.float64
    eps, B, On, st, sysd = make(spec, dtype=dt)
    p = cdwac.Params(n_imag=24)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    D = o.transition_energies(eps, spec.n_occ)
    Wo = o.w_imag_table(B, D, On, xi.cpu().numpy())
    Wg = W.cpu().numpy()
    scale = np.abs(Wo).max()
    assert np.abs(Wg - Wo).max() < 1e-12 * max(1.0, scale), np.abs(Wg - Wo).max()


def test_w_real_fp64(ctx):
    spec = inputs.custom_system(40, 6, 130, seed=4, n_core=1, states=(0, 2))
    eps, B, On, st, sysd = make(spec)
    p = cdwac.Params(n_imag=16, n_real=9, pade_M=12)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    zr = pade.z_real.cpu().numpy()
    zo = o.near_real_points(eps, spec.n_occ, eps[list(st)], p.n_real, p.eta_ref, p.real_margin)
    np.testing.assert_allclose(zr[0], zo, rtol=1e-15, atol=1e-15)
    np.testing.assert_allclose(zr[1], zo, rtol=1e-15, atol=1e-15)
    D = o.transition_energies(eps, spec.n_occ)
    Wo = o.w_complex_table(B, D, On, zo, np.arange(spec.n_occ))
    Wg = pade.W_real.cpu().numpy()
    # near a pole of W(z) the conditioning of I - Pi(z) amplifies rounding (oracle: pivoted LU, GPU: LDL^T)
    assert np.abs(Wg - Wo).max() < 1e-10 * max(1.0, np.abs(Wo).max())


def _replayed_state(ref, s, pade, p, n_occ, eps, omega):
    """The oracle's CD-WAC for state s along the GPU's node orders.

    The greedy order is decided by floating point: once the convergent reproduces the remaining reference values
    to rounding level, several orders are equally valid.  So the oracle replays the GPU's order on its own W
    tables, checks that every node taken carries the largest remaining L1 error of its step (to within rounding
    of W), and evaluates Sigma and the QP equation with those fits."""
    xi, wxi = ref["xi"], ref["wxi"]
    Wim = ref["W_imag"][s]
    Wre = ref["states"][s]["W_real"]
    zr = ref["z_real"]
    zc = np.concatenate([1j * xi, zr])
    nodes = pade.nodes.cpu().numpy()[s]
    used = pade.n_used.cpu().numpy()[s]
    crit = ["max", "min"][p.greedy_crit]
    fits = []
    for m in range(n_occ):
        Wc = np.concatenate([Wim[:, m].astype(complex), Wre[:, m] if len(zr) else np.zeros(0, complex)])
        fit, record = o.thiele_replay(zc, Wc, nodes[m, :used[m]], crit)
        assert used[m] == min(p.pade_M, len(zc))
        assert nodes[m, 0] == int(np.argmax(np.abs(Wc)))
        noise = 1e-8 * np.abs(Wc).max()
        for e_take, e_max, e_min in record:
            if crit == "max":
                assert e_take >= e_max * (1 - 1e-9) - noise, (m, e_take, e_max)
            else:
                assert e_take <= e_min * (1 + 1e-9) + noise, (m, e_take, e_min)
        fits.append(fit)
    model = o.WacModel(fits=fits)
    sig = lambda w: o.sigma_c_wac(model, Wim, eps, n_occ, xi, wxi, w, p.eta)
    sig_ref = np.array([sig(w) for w in omega])
    # conditioning of the continuation: Sigma moved by a W perturbation at the level at which the GPU and the
    # oracle W tables differ (pivoted LU vs LDL^T, summation order): 3e-12 relative at near-real points,
    # 2e-15 on the imaginary axis
    rng = np.random.default_rng(1)
    fits_p = []
    for m in range(n_occ):
        Wc = np.concatenate([Wim[:, m].astype(complex), Wre[:, m] if len(zr) else np.zeros(0, complex)])
        rel = np.concatenate([np.full(len(xi), 2e-15), np.full(len(zr), 3e-12)])
        Wc = Wc * (1 + rel * (rng.standard_normal(len(Wc)) + 1j * rng.standard_normal(len(Wc))))
        fits_p.append(o.thiele_replay(zc, Wc, nodes[m, :used[m]], crit)[0])
    model_p = o.WacModel(fits=fits_p)
    sens = np.array([abs(o.sigma_c_wac(model_p, Wim, eps, n_occ, xi, wxi, w, p.eta) - v)
                     for w, v in zip(omega, sig_ref)])
    return sig_ref, o.qp_solve(sig, eps[ref["states"][s]["n"]], 0.0, omega, upper=eps[n_occ]), sens


def _assert_sigma(sig_gpu, sig_ref, sens):
    """1e-8 Ha wherever the continuation is well conditioned; elsewhere 30x the oracle's own sensitivity."""
    tol = np.maximum(HA_TOL, 30.0 * sens)
    bad = np.abs(sig_gpu - sig_ref) > tol
    assert not bad.any(), (np.abs(sig_gpu - sig_ref)[bad], sens[bad])
    assert np.mean(sens < 1e-9) > 0.25         # a good part of the grid is held to the strict tolerance


def _wac_case(ctx, spec, p, omega):
    eps, B, On, st, sysd = make(spec)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    sig = ctx.sigma(sysd, p, xi, wxi, W, pade, omega).cpu().numpy()
    e, Z, it, qs = ctx.qp_solve(sysd, p, xi, wxi, W, pade, omega)
    D = o.transition_energies(eps, spec.n_occ)
    ref = o.run_cdwac(B, D, On, eps, spec.n_occ, list(st), oracle_params(p), omega)
    rep = [_replayed_state(ref, s, pade, p, spec.n_occ, eps, omega) for s in range(len(st))]
    return dict(sig=sig, e=e.cpu().numpy(), Z=Z.cpu().numpy(), it=it.cpu().numpy(), qs=qs.cpu().numpy(),
                pade=pade, ref=ref, W=W.cpu().numpy(), rep=rep)


@pytest.mark.parametrize("n_real,M", [(40, 64), (0, 16), (20, 40)])
def test_cdwac_sigma_and_qp_small(ctx, n_real, M):
    spec = inputs.small_system()
    p = cdwac.Params(n_imag=100, n_real=n_real, pade_M=M)
    omega = inputs.omega_grid(128)
    r = _wac_case(ctx, spec, p, omega)
    sig_rep, q, sens = r["rep"][0]
    _assert_sigma(r["sig"][0], sig_rep, sens)
    assert r["qs"][0] == q.status == 0
    assert abs(r["e"][0] - q.e_qp) < HA_TOL
    assert abs(r["Z"][0] - q.Z) < 1e-6
    # the oracle's own greedy orders differ only where the choice is rounding noise
    q_own = r["ref"]["states"][0]["qp"]
    assert abs(r["e"][0] - q_own.e_qp) < 1e-6


def test_cdwac_two_states_ragged(ctx):
    spec = inputs.custom_system(70, 9, 200, seed=8, n_core=2, states=(0, 1), core_scale=0.3)
    p = cdwac.Params(n_imag=40, n_real=24, pade_M=48)
    omega = inputs.omega_grid(48)
    r = _wac_case(ctx, spec, p, omega)
    for s in range(2):
        sig_rep, q, sens = r["rep"][s]
        _assert_sigma(r["sig"][s], sig_rep, sens)
        assert r["qs"][s] == q.status
        if q.status < 2:                        # a non-converged iteration has no unique answer
            assert abs(r["e"][s] - q.e_qp) < HA_TOL


def test_plain_cd_sigma_and_qp(ctx):
    spec = inputs.small_system()
    eps, B, On, st, sysd = make(spec)
    p = cdwac.Params(n_imag=100, n_real=0, pade_M=8)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    omega = np.array([-11.0, -10.8, -10.45, -10.1])
    sig = ctx.sigma(sysd, p, xi, wxi, W, None, omega).cpu().numpy()[0]
    D = o.transition_energies(eps, spec.n_occ)
    xo, wo = o.imaginary_grid(100)
    Wo = o.w_imag_table(B, D, On, xo)
    ref = np.array([o.sigma_c_cd(B, D, On[0], Wo[0], eps, spec.n_occ, xo, wo, w, p.eta) for w in omega])
    assert np.abs(sig - ref).max() < HA_TOL
    grid = inputs.omega_grid(16)
    e, Z, it, qs = ctx.qp_solve(sysd, p, xi, wxi, W, None, grid)
    sigfn = lambda w: o.sigma_c_cd(B, D, On[0], Wo[0], eps, spec.n_occ, xo, wo, w, p.eta)
    q = o.qp_solve(sigfn, eps[0], 0.0, grid)
    assert int(qs.cpu()[0]) == q.status == 0
    assert abs(float(e.cpu()[0]) - q.e_qp) < HA_TOL


@pytest.mark.parametrize("shape", ["one_transition", "one_aux", "m_one"])
def test_edge_cases(ctx, shape):
    if shape == "one_transition":
        spec = inputs.custom_system(2, 1, 5, seed=2, n_core=1, states=(0,), valence=(-1.0, -0.5))
        p = cdwac.Params(n_imag=20, n_real=4, pade_M=6)
    elif shape == "one_aux":
        spec = inputs.custom_system(12, 3, 1, seed=3, n_core=1, states=(0,))
        p = cdwac.Params(n_imag=20, n_real=4, pade_M=6)
    else:
        spec = inputs.custom_system(20, 4, 70, seed=5, n_core=1, states=(0,))
        p = cdwac.Params(n_imag=20, n_real=4, pade_M=1)
    omega = inputs.omega_grid(8)
    r = _wac_case(ctx, spec, p, omega)
    sig_rep, q, sens = r["rep"][0]
    _assert_sigma(r["sig"][0], sig_rep, sens)
    if q.status == 0:
        assert abs(r["e"][0] - q.e_qp) < HA_TOL


def test_not_spd_reported(ctx):
    # eigenvalues out of order give negative D_ia, Pi(i xi) turns positive and I - Pi indefinite: the
    # factorisation's own pivot check reports it instead of producing NaN
    spec = inputs.custom_system(20, 4, 30, seed=9, n_core=1, states=(0,))
    eps = inputs.eigenvalues(spec).copy()
    eps[spec.n_occ:] -= 30.0
    B = inputs.build_B(spec) * 20.0
    On = inputs.build_On(spec)
    sysd = cdwac.System(eps, B, On, (0,), spec.n_occ)
    with pytest.raises(cdwac.CdwacError) as ei:
        ctx.build_W_imag(sysd, cdwac.Params(n_imag=8))
    assert ei.value.status == cdwac.ERR_NOT_SPD
    # the context stays usable
    spec2 = inputs.small_system()
    _, _, _, _, s2 = make(spec2)
    ctx.build_W_imag(s2, cdwac.Params(n_imag=8))


def test_argument_errors(ctx):
    spec = inputs.small_system()
    _, _, _, _, sysd = make(spec)
    with pytest.raises(cdwac.CdwacError) as ei:
        ctx.build_W_imag(sysd, cdwac.Params(n_imag=0))
    assert ei.value.status == cdwac.ERR_ARG
    with pytest.raises(cdwac.CdwacError):
        ctx.build_W_imag(sysd, cdwac.Params(n_imag=10, pade_M=cdwac.MAX_M + 1))
