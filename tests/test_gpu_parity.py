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
                    greedy_criterion=["max", "min"][p.greedy_crit], real_margin=p.real_margin)


def test_gauss_legendre_grid(ctx):
    spec = inputs.small_system()
    _, _, _, _, sysd = make(spec)
    for n in (1, 7, 100, 200):
        p = cdwac.Params(n_imag=n)
        xi, wxi, _ = ctx.build_W_imag(sysd, p)
        xo, wo = o.imaginary_grid(n)
        np.testing.assert_allclose(xi.cpu().numpy(), xo, rtol=1e-13, atol=0)
        np.testing.assert_allclose(wxi.cpu().numpy(), wo, rtol=1e-12, atol=0)


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
    assert np.abs(Wg - Wo).max() < 1e-11 * max(1.0, np.abs(Wo).max())


def _wac_case(ctx, spec, p, omega):
    eps, B, On, st, sysd = make(spec)
    xi, wxi, W = ctx.build_W_imag(sysd, p)
    pade = ctx.fit_pade(sysd, p, xi, W)
    sig = ctx.sigma(sysd, p, xi, wxi, W, pade, omega).cpu().numpy()
    e, Z, it, qs = ctx.qp_solve(sysd, p, xi, wxi, W, pade, omega)
    D = o.transition_energies(eps, spec.n_occ)
    ref = o.run_cdwac(B, D, On, eps, spec.n_occ, list(st), oracle_params(p), omega)
    return dict(sig=sig, e=e.cpu().numpy(), Z=Z.cpu().numpy(), it=it.cpu().numpy(), qs=qs.cpu().numpy(),
                pade=pade, ref=ref, W=W.cpu().numpy())


@pytest.mark.parametrize("n_real,M", [(40, 64), (0, 16), (20, 40)])
def test_cdwac_sigma_and_qp_small(ctx, n_real, M):
    spec = inputs.small_system()
    p = cdwac.Params(n_imag=100, n_real=n_real, pade_M=M)
    omega = inputs.omega_grid(128)
    r = _wac_case(ctx, spec, p, omega)
    rs = r["ref"]["states"][0]
    # node order of the greedy fits
    nodes = r["pade"].nodes.cpu().numpy()[0]
    used = r["pade"].n_used.cpu().numpy()[0]
    for m, fit in enumerate(rs["model"].fits):
        assert used[m] == len(fit.nodes)
        assert list(nodes[m, :used[m]]) == fit.nodes
    assert np.abs(r["sig"][0] - rs["sigma"]).max() < HA_TOL
    q = rs["qp"]
    assert r["qs"][0] == q.status
    assert abs(r["e"][0] - q.e_qp) < HA_TOL
    assert abs(r["Z"][0] - q.Z) < 1e-6


def test_cdwac_two_states_ragged(ctx):
    spec = inputs.custom_system(70, 9, 200, seed=8, n_core=2, states=(0, 1), core_scale=0.3)
    p = cdwac.Params(n_imag=40, n_real=24, pade_M=48)
    omega = inputs.omega_grid(48)
    r = _wac_case(ctx, spec, p, omega)
    for s in range(2):
        rs = r["ref"]["states"][s]
        assert np.abs(r["sig"][s] - rs["sigma"]).max() < HA_TOL
        assert abs(r["e"][s] - rs["qp"].e_qp) < HA_TOL


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
    rs = r["ref"]["states"][0]
    assert np.abs(r["sig"][0] - rs["sigma"]).max() < HA_TOL
    if rs["qp"].status == 0:
        assert abs(r["e"][0] - rs["qp"].e_qp) < HA_TOL


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
