"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: the fully analytic sum-over-poles
self-energy (Eq. sigma_pole) from an RPA diagonalisation, closed forms, exactness of Gauss-Legendre and of
rational interpolation, and invariants of Pi, Lambda and W (Sec. 2.3).
"""
import math

import numpy as np
import pytest

from oracle import cdwac_oracle as o
from paper_2305_15955_gb300 import inputs


@pytest.fixture(scope="module")
def small():
    spec = inputs.small_system()
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec)
    On = inputs.build_On(spec)
    D = o.transition_energies(eps, spec.n_occ)
    xi, wxi = o.imaginary_grid(100)
    Wim = o.w_imag_table(B, D, On, xi)
    return dict(spec=spec, eps=eps, B=B, On=On, D=D, xi=xi, wxi=wxi, Wim=Wim)


# --- grid -------------------------------------------------------------------------------------------------

def test_imaginary_grid_exact_rational_integrals():
    # xi = (1+x)/(1-x) turns 1/(1+xi)^2 and 1/(1+xi)^4 into polynomials of x: Gauss-Legendre is exact
    for n in (4, 17, 100):
        xi, w = o.imaginary_grid(n)
        assert np.all(np.diff(xi) > 0) and xi[0] > 0
        assert abs(np.sum(w / (1 + xi) ** 2) - 1.0) < 1e-13
        assert abs(np.sum(w / (1 + xi) ** 4) - 1.0 / 3.0) < 1e-13
    xi, w = o.imaginary_grid(100, omega0=2.5)
    assert abs(np.sum(w / (2.5 + xi) ** 2) - 1.0 / 2.5) < 1e-13


def test_imaginary_grid_lorentzian():
    xi, w = o.imaginary_grid(100)
    for a in (0.3, 1.0, 10.6):
        assert abs(np.sum(w * a / (a * a + xi * xi)) - math.pi / 2) < 1e-6


def test_transition_energy_order():
    eps = np.array([-3.0, -1.0, 0.5, 2.0, 7.0])
    D = o.transition_energies(eps, 2)
    expect = [eps[a] - eps[i] for i in range(2) for a in range(2, 5)]
    assert np.array_equal(D, np.array(expect))


def test_residue_factors_cases():
    eps = np.array([-10.0, -1.0, 0.5, 2.0])
    f = o.residue_factors(eps, 2, -5.0)      # occupied m above omega contributes -1
    assert list(f) == [0.0, -1.0, 0.0, 0.0]
    f = o.residue_factors(eps, 2, 1.0)       # virtual m below omega contributes +1
    assert list(f) == [0.0, 0.0, 1.0, 0.0]
    f = o.residue_factors(eps, 2, -1.0)      # theta(0) = 1/2
    assert list(f) == [0.0, -0.5, 0.0, 0.0]


# --- screened interaction -------------------------------------------------------------------------------

def test_pi_invariants(small):
    B, D = small["B"], small["D"]
    for x in (0.01, 1.0, 300.0):
        Pi = o.polarizability(B, D, 1j * x)
        assert np.isrealobj(Pi)
        assert np.abs(Pi - Pi.T).max() < 1e-14
        ev = np.linalg.eigvalsh(Pi)
        assert ev.max() < 1e-12                          # negative semidefinite
        Lam = o.screened_lambda(Pi)
        assert np.linalg.eigvalsh(0.5 * (Lam + Lam.T)).max() < 1e-12
        assert np.linalg.eigvalsh(0.5 * (Lam + Lam.T)).min() > -1.0
    # even in the frequency: Pi(z) = Pi(-z) for complex z
    z = 0.7 + 0.05j
    assert np.abs(o.polarizability(B, D, z) - o.polarizability(B, D, -z)).max() < 1e-13


def test_w_imag_invariants(small):
    W = small["Wim"][0]                                   # [n_xi, N_b]
    assert np.all(W <= 1e-15)
    assert np.all(np.diff(W, axis=0) >= -1e-15)            # increasing towards 0 with xi
    assert np.abs(W[-1]).max() < 1e-4 * np.abs(W[0]).max()


def test_w_imag_matches_rpa_pole_form(small):
    s = small
    Wp = o.w_imag_pole_sum(s["B"], s["D"], s["On"][0], s["xi"])
    assert np.abs(s["Wim"][0] - Wp).max() < 1e-13


def test_one_pole_closed_form():
    # N_aux = 1, one transition: W(z) = 4 o^2 b^2 D / (z^2 - D^2 - 4 b^2 D)
    b, d, ov = 0.7, 0.9, 0.4
    B = np.array([[b]])
    D = np.array([d])
    for z in (0.3j, 2.0j, 0.5 + 0.01j, 1.7 + 0.001j):
        Lam = o.screened_lambda(o.polarizability(B, D, z))
        W = o.w_elements(np.array([[ov]]), Lam)[0]
        expect = 4 * ov ** 2 * b ** 2 * d / (z ** 2 - d ** 2 - 4 * b ** 2 * d)
        assert abs(W - expect) < 1e-14


# --- self-energy: plain CD is exact against the sum over poles ---------------------------------------------

@pytest.mark.parametrize("omega", [-11.0, -10.7, -10.45, -10.2, -10.0, -0.2, 0.011, 0.5, 2.6])
def test_cd_matches_sum_over_poles(small, omega):
    s = small
    eta = 1e-8
    cd = o.sigma_c_cd(s["B"], s["D"], s["On"][0], s["Wim"][0], s["eps"], s["spec"].n_occ, s["xi"], s["wxi"],
                      omega, eta)
    ps = o.sigma_c_pole_sum(s["B"], s["D"], s["On"][0], s["eps"], s["spec"].n_occ, omega, eta)
    assert abs(cd.real - ps.real) < 1e-10 * max(1.0, abs(ps)), (cd, ps)


def test_cd_matches_sum_over_poles_other_state(small):
    # a valence state n = 3 exercises O^{nm} rows that carry no core scaling
    s = small
    On3 = inputs.build_On(s["spec"], states=(3,))
    W3 = o.w_imag_table(s["B"], s["D"], On3, s["xi"])[0]
    for omega in (-0.9, -0.6, -0.45):   # away from eigenvalues: the quadrature cannot resolve |omega - eps_m| -> 0
        cd = o.sigma_c_cd(s["B"], s["D"], On3[0], W3, s["eps"], s["spec"].n_occ, s["xi"], s["wxi"], omega, 1e-8)
        ps = o.sigma_c_pole_sum(s["B"], s["D"], On3[0], s["eps"], s["spec"].n_occ, omega, 1e-8)
        assert abs(cd.real - ps.real) < 1e-10 * max(1.0, abs(ps))


def test_sigma_x_hand_example():
    # Eq. exs for two auxiliary functions and three orbitals, two of them occupied, worked by hand:
    # Sigma^x_n = -[(0.5)^2 + (-1)^2 + (0.25)^2 + 2^2] = -5.3125; the virtual column (3, -7) does not enter
    On_s = np.array([[0.5, -1.0, 3.0], [0.25, 2.0, -7.0]])
    assert o.sigma_x(On_s, 2) == -5.3125
    assert o.sigma_x(On_s, 1) == -0.3125


def test_sigma_R_poles_with_exact_rpa_poles_equals_plain_cd(small):
    # the pole-residue form of W behind Eq. sigma_pole is exact when it carries every RPA excitation Omega_s with
    # residue (w^s_nm)^2: the residue term from that model equals plain CD's W built at every residue
    s = small
    n_occ = s["spec"].n_occ
    Om, Z = o.rpa_poles(s["B"], s["D"])
    wamp = o.pole_amplitudes(s["B"], s["D"], s["On"][0], Om, Z)            # [N_b, n_poles]
    poles = np.stack([np.broadcast_to(Om, (n_occ, len(Om))), wamp[:n_occ] ** 2], axis=-1)
    for w in (-10.9, -10.3, -0.95, -0.5):
        ref = o.sigma_R_cd(s["B"], s["D"], s["On"][0], s["eps"], n_occ, w, 1e-3)
        got = o.sigma_R_poles(poles, s["eps"], n_occ, w, 1e-3)
        assert abs(ref) > 1e-3
        assert abs(got - ref) < 1e-10 * max(1.0, abs(ref)), (w, got, ref)
    # a single pole per m reproduces the closed-form one-pole W of an N_aux = 1, N_ov = 1 system
    b, o00, d, e0, e1 = 0.6, 0.7, 9.5, -10.0, -0.5
    om = math.sqrt(d * d + 4 * b * b * d)
    r = 2 * o00 ** 2 * b ** 2 * d / om
    eps2 = np.array([e0, e1, e1 + d])
    pol = np.array([[[om, 0.0]], [[om, r]]])
    w = -5.0
    z = abs(e1 - w) + 1e-3j
    expect = -(4 * o00 ** 2 * b ** 2 * d / (z * z - d * d - 4 * b * b * d))     # -f_m W(z), f_m = -1
    assert abs(o.sigma_R_poles(pol, eps2, 2, w, 1e-3) - expect) < 1e-13


def test_sigma_x_definition(small):
    s = small
    On = s["On"][0]
    assert abs(o.sigma_x(On, s["spec"].n_occ) + sum(On[p, i] ** 2 for p in range(On.shape[0]) for i in range(5))) < 1e-13


# --- Thiele continued fraction --------------------------------------------------------------------------

def _rational_w(z, c, Om):
    z = np.asarray(z, dtype=complex)
    return sum(cj / (z * z - oj * oj) for cj, oj in zip(c, Om))


def test_thiele_interpolates_its_nodes():
    rng = np.random.default_rng(5)
    z = np.concatenate([1j * np.geomspace(0.01, 50, 30), np.linspace(0.1, 9, 12) + 1e-3j])
    W = _rational_w(z, rng.uniform(0.1, 1, 9), rng.uniform(0.3, 8, 9))
    fit = o.thiele_greedy_fit(z, W, 24)
    Tn = o.thiele_eval(fit.a, fit.z2, z[fit.nodes])
    assert np.max(np.abs(Tn - W[fit.nodes]) / np.abs(W[fit.nodes])) < 1e-9


def test_thiele_one_pole_exact_with_two_nodes():
    c, Om = [-0.6], [1.3]
    z = 1j * np.array([0.2, 0.9, 3.0])
    fit = o.thiele_greedy_fit(z, _rational_w(z, c, Om), 2)
    for zz in (0.5 + 0.01j, 4.0 + 1e-3j, 7j):
        assert abs(o.thiele_eval(fit.a, fit.z2, zz) - _rational_w(zz, c, Om)) < 1e-13


def test_thiele_three_poles_exact_with_six_nodes():
    # sum of 3 poles in z^2 is rational of type [2/3] in z^2: exactly M = 6 reciprocal differences
    c, Om = [-0.5, -0.2, -0.05], [0.8, 2.1, 5.0]
    z = 1j * np.geomspace(0.05, 20, 40)
    fit = o.thiele_greedy_fit(z, _rational_w(z, c, Om), 6)
    probe = np.array([0.3 + 0.02j, 1.5 + 0.02j, 3.3 + 0.1j, 9.0 + 0.0j, 0.4j])
    got = o.thiele_eval(fit.a, fit.z2, probe)
    assert np.max(np.abs(got - _rational_w(probe, c, Om))) < 1e-10
    # even M decays at infinity, odd M does not (Sec. 2.4)
    assert abs(o.thiele_eval(fit.a, fit.z2, 1e6j)) < 1e-9
    fit5 = o.thiele_greedy_fit(z, _rational_w(z, c, Om), 5)
    assert abs(o.thiele_eval(fit5.a, fit5.z2, 1e6j)) > 1e-6


def test_thiele_first_node_is_largest_w(small):
    s = small
    fit = o.thiele_greedy_fit(1j * s["xi"], s["Wim"][0][:, 2], 8)
    assert fit.nodes[0] == int(np.argmax(np.abs(s["Wim"][0][:, 2])))
    assert fit.nodes[0] == 0                                     # |W| is largest at the smallest xi
    assert len(set(fit.nodes)) == 8


def test_thiele_breakdown_on_duplicate_nodes():
    z = 1j * np.array([0.5, 0.5, 0.5])
    W = np.array([-1.0, -1.0, -1.0])
    fit = o.thiele_greedy_fit(z, W, 3)
    assert fit.breakdown and len(fit.nodes) < 3


# --- quasiparticle solver -------------------------------------------------------------------------------

def test_qp_fixed_point_linear_sigma():
    eps_n, shift, alpha = -10.6, 0.05, 0.3
    sig = lambda w: alpha * (w - eps_n) + 0.02
    r = o.qp_solve(sig, eps_n, shift, np.linspace(-11, -10, 64))
    expect = eps_n + (shift + 0.02) / (1 - alpha)
    assert r.status == 0 and abs(r.e_qp - expect) < 1e-6 and abs(r.Z - 1 / (1 - alpha)) < 1e-6


def test_qp_bisection_fallback():
    # slope -3: the fixed-point map diverges, the bracketed root is (eps_n + 3 w*) / 4 with Z = 1/4
    eps_n, ws = -10.6, -10.3
    sig = lambda w: -3.0 * (w - ws)
    r = o.qp_solve(sig, eps_n, 0.0, np.linspace(-11, -10, 64))
    assert r.status == 1 and abs(r.e_qp - (eps_n + 3 * ws) / 4) < 1e-8 and abs(r.Z - 0.25) < 1e-6


# --- CD-WAC against plain CD: the continuation error is measured, not pinned ---------------------------------

def test_cdwac_near_real_points_span_residues(small):
    s = small
    zr = o.near_real_points(s["eps"], 5, s["eps"][0], 40)
    assert len(zr) == 40 and zr[0].real == 0.0 and np.all(zr.imag == 1e-3)
    assert abs(zr[-1].real - (abs(o.fermi_level(s["eps"], 5) - s["eps"][0]) + 0.5)) < 1e-12


def test_cdwac_core_qp_close_to_cd(small):
    s = small
    grid = inputs.omega_grid(128)
    P = o.Params(n_imag=100, n_real=40, pade_M=64, eta=1e-3)
    cd = o.run_cd(s["B"], s["D"], s["On"], s["eps"], 5, [0], P, grid, with_sigma=False)
    wac = o.run_cdwac(s["B"], s["D"], s["On"], s["eps"], 5, [0], P, grid, with_sigma=False)
    e_cd, e_wac = cd["states"][0]["qp"].e_qp, wac["states"][0]["qp"].e_qp
    assert cd["states"][0]["qp"].status == 0
    assert abs(e_cd - e_wac) * 27211.386 < 0.01          # well inside 1 meV with 40 near-real points


def test_refined_reference_set_hand_example():
    # eps_F = (eps_HOMO + eps_LUMO)/2 = 0; states 0 and 1 at -10.0 and -9.9 (Sec. 3.3, first quadrant only):
    # core centres |eps_n' - eps_n| span [0, 0.1], radius 0.2 -> [0, 0.3]; 4 points 0, 0.1, 0.2, 0.3
    # valence centres |eps_F - eps_n| span [9.9, 10.0], radius 0.5 -> [9.4, 10.5]; 3 points 9.4, 9.95, 10.5
    eps = np.array([-10.0, -9.9, -1.0, -0.5, 0.5, 2.0])
    z = o.refined_reference_points(eps, 4, eps[[0, 1]], 4, 3, 0.2, 0.5, eta_ref=2e-3)
    np.testing.assert_allclose(z.real, [0.0, 0.1, 0.2, 0.3, 9.4, 9.95, 10.5], rtol=0, atol=1e-14)
    assert np.all(z.imag == 2e-3)
    # one state: the core centre is 0, so the neighbourhood is [0, delta_c]; a single valence point sits on
    # the centre 10.0; an empty region contributes nothing
    z = o.refined_reference_points(eps, 4, eps[[0]], 3, 1, 0.2, 0.5)
    np.testing.assert_allclose(z.real, [0.0, 0.1, 0.2, 10.0], rtol=0, atol=1e-14)
    assert len(o.refined_reference_points(eps, 4, eps[[0]], 0, 2, 0.2, 0.5)) == 2
    # a valence radius wider than the centre is cut at Re z = 0
    z = o.refined_reference_points(eps, 4, eps[[0]], 0, 2, 0.2, 12.0)
    np.testing.assert_allclose(z.real, [0.0, 22.0], rtol=0, atol=1e-13)


def test_refined_set_cdwac_exact_for_few_poles():
    # n_basis 4, n_occ 2: four transitions, so W_nm(z) is a sum of four poles in z^2, a rational function of
    # type [3/4] in z^2; eight Thiele nodes reproduce it exactly and CD-WAC then equals plain CD.  With two
    # imaginary nodes the fit has to take at least six of the refined points.
    rng = np.random.default_rng(11)
    eps = np.array([-10.0, -0.6, 0.3, 1.1])
    B = rng.normal(size=(6, 4)) / np.sqrt(6)
    On = rng.normal(size=(1, 6, 4)) / np.sqrt(6)
    D = o.transition_energies(eps, 2)
    P = o.Params(n_imag=2, n_real=8, pade_M=8, eta=1e-3, real_set="refined", n_core=4, n_val=4, delta_c=0.4,
                 delta_v=0.8)
    grid = np.linspace(-10.5, -10.05, 7)
    wac = o.run_cdwac(B, D, On, eps, 2, [0], P, grid)
    cd = o.run_cd(B, D, On, eps, 2, [0], P, grid)
    assert sum(k >= 2 for k in wac["states"][0]["model"].fits[0].nodes) >= 6
    s_w, s_c = wac["states"][0]["sigma"], cd["states"][0]["sigma"]
    assert np.max(np.abs(s_w - s_c)) < 1e-9 * np.max(np.abs(s_c))


def test_refined_set_brings_core_qp_to_cd(small):
    # measured, not pinned: CD-WAC(20, 20, 100) against plain CD on the small system; without near-real points
    # the same fit is several meV off (Sec. 5.1 reports the refined set reaching meV-level MAEs)
    s = small
    grid = inputs.omega_grid(128)
    cd = o.run_cd(s["B"], s["D"], s["On"], s["eps"], 5, [0], o.Params(n_imag=100, n_real=0), grid,
                  with_sigma=False)
    e_cd = cd["states"][0]["qp"].e_qp
    P = o.Params(n_imag=100, n_real=40, pade_M=64, real_set="refined", n_core=20, n_val=20)
    wac = o.run_cdwac(s["B"], s["D"], s["On"], s["eps"], 5, [0], P, grid, with_sigma=False)
    im = o.run_cdwac(s["B"], s["D"], s["On"], s["eps"], 5, [0], o.Params(n_imag=100, n_real=0, pade_M=64), grid,
                     with_sigma=False)
    err = abs(wac["states"][0]["qp"].e_qp - e_cd) * 27211.386
    err_im = abs(im["states"][0]["qp"].e_qp - e_cd) * 27211.386
    assert err < 0.1 and err_im > 1.0, (err, err_im)
    with pytest.raises(ValueError):
        o.reference_points(s["eps"], 5, s["eps"][[0]], o.Params(n_real=39, real_set="refined"))


def test_thiele_replay_of_greedy_order_is_identical(small):
    s = small
    zr = o.near_real_points(s["eps"], 5, s["eps"][[0]], 20)
    Wre = o.w_complex_table(s["B"], s["D"], s["On"], zr, np.arange(5))[0]
    zc = np.concatenate([1j * s["xi"], zr])
    Wc = np.concatenate([s["Wim"][0][:, 1].astype(complex), Wre[:, 1]])
    fit = o.thiele_greedy_fit(zc, Wc, 30)
    rep, record = o.thiele_replay(zc, Wc, fit.nodes)
    assert np.array_equal(rep.a, fit.a)
    assert all(take == emax for take, emax, _ in record)


# ---- LDL^T without pivoting (Eq. bigLambda's factorisation) -------------------------------------------------------

def test_ldlt_two_by_two_closed_form():
    a, b, c = 3.0, 1.25, 2.0
    L, d = o.ldlt_nopivot(np.array([[a, b], [b, c]]))
    assert np.allclose(d, [a, c - b * b / a], rtol=0, atol=1e-15)
    assert L[1, 0] == pytest.approx(b / a, abs=1e-16) and L[0, 0] == 1.0 and L[1, 1] == 1.0 and L[0, 1] == 0.0


def test_ldlt_real_matches_library_cholesky(small):
    import scipy.linalg
    B = small["B"]
    D = o.transition_energies(small["eps"], small["spec"].n_occ)
    A = np.eye(B.shape[0]) - o.polarizability(B, D, 0.7j).real
    L, d = o.ldlt_nopivot(A)
    C = scipy.linalg.cholesky(A, lower=True)
    assert np.all(d > 0)
    assert np.max(np.abs(L * np.sqrt(d)[None, :] - C)) < 1e-13 * np.max(np.abs(C))


def test_ldlt_complex_symmetric_solves_like_library(small):
    B = small["B"]
    D = o.transition_energies(small["eps"], small["spec"].n_occ)
    A = np.eye(B.shape[0]) - o.polarizability(B, D, 0.31 + 1e-3j)
    L, d = o.ldlt_nopivot(A)
    assert np.max(np.abs((L * d[None, :]) @ L.T - A)) < 1e-12 * np.max(np.abs(A))
    b = np.cos(np.arange(A.shape[0]) * 0.37) + 1j * np.sin(np.arange(A.shape[0]) * 0.11)
    import scipy.linalg
    y = scipy.linalg.solve_triangular(L, b, lower=True, unit_diagonal=True)
    x = scipy.linalg.solve_triangular(L.T, y / d, lower=False, unit_diagonal=True)
    ref = np.linalg.solve(A, b)
    assert np.max(np.abs(x - ref)) < 1e-11 * np.max(np.abs(ref))


def test_ldlt_reads_only_the_lower_triangle():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((40, 40))
    A = np.eye(40) * 40 + X @ X.T
    Ag = np.tril(A) + np.triu(rng.standard_normal((40, 40)), 1)   # garbage above the diagonal
    L1, d1 = o.ldlt_nopivot(A)
    L2, d2 = o.ldlt_nopivot(Ag)
    assert np.array_equal(L1, L2) and np.array_equal(d1, d2)


# ---- spectral function (Sec. 5.5) ---------------------------------------------------------------------------------

def test_spectral_function_lorentzian_closed_form():
    """A constant Sigma = -i gamma gives the Lorentzian gamma / pi / ((omega - eps - shift)^2 + gamma^2)."""
    eps, shift, gamma = -10.6, 0.3, 0.05
    w = np.linspace(-12.0, -8.0, 2001)
    A = o.spectral_function(np.full(w.size, -1j * gamma), eps, w, shift)
    ref = gamma / np.pi / ((w - eps - shift) ** 2 + gamma ** 2)
    assert np.max(np.abs(A - ref)) < 1e-13 * ref.max()


def test_spectral_function_sum_rule_one_pole_self_energy():
    """Sigma(omega) = a / (omega - b + i eta): the quasiparticle and its satellite share unit spectral weight."""
    eps, a, b, eta = -10.6, 0.4, -12.0, 2e-3
    w = np.linspace(-40.0, 20.0, 1_200_001)
    A = o.spectral_function(a / (w - b + 1j * eta), eps, w)
    total = np.trapezoid(A, w)
    assert abs(total - 1.0) < 2e-3, total
    # both poles of G carry weight: solutions of (w - eps)(w - b) = a
    disc = math.sqrt((eps - b) ** 2 + 4 * a)
    w1, w2 = 0.5 * (eps + b + disc), 0.5 * (eps + b - disc)
    z1 = (w1 - b) / (w1 - w2)
    near1 = np.abs(w - w1) < 0.2
    assert abs(np.trapezoid(A[near1], w[near1]) - z1) < 2e-2


# ---- eigenvalue self-consistency, evGW0 and evGW (Sec. 5.4) ------------------------------------------------------

def _one_transition():
    # n_basis 2, n_occ 1, N_aux 1: W_0m(z) = 4 o_0m^2 b^2 D / (z^2 - Omega^2), Omega^2 = D^2 + 4 b^2 D, so
    # Eq. sigma_pole has one pole per orbital with weights (w_0m)^2 = 2 o_0m^2 b^2 D / Omega
    b, o00, o01, e0, e1 = 0.7, 0.5, 0.8, -10.0, 0.6
    return b, o00, o01, e0, e1, np.array([[b]]), np.array([[[o00, o01]]]), np.array([e0, e1])


def _weights(b, o00, o01, d):
    om = math.sqrt(d * d + 4 * b * b * d)
    return om, 2 * o00 ** 2 * b ** 2 * d / om, 2 * o01 ** 2 * b ** 2 * d / om


@pytest.mark.parametrize("method", ["pole", "cd", "cdwac"])
def test_evgw0_one_transition_closed_form(method):
    # evGW0: W stays at the KS transition D = e1 - e0, G carries eps_G = (e, e1); at self-consistency
    # e = e0 + A / (e - e + Omega) + B / (e - e1 - Omega), a quadratic whose root below e1 + Omega is the answer
    b, o00, o01, e0, e1, B, On, eps = _one_transition()
    om, A, Bw = _weights(b, o00, o01, e1 - e0)
    c, d = e0 + A / om, e1 + om
    expect = 0.5 * ((c + d) - math.sqrt((c - d) ** 2 + 4 * Bw))
    P = o.Params(n_imag=100, n_real=8, pade_M=2, eta=1e-8)
    r = o.run_evgw(B, On, eps, 1, [0], P, np.linspace(-11, -9.5, 64), mode="evGW0", method=method)
    assert r["status"] == 0 and r["cycles"] > 1
    assert abs(r["e_qp"][0] - expect) < 1e-9


@pytest.mark.parametrize("method", ["pole", "cd", "cdwac"])
def test_evgw_one_transition_root(method):
    # evGW: W follows eps_G too, D = e1 - e; the fixed point is the root of
    # g(e) = e - e0 - A(e) / Omega(e) - B(e) / (e - e1 - Omega(e)) near e0 (bracketed and bisected)
    from scipy.optimize import brentq
    b, o00, o01, e0, e1, B, On, eps = _one_transition()

    def g(e):
        om, A, Bw = _weights(b, o00, o01, e1 - e)
        return e - e0 - A / om - Bw / (e - e1 - om)

    expect = brentq(g, e0 - 0.5, e0 + 0.1, xtol=1e-14)
    P = o.Params(n_imag=100, n_real=8, pade_M=2, eta=1e-8)
    r = o.run_evgw(B, On, eps, 1, [0], P, np.linspace(-11, -9.5, 64), mode="evGW", method=method)
    assert r["status"] == 0
    assert abs(r["e_qp"][0] - expect) < 1e-9


def test_evgw_cd_and_cdwac_match_the_sum_over_poles():
    # 16 orbitals, 39 transitions: the exact evGW0 / evGW fixed points from Eq. sigma_pole against plain CD and
    # CD-WAC with the subtracted I term; self-consistency moves the core level by 0.3-0.7 mHa from G0W0
    spec = inputs.custom_system(16, 3, 40, seed=3, n_core=1, states=(0,), core_scale=0.3, valence=(-1.1, -0.3),
                                virtual=(0.02, 2.0))
    eps = inputs.eigenvalues(spec)
    B, On = inputs.build_B(spec), inputs.build_On(spec)
    grid = inputs.omega_grid(64)
    P = o.Params(n_imag=60, n_real=20, pade_M=40)
    ref = {}
    for mode in ("evGW0", "evGW"):
        r = {m: o.run_evgw(B, On, eps, 3, [0], P, grid, mode=mode, method=m) for m in ("pole", "cd", "cdwac")}
        assert all(v["status"] == 0 for v in r.values())
        e = r["pole"]["e_qp"][0]
        assert abs(r["cd"]["e_qp"][0] - e) < 2e-8 and abs(r["cdwac"]["e_qp"][0] - e) < 2e-8
        # cycle 1 is G0W0 (G and W from the KS energies)
        D = o.transition_energies(eps, 3)
        g0w0 = o.qp_solve(lambda w: o.sigma_c_pole_sum(B, D, On[0], eps, 3, w, P.eta), eps[0], 0.0, grid)
        assert abs(r["pole"]["history"][0][0] - g0w0.e_qp) < 1e-12
        assert abs(e - g0w0.e_qp) > 1e-4
        # the answer is self-consistent: G built with eps_G[n] = e reproduces e
        G = eps.copy()
        G[0] = e
        Dm = o.transition_energies(G if mode == "evGW" else eps, 3)
        assert abs(eps[0] + o.sigma_c_pole_sum(B, Dm, On[0], G, 3, e, P.eta).real - e) < 1e-6
        ref[mode] = e
    assert abs(ref["evGW"] - ref["evGW0"]) > 1e-4


def test_subtracted_i_term_equals_quadrature_away_from_eps_m(small):
    # far from every eps_m both forms of Eq. In_term agree; 1.6 mHa from eps_n the plain rule misses the narrow
    # Lorentzian that the closed-form part carries (against the sum over poles)
    s = small
    Wz = o.w_imag_table(s["B"], s["D"], s["On"], np.zeros(1))[0, 0]
    args = (s["eps"], 5, s["xi"], s["wxi"])
    for w in (-10.9, -10.3):
        plain = o.sigma_I(s["Wim"][0], *args, w, 1e-3)
        assert abs(plain - o.sigma_I_subtracted(s["Wim"][0], Wz, *args, w, 1e-3)) < 1e-10
    w = s["eps"][0] + 0.0016
    exact = o.sigma_c_pole_sum(s["B"], s["D"], s["On"][0], s["eps"], 5, w, 1e-3)
    R = o.sigma_R_cd(s["B"], s["D"], s["On"][0], s["eps"], 5, w, 1e-3)
    sub = R - o.sigma_I_subtracted(s["Wim"][0], Wz, *args, w, 1e-3)
    plain = R - o.sigma_I(s["Wim"][0], *args, w, 1e-3)
    assert abs(sub.real - exact.real) < 1e-10 < 1e-7 < abs(plain.real - exact.real)


def test_evgw0_one_interpolant_errs_more_than_evgw():
    # measured, not pinned (Sec. 5.4's observation): with the generic 20-point set, evGW0 keeps the interpolant
    # whose references were placed around the KS energies and ends 0.1 meV from the exact fixed point; evGW
    # rebuilds W, the references and the fits around the updated energies and stays within 10^-3 meV
    spec = inputs.custom_system(40, 5, 120, seed=2, n_core=1, states=(0,), core_scale=0.3, valence=(-1.1, -0.3),
                                virtual=(0.02, 2.0))
    eps = inputs.eigenvalues(spec)
    B, On = inputs.build_B(spec), inputs.build_On(spec)
    grid = inputs.omega_grid(128)
    P = o.Params(n_imag=100, n_real=20, pade_M=120)
    err = {}
    for mode in ("evGW0", "evGW"):
        exact = o.run_evgw(B, On, eps, 5, [0], P, grid, mode=mode, method="pole")["e_qp"][0]
        wac = o.run_evgw(B, On, eps, 5, [0], P, grid, mode=mode, method="cdwac")
        assert wac["status"] == 0
        err[mode] = abs(wac["e_qp"][0] - exact) * 27211.386
    assert err["evGW0"] > 0.05 and err["evGW"] < 2e-3 and err["evGW0"] > 30 * err["evGW"], err
