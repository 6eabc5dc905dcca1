"""Plain FP64 CPU oracle for contour-deformation G0W0 of core levels: plain CD and CD-WAC.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA library and never calls it.

Every function follows one passage of Panades-Barrueta & Golze, "Accelerating core-level GW calculations by
combining the contour deformation approach with the analytic continuation of W" (arXiv 2305.15955), written
in the paper's order and notation.  Library primitives (matrix products, Cholesky and LU factorisations,
Gauss-Legendre nodes, a symmetric eigensolver) serve as single steps; nothing is blocked, fused or reordered.

Conventions (readings of points the paper leaves open):
  * closed shell, spin factor 2 in the polarizability (Eq. piriv carries none; Sec. 2.1 drops spin);
  * the imaginary-axis grid is Gauss-Legendre on (-1, 1) mapped by xi = omega0 (1 + x) / (1 - x);
  * the Fermi level is the middle of the HOMO-LUMO gap; occupations are fixed by orbital index;
  * theta(0) = 1/2 in the residue factors f_m (Eq. ffact);
  * complex arguments z = x + i*eta carry the infinitesimal of Eq. piriv, so
    Pi(z) = 2 sum_ia O^ia [1/(z - D_ia) - 1/(z + D_ia)] O^ia, an even function of z;
  * greedy Thiele: the first node maximises |W|, every later node maximises the L1 error
    |Re(T - W)| + |Im(T - W)| of the current convergent over the remaining nodes; ties go to the lowest
    candidate index; a node whose reciprocal difference is not finite ends the fit (breakdown);
  * near-real references (Sec. 3.3): one set per system, centres taken at omega = eps_n of the requested states;
    refined core centres |eps_n' - eps_n|, valence centres |eps_F - eps_n|, neighbourhoods cut at Re z = 0;
  * evGW0 / evGW (Sec. 5.4): the requested states' QP energies replace their entries in G (and in W's transition
    energies for evGW), other orbitals keep their KS energies; the I term takes W_nm(0) out of the quadrature and
    integrates its part in closed form, because Sigma_n is then evaluated at its own G energy.

Parity pins (tests/test_oracle_pins.py): the sum-over-poles self-energy of Eq. sigma_pole from a full RPA
diagonalisation, the closed-form one-pole system, Gauss-Legendre exactness and known integrals,
Thiele interpolation and one-pole exactness, invariants of Pi, Lambda and W, a hand-worked refined reference set,
closed-form one-transition evGW0 / evGW fixed points.  The CD-WAC continuation error itself has no exact pin: it
is a measured quantity of the method.
"""
from __future__ import annotations

import dataclasses
import decimal

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------------------------------------
# Frequency grids and occupations
# ---------------------------------------------------------------------------------------------------------


def _legendre_dec(n, x):
    """P_n(x) and P_{n-1}(x) by the three-term recurrence (j P_j = (2j-1) x P_{j-1} - (j-1) P_{j-2}), Decimal."""
    p0, p1 = decimal.Decimal(1), x
    if n == 0:
        return p0, p0
    for j in range(2, n + 1):
        p0, p1 = p1, ((2 * j - 1) * x * p1 - (j - 1) * p0) / j
    return p1, p0


def imaginary_grid(n_imag: int, omega0: float = 1.0):
    """Modified Gauss-Legendre grid on [0, inf) for the I_n quadrature (Sec. 4, 'modified Gauss-Legendre grid').

    x_k, w_k are the n-point Gauss-Legendre nodes and weights on (-1, 1): the roots of P_n and
    2 / ((1 - x^2) P_n'(x)^2).  xi_k = omega0 (1+x_k)/(1-x_k) and the weight carries the Jacobian
    d xi / d x = 2 omega0 / (1 - x)^2.  Every number is computed with 50 significant digits (Newton's method on
    P_n in Python's decimal arithmetic, started from numpy's nodes) and rounded once to FP64, so the grid is the
    exact rule correctly rounded.  Returns (xi, wxi), xi ascending.
    """
    ctx = decimal.Context(prec=50)
    with decimal.localcontext(ctx):
        D = decimal.Decimal
        x0, _ = np.polynomial.legendre.leggauss(n_imag)
        om = D(float(omega0))
        xi = np.empty(n_imag)
        wxi = np.empty(n_imag)
        for k, xs in enumerate(x0):
            x = D(float(xs))
            for _ in range(100):
                pn, pn1 = _legendre_dec(n_imag, x)
                dp = n_imag * (x * pn - pn1) / (x * x - 1) if n_imag > 1 else D(1)
                dx = pn / dp
                x -= dx
                if abs(dx) < D(10) ** -45:
                    break
            pn, pn1 = _legendre_dec(n_imag, x)
            dp = n_imag * (x * pn - pn1) / (x * x - 1) if n_imag > 1 else D(1)
            w = 2 / ((1 - x * x) * dp * dp)
            xi[k] = float(om * (1 + x) / (1 - x))
            wxi[k] = float(w * 2 * om / ((1 - x) * (1 - x)))
    return xi, wxi


def fermi_level(eps, n_occ):
    """epsilon_F read as the middle of the HOMO-LUMO gap (the paper gives no number)."""
    return 0.5 * (eps[n_occ - 1] + eps[n_occ])


def transition_energies(eps, n_occ):
    """D_ia = eps_a - eps_i, flattened as ia = i * n_virt + a (the column order of O^{ia}_P)."""
    return (eps[None, n_occ:] - eps[:n_occ, None]).reshape(-1)


# ---------------------------------------------------------------------------------------------------------
# Screened Coulomb interaction in RI-V (Eqs. piriv, bigLambda, wriv; Sec. 2.3)
# ---------------------------------------------------------------------------------------------------------


def polarizability(B, D, z):
    """Pi_PQ(z), Eq. piriv with spin factor 2: 2 sum_ia O^ia_P [1/(z - D_ia) - 1/(z + D_ia)] O^ia_Q.

    B is O^{ia}_P as an [N_aux, N_occ*N_virt] array, D the matching D_ia.  For purely imaginary z the
    bracket is real (-2 D / (xi^2 + D^2)) and a real matrix is returned.
    """
    z = complex(z)
    if z.real == 0.0:
        # z = i xi: 1/(i xi - D) - 1/(i xi + D) = -2 D / (xi^2 + D^2), real
        w = 2.0 * (-2.0 * D / (z.imag ** 2 + D ** 2))
    else:
        w = 2.0 * (1.0 / (z - D) - 1.0 / (z + D))
        # B is real: the real and imaginary parts of the sum are two real products
        return (B * w.real[None, :]) @ B.T + 1j * ((B * w.imag[None, :]) @ B.T)
    return (B * w[None, :]) @ B.T


def screened_lambda(Pi):
    """Lambda = (I - Pi)^{-1} - I, Eq. bigLambda, formed as the identical (I - Pi)^{-1} Pi.

    Solving (I - Pi) Lambda = Pi avoids subtracting I from (I - Pi)^{-1}: at large imaginary frequency
    Lambda ~ Pi ~ 1/xi^2 is small and the subtraction would keep only ~1e-16 / |Lambda| of relative accuracy.
    On the imaginary axis I - Pi is real symmetric positive definite (Pi is negative semidefinite) and is
    solved through its Cholesky factor; elsewhere it is complex symmetric and an LU factorisation with
    partial pivoting is used.
    """
    n = Pi.shape[0]
    A = np.eye(n, dtype=Pi.dtype) - Pi
    if np.isrealobj(A):
        c = scipy.linalg.cho_factor(A, lower=True)
        return scipy.linalg.cho_solve(c, Pi)
    lu = scipy.linalg.lu_factor(A)
    return scipy.linalg.lu_solve(lu, Pi)


def ldlt_nopivot(A):
    """Square-root-free Cholesky A = L D L^T without pivoting of the symmetric matrix I - Pi (Eq. bigLambda):
    real symmetric positive definite on the imaginary axis, complex symmetric (transpose, not conjugate) near the
    real axis.  Column by column (Crout order):
        d_j  = A_jj - sum_{k<j} L_jk^2 d_k,
        L_ij = (A_ij - sum_{k<j} L_ik d_k L_jk) / d_j,   i > j.
    Returns (L unit lower triangular, d).  Reads only the lower triangle of A."""
    A = np.asarray(A)
    n = A.shape[0]
    L = np.eye(n, dtype=A.dtype)
    d = np.zeros(n, dtype=A.dtype)
    for j in range(n):
        d[j] = A[j, j] - np.sum(L[j, :j] ** 2 * d[:j])
        L[j + 1:, j] = (A[j + 1:, j] - (L[j + 1:, :j] * d[:j]) @ L[j, :j]) / d[j]
    return L, d


def w_elements(On_s, Lam, m_idx=None):
    """W^c_nm = sum_PQ O^{nm}_P Lambda_PQ O^{mn}_Q, Eq. wriv, for one state n and orbitals m.

    On_s is O^{n m}_P as [N_aux, N_basis] (symmetric in n, m).  Returns W for every m (or for m_idx).
    """
    O = On_s if m_idx is None else On_s[:, m_idx]
    return np.sum(O * (Lam @ O), axis=0)          # column m: o_m^T (Lambda o_m)


def w_imag_table(B, D, On, xi):
    """W_nm(i xi_k) for all states n, all k, all m: the wmatrix(F_Im) step (Sec. 3.4).  [n_states, n_xi, N_b]."""
    n_states, _, nb = On.shape
    W = np.empty((n_states, len(xi), nb))
    for k, x in enumerate(xi):
        Lam = screened_lambda(polarizability(B, D, 1j * x))
        for s in range(n_states):
            W[s, k] = w_elements(On[s], Lam)
    return W


def w_complex_table(B, D, On, z_list, m_idx):
    """W_nm(z_j) for complex points z_j and orbitals m_idx: the wmatrix(F_real) step.  [n_states, n_z, len(m)]."""
    n_states = On.shape[0]
    W = np.empty((n_states, len(z_list), len(m_idx)), dtype=complex)
    for j, z in enumerate(z_list):
        Lam = screened_lambda(polarizability(B, D, z))
        for s in range(n_states):
            W[s, j] = w_elements(On[s], Lam, m_idx)
    return W


# ---------------------------------------------------------------------------------------------------------
# Self-energy by contour deformation (Eqs. cdmain, In_term, Rn_term, ffact, cdselfe; Sec. 2.3)
# ---------------------------------------------------------------------------------------------------------


def occupation_sign(eps, n_occ):
    """sgn(eps_F - eps_m): +1 for occupied m, -1 for virtual m."""
    s = -np.ones(len(eps))
    s[:n_occ] = 1.0
    return s


def sigma_I(W_imag_s, eps, n_occ, xi, wxi, omega, eta):
    """I_n(omega), Eq. In_term, for one state from its W_nm(i xi_k) table [n_xi, N_b].

    W(i w') is even in w', so the integral over the whole imaginary axis is folded onto [0, inf):
    1/(2 pi) int dw' W(iw') / (a + iw') = 1/(2 pi) int_0^inf dw' W(iw') [1/(a + iw') + 1/(a - iw')],
    with a_m = omega - eps_m - i eta sgn(eps_F - eps_m).
    """
    a = omega - eps - 1j * eta * occupation_sign(eps, n_occ)          # [N_b]
    kern = 1.0 / (a[None, :] + 1j * xi[:, None]) + 1.0 / (a[None, :] - 1j * xi[:, None])   # [n_xi, N_b]
    return np.sum(wxi[:, None] * W_imag_s * kern) / (2.0 * np.pi)


def residue_factors(eps, n_occ, omega):
    """f_m of Eq. ffact: -theta(eF - e_m) theta(e_m - w) + theta(e_m - eF) theta(w - e_m), theta(0) = 1/2."""
    th = lambda x: np.where(x > 0, 1.0, np.where(x < 0, 0.0, 0.5))
    occ = np.zeros(len(eps))
    occ[:n_occ] = 1.0
    return -occ * th(eps - omega) + (1.0 - occ) * th(omega - eps)


def sigma_R_cd(B, D, On_s, eps, n_occ, omega, eta):
    """R_n(omega), Eq. Rn_term, plain CD: W_nm built directly at every residue |eps_m - omega| + i eta."""
    f = residue_factors(eps, n_occ, omega)
    R = 0.0 + 0.0j
    for m in np.nonzero(f)[0]:
        z = abs(eps[m] - omega) + 1j * eta
        Lam = screened_lambda(polarizability(B, D, z))
        R += f[m] * w_elements(On_s, Lam, [m])[0]
    return R


def sigma_c_cd(B, D, On_s, W_imag_s, eps, n_occ, xi, wxi, omega, eta):
    """Sigma^c_n(omega) = R_n - I_n (Eq. cdselfe without the static exchange), plain CD."""
    return sigma_R_cd(B, D, On_s, eps, n_occ, omega, eta) - sigma_I(W_imag_s, eps, n_occ, xi, wxi, omega, eta)


def sigma_x(On_s, n_occ):
    """Static exchange in RI-V, Eq. exs: Sigma^x_n = -sum_i^occ (ni|in) = -sum_i sum_P (O^{ni}_P)^2."""
    return -np.sum(On_s[:, :n_occ] ** 2)


# ---------------------------------------------------------------------------------------------------------
# Analytic continuation of W: greedy Thiele reciprocal differences (Eqs. pade, pre_rec, rec_eq; Sec. 3.2)
# ---------------------------------------------------------------------------------------------------------


def thiele_eval(a, z2_nodes, z):
    """T^M(z), Eq. pade: a_1 / (1 + a_2 (z^2 - zt_1^2) / (1 + ... a_M (z^2 - zt_{M-1}^2))).

    Evaluated from the innermost level outwards.  a has M entries, z2_nodes the M node values zt_p^2.
    """
    z2 = np.asarray(z, dtype=complex) ** 2
    t = np.ones_like(z2)
    for p in range(len(a) - 1, 0, -1):            # levels M .. 2 (0-based p = M-1 .. 1)
        t = 1.0 + a[p] * (z2 - z2_nodes[p - 1]) / t
    return a[0] / t


@dataclasses.dataclass
class ThieleFit:
    nodes: list            # candidate indices in the order they entered the fraction
    a: np.ndarray          # complex coefficients a_1..a_M
    z2: np.ndarray         # zt_p^2 of the chosen nodes
    breakdown: bool        # True if the fit stopped early on a non-finite reciprocal difference


def thiele_greedy_fit(z, W, M, first="absmax", criterion="max", tol=0.0):
    """Greedy Thiele interpolation of W over candidate nodes z (Sec. 3.2, the greedy procedure).

    g_1(z_i) = W(z_i); g_p(z_i) = (g_{p-1}(zt_{p-1}) - g_{p-1}(z_i)) / ((z_i^2 - zt_{p-1}^2) g_{p-1}(z_i)) (Eq. rec_eq),
    a_p = g_p(zt_p) (Eq. pre_rec).  The first node is argmax |W|; node p >= 2 is the remaining candidate with the
    largest (criterion 'max') or smallest ('min') L1 error of the convergent T^{p-1}.  Stops after M nodes, or
    earlier once the largest remaining L1 error is below tol * max|W| (reading: the paper fixes M only; past
    that point the candidates' errors are rounding noise and the choice among them is not defined by the data).
    """
    z = np.asarray(z, dtype=complex)
    W = np.asarray(W, dtype=complex)
    z2 = z ** 2
    n = len(z)
    M = min(M, n)
    g = W.copy()                                   # g_1 at every candidate
    stop_below = tol * np.max(np.abs(W))
    remaining = np.ones(n, dtype=bool)
    if first == "absmax":
        k = int(np.argmax(np.abs(W)))
    elif first == "max":
        k = int(np.argmax(W.real))
    else:
        k = 0
    nodes = [k]
    a = [g[k]]
    remaining[k] = False
    breakdown = False
    for p in range(2, M + 1):
        rem = np.nonzero(remaining)[0]
        if len(rem) == 0:
            break
        zt2_prev = z2[nodes[-1]]
        a_prev = a[-1]
        with np.errstate(all="ignore"):
            g[rem] = (a_prev - g[rem]) / ((z2[rem] - zt2_prev) * g[rem])
            T = thiele_eval(np.array(a), z2[np.array(nodes)], z[rem])
            err = np.abs((T - W[rem]).real) + np.abs((T - W[rem]).imag)
        err = np.where(np.isfinite(err), err, np.inf)
        if err.max() < stop_below:
            break
        pick = int(np.argmax(err)) if criterion == "max" else int(np.argmin(err))
        k = int(rem[pick])
        if not np.isfinite(g[k]):
            breakdown = True
            break
        nodes.append(k)
        a.append(g[k])
        remaining[k] = False
    return ThieleFit(nodes=nodes, a=np.array(a, dtype=complex), z2=z2[np.array(nodes)], breakdown=breakdown)


def thiele_replay(z, W, order, criterion="max"):
    """Reciprocal differences (Eqs. pre_rec, rec_eq) along a prescribed node order, with the greedy record.

    Returns the ThieleFit for `order` and, for every step p >= 2, (L1 error of the node taken, largest and
    smallest L1 error over the candidates remaining at that step).  A node order is a valid greedy order when
    each node taken carries the extreme error of its step (up to rounding).
    """
    z = np.asarray(z, dtype=complex)
    W = np.asarray(W, dtype=complex)
    z2 = z ** 2
    g = W.copy()
    remaining = np.ones(len(z), dtype=bool)
    nodes = [int(order[0])]
    a = [g[nodes[0]]]
    remaining[nodes[0]] = False
    record = []
    for k in order[1:]:
        k = int(k)
        rem = np.nonzero(remaining)[0]
        with np.errstate(all="ignore"):
            g[rem] = (a[-1] - g[rem]) / ((z2[rem] - z2[nodes[-1]]) * g[rem])
            T = thiele_eval(np.array(a), z2[np.array(nodes)], z[rem])
            err = np.abs((T - W[rem]).real) + np.abs((T - W[rem]).imag)
        err = np.where(np.isfinite(err), err, np.inf)
        record.append((float(err[list(rem).index(k)]), float(err.max()), float(err.min())))
        nodes.append(k)
        a.append(g[k])
        remaining[k] = False
    fit = ThieleFit(nodes=nodes, a=np.array(a, dtype=complex), z2=z2[np.array(nodes)], breakdown=False)
    return fit, record


def near_real_points(eps, n_occ, eps_states, n_real, eta_ref=1e-3, margin=0.5):
    """Generic near-real reference set omega_G (Sec. 3.3): n_real equidistant points x_j + i eta_ref with
    x_j spanning [0, max_n |eps_F - eps_n| + margin], i.e. every residue |eps_m - omega| up to the Fermi level
    of every requested state n (one set per system)."""
    if n_real == 0:
        return np.zeros(0, dtype=complex)
    top = max(abs(fermi_level(eps, n_occ) - e) for e in np.atleast_1d(eps_states)) + margin
    x = np.linspace(0.0, top, n_real)
    return x + 1j * eta_ref


def _neighbourhood(c_lo, c_hi, delta, n):
    """n equidistant abscissae on the neighbourhood of radius delta around the centres [c_lo, c_hi], cut to the
    first quadrant (Re z >= 0, Sec. 3.3): [max(0, c_lo - delta), c_hi + delta], both ends included; a single point
    sits at the middle of the centres."""
    if n == 0:
        return np.zeros(0)
    if n == 1:
        return np.array([max(0.0, 0.5 * (c_lo + c_hi))])
    return np.linspace(max(0.0, c_lo - delta), c_hi + delta, n)


def refined_reference_points(eps, n_occ, eps_states, n_core, n_val, delta_c, delta_v, eta_ref=1e-3):
    """Refined near-real reference set omega_C U omega_V (Sec. 3.3), n_core + n_val points x_j + i eta_ref.

    omega_C: a neighbourhood of radius delta_c around the typical core-level residue |eps_c - omega|, taken at
    omega = eps_n with eps_c a requested core level, i.e. the centres |eps_n' - eps_n| over the requested states
    (0 for one state).  omega_V: a neighbourhood of radius delta_v around the valence residue |eps_F - omega| at
    omega = eps_n, i.e. the centres |eps_F - eps_n|.  One set per system, like the generic set; points lie in the
    first quadrant.  The Pade order of the paper's CD-WAC(N_core, N_valence, N_Im) is the sum of the three sizes."""
    e = np.atleast_1d(np.asarray(eps_states, dtype=float))
    ef = fermi_level(eps, n_occ)
    xc = _neighbourhood(0.0, float(e.max() - e.min()), delta_c, n_core)
    rv = np.abs(ef - e)
    xv = _neighbourhood(float(rv.min()), float(rv.max()), delta_v, n_val)
    return np.concatenate([xc, xv]) + 1j * eta_ref


def reference_points(eps, n_occ, eps_states, params):
    """F_real of Sec. 3.3 for params.real_set: "generic" (omega_G) or "refined" (omega_C U omega_V)."""
    if params.real_set == "generic":
        return near_real_points(eps, n_occ, eps_states, params.n_real, params.eta_ref, params.real_margin)
    if params.real_set == "refined":
        if params.n_core + params.n_val != params.n_real:
            raise ValueError("the refined set needs n_real = n_core + n_val")
        return refined_reference_points(eps, n_occ, eps_states, params.n_core, params.n_val, params.delta_c,
                                        params.delta_v, params.eta_ref)
    raise ValueError(f"unknown reference set {params.real_set!r}")


@dataclasses.dataclass
class WacModel:
    """CD-WAC continuation of one state: one Thiele fit per occupied m."""
    fits: list             # ThieleFit per occupied m (index = m)


def fit_wac(W_imag_s, W_real_s, xi, z_real, n_occ, M, first="absmax", criterion="max", tol=0.0):
    """The AC step (Sec. 3.4): for each occupied m, fit W_nm over F_wac = F_Im U F_real."""
    fits = []
    zc = np.concatenate([1j * np.asarray(xi), np.asarray(z_real, dtype=complex)])
    for m in range(n_occ):
        Wc = np.concatenate([W_imag_s[:, m].astype(complex), W_real_s[:, m] if len(z_real) else np.zeros(0)])
        fits.append(thiele_greedy_fit(zc, Wc, M, first, criterion, tol))
    return WacModel(fits=fits)


def sigma_R_wac(model, eps, n_occ, omega, eta):
    """R_n(omega), Eq. Rn_term, with W_nm(|eps_m - omega| + i eta) replaced by T^M_nm (occupied m only)."""
    f = residue_factors(eps, n_occ, omega)
    R = 0.0 + 0.0j
    for m in np.nonzero(f)[0]:
        if m >= n_occ:
            raise ValueError("CD-WAC continuation covers occupied residues only (omega below the LUMO)")
        fit = model.fits[m]
        R += f[m] * thiele_eval(fit.a, fit.z2, abs(eps[m] - omega) + 1j * eta)
    return complex(R)


def sigma_R_poles(poles_s, eps, n_occ, omega, eta):
    """R_n(omega), Eq. Rn_term, with W_nm(z) = -sum_s r_s 2 Omega_s / (Omega_s^2 - z^2) from a pole model
    poles_s [n_occ][n_poles][2] = (Omega_s, r_s) per occupied m (the learned continuation; not in the paper)."""
    f = residue_factors(eps, n_occ, omega)
    R = 0.0 + 0.0j
    for m in np.nonzero(f)[0]:
        if m >= n_occ:
            raise ValueError("the pole model covers occupied residues only (omega below the LUMO)")
        z = abs(eps[m] - omega) + 1j * eta
        Om, r = poles_s[m, :, 0], poles_s[m, :, 1]
        R += f[m] * np.sum(-r * 2.0 * Om / (Om * Om - z * z))
    return complex(R)


def sigma_c_wac(model, W_imag_s, eps, n_occ, xi, wxi, omega, eta):
    """Sigma^c_n(omega) = R_n - I_n with the continued residue term (CD-WAC)."""
    return sigma_R_wac(model, eps, n_occ, omega, eta) - sigma_I(W_imag_s, eps, n_occ, xi, wxi, omega, eta)


# ---------------------------------------------------------------------------------------------------------
# Quasiparticle equation (Eq. qp_eq) and the sum-over-poles self-energy (Eq. sigma_pole)
# ---------------------------------------------------------------------------------------------------------


@dataclasses.dataclass
class QPResult:
    e_qp: float
    Z: float
    iterations: int
    status: int            # 0 converged by fixed point, 1 by bracketed bisection, 2 not converged


def spectral_function(sigma_c, eps_n, omega, shift=0.0):
    """Diagonal spectral function A_nn(omega) = |Im[(omega - eps_n - shift - Sigma^c_n(omega))^{-1}]| / pi
    (Sec. 5.5: the imaginary part of the Green's function, with shift = Sigma^x_n - v^xc_n as in Eq. qp_eq).
    The paper gives A_nn up to a factor; 1/pi makes a single quasiparticle pole integrate to one.  sigma_c holds
    Sigma^c_n at the points omega."""
    g = 1.0 / (np.asarray(omega) - eps_n - shift - np.asarray(sigma_c))
    return np.abs(g.imag) / np.pi


def qp_solve(sigma_fn, eps_n, shift, omega_grid, tol=1e-7, max_iter=100, h=1e-5, bisect_tol=1e-9, upper=np.inf):
    """Solve e = eps_n + shift + Re Sigma^c_n(e) (Eq. qp_eq with shift = Sigma^x_n - v^xc_n).

    Fixed-point iteration from eps_n until |e_new - e| < tol.  If it does not converge, every sign change of
    f(w) = w - eps_n - shift - Re Sigma(w) between neighbouring points of omega_grid is bisected to bisect_tol;
    roots with |f| < 1e-6 are kept and the one with the largest Z in (0, 1] is returned.
    Z = 1 / (1 - d Re Sigma / d w) by a central difference of step h.  An iterate at or above `upper` (for CD-WAC
    the LUMO: the continuation covers occupied residues only) ends the fixed point as not converged.
    """
    def zfac(e):
        d = (sigma_fn(e + h).real - sigma_fn(e - h).real) / (2.0 * h)
        return 1.0 / (1.0 - d)

    e = eps_n
    for it in range(1, max_iter + 1):
        e_new = eps_n + shift + sigma_fn(e).real
        if not e_new < upper:
            break
        if abs(e_new - e) < tol:
            return QPResult(e_new, zfac(e_new), it, 0)
        e = e_new
    f = lambda w: w - eps_n - shift - sigma_fn(w).real
    fv = np.array([f(w) for w in omega_grid])
    best = None
    for j in range(len(omega_grid) - 1):
        if fv[j] == 0.0 or fv[j] * fv[j + 1] < 0:
            lo, hi, flo = omega_grid[j], omega_grid[j + 1], fv[j]
            while hi - lo > bisect_tol:
                mid = 0.5 * (lo + hi)
                fm = f(mid)
                if fm * flo <= 0:
                    hi = mid
                else:
                    lo, flo = mid, fm
            r = 0.5 * (lo + hi)
            if abs(f(r)) < 1e-6:
                Zr = zfac(r)
                if 0.0 < Zr <= 1.0 and (best is None or Zr > best[1]):
                    best = (r, Zr)
    if best is not None:
        return QPResult(best[0], best[1], max_iter, 1)
    return QPResult(e, zfac(e), max_iter, 2)


def rpa_poles(B, D):
    """Neutral excitations of direct RPA in RI form: Omega_s^2 and eigenvectors of
    C = D^2 + 4 D^{1/2} B^T B D^{1/2} (closed shell), the Omega_s of Eq. sigma_pole."""
    sq = np.sqrt(D)
    C = np.diag(D ** 2) + 4.0 * (sq[:, None] * (B.T @ B) * sq[None, :])
    Om2, Z = np.linalg.eigh(C)
    return np.sqrt(Om2), Z


def pole_amplitudes(B, D, On_s, Omega, Z):
    """w^s_nm with (w^s_nm)^2 = <nm|P_s|mn> of Eq. sigma_pole: w^s_nm = sqrt(2) sum_ia (O^{nm} . O^{ia}) D^{1/2} Z_ia,s / sqrt(Omega_s).
    Returns [N_basis, n_poles]."""
    v = (On_s.T @ B) * np.sqrt(D)[None, :]          # [N_b, N_ov]
    return np.sqrt(2.0) * (v @ Z) / np.sqrt(Omega)[None, :]


def sigma_c_pole_sum(B, D, On_s, eps, n_occ, omega, eta):
    """Sigma^c_n(omega) by the sum over poles, Eq. sigma_pole (the fully analytic O(N^6) route)."""
    Omega, Z = rpa_poles(B, D)
    wamp = pole_amplitudes(B, D, On_s, Omega, Z)
    sgn = occupation_sign(eps, n_occ)
    den = omega - eps[:, None] + (Omega[None, :] - 1j * eta) * sgn[:, None]
    return np.sum(wamp ** 2 / den)


def w_imag_pole_sum(B, D, On_s, xi):
    """W^c_nm(i xi) = -sum_s (w^s_nm)^2 2 Omega_s / (xi^2 + Omega_s^2), the pole form of W behind Eq. sigma_pole."""
    Omega, Z = rpa_poles(B, D)
    wamp = pole_amplitudes(B, D, On_s, Omega, Z)
    xi = np.atleast_1d(xi)
    return -np.einsum("ms,ks->km", wamp ** 2, 2.0 * Omega[None, :] / (xi[:, None] ** 2 + Omega[None, :] ** 2))


# ---------------------------------------------------------------------------------------------------------
# The whole procedure (Sec. 3.4): CD and CD-WAC G0W0 for a list of states
# ---------------------------------------------------------------------------------------------------------


@dataclasses.dataclass
class Params:
    n_imag: int = 100
    omega0: float = 1.0
    n_real: int = 40
    eta_ref: float = 1e-3
    eta: float = 1e-3
    pade_M: int = 64
    greedy_first: str = "absmax"
    greedy_criterion: str = "max"
    real_margin: float = 0.5
    pade_tol: float = 0.0
    real_set: str = "generic"      # "generic" (omega_G) or "refined" (omega_C U omega_V), Sec. 3.3
    n_core: int = 20               # refined set sizes; CD-WAC(20, 20, N_Im) is the paper's recommendation (Sec. 5.1)
    n_val: int = 20
    delta_c: float = 0.5           # neighbourhood radii (Ha), "parameters that can be tuned" (Sec. 3.3)
    delta_v: float = 0.5


def run_cdwac(B, D, On, eps, n_occ, states, params: Params, omega_grid, shifts=None, with_sigma=True):
    """CD-WAC G0W0 (Sec. 3.4): W on the imaginary grid, W at the near-real points, greedy Thiele fit per
    occupied m, Sigma^c on omega_grid and the QP solution per state."""
    xi, wxi = imaginary_grid(params.n_imag, params.omega0)
    Wim = w_imag_table(B, D, On, xi)
    zr = reference_points(eps, n_occ, eps[list(states)], params)
    Wre_all = w_complex_table(B, D, On, zr, np.arange(n_occ)) if len(zr) else None
    out = {"xi": xi, "wxi": wxi, "W_imag": Wim, "z_real": zr, "states": []}
    for s, n in enumerate(states):
        Wre = Wre_all[s] if len(zr) else np.zeros((0, n_occ), complex)
        model = fit_wac(Wim[s], Wre, xi, zr, n_occ, params.pade_M, params.greedy_first, params.greedy_criterion,
                        params.pade_tol)
        sig = lambda w, s=s, model=model: sigma_c_wac(model, Wim[s], eps, n_occ, xi, wxi, w, params.eta)
        sh = 0.0 if shifts is None else shifts[s]
        res = {"n": n, "z_real": zr, "W_real": Wre, "model": model,
               "qp": qp_solve(sig, eps[n], sh, omega_grid, upper=eps[n_occ])}
        if with_sigma:
            res["sigma"] = np.array([sig(w) for w in omega_grid])
        out["states"].append(res)
    return out


def run_cd(B, D, On, eps, n_occ, states, params: Params, omega_grid, shifts=None, with_sigma=True):
    """Plain CD G0W0 (Sec. 3.4): the residue term builds W at every residue of every frequency."""
    xi, wxi = imaginary_grid(params.n_imag, params.omega0)
    Wim = w_imag_table(B, D, On, xi)
    out = {"xi": xi, "wxi": wxi, "W_imag": Wim, "states": []}
    for s, n in enumerate(states):
        sig = lambda w, s=s: sigma_c_cd(B, D, On[s], Wim[s], eps, n_occ, xi, wxi, w, params.eta)
        sh = 0.0 if shifts is None else shifts[s]
        res = {"n": n, "qp": qp_solve(sig, eps[n], sh, omega_grid)}
        if with_sigma:
            res["sigma"] = np.array([sig(w) for w in omega_grid])
        out["states"].append(res)
    return out


# ---------------------------------------------------------------------------------------------------------
# Eigenvalue self-consistency beyond G0W0 (Sec. 5.4): evGW0 and evGW
# ---------------------------------------------------------------------------------------------------------


def sigma_I_subtracted(W_imag_s, W_zero_s, eps, n_occ, xi, wxi, omega, eta):
    """I_n(omega) of Eq. In_term with W_nm(0) taken out of the quadrature and integrated in closed form.

    The folded kernel K(a, xi) = 1/(a + i xi) + 1/(a - i xi) = 2a / (a^2 + xi^2), a = omega - eps_m - i eta s_m,
    has width |omega - eps_m|: once omega comes closer to eps_m than the first quadrature nodes (every evGW cycle
    evaluates Sigma_n next to its own updated eps_n) the rule misses most of it.  Its integral over [0, inf) is
    pi sgn(omega - eps_m) (0 at omega = eps_m, the theta(0) = 1/2 reading), so
    I_n = 1/(2 pi) sum_m [pi sgn(omega - eps_m) W_nm(0) + sum_k w_k (W_nm(i xi_k) - W_nm(0)) K(a_m, xi_k)];
    the remaining integrand vanishes like xi^2 at the origin, where W is even and smooth.
    W_zero_s [N_b] holds W_nm(0)."""
    a = omega - eps - 1j * eta * occupation_sign(eps, n_occ)
    kern = 1.0 / (a[None, :] + 1j * xi[:, None]) + 1.0 / (a[None, :] - 1j * xi[:, None])
    closed = np.pi * np.sign(omega - eps) * W_zero_s
    return (np.sum(closed) + np.sum(wxi[:, None] * (W_imag_s - W_zero_s[None, :]) * kern)) / (2.0 * np.pi)


def _ev_tables(B, eps_W, On, n_occ, states, params, method, xi):
    """W-side tables of one cycle, built from the energies eps_W: transition energies, W(i xi), W(0) and, for
    CD-WAC, the near-real references (placed from eps_W) and the greedy Thiele fits."""
    D = transition_energies(eps_W, n_occ)
    t = {"D": D}
    if method == "pole":
        return t
    t["W_imag"] = w_imag_table(B, D, On, xi)
    t["W_zero"] = w_imag_table(B, D, On, np.zeros(1))[:, 0, :]
    if method == "cdwac":
        zr = reference_points(eps_W, n_occ, eps_W[list(states)], params)
        Wre = w_complex_table(B, D, On, zr, np.arange(n_occ)) if len(zr) else None
        t["models"] = [fit_wac(t["W_imag"][s], Wre[s] if len(zr) else np.zeros((0, n_occ), complex), xi, zr, n_occ,
                               params.pade_M, params.greedy_first, params.greedy_criterion, params.pade_tol)
                       for s in range(len(states))]
    return t


def run_evgw(B, On, eps, n_occ, states, params: Params, omega_grid, mode="evGW0", method="cdwac", shifts=None,
             cycle_tol=1e-6, max_cycles=30):
    """evGW0 or evGW (Sec. 5.4) for the requested states.

    Cycle k solves e_n = eps_n + shift_n + Re Sigma^c_n(e_n) (Eq. qp_eq, eps_n the KS energy) with G built from
    eps_G: the KS energies whose requested-state entries carry the QP energies of cycle k-1 (eps_G = eps in cycle
    1, which is G0W0); every other orbital keeps its KS energy.
      evGW0: W from the KS transition energies, built (and, for CD-WAC, fitted) once for all cycles.
      evGW:  W from the transition energies of eps_G, rebuilt every cycle together with the near-real references
             (placed from eps_G) and the Thiele fits.
    method: "cdwac" (continued residue term), "cd" (W built at every residue) or "pole" (sum over poles of
    Eq. sigma_pole, exact for both modes).  The I term is sigma_I_subtracted.  Ends when every requested state
    moves by less than cycle_tol between two cycles (converged), when a QP equation has no solution (status 2) or
    after max_cycles."""
    if mode not in ("evGW0", "evGW") or method not in ("cdwac", "cd", "pole"):
        raise ValueError("mode evGW0|evGW, method cdwac|cd|pole")
    xi, wxi = imaginary_grid(params.n_imag, params.omega0)
    epsG = np.array(eps, dtype=float)
    idx = list(states)
    tabs = None
    history = []
    for cycle in range(1, max_cycles + 1):
        if tabs is None or mode == "evGW":
            tabs = _ev_tables(B, epsG if mode == "evGW" else np.asarray(eps, float), On, n_occ, idx, params, method,
                              xi)
        res = []
        for s, n in enumerate(idx):
            if method == "pole":
                sig = lambda w, s=s, G=epsG.copy(): sigma_c_pole_sum(B, tabs["D"], On[s], G, n_occ, w, params.eta)
            elif method == "cd":
                sig = lambda w, s=s, G=epsG.copy(): (sigma_R_cd(B, tabs["D"], On[s], G, n_occ, w, params.eta) -
                                                     sigma_I_subtracted(tabs["W_imag"][s], tabs["W_zero"][s], G,
                                                                        n_occ, xi, wxi, w, params.eta))
            else:
                sig = lambda w, s=s, G=epsG.copy(): (sigma_R_wac(tabs["models"][s], G, n_occ, w, params.eta) -
                                                     sigma_I_subtracted(tabs["W_imag"][s], tabs["W_zero"][s], G,
                                                                        n_occ, xi, wxi, w, params.eta))
            sh = 0.0 if shifts is None else shifts[s]
            res.append(qp_solve(sig, eps[n], sh, omega_grid, upper=epsG[n_occ] if method == "cdwac" else np.inf))
        e = np.array([q.e_qp for q in res])
        history.append(e)
        if any(q.status == 2 for q in res):
            return {"e_qp": e, "qp": res, "cycles": cycle, "status": 2, "history": history}
        if np.max(np.abs(e - epsG[idx])) < cycle_tol:
            return {"e_qp": e, "qp": res, "cycles": cycle, "status": 0, "history": history}
        epsG[idx] = e
    return {"e_qp": e, "qp": res, "cycles": max_cycles, "status": 1, "history": history}
