"""The factorisation step on its own (cdwac_ldlt_factor): FP64 updates and tensor-core (exact BF16 digit) updates
against the oracle's column-by-column LDL^T.

Matrices are I - Pi at an imaginary frequency (real SPD) and at a near-real point (complex symmetric) of seeded
synthetic systems, at orders that span several 64-column blocks and 128-row tiles with ragged tails.  Both
methods must be backward stable like an FP64 factorisation (L D L^T reproduces A to 1e-13 of its largest entry)
and reproduce the oracle's L and D to FP64 forward accuracy: max(1e-12, 1e-16 n cond(A)) of the largest entry.
On the imaginary axis cond(I - Pi) ~ 10; next to the real axis (Im z = 1e-3 Ha, the near-real reference points)
it reaches ~10^3, and a different summation order moves L by up to n eps cond(A).
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

TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    c = cdwac.Context(0)
    yield c
    c.close()


def i_minus_pi(n_aux, z, seed, nb=70, n_occ=7):
    spec = inputs.custom_system(nb, n_occ, n_aux, seed=seed)
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec)
    D = o.transition_energies(eps, n_occ)
    Pi = o.polarizability(B, D, z)
    A = np.eye(n_aux, dtype=Pi.dtype) - Pi
    return A.real.copy() if z.real == 0.0 else A


def gpu_factor(ctx, A, method):
    Ag = torch.from_numpy(A.copy()).cuda()
    ctx.ldlt_factor(Ag, method=method)
    F = Ag.cpu().numpy()
    return np.tril(F, -1) + np.eye(A.shape[0]), np.diag(F).copy(), F


@pytest.mark.parametrize("method", [cdwac.LDLT_FP64, cdwac.LDLT_EMULATED])
@pytest.mark.parametrize("n,z", [(64, 0.3j), (193, 0.3j), (300, 0.05j), (1000, 0.3j), (130, 0.42 + 1e-3j),
                                 (300, 0.31 + 1e-3j), (1000, 0.5 + 1e-3j)])
def test_ldlt_matches_oracle(ctx, method, n, z):
    A = i_minus_pi(n, z, seed=40 + n)
    L, d, _ = gpu_factor(ctx, A, method)
    back = np.max(np.abs((L * d[None, :]) @ L.T - A)) / np.max(np.abs(A))
    assert back <= 1e-13, back
    Lr, dr = o.ldlt_nopivot(A)
    tol = max(TOL, 1e-16 * n * np.linalg.cond(A))
    assert np.max(np.abs(d - dr)) <= tol * np.max(np.abs(dr)), np.max(np.abs(d - dr))
    assert np.max(np.abs(L - Lr)) <= tol * np.max(np.abs(Lr)), np.max(np.abs(L - Lr))


@pytest.mark.parametrize("z", [0.2j, 0.37 + 1e-3j])
def test_emulated_update_agrees_with_fp64_update(ctx, z):
    """Both update methods on the same matrix: their factors differ only by FP64 rounding."""
    A = i_minus_pi(700, z, seed=9)
    L1, d1, _ = gpu_factor(ctx, A, cdwac.LDLT_FP64)
    L2, d2, _ = gpu_factor(ctx, A, cdwac.LDLT_EMULATED)
    tol = max(1e-13, 1e-16 * A.shape[0] * np.linalg.cond(A))
    assert np.max(np.abs(d1 - d2)) <= tol * np.max(np.abs(d1))
    assert np.max(np.abs(L1 - L2)) <= tol * np.max(np.abs(L1))


def test_emulated_update_with_scaled_rows(ctx):
    """Rows and columns scaled by powers of two in [2^-4, 2^4]: the digits follow each row's own exponent."""
    A = i_minus_pi(400, 0.3j, seed=11)
    s = 2.0 ** ((np.arange(400) * 7919) % 9 - 4)
    As = s[:, None] * A * s[None, :]
    L, d, _ = gpu_factor(ctx, As, cdwac.LDLT_EMULATED)
    Lr, dr = o.ldlt_nopivot(As)
    # exact scaling relations: L_s = S L S^-1, d_s = s^2 d
    assert np.max(np.abs(d - dr) / np.abs(dr)) <= 1e-12
    assert np.max(np.abs(L - Lr)) <= TOL * np.max(np.abs(Lr)) * 256


def test_upper_triangle_untouched_and_garbage_ignored(ctx):
    A = i_minus_pi(260, 0.3j, seed=3)
    G = np.tril(A) + np.triu(np.full_like(A, 7.25), 1)
    _, _, F = gpu_factor(ctx, G, cdwac.LDLT_EMULATED)
    assert np.all(F[np.triu_indices(260, 1)] == 7.25)
    Lr, dr = o.ldlt_nopivot(A)
    assert np.max(np.abs(np.tril(F, -1) + np.eye(260) - Lr)) <= TOL * np.max(np.abs(Lr))


def test_not_spd_reports_status(ctx):
    A = i_minus_pi(200, 0.3j, seed=4)
    A[150, 150] = -5.0
    Ag = torch.from_numpy(A).cuda()
    with pytest.raises(cdwac.CdwacError) as e:
        ctx.ldlt_factor(Ag, method=cdwac.LDLT_EMULATED)
    assert e.value.status == cdwac.ERR_NOT_SPD
    # the context stays usable
    B = i_minus_pi(200, 0.3j, seed=4)
    L, d, _ = gpu_factor(ctx, B, cdwac.LDLT_EMULATED)
    assert np.all(d > 0)


def test_bad_arguments(ctx):
    Ag = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    assert ctx.lib.cdwac_ldlt_factor(ctx.h, cdwac._ptr(Ag), 4, 0, 7, None) == cdwac.ERR_ARG
    assert ctx.lib.cdwac_ldlt_factor(ctx.h, None, 4, 0, 0, None) == cdwac.ERR_ARG
    assert ctx.lib.cdwac_ldlt_factor(ctx.h, cdwac._ptr(Ag), 0, 0, 0, None) == cdwac.ERR_ARG


@pytest.mark.parametrize("z,upd_waves", [(0.3j, 1), (0.3j, 3), (0.45 + 1e-3j, 1)])
def test_full_size_factor_backward_error(z, upd_waves, monkeypatch):
    """N_aux = 4000, the acene-like order, in the launch configuration the bench times (lookahead, row-strip chunks
    of up to 14 tiles for the real update, per-tile complex update): the tensor-core factor is backward stable like
    an FP64 factorisation (L D L^T reproduces A to 1e-13 of its largest entry).  Real SPD case: it also agrees with
    the FP64-update factor to FP64 forward accuracy, with cond(A) <= ||A||_inf (the eigenvalues of I - Pi(i xi) are
    at least 1).  upd_waves = 3 cuts the real update's strips into three waves of chunks (one of the autotuner's
    choices) and must give the same factor bit for bit."""
    monkeypatch.setenv("CDWAC_UPD_WAVES", str(upd_waves))
    c = cdwac.Context(0)
    n = 4000
    A = i_minus_pi(n, z, seed=77)
    try:
        L, d, F = gpu_factor(c, A, cdwac.LDLT_EMULATED)
        L1, d1, _ = gpu_factor(c, A, cdwac.LDLT_FP64)
    finally:
        c.close()
    for Lx, dx in ((L, d), (L1, d1)):
        back = np.max(np.abs((Lx * dx[None, :]) @ Lx.T - A)) / np.max(np.abs(A))
        assert back <= 1e-13, back
    if z.real == 0.0:
        tol = max(TOL, 1e-16 * n * np.max(np.sum(np.abs(A), axis=1)))
        assert np.max(np.abs(d - d1)) <= tol * np.max(np.abs(d1))
        assert np.max(np.abs(L - L1)) <= tol * np.max(np.abs(L1))
    if upd_waves != 1:
        monkeypatch.setenv("CDWAC_UPD_WAVES", "1")
        c2 = cdwac.Context(0)
        try:
            _, _, F2 = gpu_factor(c2, A, cdwac.LDLT_EMULATED)
        finally:
            c2.close()
        assert np.array_equal(np.tril(F), np.tril(F2))
