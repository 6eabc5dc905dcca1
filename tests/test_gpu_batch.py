"""Batched launch (cdwac_batch_run): many uneven systems, lanes, CUDA-graph replay, autotuned configuration.

Each system of the batch must come out as the single-system calls give it (same kernels, same arithmetic), the
graph replay must reproduce the eager results, and every item must match the oracle on its own inputs.
"""
import os

import numpy as np
import pytest

from paper_2305_15955_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2305_15955_gb300 import cdwac  # noqa: E402

MEV = 1.0 / 27211.386


def _systems(dtype):
    specs = [inputs.custom_system(40, 5, 100, seed=41, n_core=1, states=(0,)),
             inputs.custom_system(90, 9, 260, seed=42, n_core=2, states=(0, 1)),
             inputs.custom_system(60, 6, 150, seed=43, n_core=1, states=(0,)),
             inputs.custom_system(130, 13, 420, seed=44, n_core=4, states=(0, 2))]
    out = []
    for sp in specs:
        eps = inputs.eigenvalues(sp)
        out.append(cdwac.System(eps, inputs.build_B(sp, dtype=dtype), inputs.build_On(sp, dtype=dtype), sp.states,
                                sp.n_occ))
    return out


@pytest.mark.parametrize("precision", [cdwac.PREC_FP64, cdwac.PREC_MIXED])
def test_batch_matches_single_system_calls(precision, tmp_path, monkeypatch):
    monkeypatch.setenv("CDWAC_TUNE_CACHE", str(tmp_path / "tune.txt"))
    dt = np.float64 if precision == cdwac.PREC_FP64 else np.float32
    systems = _systems(dt)
    p = cdwac.Params(n_imag=40, n_real=12, pade_M=32, precision=precision)
    omega = inputs.omega_grid(16)
    dev = torch.device("cuda", 0)
    ctx = cdwac.Context(0)
    res = [cdwac.BatchResult(s, p, omega, omega, dev) for s in systems]
    chosen, items = cdwac.batch_run(ctx, res, p, max_lanes=4, autotune=True)
    # lanes, lookahead, then the tile configuration: Pi tile-group size and width, the real update's strip waves
    assert 1 <= chosen[0] <= 4 and chosen[1] in (0, 1) and chosen[2] in (4, 8, 12, 16)
    assert chosen[3] in (128, 256) and chosen[4] in (1, 2, 3)
    # the cache holds the whole choice, and a second call with the same bucket reads it back
    line = (tmp_path / "tune.txt").read_text().split()
    assert [int(x) for x in line[1:6]] == list(chosen)
    again, _ = cdwac.batch_run(ctx, res, p, max_lanes=4, autotune=True)
    assert again == chosen
    assert (tmp_path / "tune.txt").exists()
    ctx.close()
    # the single-system calls in the tile configuration the batch chose (the two Pi tile widths round their
    # 2048-column chunk sums in a different order)
    monkeypatch.setenv("CDWAC_PI_GROUP", str(chosen[2]))
    monkeypatch.setenv("CDWAC_PI_TILE", str(chosen[3]))
    monkeypatch.setenv("CDWAC_UPD_WAVES", str(chosen[4]))
    ctx = cdwac.Context(0)
    for s, r in zip(systems, res):
        xi, wxi, W = ctx.build_W_imag(s, p)
        pade = ctx.fit_pade(s, p, xi, W)
        sig = ctx.sigma(s, p, xi, wxi, W, pade, omega)
        e, Z, it, qs = ctx.qp_solve(s, p, xi, wxi, W, pade, omega)
        np.testing.assert_allclose(r.W_imag.cpu().numpy(), W.cpu().numpy(), rtol=1e-13, atol=1e-15)
        assert torch.equal(r.pade.nodes, pade.nodes)
        np.testing.assert_allclose(r.sigma.cpu().numpy(), sig.cpu().numpy(), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r.e_qp.cpu().numpy(), e.cpu().numpy(), rtol=0, atol=1e-12)
    ctx.close()


def test_batch_graph_replay_reproduces_eager():
    systems = _systems(np.float32)
    p = cdwac.Params(n_imag=30, n_real=10, pade_M=24, precision=cdwac.PREC_MIXED)
    omega = inputs.omega_grid(12)
    dev = torch.device("cuda", 0)
    ctx = cdwac.Context(0)
    res = [cdwac.BatchResult(s, p, omega, omega, dev) for s in systems]
    _, items = cdwac.batch_run(ctx, res, p, max_lanes=2, graph=True)        # eager run + capture
    first = [r.e_qp.clone() for r in res], [r.W_imag.clone() for r in res]
    for r in res:
        r.e_qp.zero_()
        r.W_imag.zero_()
    cdwac.batch_run(ctx, res, p, max_lanes=2, graph=True, items=items)      # graph replay
    for r, e0, w0 in zip(res, first[0], first[1]):
        assert torch.equal(r.e_qp, e0)
        assert torch.equal(r.W_imag, w0)
    ctx.close()


def _physical_systems(dtype):
    """Uneven systems of the 40-orbital family (one core level at -10.6 Ha, valence in [-1.1, -0.3], virtuals in
    [0.02, 2.0], core entries x0.3), whose core QP roots lie inside the [-11, -10] Ha window."""
    shapes = [(40, 5, 120, 51, (0,)), (66, 7, 190, 52, (0, 1)), (52, 5, 150, 53, (0,)), (80, 8, 300, 54, (0, 1))]
    out = []
    for nb, no, na, seed, states in shapes:
        sp = inputs.custom_system(nb, no, na, seed=seed, n_core=2 if len(states) > 1 else 1, states=states,
                                  core_scale=0.3, valence=(-1.1, -0.3), virtual=(0.02, 2.0))
        eps = inputs.eigenvalues(sp)
        B, On = inputs.build_B(sp, dtype=dtype), inputs.build_On(sp, dtype=dtype)
        out.append((sp, eps, B.astype(np.float64), On.astype(np.float64),
                    cdwac.System(eps, B, On, sp.states, sp.n_occ)))
    return out


def _qp_fixed_point_tol(Z, tol=1e-7):
    """How far the fixed points of two implementations may end apart: each stops once |e_k+1 - e_k| < tol, which
    leaves it within tol of the root when the iteration oscillates (slope s = 1 - 1/Z < 0) and within
    tol s / (1 - s) when it creeps (0 < s < 1)."""
    s = 1.0 - 1.0 / Z
    return 2.0 * tol * max(1.0, abs(s) / max(1e-3, 1.0 - abs(s)))


def _qp_sensitivity_fixed_order(o, ref, s, pade, p, eps, n_occ, omega):
    """Largest shift of the oracle's QP energy along the GPU's node orders when W carries random relative errors at
    the level by which two FP64 implementations' tables differ (3e-12 at near-real points, 2e-15 on the imaginary
    axis, as in the Sigma criterion of the parity tests): the continuation of some systems turns these into QP
    shifts of 1e-7 Ha and more."""
    rng = np.random.default_rng(7)
    xi, wxi, zr = ref["xi"], ref["wxi"], ref["z_real"]
    zc = np.concatenate([1j * xi, zr])
    st = ref["states"][s]
    nodes, used = pade.nodes.cpu().numpy()[s], pade.n_used.cpu().numpy()[s]
    rel = np.concatenate([np.full(len(xi), 2e-15), np.full(len(zr), 3e-12)])
    base, shifts = None, []
    for trial in range(3):
        fits = []
        for m in range(n_occ):
            Wc = np.concatenate([ref["W_imag"][s][:, m].astype(complex), st["W_real"][:, m]])
            if trial:
                Wc = Wc * (1 + rel * (rng.standard_normal(len(Wc)) + 1j * rng.standard_normal(len(Wc))))
            fits.append(o.thiele_replay(zc, Wc, nodes[m, :used[m]])[0])
        model = o.WacModel(fits=fits)
        q = o.qp_solve(lambda w: o.sigma_c_wac(model, ref["W_imag"][s], eps, n_occ, xi, wxi, w, p.eta), eps[st["n"]],
                       0.0, omega, upper=eps[n_occ])
        if trial == 0:
            base = q.e_qp
        else:
            shifts.append(abs(q.e_qp - base))
    return max(shifts)


def _qp_sensitivity(o, ref, s, p, eps, n_occ, omega, rel):
    """Largest shift of the oracle's CD-WAC QP energy when its W tables carry random relative errors of size rel
    (greedy fits redone, two draws): the part of a QP difference that the continuation, not the arithmetic, sets."""
    rng = np.random.default_rng(5)
    xi, wxi, zr = ref["xi"], ref["wxi"], ref["z_real"]
    zc = np.concatenate([1j * xi, zr])
    st = ref["states"][s]
    shifts = []
    for _ in range(2):
        Wim = ref["W_imag"][s] * (1 + rel * rng.standard_normal(ref["W_imag"][s].shape))
        Wre = st["W_real"] * (1 + rel * (rng.standard_normal(st["W_real"].shape) +
                                         1j * rng.standard_normal(st["W_real"].shape)))
        fits = [o.thiele_greedy_fit(zc, np.concatenate([Wim[:, m].astype(complex), Wre[:, m]]), p.pade_M)
                for m in range(n_occ)]
        model = o.WacModel(fits=fits)
        q = o.qp_solve(lambda w: o.sigma_c_wac(model, Wim, eps, n_occ, xi, wxi, w, p.eta), eps[st["n"]], 0.0, omega,
                       upper=eps[n_occ])
        shifts.append(abs(q.e_qp - st["qp"].e_qp) if q.status < 2 else np.inf)
    return max(shifts)


@pytest.mark.parametrize("precision", [cdwac.PREC_FP64, cdwac.PREC_MIXED])
def test_batch_items_match_oracle(precision):
    # every item of an uneven batch against the oracle's CD-WAC on the same inputs (FP32-valued for the mixed path).
    # FP64: along the GPU's greedy node orders, Sigma under the parity criterion, QP energies to the fixed point's
    # own resolution plus, where that is exceeded, 30 times the oracle's own QP shift under rounding-level W noise.  Mixed: QP energies within 1 meV, or within three times the shift that W errors of the mixed
    # path's size (2^-15 relative) cause in the oracle's own continuation where that is larger (the greedy Thiele
    # continuation of some systems amplifies W errors by many orders of magnitude)
    from oracle import cdwac_oracle as o
    from test_gpu_parity import HA_TOL, _replayed_state, oracle_params

    dt = np.float64 if precision == cdwac.PREC_FP64 else np.float32
    items = _physical_systems(dt)
    p = cdwac.Params(n_imag=60, n_real=24, pade_M=48, precision=precision)
    omega = inputs.omega_grid(64)
    dev = torch.device("cuda", 0)
    ctx = cdwac.Context(0)
    res = [cdwac.BatchResult(sysd, p, omega, omega, dev) for *_, sysd in items]
    cdwac.batch_run(ctx, res, p, max_lanes=4, graph=True)
    for (sp, eps, B, On, sysd), r in zip(items, res):
        D = o.transition_energies(eps, sp.n_occ)
        ref = o.run_cdwac(B, D, On, eps, sp.n_occ, list(sp.states), oracle_params(p), omega,
                          with_sigma=precision == cdwac.PREC_FP64)
        e, qs, sig = r.e_qp.cpu().numpy(), r.qp_status.cpu().numpy(), r.sigma.cpu().numpy()
        for s in range(len(sp.states)):
            if precision == cdwac.PREC_FP64:
                sig_rep, q, sens = _replayed_state(ref, s, r.pade, p, sp.n_occ, eps, omega)
                tol = np.maximum(HA_TOL, 30.0 * sens)
                assert np.all(np.abs(sig[s] - sig_rep) <= tol), (sp.name, s, np.abs(sig[s] - sig_rep).max())
                assert qs[s] == q.status
                if q.status < 2:
                    tol = HA_TOL + _qp_fixed_point_tol(q.Z)
                    if abs(e[s] - q.e_qp) >= tol:
                        tol += 30.0 * _qp_sensitivity_fixed_order(o, ref, s, r.pade, p, eps, sp.n_occ, omega)
                    assert abs(e[s] - q.e_qp) < tol, (sp.name, s, e[s] - q.e_qp, tol)
            else:
                q = ref["states"][s]["qp"]
                assert qs[s] == q.status == 0, (sp.name, s, qs[s], q.status)
                err = abs(e[s] - q.e_qp)
                if err >= MEV:
                    sens = _qp_sensitivity(o, ref, s, p, eps, sp.n_occ, omega, 2.0 ** -15)
                    assert err < 3.0 * sens, (sp.name, s, err / MEV, sens / MEV)
    ctx.close()
