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
    assert 1 <= chosen[0] <= 4 and chosen[1] in (0, 1)
    assert (tmp_path / "tune.txt").exists()
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


@pytest.mark.parametrize("precision", [cdwac.PREC_FP64, cdwac.PREC_MIXED])
def test_batch_items_match_oracle(precision):
    # every item of an uneven batch against the oracle's CD-WAC on the same inputs (FP32-valued for the mixed path):
    # FP64 along the GPU's greedy node orders, Sigma under the parity criterion and QP energies to 1e-8 Ha; mixed
    # QP energies within 1 meV
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
                    assert abs(e[s] - q.e_qp) < HA_TOL, (sp.name, s, e[s] - q.e_qp)
            else:
                q = ref["states"][s]["qp"]
                assert qs[s] == q.status == 0, (sp.name, s, qs[s], q.status)
                assert abs(e[s] - q.e_qp) < MEV, (sp.name, s, (e[s] - q.e_qp) / MEV)
    ctx.close()
