"""Conditioning of the CD-WAC continuation on the acene-like system, from a GPU table dump (CPU oracle only).

Reads the .npz that `bench.py --accuracy --dump FILE` writes (the GPU's W(i xi) and W(z) tables, greedy node
orders, Sigma over the 128-point window and the QP energy of the core state) and, with the oracle's continued
fraction arithmetic (Eqs. pade, pre_rec, rec_eq; Sec. 3.2), prints one JSON line with
  * Sigma from the GPU's tables along the GPU's node orders, against the GPU's own Sigma (the continued-fraction
    arithmetic of the two implementations on identical data);
  * how far Sigma over the window and the QP energy move when W carries random relative errors of a given size
    with the node orders held fixed (the condition number of the continuation, separate from any arithmetic);
  * with the full stored oracle tables (acene_1200_cdwac_oracle.npz, from make_acene_reference.py): Sigma and the
    QP energy from the GPU's tables along the oracle's orders against the oracle's own.

Run:  python tests/golden/analyse_acene_dump.py DUMP.npz      (a few minutes on 8 cores)
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cdwac_oracle as o  # noqa: E402
from paper_2305_15955_gb300 import inputs  # noqa: E402

HA_MEV = 27211.386
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "acene_1200_cdwac_oracle.npz")


def main(path):
    spec = inputs.acene_system(1)
    eps = inputs.eigenvalues(spec)
    n_occ = spec.n_occ
    omega = inputs.omega_grid(128)
    d = np.load(path)
    xi, wxi, zr = d["xi"], d["wxi"], d["z_real"]
    zc = np.concatenate([1j * xi, zr])

    def model_of(Wim, Wre, orders, used, rel_i=0.0, rel_r=0.0, seed=0):
        rng = np.random.default_rng(seed)
        if rel_i:
            Wim = Wim * (1 + rel_i * rng.standard_normal(Wim.shape))
        fits = []
        for m in range(n_occ):
            Wr = Wre[:, m]
            if rel_r:
                Wr = Wr * (1 + rel_r * (rng.standard_normal(len(Wr)) + 1j * rng.standard_normal(len(Wr))))
            Wc = np.concatenate([Wim[:, m].astype(complex), Wr])
            fits.append(o.thiele_replay(zc, Wc, orders[m, :used[m]])[0])
        return o.WacModel(fits=fits), Wim

    def sigma(model, Wim):
        return np.array([o.sigma_c_wac(model, Wim, eps, n_occ, xi, wxi, w, 1e-3) for w in omega])

    def qp(model, Wim):
        return o.qp_solve(lambda w: o.sigma_c_wac(model, Wim, eps, n_occ, xi, wxi, w, 1e-3), eps[0], 0.0, omega,
                          upper=eps[n_occ])

    mev = lambda x: float(np.max(np.abs(x))) * HA_MEV
    out = {"dump": os.path.basename(path)}
    base, Wim0 = model_of(d["W_imag"], d["W_real"], d["nodes"], d["n_used"])
    s0 = sigma(base, Wim0)
    q0 = qp(base, Wim0)
    out["sigma_gpu_vs_oracle_arithmetic_same_tables_and_orders_meV"] = mev(d["sigma"] - s0)
    out["qp_gpu_vs_oracle_arithmetic_same_tables_and_orders_meV"] = float(d["e_qp"] - q0.e_qp) * HA_MEV
    out["sigma_max_abs_meV"] = mev(s0)
    for rel in (1e-13, 1e-12, 1e-10):
        out[f"sigma_shift_meV_W_noise_{rel:g}_fixed_orders"] = max(
            mev(sigma(*model_of(d["W_imag"], d["W_real"], d["nodes"], d["n_used"], rel, rel, sd)) - s0)
            for sd in range(2))
    for rel in (1e-8, 1e-6, 2e-5):
        out[f"qp_shift_meV_W_imag_noise_{rel:g}_fixed_orders"] = max(
            abs(qp(*model_of(d["W_imag"], d["W_real"], d["nodes"], d["n_used"], rel, 0.0, sd)).e_qp - q0.e_qp)
            * HA_MEV for sd in range(2))
        out[f"qp_shift_meV_W_real_noise_{rel:g}_fixed_orders"] = max(
            abs(qp(*model_of(d["W_imag"], d["W_real"], d["nodes"], d["n_used"], 0.0, rel, sd)).e_qp - q0.e_qp)
            * HA_MEV for sd in range(2))
    if os.path.exists(GOLD):
        g = np.load(GOLD)
        mo, Wo = model_of(d["W_imag"], d["W_real"], g["nodes"], g["n_used"])
        out["sigma_gpu_tables_oracle_orders_vs_oracle_meV"] = mev(sigma(mo, Wo) - g["sigma"])
        out["qp_gpu_tables_oracle_orders_vs_oracle_meV"] = float(qp(mo, Wo).e_qp - g["e_qp"]) * HA_MEV
        out["node_orders_identical_fraction"] = float(np.mean(
            [np.array_equal(d["nodes"][m, :d["n_used"][m]], g["nodes"][m, :g["n_used"][m]]) for m in range(n_occ)]))
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1])
