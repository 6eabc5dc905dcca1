"""Writes acene_1200_cdwac_oracle.json and .npz: the CPU oracle's CD-WAC G0W0 for the acene-like system.

System: 1200 orbitals (6 core levels at -10.6 +- 0.01 Ha, 114 valence in [-1.2, -0.25] Ha, 1080 virtuals
log-spaced in [0.01, 5] Ha), N_aux = 4000, seed 1, core state n = 0.  Method: 100-point modified Gauss-Legendre
imaginary grid, 40 generic near-real points, greedy Thiele with M = 64, eta = 1e-3 Ha; Sigma on 128 points in
[-11, -10] Ha; QP by fixed point.  Calls only oracle/ and the seeded input generator (FP64 throughout).
The .json keeps sampled entries; the .npz keeps the whole tables of the state: xi, wxi, W_imag [100][1200],
z_real [40], W_real [40][120], the greedy node orders nodes [120][64] with n_used [120], sigma [128], e_qp.

  --f32-inputs   the same run on the O tensor rounded to FP32 (the inputs the mixed-precision path reads),
                 written to acene_1200_f32in_cdwac_oracle.json / .npz

Run:  python tests/golden/make_acene_reference.py [--f32-inputs]     (about two hours on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import cdwac_oracle as o  # noqa: E402
from paper_2305_15955_gb300 import inputs  # noqa: E402

F32 = "--f32-inputs" in sys.argv
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                   "acene_1200_f32in_cdwac_oracle.json" if F32 else "acene_1200_cdwac_oracle.json")
# sampled table entries kept for full-size parity checks
K_SAMPLES = [0, 7, 31, 63, 99]
M_SAMPLES = [0, 1, 5, 6, 60, 119, 120, 121, 600, 1199]


def main():
    t0 = time.time()
    spec = inputs.acene_system(1)
    eps = inputs.eigenvalues(spec)
    dt = np.float32 if F32 else np.float64
    B = inputs.build_B(spec, dtype=dt).astype(np.float64)
    On = inputs.build_On(spec, dtype=dt).astype(np.float64)
    D = o.transition_energies(eps, spec.n_occ)
    P = o.Params(n_imag=100, n_real=40, pade_M=64, eta=1e-3, eta_ref=1e-3)
    omega = inputs.omega_grid(128)
    res = o.run_cdwac(B, D, On, eps, spec.n_occ, [0], P, omega)
    st = res["states"][0]
    q = st["qp"]
    out = {
        "system": {"name": spec.name, "n_basis": spec.n_basis, "n_occ": spec.n_occ, "n_aux": spec.n_aux,
                   "seed": spec.seed, "states": [0]},
        "params": {"n_imag": P.n_imag, "n_real": P.n_real, "pade_M": P.pade_M, "eta": P.eta, "eta_ref": P.eta_ref,
                   "omega0": P.omega0, "real_margin": P.real_margin},
        "omega": omega.tolist(),
        "qp": {"e_qp": float(q.e_qp), "Z": float(q.Z), "iterations": int(q.iterations), "status": int(q.status)},
        "sigma_re": st["sigma"].real.tolist(),
        "sigma_im": st["sigma"].imag.tolist(),
        "W_imag_samples": [[k, m, float(res["W_imag"][0][k, m])] for k in K_SAMPLES for m in M_SAMPLES],
        "W_real_samples": [[j, m, float(st["W_real"][j, m].real), float(st["W_real"][j, m].imag)]
                           for j in (0, 13, 39) for m in (0, 5, 6, 119)],
        "oracle_seconds": time.time() - t0,
        "oracle_threads": os.cpu_count(),
    }
    if F32:
        out["system"]["inputs"] = "O^{pq}_P rounded to FP32"
    M = P.pade_M
    nodes = np.full((spec.n_occ, M), -1, dtype=np.int32)
    for m, fit in enumerate(st["model"].fits):
        nodes[m, :len(fit.nodes)] = fit.nodes
    np.savez(OUT.replace(".json", ".npz"), xi=res["xi"], wxi=res["wxi"], W_imag=res["W_imag"][0],
             z_real=res["z_real"], W_real=st["W_real"], nodes=nodes,
             n_used=np.array([len(f.nodes) for f in st["model"].fits], dtype=np.int32), sigma=st["sigma"],
             e_qp=np.float64(q.e_qp))
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT}: e_qp = {q.e_qp:.10f} Ha, status {q.status}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
