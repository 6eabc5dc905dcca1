"""Benchmark of the CD-WAC core-level G0W0 hot path on GB300 (one JSON line on stdout).

A step is one pass of the whole path for one synthetic system: W_nm(i xi) on the 100-point imaginary grid
(Pi on the tensor cores, FP64 LDL^T, W projection), 40 near-real reference points (complex Pi, complex LDL^T),
greedy Thiele fits for every occupied m, Sigma_c on a 128-point real-frequency grid and the QP equation.
The headline value is core-state Sigma_c(omega) evaluations per second over whole steps; the line also carries
the QP solve time (= ms_per_step), Sigma evals/s with the W tables already built, the plain-CD cost on the same
GPU, the accuracy against the FP64 oracle, the roofline of the dominant kernel and the CPU oracle baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload acene|small]
  torchrun --nproc-per-node N bench.py --gpus N ...   (N > 1: independent replicas, one system per rank)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# The step runs ~25 streams (frequency lanes, each with critical-path and side streams); 32 hardware work queues
# instead of the default 8 avoid false dependencies between them.  Read when CUDA initialises, so set before torch.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "core-state Sigma_c(w) evals/sec and QP solve time, CD-WAC vs plain CD on 1 GB300 at <=1 meV"
UNIT = "Sigma_c evals/s"
HA_PER_MEV = 1.0 / 27211.386


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["acene", "medium", "small", "batch", "acarbon"], default="acene")
    ap.add_argument("--batch-systems", type=int, default=16, help="systems in the batch workload")
    ap.add_argument("--qp-max-iter", type=int, default=100,
                    help="fixed-point iterations of the QP solve before the bisection fallback (100 = the method's)")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, plain-CD and CPU-baseline measurements")
    ap.add_argument("--n-imag", type=int, default=100, help="imaginary grid points (100 = the workload's value)")
    ap.add_argument("--n-real", type=int, default=40, help="near-real reference points (40 = the workload's value)")
    ap.add_argument("--refined-map", action="store_true",
                    help="instead of the step: QP error of CD-WAC(N_core, N_val, N_Im) against plain CD over a grid "
                         "of refined-set sizes (one JSON line)")
    ap.add_argument("--delta-c", type=float, default=0.5, help="refined core neighbourhood radius (Ha) of the map")
    ap.add_argument("--delta-v", type=float, default=0.5, help="refined valence neighbourhood radius (Ha) of the map")
    ap.add_argument("--accuracy", action="store_true",
                    help="instead of the timed steps: one step of --workload at --precision, its W tables, greedy node "
                         "orders and Sigma compared with the stored FP64 oracle result (one JSON line)")
    ap.add_argument("--dump", default=None, help="with --accuracy: write the GPU tables to this .npz file")
    return ap.parse_args()


def workload(name):
    from paper_2305_15955_gb300 import inputs
    if name == "acene":
        spec = inputs.acene_system(1)
        desc = ("acene-like: N_basis=1200 (6 core at -10.6+-0.01 Ha, 114 valence in [-1.2,-0.25], 1080 virtual "
                "log-spaced in [0.01,5]), N_aux=4000, seed 1, core state n=0; 100 imaginary GL points, 40 near-real "
                "points, greedy Thiele M=64, 128 omega in [-11,-10] Ha")
    elif name == "medium":
        spec = inputs.custom_system(600, 60, 2000, seed=1, n_core=6, states=(0,))
        desc = ("medium acene-like: N_basis=600 (6 core, 54 valence, 540 virtual), N_aux=2000, seed 1, core state "
                "n=0; O^ia = 0.26 GB FP32 (above L2); 100 GL points, 40 near-real, M=64, 128 omega")
    else:
        spec = inputs.small_system()
        desc = "small: N_basis=40, N_aux=120, seed 0, core state n=0; 100 GL points, 40 near-real, M=64, 128 omega"
    return spec, desc


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch
    import torch.distributed as dist
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    return dist.get_rank(), ws, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value, device):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands, on a bounded sample of the same workload
# ------------------------------------------------------------------------------------------------------------

def oracle_sample(spec, B, On, eps):
    """Time the oracle on one imaginary frequency (Pi, Cholesky solve, W for every m) and scale to a whole step:
    100 imaginary points + 40 near-real points (complex arithmetic, counted as 4x an imaginary point).
    Returns (seconds per step, seconds measured)."""
    from oracle import cdwac_oracle as o
    D = o.transition_energies(eps, spec.n_occ)
    xi, _ = o.imaginary_grid(100)
    t0 = time.perf_counter()
    Lam = o.screened_lambda(o.polarizability(B, D, 1j * xi[50]))
    o.w_elements(On[0], Lam)
    t_imag = time.perf_counter() - t0
    return t_imag * (100 + 4 * 40), t_imag


def run_reference(args, rank, ws, dist):
    if rank != 0:
        return
    from paper_2305_15955_gb300 import inputs
    spec, desc = workload(args.workload)
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec)
    On = inputs.build_On(spec)
    for _ in range(args.warmup):
        oracle_sample(spec, B, On, eps)
    est, meas = [], 0.0
    for _ in range(args.steps):
        s, m = oracle_sample(spec, B, On, eps)
        est.append(s)
        meas += m
    t_step = float(np.mean(est))
    value = len(spec.states) * 128 / t_step
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc,
                       "timing": "extrapolated: each step times the oracle's W(i xi) at one of the 100 imaginary "
                                 "frequencies and scales it by 100 + 4 x 40 frequency-equivalents (a near-real point "
                                 "is a complex build, about four real ones); the whole step is about 2000 s of CPU"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "W_nm(i xi) at 1 of 100 imaginary frequencies per step (numpy/OpenBLAS FP64), "
                                       "scaled by 100 + 4*40 points; fits and Sigma not counted (negligible)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------------------

def ldlt_update_macs(n):
    """Multiply-adds of the blocked LDL^T's trailing updates (64-column panels, lower triangle with the diagonal):
    sum over block steps of R (R + 1) / 2 * 64, R the rows below the panel."""
    return sum((n - k1) * (n - k1 + 1) // 2 * 64 for k1 in range(64, n, 64))


def isolated_profile(cdwac, sysd, mixed, dev):
    """Per-launch device times of the step's kernels with every launch alone on the GPU: a second context with one
    frequency lane and the LDL^T updates in line (no side stream), level-2 event timers, a few imaginary frequencies
    and near-real points of the same system, each measured on a second pass after a warm-up pass.
    Returns ({class: (launches, ms)} of the imaginary-axis W build, the same of the near-real points)."""
    import torch
    saved = {k: os.environ.get(k) for k in ("CDWAC_FREQ_LANES", "CDWAC_LOOKAHEAD")}
    os.environ["CDWAC_FREQ_LANES"], os.environ["CDWAC_LOOKAHEAD"] = "1", "0"
    try:
        ctx = cdwac.Context(dev.index if dev.index is not None else 0)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    prec = cdwac.PREC_MIXED if mixed else cdwac.PREC_FP64
    p_i = cdwac.Params(n_imag=4, n_real=0, pade_M=4, precision=prec)
    p_r = cdwac.Params(n_imag=4, n_real=2, pade_M=6, precision=prec)
    out = []
    for _ in range(2):
        ctx.profile(2)
        ctx.profile_read()
        xi, wxi, W = ctx.build_W_imag(sysd, p_i)
        torch.cuda.synchronize()
        prof_i = ctx.profile_read()
        ctx.fit_pade(sysd, p_r, xi, W)
        torch.cuda.synchronize()
        prof_r = ctx.profile_read()
        out = (prof_i, prof_r, p_i.n_imag, p_r.n_real)
    ctx.profile(False)
    ctx.close()
    return out


def rooflines(spec, prm, iso, peaks, peak_kind, mixed):
    """Rooflines of the step's heavy kernels from the isolated per-launch times, and each kernel class's share of
    the serialised step (per-launch time x launches in a step of prm.n_imag imaginary and prm.n_real near-real
    points).  Peaks: the measured BF16 burst rate (kernels timed alone), divided by the BF16 products issued per
    algorithmic multiply-add where the algorithmic count is of FP32/FP64 multiply-adds."""
    prof_i, prof_r, ni_iso, nr_iso = iso
    n, nov = spec.n_aux, spec.n_ov
    per = lambda prof, k: (prof[k][1] / max(1, prof[k][0])) if k in prof else None
    tot = lambda prof, k: prof[k][1] if k in prof else 0.0
    step_ms = {}
    for k in set(prof_i) | set(prof_r):
        if k in ("ldlt",):    # the whole factorisation; its parts are the ldlt_* classes
            continue
        step_ms[k] = tot(prof_i, k) / ni_iso * prm.n_imag + tot(prof_r, k) / max(1, nr_iso) * prm.n_real
    total = sum(step_ms.values()) or 1.0
    shares = {k: {"serialised_ms_per_step": v, "share": v / total} for k, v in
              sorted(step_ms.items(), key=lambda kv: -kv[1])}
    bf16 = peaks["bf16_tflops"]
    rl = {}
    pi_flops = n * (n + 1) / 2 * nov * 2.0
    if per(prof_i, "pi_tc_imag"):
        ach = pi_flops / (per(prof_i, "pi_tc_imag") / 1e3) / 1e12
        rl["pi_tc_imag"] = {"bound": "tensor", "achieved": ach, "peak": bf16 / 3, "unit": "TFLOP/s",
                            "frac": ach / (bf16 / 3), "traffic": None,
                            "peak_basis": f"bf16_tflops/3 ({peak_kind}, burst: timed alone): three BF16 products "
                                          "per FP32 multiply-add",
                            "algorithmic_flops_per_launch": pi_flops, "launch_ms": per(prof_i, "pi_tc_imag"),
                            "serialised_ms_per_step": per(prof_i, "pi_tc_imag") * prm.n_imag}
    if per(prof_r, "pi_tc_complex"):
        ach = 2 * pi_flops / (per(prof_r, "pi_tc_complex") / 1e3) / 1e12
        rl["pi_tc_complex"] = {"bound": "tensor", "achieved": ach, "peak": bf16 / 3, "unit": "TFLOP/s",
                               "frac": ach / (bf16 / 3), "traffic": None,
                               "peak_basis": f"bf16_tflops/3 ({peak_kind}, burst)",
                               "algorithmic_flops_per_launch": 2 * pi_flops,
                               "launch_ms": per(prof_r, "pi_tc_complex"),
                               "serialised_ms_per_step": per(prof_r, "pi_tc_complex") * prm.n_real}
    macs = ldlt_update_macs(n)
    for name, prof, cnt, digits in (("oz_update_real", prof_i, ni_iso, 28), ("oz_update_complex", prof_r, nr_iso, 144)):
        if mixed and tot(prof, "ldlt_update") > 0:
            t_fact = tot(prof, "ldlt_update") / cnt                      # ms of trailing updates per factorisation
            flops = digits * macs * 2.0
            ach = flops / (t_fact / 1e3) / 1e12
            rl[name] = {"bound": "tensor", "achieved": ach, "peak": bf16, "unit": "TFLOP/s", "frac": ach / bf16,
                        "traffic": None, "peak_basis": f"bf16_tflops ({peak_kind}, burst)",
                        "algorithmic_flops_per_factorisation": flops,
                        "ms_per_factorisation": t_fact,
                        "serialised_ms_per_step": t_fact * (prm.n_imag if digits == 28 else prm.n_real),
                        "note": f"{digits} exact BF16 digit products per FP64-equivalent multiply-add of the "
                                "trailing updates (lower triangle, 64-column panels); the kernel's own launches"}
    return rl, shares

def run_ours(args, rank, ws, dist):
    import torch

    import __graft_entry__ as g
    from paper_2305_15955_gb300 import cdwac, inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        g.build()
    barrier(dist)
    g.build()
    spec, desc = workload(args.workload)
    mixed = args.precision == "mixed"
    odt = np.float32 if mixed else np.float64
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec, dtype=odt)
    On = inputs.build_On(spec, dtype=odt)
    omega = inputs.omega_grid(128)
    sysd = cdwac.System(eps, B, On, spec.states, spec.n_occ, device=dev)
    prm = cdwac.Params(n_imag=args.n_imag, n_real=args.n_real, pade_M=min(64, args.n_imag + args.n_real),
                       precision=cdwac.PREC_MIXED if mixed else cdwac.PREC_FP64)
    ctx = cdwac.Context(local)
    omega_d = torch.as_tensor(omega, device=dev)
    pade = ctx.alloc_pade(sysd, prm)

    def step(system):
        xi, wxi, W = ctx.build_W_imag(system, prm, sync=False)
        ctx.fit_pade(system, prm, xi, W, pade, sync=False)
        sig = ctx.sigma(system, prm, xi, wxi, W, pade, omega_d, sync=False)
        e, Z, it, qs = ctx.qp_solve(system, prm, xi, wxi, W, pade, omega_d, sync=False)
        return xi, wxi, W, sig, e, Z, it, qs

    allow = (cdwac.ERR_PADE_BREAKDOWN, cdwac.ERR_QP_NOT_CONVERGED)   # recorded in the line, not fatal
    for _ in range(args.warmup):
        out = step(sysd)
    ctx.sync_status(allow)
    torch.cuda.synchronize()
    barrier(dist)

    stream = torch.cuda.current_stream()
    ctx.profile(True)
    ctx.profile_read()
    launches0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        barrier(dist)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            out = step(sysd)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(dist)
    ctx.sync_status(allow)
    launches = ctx.launch_count() - launches0
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(dist, ms, dev)
    n_eval = len(spec.states) * len(omega)
    value = ws * n_eval / (ms / 1e3)
    xi, wxi, W, sig, e, Z, it, qs = out
    e_qp = float(e.cpu()[0])

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x3-f32acc+f64" if mixed else "f64", "data": "synthetic",
            "config": {"workload": desc if (args.n_imag, args.n_real) == (100, 40) else
                       desc + f" [reduced: n_imag={args.n_imag}, n_real={args.n_real}]", "precision": args.precision,
                       "l2": "inputs larger than L2 (O^ia = %.2f GB)" % (B.nbytes / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "qp_solve_ms": ms, "qp": {"e_qp_Ha": e_qp, "Z": float(Z.cpu()[0]), "iterations": int(it.cpu()[0]),
                                      "status": int(qs.cpu()[0])},
            "gpu_launches": int(launches // args.steps)}

    # per-kernel breakdown inside the timed step (classes overlap across the concurrent lanes)
    peaks, peak_kind = measured_peaks()
    tot = sum(v[1] for v in prof.values()) or 1.0
    line["kernels_in_step"] = {k: {"regions": v[0] // args.steps, "ms_per_step": v[1] / args.steps,
                                   "share": v[1] / tot} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}
    n, nov = spec.n_aux, spec.n_ov
    pi_flops = n * (n + 1) / 2 * nov * 2.0               # lower triangle, 1 MAC = 2 flops
    in_step = {}
    if "pi_tc_imag" in prof:
        cnt, tms = prof["pi_tc_imag"]
        ach = pi_flops / (tms / cnt / 1e3) / 1e12
        pk = peaks["bf16_tflops_sustained"] / 3.0
        in_step["pi_tc_imag"] = {"achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                                 "peak_basis": f"bf16_tflops_sustained/3 ({peak_kind}): inside the long step, with "
                                               "the other lanes' kernels sharing the GPU"}
    line["pi_in_step"] = in_step
    line["clocks"] = clk.summary()

    if rank == 0 and not args.no_extras:
        # rooflines from per-launch times of kernels running alone, and the serialised shares that pick the dominant
        # kernel
        iso = isolated_profile(cdwac, sysd, mixed, dev)
        rl, shares = rooflines(spec, prm, iso, peaks, peak_kind, mixed)
        line["kernels_serialised"] = shares
        if rl:
            dom = max(rl, key=lambda k: rl[k]["serialised_ms_per_step"])
            line["roofline"] = dict(rl[dom], kernel=dom,
                                    basis="kernel timed alone (one lane, updates in line) with CUDA events; the "
                                          "dominant class of the serialised step")
        line["roofline_all"] = rl

        # Sigma throughput with the W tables and fits already built (the CD-WAC residue term is a fraction)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        many = torch.linspace(-11.0, -10.0, 4096, dtype=torch.float64, device=dev)
        ctx.sigma(sysd, prm, xi, wxi, W, pade, many, sync=False)
        t0.record(stream)
        for _ in range(5):
            ctx.sigma(sysd, prm, xi, wxi, W, pade, many, sync=False)
        t1.record(stream)
        torch.cuda.synchronize()
        line["sigma_evals_per_s_after_setup"] = 5 * 4096 / (t0.elapsed_time(t1) / 1e3)

        # plain CD on the same GPU: one Sigma evaluation builds Pi(z) and a complex LDL^T per residue
        w1 = torch.tensor([e_qp], dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        tp = time.perf_counter()
        ctx.sigma(sysd, prm, xi, wxi, W, None, w1, sync=True)
        t_cd = time.perf_counter() - tp
        n_res = int(np.sum(eps[:spec.n_occ] > e_qp))
        line["plain_cd"] = {"precision": args.precision, "sigma_eval_s": t_cd, "residues_per_eval": n_res,
                            "per_residue_ms": 1e3 * t_cd / max(1, n_res), "sigma_evals_per_s": 1.0 / t_cd,
                            "qp_solve_s_extrapolated": t_cd * (int(it.cpu()[0]) + 2),
                            "note": "one plain-CD Sigma(omega) timed at omega = e_qp in the step's precision; the QP "
                                    "time is that cost times the CD-WAC iteration count + 2 (Z), extrapolated"}
        line["cdwac_vs_plain_cd_qp_speedup_extrapolated"] = line["plain_cd"]["qp_solve_s_extrapolated"] / (ms / 1e3)
        if mixed:
            # plain CD in FP64 on the same GPU (the reference CD-WAC is compared with): one Sigma evaluation at an
            # omega with exactly five occupied levels above it, i.e. five residues, each an FP64 Pi(z), complex LDL^T
            # and W; per-residue cost times the residues and Sigma evaluations of a QP solve, extrapolated
            sys64 = cdwac.System(eps, B.astype(np.float64), On.astype(np.float64), spec.states, spec.n_occ,
                                 device=dev)
            p64 = cdwac.Params(n_imag=prm.n_imag, n_real=prm.n_real, pade_M=prm.pade_M, precision=cdwac.PREC_FP64)
            w5 = torch.tensor([0.5 * (eps[spec.n_occ - 6] + eps[spec.n_occ - 5])], dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            tp = time.perf_counter()
            ctx.sigma(sys64, p64, xi, wxi, W, None, w5, sync=True)
            t5 = time.perf_counter() - tp
            del sys64
            torch.cuda.empty_cache()
            per_res = t5 / 5.0
            line["plain_cd_fp64"] = {"per_residue_s": per_res, "residues_timed": 5,
                                     "residues_per_eval_at_e_qp": n_res,
                                     "sigma_eval_s_extrapolated": per_res * n_res,
                                     "qp_solve_s_extrapolated": per_res * n_res * (int(it.cpu()[0]) + 2),
                                     "note": "FP64 Pi(z) on the CUDA cores, FP64 complex LDL^T and W per residue; "
                                             "five residues timed, extrapolated to the QP solve"}
            line["cdwac_mixed_vs_plain_cd_fp64_qp_speedup_extrapolated"] = (
                line["plain_cd_fp64"]["qp_solve_s_extrapolated"] / (ms / 1e3))

        # diagonal spectral function over the paper's window (Sec. 5.5): 50 eV at 0.01 eV, 5000 points from 15 eV
        # below the core level (inside the near-real grid's reach), from the continued fractions; plain CD needs one
        # Pi(z) + LDL^T per residue at every point
        ev = 1.0 / 27.211386
        n_state = int(spec.states[0])
        win = torch.as_tensor(eps[n_state] - 15.0 * ev + np.arange(5000) * (0.01 * ev), dtype=torch.float64,
                              device=dev)
        ctx.spectral(sysd, prm, xi, wxi, W, pade, win, sync=True)
        t0.record(stream)
        for _ in range(5):
            ctx.spectral(sysd, prm, xi, wxi, W, pade, win, sync=False)
        t1.record(stream)
        torch.cuda.synchronize()
        t_spec = t0.elapsed_time(t1) / 5 / 1e3
        line["spectral_function"] = {"points": 5000, "window_eV": 50.0, "spacing_eV": 0.01, "cdwac_s": t_spec,
                                     "plain_cd_s_extrapolated": 5000 * t_cd,
                                     "cdwac_vs_plain_cd": 5000 * t_cd / t_spec,
                                     "note": "CD-WAC timed after set-up (W tables and fits built); plain CD = 5000 x "
                                             "the timed plain-CD Sigma evaluation, extrapolated"}

        # accuracy against the FP64 oracle (stored by tests/golden/make_acene_reference.py)
        gold = os.path.join(ROOT, "tests", "golden", "acene_1200_cdwac_oracle.json")
        if args.workload == "acene" and os.path.exists(gold):
            with open(gold) as f:
                ref = json.load(f)
            sig_ref = np.asarray(ref["sigma_re"]) + 1j * np.asarray(ref["sigma_im"])
            sig_gpu = sig.cpu().numpy()[0]
            Wn = W.cpu().numpy()[0]
            Wr = pade.W_real.cpu().numpy()[0]
            w_err = max(abs(Wn[k, m] - v) / max(abs(v), 1e-300) for k, m, v in ref["W_imag_samples"])
            wr_err = max(abs(Wr[j, m] - complex(a, b)) / abs(complex(a, b)) for j, m, a, b in ref["W_real_samples"])
            acc = {"oracle": "tests/golden/acene_1200_cdwac_oracle.json (FP64 CPU oracle, FP64 inputs)",
                   "W_imag_samples_max_rel_err": float(w_err), "W_real_samples_max_rel_err": float(wr_err),
                   "sigma_window_max_abs_err_meV": float(np.max(np.abs(sig_gpu - sig_ref))) / HA_PER_MEV,
                   "sigma_window_max_abs_meV": float(np.max(np.abs(sig_ref))) / HA_PER_MEV}
            st_gpu = int(qs.cpu()[0])
            if st_gpu == 0 and ref["qp"]["status"] == 0:
                acc["qp_vs_fp64_oracle_meV"] = (e_qp - ref["qp"]["e_qp"]) / HA_PER_MEV
                acc["qp_within_1_meV"] = bool(abs(e_qp - ref["qp"]["e_qp"]) < HA_PER_MEV)
            acc["note"] = ("the core QP energy (e_qp_Ha) is the accuracy target; Sigma over the window is reported "
                           "but not determined to 1 meV by any arithmetic at this size: the greedy M = 64 Thiele "
                           "continuation moves it by eV under 1e-13 relative changes of W with the node order fixed "
                           "(tests/golden/analyse_acene_dump.py on a bench.py --accuracy --dump file)")
            line["accuracy"] = acc

        # end to end through the C ABI with host buffers: copies of the inputs in, QP energy and Sigma out
        Bh = torch.from_numpy(B).pin_memory()
        Onh = torch.from_numpy(On).pin_memory()
        epsh = torch.from_numpy(eps).pin_memory()
        Bd, Ond, epsd = torch.empty_like(Bh, device=dev), torch.empty_like(Onh, device=dev), torch.empty_like(epsh, device=dev)
        sys_e2e = cdwac.System(epsd, Bd, Ond, spec.states, spec.n_occ, device=dev)
        e_host = torch.empty(len(spec.states), dtype=torch.float64).pin_memory()
        s_host = torch.empty(len(spec.states), len(omega), dtype=torch.complex128).pin_memory()

        def e2e_step():
            Bd.copy_(Bh, non_blocking=True)
            Ond.copy_(Onh, non_blocking=True)
            epsd.copy_(epsh, non_blocking=True)
            o = step(sys_e2e)
            e_host.copy_(o[4], non_blocking=True)
            s_host.copy_(o[3], non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        t1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = t0.elapsed_time(t1) / args.steps
        line["e2e"] = {"value": n_eval / (ms_e2e / 1e3), "unit": UNIT,
                       "h2d_bytes_per_step": int(Bh.numel() * Bh.element_size() + Onh.numel() * Onh.element_size()
                                                 + epsh.numel() * 8),
                       "d2h_bytes_per_step": int(e_host.numel() * 8 + s_host.numel() * 16), "ms_per_step": ms_e2e}

        # CPU oracle on this host's cores (bounded sample)
        B64 = B.astype(np.float64)
        On64 = On.astype(np.float64)
        t_step, t_meas = oracle_sample(spec, B64, On64, eps)
        line["cpu_baseline"] = {"value": n_eval / t_step, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"W_nm(i xi) at 1 of 100 imaginary frequencies ({t_meas:.1f} s, numpy FP64), "
                                          "scaled by 100 + 4*40 points per step"}
    ctx.sync_status(allow)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_batch(args, rank, ws, dist):
    """Uneven batch: 16 systems (N_basis uniform in [200, 1500] from seeds 2..17, N_aux = 3.3 N_basis,
    n_occ = N_basis/10, 4 core states each) in one graph-captured cdwac_batch_run; a step replays the graph."""
    import torch

    import __graft_entry__ as g
    from paper_2305_15955_gb300 import cdwac, inputs

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    g.build()
    specs = inputs.batched_systems(args.batch_systems)
    t0 = time.time()
    systems = []
    for sp in specs:
        eps = inputs.eigenvalues(sp)
        systems.append(cdwac.System(eps, inputs.build_B(sp, dtype=np.float32), inputs.build_On(sp, dtype=np.float32),
                                    sp.states, sp.n_occ, device=dev))
    t_gen = time.time() - t0
    prm = cdwac.Params(n_imag=args.n_imag, n_real=args.n_real, pade_M=min(64, args.n_imag + args.n_real),
                       precision=cdwac.PREC_MIXED)
    omega = inputs.omega_grid(128)
    ctx = cdwac.Context(local)
    res = [cdwac.BatchResult(s, prm, omega, omega, dev) for s in systems]
    lanes = 4
    l0 = ctx.launch_count()
    chosen, items = cdwac.batch_run(ctx, res, prm, max_lanes=lanes, graph=True,   # eager run + capture
                                    max_iter=args.qp_max_iter)
    ln, la, pg, pt, uw = chosen
    graph_kernels = (ctx.launch_count() - l0) // 2   # the eager run and the capture enqueue the same kernels
    for _ in range(max(0, args.warmup - 1)):
        cdwac.batch_run(ctx, res, prm, max_lanes=lanes, graph=True, items=items, sync=False,
                        max_iter=args.qp_max_iter)
    torch.cuda.synchronize()
    barrier(dist)
    stream = torch.cuda.current_stream()
    launches0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            cdwac.batch_run(ctx, res, prm, max_lanes=lanes, graph=True, items=items, sync=False,
                            max_iter=args.qp_max_iter)
        e1.record(stream)
        torch.cuda.synchronize()
    ctx.sync_status((cdwac.ERR_PADE_BREAKDOWN, cdwac.ERR_QP_NOT_CONVERGED))
    ms = max_over_ranks(dist, e0.elapsed_time(e1) / args.steps, dev)
    n_states = sum(len(sp.states) for sp in specs)
    peaks, _ = measured_peaks()
    pi_flops = sum(prm.n_imag * sp.n_aux * (sp.n_aux + 1) / 2 * sp.n_ov * 2 + prm.n_real * sp.n_aux * (sp.n_aux + 1) *
                   sp.n_ov * 2 for sp in specs)
    line = {"metric": METRIC, "value": ws * n_states * len(omega) / (ms / 1e3), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3-f32acc+f64", "data": "synthetic",
            "config": {"workload": f"uneven batch: {len(specs)} systems, N_basis " +
                                   ",".join(str(sp.n_basis) for sp in specs) +
                                   ", N_aux = 3.3 N_basis, 4 core states each, one CUDA graph per step",
                       "lanes": ln, "lookahead": la, "pi_tile_group": pg, "pi_tile_width": pt,
                       "update_waves": uw,
                       "n_states_total": n_states, "qp_max_iter": args.qp_max_iter,
                       "input_generation_s": t_gen},
            "pi_tflop_per_step": pi_flops / 1e12,
            "gpu_launches": int(graph_kernels), "gpu_launches_note": "kernel nodes of the CUDA graph replayed per step",
            "qp_status_counts": np.bincount(np.concatenate([r.qp_status.cpu().numpy() for r in res]), minlength=3).tolist(),
            "qp_by_system": qp_report(specs, res, omega, prm),
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def qp_report(specs, res, omega, prm):
    """Where each batch state's QP equation ended, against the 128-point window (the bisection fallback's bracket)
    and the reach of the near-real grid (|eps_F - eps_n| + real_margin): status 0 fixed point, 1 bisection, 2 none
    (the last fixed-point iterate is reported).  The residues of a state evaluated at omega run up to
    eps_HOMO - omega; beyond the grid's reach the continuation extrapolates."""
    from paper_2305_15955_gb300 import inputs
    out = []
    for sp, r in zip(specs, res):
        eps = inputs.eigenvalues(sp)
        ef = inputs.fermi_level(eps, sp.n_occ)
        e, st, Z = r.e_qp.cpu().numpy(), r.qp_status.cpu().numpy(), r.Z.cpu().numpy()
        reach = max(abs(ef - eps[n]) for n in sp.states) + prm.real_margin
        out.append({"system": sp.name, "states": [int(n) for n in sp.states], "status": st.tolist(),
                    "e_qp_Ha": [round(float(x), 6) for x in e], "Z": [round(float(x), 4) for x in Z],
                    "in_window": [bool(omega[0] <= x <= omega[-1]) for x in e],
                    "largest_residue_Ha": [round(float(eps[sp.n_occ - 1] - x), 3) for x in e],
                    "near_real_reach_Ha": round(float(reach), 3)})
    return out


def run_refined_map(args, rank, ws, dist):
    """QP error of CD-WAC(N_core, N_val, N_Im) against plain CD, both FP64 on the same GPU: the synthetic analogue
    of the reference-set calibration of Sec. 5.1 (an MAE over a set of core levels).  Eight seeded systems of the
    small recipe (N_basis 40: one core level at -10.6 Ha, 4 valence levels in [-1.1, -0.3], 35 virtuals log-spaced
    in [0.02, 2.0]; N_aux 120; core entries x0.3; seeds 0-7), whose core QP equations have their root inside the
    128-point window [-11, -10] Ha; 100 imaginary points; Pade order M = N_core + N_val + N_Im as in the paper;
    neighbourhood radii from --delta-c / --delta-v.  Also the generic set at the same point counts, and evGW0 / evGW
    cycles of CD-WAC against plain-CD cycles.  Larger systems of the acene-like recipe carry correlation
    self-energies of tens of Ha, whose QP roots leave the window."""
    import torch

    import __graft_entry__ as g
    from paper_2305_15955_gb300 import cdwac, inputs

    if rank != 0:
        return
    torch.cuda.set_device(0)
    g.build()
    ctx = cdwac.Context(0)
    omega = inputs.omega_grid(128)
    ni = args.n_imag
    base = cdwac.Params(n_imag=ni, n_real=0, pade_M=min(cdwac.MAX_M, ni))
    systems = []
    t0 = time.perf_counter()
    for seed in range(8):
        spec = inputs.custom_system(40, 5, 120, seed=seed, n_core=1, states=(0,), core_scale=0.3,
                                    valence=(-1.1, -0.3), virtual=(0.02, 2.0))
        sysd = cdwac.System(inputs.eigenvalues(spec), inputs.build_B(spec), inputs.build_On(spec), spec.states,
                            spec.n_occ)
        xi, wxi, W = ctx.build_W_imag(sysd, base)
        e, _, _, qs = ctx.qp_solve(sysd, base, xi, wxi, W, None, omega)
        systems.append((sysd, xi, wxi, W, float(e.cpu()[0]), int(qs.cpu()[0])))
    t_cd = time.perf_counter() - t0

    def errors(p):
        """|e_QP(CD-WAC) - e_QP(CD)| in meV per system (None where either QP did not converge)."""
        out = []
        for sysd, xi, wxi, W, e_cd, s_cd in systems:
            pade = ctx.fit_pade(sysd, p, xi, W)
            e, _, _, qs = ctx.qp_solve(sysd, p, xi, wxi, W, pade, omega)
            ok = s_cd == 0 and int(qs.cpu()[0]) == 0
            out.append(abs(float(e.cpu()[0]) - e_cd) / HA_PER_MEV if ok else None)
        return out

    def stats(errs):
        v = [x for x in errs if x is not None]
        return (sum(v) / len(v) if v else None), (max(v) if v else None), len(errs) - len(v)

    sizes = (0, 2, 5, 10, 20, 40)
    mae, mx, bad = ([[None] * len(sizes) for _ in sizes] for _ in range(3))
    for i, nc in enumerate(sizes):
        for j, nv in enumerate(sizes):
            p = (cdwac.Params.refined(nc, nv, args.delta_c, args.delta_v, n_imag=ni,
                                      pade_M=min(cdwac.MAX_M, ni + nc + nv)) if nc + nv else base)
            mae[i][j], mx[i][j], bad[i][j] = stats(errors(p))
    generic = {}
    for nr in (10, 20, 40, 80):
        m, x, b = stats(errors(cdwac.Params(n_imag=ni, n_real=nr, pade_M=min(cdwac.MAX_M, ni + nr))))
        generic[str(nr)] = {"mae_meV": m, "max_meV": x, "not_converged": b}
    # evGW0 / evGW (Sec. 5.4): CD-WAC cycles against plain-CD cycles on the same systems
    evgw = {}
    for mode_name, mode in (("evGW0", cdwac.EVGW0), ("evGW", cdwac.EVGW)):
        ref = []
        for sysd, *_ in systems:
            e, _, _, _, st = ctx.evgw(sysd, base, mode, omega, plain_cd=True)
            ref.append(float(e.cpu()[0]) if st == cdwac.OK else None)
        for name, p in (("generic 20", cdwac.Params(n_imag=ni, n_real=20, pade_M=min(cdwac.MAX_M, ni + 20))),
                        ("refined (10, 10), delta_c 0.5, delta_v 0.25 (fixed radii, not --delta-c/--delta-v)",
                         cdwac.Params.refined(10, 10, 0.5, 0.25, n_imag=ni, pade_M=min(cdwac.MAX_M, ni + 20)))):
            errs = []
            for (sysd, *_), r in zip(systems, ref):
                e, _, _, _, st = ctx.evgw(sysd, p, mode, omega)
                errs.append(abs(float(e.cpu()[0]) - r) / HA_PER_MEV if st == cdwac.OK and r is not None else None)
            m, x, b = stats(errs)
            evgw[f"{mode_name}, {name}"] = {"mae_meV": m, "max_meV": x, "not_converged": b}
    line = {"metric": "core QP error of CD-WAC(N_core, N_val, N_Im) against plain CD (MAE over 8 systems)",
            "unit": "meV", "dtype": "f64", "data": "synthetic",
            "config": {"workload": "8 small systems: N_basis=40 (1 core at -10.6 Ha, 4 valence in [-1.1,-0.3], 35 "
                                   "virtual log-spaced in [0.02,2.0]), N_aux=120, core entries x0.3, seeds 0-7; "
                                   "core state n=0; 128 omega in [-11,-10] Ha", "n_imag": ni,
                       "delta_c_Ha": args.delta_c, "delta_v_Ha": args.delta_v, "pade_M": "N_core + N_val + N_Im"},
            "sizes": list(sizes), "rows": "N_core", "cols": "N_val", "mae_meV": mae, "max_meV": mx,
            "not_converged": bad, "generic": generic, "evgw_vs_plain_cd": evgw, "plain_cd_qp_s": t_cd,
            "plain_cd_qp_status": [s[5] for s in systems]}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_accuracy(args, rank, ws, dist):
    """One untimed step of the workload in the chosen precision and its accuracy against the stored oracle result
    (tests/golden/acene_1200_cdwac_oracle.json and, when present, the full tables in the matching .npz written by
    tests/golden/make_acene_reference.py): W(i xi) and W(z) at every stored entry, the greedy node orders, Sigma
    over the 128-point window and the QP energy.  --dump writes the GPU's tables for
    tests/golden/analyse_acene_dump.py."""
    import torch

    import __graft_entry__ as g
    from paper_2305_15955_gb300 import cdwac, inputs

    if rank != 0:
        return
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    g.build()
    spec, desc = workload(args.workload)
    mixed = args.precision == "mixed"
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec, dtype=np.float32 if mixed else np.float64)
    On = inputs.build_On(spec, dtype=np.float32 if mixed else np.float64)
    omega = inputs.omega_grid(128)
    sysd = cdwac.System(eps, B, On, spec.states, spec.n_occ, device=dev)
    prm = cdwac.Params(n_imag=args.n_imag, n_real=args.n_real, pade_M=min(64, args.n_imag + args.n_real),
                       precision=cdwac.PREC_MIXED if mixed else cdwac.PREC_FP64)
    ctx = cdwac.Context(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xi, wxi, W = ctx.build_W_imag(sysd, prm)
    pade = ctx.fit_pade(sysd, prm, xi, W)
    sig = ctx.sigma(sysd, prm, xi, wxi, W, pade, torch.as_tensor(omega, device=dev))
    e, Z, it, qs = ctx.qp_solve(sysd, prm, xi, wxi, W, pade, torch.as_tensor(omega, device=dev))
    torch.cuda.synchronize()
    t_step = time.perf_counter() - t0
    tab = {"xi": xi.cpu().numpy(), "wxi": wxi.cpu().numpy(), "W_imag": W.cpu().numpy()[0],
           "z_real": pade.z_real.cpu().numpy()[0], "W_real": pade.W_real.cpu().numpy()[0],
           "nodes": pade.nodes.cpu().numpy()[0], "n_used": pade.n_used.cpu().numpy()[0],
           "sigma": sig.cpu().numpy()[0], "e_qp": float(e.cpu()[0]), "qp_status": int(qs.cpu()[0])}
    ctx.close()
    if args.dump:
        np.savez(args.dump, **{k: np.asarray(v) for k, v in tab.items()})
    line = {"mode": "accuracy", "workload": desc, "precision": args.precision, "step_s_untimed": t_step,
            "qp": {"e_qp_Ha": tab["e_qp"], "status": tab["qp_status"]}}
    gold = os.path.join(ROOT, "tests", "golden", "acene_1200_cdwac_oracle.json")
    if args.workload == "acene" and os.path.exists(gold):
        with open(gold) as f:
            ref = json.load(f)
        Wn, Wr = tab["W_imag"], tab["W_real"]
        rel_i = [abs(Wn[k, m] - v) / abs(v) for k, m, v in ref["W_imag_samples"]]
        rel_r = [abs(Wr[j, m] - complex(vr, vi)) / abs(complex(vr, vi)) for j, m, vr, vi in ref["W_real_samples"]]
        sig_ref = np.asarray(ref["sigma_re"]) + 1j * np.asarray(ref["sigma_im"])
        line["vs_stored_oracle"] = {
            "W_imag_samples_max_rel_err": float(max(rel_i)), "W_real_samples_max_rel_err": float(max(rel_r)),
            "W_real_samples_rel_err_by_point": {str(j): float(max(abs(Wr[jj, m] - complex(vr, vi)) / abs(complex(vr, vi))
                                                                  for jj, m, vr, vi in ref["W_real_samples"] if jj == j))
                                                for j in sorted({int(x[0]) for x in ref["W_real_samples"]})},
            "sigma_max_abs_err_meV": float(np.max(np.abs(tab["sigma"] - sig_ref))) / HA_PER_MEV,
            "sigma_max_abs_meV": float(np.max(np.abs(sig_ref))) / HA_PER_MEV,
            "qp_oracle_Ha": ref["qp"]["e_qp"]}
        line["vs_stored_oracle"]["qp_vs_oracle_meV"] = (tab["e_qp"] - ref["qp"]["e_qp"]) / HA_PER_MEV
        full = gold.replace(".json", ".npz")
        if os.path.exists(full):
            line["vs_stored_oracle"].update(_full_table_comparison(full, tab))
    print(json.dumps(line), flush=True)


def _full_table_comparison(path, tab):
    """Every stored oracle table entry against the GPU's (numpy on stored values; the continuation's own
    conditioning is analysed by tests/golden/analyse_acene_dump.py, which runs the oracle on a --dump file)."""
    ref = np.load(path)
    rel = lambda a, b: np.abs(a - b) / np.maximum(np.abs(b).max(axis=-1, keepdims=True), 1e-300)
    out = {"W_imag_max_rel_err_by_k": rel(tab["W_imag"], ref["W_imag"]).max(axis=1).tolist(),
           "W_real_max_rel_err_by_point": rel(tab["W_real"], ref["W_real"]).max(axis=1).tolist()}
    n_occ = tab["nodes"].shape[0]
    out["node_orders_identical_fraction"] = float(np.mean([np.array_equal(tab["nodes"][m, :tab["n_used"][m]],
                                                                          ref["nodes"][m, :ref["n_used"][m]])
                                                           for m in range(n_occ)]))
    return out


def run_acarbon(args, rank, ws, dist):
    """The amorphous-carbon-like system (N_basis 3500: 116 core levels at -10.6 +- 0.02 Ha, 184 valence in
    [-1.2, -0.25], 3200 virtuals log-spaced in [0.005, 8]; N_aux 10 000; O^{ia} in FP32, 38.4 GB; seed 3; 8 core
    states), mixed precision.  A whole step (100 imaginary + 40 near-real points) takes minutes, so it is timed on a
    sample and extrapolated, and labelled so: two imaginary frequencies (one W build over a 2-point grid) and two
    near-real points (one near-real build), scaled to 100 + 40; the Thiele fits, Sigma on the 128-point window and
    the QP equations of the 8 states on W tables of the full shape (values of the sampled build repeated); plain
    CD (mixed) timed on two residues."""
    import torch

    import __graft_entry__ as g
    from paper_2305_15955_gb300 import cdwac, inputs

    if rank != 0:
        return
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    g.build()
    spec = inputs.amorphous_carbon_system()
    t0 = time.time()
    eps = inputs.eigenvalues(spec)
    B = inputs.build_B(spec, dtype=np.float32)
    On = inputs.build_On(spec, dtype=np.float32)
    t_gen = time.time() - t0
    sysd = cdwac.System(eps, torch.from_numpy(B).to(dev), torch.from_numpy(On).to(dev), spec.states, spec.n_occ,
                        device=dev)
    del B
    omega = torch.as_tensor(inputs.omega_grid(128), device=dev)
    prm = cdwac.Params(n_imag=100, n_real=40, pade_M=64, precision=cdwac.PREC_MIXED)

    def timed(fn, reps=1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            r = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / reps, r

    # plain CD (mixed) on the same GPU, first and in a context of its own (its operand planes, ~115 GB, are freed
    # before the W builds): one Sigma evaluation with exactly two residues, after a warm-up evaluation
    ctx = cdwac.Context(0)
    one = cdwac.System(eps, sysd.O_ia, sysd.O_n[:1], (0,), spec.n_occ, device=dev)
    p1 = cdwac.Params(n_imag=1, n_real=0, precision=cdwac.PREC_MIXED)
    xi1, wxi1, W1 = ctx.build_W_imag(one, p1)
    w2 = torch.tensor([0.5 * (eps[spec.n_occ - 3] + eps[spec.n_occ - 2])], dtype=torch.float64, device=dev)
    timed(lambda: ctx.sigma(one, p1, xi1, wxi1, W1, None, w2))
    t_cd, _ = timed(lambda: ctx.sigma(one, p1, xi1, wxi1, W1, None, w2))
    per_res = t_cd / 2.0
    n_res = spec.n_occ                       # a core-state Sigma near -10.6 Ha has every occupied level above it
    ctx.close()
    del one
    torch.cuda.empty_cache()
    ctx = cdwac.Context(0)

    p2 = cdwac.Params(n_imag=2, n_real=2, pade_M=4, precision=cdwac.PREC_MIXED)
    timed(lambda: ctx.build_W_imag(sysd, p2))                        # warm-up: scratch, lanes, tensor maps
    t_imag, (xi2, wxi2, W2) = timed(lambda: ctx.build_W_imag(sysd, p2))
    timed(lambda: ctx.fit_pade(sysd, p2, xi2, W2))
    t_real, _ = timed(lambda: ctx.fit_pade(sysd, p2, xi2, W2))
    # full-shape tables for the fit, Sigma and QP timings (the sampled values repeated over the grid)
    xi, wxi, _ = ctx.build_W_imag(cdwac.System(eps[:4], torch.zeros(1, 3, device=dev, dtype=torch.float32),
                                               torch.zeros(1, 1, 4, device=dev, dtype=torch.float32), [0], 1,
                                               device=dev), cdwac.Params(n_imag=100, n_real=0))
    W = W2[:, :1, :].repeat(1, 100, 1).contiguous()
    pade = ctx.alloc_pade(sysd, prm)
    t_rest, _ = timed(lambda: (ctx.fit_pade(sysd, cdwac.Params(n_imag=100, n_real=0, pade_M=64,
                                                                precision=cdwac.PREC_MIXED), xi, W, pade),
                               ctx.sigma(sysd, prm, xi, wxi, W, pade, omega),
                               ctx.qp_solve(sysd, prm, xi, wxi, W, pade, omega)))
    step_s = t_imag * 50 + t_real * 20 + t_rest
    n_eval = len(spec.states) * 128
    line = {"metric": METRIC, "value": n_eval / step_s, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3-f32acc+f64", "data": "synthetic", "extrapolated": True,
            "config": {"workload": "a-C-like: N_basis=3500 (116 core at -10.6+-0.02 Ha, 184 valence in [-1.2,-0.25], "
                                   "3200 virtual log-spaced in [0.005,8]), N_aux=10000, O^ia FP32 (38.4 GB), seed 3, "
                                   "8 core states; 100 imaginary GL points, 40 near-real points, M=64, 128 omega in "
                                   "[-11,-10] Ha",
                       "sample": "2 imaginary frequencies and 2 near-real points timed, scaled to 100 + 40; fits, "
                                 "Sigma and QP timed on full-shape tables",
                       "input_generation_s": t_gen},
            "imag_2_freq_s": t_imag, "near_real_2_points_s": t_real, "fits_sigma_qp_s": t_rest,
            "plain_cd_mixed": {"per_residue_s": per_res, "residues_timed": 2,
                               "sigma_eval_s_extrapolated": per_res * n_res,
                               "note": "Pi(z) on the tensor cores and a complex LDL^T per residue; a core-state "
                                       "Sigma evaluation has n_occ = 300 residues"},
            "gpu_launches": None}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    rank, ws, dist = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws, dist)
    elif args.refined_map:
        run_refined_map(args, rank, ws, dist)
    elif args.accuracy:
        run_accuracy(args, rank, ws, dist)
    elif args.workload == "batch":
        run_batch(args, rank, ws, dist)
    elif args.workload == "acarbon":
        run_acarbon(args, rank, ws, dist)
    else:
        run_ours(args, rank, ws, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
