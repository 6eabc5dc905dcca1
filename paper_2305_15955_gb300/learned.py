"""Learned continuation of W (pole-residue MLP): data from the method itself, training and evaluation on the GPU.

The arithmetic runs in libcdwac's kernels (cdwac_mlp_features, cdwac_mlp_loss_grad, cdwac_mlp_adam,
cdwac_mlp_poles, cdwac_qp_solve_poles); this module only sequences the calls.

Data: for each training system, W_nm(i xi) on the imaginary grid (cdwac_build_W_imag) and W_nm at the generic
near-real points (cdwac_fit_pade) for every pair of occupied n, m.  The network sees the 32 imaginary samples and
is trained to reproduce W at the imaginary nodes and the near-real points.  At inference it needs only the
imaginary axis, so it replaces the near-real W builds (half of the CD-WAC cost) for the residue term.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import cdwac, inputs


def training_systems(seeds, nb_range=(30, 60)):
    """Small core-level systems (the 40-orbital family: one core level at -10.6 Ha, 4 valence levels, core rows
    x0.3, N_aux = 3 N_basis) with N_basis drawn per seed; every occupied orbital is a requested state."""
    out = []
    for sd in seeds:
        nb = nb_range[0] + int(inputs.counter_uniform(sd, 7) * (nb_range[1] - nb_range[0] + 1) - 1e-12)
        out.append(inputs.custom_system(nb, 5, 3 * nb, seed=sd, n_core=1, states=tuple(range(5)), core_scale=0.3,
                                        valence=(-1.1, -0.3), virtual=(0.02, 2.0)))
    return out


def _device_system(spec, states=None):
    eps = inputs.eigenvalues(spec)
    st = spec.states if states is None else states
    return cdwac.System(eps, inputs.build_B(spec), inputs.build_On(spec, states=st), st, spec.n_occ), eps


@dataclasses.dataclass
class Dataset:
    x: torch.Tensor
    scale: torch.Tensor
    z_ref: torch.Tensor
    w_ref: torch.Tensor


def generate(ctx: cdwac.Context, specs, params: cdwac.Params) -> Dataset:
    parts = []
    for sp in specs:
        sysd, _ = _device_system(sp)
        xi, wxi, W = ctx.build_W_imag(sysd, params)
        pade = ctx.fit_pade(sysd, params, xi, W)
        parts.append(ctx.mlp_features(xi, W, sp.n_occ, pade, params.n_real))
    return Dataset(*[torch.cat([p[i] for p in parts]) for i in range(4)])


def init_params(dev, seed=0):
    """Same deterministic initialisation as the CPU reference of the network."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in [(32, 256), (256, 256), (256, 256), (256, 16)]:
        lim = np.sqrt(6.0 / i) * (0.25 if o == 16 else 1.0)
        parts.append(rng.uniform(-lim, lim, size=i * o))
        parts.append(np.zeros(o))
    return torch.as_tensor(np.concatenate(parts), dtype=torch.float32, device=dev)


def train(ctx: cdwac.Context, data: Dataset, steps=2000, batch=512, lr=1e-3, seed=0, log_every=0, lr_final=None):
    """Adam on random minibatches; the learning rate decays along a cosine from lr to lr_final (default lr/100)."""
    dev = data.x.device
    params = init_params(dev, seed)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    n = data.x.shape[0]
    history = []
    for step in range(1, steps + 1):
        idx = torch.randint(0, n, (min(batch, n),), generator=gen).to(dev)
        ctx.mlp_loss_grad(params, data.x[idx].contiguous(), data.scale[idx].contiguous(),
                          data.z_ref[idx].contiguous(), data.w_ref[idx].contiguous(), grad, loss)
        lf = lr / 100.0 if lr_final is None else lr_final
        lr_t = lf + 0.5 * (lr - lf) * (1.0 + np.cos(np.pi * (step - 1) / max(1, steps - 1)))
        ctx.mlp_adam(params, grad, m, v, step, lr=lr_t)
        if log_every and (step % log_every == 0 or step == 1):
            history.append((step, float(loss.item())))
    return params, history


def mean_loss(ctx: cdwac.Context, params, data: Dataset, batch=4096):
    tot, n = 0.0, data.x.shape[0]
    for i in range(0, n, batch):
        sl = slice(i, min(n, i + batch))
        _, l = ctx.mlp_loss_grad(params, data.x[sl].contiguous(), data.scale[sl].contiguous(),
                                 data.z_ref[sl].contiguous(), data.w_ref[sl].contiguous())
        tot += float(l.item()) * (sl.stop - sl.start)
    return tot / n


def evaluate(ctx: cdwac.Context, params, specs, prm_wac: cdwac.Params, omega_grid):
    """Core-state (n = 0) QP energies by plain CD (direct W at every residue: the reference), CD-WAC with near-real
    points, CD-WAC on the imaginary axis only, and the learned continuation (imaginary axis only).
    Returns per-system errors in meV against plain CD and the statuses."""
    rows = []
    p_imag = dataclasses.replace(prm_wac, n_real=0)
    for sp in specs:
        sysd, eps = _device_system(sp, states=(0,))
        xi, wxi, W = ctx.build_W_imag(sysd, prm_wac)
        e_cd, _, _, s_cd = ctx.qp_solve(sysd, prm_wac, xi, wxi, W, None, omega_grid)
        pade = ctx.fit_pade(sysd, prm_wac, xi, W)
        e_wac, _, _, s_wac = ctx.qp_solve(sysd, prm_wac, xi, wxi, W, pade, omega_grid)
        pade_i = ctx.fit_pade(sysd, p_imag, xi, W)
        e_im, _, _, s_im = ctx.qp_solve(sysd, p_imag, xi, wxi, W, pade_i, omega_grid)
        x, scale, _, _ = ctx.mlp_features(xi, W, sp.n_occ)
        poles = ctx.mlp_poles(params, x, scale)
        e_ml, _, _, s_ml = ctx.qp_solve_poles(sysd, prm_wac, xi, wxi, W, poles, omega_grid)
        ref = float(e_cd.cpu()[0])
        mev = 27211.386
        rows.append({"n_basis": sp.n_basis, "seed": sp.seed, "status_cd": int(s_cd.cpu()[0]),
                     "wac_near_real_meV": (float(e_wac.cpu()[0]) - ref) * mev,
                     "wac_imag_only_meV": (float(e_im.cpu()[0]) - ref) * mev,
                     "mlp_imag_only_meV": (float(e_ml.cpu()[0]) - ref) * mev,
                     "status": [int(s_wac.cpu()[0]), int(s_im.cpu()[0]), int(s_ml.cpu()[0])]})
    return rows
