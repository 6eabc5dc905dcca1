"""Seeded synthetic inputs for CD-WAC: Kohn-Sham-like eigenvalues and RI-V three-centre tensors.

This module holds none of the method's arithmetic.  It only draws the mean-field input of a G0W0 run
(the eigenvalues eps_m and the RI-V tensors O^{nm}_P of Eq. 3c_OnmP in Sec. 2.2) for synthetic systems whose
shapes follow the paper's acene and amorphous-carbon workloads (Sec. 5.5).  Both the CUDA path and the CPU
oracle consume the buffers built here.

Random numbers are counter based, so any block of the symmetric tensor O^{pq}_P can be drawn without
materialising the rest: entry (P, p, q) with p <= q is the standard normal built by Box-Muller from two
splitmix64 outputs (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
keyed on (seed, P, p, q), divided by sqrt(N_aux).  O^{pq}_P = O^{qp}_P holds by construction, and the
occupied-virtual block B[P, i*n_virt + a] = O^{i,a}_P is the same number as the (n=i, m=a) entry of the
state rows, so the polarizability and the projection see one consistent tensor.
"""
from __future__ import annotations

import concurrent.futures as _cf
import dataclasses
import math
import os

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser of (x + golden gamma), on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _uniform01(h: np.ndarray) -> np.ndarray:
    """Top 53 bits of a uint64 hash mapped to (0, 1]."""
    return ((h >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def counter_normals(seed: int, keys: np.ndarray) -> np.ndarray:
    """Standard normals, one per uint64 counter in ``keys`` (Box-Muller on two splitmix64 draws)."""
    with np.errstate(over="ignore"):
        base = _splitmix64(np.uint64(seed) * _GOLDEN + np.uint64(0x5DEECE66D))
        k2 = keys.astype(np.uint64) * np.uint64(2) + base
        u1 = _uniform01(_splitmix64(k2))
        u2 = _uniform01(_splitmix64(k2 + np.uint64(1)))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def counter_uniform(seed: int, key: int) -> float:
    """One uniform draw in (0, 1] for scalar choices (e.g. the size of a batched system)."""
    with np.errstate(over="ignore"):
        h = _splitmix64(np.array([np.uint64(seed) * _GOLDEN + np.uint64(key) + np.uint64(0xA5A5)], dtype=np.uint64))
    return float(_uniform01(h)[0])


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    """A synthetic closed-shell system.

    Orbitals are ordered by ascending energy: ``n_core`` core levels, then valence levels (together ``n_occ``
    occupied), then ``n_basis - n_occ`` virtual levels.  ``states`` are the orbital indices whose G0W0
    quasiparticle energies are wanted (the core levels n of the paper).  ``core_scale`` multiplies every
    entry O^{pq}_P with p or q a core orbital (once, so O^{cc}_P also gets a single factor).
    """

    n_basis: int
    n_occ: int
    n_aux: int
    seed: int
    n_core: int
    core_center: float
    core_halfwidth: float
    valence: tuple
    virtual: tuple
    states: tuple
    core_scale: float = 1.0
    name: str = ""

    @property
    def n_virt(self) -> int:
        return self.n_basis - self.n_occ

    @property
    def n_ov(self) -> int:
        return self.n_occ * self.n_virt


def eigenvalues(spec: SystemSpec) -> np.ndarray:
    """Ascending eigenvalues (Ha): core linspace, valence linspace, virtuals geometric (log) spacing."""
    if spec.n_core == 1:
        core = np.array([spec.core_center])
    else:
        core = np.linspace(spec.core_center - spec.core_halfwidth, spec.core_center + spec.core_halfwidth, spec.n_core)
    n_val = spec.n_occ - spec.n_core
    val = np.linspace(spec.valence[0], spec.valence[1], n_val) if n_val > 1 else np.array([spec.valence[1]])[:n_val]
    virt = np.geomspace(spec.virtual[0], spec.virtual[1], spec.n_virt)
    eps = np.concatenate([core, val, virt]).astype(np.float64)
    if np.any(np.diff(eps) < 0):
        raise ValueError("eigenvalue ranges overlap; eps must be ascending")
    return eps


def _o_entries(spec: SystemSpec, P: np.ndarray, p: np.ndarray, q: np.ndarray) -> np.ndarray:
    """O^{pq}_P for broadcastable index arrays (symmetric in p, q)."""
    lo = np.minimum(p, q).astype(np.uint64)
    hi = np.maximum(p, q).astype(np.uint64)
    nb = np.uint64(spec.n_basis)
    with np.errstate(over="ignore"):
        keys = (P.astype(np.uint64) * nb + lo) * nb + hi
    vals = counter_normals(spec.seed, keys) / math.sqrt(spec.n_aux)
    if spec.core_scale != 1.0 and spec.n_core > 0:
        core = (lo < np.uint64(spec.n_core))
        vals = np.where(core, vals * spec.core_scale, vals)
    return vals


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def build_B(spec: SystemSpec, dtype=np.float64, out: np.ndarray | None = None) -> np.ndarray:
    """Occupied-virtual block B[P, i*n_virt + a] = O^{i, n_occ + a}_P, shape [n_aux, n_occ*n_virt]."""
    n_occ, n_virt = spec.n_occ, spec.n_virt
    if out is None:
        out = np.empty((spec.n_aux, n_occ * n_virt), dtype=dtype)
    i_idx = np.repeat(np.arange(n_occ, dtype=np.uint64), n_virt)
    a_idx = np.tile(np.arange(n_occ, n_occ + n_virt, dtype=np.uint64), n_occ)

    def rows(r0, r1):
        for P in range(r0, r1):
            out[P, :] = _o_entries(spec, np.full(1, P, dtype=np.uint64), i_idx, a_idx)

    nt = _threads()
    step = max(1, (spec.n_aux + nt - 1) // nt)
    with _cf.ThreadPoolExecutor(nt) as ex:
        list(ex.map(lambda r: rows(r, min(spec.n_aux, r + step)), range(0, spec.n_aux, step)))
    return out


def build_On(spec: SystemSpec, states=None, dtype=np.float64) -> np.ndarray:
    """State rows O_n[s, P, m] = O^{n_s, m}_P for every orbital m, shape [n_states, n_aux, n_basis]."""
    states = spec.states if states is None else tuple(states)
    out = np.empty((len(states), spec.n_aux, spec.n_basis), dtype=dtype)
    m = np.arange(spec.n_basis, dtype=np.uint64)
    for s, n in enumerate(states):
        P = np.arange(spec.n_aux, dtype=np.uint64)[:, None]
        out[s] = _o_entries(spec, P, np.full_like(m, n)[None, :], m[None, :])
    return out


def fermi_level(eps: np.ndarray, n_occ: int) -> float:
    """Midpoint of the HOMO-LUMO gap (occupations are fixed by index, not by this value)."""
    return 0.5 * (float(eps[n_occ - 1]) + float(eps[n_occ]))


# --- the workloads -------------------------------------------------------------------------------------

def small_system() -> SystemSpec:
    """40 orbitals (1 core at -10.6 Ha, 4 valence in [-1.1, -0.3], 35 virtuals log-spaced in [0.02, 2.0]),
    N_aux = 120, seed 0, core entries x0.3: small enough for the brute-force pole sum."""
    return SystemSpec(n_basis=40, n_occ=5, n_aux=120, seed=0, n_core=1, core_center=-10.6, core_halfwidth=0.0,
                      valence=(-1.1, -0.3), virtual=(0.02, 2.0), states=(0,), core_scale=0.3, name="small-40")


def acene_system(n_states: int = 1) -> SystemSpec:
    """Acene-like: 1200 orbitals (6 core at -10.6 +- 0.01 Ha, 114 valence in [-1.2, -0.25], 1080 virtuals
    log-spaced in [0.01, 5]), N_aux = 4000, seed 1."""
    return SystemSpec(n_basis=1200, n_occ=120, n_aux=4000, seed=1, n_core=6, core_center=-10.6, core_halfwidth=0.01,
                      valence=(-1.2, -0.25), virtual=(0.01, 5.0), states=tuple(range(n_states)), name="acene-1200")


def amorphous_carbon_system() -> SystemSpec:
    """a-C46H70-like: 3500 orbitals (116 core at -10.6 +- 0.02 Ha, 184 valence in [-1.2, -0.25], 3200 virtuals
    log-spaced in [0.005, 8]), N_aux = 10000, seed 3, 8 core states."""
    return SystemSpec(n_basis=3500, n_occ=300, n_aux=10000, seed=3, n_core=116, core_center=-10.6,
                      core_halfwidth=0.02, valence=(-1.2, -0.25), virtual=(0.005, 8.0), states=tuple(range(8)),
                      name="a-C-3500")


def batched_systems(n_systems: int = 16, first_seed: int = 2, nb_range=(200, 1500)) -> list:
    """Uneven batch: N_basis drawn uniformly in nb_range per seed, N_aux = round(3.3 N_basis),
    n_occ = round(N_basis / 10), 4 core states each, energy ranges as in the acene-like system."""
    out = []
    for k in range(n_systems):
        seed = first_seed + k
        nb = nb_range[0] + int(counter_uniform(seed, 1) * (nb_range[1] - nb_range[0] + 1) - 1e-12)
        nb = min(max(nb, nb_range[0]), nb_range[1])
        n_occ = int(round(nb / 10))
        out.append(SystemSpec(n_basis=nb, n_occ=n_occ, n_aux=int(round(3.3 * nb)), seed=seed, n_core=4,
                              core_center=-10.6, core_halfwidth=0.01, valence=(-1.2, -0.25), virtual=(0.01, 5.0),
                              states=(0, 1, 2, 3), name=f"batch-{seed}-{nb}"))
    return out


def custom_system(n_basis, n_occ, n_aux, seed, n_core=1, states=(0,), core_scale=1.0,
                  valence=(-1.2, -0.25), virtual=(0.01, 5.0), core_center=-10.6, core_halfwidth=0.01) -> SystemSpec:
    """Any size with the acene-like energy distributions (used for parity tests of ragged shapes)."""
    return SystemSpec(n_basis=n_basis, n_occ=n_occ, n_aux=n_aux, seed=seed, n_core=n_core, core_center=core_center,
                      core_halfwidth=core_halfwidth if n_core > 1 else 0.0, valence=valence, virtual=virtual,
                      states=tuple(states), core_scale=core_scale, name=f"custom-{n_basis}-{n_aux}-{seed}")


def omega_grid(n: int = 128, lo: float = -11.0, hi: float = -10.0) -> np.ndarray:
    """Real-frequency grid (Ha) on which Sigma_c is tabulated around the core level."""
    return np.linspace(lo, hi, n)
