"""Thin ctypes binding of libcdwac.so (declared in include/cdwac.h).

Argument marshalling only: PyTorch provides device memory and the current CUDA stream; every step of the
computation runs in the library's CUDA kernels.  There is no CPU fallback: if the library or a GPU is missing,
``load()`` raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libcdwac.so")
_lib = None

OK, ERR_ARG, ERR_CUDA, ERR_NOT_SPD, ERR_SINGULAR, ERR_PADE_BREAKDOWN, ERR_QP_NOT_CONVERGED, ERR_TIMEOUT, ERR_OOM, \
    ERR_UNSUPPORTED = range(10)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_CUDA", "ERR_NOT_SPD", "ERR_SINGULAR", "ERR_PADE_BREAKDOWN",
                "ERR_QP_NOT_CONVERGED", "ERR_TIMEOUT", "ERR_OOM", "ERR_UNSUPPORTED"]
F64, F32 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
LDLT_FP64, LDLT_EMULATED = 0, 1
REAL_GENERIC, REAL_REFINED = 0, 1
EVGW0, EVGW = 0, 1
MAX_M = 256
EXPORTED = ["cdwac_create", "cdwac_destroy", "cdwac_last_error", "cdwac_default_params", "cdwac_sync_status",
            "cdwac_scratch_bytes", "cdwac_build_W_imag", "cdwac_fit_pade", "cdwac_sigma", "cdwac_qp_solve",
            "cdwac_profile_enable", "cdwac_profile_read", "cdwac_launch_count", "cdwac_build_W_imag_noalloc",
            "cdwac_batch_run", "cdwac_mlp_features", "cdwac_mlp_loss_grad", "cdwac_mlp_adam", "cdwac_mlp_poles",
            "cdwac_sigma_poles", "cdwac_qp_solve_poles", "cdwac_spectral", "cdwac_ldlt_factor", "cdwac_evgw"]
MLP_IN, MLP_HIDDEN, MLP_POLES = 32, 256, 8
MLP_NPARAMS = 32 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 16 + 16
BATCH_GRAPH, BATCH_AUTOTUNE = 1, 2
NOALLOC_SCRATCH_BYTES = 16 << 20


class CdwacError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class _System(ctypes.Structure):
    _fields_ = [("n_basis", ctypes.c_int), ("n_occ", ctypes.c_int), ("n_aux", ctypes.c_int),
                ("n_states", ctypes.c_int), ("O_dtype", ctypes.c_int), ("eps", ctypes.c_void_p),
                ("O_ia", ctypes.c_void_p), ("O_n", ctypes.c_void_p), ("states", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("n_imag", ctypes.c_int), ("omega0", ctypes.c_double), ("n_real", ctypes.c_int),
                ("eta_ref", ctypes.c_double), ("real_margin", ctypes.c_double), ("eta", ctypes.c_double),
                ("pade_M", ctypes.c_int), ("greedy_first", ctypes.c_int), ("greedy_crit", ctypes.c_int),
                ("precision", ctypes.c_int), ("pade_tol", ctypes.c_double), ("real_set", ctypes.c_int),
                ("n_core", ctypes.c_int), ("n_val", ctypes.c_int), ("delta_c", ctypes.c_double),
                ("delta_v", ctypes.c_double)]


class _ProfEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double)]


class _Pade(ctypes.Structure):
    _fields_ = [("n_states", ctypes.c_int), ("n_occ", ctypes.c_int), ("M", ctypes.c_int),
                ("a", ctypes.c_void_p), ("z2", ctypes.c_void_p), ("nodes", ctypes.c_void_p),
                ("n_used", ctypes.c_void_p)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("sys", _System), ("xi", ctypes.c_void_p), ("wxi", ctypes.c_void_p), ("W_imag", ctypes.c_void_p),
                ("z_real", ctypes.c_void_p), ("W_real", ctypes.c_void_p), ("pade", _Pade),
                ("omega", ctypes.c_void_p), ("n_omega", ctypes.c_int), ("sigma", ctypes.c_void_p),
                ("shift", ctypes.c_void_p), ("qp_grid", ctypes.c_void_p), ("n_grid", ctypes.c_int),
                ("e_qp", ctypes.c_void_p), ("Z", ctypes.c_void_p), ("iters", ctypes.c_void_p),
                ("qp_status", ctypes.c_void_p)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libcdwac.so (built by paper_2305_15955_gb300.build); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: run paper_2305_15955_gb300.build.build() first")
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    lib.cdwac_create.argtypes = [ctypes.POINTER(P), ctypes.c_int]
    lib.cdwac_destroy.argtypes = [P]
    lib.cdwac_destroy.restype = None
    lib.cdwac_last_error.argtypes = [P]
    lib.cdwac_last_error.restype = ctypes.c_char_p
    lib.cdwac_default_params.argtypes = [ctypes.POINTER(_Params)]
    lib.cdwac_default_params.restype = None
    lib.cdwac_sync_status.argtypes = [P, P]
    lib.cdwac_scratch_bytes.argtypes = [P]
    lib.cdwac_scratch_bytes.restype = ctypes.c_size_t
    sysp, prmp, padep = ctypes.POINTER(_System), ctypes.POINTER(_Params), ctypes.POINTER(_Pade)
    lib.cdwac_build_W_imag.argtypes = [P, sysp, prmp, P, P, P, P]
    lib.cdwac_fit_pade.argtypes = [P, sysp, prmp, P, P, P, P, padep, P]
    lib.cdwac_sigma.argtypes = [P, sysp, prmp, P, P, P, padep, P, ctypes.c_int, P, P]
    lib.cdwac_qp_solve.argtypes = [P, sysp, prmp, P, P, P, padep, P, P, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_int, P, P, P, P, P]
    lib.cdwac_profile_enable.argtypes = [P, ctypes.c_int]
    lib.cdwac_profile_enable.restype = None
    lib.cdwac_profile_read.argtypes = [P, ctypes.POINTER(_ProfEntry), ctypes.c_int]
    lib.cdwac_launch_count.argtypes = [P]
    lib.cdwac_launch_count.restype = ctypes.c_longlong
    lib.cdwac_build_W_imag_noalloc.argtypes = [sysp, prmp, P, P, P, P, P]
    lib.cdwac_ldlt_factor.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
    lib.cdwac_spectral.argtypes = [P, sysp, prmp, P, P, P, padep, P, P, ctypes.c_int, P, P, P]
    lib.cdwac_evgw.argtypes = [P, sysp, prmp, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, P, P, P, ctypes.POINTER(ctypes.c_int), P]
    lib.cdwac_mlp_features.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P,
                                       ctypes.c_int, P, P, P, P, P]
    lib.cdwac_mlp_loss_grad.argtypes = [P, P, ctypes.c_int, P, P, ctypes.c_int, P, P, P, P, P]
    lib.cdwac_mlp_adam.argtypes = [P, P, P, P, P, ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, P]
    lib.cdwac_mlp_poles.argtypes = [P, P, ctypes.c_int, P, P, P, P]
    lib.cdwac_sigma_poles.argtypes = [P, sysp, prmp, P, P, P, P, P, ctypes.c_int, P, P]
    lib.cdwac_qp_solve_poles.argtypes = [P, sysp, prmp, P, P, P, P, P, P, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, P, P, P, P, P]
    lib.cdwac_batch_run.argtypes = [P, ctypes.POINTER(_BatchItem), ctypes.c_int, prmp, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_uint, ctypes.POINTER(ctypes.c_int), P]
    _lib = lib
    return lib


@dataclasses.dataclass
class Params:
    """Mirror of cdwac_params (defaults as cdwac_default_params)."""
    n_imag: int = 100
    omega0: float = 1.0
    n_real: int = 40
    eta_ref: float = 1e-3
    real_margin: float = 0.5
    eta: float = 1e-3
    pade_M: int = 64
    greedy_first: int = 0
    greedy_crit: int = 0
    precision: int = PREC_FP64
    pade_tol: float = 0.0
    real_set: int = REAL_GENERIC
    n_core: int = 20
    n_val: int = 20
    delta_c: float = 0.5
    delta_v: float = 0.5

    @classmethod
    def refined(cls, n_core=20, n_val=20, delta_c=0.5, delta_v=0.5, **kw):
        """CD-WAC(n_core, n_val, n_imag): the refined near-real set omega_C U omega_V (Sec. 3.3)."""
        return cls(n_real=n_core + n_val, real_set=REAL_REFINED, n_core=n_core, n_val=n_val, delta_c=delta_c,
                   delta_v=delta_v, **kw)

    def c(self) -> _Params:
        return _Params(self.n_imag, self.omega0, self.n_real, self.eta_ref, self.real_margin, self.eta, self.pade_M,
                       self.greedy_first, self.greedy_crit, self.precision, self.pade_tol, self.real_set,
                       self.n_core, self.n_val, self.delta_c, self.delta_v)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class System:
    """Device-resident system: eps [n_basis] f64, O_ia [n_aux, n_occ*n_virt], O_n [n_states, n_aux, n_basis]
    (both f64 or both f32), states [n_states] int32."""

    def __init__(self, eps, O_ia, O_n, states, n_occ, device="cuda"):
        dev = torch.device(device)
        self.eps = torch.as_tensor(eps, dtype=torch.float64).to(dev).contiguous()
        self.O_ia = torch.as_tensor(O_ia).to(dev).contiguous()
        self.O_n = torch.as_tensor(O_n).to(dev, dtype=self.O_ia.dtype).contiguous()
        self.states = torch.as_tensor(np.asarray(states, dtype=np.int32)).to(dev).contiguous()
        if self.O_ia.dtype not in (torch.float64, torch.float32):
            raise ValueError("O must be float64 or float32")
        self.n_basis = int(self.eps.numel())
        self.n_occ = int(n_occ)
        self.n_aux = int(self.O_ia.shape[0])
        self.n_states = int(self.states.numel())
        if tuple(self.O_ia.shape) != (self.n_aux, self.n_occ * (self.n_basis - self.n_occ)):
            raise ValueError(f"O_ia shape {tuple(self.O_ia.shape)} does not match the sizes")
        if tuple(self.O_n.shape) != (self.n_states, self.n_aux, self.n_basis):
            raise ValueError(f"O_n shape {tuple(self.O_n.shape)} does not match the sizes")
        self._c = _System(self.n_basis, self.n_occ, self.n_aux, self.n_states,
                          F64 if self.O_ia.dtype == torch.float64 else F32, self.eps.data_ptr(),
                          self.O_ia.data_ptr(), self.O_n.data_ptr(), self.states.data_ptr())

    @property
    def c(self):
        return self._c


@dataclasses.dataclass
class PadeModel:
    a: torch.Tensor        # [n_states, n_occ, M] complex128
    z2: torch.Tensor       # [n_states, n_occ, M] complex128
    nodes: torch.Tensor    # [n_states, n_occ, M] int32
    n_used: torch.Tensor   # [n_states, n_occ] int32
    z_real: torch.Tensor   # [n_states, n_real] complex128
    W_real: torch.Tensor   # [n_states, n_real, n_occ] complex128
    M: int

    def c(self) -> _Pade:
        ns, no, M = self.a.shape
        return _Pade(ns, no, M, self.a.data_ptr(), self.z2.data_ptr(), self.nodes.data_ptr(), self.n_used.data_ptr())


class Context:
    """A libcdwac context bound to one CUDA device; calls run on torch's current stream."""

    def __init__(self, device: int = 0):
        self.lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("libcdwac needs a CUDA device")
        self.device = device
        h = ctypes.c_void_p()
        st = self.lib.cdwac_create(ctypes.byref(h), device)
        if st != OK:
            raise CdwacError(st, "cdwac_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            torch.cuda.synchronize(self.device)
            self.lib.cdwac_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _check(self, st):
        if st != OK:
            raise CdwacError(st, self.lib.cdwac_last_error(self.h).decode())

    def sync_status(self, allow=(ERR_PADE_BREAKDOWN,)):
        """Wait for the stream and raise on a device error (statuses in `allow` are returned, not raised)."""
        st = self.lib.cdwac_sync_status(self.h, self._stream())
        if st != OK and st not in allow:
            raise CdwacError(st, self.lib.cdwac_last_error(self.h).decode())
        return st

    def scratch_bytes(self) -> int:
        return int(self.lib.cdwac_scratch_bytes(self.h))

    def profile(self, on=True):
        """Per-kernel-class CUDA-event timers (recorded on the calls' stream); on=2 also times the LDL^T steps."""
        self.lib.cdwac_profile_enable(self.h, int(on))

    def profile_read(self) -> dict:
        """{class: (launch groups timed, total ms)} accumulated since the last read (waits for the events)."""
        buf = (_ProfEntry * 32)()
        k = self.lib.cdwac_profile_read(self.h, buf, 32)
        if k < 0:
            raise CdwacError(ERR_CUDA, "cdwac_profile_read failed")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(k)}

    def launch_count(self) -> int:
        return int(self.lib.cdwac_launch_count(self.h))

    # ---- learned continuation -------------------------------------------------------------------------
    def mlp_features(self, xi, W_imag, n_occ, pade: PadeModel | None = None, n_real=0):
        """x [B, 32], scale [B], z_ref, w_ref [B, 32 + n_real] for every (state, occupied m) pair."""
        dev = self._dev()
        ns, n_imag, nb = W_imag.shape
        B, J = ns * n_occ, MLP_IN + n_real
        x = torch.empty(B, MLP_IN, dtype=torch.float32, device=dev)
        scale = torch.empty(B, dtype=torch.float32, device=dev)
        z_ref = torch.empty(B, J, dtype=torch.complex128, device=dev)
        w_ref = torch.empty(B, J, dtype=torch.complex128, device=dev)
        zr = _ptr(pade.z_real) if (pade is not None and n_real > 0) else None
        wr = _ptr(pade.W_real) if (pade is not None and n_real > 0) else None
        self._check(self.lib.cdwac_mlp_features(self.h, _ptr(xi), _ptr(W_imag), ns, n_imag, nb, n_occ, zr, wr,
                                                n_real, _ptr(x), _ptr(scale), _ptr(z_ref), _ptr(w_ref),
                                                self._stream()))
        return x, scale, z_ref, w_ref

    def mlp_loss_grad(self, params, x, scale, z_ref, w_ref, grad=None, loss=None):
        grad = torch.empty_like(params) if grad is None else grad
        loss = torch.empty(1, dtype=torch.float64, device=params.device) if loss is None else loss
        self._check(self.lib.cdwac_mlp_loss_grad(self.h, _ptr(params), int(x.shape[0]), _ptr(x), _ptr(scale),
                                                 int(z_ref.shape[1]), _ptr(z_ref), _ptr(w_ref), _ptr(grad),
                                                 _ptr(loss), self._stream()))
        return grad, loss

    def mlp_adam(self, params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.lib.cdwac_mlp_adam(self.h, _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step),
                                            float(lr), float(beta1), float(beta2), float(eps), self._stream()))

    def mlp_poles(self, params, x, scale):
        poles = torch.empty(x.shape[0], MLP_POLES, 2, dtype=torch.float64, device=params.device)
        self._check(self.lib.cdwac_mlp_poles(self.h, _ptr(params), int(x.shape[0]), _ptr(x), _ptr(scale),
                                             _ptr(poles), self._stream()))
        return poles

    def sigma_poles(self, system: System, params: Params, xi, wxi, W_imag, poles, omega, sync=True):
        dev = self._dev()
        omega = torch.as_tensor(omega, dtype=torch.float64).to(dev).contiguous()
        out = torch.empty(system.n_states, omega.numel(), dtype=torch.complex128, device=dev)
        p = params.c()
        self._check(self.lib.cdwac_sigma_poles(self.h, ctypes.byref(system.c), ctypes.byref(p), _ptr(xi), _ptr(wxi),
                                               _ptr(W_imag), _ptr(poles), _ptr(omega), int(omega.numel()), _ptr(out),
                                               self._stream()))
        if sync:
            self.sync_status()
        return out

    def qp_solve_poles(self, system: System, params: Params, xi, wxi, W_imag, poles, omega_grid, shift=None,
                       tol=1e-7, max_iter=100, sync=True):
        dev = self._dev()
        grid = torch.as_tensor(omega_grid, dtype=torch.float64).to(dev).contiguous()
        sh = None if shift is None else torch.as_tensor(shift, dtype=torch.float64).to(dev).contiguous()
        ns = system.n_states
        e = torch.empty(ns, dtype=torch.float64, device=dev)
        Z = torch.empty_like(e)
        it = torch.empty(ns, dtype=torch.int32, device=dev)
        qs = torch.empty_like(it)
        p = params.c()
        self._check(self.lib.cdwac_qp_solve_poles(self.h, ctypes.byref(system.c), ctypes.byref(p), _ptr(xi),
                                                  _ptr(wxi), _ptr(W_imag), _ptr(poles), _ptr(sh), _ptr(grid),
                                                  int(grid.numel()), float(tol), int(max_iter), _ptr(e), _ptr(Z),
                                                  _ptr(it), _ptr(qs), self._stream()))
        if sync:
            self.sync_status(allow=(ERR_PADE_BREAKDOWN, ERR_QP_NOT_CONVERGED))
        return e, Z, it, qs

    def _dev(self):
        return torch.device("cuda", self.device)

    def evgw(self, system: System, params: Params, mode, omega_grid, shift=None, cycle_tol=1e-6, max_cycles=30,
             plain_cd=False):
        """cdwac_evgw: (e_qp, Z, qp_status [n_states] on the device, cycles, status).  status is OK or
        ERR_QP_NOT_CONVERGED (no solution in a cycle, or max_cycles without self-consistency); other errors raise.
        plain_cd: residues from W built at every residue instead of the continued fractions."""
        dev = self._dev()
        grid = torch.as_tensor(omega_grid, dtype=torch.float64).to(dev).contiguous()
        sh = None if shift is None else torch.as_tensor(shift, dtype=torch.float64).to(dev).contiguous()
        ns = system.n_states
        e = torch.empty(ns, dtype=torch.float64, device=dev)
        Z = torch.empty_like(e)
        qs = torch.empty(ns, dtype=torch.int32, device=dev)
        cycles = ctypes.c_int(0)
        p = params.c()
        st = self.lib.cdwac_evgw(self.h, ctypes.byref(system.c), ctypes.byref(p), int(mode), int(bool(plain_cd)),
                                 _ptr(sh), _ptr(grid), int(grid.numel()), float(cycle_tol), int(max_cycles), _ptr(e),
                                 _ptr(Z), _ptr(qs), ctypes.byref(cycles), self._stream())
        if st not in (OK, ERR_QP_NOT_CONVERGED):
            self._check(st)
        self.sync_status(allow=(ERR_PADE_BREAKDOWN, ERR_QP_NOT_CONVERGED))
        return e, Z, qs, cycles.value, st

    def spectral(self, system: System, params: Params, xi, wxi, W_imag, pade: PadeModel | None, omega, shift=None,
                 sync=True):
        """cdwac_spectral: (Sigma^c [n_states, n_omega] complex, A [n_states, n_omega]) on the device."""
        dev = self._dev()
        omega = torch.as_tensor(omega, dtype=torch.float64).to(dev).contiguous()
        sig = torch.empty(system.n_states, omega.numel(), dtype=torch.complex128, device=dev)
        A = torch.empty(system.n_states, omega.numel(), dtype=torch.float64, device=dev)
        sh = None if shift is None else torch.as_tensor(shift, dtype=torch.float64).to(dev).contiguous()
        p = params.c()
        pc = pade.c() if pade is not None else None
        self._check(self.lib.cdwac_spectral(self.h, ctypes.byref(system.c), ctypes.byref(p), _ptr(xi), _ptr(wxi),
                                            _ptr(W_imag), ctypes.byref(pc) if pc is not None else None, _ptr(sh),
                                            _ptr(omega), int(omega.numel()), _ptr(sig), _ptr(A), self._stream()))
        if sync:
            self.sync_status()
        return sig, A

    def ldlt_factor(self, A, method: int = LDLT_FP64, sync: bool = True):
        """cdwac_ldlt_factor in place on a square float64 or complex128 CUDA tensor (row-major, contiguous): the
        lower triangle becomes the unit-lower L (below the diagonal) and D (on it)."""
        if A.dim() != 2 or A.shape[0] != A.shape[1] or not A.is_contiguous():
            raise ValueError("A must be a contiguous square matrix")
        if A.dtype not in (torch.float64, torch.complex128):
            raise ValueError("A must be float64 or complex128")
        self._check(self.lib.cdwac_ldlt_factor(self.h, _ptr(A), A.shape[0], int(A.dtype == torch.complex128),
                                               int(method), self._stream()))
        if sync:
            self.sync_status()
        return A

    def build_W_imag(self, system: System, params: Params, sync: bool = True):
        dev = self._dev()
        xi = torch.empty(params.n_imag, dtype=torch.float64, device=dev)
        wxi = torch.empty_like(xi)
        W = torch.empty(system.n_states, params.n_imag, system.n_basis, dtype=torch.float64, device=dev)
        p = params.c()
        self._check(self.lib.cdwac_build_W_imag(self.h, ctypes.byref(system.c), ctypes.byref(p), _ptr(xi),
                                                _ptr(wxi), _ptr(W), self._stream()))
        if sync:
            self.sync_status()
        return xi, wxi, W

    def alloc_pade(self, system: System, params: Params, M: int | None = None) -> PadeModel:
        dev = self._dev()
        M = params.pade_M if M is None else M
        ns, no = system.n_states, system.n_occ
        return PadeModel(a=torch.zeros(ns, no, M, dtype=torch.complex128, device=dev),
                         z2=torch.zeros(ns, no, M, dtype=torch.complex128, device=dev),
                         nodes=torch.full((ns, no, M), -1, dtype=torch.int32, device=dev),
                         n_used=torch.zeros(ns, no, dtype=torch.int32, device=dev),
                         z_real=torch.zeros(ns, max(params.n_real, 1), dtype=torch.complex128, device=dev),
                         W_real=torch.zeros(ns, max(params.n_real, 1), no, dtype=torch.complex128, device=dev),
                         M=M)

    def fit_pade(self, system: System, params: Params, xi, W_imag, pade: PadeModel | None = None, sync=True):
        pade = self.alloc_pade(system, params) if pade is None else pade
        p = params.c()
        pc = pade.c()
        self._check(self.lib.cdwac_fit_pade(self.h, ctypes.byref(system.c), ctypes.byref(p), _ptr(xi), _ptr(W_imag),
                                            _ptr(pade.z_real), _ptr(pade.W_real), ctypes.byref(pc), self._stream()))
        if sync:
            self.sync_status()
        return pade

    def sigma(self, system: System, params: Params, xi, wxi, W_imag, pade: PadeModel | None, omega, sync=True):
        dev = self._dev()
        omega = torch.as_tensor(omega, dtype=torch.float64).to(dev).contiguous()
        out = torch.empty(system.n_states, omega.numel(), dtype=torch.complex128, device=dev)
        p = params.c()
        pc = pade.c() if pade is not None else None
        self._check(self.lib.cdwac_sigma(self.h, ctypes.byref(system.c), ctypes.byref(p), _ptr(xi), _ptr(wxi),
                                         _ptr(W_imag), ctypes.byref(pc) if pc is not None else None, _ptr(omega),
                                         int(omega.numel()), _ptr(out), self._stream()))
        if sync:
            self.sync_status()
        return out

    def qp_solve(self, system: System, params: Params, xi, wxi, W_imag, pade: PadeModel | None, omega_grid,
                 shift=None, tol=1e-7, max_iter=100, sync=True):
        dev = self._dev()
        grid = torch.as_tensor(omega_grid, dtype=torch.float64).to(dev).contiguous()
        sh = None if shift is None else torch.as_tensor(shift, dtype=torch.float64).to(dev).contiguous()
        ns = system.n_states
        e = torch.empty(ns, dtype=torch.float64, device=dev)
        Z = torch.empty_like(e)
        it = torch.empty(ns, dtype=torch.int32, device=dev)
        qs = torch.empty_like(it)
        p = params.c()
        pc = pade.c() if pade is not None else None
        self._check(self.lib.cdwac_qp_solve(self.h, ctypes.byref(system.c), ctypes.byref(p), _ptr(xi), _ptr(wxi),
                                            _ptr(W_imag), ctypes.byref(pc) if pc is not None else None, _ptr(sh),
                                            _ptr(grid), int(grid.numel()), float(tol), int(max_iter), _ptr(e),
                                            _ptr(Z), _ptr(it), _ptr(qs), self._stream()))
        if sync:
            self.sync_status(allow=(ERR_PADE_BREAKDOWN, ERR_QP_NOT_CONVERGED))
        return e, Z, it, qs


class BatchResult:
    """Device outputs of one system of a batch (same layouts as the single-system calls)."""

    def __init__(self, system: System, params: Params, omega, qp_grid, dev):
        ns, nb, no = system.n_states, system.n_basis, system.n_occ
        self.system = system
        self.xi = torch.empty(params.n_imag, dtype=torch.float64, device=dev)
        self.wxi = torch.empty_like(self.xi)
        self.W_imag = torch.empty(ns, params.n_imag, nb, dtype=torch.float64, device=dev)
        nr = max(params.n_real, 1)
        self.pade = PadeModel(a=torch.zeros(ns, no, params.pade_M, dtype=torch.complex128, device=dev),
                              z2=torch.zeros(ns, no, params.pade_M, dtype=torch.complex128, device=dev),
                              nodes=torch.full((ns, no, params.pade_M), -1, dtype=torch.int32, device=dev),
                              n_used=torch.zeros(ns, no, dtype=torch.int32, device=dev),
                              z_real=torch.zeros(ns, nr, dtype=torch.complex128, device=dev),
                              W_real=torch.zeros(ns, nr, no, dtype=torch.complex128, device=dev), M=params.pade_M)
        self.omega = torch.as_tensor(omega, dtype=torch.float64).to(dev).contiguous()
        self.sigma = torch.empty(ns, self.omega.numel(), dtype=torch.complex128, device=dev)
        self.qp_grid = torch.as_tensor(qp_grid, dtype=torch.float64).to(dev).contiguous()
        self.e_qp = torch.empty(ns, dtype=torch.float64, device=dev)
        self.Z = torch.empty_like(self.e_qp)
        self.iters = torch.empty(ns, dtype=torch.int32, device=dev)
        self.qp_status = torch.empty_like(self.iters)

    def c(self) -> _BatchItem:
        return _BatchItem(self.system.c, self.xi.data_ptr(), self.wxi.data_ptr(), self.W_imag.data_ptr(),
                          self.pade.z_real.data_ptr(), self.pade.W_real.data_ptr(), self.pade.c(),
                          self.omega.data_ptr(), int(self.omega.numel()), self.sigma.data_ptr(), None,
                          self.qp_grid.data_ptr(), int(self.qp_grid.numel()), self.e_qp.data_ptr(),
                          self.Z.data_ptr(), self.iters.data_ptr(), self.qp_status.data_ptr())


def batch_run(ctx: "Context", results, params: Params, max_lanes=4, graph=False, autotune=False, tol=1e-7,
              max_iter=100, sync=True, items=None):
    """cdwac_batch_run over BatchResult objects; returns (lanes, lookahead, Pi tile-group size, Pi tile width,
    update waves) the call used and the ctypes items (pass them back as `items` to replay a captured graph with the
    identical item array)."""
    if items is None:
        items = (_BatchItem * len(results))(*[r.c() for r in results])
    p = params.c()
    chosen = (ctypes.c_int * 5)()
    flags = (BATCH_GRAPH if graph else 0) | (BATCH_AUTOTUNE if autotune else 0)
    ctx._check(ctx.lib.cdwac_batch_run(ctx.h, items, len(results), ctypes.byref(p), float(tol), int(max_iter),
                                       int(max_lanes), flags, chosen, ctx._stream()))
    if sync:
        ctx.sync_status(allow=(ERR_PADE_BREAKDOWN, ERR_QP_NOT_CONVERGED))
    return tuple(int(c) for c in chosen), items


def build_W_imag_noalloc(system: System, params: Params, xi, wxi, W_imag, dev_status=None, stream=None) -> int:
    """cdwac_build_W_imag_noalloc: FP64 W(i xi) into caller-provided tensors, no device allocation by the library.

    xi, wxi [n_imag], W_imag [n_states, n_imag, n_basis] float64 CUDA tensors; dev_status an int32 CUDA tensor of
    one element (pivot errors are OR-ed into it) or None.  Returns the call's status code (asynchronous)."""
    lib = load()
    p = params.c()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else stream)
    return int(lib.cdwac_build_W_imag_noalloc(ctypes.byref(system.c), ctypes.byref(p), _ptr(xi), _ptr(wxi),
                                              _ptr(W_imag), _ptr(dev_status), st))
