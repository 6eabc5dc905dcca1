"""Error bound of the mixed path's W tables, shared by the mixed-precision GPU tests.

With hi = bf16(x) and lo = bf16(x - hi) an FP32 operand keeps x - hi - lo <= 2^-17 |x|, the dropped lo*lo product
is <= 2^-18 |x y|, and the weighted operand S = fp32(w) * x adds two FP32 roundings: every term S_Pk B_Qk of Pi
carries a relative error below 2^-16, with signs that vary from term to term (the tensor-core accumulation runs in
short chains summed with round-to-nearest, so it adds only a bias of order 1e-7), and the normwise error of Pi is
taken as 2^-16 ||Pi||_2.  The W solves' split-BF16 products and FP32 block solves act as a backward error of the
same size on the factor.  Together u = 2^-15 of ||I - Pi||_2, and first-order perturbation of
W_nm = o_m^T [(I - Pi)^-1 - I] o_m bounds |dW_nm| <= u kappa(I - Pi) ||(I - Pi)^-1||_2 ||o_m||^2 with kappa the
2-norm condition number, evaluated from the oracle's matrices (FP64) with a safety factor of 4.
"""
import numpy as np

from oracle import cdwac_oracle as o

U_BF16X3 = 2.0 ** -15
SAFETY = 4.0


def w_bound(B, D, On, z, m_idx):
    """Per-state bound on |dW_nm| over m_idx at frequency z, and kappa(I - Pi(z))."""
    A = np.eye(B.shape[0]) - o.polarizability(B, D, complex(z))
    sv = np.linalg.svd(A, compute_uv=False)
    kappa, inv_norm = sv[0] / sv[-1], 1.0 / sv[-1]
    on2 = np.sum(On[:, :, m_idx] ** 2, axis=1)                      # [n_states, len(m_idx)]
    return SAFETY * U_BF16X3 * kappa * inv_norm * on2, kappa
