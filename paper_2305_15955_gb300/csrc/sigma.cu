// Correlation self-energy by contour deformation, Sigma^c_n(omega) = R_n(omega) - I_n(omega)
// (Eqs. cdmain, In_term, Rn_term, ffact, cdselfe), and the quasiparticle equation (Eq. qp_eq).
//
// I_n(omega) = 1/(2 pi) sum_m int dw' W_nm(i w') / (a_m + i w'),  a_m = omega - eps_m - i eta sgn(eps_F - eps_m).
// W(iw') is even, so on the [0, inf) grid each node carries 1/(a + i xi) + 1/(a - i xi) = 2a / (a^2 + xi^2):
//   I_n(omega) = (1/pi) sum_k wxi_k sum_m W_nm(i xi_k) a_m / (a_m^2 + xi_k^2).
// R_n(omega) = sum_m f_m W_nm(|eps_m - omega| + i eta) with f_m of Eq. ffact (theta(0) = 1/2); in CD-WAC the
// occupied-m values come from the Thiele continued fractions T_nm (Eq. pade), evaluated innermost level
// outwards in FP64.
//
// Precision: FP64 throughout in CDWAC_PREC_FP64.  In CDWAC_PREC_MIXED the I_n terms are formed in FP32 and
// summed per thread in FP32 over at most a few hundred terms before FP64 accumulation; R_n stays FP64.
#include "common.cuh"

namespace {

constexpr int SIG_THREADS = 256;
constexpr double INV_PI = 0.318309886183790671537767526745;

struct SigmaArgs {
  int n_basis, n_occ, n_imag, n_states;
  const double* eps;
  const int* states;
  const double* xi;
  const double* wxi;
  const double* W_imag;     // [n_states][n_imag][n_basis]
  double eta;
  int mixed;
  // CD-WAC model (may be null: I term only)
  const cplx* pa;
  const cplx* pz2;
  const int* n_used;
  int M_cap;
  // learned continuation (may be null): [n_states][n_occ][CDWAC_MLP_POLES][2] (Omega, residue)
  const double* poles;
  // W_nm(0) [n_states][n_basis] (may be null): the I term's xi -> 0 part integrated in closed form
  const double* W_zero;
  // energies eps_n of the QP equation (may be null: eps); eps then holds the energies of G
  const double* eps_qp;
};

__device__ inline double theta(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? 0.0 : 0.5); }

// Block-wide complex sum; result returned to every thread.
__device__ inline cplx block_sum(cplx v, cplx* red) {
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32, nw = blockDim.x / 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < nw) ? red[l] : mkc(0.0, 0.0);
    for (int off = 16; off > 0; off >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    if (l == 0) red[32] = v;
  }
  __syncthreads();
  return red[32];
}

// This thread's share of I_n(omega) for state s (sum over m strided by the block, all k).
// With W_zero: I_n = sum_m [sgn(omega - eps_m) W_nm(0) / 2 + 1/pi sum_k wxi_k (W_nm(i xi_k) - W_nm(0)) a/(a^2+xi^2)]:
// the Lorentzian of width |omega - eps_m| integrates to pi/2 sgn(omega - eps_m) over [0, inf) whatever the grid,
// and what is left vanishes like xi^2 at the origin (needed when omega sits next to eps_m, as at evGW
// self-consistency).
__device__ inline cplx partial_I(const SigmaArgs& A, int s, double omega) {
  const double* W = A.W_imag + (long)s * A.n_imag * A.n_basis;
  const double* W0 = A.W_zero ? A.W_zero + (long)s * A.n_basis : nullptr;
  cplx acc = mkc(0.0, 0.0);
  double closed = 0.0;
  for (int m = threadIdx.x; m < A.n_basis; m += blockDim.x) {
    const double al = omega - A.eps[m];
    const double be = -A.eta * (m < A.n_occ ? 1.0 : -1.0);
    const double w0 = W0 ? W0[m] : 0.0;
    closed += al > 0.0 ? 0.5 * w0 : (al < 0.0 ? -0.5 * w0 : 0.0);
    if (!A.mixed) {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < A.n_imag; ++k) {
        const double x = A.xi[k];
        const double u = al * al - be * be + x * x, v = 2.0 * al * be;
        const double c = A.wxi[k] * (W[(long)k * A.n_basis + m] - w0) / (u * u + v * v);
        sr += c * (al * u + be * v);
        si += c * (be * u - al * v);
      }
      acc.x += sr;
      acc.y += si;
    } else {
      const float alf = (float)al, bef = (float)be;
      float sr = 0.f, si = 0.f;
      for (int k = 0; k < A.n_imag; ++k) {
        const float x = (float)A.xi[k];
        const float u = alf * alf - bef * bef + x * x, v = 2.f * alf * bef;
        const float c = (float)A.wxi[k] * (float)(W[(long)k * A.n_basis + m] - w0) / (u * u + v * v);
        sr += c * (alf * u + bef * v);
        si += c * (bef * u - alf * v);
      }
      acc.x += (double)sr;
      acc.y += (double)si;
    }
  }
  return mkc(acc.x * INV_PI + closed, acc.y * INV_PI);
}

// This thread's share of R_n(omega) from the continued fractions (occupied m).
__device__ inline cplx partial_R_wac(const SigmaArgs& A, int s, double omega, unsigned* status, bool report) {
  cplx acc = mkc(0.0, 0.0);
  for (int m = threadIdx.x; m < A.n_occ; m += blockDim.x) {
    const double f = -theta(A.eps[m] - omega);
    if (f == 0.0) continue;
    const double x = fabs(A.eps[m] - omega);
    const cplx z2 = mkc(x * x - A.eta * A.eta, 2.0 * x * A.eta);
    const long base = ((long)s * A.n_occ + m) * A.M_cap;
    const int M = A.n_used[(long)s * A.n_occ + m];
    cplx t = mkc(1.0, 0.0);
    for (int q = M - 1; q >= 1; --q) {
      cplx v = (A.pa[base + q] * (z2 - A.pz2[base + q - 1])) / t;
      t = mkc(1.0 + v.x, v.y);
    }
    cplx T = A.pa[base] / t;
    acc = acc + f * T;
  }
  // a virtual residue (omega above a virtual level) has no continuation
  if (report && threadIdx.x == 0 && omega > A.eps[A.n_occ]) raise_status(status, DEV_ERR_BOUNDS);
  return acc;
}

// This thread's share of R_n(omega) from the learned pole model: T(z) = -sum_s r_s 2 Omega_s / (Omega_s^2 - z^2).
__device__ inline cplx partial_R_poles(const SigmaArgs& A, int s, double omega, unsigned* status, bool report) {
  cplx acc = mkc(0.0, 0.0);
  for (int m = threadIdx.x; m < A.n_occ; m += blockDim.x) {
    const double f = -theta(A.eps[m] - omega);
    if (f == 0.0) continue;
    const double x = fabs(A.eps[m] - omega);
    const cplx z2 = mkc(x * x - A.eta * A.eta, 2.0 * x * A.eta);
    const double* P = A.poles + ((long)s * A.n_occ + m) * CDWAC_MLP_POLES * 2;
    cplx T = mkc(0.0, 0.0);
    for (int q = 0; q < CDWAC_MLP_POLES; ++q) {
      const double Om = P[2 * q], r = P[2 * q + 1];
      T = T - (r * 2.0 * Om) * (mkc(1.0, 0.0) / (mkc(Om * Om, 0.0) - z2));
    }
    acc = acc + f * T;
  }
  if (report && threadIdx.x == 0 && omega > A.eps[A.n_occ]) raise_status(status, DEV_ERR_BOUNDS);
  return acc;
}

__device__ inline cplx block_sigma(const SigmaArgs& A, int s, double omega, cplx* red, unsigned* status,
                                   bool report = true) {
  cplx v = mkc(0.0, 0.0) - partial_I(A, s, omega);
  if (A.pa) v = v + partial_R_wac(A, s, omega, status, report);
  else if (A.poles) v = v + partial_R_poles(A, s, omega, status, report);
  return block_sum(v, red);
}

__global__ void __launch_bounds__(SIG_THREADS) sigma_kernel(SigmaArgs A, const double* omega, int n_omega,
                                                            cplx* sigma, unsigned* status) {
  __shared__ cplx red[33];
  const int j = blockIdx.x, s = blockIdx.y;
  cplx v = block_sigma(A, s, omega[j], red, status);
  if (threadIdx.x == 0) sigma[(long)s * n_omega + j] = v;
}

// Fixed point e <- eps_n + shift + Re Sigma(e) (for CD-WAC it stops if an iterate leaves the range below the
// LUMO); fallback: bisect every sign change of
// f(w) = w - eps_n - shift - Re Sigma(w) on the grid, keep roots with |f| < 1e-6 and the largest Z in (0, 1].
__global__ void __launch_bounds__(SIG_THREADS) qp_kernel(SigmaArgs A, const double* shift, const double* grid,
                                                         int n_grid, double tol, int max_iter, double* e_qp,
                                                         double* Zout, int* iters, int* qst, unsigned* status) {
  __shared__ cplx red[33];
  const int s = blockIdx.x;
  const double en = A.eps_qp ? A.eps_qp[A.states[s]] : A.eps[A.states[s]];
  const double sh = shift ? shift[s] : 0.0;
  const double h = 1e-5;
  auto resig = [&](double w) { return block_sigma(A, s, w, red, status, false).x; };
  // the continuation covers residues of occupied orbitals only: an iterate above the LUMO ends the fixed point
  const double upper = (A.pa || A.poles) ? A.eps[A.n_occ] : INFINITY;
  auto zfac = [&](double e) {
    double d = (resig(e + h) - resig(e - h)) / (2.0 * h);
    return 1.0 / (1.0 - d);
  };
  double e = en;     // the fixed point starts from eps_n of the equation (the KS level, in every evGW cycle too)
  int it = 1;
  int conv = 0;
  double e_new = e;
  for (it = 1; it <= max_iter; ++it) {
    e_new = en + sh + resig(e);
    if (!(e_new < upper)) break;
    if (fabs(e_new - e) < tol) {
      conv = 1;
      break;
    }
    e = e_new;
  }
  double res_e, res_z;
  int st;
  if (conv) {
    res_e = e_new;
    res_z = zfac(e_new);
    st = 0;
  } else {
    it = max_iter;
    bool found = false;
    double be = 0.0, bz = 0.0;
    double fprev = grid[0] - en - sh - resig(grid[0]);
    for (int j = 0; j + 1 < n_grid; ++j) {
      double fnext = grid[j + 1] - en - sh - resig(grid[j + 1]);
      if (fprev == 0.0 || fprev * fnext < 0.0) {
        double lo = grid[j], hi = grid[j + 1], flo = fprev;
        for (int b = 0; b < 200 && hi - lo > 1e-9; ++b) {
          double mid = 0.5 * (lo + hi);
          double fm = mid - en - sh - resig(mid);
          if (fm * flo <= 0.0) {
            hi = mid;
          } else {
            lo = mid;
            flo = fm;
          }
        }
        double r = 0.5 * (lo + hi);
        double fr = r - en - sh - resig(r);
        if (fabs(fr) < 1e-6) {
          double zr = zfac(r);
          if (zr > 0.0 && zr <= 1.0 && (!found || zr > bz)) {
            found = true;
            be = r;
            bz = zr;
          }
        }
      }
      fprev = fnext;
    }
    if (found) {
      res_e = be;
      res_z = bz;
      st = 1;
    } else {
      res_e = e;
      res_z = zfac(e);
      st = 2;
      if (threadIdx.x == 0) raise_status(status, DEV_INFO_QP_NOT_CONVERGED);
    }
  }
  if (threadIdx.x == 0) {
    e_qp[s] = res_e;
    Zout[s] = res_z;
    iters[s] = it;
    qst[s] = st;
  }
}

SigmaArgs make_args(const cdwac_system* sys, const cdwac_params* prm, const double* xi, const double* wxi,
                    const double* W_imag, const cdwac_pade* pade) {
  SigmaArgs A;
  A.n_basis = sys->n_basis;
  A.n_occ = sys->n_occ;
  A.n_imag = prm->n_imag;
  A.n_states = sys->n_states;
  A.eps = sys->eps;
  A.states = sys->states;
  A.xi = xi;
  A.wxi = wxi;
  A.W_imag = W_imag;
  A.eta = prm->eta;
  A.mixed = prm->precision == CDWAC_PREC_MIXED;
  A.pa = pade ? reinterpret_cast<const cplx*>(pade->a) : nullptr;
  A.pz2 = pade ? reinterpret_cast<const cplx*>(pade->z2) : nullptr;
  A.n_used = pade ? pade->n_used : nullptr;
  A.M_cap = pade ? pade->M : 0;
  A.poles = nullptr;
  A.W_zero = nullptr;
  A.eps_qp = nullptr;
  return A;
}

__global__ void scatter_states_kernel(double* __restrict__ eps, const int* __restrict__ states,
                                      const double* __restrict__ e, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) eps[states[i]] = e[i];
}

// Diagonal spectral function (Sec. 5.5): A = |Im[(omega - eps_n - shift_n - Sigma^c_n(omega))^-1]| / pi
//   = |Im d| / |d|^2 / pi,  d = omega - eps_n - shift_n - Sigma^c_n(omega).
__global__ void spectral_kernel(const double* __restrict__ eps, const int* __restrict__ states, int n_states,
                                const double* __restrict__ shift, const double* __restrict__ omega, int n_omega,
                                const cplx* __restrict__ sigma, double* __restrict__ Aout) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= (long)n_states * n_omega) return;
  const int s = (int)(e / n_omega), j = (int)(e % n_omega);
  const double dre = omega[j] - eps[states[s]] - (shift ? shift[s] : 0.0) - sigma[e].x;
  const double dim = -sigma[e].y;
  Aout[e] = fabs(dim) / (dre * dre + dim * dim) / 3.14159265358979323846;
}

}  // namespace

cdwac_status launch_spectral(cdwac_ctx* ctx, const double* eps, const int* states, int n_states, const double* shift,
                             const double* omega, int n_omega, const double* sigma, double* A, cudaStream_t st) {
  const long total = (long)n_states * n_omega;
  if (total <= 0) return CDWAC_OK;
  spectral_kernel<<<(int)((total + 255) / 256), 256, 0, st>>>(eps, states, n_states, shift, omega, n_omega,
                                                              reinterpret_cast<const cplx*>(sigma), A);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status launch_sigma_wac(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                              const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* omega,
                              int n_omega, double* sigma, cudaStream_t st, const double* W_zero) {
  if (n_omega <= 0) return CDWAC_OK;
  SigmaArgs A = make_args(sys, prm, xi, wxi, W_imag, pade);
  A.W_zero = W_zero;
  dim3 grid(n_omega, sys->n_states);
  sigma_kernel<<<grid, SIG_THREADS, 0, st>>>(A, omega, n_omega, reinterpret_cast<cplx*>(sigma), ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status launch_sigma_I_only(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm,
                                 const double* xi, const double* wxi, const double* W_imag, const double* omega,
                                 int n_omega, double* sigma, cudaStream_t st) {
  return launch_sigma_wac(ctx, sys, prm, xi, wxi, W_imag, nullptr, omega, n_omega, sigma, st);
}

cdwac_status launch_qp_wac(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                           const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* shift,
                           const double* omega, int n_grid, double tol, int max_iter, double* e_qp, double* Z,
                           int* iters, int* qp_status, cudaStream_t st, const double* W_zero, const double* eps_qp) {
  SigmaArgs A = make_args(sys, prm, xi, wxi, W_imag, pade);
  A.W_zero = W_zero;
  A.eps_qp = eps_qp;
  qp_kernel<<<sys->n_states, SIG_THREADS, 0, st>>>(A, shift, omega, n_grid, tol, max_iter, e_qp, Z, iters,
                                                     qp_status, ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status launch_sigma_poles(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                                const double* wxi, const double* W_imag, const double* poles, const double* omega,
                                int n_omega, double* sigma, cudaStream_t st) {
  if (n_omega <= 0) return CDWAC_OK;
  SigmaArgs A = make_args(sys, prm, xi, wxi, W_imag, nullptr);
  A.poles = poles;
  dim3 grid(n_omega, sys->n_states);
  sigma_kernel<<<grid, SIG_THREADS, 0, st>>>(A, omega, n_omega, reinterpret_cast<cplx*>(sigma), ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status launch_qp_poles(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                             const double* wxi, const double* W_imag, const double* poles, const double* shift,
                             const double* omega, int n_grid, double tol, int max_iter, double* e_qp, double* Z,
                             int* iters, int* qp_status, cudaStream_t st) {
  SigmaArgs A = make_args(sys, prm, xi, wxi, W_imag, nullptr);
  A.poles = poles;
  qp_kernel<<<sys->n_states, SIG_THREADS, 0, st>>>(A, shift, omega, n_grid, tol, max_iter, e_qp, Z, iters, qp_status,
                                                     ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status launch_scatter_states(cdwac_ctx* ctx, double* eps, const int* states, const double* e, int n,
                                   cudaStream_t st) {
  if (n <= 0) return CDWAC_OK;
  scatter_states_kernel<<<ceil_div(n, 128), 128, 0, st>>>(eps, states, e, n);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}
