// Modified Gauss-Legendre grid on [0, inf) for the imaginary-axis quadrature of I_n (Sec. 4) and the
// transition energies D_ia of the polarizability (Eq. piriv).
#include "common.cuh"

// Double-double arithmetic (Dekker 1971; Bailey's QD library): a value is hi + lo with |lo| <= ulp(hi)/2.
// This file is compiled without FMA contraction; two_prod uses an explicit fma for the exact product error.
namespace {
struct dd {
  double hi, lo;
};
__device__ inline dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
__device__ inline dd two_prod(double a, double b) {
  double p = a * b;
  return {p, fma(a, b, -p)};
}
__device__ inline dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
__device__ inline dd dd_sub(dd a, dd b) { return dd_add(a, dd{-b.hi, -b.lo}); }
__device__ inline dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  p.lo += a.hi * b.lo + a.lo * b.hi;
  return quick_two_sum(p.hi, p.lo);
}
__device__ inline dd dd_muld(dd a, double b) {
  dd p = two_prod(a.hi, b);
  p.lo += a.lo * b;
  return quick_two_sum(p.hi, p.lo);
}
__device__ inline dd dd_div(dd a, dd b) {
  double q1 = a.hi / b.hi;
  dd r = dd_sub(a, dd_muld(b, q1));
  double q2 = r.hi / b.hi;
  r = dd_sub(r, dd_muld(b, q2));
  double q3 = r.hi / b.hi;
  return dd_add(quick_two_sum(q1, q2), dd{q3, 0.0});
}
__device__ inline dd ddv(double v) { return {v, 0.0}; }

// P_n(x), P_{n-1}(x) by j P_j = (2j - 1) x P_{j-1} - (j - 1) P_{j-2}
__device__ inline void legendre_dd(int n, dd x, dd& pn, dd& pn1) {
  dd p0 = ddv(1.0), p1 = x;
  for (int j = 2; j <= n; ++j) {
    dd p2 = dd_div(dd_sub(dd_muld(dd_mul(x, p1), 2.0 * j - 1.0), dd_muld(p0, j - 1.0)), ddv((double)j));
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pn1 = p0;
}
}  // namespace

// One thread per node.  Newton's method on the Legendre polynomial P_n from the asymptotic guess
// x ~ cos(pi (k + 3/4) / (n + 1/2)) (Tricomi), first in double, then refined in double-double; the weight is
// 2 / ((1 - x^2) P_n'(x)^2) with P_n' = n (x P_n - P_{n-1}) / (x^2 - 1).  xi = omega0 (1 + x) / (1 - x) and the
// weight times the Jacobian 2 omega0 / (1 - x)^2 are formed in double-double and rounded once, so the grid is
// the exact rule correctly rounded to FP64.  Node k is the k-th largest root, stored at n-1-k (ascending).
__global__ void gauss_legendre_kernel(int n, double omega0, double* xi, double* wxi) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double pi = 3.14159265358979323846;
  double x = (n == 1) ? 0.0 : cos(pi * (k + 0.75) / (n + 0.5));
  for (int it = 0; it < 100 && n > 1; ++it) {
    double p0 = 1.0, p1 = x;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (x * p1 - p0) / (x * x - 1.0);
    double dx = p1 / dp;
    x -= dx;
    if (fabs(dx) <= 1e-15 * fabs(x) + 1e-300) break;
  }
  dd X = ddv(x), dP = ddv(1.0);
  if (n > 1) {
    for (int it = 0; it < 4; ++it) {
      dd pn, pn1;
      legendre_dd(n, X, pn, pn1);
      dP = dd_div(dd_muld(dd_sub(dd_mul(X, pn), pn1), (double)n), dd_sub(dd_mul(X, X), ddv(1.0)));
      dd dx = dd_div(pn, dP);
      X = dd_sub(X, dx);
      if (fabs(dx.hi) <= 1e-33 * fabs(X.hi) + 1e-300) break;
    }
    dd pn, pn1;
    legendre_dd(n, X, pn, pn1);
    dP = dd_div(dd_muld(dd_sub(dd_mul(X, pn), pn1), (double)n), dd_sub(dd_mul(X, X), ddv(1.0)));
  }
  dd one = ddv(1.0), om = ddv(omega0);
  dd onepx = dd_add(one, X), onemx = dd_sub(one, X);
  dd w = dd_div(ddv(2.0), dd_mul(dd_sub(one, dd_mul(X, X)), dd_mul(dP, dP)));
  dd xv = dd_div(dd_mul(om, onepx), onemx);
  dd wv = dd_div(dd_muld(dd_mul(w, om), 2.0), dd_mul(onemx, onemx));
  int out = n - 1 - k;
  xi[out] = xv.hi + xv.lo;
  wxi[out] = wv.hi + wv.lo;
}

cdwac_status launch_gauss_legendre(cdwac_ctx* ctx, int n, double omega0, double* xi, double* wxi, cudaStream_t st) {
  gauss_legendre_kernel<<<ceil_div(n, 128), 128, 0, st>>>(n, omega0, xi, wxi);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

// D[i * n_virt + a] = eps[n_occ + a] - eps[i]
__global__ void transition_energy_kernel(const double* eps, int n_occ, int n_virt, double* D) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long n = (long)n_occ * n_virt;
  if (idx >= n) return;
  int i = int(idx / n_virt), a = int(idx % n_virt);
  D[idx] = eps[n_occ + a] - eps[i];
}

cdwac_status launch_transition_energies(cdwac_ctx* ctx, const double* eps, int n_occ, int n_virt, double* D,
                                        cudaStream_t st) {
  long n = (long)n_occ * n_virt;
  transition_energy_kernel<<<ceil_div(n, 256), 256, 0, st>>>(eps, n_occ, n_virt, D);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}
