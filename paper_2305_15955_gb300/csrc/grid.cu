// Modified Gauss-Legendre grid on [0, inf) for the imaginary-axis quadrature of I_n (Sec. 4) and the
// transition energies D_ia of the polarizability (Eq. piriv).
#include "common.cuh"

// One thread per node: Newton's method on the Legendre polynomial P_n from the asymptotic guess
// x ~ cos(pi (k + 3/4) / (n + 1/2)) (Tricomi), P_n and P_n' by the three-term recurrence; the weight is
// 2 / ((1 - x^2) P_n'(x)^2).  Node k is the k-th largest root; it is stored at index n-1-k so that x (and xi)
// ascend.  xi = omega0 (1 + x) / (1 - x), and the weight takes the Jacobian 2 omega0 / (1 - x)^2.
__global__ void gauss_legendre_kernel(int n, double omega0, double* xi, double* wxi) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double pi = 3.14159265358979323846;
  double x = cos(pi * (k + 0.75) / (n + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = x;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? x : p1, pn1 = (n == 1) ? 1.0 : p0;
    dp = n * (x * pn - pn1) / (x * x - 1.0);
    double dx = pn / dp;
    x -= dx;
    if (fabs(dx) <= 1e-16 * fabs(x) + 1e-300) break;
  }
  {  // derivative at the converged root
    double p0 = 1.0, p1 = x;
    for (int j = 2; j <= n; ++j) {
      double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    double pn = (n == 1) ? x : p1, pn1 = (n == 1) ? 1.0 : p0;
    dp = n * (x * pn - pn1) / (x * x - 1.0);
  }
  double w = 2.0 / ((1.0 - x * x) * dp * dp);
  int out = n - 1 - k;
  xi[out] = omega0 * (1.0 + x) / (1.0 - x);
  wxi[out] = w * 2.0 * omega0 / ((1.0 - x) * (1.0 - x));
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
