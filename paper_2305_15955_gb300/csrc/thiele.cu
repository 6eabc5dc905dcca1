// Greedy Thiele continued-fraction fit of W_nm (Sec. 3.2; Eqs. pade, pre_rec, rec_eq) and the generic
// near-real reference points omega_G (Sec. 3.3).
//
// One warp per (state n, occupied m).  The candidate set F_wac = {i xi_k} U {x_j + i eta_ref} lives in shared
// memory; lanes stride over it.  Step p updates the reciprocal differences of every remaining candidate,
//   g_p(z_i) = (g_{p-1}(zt_{p-1}) - g_{p-1}(z_i)) / ((z_i^2 - zt_{p-1}^2) g_{p-1}(z_i)),
// evaluates the convergent T^{p-1} at the remaining candidates (innermost level outwards), and takes the
// candidate with the largest (or smallest) L1 error |Re(T - W)| + |Im(T - W)| as node p, a_p = g_p(node).
// The first node maximises |W|.  Ties go to the lowest candidate index; a non-finite error counts as +inf;
// a non-finite a_p ends the fit early (breakdown) and the first n_used nodes stay valid.  The fit also ends
// once the largest remaining error is below pade_tol * max|W|: beyond that point the choice among candidates
// would be decided by rounding.
// This file is compiled without FMA contraction so that every product and sum rounds as written.
#include "common.cuh"

namespace {

struct WarpPick {
  int valid;
  double err;
  int idx;
};

__device__ inline bool better(const WarpPick& a, const WarpPick& b, bool want_max) {
  if (a.valid != b.valid) return a.valid > b.valid;
  if (!a.valid) return false;
  if (a.err != b.err) return want_max ? (a.err > b.err) : (a.err < b.err);
  return a.idx < b.idx;
}

__device__ inline WarpPick warp_best(WarpPick p, bool want_max) {
  for (int off = 16; off > 0; off >>= 1) {
    WarpPick o;
    o.valid = __shfl_xor_sync(0xffffffffu, p.valid, off);
    o.err = __shfl_xor_sync(0xffffffffu, p.err, off);
    o.idx = __shfl_xor_sync(0xffffffffu, p.idx, off);
    if (better(o, p, want_max)) p = o;
  }
  return p;
}

__global__ void thiele_fit_kernel(int n_states, int n_occ, int n_imag, int n_real, const double* __restrict__ xi,
                                  const double* __restrict__ W_imag, int n_basis, const cplx* __restrict__ z_real,
                                  const cplx* __restrict__ W_real, int M, int first_mode, int crit, double tol,
                                  int M_cap,
                                  cplx* __restrict__ a_out, cplx* __restrict__ z2_out, int* __restrict__ nodes_out,
                                  int* __restrict__ n_used_out, unsigned* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = n_imag + n_real;
  const int warps = blockDim.x / 32;
  const int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  const size_t per_warp = ((size_t)nc * (3 * sizeof(cplx) + sizeof(int)) + (size_t)2 * M * sizeof(cplx) + 15) & ~size_t(15);
  unsigned char* base = smem_raw + wid * per_warp;
  cplx* z2 = reinterpret_cast<cplx*>(base);
  cplx* Wv = z2 + nc;
  cplx* g = Wv + nc;
  cplx* a = g + nc;
  cplx* zt2 = a + M;
  int* rem = reinterpret_cast<int*>(zt2 + M);

  const int fit = blockIdx.x * warps + wid;
  if (fit >= n_states * n_occ) return;            // whole warp leaves together
  const int s = fit / n_occ, m = fit % n_occ;

  for (int i = lane; i < nc; i += 32) {
    if (i < n_imag) {
      double x = xi[i];
      z2[i] = mkc(-(x * x), 0.0);
      Wv[i] = mkc(W_imag[((long)s * n_imag + i) * n_basis + m], 0.0);
    } else {
      int j = i - n_imag;
      cplx z = z_real[(long)s * n_real + j];
      z2[i] = mkc(z.x * z.x - z.y * z.y, z.x * z.y + z.y * z.x);
      Wv[i] = W_real[((long)s * n_real + j) * n_occ + m];
    }
    g[i] = Wv[i];
    rem[i] = 1;
  }
  __syncwarp();

  // largest |W| over the candidates (scale of the stopping rule)
  double wmax = 0.0;
  for (int i = lane; i < nc; i += 32) wmax = fmax(wmax, hypot(Wv[i].x, Wv[i].y));
  for (int off = 16; off > 0; off >>= 1) wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, off));
  const double stop_below = tol * wmax;

  // node 1
  WarpPick pk{0, 0.0, 0};
  for (int i = lane; i < nc; i += 32) {
    double key = first_mode == 0 ? hypot(Wv[i].x, Wv[i].y) : (first_mode == 1 ? Wv[i].x : -(double)i);
    WarpPick c{1, isfinite(key) ? key : INFINITY, i};
    if (better(c, pk, true)) pk = c;
  }
  pk = warp_best(pk, true);
  int k = pk.idx;
  if (lane == 0) {
    a[0] = g[k];
    zt2[0] = z2[k];
    rem[k] = 0;
  }
  __syncwarp();
  int used = 1;
  int broke = 0;
  const int Mx = min(M, nc);
  for (int p = 1; p < Mx; ++p) {
    const cplx ap = a[p - 1], zp = zt2[p - 1];
    WarpPick best{0, 0.0, 0};
    double emax = 0.0;
    for (int i = lane; i < nc; i += 32) {
      if (!rem[i]) continue;
      cplx gi = g[i];
      gi = (ap - gi) / ((z2[i] - zp) * gi);
      g[i] = gi;
      // convergent T^{p} built from a[0..p-1] at z2[i]
      cplx t = mkc(1.0, 0.0);
      for (int q = p - 1; q >= 1; --q) {
        cplx v = (a[q] * (z2[i] - zt2[q - 1])) / t;
        t = mkc(1.0 + v.x, v.y);
      }
      cplx T = a[0] / t;
      cplx d = T - Wv[i];
      double err = fabs(d.x) + fabs(d.y);
      if (!isfinite(err)) err = INFINITY;
      emax = fmax(emax, err);
      WarpPick c{1, err, i};
      if (better(c, best, crit == 0)) best = c;
    }
    best = warp_best(best, crit == 0);
    for (int off = 16; off > 0; off >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, off));
    __syncwarp();
    if (!best.valid) break;
    if (emax < stop_below) break;     // every remaining value is already reproduced
    k = best.idx;
    cplx gk = g[k];
    if (!finite_c(gk)) {
      broke = 1;
      break;
    }
    if (lane == 0) {
      a[p] = gk;
      zt2[p] = z2[k];
      rem[k] = 0;
      nodes_out[(long)fit * M_cap + p] = k;
    }
    __syncwarp();
    ++used;
  }
  __syncwarp();
  for (int p = lane; p < used; p += 32) {
    a_out[(long)fit * M_cap + p] = a[p];
    z2_out[(long)fit * M_cap + p] = zt2[p];
  }
  if (lane == 0) {
    nodes_out[(long)fit * M_cap + 0] = pk.idx;
    n_used_out[fit] = used;
    if (broke) raise_status(status, DEV_INFO_PADE_BREAKDOWN);
  }
}

// n equidistant abscissae on the neighbourhood of radius delta around the centres [c_lo, c_hi], cut to Re z >= 0:
// [max(0, c_lo - delta), c_hi + delta] with both ends; x_j = j * step + lo (product and sum rounded separately),
// the last one exactly hi; a single point at the middle of the centres.
__device__ double region_point(double c_lo, double c_hi, double delta, int n, int j) {
  if (n == 1) return fmax(0.0, 0.5 * (c_lo + c_hi));
  const double lo = fmax(0.0, c_lo - delta), hi = c_hi + delta;
  if (j == n - 1) return hi;
  return __dadd_rn(__dmul_rn((double)j, (hi - lo) / (double)(n - 1)), lo);
}

// Near-real reference points z_j = x_j + i eta_ref (Sec. 3.3), one set per system spanning the residues of every
// requested state n, so that each Pi(z_j) + LDL^T serves all of them.
//   generic  omega_G: x_j = j * top / (n_real - 1), x_{n_real-1} = top, top = max_n |eps_F - eps_n| + margin
//   refined  omega_C: n_core points around the core-level residues |eps_n' - eps_n| at omega = eps_n (radius
//            delta_c), then omega_V: n_real - n_core points around r_n = |eps_F - eps_n| (radius delta_v)
__global__ void near_real_kernel(const double* eps, int n_occ, const int* states, int n_states, int n_real,
                                 int refined, int n_core, double delta_c, double delta_v, double eta_ref,
                                 double margin, cplx* z_real) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_states * n_real) return;
  const int j = idx % n_real;
  const double ef = 0.5 * (eps[n_occ - 1] + eps[n_occ]);
  double e_lo = eps[states[0]], e_hi = e_lo, r_lo = fabs(ef - e_lo), r_hi = r_lo;
  for (int t = 1; t < n_states; ++t) {
    const double e = eps[states[t]], r = fabs(ef - e);
    e_lo = fmin(e_lo, e);
    e_hi = fmax(e_hi, e);
    r_lo = fmin(r_lo, r);
    r_hi = fmax(r_hi, r);
  }
  double x;
  if (!refined) {
    const double top = r_hi + margin;
    x = n_real == 1 ? 0.0 : (j == n_real - 1 ? top : (double)j * (top / (double)(n_real - 1)));
  } else if (j < n_core) {
    x = region_point(0.0, e_hi - e_lo, delta_c, n_core, j);
  } else {
    x = region_point(r_lo, r_hi, delta_v, n_real - n_core, j - n_core);
  }
  z_real[idx] = mkc(x, eta_ref);
}

}  // namespace

cdwac_status launch_near_real_points(cdwac_ctx* ctx, const double* eps, int n_occ, const int* states, int n_states,
                                     const cdwac_params* prm, double* z_real, cudaStream_t st) {
  const int n = n_states * prm->n_real;
  if (n == 0) return CDWAC_OK;
  const bool refined = prm->real_set == CDWAC_REAL_REFINED;
  near_real_kernel<<<ceil_div(n, 128), 128, 0, st>>>(eps, n_occ, states, n_states, prm->n_real, refined ? 1 : 0,
                                                      refined ? prm->n_core : 0, prm->delta_c, prm->delta_v,
                                                      prm->eta_ref, prm->real_margin, reinterpret_cast<cplx*>(z_real));
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status launch_thiele_fit(cdwac_ctx* ctx, int n_states, int n_occ, int n_imag, int n_real, const double* xi,
                               const double* W_imag, int n_basis, const double* z_real, const double* W_real,
                               const cdwac_params* prm, const cdwac_pade* pade, cudaStream_t st) {
  const int nc = n_imag + n_real;
  const int M = prm->pade_M;
  const size_t per_warp = ((size_t)nc * (3 * sizeof(cplx) + sizeof(int)) + (size_t)2 * M * sizeof(cplx) + 15) & ~size_t(15);
  int warps = 4;
  while (warps > 1 && per_warp * warps > 200 * 1024) warps >>= 1;
  const size_t smem = per_warp * warps;
  if (smem > 220 * 1024) return set_error(ctx, CDWAC_ERR_ARG, "thiele: candidate set too large for shared memory");
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(thiele_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int fits = n_states * n_occ;
  thiele_fit_kernel<<<ceil_div(fits, warps), warps * 32, smem, st>>>(
      n_states, n_occ, n_imag, n_real, xi, W_imag, n_basis, reinterpret_cast<const cplx*>(z_real),
      reinterpret_cast<const cplx*>(W_real), M, prm->greedy_first, prm->greedy_crit, prm->pade_tol, pade->M,
      reinterpret_cast<cplx*>(pade->a), reinterpret_cast<cplx*>(pade->z2), pade->nodes, pade->n_used,
      ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}
