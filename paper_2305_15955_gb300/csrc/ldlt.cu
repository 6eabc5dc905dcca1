// Square-root-free Cholesky factorisation A = L D L^T of I - Pi (Eq. bigLambda) and the quadratic forms
// W_nm = o^T [(I - Pi)^-1 - I] o = sum_P y_P^2 / d_P - sum_P o_P^2,  y = L^-1 o   (Eq. wriv),
// in FP64, for real symmetric positive definite A (imaginary axis, Cholesky without square roots) and for
// complex symmetric A (near-real points and residues; no conjugation, no pivoting).
//
// Blocked right-looking factorisation with NB = 64 column blocks, three launches per block step:
//   diag  : one CTA factors the NB x NB diagonal block in shared memory;
//   panel : rows below: W_ik = A_ik L_kk^-T by forward substitution, L_ik = W_ik D_k^-1 (W_ik kept in a panel
//           buffer);
//   update: trailing lower triangle A_ij -= W_ik L_jk^T, with FP64 FMAs (update_kernel) or, given tensor-core
//           scratch, as exact BF16 digit products on the tcgen05 tensor cores (ozaki.cu; FP64-equivalent).
// After the last step one launch inverts every unit-lower diagonal block L_kk (the blocked solves use them).
// Only the lower triangle of A is read or written.  A non-positive (real) or vanishing (complex) pivot sets
// CDWAC_ERR_NOT_SPD / CDWAC_ERR_SINGULAR in the status word and the factorisation continues with a unit pivot,
// so no NaN reaches later kernels.
#include "common.cuh"
#include "ozaki.cuh"

__device__ inline double mkT(double v, double*) { return v; }
__device__ inline cplx mkT(double v, cplx*) { return mkc(v, 0.0); }

namespace {

constexpr int NB = 64;
constexpr int TK = 16;
constexpr int TP = 64 + 1;

template <class T>
__device__ inline T ld_as(const void* p, int dtype, long idx);
template <>
__device__ inline double ld_as<double>(const void* p, int dtype, long idx) {
  return dtype == CDWAC_F64 ? ((const double*)p)[idx] : (double)((const float*)p)[idx];
}

__device__ inline double shfl_xor_T(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ inline cplx shfl_xor_T(cplx v, int m) {
  return mkc(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// 1/d by Newton's iteration x <- x + x (1 - d x), started from the single-precision reciprocal of d: each step
// squares the relative error, so two steps take the 2^-23 start to the FP64 rounding level (the last step's
// rounding leaves x within an ulp or so of 1/d; the factorisation tests bound the result through its backward
// error).  Four FP64 FMAs and two conversions: GB300 issues one FP64 warp instruction in about 64 cycles, and the
// pivot reciprocal is on the factorisation's critical path.  Outside single precision's exponent range (|d|
// beyond 2^+-99) the division.
__device__ inline double rcp_T(double d) {
  const int E = (int)(((unsigned long long)__double_as_longlong(d) >> 52) & 0x7FF);
  if (E < 1023 - 99 || E > 1023 + 99) return 1.0 / d;
  double x = (double)__frcp_rn((float)d);
  double e = fma(-d, x, 1.0);
  x = fma(x, e, x);
  e = fma(-d, x, 1.0);
  return fma(x, e, x);
}
// 1/z = conj(z) / |z|^2 with the reciprocal above
__device__ inline cplx rcp_T(cplx z) {
  const double r = rcp_T(fma(z.x, z.x, z.y * z.y));
  return mkc(z.x * r, -z.y * r);
}

__device__ inline double shfl_T(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ inline cplx shfl_T(cplx v, int src) {
  return mkc(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

__device__ inline unsigned pivot_err(double) { return DEV_ERR_NOT_SPD; }
__device__ inline unsigned pivot_err(cplx) { return DEV_ERR_SINGULAR; }

// ---- diagonal block --------------------------------------------------------------------------------------
// One CTA (256 threads) factors the NB x NB block held in shared memory (row stride NB + 1).  Step j: the threads
// of rows i > j scale column j by 1/d_j (only they evaluate the pivot; GB300's FP64 units are scarce), then the
// trailing triangle j < k <= i is updated with l_i u_k (u = the unscaled column).  The triangle's elements are
// numbered by k from the last column down and i upwards, so that the elements of step j are the first
// (63 - j)(64 - j) / 2 numbers: every lane of every warp has work until the last steps.
__device__ inline bool bad_pivot_fast(double d) { return !(d > 0.0); }
__device__ inline bool bad_pivot_fast(cplx d) { return !(fabs(d.x) + fabs(d.y) > 1e-300); }

constexpr int SD = NB + 1;                 // shared-memory row stride of the diagonal block
constexpr int TRI = NB * (NB - 1) / 2;     // elements j < k <= i < NB of the first step, the largest
constexpr int PER_THREAD = (TRI + 255) / 256;

template <class T>
__global__ void __launch_bounds__(256) diag_kernel(T* A, int n, int k0, T* dinv, unsigned* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);            // [NB][SD]
  __shared__ T lcol[NB], ucol[NB];
  __shared__ int bad_step;
  using N = Num<T>;
  const int nb = min(NB, n - k0);
  const int tid = threadIdx.x;
#pragma unroll
  for (int it = 0; it < NB * NB / 256; ++it) {   // fixed count: every load of the block in flight at once
    const int e = tid + 256 * it, i = e / NB, j = e % NB;
    S[i * SD + j] = (i < nb && j <= i) ? A[(long)(k0 + i) * n + (k0 + j)] : (i == j ? N::one() : N::zero());
  }
  // this thread's trailing-triangle elements: number e -> (i, k), u = 63 - k, e in [u(u+1)/2, u(u+1)/2 + u]
  short ti[PER_THREAD], tk[PER_THREAD];
#pragma unroll
  for (int q = 0; q < PER_THREAD; ++q) {
    const int e = tid + 256 * q;
    int u = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while ((u + 1) * (u + 2) / 2 <= e) ++u;
    while (u * (u + 1) / 2 > e) --u;
    tk[q] = (short)(NB - 1 - u);
    ti[q] = (short)(NB - 1 - u + (e - u * (u + 1) / 2));
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (tid < NB) {                                   // warps 0 and 1, whole
      const T d0 = S[j * SD + j];
      const bool bad = bad_pivot_fast(d0);
      if (tid == 0) bad_step = bad ? 1 : 0;
      // one reciprocal per warp, broadcast (FP64 division is a multi-instruction sequence on the scarce FP64 units)
      T rinv = N::one();
      if ((tid & 31) == 0) rinv = bad ? N::one() : rcp_T(d0);
      rinv = shfl_T(rinv, 0);
      if (tid > j && tid < nb) {
        const T u = S[tid * SD + j];
        ucol[tid] = u;
        lcol[tid] = N::mul(u, rinv);
      }
    }
    __syncthreads();                                 // pivot read by every thread that needs it; l and u ready
    if (tid == 0 && bad_step) {
      raise_status(status, pivot_err(S[j * SD + j]));
      S[j * SD + j] = N::one();
    }
    if (tid > j && tid < nb) S[tid * SD + j] = lcol[tid];
    const int count = (NB - 1 - j) * (NB - j) / 2;   // elements with k > j
#pragma unroll
    for (int q = 0; q < PER_THREAD; ++q) {
      const int e = tid + 256 * q;
      const int i = ti[q], k = tk[q];
      if (e < count && i < nb) S[i * SD + k] = N::fms(lcol[i], ucol[k], S[i * SD + k]);
    }
    __syncthreads();
  }
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e % NB;
    if (i < nb && j <= i) A[(long)(k0 + i) * n + (k0 + j)] = S[i * SD + j];   // diagonal holds d_i
  }
  if (tid < nb) dinv[k0 + tid] = rcp_T(S[tid * SD + tid]);
}

// ---- inverses of the unit-lower diagonal blocks, for the solves after the factorisation ------------------------
// One CTA per block: X = L_kk^-1, X[c][c] = 1, X[i][c] = -sum_{c <= t < i} L[i][t] X[t][c]; thread (c, part)
// sums t = c + part mod 4.
template <class T>
__global__ void __launch_bounds__(256) inverse_kernel(const T* A, int n, T* linv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);            // [NB][NB] strict lower part of the block
  T* X = S + NB * NB;
  using N = Num<T>;
  const int k0 = blockIdx.x * NB, nb = min(NB, n - k0);
  const int tid = threadIdx.x;
#pragma unroll
  for (int it = 0; it < NB * NB / 256; ++it) {
    const int e = tid + 256 * it, i = e / NB, j = e % NB;
    S[e] = (i < nb && j < i) ? A[(long)(k0 + i) * n + (k0 + j)] : N::zero();
  }
  __syncthreads();
  const int c = tid / 4, part = tid % 4;
  for (int i = 0; i < NB; ++i)
    if (part == 0) X[i * NB + c] = (i == c && c < nb) ? N::one() : N::zero();
  __syncwarp();
  for (int i = 1; i < nb; ++i) {                    // uniform trip count: the shuffles need the whole warp
    const bool active = c < i;
    T s = N::zero();
    if (active)
      for (int t = c + part; t < i; t += 4) s = N::fma_(S[i * NB + t], X[t * NB + c], s);
    s = N::add(s, shfl_xor_T(s, 1));
    s = N::add(s, shfl_xor_T(s, 2));
    if (active && part == 0) X[i * NB + c] = N::sub(N::zero(), s);
    __syncwarp();
  }
  __syncthreads();
  for (int e = tid; e < NB * NB; e += blockDim.x) linv[(long)blockIdx.x * NB * NB + e] = X[e];
}

// ---- panel: W_i = A_i L_kk^-T (forward substitution), L_i = W_i D^-1 -------------------------------------------
// One CTA (4 warps) per 32 rows below the diagonal block: all threads stage the rows and the strict lower L_kk in
// shared memory (coalesced); four lanes share each row, w_c = a_c - sum_{t<c} w_t L_ct with lane q summing
// t = q mod 4 and two shuffles joining the parts; then all threads write the rows back as W (panel buffer) and L
// (in A).  Half the FP64 work of multiplying by an explicit inverse, and no inverse on the critical path.
constexpr int PR = 32;            // rows per CTA
constexpr int PT = 128;           // threads per CTA
template <class T>
__global__ void __launch_bounds__(PT) panel_kernel(T* A, int n, int k0, const T* dinv, T* wpanel) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);           // [NB][SD]: Ls[c][t] = L_kk[c][t], t < c
  T* Ws = Ls + NB * SD;                              // [NB][PR + 1]: Ws[c][r] = row r, column c
  using N = Num<T>;
  const int tid = threadIdx.x;
  const int r0 = k0 + NB + blockIdx.x * PR;
#pragma unroll 16
  for (int it = 0; it < NB * NB / PT; ++it) {     // fixed counts: the loads are issued back to back
    const int e = tid + PT * it, c = e / NB, t = e % NB;
    Ls[c * SD + t] = t < c ? A[(long)(k0 + c) * n + k0 + t] : N::zero();
  }
#pragma unroll
  for (int it = 0; it < PR * NB / PT; ++it) {
    const int e = tid + PT * it, rr = e / NB, c = e % NB, row = r0 + rr;
    Ws[c * (PR + 1) + rr] = row < n ? A[(long)row * n + k0 + c] : N::zero();
  }
  __syncthreads();
  const int r = tid / 4, q = tid % 4;               // row of this lane group, part of the sum
  for (int c = 1; c < NB; ++c) {
    T s = N::zero();
    for (int t = q; t < c; t += 4) s = N::fma_(Ws[t * (PR + 1) + r], Ls[c * SD + t], s);
    s = N::add(s, shfl_xor_T(s, 1));
    s = N::add(s, shfl_xor_T(s, 2));
    if (q == 0) Ws[c * (PR + 1) + r] = N::sub(Ws[c * (PR + 1) + r], s);
    __syncwarp();
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < PR * NB / PT; ++it) {
    const int e = tid + PT * it, rr = e / NB, c = e % NB, row = r0 + rr;
    if (row < n) {
      const T w = Ws[c * (PR + 1) + rr];
      wpanel[(long)row * NB + c] = w;
      A[(long)row * n + k0 + c] = N::mul(w, dinv[k0 + c]);
    }
  }
}

__device__ inline void lower_tile_coords(int b, int& ti, int& tj) {
  int t = int((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((t + 1) * (t + 2) / 2 <= b) ++t;
  while (t * (t + 1) / 2 > b) --t;
  ti = t;
  tj = b - t * (t + 1) / 2;
}

// ---- trailing update: A_ij -= W_i L_j^T over the lower triangle of rows/cols >= k1 -----------------------
// part 0: every lower tile of the trailing matrix; part 1: its first block column only (the next panel);
// part 2: every lower tile except the first block column.
template <class T>
__global__ void __launch_bounds__(256) update_kernel(T* A, int n, int k0, const T* wpanel, int part) {
  __shared__ T Ws[TK][TP];
  __shared__ T Ls[TK][TP];
  using N = Num<T>;
  const int nb = min(NB, n - k0);
  const int k1 = k0 + NB;
  int ti, tj;
  if (part == 1) {
    ti = blockIdx.x;
    tj = 0;
  } else {
    lower_tile_coords(blockIdx.x, ti, tj);
    if (part == 2) {
      ++ti;
      ++tj;
    }
  }
  const int row0 = k1 + ti * 64, col0 = k1 + tj * 64;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = N::zero();
  for (int c0 = 0; c0 < nb; c0 += TK) {
    for (int e = tid; e < TK * 64; e += 256) {
      int cc = e % TK, r = e / TK;
      int c = c0 + cc;
      int ra = row0 + r, rb = col0 + r;
      Ws[cc][r] = (ra < n && c < nb) ? wpanel[(long)ra * NB + c] : N::zero();
      Ls[cc][r] = (rb < n && c < nb) ? A[(long)rb * n + k0 + c] : N::zero();
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TK; ++q) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ws[q][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Ls[q][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = N::fma_(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int P = row0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int Q = col0 + tx * 4 + j;
      if (P < n && Q <= P) {
        long idx = (long)P * n + Q;
        A[idx] = N::sub(A[idx], acc[i][j]);
      }
    }
  }
}

// ---- quadratic forms through forward substitution -----------------------------------------------------------
// One CTA owns QC columns of O and walks all 64-row blocks: t_i = o_i - L_i,<i y_<i, y_i = L_ii^-1 t_i.
constexpr int QC = 8;    // columns per CTA
constexpr int QK = 16;   // K chunk of the off-diagonal product

template <class T>
__global__ void __launch_bounds__(256) quadform_kernel(const T* __restrict__ L, const T* __restrict__ dinv,
                                                       const T* __restrict__ linv, int n, const void* O, int dtype,
                                                       long o_state_stride, long ld_o, int cols_per_state,
                                                       int n_cols, T* ywork, T* W_out, long w_state_stride) {
  __shared__ T Ls[64][QK + 1];
  __shared__ T Ys[QK][QC];
  __shared__ T Ts[64][QC];
  __shared__ T red[256];
  __shared__ double ored[256];
  using N = Num<T>;
  const int tid = threadIdx.x;
  const int c_base = blockIdx.x * QC;          // first column (relative to m0) of this CTA
  const int npad = ((n + 63) / 64) * 64;
  T* Y = ywork + (long)blockIdx.x * npad * QC; // this CTA's y, [npad][QC]
  const int r = tid / 4, cg = tid % 4;          // thread owns row r of the block, columns 2cg, 2cg+1
  T wacc[2] = {N::zero(), N::zero()};
  double oacc[2] = {0.0, 0.0};
  const int nblk = (n + 63) / 64;
  for (int ib = 0; ib < nblk; ++ib) {
    const int i0 = ib * 64;
    T t[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      int c = cg * 2 + u, col = c_base + c;
      int row = i0 + r;
      if (row < n && col < n_cols) {
        const int cs = col / cols_per_state, cm = col % cols_per_state;
        double ov = ld_as<double>(O, dtype, cs * o_state_stride + (long)row * ld_o + cm);
        oacc[u] += ov * ov;
        t[u] = mkT(ov, (T*)nullptr);
      } else {
        t[u] = N::zero();
      }
    }
    for (int k0 = 0; k0 < i0; k0 += QK) {
      for (int e = tid; e < 64 * QK; e += 256) {
        int rr = e / QK, kk = e % QK;
        int row = i0 + rr, col = k0 + kk;
        Ls[rr][kk] = (row < n) ? L[(long)row * n + col] : N::zero();
      }
      for (int e = tid; e < QK * QC; e += 256) {
        int kk = e / QC, c = e % QC;
        Ys[kk][c] = Y[(long)(k0 + kk) * QC + c];
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < QK; ++kk) {
        T lv = Ls[r][kk];
        t[0] = N::fms(lv, Ys[kk][cg * 2 + 0], t[0]);
        t[1] = N::fms(lv, Ys[kk][cg * 2 + 1], t[1]);
      }
      __syncthreads();
    }
    Ts[r][cg * 2 + 0] = t[0];
    Ts[r][cg * 2 + 1] = t[1];
    __syncthreads();
    // y_i = Linv_ii t_i  (unit lower 64 x 64)
    const T* X = linv + (long)ib * 64 * 64;
    T y[2] = {N::zero(), N::zero()};
    for (int c = 0; c <= r; ++c) {
      T xv = X[r * 64 + c];
      y[0] = N::fma_(xv, Ts[c][cg * 2 + 0], y[0]);
      y[1] = N::fma_(xv, Ts[c][cg * 2 + 1], y[1]);
    }
    const int row = i0 + r;
    if (row < n) {
      T di = dinv[row];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        Y[(long)row * QC + cg * 2 + u] = y[u];
        wacc[u] = N::fma_(N::mul(y[u], y[u]), di, wacc[u]);
      }
    } else {
#pragma unroll
      for (int u = 0; u < 2; ++u) Y[(long)row * QC + cg * 2 + u] = N::zero();
    }
    __syncthreads();
  }
  // reduce over the 64 rows for each of the QC columns: thread (r, cg) holds columns 2cg, 2cg+1
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    red[tid] = wacc[u];
    ored[tid] = oacc[u];
    __syncthreads();
    for (int s = 128; s >= 4; s >>= 1) {   // tid = 4 r + cg: partners differ in r
      if (tid < s) {
        red[tid] = N::add(red[tid], red[tid + s]);
        ored[tid] += ored[tid + s];
      }
      __syncthreads();
    }
    if (tid < 4) {
      int col = c_base + tid * 2 + u;
      if (col < n_cols) {
        const int cs = col / cols_per_state, cm = col % cols_per_state;
        W_out[cs * w_state_stride + cm] = N::sub(red[tid], mkT(ored[tid], (T*)nullptr));
      }
    }
    __syncthreads();
  }
}

// Two right-hand sides per column: y = L^-1 o, u = L^-1 v, W = sum_P y_P u_P / d_P  (real case).
__global__ void __launch_bounds__(256) quadform_pi_kernel(const double* __restrict__ L, const double* __restrict__ dinv,
                                                          const double* __restrict__ linv, int n, const void* O,
                                                          int dtype, const double* __restrict__ V,
                                                          long o_state_stride, long ld_o, int cols_per_state,
                                                          int n_cols, double* ywork, double* W_out,
                                                          long w_state_stride) {
  __shared__ double Ls[64][QK + 1];
  __shared__ double Ys[QK][2 * QC];
  __shared__ double Ts[64][2 * QC];
  __shared__ double red[256];
  const int tid = threadIdx.x;
  const int c_base = blockIdx.x * QC;
  const int npad = ((n + 63) / 64) * 64;
  double* Y = ywork + (long)blockIdx.x * npad * 2 * QC;   // [npad][2 QC]: columns 0..QC-1 y, QC..2QC-1 u
  const int r = tid / 4, cg = tid % 4;
  double wacc[2] = {0.0, 0.0};
  const int nblk = (n + 63) / 64;
  for (int ib = 0; ib < nblk; ++ib) {
    const int i0 = ib * 64;
    double t[4];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      int col = c_base + cg * 2 + u;
      int row = i0 + r;
      t[u] = 0.0;
      t[2 + u] = 0.0;
      if (row < n && col < n_cols) {
        const int cs = col / cols_per_state, cm = col % cols_per_state;
        const long off = cs * o_state_stride + (long)row * ld_o + cm;
        t[u] = ld_as<double>(O, dtype, off);
        t[2 + u] = V[off];
      }
    }
    for (int k0 = 0; k0 < i0; k0 += QK) {
      for (int e = tid; e < 64 * QK; e += 256) {
        int rr = e / QK, kk = e % QK;
        int row = i0 + rr;
        Ls[rr][kk] = (row < n) ? L[(long)row * n + k0 + kk] : 0.0;
      }
      for (int e = tid; e < QK * 2 * QC; e += 256) {
        int kk = e / (2 * QC), c = e % (2 * QC);
        Ys[kk][c] = Y[(long)(k0 + kk) * 2 * QC + c];
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < QK; ++kk) {
        double lv = Ls[r][kk];
        t[0] = fma(-lv, Ys[kk][cg * 2 + 0], t[0]);
        t[1] = fma(-lv, Ys[kk][cg * 2 + 1], t[1]);
        t[2] = fma(-lv, Ys[kk][QC + cg * 2 + 0], t[2]);
        t[3] = fma(-lv, Ys[kk][QC + cg * 2 + 1], t[3]);
      }
      __syncthreads();
    }
    Ts[r][cg * 2 + 0] = t[0];
    Ts[r][cg * 2 + 1] = t[1];
    Ts[r][QC + cg * 2 + 0] = t[2];
    Ts[r][QC + cg * 2 + 1] = t[3];
    __syncthreads();
    const double* X = linv + (long)ib * 64 * 64;
    double y[4] = {0.0, 0.0, 0.0, 0.0};
    for (int c = 0; c <= r; ++c) {
      double xv = X[r * 64 + c];
      y[0] = fma(xv, Ts[c][cg * 2 + 0], y[0]);
      y[1] = fma(xv, Ts[c][cg * 2 + 1], y[1]);
      y[2] = fma(xv, Ts[c][QC + cg * 2 + 0], y[2]);
      y[3] = fma(xv, Ts[c][QC + cg * 2 + 1], y[3]);
    }
    const int row = i0 + r;
    if (row < n) {
      double di = dinv[row];
      wacc[0] = fma(y[0] * y[2], di, wacc[0]);
      wacc[1] = fma(y[1] * y[3], di, wacc[1]);
    } else {
      y[0] = y[1] = y[2] = y[3] = 0.0;
    }
    Y[(long)row * 2 * QC + cg * 2 + 0] = y[0];
    Y[(long)row * 2 * QC + cg * 2 + 1] = y[1];
    Y[(long)row * 2 * QC + QC + cg * 2 + 0] = y[2];
    Y[(long)row * 2 * QC + QC + cg * 2 + 1] = y[3];
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    red[tid] = wacc[u];
    __syncthreads();
    for (int s = 128; s >= 4; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    if (tid < 4) {
      int col = c_base + tid * 2 + u;
      if (col < n_cols) {
        const int cs = col / cols_per_state, cm = col % cols_per_state;
        W_out[cs * w_state_stride + cm] = red[tid];
      }
    }
    __syncthreads();
  }
}

}  // namespace

cdwac_status ldlt_quadform_pi(cdwac_ctx* ctx, const double* L, const double* dinv, const double* linv_blocks, int n,
                              const void* O, int dtype, const double* V, long o_state_stride, long ld_o, int n_states,
                              int cols_per_state, double* W_out, long w_state_stride, double* ywork, cudaStream_t st) {
  const int n_cols = n_states * cols_per_state;
  if (n_cols <= 0) return CDWAC_OK;
  quadform_pi_kernel<<<ceil_div(n_cols, QC), 256, 0, st>>>(L, dinv, linv_blocks, n, O, dtype, V, o_state_stride,
                                                            ld_o, cols_per_state, n_cols, ywork, W_out,
                                                            w_state_stride);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

template <class T>
size_t ldlt_scratch_elems(int n) {
  int nblk = (n + NB - 1) / NB;
  return (size_t)n /*dinv*/ + (size_t)nblk * NB * NB /*linv*/ + 2 * (size_t)(nblk + 1) * NB * NB /*2 panels*/;
}

// Lookahead schedule on two streams (when the context owns a side stream): after panel k, the critical-path
// stream (high priority, forked from and joined back to the caller's stream) updates only the next block column,
// factors the next diagonal block and builds the next panel, while the side stream (lowest priority) updates the
// rest of the trailing matrix; the following step waits for both.  The panel buffer is
// double-buffered because the side stream still reads panel k while panel k+1 is written.
template <class T>
static cdwac_status ldlt_factor_lookahead(cdwac_ctx* ctx, T* A, int n, T* dinv, T* linv_blocks, T* wpanel,
                                          cudaStream_t st, size_t dsmem, size_t psmem, const OzakiPlan* oz) {
  const int nblk = (n + NB - 1) / NB;
  T* wp[2] = {wpanel, wpanel + (size_t)(nblk + 1) * NB * NB};
  cudaStream_t side = ctx->side_stream;
  const cudaStream_t caller = st;
  if (ctx->crit_stream) {   // the critical path moves to the high-priority stream, joined back at the end
    st = ctx->crit_stream;
    CDWAC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_crit_in, caller));
    CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_crit_in, 0));
  }
  {
    ProfScope ps(ctx, PROF_LDLT_DIAG, st, 2);
    diag_kernel<T><<<1, 256, dsmem, st>>>(A, n, 0, dinv, ctx->d_status);
    CDWAC_LAUNCH_CHECK(ctx);
  }
  // Step kb: panel kb (overlaps the side stream's update kb-1), then wait for that update (it touched block
  // column kb+1), hand the bulk of update kb to the side stream, and update column kb+1 / factor block kb+1 here.
  bool bulk_pending = false;
  for (int kb = 0; kb < nblk - 1; ++kb) {
    const int k0 = kb * NB, rest = n - (k0 + NB), m = ceil_div(rest, 64);
    T* w = wp[kb & 1];
    cdwac_status rc;
    {
      ProfScope ps(ctx, PROF_LDLT_PANEL, st, 2);
      panel_kernel<T><<<ceil_div(rest, PR), PT, psmem, st>>>(A, n, k0, dinv, w);
      CDWAC_LAUNCH_CHECK(ctx);
    }
    if (oz) {
      // digit planes of this step (double-buffered like the panel: the side stream may still read step kb - 1)
      ProfScope pss(ctx, PROF_LDLT_SLICE, st, 2);
      if ((rc = ozaki_slice<T>(ctx, *oz, kb & 1, A, n, k0, w, st))) return rc;
    }
    if (bulk_pending) CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_bulk, 0));
    bulk_pending = false;
    if (m > 1) CDWAC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_panel, st));
    {
      // the next block column first: its CTAs are queued ahead of the bulk update's
      ProfScope ps(ctx, PROF_LDLT_UPDATE, st, 2);
      if (oz) {
        if ((rc = ozaki_update<T>(ctx, *oz, kb & 1, A, n, k0, 1, st))) return rc;
      } else {
        update_kernel<T><<<m, 256, 0, st>>>(A, n, k0, w, 1);
        CDWAC_LAUNCH_CHECK(ctx);
      }
    }
    if (m > 1) {
      CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(side, ctx->ev_panel, 0));
      if (oz) {
        if ((rc = ozaki_update<T>(ctx, *oz, kb & 1, A, n, k0, 2, side))) return rc;
      } else {
        update_kernel<T><<<m * (m - 1) / 2, 256, 0, side>>>(A, n, k0, w, 2);
        CDWAC_LAUNCH_CHECK(ctx);
      }
      CDWAC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_bulk, side));
      bulk_pending = true;
    }
    {
      ProfScope ps(ctx, PROF_LDLT_DIAG, st, 2);
      diag_kernel<T><<<1, 256, dsmem, st>>>(A, n, k0 + NB, dinv, ctx->d_status);
      CDWAC_LAUNCH_CHECK(ctx);
    }
  }
  if (bulk_pending) CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->ev_bulk, 0));
  if (st != caller) {
    CDWAC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_crit_out, st));
    CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(caller, ctx->ev_crit_out, 0));
  }
  return CDWAC_OK;
}

size_t ldlt_tc_scratch_bytes(int n, bool cplx) { return ozaki_scratch_bytes(n, cplx); }

// Inverses of every diagonal block at once (needed by the solves, not by the factorisation itself).
template <class T>
static cdwac_status launch_inverses(cdwac_ctx* ctx, const T* A, int n, T* linv_blocks, size_t ismem, cudaStream_t st) {
  ProfScope ps(ctx, PROF_LDLT_DIAG, st, 2);
  inverse_kernel<T><<<ceil_div(n, NB), 256, ismem, st>>>(A, n, linv_blocks);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

template <class T>
cdwac_status ldlt_factor(cdwac_ctx* ctx, T* A, int n, T* dinv, T* linv_blocks, T* wpanel, cudaStream_t st,
                         void* oz_scratch) {
  const size_t dsmem = (size_t)NB * SD * sizeof(T);
  const size_t psmem = (size_t)(NB * SD + NB * (PR + 1)) * sizeof(T);
  const size_t ismem = 2 * (size_t)NB * NB * sizeof(T);
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem));
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem));
  OzakiPlan plan;
  const OzakiPlan* oz = nullptr;
  if (oz_scratch && n > NB) {
    cdwac_status rc = ozaki_plan(ctx, oz_scratch, n, sizeof(T) == sizeof(cplx), &plan);
    if (rc) return rc;
    oz = &plan;
  }
  if (ctx->side_stream && ctx->ev_panel && ctx->ev_bulk) {
    cdwac_status rc = ldlt_factor_lookahead<T>(ctx, A, n, dinv, linv_blocks, wpanel, st, dsmem, psmem, oz);
    if (rc) return rc;
    return launch_inverses<T>(ctx, A, n, linv_blocks, ismem, st);
  }
  for (int k0 = 0; k0 < n; k0 += NB) {
    {
      ProfScope ps(ctx, PROF_LDLT_DIAG, st, 2);
      diag_kernel<T><<<1, 256, dsmem, st>>>(A, n, k0, dinv, ctx->d_status);
      CDWAC_LAUNCH_CHECK(ctx);
    }
    int rest = n - (k0 + NB);
    if (rest <= 0) break;
    int rblk = ceil_div(rest, 64);
    {
      ProfScope ps(ctx, PROF_LDLT_PANEL, st, 2);
      panel_kernel<T><<<ceil_div(rest, PR), PT, psmem, st>>>(A, n, k0, dinv, wpanel);
      CDWAC_LAUNCH_CHECK(ctx);
    }
    if (oz) {
      cdwac_status rc;
      {
        ProfScope pss(ctx, PROF_LDLT_SLICE, st, 2);
        if ((rc = ozaki_slice<T>(ctx, *oz, 0, A, n, k0, wpanel, st))) return rc;
      }
      ProfScope ps(ctx, PROF_LDLT_UPDATE, st, 2);
      if ((rc = ozaki_update<T>(ctx, *oz, 0, A, n, k0, 0, st))) return rc;
    } else {
      ProfScope ps(ctx, PROF_LDLT_UPDATE, st, 2);
      update_kernel<T><<<rblk * (rblk + 1) / 2, 256, 0, st>>>(A, n, k0, wpanel, 0);
      CDWAC_LAUNCH_CHECK(ctx);
    }
  }
  return launch_inverses<T>(ctx, A, n, linv_blocks, ismem, st);
}

template <class T>
size_t quadform_scratch_elems(int n, int n_cols) {
  int blocks = (n_cols + QC - 1) / QC;
  int npad = ((n + 63) / 64) * 64;
  return (size_t)blocks * npad * QC;
}

template <class T>
cdwac_status ldlt_quadform(cdwac_ctx* ctx, const T* L, const T* dinv, const T* linv_blocks, int n, const void* O,
                           int dtype, long o_state_stride, long ld_o, int n_states, int cols_per_state, T* W_out,
                           long w_state_stride, T* ywork, cudaStream_t st) {
  const int n_cols = n_states * cols_per_state;
  if (n_cols <= 0) return CDWAC_OK;
  int blocks = ceil_div(n_cols, QC);
  quadform_kernel<T><<<blocks, 256, 0, st>>>(L, dinv, linv_blocks, n, O, dtype, o_state_stride, ld_o,
                                             cols_per_state, n_cols, ywork, W_out, w_state_stride);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

template size_t ldlt_scratch_elems<double>(int);
template size_t ldlt_scratch_elems<cplx>(int);
template size_t quadform_scratch_elems<double>(int, int);
template size_t quadform_scratch_elems<cplx>(int, int);
template cdwac_status ldlt_factor<double>(cdwac_ctx*, double*, int, double*, double*, double*, cudaStream_t, void*);
template cdwac_status ldlt_factor<cplx>(cdwac_ctx*, cplx*, int, cplx*, cplx*, cplx*, cudaStream_t, void*);
template cdwac_status ldlt_quadform<double>(cdwac_ctx*, const double*, const double*, const double*, int,
                                            const void*, int, long, long, int, int, double*, long, double*,
                                            cudaStream_t);
template cdwac_status ldlt_quadform<cplx>(cdwac_ctx*, const cplx*, const cplx*, const cplx*, int, const void*, int,
                                          long, long, int, int, cplx*, long, cplx*, cudaStream_t);
