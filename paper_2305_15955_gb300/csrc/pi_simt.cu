// FP64 polarizability on the CUDA cores (the parity path): A = I - Pi(z), lower triangle only.
//
// Pi_PQ(z) = 2 sum_ia O^ia_P [1/(z - D_ia) - 1/(z + D_ia)] O^ia_Q   (Eq. piriv, closed-shell spin factor 2)
// On the imaginary axis z = i xi the weight is -4 D / (xi^2 + D^2) and A is real symmetric positive definite;
// for complex z the weight 4 D / (z^2 - D^2) is complex and A is complex symmetric.
//
// Tiling: 64 x 64 output tiles of the lower triangle, 256 threads with 4 x 4 outputs each, K staged through
// shared memory 16 columns at a time.  FP64 FMA throughput bounds this kernel on GB300, so the tile is
// chosen for simplicity; the mixed-precision path uses the tensor cores instead.
#include "common.cuh"

namespace {

constexpr int TM = 64, TK = 16, TPAD = TM + 1;

__device__ inline void lower_tile_coords(int b, int& ti, int& tj) {
  int t = int((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((t + 1) * (t + 2) / 2 <= b) ++t;
  while (t * (t + 1) / 2 > b) --t;
  ti = t;
  tj = b - t * (t + 1) / 2;
}

template <class TIn>
__device__ inline double ld(const TIn* p) { return (double)*p; }

// Real weight on the imaginary axis: A = I + 4 sum B B D/(xi^2 + D^2)
template <class TIn>
__global__ void __launch_bounds__(256) pi_imag_kernel(const TIn* __restrict__ B, const double* __restrict__ D,
                                                      int n_aux, int n_ov, const double* __restrict__ xi_dev,
                                                      double* __restrict__ A, double* __restrict__ pidiag) {
  const double xi2 = xi_dev[0] * xi_dev[0];
  __shared__ double As[TK][TPAD];
  __shared__ double Bs[TK][TPAD];
  __shared__ double wk[TK];
  int ti, tj;
  lower_tile_coords(blockIdx.x, ti, tj);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int row0 = ti * TM, col0 = tj * TM;
  double acc[4][4] = {};
  for (long k0 = 0; k0 < n_ov; k0 += TK) {
    if (tid < TK) {
      long k = k0 + tid;
      double d = (k < n_ov) ? D[k] : 1.0;
      wk[tid] = (k < n_ov) ? 4.0 * d / (xi2 + d * d) : 0.0;
    }
    __syncthreads();
    const int kk = tid % TK;
    const long k = k0 + kk;
    for (int r = tid / TK; r < TM; r += 256 / TK) {
      int pr = row0 + r, pc = col0 + r;
      double va = (pr < n_aux && k < n_ov) ? ld(B + (long)pr * n_ov + k) : 0.0;
      double vb = (pc < n_aux && k < n_ov) ? ld(B + (long)pc * n_ov + k) : 0.0;
      As[kk][r] = va * wk[kk];
      Bs[kk][r] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TK; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[q][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[q][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int P = row0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int Q = col0 + tx * 4 + j;
      if (P < n_aux && Q < n_aux && Q <= P) {
        A[(long)P * n_aux + Q] = (P == Q ? 1.0 : 0.0) + acc[i][j];
        if (P == Q) {
          if (pidiag) pidiag[P] = -acc[i][j];
        } else {
          A[(long)Q * n_aux + P] = acc[i][j];    // strict upper triangle keeps -Pi for the product Pi O
        }
      }
    }
  }
}

// V = Pi O for the columns of every state (FP64), with Pi read from the strict upper triangle of A (which the
// LDL^T factorisation leaves untouched: there A_PQ = -Pi_PQ) and from the separate diagonal pidiag.
// Output V[s][P][m], same layout as O_n.  Tiles of 64 rows x 64 columns, K staged 16 at a time.
template <class TIn>
__global__ void __launch_bounds__(256) pi_times_o_kernel(const double* __restrict__ A, const double* __restrict__ pidiag,
                                                         int n, const TIn* __restrict__ O, long o_state_stride,
                                                         long ld_o, int cols_per_state, int n_cols,
                                                         double* __restrict__ V) {
  __shared__ double Ps[TK][TPAD];
  __shared__ double Os[TK][TPAD];
  const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TM;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  double acc[4][4] = {};
  for (int q0 = 0; q0 < n; q0 += TK) {
    for (int e = tid; e < TK * TM; e += 256) {
      int r = e / TK, qq = e % TK;
      int P = row0 + r, Q = q0 + qq;
      double v = 0.0;
      if (P < n && Q < n) v = (P == Q) ? pidiag[P] : -A[(long)min(P, Q) * n + max(P, Q)];
      Ps[qq][r] = v;
      int c = col0 + r;
      double ov = 0.0;
      if (c < n_cols && Q < n) {
        int cs = c / cols_per_state, cm = c % cols_per_state;
        ov = (double)O[cs * o_state_stride + (long)Q * ld_o + cm];
      }
      Os[qq][r] = ov;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TK; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Ps[q][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Os[q][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int P = row0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = col0 + tx * 4 + j;
      if (P < n && c < n_cols) {
        int cs = c / cols_per_state, cm = c % cols_per_state;
        V[cs * o_state_stride + (long)P * ld_o + cm] = acc[i][j];
      }
    }
  }
}

// Complex weight: A = I - 4 sum B B D/(z^2 - D^2)
template <class TIn>
__global__ void __launch_bounds__(256) pi_complex_kernel(const TIn* __restrict__ B, const double* __restrict__ D,
                                                         int n_aux, int n_ov, const cplx* __restrict__ z_dev,
                                                         cplx* __restrict__ A) {
  const cplx z = z_dev[0];
  __shared__ double Ar[TK][TPAD];
  __shared__ double Ai[TK][TPAD];
  __shared__ double Bs[TK][TPAD];
  __shared__ cplx wk[TK];
  int ti, tj;
  lower_tile_coords(blockIdx.x, ti, tj);
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int row0 = ti * TM, col0 = tj * TM;
  double accr[4][4] = {}, acci[4][4] = {};
  const cplx z2 = z * z;
  for (long k0 = 0; k0 < n_ov; k0 += TK) {
    if (tid < TK) {
      long k = k0 + tid;
      if (k < n_ov) {
        double d = D[k];
        // 2 [1/(z - d) - 1/(z + d)] = 4 d / (z^2 - d^2); A takes minus this
        cplx w = mkc(-4.0 * d, 0.0) / (z2 - mkc(d * d, 0.0));
        wk[tid] = w;
      } else {
        wk[tid] = mkc(0.0, 0.0);
      }
    }
    __syncthreads();
    const int kk = tid % TK;
    const long k = k0 + kk;
    for (int r = tid / TK; r < TM; r += 256 / TK) {
      int pr = row0 + r, pc = col0 + r;
      double va = (pr < n_aux && k < n_ov) ? ld(B + (long)pr * n_ov + k) : 0.0;
      double vb = (pc < n_aux && k < n_ov) ? ld(B + (long)pc * n_ov + k) : 0.0;
      Ar[kk][r] = va * wk[kk].x;
      Ai[kk][r] = va * wk[kk].y;
      Bs[kk][r] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TK; ++q) {
      double ar[4], ai[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ar[i] = Ar[q][ty * 4 + i];
        ai[i] = Ai[q][ty * 4 + i];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[q][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accr[i][j] = fma(ar[i], b[j], accr[i][j]);
          acci[i][j] = fma(ai[i], b[j], acci[i][j]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int P = row0 + ty * 4 + i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int Q = col0 + tx * 4 + j;
      if (P < n_aux && Q < n_aux && Q <= P)
        A[(long)P * n_aux + Q] = mkc((P == Q ? 1.0 : 0.0) + accr[i][j], acci[i][j]);
    }
  }
}

}  // namespace

cdwac_status launch_pi_imag_fp64(cdwac_ctx* ctx, const void* B, int dtype, const double* D, int n_aux, int n_ov,
                                 const double* xi, double* A, double* pidiag, cudaStream_t st) {
  int nt = ceil_div(n_aux, TM);
  int blocks = nt * (nt + 1) / 2;
  if (dtype == CDWAC_F64)
    pi_imag_kernel<double><<<blocks, 256, 0, st>>>((const double*)B, D, n_aux, n_ov, xi, A, pidiag);
  else
    pi_imag_kernel<float><<<blocks, 256, 0, st>>>((const float*)B, D, n_aux, n_ov, xi, A, pidiag);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status launch_pi_times_o(cdwac_ctx* ctx, const double* A, const double* pidiag, int n, const void* O, int dtype,
                               long o_state_stride, long ld_o, int n_states, int cols_per_state, double* V,
                               cudaStream_t st) {
  const int n_cols = n_states * cols_per_state;
  dim3 grid(ceil_div(n_cols, TM), ceil_div(n, TM));
  if (dtype == CDWAC_F64)
    pi_times_o_kernel<double><<<grid, 256, 0, st>>>(A, pidiag, n, (const double*)O, o_state_stride, ld_o,
                                                    cols_per_state, n_cols, V);
  else
    pi_times_o_kernel<float><<<grid, 256, 0, st>>>(A, pidiag, n, (const float*)O, o_state_stride, ld_o,
                                                   cols_per_state, n_cols, V);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status launch_pi_complex_fp64(cdwac_ctx* ctx, const void* B, int dtype, const double* D, int n_aux,
                                    int n_ov, const cplx* z, cplx* A, cudaStream_t st) {
  int nt = ceil_div(n_aux, TM);
  int blocks = nt * (nt + 1) / 2;
  if (dtype == CDWAC_F64)
    pi_complex_kernel<double><<<blocks, 256, 0, st>>>((const double*)B, D, n_aux, n_ov, z, A);
  else
    pi_complex_kernel<float><<<blocks, 256, 0, st>>>((const float*)B, D, n_aux, n_ov, z, A);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}
