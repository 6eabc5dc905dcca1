// Mixed-precision W projection on the CUDA cores (FP32), for the imaginary axis:
//   W_nm = o^T (I - Pi)^-1 Pi o = sum_P y_P u_P / d_P,   y = L^-1 o,   u = L^-1 (Pi o)      (Eqs. wriv, bigLambda)
// with L D L^T = I - Pi the FP64 factor.  The (I - Pi)^-1 Pi form keeps the small W at large xi to relative
// accuracy; the products and the forward substitutions run in FP32 (the tensor-core Pi already carries ~1e-5
// relative error), the sum over P in FP64.
#include "common.cuh"

namespace {

constexpr int TM = 64, TK = 16;

// V[s][P][m] = sum_Q Pi_PQ O[s][Q][m], Pi_PQ = -negpi[P][Q] (full symmetric -Pi, FP32)
template <class TIn>
__global__ void __launch_bounds__(256) symm_f32_kernel(const float* __restrict__ negpi, int n, const TIn* __restrict__ O,
                                                       long o_state_stride, long ld_o, int cols_per_state,
                                                       int n_cols, float* __restrict__ V) {
  __shared__ __align__(16) float Ps[TK][TM];
  __shared__ __align__(16) float Os[TK][TM];
  const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TM;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float acc[4][4] = {};
  for (int q0 = 0; q0 < n; q0 += TK) {
    for (int e = tid; e < TK * TM; e += 256) {
      // Pi is symmetric: read row Q (consecutive threads -> consecutive P) to keep the loads coalesced
      const int qq = e / TM, r = e % TM;
      const int P = row0 + r, Q = q0 + qq;
      Ps[qq][r] = (P < n && Q < n) ? -negpi[(long)Q * n + P] : 0.f;
      const int c = col0 + r;
      float ov = 0.f;
      if (c < n_cols && Q < n) {
        const int cs = c / cols_per_state, cm = c % cols_per_state;
        ov = (float)O[cs * o_state_stride + (long)Q * ld_o + cm];
      }
      Os[qq][r] = ov;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TK; ++q) {
      const float4 a = *reinterpret_cast<const float4*>(&Ps[q][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Os[q][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
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
        V[(long)cs * n * cols_per_state + (long)P * cols_per_state + cm] = acc[i][j];
      }
    }
  }
}

// lower triangle of the FP64 factor (unit diagonal implied) -> FP32, and the diagonal-block inverses -> FP32
__global__ void factor_to_f32_kernel(const double* __restrict__ L, int n, const double* __restrict__ linv, int nblk,
                                     float* __restrict__ L32, float* __restrict__ linv32) {
  const long total = (long)n * n, tl = (long)nblk * 64 * 64;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total + tl; e += (long)gridDim.x * blockDim.x) {
    if (e < total) {
      const long r = e / n, c = e % n;
      if (c < r) L32[e] = (float)L[e];
    } else {
      linv32[e - total] = (float)linv[e - total];
    }
  }
}

constexpr int QC = 8, QK = 32;

// One CTA per QC columns: forward substitution for o and v = Pi o together, W = sum y u / d in FP64.
template <class TIn>
__global__ void __launch_bounds__(256) quadform_f32_kernel(const float* __restrict__ L32, const double* __restrict__ dinv,
                                                           const float* __restrict__ linv32, int n, const TIn* O,
                                                           const float* __restrict__ V, long o_state_stride, long ld_o,
                                                           int cols_per_state, int n_cols, float* ywork, double* W_out,
                                                           long w_state_stride) {
  __shared__ float Ls[64][QK + 1];
  __shared__ float Ys[QK][2 * QC];
  __shared__ float Ts[64][2 * QC];
  __shared__ double red[256];
  const int tid = threadIdx.x;
  const int c_base = blockIdx.x * QC;
  const int npad = ((n + 63) / 64) * 64;
  float* Y = ywork + (long)blockIdx.x * npad * 2 * QC;
  const int r = tid / 4, cg = tid % 4;
  double wacc[2] = {0.0, 0.0};
  const int nblk = (n + 63) / 64;
  for (int ib = 0; ib < nblk; ++ib) {
    const int i0 = ib * 64;
    float t[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int col = c_base + cg * 2 + u, row = i0 + r;
      if (row < n && col < n_cols) {
        const int cs = col / cols_per_state, cm = col % cols_per_state;
        t[u] = (float)O[cs * o_state_stride + (long)row * ld_o + cm];
        t[2 + u] = V[(long)cs * n * cols_per_state + (long)row * cols_per_state + cm];
      }
    }
    for (int k0 = 0; k0 < i0; k0 += QK) {
      for (int e = tid; e < 64 * QK; e += 256) {
        const int rr = e / QK, kk = e % QK, row = i0 + rr;
        Ls[rr][kk] = (row < n) ? L32[(long)row * n + k0 + kk] : 0.f;
      }
      for (int e = tid; e < QK * 2 * QC; e += 256) {
        const int kk = e / (2 * QC), c = e % (2 * QC);
        Ys[kk][c] = Y[(long)(k0 + kk) * 2 * QC + c];
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < QK; ++kk) {
        const float lv = Ls[r][kk];
        t[0] = fmaf(-lv, Ys[kk][cg * 2 + 0], t[0]);
        t[1] = fmaf(-lv, Ys[kk][cg * 2 + 1], t[1]);
        t[2] = fmaf(-lv, Ys[kk][QC + cg * 2 + 0], t[2]);
        t[3] = fmaf(-lv, Ys[kk][QC + cg * 2 + 1], t[3]);
      }
      __syncthreads();
    }
    Ts[r][cg * 2 + 0] = t[0];
    Ts[r][cg * 2 + 1] = t[1];
    Ts[r][QC + cg * 2 + 0] = t[2];
    Ts[r][QC + cg * 2 + 1] = t[3];
    __syncthreads();
    const float* X = linv32 + (long)ib * 64 * 64;
    float y[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c = 0; c <= r; ++c) {
      const float xv = X[r * 64 + c];
      y[0] = fmaf(xv, Ts[c][cg * 2 + 0], y[0]);
      y[1] = fmaf(xv, Ts[c][cg * 2 + 1], y[1]);
      y[2] = fmaf(xv, Ts[c][QC + cg * 2 + 0], y[2]);
      y[3] = fmaf(xv, Ts[c][QC + cg * 2 + 1], y[3]);
    }
    const int row = i0 + r;
    if (row < n) {
      const double di = dinv[row];
      wacc[0] += (double)y[0] * (double)y[2] * di;
      wacc[1] += (double)y[1] * (double)y[3] * di;
    } else {
      y[0] = y[1] = y[2] = y[3] = 0.f;
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
      const int col = c_base + tid * 2 + u;
      if (col < n_cols) {
        const int cs = col / cols_per_state, cm = col % cols_per_state;
        W_out[cs * w_state_stride + cm] = red[tid];
      }
    }
    __syncthreads();
  }
}

// ---- complex symmetric case (near-real points, residues): W = sum_P y_P^2 / d_P - sum_P o_P^2, y = L^-1 o ------
// W is O(1) there, so the single-solve form has no cancellation; FP32 complex arithmetic, FP64 sums.
struct c32 {
  float x, y;
};
__device__ inline c32 c32fms(c32 a, c32 b, c32 c) {   // c - a b
  return {fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y))};
}
__device__ inline c32 c32fma(c32 a, c32 b, c32 c) {   // c + a b
  return {fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y))};
}

__global__ void cfactor_to_c32_kernel(const cplx* __restrict__ L, int n, const cplx* __restrict__ linv, int nblk,
                                      c32* __restrict__ L32, c32* __restrict__ linv32) {
  const long total = (long)n * n, tl = (long)nblk * 64 * 64;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total + tl; e += (long)gridDim.x * blockDim.x) {
    if (e < total) {
      const long r = e / n, c = e % n;
      if (c < r) L32[e] = {(float)L[e].x, (float)L[e].y};
    } else {
      const cplx v = linv[e - total];
      linv32[e - total] = {(float)v.x, (float)v.y};
    }
  }
}

constexpr int QCC = 2, QKC = 32;   // columns per CTA (128 threads = 64 rows x 2 columns), K chunk

template <class TIn>
__global__ void __launch_bounds__(128) cquadform_c32_kernel(const c32* __restrict__ L32, const cplx* __restrict__ dinv,
                                                            const c32* __restrict__ linv32, int n, const TIn* O,
                                                            long o_state_stride, long ld_o, int cols_per_state,
                                                            int n_cols, c32* ywork, cplx* W_out, long w_state_stride) {
  __shared__ c32 Ls[64][QKC + 1];
  __shared__ c32 Ys[QKC][QCC];
  __shared__ c32 Ts[64][QCC];
  __shared__ double rr_[128], ri_[128], ro_[128];
  const int tid = threadIdx.x, r = tid / QCC, cc = tid % QCC;
  const int col = blockIdx.x * QCC + cc;
  const int npad = ((n + 63) / 64) * 64;
  c32* Y = ywork + (long)blockIdx.x * npad * QCC;
  double wr = 0.0, wi = 0.0, oo = 0.0;
  const int nblk = (n + 63) / 64;
  int cs = 0, cm = 0;
  if (col < n_cols) {
    cs = col / cols_per_state;
    cm = col % cols_per_state;
  }
  for (int ib = 0; ib < nblk; ++ib) {
    const int i0 = ib * 64, row = i0 + r;
    c32 t = {0.f, 0.f};
    if (row < n && col < n_cols) {
      const double ov = (double)O[cs * o_state_stride + (long)row * ld_o + cm];
      oo += ov * ov;
      t.x = (float)ov;
    }
    for (int k0 = 0; k0 < i0; k0 += QKC) {
      for (int e = tid; e < 64 * QKC; e += 128) {
        const int rr = e / QKC, kk = e % QKC, lr = i0 + rr;
        Ls[rr][kk] = (lr < n) ? L32[(long)lr * n + k0 + kk] : c32{0.f, 0.f};
      }
      if (tid < QKC * QCC) Ys[tid / QCC][tid % QCC] = Y[(long)(k0 + tid / QCC) * QCC + tid % QCC];
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < QKC; ++kk) t = c32fms(Ls[r][kk], Ys[kk][cc], t);
      __syncthreads();
    }
    Ts[r][cc] = t;
    __syncthreads();
    const c32* X = linv32 + (long)ib * 64 * 64;
    c32 y = {0.f, 0.f};
    for (int c = 0; c <= r; ++c) y = c32fma(X[r * 64 + c], Ts[c][cc], y);
    if (row < n) {
      const cplx di = dinv[row];
      const double yr = y.x, yi = y.y;
      const double sr = yr * yr - yi * yi, si = 2.0 * yr * yi;     // y^2
      wr += sr * di.x - si * di.y;
      wi += sr * di.y + si * di.x;
    } else {
      y = {0.f, 0.f};
    }
    Y[(long)row * QCC + cc] = y;
    __syncthreads();
  }
  rr_[tid] = wr;
  ri_[tid] = wi;
  ro_[tid] = oo;
  __syncthreads();
  for (int s = 64; s >= QCC; s >>= 1) {
    if (tid < s) {
      rr_[tid] += rr_[tid + s];
      ri_[tid] += ri_[tid + s];
      ro_[tid] += ro_[tid + s];
    }
    __syncthreads();
  }
  if (tid < QCC) {
    const int c = blockIdx.x * QCC + tid;
    if (c < n_cols) {
      const int s2 = c / cols_per_state, m2 = c % cols_per_state;
      W_out[s2 * w_state_stride + m2] = mkc(rr_[tid] - ro_[tid], ri_[tid]);
    }
  }
}

}  // namespace

size_t wsolve_c32_scratch_bytes(int n, int n_cols) {
  const int nblk = (n + 63) / 64, npad = nblk * 64, blocks = (n_cols + QCC - 1) / QCC;
  return sizeof(c32) * ((size_t)n * n + (size_t)nblk * 4096 + (size_t)blocks * npad * QCC) + 3 * 256;
}

cdwac_status wsolve_c32(cdwac_ctx* ctx, const cplx* L, const cplx* dinv, const cplx* linv, int n, const void* O,
                        int dtype, long o_state_stride, long ld_o, int n_states, int cols_per_state, cplx* W_out,
                        long w_state_stride, void* scratch, cudaStream_t st) {
  const int n_cols = n_states * cols_per_state;
  if (n_cols <= 0) return CDWAC_OK;
  const int nblk = (n + 63) / 64;
  Arena ar(scratch);
  c32* L32 = ar.take<c32>((size_t)n * n);
  c32* linv32 = ar.take<c32>((size_t)nblk * 4096);
  c32* Y = ar.take<c32>((size_t)((n_cols + QCC - 1) / QCC) * nblk * 64 * QCC);
  {
    long total = (long)n * n + (long)nblk * 4096;
    int blocks = (int)std::min<long>((total + 255) / 256, (long)ctx->num_sms * 16);
    cfactor_to_c32_kernel<<<blocks, 256, 0, st>>>(L, n, linv, nblk, L32, linv32);
    CDWAC_LAUNCH_CHECK(ctx);
  }
  const int qb = ceil_div(n_cols, QCC);
  if (dtype == CDWAC_F64)
    cquadform_c32_kernel<double><<<qb, 128, 0, st>>>(L32, dinv, linv32, n, (const double*)O, o_state_stride, ld_o,
                                                     cols_per_state, n_cols, Y, W_out, w_state_stride);
  else
    cquadform_c32_kernel<float><<<qb, 128, 0, st>>>(L32, dinv, linv32, n, (const float*)O, o_state_stride, ld_o,
                                                    cols_per_state, n_cols, Y, W_out, w_state_stride);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

size_t wsolve32_scratch_bytes(int n, int n_cols) {
  const int nblk = (n + 63) / 64, npad = nblk * 64, blocks = (n_cols + QC - 1) / QC;
  return sizeof(float) * ((size_t)n * n /*L32*/ + (size_t)nblk * 4096 /*linv32*/ + (size_t)n * n_cols /*V*/ +
                          (size_t)blocks * npad * 2 * QC /*ywork*/) +
         4 * 256;
}

cdwac_status wsolve32(cdwac_ctx* ctx, const double* L, const double* dinv, const double* linv, const float* negpi32,
                      int n, const void* O, int dtype, long o_state_stride, long ld_o, int n_states,
                      int cols_per_state, double* W_out, long w_state_stride, void* scratch, cudaStream_t st) {
  const int n_cols = n_states * cols_per_state;
  if (n_cols <= 0) return CDWAC_OK;
  const int nblk = (n + 63) / 64;
  Arena ar(scratch);
  float* L32 = ar.take<float>((size_t)n * n);
  float* linv32 = ar.take<float>((size_t)nblk * 4096);
  float* V = ar.take<float>((size_t)n * n_cols);
  float* Y = ar.take<float>((size_t)((n_cols + QC - 1) / QC) * nblk * 64 * 2 * QC);
  {
    long total = (long)n * n + (long)nblk * 4096;
    int blocks = (int)std::min<long>((total + 255) / 256, (long)ctx->num_sms * 16);
    factor_to_f32_kernel<<<blocks, 256, 0, st>>>(L, n, linv, nblk, L32, linv32);
    CDWAC_LAUNCH_CHECK(ctx);
  }
  dim3 grid(ceil_div(n_cols, TM), ceil_div(n, TM));
  if (dtype == CDWAC_F64)
    symm_f32_kernel<double><<<grid, 256, 0, st>>>(negpi32, n, (const double*)O, o_state_stride, ld_o, cols_per_state,
                                                  n_cols, V);
  else
    symm_f32_kernel<float><<<grid, 256, 0, st>>>(negpi32, n, (const float*)O, o_state_stride, ld_o, cols_per_state,
                                                 n_cols, V);
  CDWAC_LAUNCH_CHECK(ctx);
  const int qb = ceil_div(n_cols, QC);
  if (dtype == CDWAC_F64)
    quadform_f32_kernel<double><<<qb, 256, 0, st>>>(L32, dinv, linv32, n, (const double*)O, V, o_state_stride, ld_o,
                                                    cols_per_state, n_cols, Y, W_out, w_state_stride);
  else
    quadform_f32_kernel<float><<<qb, 256, 0, st>>>(L32, dinv, linv32, n, (const float*)O, V, o_state_stride, ld_o,
                                                   cols_per_state, n_cols, Y, W_out, w_state_stride);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}
