// Learned continuation of W: a pole-residue MLP (32 -> 3 x 256 GELU -> 16), trained and evaluated on the GPU.
//
// Input of one (n, m) pair: x_k = W_nm(i xi_{3k}) / s, k < 32, s = |W_nm(i xi_1)|.  Outputs o map to 8 poles
// Omega_s = softplus(o_s) + 0.05 Ha and residues r_s = softplus(o_{8+s}); the model is the sum-over-poles form
//   W(z) = -s sum_s r_s 2 Omega_s / (Omega_s^2 - z^2),
// which is <= 0 on the imaginary axis by construction (the pole form behind Eq. sigma_pole).  Training minimises
// mean_b (1/J) sum_j |W(z_j) - W_ref(z_j)|^2 / (s_b^2 + |W_ref(z_j)|^2) over reference points the method itself
// computed (the 32 imaginary nodes and the near-real points of Sec. 3.3).  FP32 training (tiled SIMT GEMMs,
// exact-erf GELU, Adam); inference reads BF16 copies of the weights with FP32 accumulation.
//
// Parameter layout (row-major weights [in][out], then the bias, per layer): 32x256, 256 | 256x256, 256 |
// 256x256, 256 | 256x16, 16  = CDWAC_MLP_NPARAMS floats.
#include <cuda_bf16.h>

#include "common.cuh"

namespace {

constexpr int NIN = CDWAC_MLP_IN, NH = CDWAC_MLP_HIDDEN, NP = CDWAC_MLP_POLES, NOUT = 2 * CDWAC_MLP_POLES;
constexpr float OMEGA_FLOOR = 0.05f;
constexpr int EVERY = 3;

struct Layer {
  int in, out;
  long w_off, b_off;
};
__host__ __device__ inline Layer layer(int l) {
  const int ins[4] = {NIN, NH, NH, NH}, outs[4] = {NH, NH, NH, NOUT};
  long off = 0;
  for (int i = 0; i < l; ++i) off += (long)ins[i] * outs[i] + outs[i];
  return {ins[l], outs[l], off, off + (long)ins[l] * outs[l]};
}

template <class T>
__device__ inline float ldf(const T* p, long i);
template <>
__device__ inline float ldf<float>(const float* p, long i) {
  return p[i];
}
template <>
__device__ inline float ldf<__nv_bfloat16>(const __nv_bfloat16* p, long i) {
  return __bfloat162float(p[i]);
}

// C[M][N] = op(A) op(B) (+ C if accumulate); A row-major [M][K] (or [K][M] if transA), B [K][N] (or [N][K]).
constexpr int GT = 64, GK = 16;
template <class TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                   int transA, const TB* __restrict__ B, int ldb, int transB,
                                                   float* __restrict__ C, int ldc, int accumulate) {
  __shared__ float As[GK][GT + 1];
  __shared__ float Bs[GK][GT + 1];
  const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = tid; e < GK * GT; e += 256) {
      int i, k;
      if (transA) {
        k = e / GT;
        i = e % GT;
      } else {
        i = e / GK;
        k = e % GK;
      }
      const int gi = row0 + i, gk = k0 + k;
      As[k][i] = (gi < M && gk < K) ? (transA ? A[(long)gk * lda + gi] : A[(long)gi * lda + gk]) : 0.f;
      int j, kb;
      if (transB) {
        j = e / GK;
        kb = e % GK;
      } else {
        kb = e / GT;
        j = e % GT;
      }
      const int gj = col0 + j, gkb = k0 + kb;
      Bs[kb][j] = (gj < N && gkb < K) ? (transB ? ldf(B, (long)gj * ldb + gkb) : ldf(B, (long)gkb * ldb + gj)) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[q][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[q][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = row0 + ty * 4 + r;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = col0 + tx * 4 + c;
      if (gi < M && gj < N) {
        float* p = C + (long)gi * ldc + gj;
        *p = accumulate ? *p + acc[r][c] : acc[r][c];
      }
    }
  }
}

__device__ inline float gelu(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }
__device__ inline float gelu_prime(float a) {
  return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}
__device__ inline double softplus(double y) { return fmax(y, 0.0) + log1p(exp(-fabs(y))); }
__device__ inline double sigmoid(double y) { return 1.0 / (1.0 + exp(-y)); }

// a[b][j] += bias[j]; if act: h = gelu(a)
template <class TB>
__global__ void bias_act_kernel(float* a, float* h, const TB* bias, int rows, int cols, int act) {
  const long total = (long)rows * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const float v = a[e] + ldf(bias, e % cols);
    a[e] = v;
    if (act) h[e] = gelu(v);
  }
}

__global__ void gelu_back_kernel(float* d, const float* a, long total) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x)
    d[e] *= gelu_prime(a[e]);
}

__global__ void colsum_kernel(const float* d, int rows, int cols, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += d[(long)r * cols + j];
  out[j] = s;
}

// per sample: poles from o, model at the reference points, loss share, dL/do
__global__ void head_loss_kernel(const float* o, const float* scale, int B, int J, const cplx* z_ref, const cplx* w_ref,
                                 float* d_o, double* loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double yo[NP], yr[NP], Om[NP], r[NP], dOm[NP] = {}, dr[NP] = {};
  for (int s = 0; s < NP; ++s) {
    yo[s] = o[(long)b * NOUT + s];
    yr[s] = o[(long)b * NOUT + NP + s];
    Om[s] = softplus(yo[s]) + OMEGA_FLOOR;
    r[s] = softplus(yr[s]);
  }
  const double sc = scale[b];
  double L = 0.0;
  for (int j = 0; j < J; ++j) {
    const cplx z = z_ref[(long)b * J + j];
    const cplx z2 = z * z;
    cplx W = mkc(0.0, 0.0);
    cplx g[NP], dg[NP];
    for (int s = 0; s < NP; ++s) {
      const cplx den = mkc(Om[s] * Om[s], 0.0) - z2;
      g[s] = mkc(2.0 * Om[s], 0.0) / den;
      dg[s] = mkc(-2.0, 0.0) * (mkc(Om[s] * Om[s], 0.0) + z2) / (den * den);
      W = W + r[s] * g[s];
    }
    W = (-sc) * W;
    const cplx wref = w_ref[(long)b * J + j];
    const cplx e = W - wref;
    const double wgt = 1.0 / (sc * sc + wref.x * wref.x + wref.y * wref.y);   // relative error, scale as floor
    L += (e.x * e.x + e.y * e.y) * wgt;
    const double c = 2.0 * wgt / ((double)J * B);
    for (int s = 0; s < NP; ++s) {
      // c Re(conj(e) dW/dp) with dW/dr = -s g, dW/dOmega = -s r dg
      const cplx wr = (-sc) * g[s], wo = (-sc * r[s]) * dg[s];
      dr[s] += c * (e.x * wr.x + e.y * wr.y);
      dOm[s] += c * (e.x * wo.x + e.y * wo.y);
    }
  }
  for (int s = 0; s < NP; ++s) {
    d_o[(long)b * NOUT + s] = (float)(dOm[s] * sigmoid(yo[s]));
    d_o[(long)b * NOUT + NP + s] = (float)(dr[s] * sigmoid(yr[s]));
  }
  atomicAdd(loss, L / ((double)J * B));
}

__global__ void poles_kernel(const float* o, const float* scale, int B, double* poles) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  for (int s = 0; s < NP; ++s) {
    poles[((long)b * NP + s) * 2 + 0] = softplus((double)o[(long)b * NOUT + s]) + OMEGA_FLOOR;
    poles[((long)b * NP + s) * 2 + 1] = softplus((double)o[(long)b * NOUT + NP + s]) * (double)scale[b];
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* p, __nv_bfloat16* q, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) q[i] = __float2bfloat16_rn(p[i]);
}

// features and targets of every (state s, occupied m) pair
__global__ void features_kernel(const double* xi, const double* W_imag, int n_states, int n_imag, int n_basis,
                                int n_occ, const cplx* z_real, const cplx* W_real, int n_real, float* x, float* scale,
                                cplx* z_ref, cplx* w_ref) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_states * n_occ) return;
  const int s = b / n_occ, m = b % n_occ;
  const double* W = W_imag + (long)s * n_imag * n_basis + m;
  const double sc = fabs(W[0]) > 0 ? fabs(W[0]) : 1.0;
  scale[b] = (float)sc;
  const int J = NIN + n_real;
  for (int k = 0; k < NIN; ++k) {
    const double v = W[(long)(k * EVERY) * n_basis];
    x[(long)b * NIN + k] = (float)(v / sc);
    z_ref[(long)b * J + k] = mkc(0.0, xi[k * EVERY]);
    w_ref[(long)b * J + k] = mkc(v, 0.0);
  }
  for (int j = 0; j < n_real; ++j) {
    z_ref[(long)b * J + NIN + j] = z_real[(long)s * n_real + j];
    w_ref[(long)b * J + NIN + j] = W_real[((long)s * n_real + j) * n_occ + m];
  }
}

int grid_for(cdwac_ctx* ctx, long n) {
  long b = (n + 255) / 256;
  long cap = (long)ctx->num_sms * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <class TB>
cdwac_status gemm(cdwac_ctx* ctx, int M, int N, int K, const float* A, int lda, int tA, const TB* B, int ldb, int tB,
                  float* C, int ldc, int acc, cudaStream_t st) {
  dim3 g(ceil_div(N, GT), ceil_div(M, GT));
  gemm_kernel<TB><<<g, 256, 0, st>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, acc);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

// forward pass; act[l] = pre-activation a_l, act[l] + B*NH = gelu(a_l) (l = 0..2), out = o [B][16]
template <class TW>
cdwac_status forward(cdwac_ctx* ctx, const TW* P, int B, const float* x, float* act, float* out, cudaStream_t st) {
  const float* h = x;
  cdwac_status rc;
  for (int l = 0; l < 4; ++l) {
    const Layer L = layer(l);
    float* a = (l < 3) ? act + (long)l * 2 * B * NH : out;
    float* hn = (l < 3) ? a + (long)B * NH : nullptr;
    if ((rc = gemm<TW>(ctx, B, L.out, L.in, h, L.in, 0, P + L.w_off, L.out, 0, a, L.out, 0, st))) return rc;
    bias_act_kernel<TW><<<grid_for(ctx, (long)B * L.out), 256, 0, st>>>(a, hn, P + L.b_off, B, L.out, l < 3);
    CDWAC_LAUNCH_CHECK(ctx);
    h = hn;
  }
  return CDWAC_OK;
}

}  // namespace

extern "C" {

cdwac_status cdwac_mlp_features(cdwac_ctx* ctx, const double* xi, const double* W_imag, int n_states, int n_imag,
                                int n_basis, int n_occ, const double* z_real, const double* W_real, int n_real,
                                float* x, float* scale, double* z_ref, double* w_ref, void* stream) {
  if (!ctx) return CDWAC_ERR_ARG;
  if (!xi || !W_imag || !x || !scale || !z_ref || !w_ref || n_states < 1 || n_occ < 1 || n_occ > n_basis ||
      n_imag < EVERY * (NIN - 1) + 1 || n_real < 0 || (n_real > 0 && (!z_real || !W_real)))
    return set_error(ctx, CDWAC_ERR_ARG, "bad mlp_features arguments (n_imag must be >= %d)", EVERY * (NIN - 1) + 1);
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const int B = n_states * n_occ;
  features_kernel<<<ceil_div(B, 128), 128, 0, (cudaStream_t)stream>>>(
      xi, W_imag, n_states, n_imag, n_basis, n_occ, reinterpret_cast<const cplx*>(z_real),
      reinterpret_cast<const cplx*>(W_real), n_real, x, scale, reinterpret_cast<cplx*>(z_ref),
      reinterpret_cast<cplx*>(w_ref));
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status cdwac_mlp_loss_grad(cdwac_ctx* ctx, const float* params, int batch, const float* x, const float* scale,
                                 int n_ref, const double* z_ref, const double* w_ref, float* grad, double* loss,
                                 void* stream) {
  if (!ctx) return CDWAC_ERR_ARG;
  if (!params || batch < 1 || !x || !scale || n_ref < 1 || !z_ref || !w_ref || !grad || !loss)
    return set_error(ctx, CDWAC_ERR_ARG, "bad mlp_loss_grad arguments");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int B = batch;
  const size_t bytes = sizeof(float) * ((size_t)6 * B * NH + (size_t)2 * B * NOUT + (size_t)2 * B * NH) + 4096;
  cdwac_status rc = ensure_scratch(ctx, bytes);
  if (rc) return rc;
  Arena ar(ctx->scratch);
  float* act = ar.take<float>((size_t)6 * B * NH);
  float* o = ar.take<float>((size_t)B * NOUT);
  float* d_o = ar.take<float>((size_t)B * NOUT);
  float* dA = ar.take<float>((size_t)B * NH);
  float* dB = ar.take<float>((size_t)B * NH);
  ProfScope ps(ctx, PROF_MLP, st);
  if ((rc = forward<float>(ctx, params, B, x, act, o, st))) return rc;
  CDWAC_CUDA_TRY(ctx, cudaMemsetAsync(loss, 0, sizeof(double), st));
  head_loss_kernel<<<ceil_div(B, 128), 128, 0, st>>>(o, scale, B, n_ref, reinterpret_cast<const cplx*>(z_ref),
                                                     reinterpret_cast<const cplx*>(w_ref), d_o, loss);
  CDWAC_LAUNCH_CHECK(ctx);
  // backward: d of the layer output in `cur` ([B][out]); h_in = input of the layer
  const float* cur = d_o;
  for (int l = 3; l >= 0; --l) {
    const Layer L = layer(l);
    const float* h_in = (l == 0) ? x : act + (long)(l - 1) * 2 * B * NH + (long)B * NH;
    if ((rc = gemm<float>(ctx, L.in, L.out, B, h_in, L.in, 1, cur, L.out, 0, grad + L.w_off, L.out, 0, st))) return rc;
    colsum_kernel<<<ceil_div(L.out, 128), 128, 0, st>>>(cur, B, L.out, grad + L.b_off);
    CDWAC_LAUNCH_CHECK(ctx);
    if (l == 0) break;
    float* nxt = (cur == dA) ? dB : dA;
    if ((rc = gemm<float>(ctx, B, L.in, L.out, cur, L.out, 0, params + L.w_off, L.out, 1, nxt, L.in, 0, st))) return rc;
    gelu_back_kernel<<<grid_for(ctx, (long)B * L.in), 256, 0, st>>>(nxt, act + (long)(l - 1) * 2 * B * NH,
                                                                      (long)B * L.in);
    CDWAC_LAUNCH_CHECK(ctx);
    cur = nxt;
  }
  return CDWAC_OK;
}

cdwac_status cdwac_mlp_adam(cdwac_ctx* ctx, float* params, const float* grad, float* m, float* v, int step, float lr,
                            float beta1, float beta2, float eps, void* stream) {
  if (!ctx) return CDWAC_ERR_ARG;
  if (!params || !grad || !m || !v || step < 1) return set_error(ctx, CDWAC_ERR_ARG, "bad mlp_adam arguments");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  adam_kernel<<<grid_for(ctx, CDWAC_MLP_NPARAMS), 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, CDWAC_MLP_NPARAMS,
                                                                                  lr, beta1, beta2, eps, c1, c2);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status cdwac_mlp_poles(cdwac_ctx* ctx, const float* params, int batch, const float* x, const float* scale,
                             double* poles, void* stream) {
  if (!ctx) return CDWAC_ERR_ARG;
  if (!params || batch < 1 || !x || !scale || !poles) return set_error(ctx, CDWAC_ERR_ARG, "bad mlp_poles arguments");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int B = batch;
  const size_t bytes = sizeof(__nv_bfloat16) * CDWAC_MLP_NPARAMS + sizeof(float) * ((size_t)6 * B * NH + (size_t)B * NOUT) +
                       4096;
  cdwac_status rc = ensure_scratch(ctx, bytes);
  if (rc) return rc;
  Arena ar(ctx->scratch);
  __nv_bfloat16* pb = ar.take<__nv_bfloat16>(CDWAC_MLP_NPARAMS);
  float* act = ar.take<float>((size_t)6 * B * NH);
  float* o = ar.take<float>((size_t)B * NOUT);
  ProfScope ps(ctx, PROF_MLP, st);
  to_bf16_kernel<<<grid_for(ctx, CDWAC_MLP_NPARAMS), 256, 0, st>>>(params, pb, CDWAC_MLP_NPARAMS);
  CDWAC_LAUNCH_CHECK(ctx);
  if ((rc = forward<__nv_bfloat16>(ctx, pb, B, x, act, o, st))) return rc;
  poles_kernel<<<ceil_div(B, 128), 128, 0, st>>>(o, scale, B, poles);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

}  // extern "C"
