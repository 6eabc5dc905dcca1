// Mixed-precision W projection on the tcgen05 tensor cores, imaginary axis (Eqs. wriv, bigLambda):
//
//   W_nm = o^T (I - Pi)^-1 Pi o = sum_P y_P u_P / d_P,   [y | u] = L^-1 [o | Pi o],   L D L^T = I - Pi.
//
// The right-hand sides of all columns m (every state, every orbital) are solved together as one blocked forward
// substitution over the 64-row blocks b of the factor:
//
//   T = [O | Pi O]                              split-BF16 tensor-core GEMM for Pi O (three products, FP32 sums)
//   for b:  Y_b = L_bb^-1 T_b                   CUDA cores, FP32 (64 x 64 times 64 x 2C), W partial sums in FP64
//           T_>b -= L_>b,b Y_b                  split-BF16 tensor-core GEMM with K = 64
//
// The updates are grouped by eight blocks (512 rows): inside a group each step updates only the group's remaining
// rows, and after a group's last block one GEMM with K = 512 updates every row below it, so the FP32 right-hand
// sides below a group are read and written once per group instead of once per block.
//
// Near the real axis (complex symmetric L, real o) the same blocked substitution gives y = L^-1 o and
// W_nm = sum_P y_P^2 / d_P - sum_P o_P^2 (W is O(1) there: no cancellation).  The complex update is one real GEMM
// with K = 128 per block: A = [Re L | -Im L], and the rows of B are [Re y | Im y] for the real parts of T and
// [Im y | -Re y] for the imaginary parts.
//
// T is held column-major (T[col][row], col < 2C) so that both the GEMM epilogue (a warp writes 32 consecutive rows
// of one column) and the block solve (64 consecutive rows of a column) touch contiguous memory.  The BF16 planes of
// the factor, of Pi and of O^T are K-major for TMA (128-byte swizzle); the planes of a group's Y_b are [2C][512]
// (complex [2C][1024]).  The
// products carry ~2^-16 relative error per term like the tensor-core Pi, which dominates the mixed path's error.
#include <cuda.h>
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "tcgen05.cuh"

namespace {
using namespace tc;

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int PLANE = BM * BK * 2;       // bytes of one 128 x 64 BF16 tile
constexpr int STAGES = 3;
constexpr int STAGE = 4 * PLANE;         // A hi, A lo, B hi, B lo
constexpr int SMEM = STAGES * STAGE + 1024;
constexpr int NHH = STAGES;        // hi*hi accumulator buffers, one per operand stage (see tc_gemm_kernel)
constexpr int CORR = 32;           // K-tiles per correction accumulator (one buffer)
constexpr int TMEM_COLS = 4 * BN;  // three hi*hi buffers and the corrections
constexpr int GB = 8;              // 64-row blocks per group of the blocked substitution's updates

struct GemmMaps {
  CUtensorMap ah, al, bh, bl;
};

// out[(col) * ld + row_off + row] (=, -=) sum_k A[a_y0 + row][a_x0 + k] B[b_y0 + col][b_x0 + k], row < M, col < N.
// The tensor cores' FP32 accumulation loses a fraction of an ulp towards zero at every instruction, a bias over
// long chains (the Pi O product runs over K = N_aux), so the hi*hi products of every K-tile go to a fresh
// accumulator (three in turn) and the hi*lo + lo*hi corrections to one refreshed every CORR K-tiles, and warps 4-11 (two warpgroups, half the columns each) add every finished accumulator into FP32
// running sums with round-to-nearest adds.  Warp 0 lane 0 drives TMA, warp 1 owns the tensor memory and lane 0
// issues the MMAs, warps 2-3 are idle.
template <bool SUB>
__global__ void __launch_bounds__(384, 1) tc_gemm_kernel(const __grid_constant__ GemmMaps maps, int M, int N,
                                                         int k_tiles, int a_x0, int a_y0, int b_x0, int b_y0,
                                                         float* out, long ld, int row_off, unsigned* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t hh_empty[NHH], cr_empty;
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int issued, consumed;

  const int mt = (M + BM - 1) / BM;
  const int tm = blockIdx.x % mt, tn = blockIdx.x / mt;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < NHH; ++b) mbar_init(&hh_empty[b], 8);
    mbar_init(&cr_empty, 8);
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    int kt = 0;
    for (; kt < k_tiles; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      mbar_expect_tx(&full_bar[s], (uint32_t)STAGE);
      uint8_t* st = smem + s * STAGE;
      const int x = a_x0 + kt * BK;
      tma_load_2d(&maps.ah, &full_bar[s], st + 0 * PLANE, x, a_y0 + tm * BM);
      tma_load_2d(&maps.al, &full_bar[s], st + 1 * PLANE, x, a_y0 + tm * BM);
      tma_load_2d(&maps.bh, &full_bar[s], st + 2 * PLANE, b_x0 + kt * BK, b_y0 + tn * BN);
      tma_load_2d(&maps.bl, &full_bar[s], st + 3 * PLANE, b_x0 + kt * BK, b_y0 + tn * BN);
    }
    issued = kt;
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    int kt = 0;
    for (; kt < k_tiles; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      const int hb = kt % NHH, g = kt / CORR;
      const bool g_first = kt % CORR == 0;
      if (kt >= NHH && !mbar_wait(&hh_empty[hb], (uint32_t)(kt / NHH - 1) & 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      if (g_first && g >= 1 && !mbar_wait(&cr_empty, (uint32_t)(g - 1) & 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      if (!mbar_wait(&full_bar[s], ph, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t base = smem_u32(smem + s * STAGE);
      const uint32_t dh = tmem + (uint32_t)(hb * BN), dc = tmem + (uint32_t)(NHH * BN);
      // the hi*hi products of the K-tile first, then its corrections: consecutive instructions share an accumulator
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        umma(dh, sdesc(base + 0 * PLANE + kk * 32), sdesc(base + 2 * PLANE + kk * 32), idesc,
             kk == 0 ? 0u : 1u);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t ko = kk * 32;
        umma(dc, sdesc(base + 0 * PLANE + ko), sdesc(base + 3 * PLANE + ko), idesc, (g_first && kk == 0) ? 0u : 1u);
        umma(dc, sdesc(base + 1 * PLANE + ko), sdesc(base + 2 * PLANE + ko), idesc, 1u);
      }
      umma_commit(&empty_bar[s]);

    }
    consumed = kt;
    umma_commit(&done_bar);
  } else if (warp >= 4) {
    // two drain warpgroups: group g sums columns [64 g, 64 g + 64); warp w reads lanes 32 (w % 4) .. + 31 = rows
    const int g = (warp - 4) >> 2, q = warp & 3;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float run[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) run[j] = 0.f;
    bool ok = true;
    // adds accumulator set `set` (0 .. NHH - 1: hi*hi buffers; NHH: the correction buffer) into the running sums
    auto drain = [&](uint64_t* empty, int set) {
      tc_fence_after();
      tmem_add64(tmem + lane_base + (uint32_t)(set * BN + g * 64), run);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(empty);
      return true;
    };
    for (int kt = 0; kt < k_tiles && ok; ++kt) {
      // the commit that releases K-tile kt's operand stage arrives once every MMA up to kt has completed, so its
      // phase also marks the K-tile's accumulators complete; the MMAs of K-tile kt + STAGES, whose commit ends the
      // stage's next phase, wait for this drain (NHH = STAGES), so the phase cannot pass unobserved
      const uint32_t parity = (uint32_t)(kt / STAGES) & 1u;
      ok = __all_sync(0xffffffffu, mbar_wait(&empty_bar[kt % STAGES], parity, &abort_flag));
      if (!ok) break;
      drain(&hh_empty[kt % NHH], kt % NHH);
      if (kt % CORR == CORR - 1 || kt == k_tiles - 1) drain(&cr_empty, NHH);
    }
    if (!ok) {
      abort_flag = 1;
    } else {
      // out is column-major (out[col][row]): the 32 lanes hold consecutive rows, so every access is coalesced
      const int row = tm * BM + q * 32 + lane;
      if (row < M) {
        float* o = out + row_off + row;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 32) {
          // every load of 32 columns before any store: the compiler cannot prove o[j ld] and o[k ld] distinct
          float cur[32];
          if (SUB) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int col = tn * BN + g * 64 + c0 + j;
              cur[j] = col < N ? o[(long)col * ld] : 0.f;
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = tn * BN + g * 64 + c0 + j;
            if (col < N) o[(long)col * ld] = SUB ? cur[j] - run[c0 + j] : run[c0 + j];
          }
        }
      }
    }
  }
  __syncwarp();

  // every MMA issued has completed before the tensor memory is released, on every path
  const bool done_ok = mbar_wait(&done_bar, 0, nullptr);
  tc_fence_after();
  __syncthreads();
  if (threadIdx.x == 0 && (!done_ok || abort_flag)) {
    raise_status(status, DEV_ERR_TIMEOUT);
    for (int kt = consumed; kt < issued; ++kt) mbar_wait(&full_bar[kt % STAGES], (uint32_t)(kt / STAGES) & 1u, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TMEM_COLS)
                 : "memory");
  }
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Strict lower triangle of the FP64 factor -> BF16 hi/lo planes [n][npad] (zero elsewhere, including the K
// padding); the diagonal-block inverses -> FP32.
__global__ void factor_split_kernel(const double* __restrict__ L, int n, int npad, const double* __restrict__ linv,
                                    int nblk, __nv_bfloat16* __restrict__ lh, __nv_bfloat16* __restrict__ ll,
                                    float* __restrict__ linv32) {
  const long total = (long)n * npad, tl = (long)nblk * 64 * 64;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total + tl; e += (long)gridDim.x * blockDim.x) {
    if (e < total) {
      const long r = e / npad, c = e % npad;
      const float v = (c < r) ? (float)L[r * n + c] : 0.f;
      split_bf16(v, lh[e], ll[e]);
    } else {
      linv32[e - total] = (float)linv[e - total];
    }
  }
}

// Pi = -negpi (FP32, full symmetric [n][n]) -> BF16 hi/lo planes [n][npad]
__global__ void pi_split_kernel(const float* __restrict__ negpi, int n, int npad, __nv_bfloat16* __restrict__ ph,
                                __nv_bfloat16* __restrict__ pl) {
  const long total = (long)n * npad;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / npad, c = e % npad;
    const float v = c < n ? -negpi[r * n + c] : 0.f;
    split_bf16(v, ph[e], pl[e]);
  }
}

// O^T: column c = (state s, orbital m) -> FP32 row T[c][0..n) (zero padded to npad) and, if oh is given, its
// BF16 hi/lo planes
template <class TIn>
__global__ void o_transpose_kernel(const TIn* __restrict__ O, long o_state_stride, long ld_o, int cols_per_state,
                                   int n_cols, int n, int npad, float* __restrict__ t32, __nv_bfloat16* __restrict__ oh,
                                   __nv_bfloat16* __restrict__ ol) {
  __shared__ float tile[32][33];
  const int P0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const int P = P0 + k, c = c0 + tx;
    float v = 0.f;
    if (P < n && c < n_cols) {
      const int s = c / cols_per_state, m = c % cols_per_state;
      v = (float)O[s * o_state_stride + (long)P * ld_o + m];
    }
    tile[k][tx] = v;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int c = c0 + k, P = P0 + tx;
    if (c < n_cols && P < npad) {
      const float v = tile[tx][k];
      const long e = (long)c * npad + P;
      t32[e] = v;
      if (oh) split_bf16(v, oh[e], ol[e]);
    }
  }
}

// Block step b: Y_b = X_b T_b for every column (X_b = L_bb^-1, unit lower), written as BF16 hi/lo planes into
// columns yo .. yo + 63 of [2C][ys] for the updates, and the W partial sums  part[b][m] = sum_r y[m][r] y[C + m][r]
// / d_r.
// One CTA per 16 column pairs (m, C + m); thread (r, g) owns row r and columns {4 of m, their 4 partners}.
constexpr int SP = 16;
__global__ void __launch_bounds__(256) block_solve_kernel(const float* __restrict__ T, long ld, int n, int C, int b,
                                                          const float* __restrict__ linv32,
                                                          const double* __restrict__ dinv,
                                                          __nv_bfloat16* __restrict__ yh,
                                                          __nv_bfloat16* __restrict__ yl, int ys, int yo,
                                                          double* __restrict__ part) {
  __shared__ float Xs[64][65];
  __shared__ float Ts[2 * SP][65];
  __shared__ double red[4][64][4];
  const int m0 = blockIdx.x * SP;
  const int tid = threadIdx.x, r = tid % 64, g = tid / 64;
  const int r0 = b * 64;
  const float* X = linv32 + (long)b * 64 * 64;
#pragma unroll
  for (int it = 0; it < 64 * 64 / 256; ++it) {
    const int e = tid + 256 * it;
    Xs[e / 64][e % 64] = X[e];
  }
#pragma unroll
  for (int it = 0; it < 2 * SP * 64 / 256; ++it) {
    const int e = tid + 256 * it, cc = e / 64, k = e % 64;
    const int col = cc < SP ? m0 + cc : C + m0 + (cc - SP);
    const bool ok = (cc < SP ? m0 + cc : m0 + cc - SP) < C && r0 + k < n;
    Ts[cc][k] = ok ? T[(long)col * ld + r0 + k] : 0.f;
  }
  __syncthreads();
  float y[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) y[j] = 0.f;
  for (int k = 0; k <= r; ++k) {
    const float x = Xs[r][k];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      y[j] = fmaf(x, Ts[g * 4 + j][k], y[j]);
      y[4 + j] = fmaf(x, Ts[SP + g * 4 + j][k], y[4 + j]);
    }
  }
  const int row = r0 + r;
  const double di = row < n ? dinv[row] : 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int m = m0 + g * 4 + j;
    red[g][r][j] = (double)y[j] * (double)y[4 + j] * di;
    if (m < C) {
      __nv_bfloat16 h, l;
      split_bf16(y[j], h, l);
      yh[(long)m * ys + yo + r] = h;
      yl[(long)m * ys + yo + r] = l;
      split_bf16(y[4 + j], h, l);
      yh[(long)(C + m) * ys + yo + r] = h;
      yl[(long)(C + m) * ys + yo + r] = l;
    }
  }
  __syncthreads();
  if (tid < SP) {
    const int gg = tid / 4, j = tid % 4, m = m0 + tid;
    double s = 0.0;
    for (int k = 0; k < 64; ++k) s += red[gg][k][j];
    if (m < C) part[(long)b * C + m] = s;
  }
}

// W[c] = sum_b part[b][c], written to W_out[s * w_state_stride + m] for c = (s, m)
__global__ void w_reduce_kernel(const double* __restrict__ part, int nblk, int C, int cols_per_state,
                                double* __restrict__ W_out, long w_state_stride) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long)b * C + c];
  W_out[(long)(c / cols_per_state) * w_state_stride + c % cols_per_state] = s;
}

// ---- near-real (complex symmetric) solve ---------------------------------------------------------------------

struct f2 {
  float x, y;
};

// Strict lower complex factor -> BF16 hi/lo planes [n][2 npad]: block b occupies columns 128b..128b+127 as
// [Re L(:, 64b..64b+63) | -Im L(:, 64b..64b+63)]; complex diagonal-block inverses -> FP32 pairs.
__global__ void cfactor_split_kernel(const cplx* __restrict__ L, int n, int npad, const cplx* __restrict__ linv,
                                     int nblk, __nv_bfloat16* __restrict__ lh, __nv_bfloat16* __restrict__ ll,
                                     f2* __restrict__ linv32) {
  const long w2 = 2L * npad, total = (long)n * w2, tl = (long)nblk * 64 * 64;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total + tl; e += (long)gridDim.x * blockDim.x) {
    if (e < total) {
      const long r = e / w2, cc = e % w2;
      const long b = cc / 128, k = cc % 128, col = 64 * b + (k % 64);
      float v = 0.f;
      if (col < r) {
        const cplx x = L[r * n + col];
        v = k < 64 ? (float)x.x : (float)-x.y;
      }
      split_bf16(v, lh[e], ll[e]);
    } else {
      const cplx x = linv[e - total];
      linv32[e - total] = f2{(float)x.x, (float)x.y};
    }
  }
}

// Block step b, complex: Y_b = X_b T_b (T rows c = Re, C + c = Im), planes in columns yo .. yo + 127 of [2C][ys]
// for the updates (row c: [Re y | Im y], row C + c: [Im y | -Re y]) and part[b][c] = sum_r y_r^2 / d_r (complex,
// FP64).
// One CTA per 8 columns; thread (r, g) owns row r of columns 2g and 2g + 1.
constexpr int SPC = 8;
__global__ void __launch_bounds__(256) block_solve_c_kernel(const float* __restrict__ T, long ld, int n, int C, int b,
                                                            const f2* __restrict__ linv32,
                                                            const cplx* __restrict__ dinv,
                                                            __nv_bfloat16* __restrict__ yh,
                                                            __nv_bfloat16* __restrict__ yl, int ys, int yo,
                                                            double* __restrict__ part) {
  __shared__ f2 Xs[64][65];
  __shared__ float Tr[SPC][65], Ti[SPC][65];
  __shared__ double red[4][64][2][2];
  const int m0 = blockIdx.x * SPC;
  const int tid = threadIdx.x, r = tid % 64, g = tid / 64;
  const int r0 = b * 64;
  const f2* X = linv32 + (long)b * 64 * 64;
#pragma unroll
  for (int it = 0; it < 64 * 64 / 256; ++it) {
    const int e = tid + 256 * it;
    Xs[e / 64][e % 64] = X[e];
  }
#pragma unroll
  for (int it = 0; it < 2 * SPC * 64 / 256; ++it) {
    const int e = tid + 256 * it, cc = e / 64, k = e % 64;
    const int m = m0 + (cc % SPC);
    const bool ok = m < C && r0 + k < n;
    const float v = ok ? T[(long)(cc < SPC ? m : C + m) * ld + r0 + k] : 0.f;
    if (cc < SPC)
      Tr[cc][k] = v;
    else
      Ti[cc - SPC][k] = v;
  }
  __syncthreads();
  float yr[2] = {0.f, 0.f}, yi[2] = {0.f, 0.f};
  for (int k = 0; k <= r; ++k) {
    const f2 x = Xs[r][k];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float tr = Tr[2 * g + j][k], ti = Ti[2 * g + j][k];
      yr[j] = fmaf(x.x, tr, fmaf(-x.y, ti, yr[j]));
      yi[j] = fmaf(x.x, ti, fmaf(x.y, tr, yi[j]));
    }
  }
  const int row = r0 + r;
  const cplx di = row < n ? dinv[row] : mkc(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int m = m0 + 2 * g + j;
    const double a = yr[j], bb = yi[j];
    const double sr = a * a - bb * bb, si = 2.0 * a * bb;   // y^2
    red[g][r][j][0] = sr * di.x - si * di.y;
    red[g][r][j][1] = sr * di.y + si * di.x;
    if (m < C) {
      __nv_bfloat16 h, l;
      split_bf16(yr[j], h, l);
      yh[(long)m * ys + yo + r] = h;
      yl[(long)m * ys + yo + r] = l;
      split_bf16(yi[j], h, l);
      yh[(long)m * ys + yo + 64 + r] = h;
      yl[(long)m * ys + yo + 64 + r] = l;
      yh[(long)(C + m) * ys + yo + r] = h;
      yl[(long)(C + m) * ys + yo + r] = l;
      split_bf16(-yr[j], h, l);
      yh[(long)(C + m) * ys + yo + 64 + r] = h;
      yl[(long)(C + m) * ys + yo + 64 + r] = l;
    }
  }
  __syncthreads();
  if (tid < 2 * SPC) {
    const int mm = tid / 2, part_ri = tid % 2, gg = mm / 2, j = mm % 2, m = m0 + mm;
    double acc = 0.0;
    for (int k = 0; k < 64; ++k) acc += red[gg][k][j][part_ri];
    if (m < C) part[((long)b * C + m) * 2 + part_ri] = acc;
  }
}

// W[c] = sum_b part[b][c] - sum_P o_P^2 for column c = (s, m), written to W_out[s * w_state_stride + m]; one
// CTA per column, the sums over P and b split across its threads
template <class TIn>
__global__ void __launch_bounds__(256) w_reduce_c_kernel(const double* __restrict__ part, int nblk, int C, int n,
                                                         const TIn* __restrict__ O, long o_state_stride, long ld_o,
                                                         int cols_per_state, cplx* __restrict__ W_out,
                                                         long w_state_stride) {
  __shared__ double sre[256], sim[256];
  const int c = blockIdx.x, tid = threadIdx.x;
  const int s = c / cols_per_state, m = c % cols_per_state;
  double re = 0.0, im = 0.0;
  for (int P = tid; P < n; P += 256) {
    const double o = (double)O[s * o_state_stride + (long)P * ld_o + m];
    re -= o * o;
  }
  for (int b = tid; b < nblk; b += 256) {
    re += part[((long)b * C + c) * 2];
    im += part[((long)b * C + c) * 2 + 1];
  }
  sre[tid] = re;
  sim[tid] = im;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (tid < h) {
      sre[tid] += sre[tid + h];
      sim[tid] += sim[tid + h];
    }
    __syncthreads();
  }
  if (tid == 0) W_out[(long)s * w_state_stride + m] = mkc(sre[0], sim[0]);
}

bool make_map(CUtensorMap* m, const void* base, int rows, long kpad) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct Bufs {
  __nv_bfloat16 *lh, *ll, *ph, *pl, *oh, *ol, *yh, *yl;
  float *t, *linv32;
  double* part;
  int npad, nblk;
};

Bufs carve(void* scratch, int n, int C) {
  Bufs b;
  b.npad = ((n + 63) / 64) * 64;
  b.nblk = (n + 63) / 64;
  Arena ar(scratch);
  const size_t sq = (size_t)n * b.npad, oc = (size_t)C * b.npad;
  b.lh = ar.take<__nv_bfloat16>(sq);
  b.ll = ar.take<__nv_bfloat16>(sq);
  b.ph = ar.take<__nv_bfloat16>(sq);
  b.pl = ar.take<__nv_bfloat16>(sq);
  b.oh = ar.take<__nv_bfloat16>(oc);
  b.ol = ar.take<__nv_bfloat16>(oc);
  b.yh = ar.take<__nv_bfloat16>((size_t)2 * C * 64 * GB);
  b.yl = ar.take<__nv_bfloat16>((size_t)2 * C * 64 * GB);
  b.t = ar.take<float>(2 * oc);
  b.linv32 = ar.take<float>((size_t)b.nblk * 64 * 64);
  b.part = ar.take<double>((size_t)b.nblk * C);
  return b;
}

int grid_of(cdwac_ctx* ctx, long work) {
  long b = (work + 255) / 256, cap = (long)ctx->num_sms * 8;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

template <bool SUB>
cdwac_status gemm(cdwac_ctx* ctx, const GemmMaps& maps, int M, int N, int k_tiles, int a_x0, int a_y0, float* out,
                  long ld, int row_off, cudaStream_t st, int b_x0 = 0) {
  if (M <= 0 || N <= 0) return CDWAC_OK;
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(tc_gemm_kernel<SUB>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
  const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
  tc_gemm_kernel<SUB><<<mt * nt, 384, SMEM, st>>>(maps, M, N, k_tiles, a_x0, a_y0, b_x0, 0, out, ld, row_off,
                                                  ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

// The updates after block step blk of the blocked substitution, with blocks taken in groups of GB (512 rows): the
// rows of the rest of blk's group get Y_blk alone (K = 64 columns of the factor, kpb K-tiles of 64 per block),
// and after the last block of a group every row below the group gets the whole group's Y at once
// (K = 64 x GB), so the RHS matrix T below the group is read and written once per group instead of once per block.
cdwac_status group_update(cdwac_ctx* ctx, const GemmMaps& upd, int n, int C, int blk, int nblk, int kpb, float* t,
                          long ld, cudaStream_t st) {
  const int g = blk / GB, gend = std::min(nblk, (g + 1) * GB), r1 = (blk + 1) * 64;
  if (r1 >= n) return CDWAC_OK;
  const int kw = 64 * kpb;   // factor (and Y) columns per block
  if (blk + 1 < gend) {
    const int rend = std::min(n, gend * 64);
    return gemm<true>(ctx, upd, rend - r1, 2 * C, kpb, blk * kw, r1, t, ld, r1, st, (blk % GB) * kw);
  }
  const int nb = blk + 1 - g * GB;
  return gemm<true>(ctx, upd, n - r1, 2 * C, kpb * nb, g * GB * kw, r1, t, ld, r1, st, 0);
}

}  // namespace

namespace {
struct CBufs {
  __nv_bfloat16 *lh, *ll, *yh, *yl;
  float* t;
  f2* linv32;
  double* part;
  int npad, nblk;
};

CBufs carve_c(void* scratch, int n, int C) {
  CBufs b;
  b.npad = ((n + 63) / 64) * 64;
  b.nblk = (n + 63) / 64;
  Arena ar(scratch);
  const size_t sq = (size_t)n * 2 * b.npad;
  b.lh = ar.take<__nv_bfloat16>(sq);
  b.ll = ar.take<__nv_bfloat16>(sq);
  b.yh = ar.take<__nv_bfloat16>((size_t)2 * C * 128 * GB);
  b.yl = ar.take<__nv_bfloat16>((size_t)2 * C * 128 * GB);
  b.t = ar.take<float>((size_t)2 * C * b.npad);
  b.linv32 = ar.take<f2>((size_t)b.nblk * 64 * 64);
  b.part = ar.take<double>((size_t)b.nblk * C * 2);
  return b;
}
}  // namespace

size_t wsolve_tc_c_scratch_bytes(int n, int n_cols) {
  const size_t npad = ((size_t)n + 63) / 64 * 64, nblk = npad / 64;
  return 2 * ((size_t)n * 2 * npad * 2 + 256) + 2 * ((size_t)2 * n_cols * 128 * GB * 2 + 256) +
         ((size_t)2 * n_cols * npad * 4 + 256) + (nblk * 64 * 64 * 8 + 256) + (nblk * n_cols * 16 + 256) + 1024;
}

cdwac_status wsolve_tc_c(cdwac_ctx* ctx, const cplx* L, const cplx* dinv, const cplx* linv, int n, const void* O,
                         int dtype, long o_state_stride, long ld_o, int n_states, int cols_per_state, cplx* W_out,
                         long w_state_stride, void* scratch, cudaStream_t st) {
  const int C = n_states * cols_per_state;
  if (C <= 0) return CDWAC_OK;
  CBufs b = carve_c(scratch, n, C);
  const long ld = b.npad;
  {
    const long work = (long)n * 2 * b.npad + (long)b.nblk * 4096;
    cfactor_split_kernel<<<grid_of(ctx, work), 256, 0, st>>>(L, n, b.npad, linv, b.nblk, b.lh, b.ll, b.linv32);
    CDWAC_LAUNCH_CHECK(ctx);
    dim3 tg((b.npad + 31) / 32, (C + 31) / 32);
    if (dtype == CDWAC_F64)
      o_transpose_kernel<double><<<tg, 256, 0, st>>>((const double*)O, o_state_stride, ld_o, cols_per_state, C, n,
                                                     b.npad, b.t, nullptr, nullptr);
    else
      o_transpose_kernel<float><<<tg, 256, 0, st>>>((const float*)O, o_state_stride, ld_o, cols_per_state, C, n,
                                                    b.npad, b.t, nullptr, nullptr);
    CDWAC_LAUNCH_CHECK(ctx);
    CDWAC_CUDA_TRY(ctx, cudaMemsetAsync(b.t + (long)C * ld, 0, sizeof(float) * (size_t)C * ld, st));
  }
  GemmMaps upd;
  if (!make_map(&upd.ah, b.lh, n, 2L * b.npad) || !make_map(&upd.al, b.ll, n, 2L * b.npad) ||
      !make_map(&upd.bh, b.yh, 2 * C, 128L * GB) || !make_map(&upd.bl, b.yl, 2 * C, 128L * GB))
    return set_error(ctx, CDWAC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the complex W solve (n=%d, C=%d)", n, C);
  cdwac_status rc;
  for (int blk = 0; blk < b.nblk; ++blk) {
    block_solve_c_kernel<<<(C + SPC - 1) / SPC, 256, 0, st>>>(b.t, ld, n, C, blk, b.linv32, dinv, b.yh, b.yl,
                                                               128 * GB, 128 * (blk % GB), b.part);
    CDWAC_LAUNCH_CHECK(ctx);
    if ((rc = group_update(ctx, upd, n, C, blk, b.nblk, 2, b.t, ld, st))) return rc;
  }
  if (dtype == CDWAC_F64)
    w_reduce_c_kernel<double><<<C, 256, 0, st>>>(b.part, b.nblk, C, n, (const double*)O,
                                                               o_state_stride, ld_o, cols_per_state, W_out,
                                                               w_state_stride);
  else
    w_reduce_c_kernel<float><<<C, 256, 0, st>>>(b.part, b.nblk, C, n, (const float*)O,
                                                              o_state_stride, ld_o, cols_per_state, W_out,
                                                              w_state_stride);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

size_t wsolve_tc_scratch_bytes(int n, int n_cols) {
  const size_t npad = ((size_t)n + 63) / 64 * 64, nblk = npad / 64;
  const size_t sq = (size_t)n * npad, oc = (size_t)n_cols * npad;
  return 4 * (sq * 2 + 256) + 2 * (oc * 2 + 256) + 2 * ((size_t)2 * n_cols * 64 * GB * 2 + 256) + (2 * oc * 4 + 256) +
         (nblk * 64 * 64 * 4 + 256) + (nblk * n_cols * 8 + 256) + 1024;
}

cdwac_status wsolve_tc(cdwac_ctx* ctx, const double* L, const double* dinv, const double* linv, const float* negpi32,
                       int n, const void* O, int dtype, long o_state_stride, long ld_o, int n_states,
                       int cols_per_state, double* W_out, long w_state_stride, void* scratch, cudaStream_t st) {
  const int C = n_states * cols_per_state;
  if (C <= 0) return CDWAC_OK;
  Bufs b = carve(scratch, n, C);
  const long ld = b.npad;
  {
    const long work = (long)n * b.npad + (long)b.nblk * 4096;
    factor_split_kernel<<<grid_of(ctx, work), 256, 0, st>>>(L, n, b.npad, linv, b.nblk, b.lh, b.ll, b.linv32);
    CDWAC_LAUNCH_CHECK(ctx);
    pi_split_kernel<<<grid_of(ctx, (long)n * b.npad), 256, 0, st>>>(negpi32, n, b.npad, b.ph, b.pl);
    CDWAC_LAUNCH_CHECK(ctx);
    dim3 tg((b.npad + 31) / 32, (C + 31) / 32);
    if (dtype == CDWAC_F64)
      o_transpose_kernel<double><<<tg, 256, 0, st>>>((const double*)O, o_state_stride, ld_o, cols_per_state, C, n,
                                                     b.npad, b.t, b.oh, b.ol);
    else
      o_transpose_kernel<float><<<tg, 256, 0, st>>>((const float*)O, o_state_stride, ld_o, cols_per_state, C, n,
                                                    b.npad, b.t, b.oh, b.ol);
    CDWAC_LAUNCH_CHECK(ctx);
  }
  GemmMaps pio, upd;
  if (!make_map(&pio.ah, b.ph, n, b.npad) || !make_map(&pio.al, b.pl, n, b.npad) ||
      !make_map(&pio.bh, b.oh, C, b.npad) || !make_map(&pio.bl, b.ol, C, b.npad) ||
      !make_map(&upd.ah, b.lh, n, b.npad) || !make_map(&upd.al, b.ll, n, b.npad) ||
      !make_map(&upd.bh, b.yh, 2 * C, 64L * GB) || !make_map(&upd.bl, b.yl, 2 * C, 64L * GB))
    return set_error(ctx, CDWAC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the W solve (n=%d, C=%d)", n, C);
  cdwac_status rc;
  // second half of T: Pi O
  if ((rc = gemm<false>(ctx, pio, n, C, b.npad / BK, 0, 0, b.t + (long)C * ld, ld, 0, st))) return rc;
  for (int blk = 0; blk < b.nblk; ++blk) {
    block_solve_kernel<<<(C + SP - 1) / SP, 256, 0, st>>>(b.t, ld, n, C, blk, b.linv32, dinv, b.yh, b.yl, 64 * GB,
                                                          64 * (blk % GB), b.part);
    CDWAC_LAUNCH_CHECK(ctx);
    if ((rc = group_update(ctx, upd, n, C, blk, b.nblk, 1, b.t, ld, st))) return rc;
  }
  w_reduce_kernel<<<(C + 127) / 128, 128, 0, st>>>(b.part, b.nblk, C, cols_per_state, W_out, w_state_stride);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}
