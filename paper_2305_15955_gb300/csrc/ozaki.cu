// FP64-equivalent trailing update of the blocked LDL^T (mixed path) on the tcgen05 tensor cores.
//
//   A_ij -= sum_c W_ic L_jc,   c over the 64 columns of the current panel, i >= j >= k0 + 64,
//
// with W = L D the panel rows (row stride 64) and L the factor's panel columns.  GB300 issues FP64 FMAs at about
// 1.2 TFLOP/s and BF16 tensor products at about 2 PFLOP/s, so the update is formed from exact integer slices (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012) 95-118):
//
//   * every row x of W and of L is scaled by 2^-e, e the exponent of its largest magnitude, and cut into S signed
//     integer digits of B bits: x 2^-e = sum_s d_s 2^-Bs + r, |d_1| <= 2^B, |d_s| <= 2^(B-1) for s > 1,
//     |r| <= 2^-57 (the rounding of x 2^-e to SB fractional bits; the digits are then exact).  Real: S = 7, B = 8;
//     complex: S = 8, B = 7.  Each digit is exact in BF16 and each digit product is exact in FP32.  The digits are
//     cut with integer arithmetic from the bit patterns: GB300's FP64 units are its scarcest resource.
//   * tcgen05.mma sums, for each level L = s + t (S(S+1)/2 digit pairs), the products over the panel columns in
//     its own FP32 tensor-memory accumulator.  All partial sums of one level are integers of magnitude below
//     64 x 147 456 < 2^24 (real, largest level) or 128 x 40 960 < 2^23 (complex, K = 128), so every
//     accumulation is exact.
//   * the epilogue forms sum_L 2^-BL acc_L exactly in 64-bit integers (GB300's FP64 units are the scarce
//     resource), converts it once to FP64, scales it by 2^(e_i + e_j) with an integer add to the exponent field
//     and subtracts it from A.
//
// The digits dropped (levels above S + 1 and the remainders r) are below about 2^-54 max|W_i| max|L_j| per
// column, the size of the rounding error of an FP64 dot product of this length.
//
// Complex symmetric A (no conjugation): Re -= Wr Lr - Wi Li, Im -= Wr Li + Wi Lr.  The CTA loads the digits of
// Wr with those of Lr and Li, issues Re += Wr Lr and Im += Wr Li, then reloads the operand buffer with the digits
// of Wi and issues Re += -(Wi Li) (negated-A instruction descriptor) and Im += Wi Lr.
//
// One CTA per 128 x BN tile of the trailing lower triangle (BN = 64 real, 32 complex): one elected thread issues
// TMA (3-D maps over the digit planes, 128-byte swizzle), one issues the MMAs, all warps drain tensor memory
// (tcgen05.ld 32x32b; eight warps, two per lane quarter), stage the FP64 result in shared memory and update A with
// coalesced row segments.  Every
// mbarrier wait is bounded; on expiry the kernel records CDWAC_ERR_TIMEOUT, waits for the copies it issued and
// frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <string.h>

#include <type_traits>

#include "ozaki.cuh"
#include "tcgen05.cuh"

namespace {
using namespace tc;

constexpr int K = 64;       // panel width (the factorisation's block size)
constexpr int BM = 128;     // W rows per tile
constexpr int ROWB = K * 2; // bytes of one digit row: 64 BF16 = one 128-byte swizzle row
constexpr uint32_t NEG_A = 1u << 13;   // instruction-descriptor bit: negate the A operand

template <bool CPLX>
struct OzCfg {
  // digits per operand and bits per digit: real 7 x 8 bits (level sums over K = 64 stay below 9.5e6 < 2^24),
  // complex 8 x 7 bits (its level sums run over K = 128 products and must stay below 2^24 as well)
  static constexpr int S = CPLX ? 8 : 7;
  static constexpr int BETA = CPLX ? 7 : 8;
  static constexpr int NPART = CPLX ? 2 : 1;
  static constexpr int BN = CPLX ? 32 : 64;
  static constexpr int A_TILE = BM * ROWB;          // one digit of 128 W rows (16 KB)
  static constexpr int B_TILE = BN * ROWB;          // one digit of BN L rows
  static constexpr int A_BYTES = S * A_TILE;        // the digits of one part of W
  static constexpr int B_BYTES = NPART * S * B_TILE;
  static constexpr int SMEM = A_BYTES + B_BYTES + 1024;
  static constexpr int TMEM_COLS = 512;             // 7 levels x 64 columns, or (re, im) x 8 levels x 32 columns
  static constexpr int IM_COL = 256;                // first tensor-memory column of the imaginary accumulators
  // recombination scale 2^SHIFT: the level-2 sum (|acc_2| <= K d_1^2 = 64 * 2^16 real, 128 * 2^14 complex) times
  // 2^(SHIFT - 2 BETA) stays below 2^63, so the int64 sum of all levels cannot overflow
  static constexpr int SHIFT = CPLX ? 55 : 56;
};

struct OzMaps {
  CUtensorMap w, l;
};

// RN(a) 2^k as an FP64 number: the hardware conversion of a (round to nearest), then the power of two applied to
// the exponent field with an integer add instead of an FP64 multiply (GB300 issues an FP64 warp instruction in about
// 64 cycles).  Exact as long as the result stays in the normal range, which these updates do.
__device__ inline double scaled_int64(long long a, int k) {
  const long long b = __double_as_longlong(__ll2double_rn(a));
  return __longlong_as_double((b & 0x7FF0000000000000ll) ? b + ((long long)k << 52) : b);
}

template <bool CPLX>
__global__ void __launch_bounds__(256, 1) oz_update_kernel(const __grid_constant__ OzMaps maps, void* A_out, int n,
                                                           int k1, const int* __restrict__ ew,
                                                           const int* __restrict__ el, int part, unsigned* status) {
  using C = OzCfg<CPLX>;
  constexpr int S = C::S, BETA = C::BETA;
  constexpr int BN = C::BN;
  constexpr int Q = K / BN;     // column tiles in the next 64-column block
  constexpr int CT = BM / BN;   // column tiles per 128 rows
  int b = blockIdx.x, ti = 0;
  for (; ti < (1 << 20); ++ti) {
    const int cnt = part == 1 ? Q : (part == 0 ? CT * (ti + 1) : CT * (ti + 1) - Q);
    if (b < cnt) break;
    b -= cnt;
  }
  const int tj = part == 2 ? b + Q : b;
  const int row0 = k1 + ti * BM, col0 = k1 + tj * BN;
  if (row0 >= n || col0 >= n) return;   // the whole CTA leaves before any barrier or allocation

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + C::A_BYTES;
  __shared__ __align__(8) uint64_t bar_a0, bar_a1, bar_mma0, bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int loads_issued;
  __shared__ int exp_w[BM], exp_l[BN];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    mbar_init(&bar_a0, 1);
    mbar_init(&bar_a1, 1);
    mbar_init(&bar_mma0, 1);
    mbar_init(&bar_done, 1);
    abort_flag = 0;
    loads_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int r = threadIdx.x; r < BM; r += blockDim.x) exp_w[r] = row0 + r < n ? ew[row0 + r] : 0;
  for (int c = threadIdx.x; c < BN; c += blockDim.x) exp_l[c] = col0 + c < n ? el[col0 + c] : 0;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: digits of W (part 0) and of every part of L; for complex A then the digits of Wi
    mbar_expect_tx(&bar_a0, (uint32_t)(C::A_BYTES + C::B_BYTES));
    for (int s = 0; s < S; ++s) tma_load_3d(&maps.w, &bar_a0, sA + s * C::A_TILE, 0, row0, s);
    for (int p = 0; p < C::NPART; ++p)
      for (int s = 0; s < S; ++s) tma_load_3d(&maps.l, &bar_a0, sB + (p * S + s) * C::B_TILE, 0, col0, p * S + s);
    loads_issued = 1;
    if (CPLX) {
      if (mbar_wait(&bar_mma0, 0, &abort_flag)) {   // the phase-0 MMAs have finished reading sA
        mbar_expect_tx(&bar_a1, (uint32_t)C::A_BYTES);
        for (int s = 0; s < S; ++s) tma_load_3d(&maps.w, &bar_a1, sA + s * C::A_TILE, 0, row0, S + s);
        loads_issued = 3;
      } else {
        abort_flag = 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: level idx = s + t (0-based digits) accumulates in columns idx * BN (+ IM_COL)
    constexpr uint32_t id = idesc_bf16(BM, BN);
    bool ok = mbar_wait(&bar_a0, 0, &abort_flag);
    if (ok) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      for (int s = 0; s < S; ++s)
        for (int t = 0; s + t < S; ++t) {
          const uint32_t d = tmem + (uint32_t)((s + t) * BN);
#pragma unroll
          for (int kk = 0; kk < K / 16; ++kk) {
            const uint32_t acc = (s > 0 || kk > 0) ? 1u : 0u;   // digit 0 is the first to reach every level
            const uint64_t ad = sdesc(a0 + s * C::A_TILE + kk * 32);
            umma(d, ad, sdesc(b0 + t * C::B_TILE + kk * 32), id, acc);
            if (CPLX) umma(d + C::IM_COL, ad, sdesc(b0 + (S + t) * C::B_TILE + kk * 32), id, acc);
          }
        }
      umma_commit(&bar_mma0);
      if (CPLX) {
        ok = mbar_wait(&bar_a1, 0, &abort_flag);
        if (ok) {
          tc_fence_after();
          for (int s = 0; s < S; ++s)
            for (int t = 0; s + t < S; ++t) {
              const uint32_t d = tmem + (uint32_t)((s + t) * BN);
#pragma unroll
              for (int kk = 0; kk < K / 16; ++kk) {
                const uint64_t ad = sdesc(a0 + s * C::A_TILE + kk * 32);
                umma(d, ad, sdesc(b0 + (S + t) * C::B_TILE + kk * 32), id | NEG_A, 1u);   // Re += -(Wi Li)
                umma(d + C::IM_COL, ad, sdesc(b0 + t * C::B_TILE + kk * 32), id, 1u);     // Im += Wi Lr
              }
            }
        }
      }
    }
    if (!ok) abort_flag = 1;
    umma_commit(&bar_done);   // arrives once every MMA issued above has completed
  }
  __syncwarp();

  const bool done_ok = mbar_wait(&bar_done, 0, nullptr);
  tc_fence_after();
  // CTA-uniform verdict (the epilogue below has block-wide barriers)
  const bool good = __syncthreads_and(done_ok ? 1 : 0) && !abort_flag;
  if (threadIdx.x == 0 && !good) {
    raise_status(status, DEV_ERR_TIMEOUT);
    if (loads_issued & 1) mbar_wait(&bar_a0, 0, nullptr);   // no copy may land after the CTA exits
    if (loads_issued & 2) mbar_wait(&bar_a1, 0, nullptr);
  }
  if (good) {
    // Every MMA has completed, so the operand buffers are free for staging: slot [unit][quarter][32 rows][33].
    // Warp w reads tensor-memory lanes 32 (w % 4) .. + 31, i.e. tile rows of quarter q = w % 4; the two warpgroups
    // g = w / 4 take one unit each: column chunk g (real, 64 columns) or part g = re, im (complex, 32 columns).
    // In the read-modify-write lane = column, so each row segment is one coalesced access; the A values are
    // fetched before the tensor-memory drain so that their latency hides behind the integer recombination.
    using T = typename std::conditional<CPLX, cplx, double>::type;
    T* Ab = reinterpret_cast<T*>(A_out);
    double* stage = reinterpret_cast<double*>(smem);
    const int wq = warp & 3, wg = warp >> 2;
    const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
    const int c0 = CPLX ? 0 : 32 * wg;                 // column chunk of this warpgroup
    const int pp = CPLX ? wg : 0;                      // part drained by this warpgroup
    const int rbase = row0 + wq * 32 + (CPLX ? 16 * wg : 0);   // first row written by this warp
    const int col = col0 + c0 + lane;
    T cv0[16], cv1[16];
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      const int row = rbase + rr;
      if (row < n && col <= row) cv0[rr] = Ab[(long)row * n + col];
    }
    {
      // exact integer recombination N = sum_L acc_L 2^(SH - 7L) on the integer pipe (bits of the lowest levels
      // below 2^-SH are rounded off, < 2^-60 of the largest term)
      long long acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0;
#pragma unroll 1
      for (int idx = 0; idx < S; ++idx) {
        uint32_t v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)(pp * C::IM_COL + idx * BN + c0), v);
        constexpr int SH = C::SHIFT;
        const int sh = SH - BETA * (idx + 2);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const long long a = (long long)__float2int_rn(__uint_as_float(v[j]));   // exact: an integer < 2^23
          acc[j] += sh >= 0 ? (a << sh) : ((a + (1LL << (-sh - 1))) >> -sh);   // rounded, not floored
        }
      }
      // staged: the scaled update N 2^(e_row + e_col - SHIFT) of element (tile row wq * 32 + lane, column c0 + j);
      // the read-modify-write below is then one FP64 subtraction per element
      double* st = stage + ((wg * 4 + wq) * 32) * 33;
      const int kr = exp_w[wq * 32 + lane] - C::SHIFT;
#pragma unroll
      for (int j = 0; j < 32; ++j) st[lane * 33 + j] = scaled_int64(acc[j], kr + exp_l[c0 + j]);
    }
    if (CPLX)
      __syncthreads();   // both parts of every row staged
    else
      __syncwarp();
    if (!CPLX) {
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        const int row = rbase + 16 + rr;
        if (row < n && col <= row) cv1[rr] = Ab[(long)row * n + col];
      }
    }
    const double* st0 = stage + ((CPLX ? 0 : wg) * 4 + wq) * 32 * 33;
    const double* st1 = stage + (4 + wq) * 32 * 33;
    const int r_off = CPLX ? 16 * wg : 0;              // first staged row of this warp within its quarter
#pragma unroll
    for (int h = 0; h < (CPLX ? 1 : 2); ++h) {
#pragma unroll
      for (int rr = 0; rr < 16; ++rr) {
        const int r = r_off + h * 16 + rr, row = row0 + wq * 32 + r;
        if (row < n && col <= row) {
          T v = h == 0 ? cv0[rr] : cv1[rr];
          if constexpr (!CPLX) {
            v = v - st0[r * 33 + lane];
          } else {
            v.x = v.x - st0[r * 33 + lane];
            v.y = v.y - st1[r * 33 + lane];
          }
          Ab[(long)row * n + col] = v;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
}

// ---- digits: one warp per (row, operand); lane l holds columns 2l and 2l + 1 --------------------------------------
__device__ inline void load2(const double* p, double (&x)[2][2]) {   // rows of A need not be 16-byte aligned
  x[0][0] = p[0];
  x[0][1] = p[1];
  x[1][0] = x[1][1] = 0.0;
}
__device__ inline void load2(const cplx* p, double (&x)[2][2]) {
  const cplx a = p[0], b = p[1];
  x[0][0] = a.x;
  x[0][1] = b.x;
  x[1][0] = a.y;
  x[1][1] = b.y;
}

// Fixed-point value round(|x| 2^(F - e)) of an FP64 number with the sign of x, for a row whose largest magnitude is
// below 2^e (|result| < 2^F), from the bit pattern alone: GB300's FP64 pipe issues one warp instruction in about 64
// cycles, its integer pipe one per cycle.  Zero and subnormal inputs give 0 (their size is far below 2^(e - F)).
__device__ inline long long fixed_point(double x, int e, int F) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));   // |x| = mant 2^(E - 1075)
  const int sh = E - 1075 + F - e;                                                 // <= F - 53
  long long v;
  if (sh >= 0)
    v = mant << sh;
  else if (sh > -62)
    v = (mant + (1ll << (-sh - 1))) >> -sh;                                        // rounded to nearest
  else
    v = 0;
  return (b >> 63) ? -v : v;
}

// Signed digits of v (|v| < 2^F, F = S BETA): v = sum_s d_s 2^(F - BETA (s + 1)), d_0 the nearest integer to
// v / 2^(F - BETA) and every later digit the nearest integer to what remains at its weight, so |d_0| <= 2^BETA,
// |d_s| <= 2^(BETA - 1) and the last digit takes the exact remainder.
template <int S, int BETA>
__device__ inline void signed_digits(long long v, float (&d)[S]) {
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int k = BETA * (S - 1 - s);
    const long long q = k ? (v + (1ll << (k - 1))) >> k : v;
    d[s] = (float)q;   // |q| <= 2^BETA: exact
    v -= q * (1ll << k);
  }
}

template <class T>
__global__ void __launch_bounds__(256) oz_slice_kernel(const T* __restrict__ A, int n, int k0,
                                                       const T* __restrict__ wpanel, __nv_bfloat16* __restrict__ wpl,
                                                       __nv_bfloat16* __restrict__ lpl, int* __restrict__ ew,
                                                       int* __restrict__ el) {
  constexpr int NPART = sizeof(T) == sizeof(cplx) ? 2 : 1;
  constexpr int S = OzCfg<(NPART == 2)>::S, BETA = OzCfg<(NPART == 2)>::BETA;
  const int k1 = k0 + K, rows = n - k1;
  const long gw = (blockIdx.x * (long)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (gw >= 2L * rows) return;   // warp-uniform
  const int op = (int)(gw & 1), row = k1 + (int)(gw >> 1);
  const T* src = op == 0 ? wpanel + (long)row * K : A + (long)row * n + k0;
  double x[2][2];
  load2(src + 2 * lane, x);
  // largest magnitude of the row: the bit patterns of non-negative doubles order like the numbers
  unsigned long long m = 0;
#pragma unroll
  for (int p = 0; p < NPART; ++p)
#pragma unroll
    for (int c = 0; c < 2; ++c)
      m = max(m, (unsigned long long)__double_as_longlong(x[p][c]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)m, o));
  // e with max|x| < 2^e (the exponent frexp returns); 0 for an all-zero row
  const int e = m ? (int)(m >> 52) - 1022 : 0;
  __nv_bfloat16* pl = op == 0 ? wpl : lpl;
#pragma unroll
  for (int p = 0; p < NPART; ++p) {
    float d0[S], d1[S];
    signed_digits<S, BETA>(fixed_point(x[p][0], e, S * BETA), d0);
    signed_digits<S, BETA>(fixed_point(x[p][1], e, S * BETA), d1);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      __nv_bfloat162 v;
      v.x = __float2bfloat16_rn(d0[s]);
      v.y = __float2bfloat16_rn(d1[s]);
      *reinterpret_cast<__nv_bfloat162*>(pl + ((size_t)(p * S + s) * n + row) * K + 2 * lane) = v;
    }
  }
  if (lane == 0) (op == 0 ? ew : el)[row] = e;
}

bool make_map3(CUtensorMap* m, const void* base, int n, int planes, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)n, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)ROWB, (cuuint64_t)n * ROWB};
  cuuint32_t box[3] = {(cuuint32_t)K, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t plane_bytes(int n, bool cplx) {
  return cplx ? (size_t)2 * OzCfg<true>::S * n * ROWB : (size_t)OzCfg<false>::S * n * ROWB;
}

}  // namespace

size_t ozaki_scratch_bytes(int n, bool cplx) {
  return 4 * (plane_bytes(n, cplx) + 256) + 4 * ((size_t)n * sizeof(int) + 256) + 256;
}

cdwac_status ozaki_plan(cdwac_ctx* ctx, void* scratch, int n, bool cplx, OzakiPlan* plan) {
  memset(plan, 0, sizeof(*plan));
  plan->n = n;
  plan->cplx = cplx;
  Arena ar(scratch);
  const int planes = cplx ? 2 * OzCfg<true>::S : OzCfg<false>::S;
  const int bn = cplx ? OzCfg<true>::BN : OzCfg<false>::BN;
  for (int b = 0; b < 2; ++b) {
    plan->wpl[b] = ar.take<char>(plane_bytes(n, cplx));
    plan->lpl[b] = ar.take<char>(plane_bytes(n, cplx));
    plan->ew[b] = ar.take<int>(n);
    plan->el[b] = ar.take<int>(n);
    if (!make_map3(&plan->wmap[b], plan->wpl[b], n, planes, BM) || !make_map3(&plan->lmap[b], plan->lpl[b], n, planes, bn))
      return set_error(ctx, CDWAC_ERR_CUDA, "cuTensorMapEncodeTiled failed for the digit planes (n=%d)", n);
  }
  return CDWAC_OK;
}

template <class T>
cdwac_status ozaki_slice(cdwac_ctx* ctx, const OzakiPlan& plan, int buf, const T* A, int n, int k0, const T* wpanel,
                         cudaStream_t st) {
  const int rows = n - (k0 + K);
  if (rows <= 0) return CDWAC_OK;
  const long threads = 2L * rows * 32;
  oz_slice_kernel<T><<<(int)((threads + 255) / 256), 256, 0, st>>>(
      A, n, k0, wpanel, static_cast<__nv_bfloat16*>(plan.wpl[buf]), static_cast<__nv_bfloat16*>(plan.lpl[buf]),
      plan.ew[buf], plan.el[buf]);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

template <class T>
cdwac_status ozaki_update(cdwac_ctx* ctx, const OzakiPlan& plan, int buf, T* A, int n, int k0, int part,
                          cudaStream_t st) {
  constexpr bool CPLX = sizeof(T) == sizeof(cplx);
  using C = OzCfg<CPLX>;
  const int k1 = k0 + K, rows = n - k1;
  if (rows <= 0) return CDWAC_OK;
  const long mb = (rows + BM - 1) / BM, ct = BM / C::BN, q = K / C::BN;
  const long all = ct * mb * (mb + 1) / 2;
  const long grid = part == 0 ? all : (part == 1 ? q * mb : all - q * mb);
  if (grid <= 0) return CDWAC_OK;
  OzMaps maps;
  maps.w = plan.wmap[buf];
  maps.l = plan.lmap[buf];
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(oz_update_kernel<CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           C::SMEM));
  oz_update_kernel<CPLX><<<(unsigned)grid, 256, C::SMEM, st>>>(maps, A, n, k1, plan.ew[buf], plan.el[buf], part,
                                                              ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

template cdwac_status ozaki_slice<double>(cdwac_ctx*, const OzakiPlan&, int, const double*, int, int, const double*,
                                          cudaStream_t);
template cdwac_status ozaki_slice<cplx>(cdwac_ctx*, const OzakiPlan&, int, const cplx*, int, int, const cplx*,
                                        cudaStream_t);
template cdwac_status ozaki_update<double>(cdwac_ctx*, const OzakiPlan&, int, double*, int, int, int, cudaStream_t);
template cdwac_status ozaki_update<cplx>(cdwac_ctx*, const OzakiPlan&, int, cplx*, int, int, int, cudaStream_t);
