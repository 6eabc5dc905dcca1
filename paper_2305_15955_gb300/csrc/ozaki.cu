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
//   * the epilogue forms sum_L 2^-BL acc_L exactly in 64-bit integers, rounds it once to FP64 scaled by
//     2^(e_i + e_j) (both with integer instructions: GB300's FP64 units are the scarce resource) and subtracts it
//     from A, the one FP64 instruction per element.
//
// The digits dropped (levels above S + 1 and the remainders r) are below about 2^-54 max|W_i| max|L_j| per
// column, the size of the rounding error of an FP64 dot product of this length.
//
// Complex symmetric A (no conjugation): Re -= Wr Lr - Wi Li, Im -= Wr Li + Wi Lr.  Two CTAs share a complex
// tile, one per part of A: the re CTA issues Re += Wr Lr and then Re += -(Wi Li) (negated-A instruction
// descriptor), the im CTA Im += Wr Li and then Im += Wi Lr.
//
// Real A: `oz_strip_kernel`, one CTA per chunk of 128 x 32 tiles of one 128-row strip (640 threads, one CTA per
// SM): the strip's W digits stay resident, the L digits and two tensor-memory accumulator sets are double-buffered,
// one MMA per W digit and k-step with the L digits stacked along N, sixteen independent epilogue warps.
// Complex A: `oz_update_kernel<true>`, one CTA per 128 x 32 tile and part of A (256 threads, two CTAs per SM with
// 97 KB of shared memory and 256 tensor-memory columns each, so that one CTA's epilogue overlaps the other's loads
// and MMAs): the tile's L digits stay resident, the W digits stream through a ring, N-stacked MMAs as above.
// Both: one elected thread issues TMA (3-D maps over the digit planes, 128-byte swizzle), one issues the MMAs, the
// epilogue warps drain tensor memory (tcgen05.ld 32x32b), recombine the levels exactly in integers, assemble the
// FP64 update with integer instructions, stage it per warp in shared memory and update A with coalesced row
// segments.  Every mbarrier wait is bounded; on expiry a kernel records CDWAC_ERR_TIMEOUT, waits for the copies it
// issued and frees its tensor memory.
#include <cuda.h>
#include <cuda_bf16.h>
#include <string.h>

#include <algorithm>
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
  static constexpr int NPART = CPLX ? 2 : 1;        // parts (re, im) of W and of L
  static constexpr int BN = 32;                     // tile columns
  static constexpr int NT = 256;                    // threads: eight warps, two per tensor-memory lane quarter
  static constexpr int A_TILE = BM * ROWB;          // one digit of 128 W rows (16 KB)
  static constexpr int B_TILE = BN * ROWB;          // one digit of 32 L rows (4 KB)
  static constexpr int B_BYTES = NPART * S * B_TILE;   // every digit of every part of L: 28 KB real, 64 KB complex
  static constexpr int NS = 2;                      // stages of the W-digit ring
  static constexpr int WLOADS = NPART * S;          // W digit planes per tile: Wr digits, then (complex) Wi digits
  // 97 KB (complex) of dynamic shared memory: two CTAs per SM (the real update runs by strips, oz_strip_kernel;
  // the real instance gives the digit and plane sizes)
  static constexpr int SMEM = B_BYTES + NS * A_TILE + 1024;
  static constexpr int MIN_CTAS = 2;
  static constexpr int TMEM_COLS = 256;             // S levels x 32 columns (224 real, 256 complex)
  // recombination scale 2^SHIFT: the level-2 sum (|acc_2| <= K d_1^2 = 64 * 2^16 real, 128 * 2^14 complex) times
  // 2^(SHIFT - 2 BETA) stays below 2^63, so the int64 sum of all levels cannot overflow
  static constexpr int SHIFT = CPLX ? 55 : 56;
};

struct OzMaps {
  CUtensorMap w, l;
};

// RN(a) 2^k as an FP64 number, assembled with integer instructions (GB300 issues an FP64 warp instruction, the
// conversion included, in about 64 cycles, an integer one in one or two): the magnitude is normalised with a
// count of leading zeros, its top 53 bits are rounded to nearest (ties to even) on the 11 bits below them, and
// the biased exponent 1086 - lz + k is added above the mantissa (a carry out of the rounding moves into the
// exponent field, as it should).  Results outside the normal range take the FP64 path (not reached by these
// updates).
__device__ inline double scaled_int64(long long a, int k) {
  if (a == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)a & 0x8000000000000000ull;
  unsigned long long m = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
  const int lz = __clzll((long long)m);
  const int E = 1086 - lz + k;
  if (E < 2 || E > 2045) return ldexp((double)a, k);
  m <<= lz;
  const unsigned rem = (unsigned)(m & 0x7FFull);
  m >>= 11;
  m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
  return __longlong_as_double((long long)(sgn | (((unsigned long long)(E - 1) << 52) + m)));
}

// The integer held by a level accumulator (FP32 bits of an integer below 2^24, exact).  fint22: for values
// within 2^22, adding 1.5 2^23 puts the integer in the low mantissa bits (one FP32 add and one integer subtract
// instead of the conversion instruction).  Real digits keep levels 0 and 1 within 2^22 (64 products of at most
// 2^16, and 2 x 64 of at most 2^15), complex digits levels 0-5 (at most 6 x 128 products of at most 2^13 or
// 2^14).
__device__ __forceinline__ int fint22(uint32_t bits) {
  return (int)(__float_as_uint(__uint_as_float(bits) + 12582912.0f) - 0x4B400000u);
}
__device__ __forceinline__ int level_int(uint32_t bits, int L) {
  return L <= 1 ? fint22(bits) : __float2int_rn(__uint_as_float(bits));
}

// One CTA per 128 x 32 tile of the trailing lower triangle (complex: two CTAs per tile, one per part of A), two
// CTAs per SM, so that one CTA's epilogue (tensor-memory drain, integer recombination, read-modify-write of A)
// overlaps the other's loads and MMAs.  The L digits of the tile stay in shared memory; the W digits stream
// through a ring of NS stages (the MMAs of W digit s pair it with L digits t <= S - 1 - s).
template <bool CPLX>
__global__ void __launch_bounds__(OzCfg<CPLX>::NT, OzCfg<CPLX>::MIN_CTAS) oz_update_kernel(const __grid_constant__ OzMaps maps, void* A_out, int n,
                                                           int k1, const int* __restrict__ ew,
                                                           const int* __restrict__ el, int part, unsigned* status) {
  using C = OzCfg<CPLX>;
  constexpr int S = C::S, BETA = C::BETA, BN = C::BN, NS = C::NS;
  constexpr int Q = K / BN;     // column tiles in the next 64-column block
  constexpr int CT = BM / BN;   // column tiles per 128 rows
  int b = CPLX ? (int)(blockIdx.x >> 1) : (int)blockIdx.x, ti = 0;
  const int pr = CPLX ? (int)(blockIdx.x & 1) : 0;   // part of A this CTA updates: 0 = re, 1 = im
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
  uint8_t* sB = smem;                  // L digits: plane p S + t at p S + t
  uint8_t* sA = smem + C::B_BYTES;     // W-digit ring
  __shared__ __align__(8) uint64_t bar_l, full_bar[NS], empty_bar[NS], bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int l_issued, w_issued, w_consumed;
  __shared__ int exp_w[BM], exp_l[BN];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    mbar_init(&bar_l, 1);
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&bar_done, 1);
    abort_flag = 0;
    l_issued = 0;
    w_issued = 0;
    w_consumed = 0;
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
    // ---- TMA producer: every digit of every part of L, then the W digit planes q = 0 .. WLOADS - 1 (Wr digits,
    // then Wi digits) through the ring
    mbar_expect_tx(&bar_l, (uint32_t)C::B_BYTES);
    for (int p = 0; p < C::NPART; ++p)
      for (int s = 0; s < S; ++s) tma_load_3d(&maps.l, &bar_l, sB + (p * S + s) * C::B_TILE, 0, col0, p * S + s);
    l_issued = 1;
    int q = 0;
    for (; q < C::WLOADS; ++q) {
      const int st = q % NS;
      if (q >= NS && !mbar_wait(&empty_bar[st], (uint32_t)(q / NS - 1) & 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      mbar_expect_tx(&full_bar[st], (uint32_t)C::A_TILE);
      tma_load_3d(&maps.w, &full_bar[st], sA + st * C::A_TILE, 0, row0, q);
    }
    w_issued = q;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: W digit s (part ph) times L digit t of the paired part accumulates in level s + t, columns
    // (s + t) BN.  Real: W L.  Complex, re CTA: Wr Lr - Wi Li (negated-A descriptor); im CTA: Wr Li + Wi Lr.
    bool ok = mbar_wait(&bar_l, 0, &abort_flag);
    int q = 0;
    if (ok) {
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      for (; q < C::WLOADS; ++q) {
        const int st = q % NS;
        if (!mbar_wait(&full_bar[st], (uint32_t)(q / NS) & 1u, &abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int ph = q / S, s = q % S;
        const int lp = CPLX ? (ph ^ pr) : 0;
        const uint32_t neg = (CPLX && ph == 1 && pr == 0) ? NEG_A : 0u;
        // the L digit planes t = 0 .. S - 1 of part lp lie one after another (BN rows each): one MMA of
        // N = BN (S - s) multiplies W digit s by L digits 0 .. S - 1 - s, its accumulator starting at level s
        const uint32_t abase = a0 + st * C::A_TILE, bbase = b0 + lp * S * C::B_TILE;
        const uint32_t idn = idesc_bf16(BM, BN * (S - s)) | neg;
        const uint32_t d = tmem + (uint32_t)(s * BN);
#pragma unroll
        for (int kk = 0; kk < K / 16; ++kk)   // q = 0 (digit 0 of Wr) is the first to reach every level
          umma(d, sdesc(abase + kk * 32), sdesc(bbase + kk * 32), idn, (q > 0 || kk > 0) ? 1u : 0u);
        umma_commit(&empty_bar[st]);   // the stage is free once these MMAs have read it
      }
    }
    w_consumed = q;
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
    // no copy may land after the CTA exits: wait for the L digits and for every W load not consumed
    if (l_issued) mbar_wait(&bar_l, 0, nullptr);
    for (int q = w_consumed; q < w_issued; ++q) mbar_wait(&full_bar[q % NS], (uint32_t)(q / NS) & 1u, nullptr);
  }
  if (good) {
    // Every MMA has completed, so the operand buffers are free: each warp stages its own 32 x 16 block there.
    // Warp w drains tensor-memory lanes 32 (w % 4) .. + 31 (tile rows 32 (w % 4) + lane) and the 16 columns
    // 16 (w / 4) .. + 15 of every level, recombines them exactly, and updates its block of A (part pr), two rows of
    // 16 columns per instruction; no block-wide barrier, so the warps' integer and FP64 phases overlap.
    static_assert(CPLX && S == 8 && BETA == 7 && C::SHIFT == 55 && BN == 32 && C::NT == 256,
                  "recombination written for complex 8 x 7-bit digits, 32-column tiles and eight warps");
    double* Ad = reinterpret_cast<double*>(A_out);
    const int wq = warp & 3, h = warp >> 2;
    const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
    double* stw = reinterpret_cast<double*>(smem) + warp * (32 * 17);
    const int rr = lane >> 4, cc = lane & 15, c0 = col0 + 16 * h;
    // N = sum_L a_L 2^(41 - 7 L): levels 0 and 1 only reach the high word (a_0 2^9 + a_1 2^2 < 2^31), levels 2-5
    // are 32 x 32 -> 64-bit multiply-adds by constant powers of two, levels 6 and 7 are rounded to 2^-1 and 2^-8
    long long acc[16];
    {
      const uint32_t ta = tmem + lane_base + (uint32_t)(16 * h);
      uint32_t v0[16], v1[16];
      tmem_ld16_async(ta + 0 * BN, v0);
      tmem_ld16_async(ta + 1 * BN, v1);
      tmem_wait_ld16(v0, v1);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int hi = fint22(v0[c]) * 512 + fint22(v1[c]) * 4;
        acc[c] = (long long)((unsigned long long)(unsigned)hi << 32);
      }
      tmem_ld16_async(ta + 2 * BN, v0);
      tmem_ld16_async(ta + 3 * BN, v1);
      tmem_wait_ld16(v0, v1);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        acc[c] += (long long)fint22(v0[c]) * (1 << 27) + (long long)fint22(v1[c]) * (1 << 20);
      tmem_ld16_async(ta + 4 * BN, v0);
      tmem_ld16_async(ta + 5 * BN, v1);
      tmem_wait_ld16(v0, v1);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        acc[c] += (long long)fint22(v0[c]) * (1 << 13) + (long long)fint22(v1[c]) * (1 << 6);
      tmem_ld16_async(ta + 6 * BN, v0);
      tmem_ld16_async(ta + 7 * BN, v1);
      tmem_wait_ld16(v0, v1);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        acc[c] += (long long)((__float2int_rn(__uint_as_float(v0[c])) + 1) >> 1) +
                  (long long)((__float2int_rn(__uint_as_float(v1[c])) + 128) >> 8);
    }
    const int kr = exp_w[wq * 32 + lane] - C::SHIFT;
#pragma unroll
    for (int c = 0; c < 16; ++c) stw[lane * 17 + c] = scaled_int64(acc[c], kr + exp_l[16 * h + c]);
    __syncwarp();
    double cv[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int row = row0 + wq * 32 + 2 * i + rr, col = c0 + cc;
      cv[i] = (row < n && col <= row) ? Ad[((long)row * n + col) * 2 + pr] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int row = row0 + wq * 32 + 2 * i + rr, col = c0 + cc;
      if (row < n && col <= row) Ad[((long)row * n + col) * 2 + pr] = cv[i] - stw[(2 * i + rr) * 17 + cc];
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

// ---- real trailing update by row strips -----------------------------------------------------------------------
// One CTA per chunk of up to `chunk` consecutive 128 x 32 tiles of one 128-row strip (real A).  The strip's seven
// W digit planes (112 KB) are loaded once and stay in shared memory; the L digits of successive tiles (28 KB each)
// and their tensor-memory accumulators (7 levels x 32 columns) are double-buffered, so the MMAs of tile j + 1 run
// while the epilogue warps drain, recombine and write tile j.  640 threads: warp 0 issues TMA, warp 1 the MMAs,
// warps 4-19 form the epilogue (they stage the FP64 update in shared memory and update A with coalesced row
// segments).
constexpr int SBN = 32;                            // tile columns
constexpr int SS = 7, SBETA = 8, SSHIFT = 56;      // real digits (as OzCfg<false>)
constexpr int S_WB = SS * BM * ROWB;               // the strip's W digits: 112 KB
constexpr int S_LB = SS * SBN * ROWB;              // one tile's L digits: 28 KB
constexpr int S_SLD = 9;                           // staging row stride (doubles): 8 columns + 1
constexpr int S_STG = 16 * 32 * S_SLD * 8;         // a 32 x 8 slot per epilogue warp: 36 KB
constexpr int S_SMEM = S_WB + 2 * S_LB + S_STG + 1024;
constexpr int S_ACC = 256;                         // tensor-memory columns per accumulator set (224 used)

// Tiles of the trailing lower triangle handled by block b: strip ti, first column tile, count (0: nothing).
__device__ inline void strip_chunk(int b, int part, int chunk, int& ti, int& first, int& count) {
  constexpr int Q = K / SBN, CT = BM / SBN;
  int cnt = 0;
  for (ti = 0; ti < (1 << 20); ++ti) {
    cnt = part == 1 ? Q : (part == 0 ? CT * (ti + 1) : CT * (ti + 1) - Q);
    const int nch = (cnt + chunk - 1) / chunk;
    if (b < nch) break;
    b -= nch;
  }
  first = (part == 2 ? Q : 0) + b * chunk;
  count = min(chunk, cnt - b * chunk);
}

__global__ void __launch_bounds__(640, 1) oz_strip_kernel(const __grid_constant__ OzMaps maps, double* __restrict__ A,
                                                          int n, int k1, const int* __restrict__ ew,
                                                          const int* __restrict__ el, int part, int chunk,
                                                          unsigned* status) {
  int ti, first, count;
  strip_chunk(blockIdx.x, part, chunk, ti, first, count);
  const int row0 = k1 + ti * BM;
  count = min(count, (n - k1 + SBN - 1) / SBN - first);   // column tiles past n (ragged last strip) are skipped
  if (row0 >= n || count <= 0) return;   // the whole CTA leaves before any barrier or allocation

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sW = smem;
  uint8_t* sL = smem + S_WB;                                       // two buffers of S_LB
  double* stage = reinterpret_cast<double*>(smem + S_WB + 2 * S_LB);
  __shared__ __align__(8) uint64_t bar_w, lfull[2], lempty[2], afull[2], aempty[2], bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int w_issued, l_issued;
  __shared__ int exp_w[BM];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    mbar_init(&bar_w, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&lfull[i], 1);
      mbar_init(&lempty[i], 1);
      mbar_init(&afull[i], 1);
      mbar_init(&aempty[i], 16);
    }
    mbar_init(&bar_done, 1);
    abort_flag = 0;
    w_issued = 0;
    l_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int r = threadIdx.x; r < BM; r += blockDim.x) exp_w[r] = row0 + r < n ? ew[row0 + r] : 0;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(2u * S_ACC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer: the strip's W digits once, then the L digits of each tile into buffer j % 2
    mbar_expect_tx(&bar_w, (uint32_t)S_WB);
    for (int s = 0; s < SS; ++s) tma_load_3d(&maps.w, &bar_w, sW + s * (BM * ROWB), 0, row0, s);
    w_issued = 1;
    int j = 0;
    for (; j < count; ++j) {
      const int lb = j & 1;
      if (j >= 2 && !mbar_wait(&lempty[lb], (uint32_t)(j / 2 - 1) & 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      mbar_expect_tx(&lfull[lb], (uint32_t)S_LB);
      const int col0 = k1 + (first + j) * SBN;
      for (int t = 0; t < SS; ++t) tma_load_3d(&maps.l, &lfull[lb], sL + lb * S_LB + t * (SBN * ROWB), 0, col0, t);
    }
    l_issued = j;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: tile j's level s + t in columns (j % 2) S_ACC + (s + t) SBN
    bool ok = mbar_wait(&bar_w, 0, &abort_flag);
    const uint32_t w0 = smem_u32(sW);
    for (int j = 0; ok && j < count; ++j) {
      const int ab = j & 1;
      if (j >= 2 && !mbar_wait(&aempty[ab], (uint32_t)(j / 2 - 1) & 1u, &abort_flag)) {
        ok = false;
        break;
      }
      if (!mbar_wait(&lfull[ab], (uint32_t)(j / 2) & 1u, &abort_flag)) {
        ok = false;
        break;
      }
      tc_fence_after();
      // The L digit planes t = 0 .. 6 lie one after another in shared memory (32 rows each), so one MMA of
      // N = 32 (7 - s) multiplies W digit s by L digits 0 .. 6 - s at once; its accumulator starts at level s,
      // so the product with L digit t lands in level s + t.
      const uint32_t l0 = smem_u32(sL + ab * S_LB);
#pragma unroll
      for (int s = 0; s < SS; ++s) {
        const uint32_t id = idesc_bf16(BM, SBN * (SS - s));
        const uint32_t d = tmem + (uint32_t)(ab * S_ACC + s * SBN);
#pragma unroll
        for (int kk = 0; kk < K / 16; ++kk)   // digit 0 of W is the first to reach every level
          umma(d, sdesc(w0 + s * (BM * ROWB) + kk * 32), sdesc(l0 + kk * 32), id, (s > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(&lempty[ab]);   // the L buffer is free once these MMAs have read it
      umma_commit(&afull[ab]);    // and the accumulators are complete
    }
    if (!ok) abort_flag = 1;
    umma_commit(&bar_done);   // arrives once every MMA issued above has completed
  } else if (warp >= 4) {
    // ---- epilogue: sixteen independent warps (no block-wide barrier, so that warps in their integer phase
    // overlap warps in their FP64 phase); warp 4 + e drains tensor-memory lanes 32 (e % 4) .. + 31 (tile rows
    // 32 (e % 4) + lane) and the 8 columns 8 (e / 4) .. + 7 of every level, stages that 32 x 8 block in its own
    // shared-memory slot and updates it in A, four rows of 64 contiguous bytes per instruction.
    const int e = warp - 4, wq = warp & 3, h = e >> 2;
    const uint32_t lane_base = (uint32_t)(wq * 32) << 16;
    const int kr = exp_w[wq * 32 + lane] - SSHIFT;
    double* st = stage + e * (32 * S_SLD);
    const int rr = lane >> 3, cc = lane & 7;   // read-modify-write: rows 4 i + rr, column cc of the block
    bool ok = true;
    for (int j = 0; j < count; ++j) {
      const int ab = j & 1;
      const int c0 = k1 + (first + j) * SBN + 8 * h;   // first column of this warp's block
      // A values of the block first: their latency hides behind the wait and the recombination
      double cv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int row = row0 + wq * 32 + 4 * i + rr, col = c0 + cc;
        cv[i] = (ok && row < n && col <= row) ? A[(long)row * n + col] : 0.0;
      }
      int el8[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) el8[c] = c0 + c < n ? __ldg(el + c0 + c) : 0;
      if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&afull[ab], (uint32_t)(j / 2) & 1u, &abort_flag));
      tc_fence_after();
      long long acc[8];
      if (ok) {
        // exact integer recombination N = sum_L a_L 2^(40 - 8 L) (SSHIFT = 56, SBETA = 8): levels 0 and 1 only
        // reach the high word (a_0 2^8 + a_1 < 2^31), levels 2-5 are 32 x 32 -> 64-bit multiply-adds by
        // constant powers of two, level 6 is rounded to 2^-8
        static_assert(SSHIFT == 56 && SBETA == 8 && SS == 7, "recombination written for 7 x 8-bit digits");
        const uint32_t ta = tmem + lane_base + (uint32_t)(ab * S_ACC + 8 * h);
        uint32_t v[32];
        tmem_ld8_at<0>(ta + 0 * SBN, v);
        tmem_ld8_at<8>(ta + 1 * SBN, v);
        tmem_ld8_at<16>(ta + 2 * SBN, v);
        tmem_ld8_at<24>(ta + 3 * SBN, v);
        tmem_wait_ld1(v);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int hi = level_int(v[c], 0) * 256 + level_int(v[8 + c], 1);
          acc[c] = (long long)((unsigned long long)(unsigned)hi << 32) + (long long)level_int(v[16 + c], 2) * (1 << 24) +
                   (long long)level_int(v[24 + c], 3) * (1 << 16);
        }
        tmem_ld8_at<0>(ta + 4 * SBN, v);
        tmem_ld8_at<8>(ta + 5 * SBN, v);
        tmem_ld8_at<16>(ta + 6 * SBN, v);
        tmem_wait_ld1(v);
#pragma unroll
        for (int c = 0; c < 8; ++c)
          acc[c] += (long long)level_int(v[c], 4) * (1 << 8) + (long long)level_int(v[8 + c], 5) +
                    (long long)((level_int(v[16 + c], 6) + 128) >> 8);
      }
      tc_fence_before();
      __syncwarp();
      if (ok && lane == 0) mbar_arrive(&aempty[ab]);   // the MMAs of tile j + 2 may overwrite this set
      if (ok) {
#pragma unroll
        for (int c = 0; c < 8; ++c) st[lane * S_SLD + c] = scaled_int64(acc[c], kr + el8[c]);
      }
      __syncwarp();
      if (ok) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int row = row0 + wq * 32 + 4 * i + rr, col = c0 + cc;
          if (row < n && col <= row) A[(long)row * n + col] = cv[i] - st[(4 * i + rr) * S_SLD + cc];
        }
      }
      __syncwarp();   // the slot is read before the next tile overwrites it
    }
    if (!ok) abort_flag = 1;
  }
  __syncwarp();

  const bool done_ok = mbar_wait(&bar_done, 0, nullptr);
  tc_fence_after();
  const bool good = __syncthreads_and(done_ok ? 1 : 0) && !abort_flag;
  if (threadIdx.x == 0 && !good) {
    raise_status(status, DEV_ERR_TIMEOUT);
    // no copy may land after the CTA exits: the W digits and the (at most two) L loads not known to be consumed
    if (w_issued) mbar_wait(&bar_w, 0, nullptr);
    for (int j = l_issued > 2 ? l_issued - 2 : 0; j < l_issued; ++j)
      mbar_wait(&lfull[j & 1], (uint32_t)(j / 2) & 1u, nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * S_ACC) : "memory");
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
  if constexpr (!CPLX) {
    // row strips in chunks of about tiles / (SMs x upd_waves) tiles: upd_waves waves of CTAs (1 unless the batch
    // autotuner chose more), each loading its W digits once
    const long mbs = (rows + BM - 1) / BM, cts = BM / SBN, qs = K / SBN;
    const long all = cts * mbs * (mbs + 1) / 2;
    const long tiles = part == 0 ? all : (part == 1 ? qs * mbs : all - qs * mbs);
    if (tiles <= 0) return CDWAC_OK;
    const long slots = (long)ctx->num_sms * std::max(1, std::min(8, ctx->upd_waves));
    const int chunk = (int)std::min<long>(32, std::max<long>(1, (tiles + slots - 1) / slots));
    long grid = 0;
    for (long t = 0; t < mbs; ++t) {
      const long cnt = part == 1 ? qs : (part == 0 ? cts * (t + 1) : cts * (t + 1) - qs);
      grid += (cnt + chunk - 1) / chunk;
    }
    OzMaps maps;
    maps.w = plan.wmap[buf];
    maps.l = plan.lmap[buf];
    CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(oz_strip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, S_SMEM));
    oz_strip_kernel<<<(unsigned)grid, 640, S_SMEM, st>>>(maps, reinterpret_cast<double*>(A), n, k1, plan.ew[buf],
                                                         plan.el[buf], part, chunk, ctx->d_status);
    CDWAC_LAUNCH_CHECK(ctx);
    return CDWAC_OK;
  } else {
  const long mb = (rows + BM - 1) / BM, ct = BM / C::BN, q = K / C::BN;
  const long all = ct * mb * (mb + 1) / 2;
  const long tiles = part == 0 ? all : (part == 1 ? q * mb : all - q * mb);
  if (tiles <= 0) return CDWAC_OK;
  const long grid = tiles * C::NPART;   // complex: one CTA per part of A
  OzMaps maps;
  maps.w = plan.wmap[buf];
  maps.l = plan.lmap[buf];
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(oz_update_kernel<CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           C::SMEM));
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(oz_update_kernel<CPLX>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                           (int)cudaSharedmemCarveoutMaxShared));
  oz_update_kernel<CPLX><<<(unsigned)grid, C::NT, C::SMEM, st>>>(maps, A, n, k1, plan.ew[buf], plan.el[buf], part,
                                                              ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
  }
}

template cdwac_status ozaki_slice<double>(cdwac_ctx*, const OzakiPlan&, int, const double*, int, int, const double*,
                                          cudaStream_t);
template cdwac_status ozaki_slice<cplx>(cdwac_ctx*, const OzakiPlan&, int, const cplx*, int, int, const cplx*,
                                        cudaStream_t);
template cdwac_status ozaki_update<double>(cdwac_ctx*, const OzakiPlan&, int, double*, int, int, int, cudaStream_t);
template cdwac_status ozaki_update<cplx>(cdwac_ctx*, const OzakiPlan&, int, cplx*, int, int, int, cudaStream_t);
