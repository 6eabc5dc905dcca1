// Mixed-precision polarizability on the 5th-generation tensor cores (tcgen05), GB300 / sm_103a.
//
//   A = I - Pi(z),  Pi(z) = B diag(w(z)) B^T,  w = 2 [1/(z - D) - 1/(z + D)] = 4 D / (z^2 - D^2)   (Eq. piriv)
//
// The weight is folded into one operand: S = B diag(-w) (per column ia), so that A = I + S B^T.  Each of S and B is
// split into BF16 planes hi + lo (hi = bf16(x), lo = bf16(x - hi)) and the product is formed from three BF16
// products hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory (the lo*lo term, ~2^-16 relative, is
// dropped).  On the imaginary axis -w = 4 D / (xi^2 + D^2) > 0; for complex z the real and imaginary parts of -w
// give two weighted operands, whose contractions write the real and the imaginary parts of A.
//
// Two kernels: `tc_syrk256_kernel` on 128 x 256 tiles (the default; described at its definition) and
// `tc_syrk_kernel` on 128 x 128 tiles (the batch autotuner's alternative), described here.
//
// tc_syrk_kernel: one CTA per 128 x 128 tile of the lower triangle of A (A is symmetric), 384 threads.  Warp 0 lane 0
// drives TMA (cp.async.bulk.tensor, 128-byte swizzle) through a ring of shared-memory stages; warp 1 owns the
// tensor memory and lane 0 issues tcgen05.mma (M = N = 128, K = 16 per instruction, both operands K-major);
// tcgen05.commit releases a stage when the MMAs reading it finish.  The hi*hi products of every K-tile (one buffer
// per operand stage, in turn) and the corrections of every 32 K-tiles go to fresh accumulators in tensor memory;
// warps 4-11 read each finished one (tcgen05.ld 32x32b, the accumulator rows they own), add it into FP32 running
// sums and at the end write A in FP64.  Every wait on an mbarrier is bounded (5 s): on expiry the kernel records
// CDWAC_ERR_TIMEOUT, stops issuing, drains what it issued and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <string.h>

#include "tc_pi.cuh"
#include "tcgen05.cuh"

namespace {
using namespace tc;

constexpr int BM = 128, BK = 64;                     // tile rows and K-tile width
constexpr int PLANE = BM * BK * 2;                       // bytes of one 128 x 64 BF16 operand tile
struct Maps {
  CUtensorMap sh, sl, bh, bl;   // planes of the weighted operand S and of B
};

__device__ inline void lower_tile_coords(int b, int& ti, int& tj) {
  int t = int((sqrt(8.0 * b + 1.0) - 1.0) * 0.5);
  while ((t + 1) * (t + 2) / 2 <= b) ++t;
  while (t * (t + 1) / 2 > b) --t;
  ti = t;
  tj = b - t * (t + 1) / 2;
}

// Tile b of the lower triangle of nt x nt tiles, in groups of G x G tiles (lower-triangle order of the groups,
// row-major inside a group): the CTAs of one wave then share about 2G operand row blocks, so that each K-slice of
// them comes from DRAM once per wave instead of once per row block of the whole triangle.  G is the context's
// pi_group (12 unless the batch autotuner chose another).
__device__ inline void grouped_tile_coords(int b, int nt, int G, int& ti, int& tj) {
  const int ns = (nt + G - 1) / G;
  int rem = b;
  for (int I = 0; I < ns; ++I) {
    const int rI = min(G, nt - I * G);
    for (int J = 0; J <= I; ++J) {
      const int cJ = min(G, nt - J * G);
      const int cnt = J < I ? rI * cJ : rI * (rI + 1) / 2;
      if (rem < cnt) {
        if (J < I) {
          ti = I * G + rem / cJ;
          tj = J * G + rem % cJ;
        } else {
          int r, c;
          lower_tile_coords(rem, r, c);
          ti = I * G + r;
          tj = J * G + c;
        }
        return;
      }
      rem -= cnt;
    }
  }
  ti = tj = nt;   // past the triangle: not reached for b < nt (nt + 1) / 2
}

// Accumulation in chunks.  The FP32 accumulation of the tensor cores is not unbiased over a long chain: each
// instruction that adds into an accumulator loses a fraction of an ulp of it, always towards zero.  Summed over all
// K = 129 600 columns of the acene-like system (8100 K-steps of three products into one accumulator) Pi came out
// about 1.2e-3 too small in magnitude, a bias that survives in W at large xi.  So the hi*hi products of every
// K-tile (64 columns, a chain of four instructions) go to a fresh accumulator, one per operand stage in turn, and
// the hi*lo + lo*hi corrections (2^-8 of the size, so a chain of 32 K-tiles biases Pi by less than 1e-7) to one
// more refreshed every CORR K-tiles; the drain warps add every finished accumulator into FP32 running sums with
// round-to-nearest adds on the CUDA cores while the MMAs fill the others.  The drain needs no commit of its own:
// the one that frees a K-tile's operand stage also marks its accumulators complete.
constexpr int CORR = 32;  // K-tiles per correction accumulator (one buffer)

constexpr int BN = 128;                            // tile columns
constexpr int STAGE = 4 * PLANE;                   // S hi, S lo, B hi, B lo of one K-tile
constexpr int STAGES = 3;
constexpr int SMEM = STAGES * STAGE + 1024;        // + alignment slack
constexpr int NHH = STAGES;                        // hi*hi accumulator buffers, one per operand stage
constexpr int TMEM_COLS = (NHH + 1) * BN;          // and the correction accumulator: 512 columns

// A = I + S B^T, lower triangle, written as `part`: -1 the real matrix A (double*), 0 the real parts of a complex
// matrix (cplx*, with the identity), 1 its imaginary parts (without it); a complex Pi(z) is two launches, one per
// weight (two 128 x 128 real contractions keep the full-width instructions and the drain's 128 running sums).
// Warps: 0 = TMA producer (lane 0), 1 = tensor-memory owner and MMA issuer (lane 0), 4..11 = two drain warpgroups
// (warp w reads tensor-memory lanes 32 (w % 4) .. + 31, the tile rows it later writes); 2, 3 idle.
__global__ void __launch_bounds__(384, 1) tc_syrk_kernel(const __grid_constant__ Maps maps, int n, int k_tiles,
                                                         int group, void* A_out, int part, float* negpi32,
                                                         unsigned* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t hh_empty[NHH], cr_empty;
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int issued, consumed;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nt = (n + BM - 1) / BM;
  int ti, tj;
  grouped_tile_coords(blockIdx.x, nt, group, ti, tj);
  const int row0 = ti * BM, col0 = tj * BN;
  if (col0 >= n) return;   // past the triangle: the whole CTA leaves before any barrier or allocation

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
    // ---- TMA producer
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
      const int x = kt * BK;
      tma_load_2d(&maps.sh, &full_bar[s], st + 0 * PLANE, x, row0);
      tma_load_2d(&maps.sl, &full_bar[s], st + 1 * PLANE, x, row0);
      tma_load_2d(&maps.bh, &full_bar[s], st + 2 * PLANE, x, col0);
      tma_load_2d(&maps.bl, &full_bar[s], st + 3 * PLANE, x, col0);
    }
    issued = kt;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: K-tile kt puts its hi*hi products in hh buffer kt % NHH and its corrections in the
    // correction buffer (group g = kt / CORR); tensor-memory columns [hh0 | hh1 | hh2 | cr], BN each
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    int kt = 0;
    for (; kt < k_tiles; ++kt) {
      const int s = kt % STAGES;
      const uint32_t ph = (uint32_t)(kt / STAGES) & 1u;
      const int hb = kt % NHH, g = kt / CORR;
      const bool g_first = kt % CORR == 0;
      // the drain must have read a buffer's previous contents before it is overwritten
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
      for (int kk = 0; kk < BK / 16; ++kk)   // 16 BF16 = 32 bytes along K inside the 128-byte swizzle row
        umma(dh, sdesc(base + 0 * PLANE + kk * 32), sdesc(base + 2 * PLANE + kk * 32), idesc, kk == 0 ? 0u : 1u);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t ko = kk * 32;
        umma(dc, sdesc(base + 0 * PLANE + ko), sdesc(base + 3 * PLANE + ko), idesc, (g_first && kk == 0) ? 0u : 1u);
        umma(dc, sdesc(base + 1 * PLANE + ko), sdesc(base + 2 * PLANE + ko), idesc, 1u);
      }
      umma_commit(&empty_bar[s]);
    }
    consumed = kt;
    umma_commit(&done_bar);   // arrives once every MMA issued above has completed
  } else if (warp >= 4) {
    // ---- drain: two warpgroups; group g (warps 4 + 4g .. 7 + 4g) sums columns [64 g, 64 g + 64) of every
    // accumulator into FP32 running sums with round-to-nearest adds; warp w reads tensor-memory lanes
    // 32 (w % 4) .. + 31, the tile rows it owns
    const int g = (warp - 4) >> 2, q = warp & 3;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    constexpr int HALF = BN / 2;
    float run[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) run[j] = 0.f;
    bool ok = true;
    // adds accumulator `set` (0 .. NHH - 1: hi*hi buffers; NHH: the correction buffer) into the running sums
    auto drain = [&](uint64_t* empty, int set) {
      tc_fence_after();
      tmem_add64(tmem + lane_base + (uint32_t)(set * BN + g * HALF), run);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(empty);
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
    if (!ok) abort_flag = 1;
    // every drain warp is done (a timeout in one ends the others' bounded waits too); the verdict is the AND over
    // the eight drain warps, the same in all of them, so the barrier below is reached by all or none
    if (drain_and256(ok && !abort_flag)) {
      // The last drain means every MMA has completed and every operand stage has been consumed, so the operand
      // ring is free: the tile is staged there (row stride BN + 1 floats: conflict-free both ways) and written
      // out as coalesced row segments, this warp's 32 rows and its group's 64 columns.
      constexpr int LDS = BN + 1;
      float* stg = reinterpret_cast<float*>(smem);
#pragma unroll
      for (int j = 0; j < HALF; ++j) stg[(q * 32 + lane) * LDS + g * HALF + j] = run[j];
      drain_bar();
      const int c_lo = g * HALF;
      for (int rr = 0; rr < 32; ++rr) {
        const int row = row0 + q * 32 + rr;
        if (row >= n) break;
        const float* src = stg + (q * 32 + rr) * LDS;
        for (int j = c_lo + lane; j < c_lo + HALF; j += 32) {
          const int col = col0 + j;
          if (col > row || col >= n) continue;
          const double diag = col == row ? 1.0 : 0.0;
          if (part < 0) {
            reinterpret_cast<double*>(A_out)[(long)row * n + col] = diag + (double)src[j];
            if (negpi32) negpi32[(long)row * n + col] = src[j];   // -Pi in FP32 for the Pi O product
          } else {
            double* Ac = reinterpret_cast<double*>(A_out) + 2 * ((long)row * n + col) + part;
            *Ac = (part == 0 ? diag : 0.0) + (double)src[j];
          }
        }
      }
      if (part < 0 && negpi32) {
        // the transposed (upper) entries: the 32 lanes hold consecutive rows, so every store is coalesced
        const int row = row0 + q * 32 + lane;
        for (int j = c_lo; j < c_lo + HALF; ++j) {
          const int col = col0 + j;
          if (row < n && col < row) negpi32[(long)col * n + row] = stg[(q * 32 + lane) * LDS + j];
        }
      }
    }
  }
  __syncwarp();

  // every MMA issued has completed before the tensor memory is released, on every path
  const bool done_ok = mbar_wait(&done_bar, 0, nullptr);
  tc_fence_after();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!done_ok || abort_flag) {
      raise_status(status, DEV_ERR_TIMEOUT);
      // drain loads that were issued but never consumed, so no copy lands after the CTA exits
      for (int kt = consumed; kt < issued; ++kt)
        mbar_wait(&full_bar[kt % STAGES], (uint32_t)(kt / STAGES) & 1u, nullptr);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TMEM_COLS)
                 : "memory");
  }
}

// ---- 128 x 256 tiles ---------------------------------------------------------------------------------------------
// The same contraction on 128 x 256 output tiles with 32-column K-tiles (64-byte swizzle).  Each 128 x 256 x 16
// MMA reads 4 KB of S and 8 KB of B from shared memory for twice the work of a 128 x 128 one, and a K-tile brings
// 48 KB by TMA for 6 MMAs of 256 columns; at the tensor cores' rate per SM that is about 150 B of shared-memory
// traffic per cycle against about 210 for the 128 x 128 kernel, whose operand reads plus TMA fills exceed the
// shared memory's bandwidth.
// Accumulation: every two K-tiles form one chain of twelve instructions in a fresh 256-column tensor-memory
// accumulator, two accumulators in turn (all 512 columns); each K-tile issues its hi*lo and lo*hi corrections
// first and its two hi*hi products last.  The tensor cores' accumulation loses a fraction of an ulp of the
// accumulator towards zero per instruction; in this order a chain's bias stays near 4.5 x 2^-25 of its value
// (1.3e-7; chains of one K-tile's four hi*hi instructions: 2.5 x 2^-25), and the acene-like core QP energy moves
// by 0.03 meV (0.20 -> 0.23 meV from the FP64 oracle, W(i xi) within 5.4e-7).
// Sixteen drain warps (warps 2-17: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 and the 64 columns
// 64 ((w - 2) / 4) .. + 63) add each finished chain into FP32 running sums with round-to-nearest adds while the
// MMAs fill the other accumulator: a drain has two K-tiles (12 MMAs) of time, where a single hi*hi accumulator
// beside a correction accumulator left it the four correction MMAs of one K-tile and stalled the tensor cores.  Lower triangle:
// tile (ti, tp) covers rows 128 ti .. + 127 and columns 256 tp .. + 255 with 2 tp <= ti; entries above the
// diagonal are computed and not written.
namespace w256 {
constexpr int BM = 128, BN = 256, BK = 32;
constexpr int SPL = BM * BK * 2;           // one S plane of a K-tile: 128 rows x 64 B = 8 KB
constexpr int BPL = BN * BK * 2;           // one B plane of a K-tile: 256 rows x 64 B = 16 KB
constexpr int STAGE = 2 * SPL + 2 * BPL;   // S hi, S lo, B hi, B lo: 48 KB
constexpr int STAGES = 4;
constexpr int SMEM = STAGES * STAGE + 1024;
constexpr int NT = 576;                    // warps 0 (TMA), 1 (MMA, tensor memory), 2-17 (drain)
constexpr int NDRAIN = 16;
constexpr int LDS = BN + 1;                // staging row stride (floats)
static_assert(BM * LDS * 4 <= STAGES * STAGE, "the staged tile fits in the operand ring");
}  // namespace w256

// Shared-memory descriptor for a K-major operand in the 64-byte swizzle layout written by TMA: rows of 64 B,
// 8-row groups 512 B apart (stride byte offset), version 1, layout type 4 (64-byte swizzle).
__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Tile b of the lower triangle of 128 x 256 tiles: groups of G row blocks; inside a group, column pairs tp in
// order and the group's rows ti >= 2 tp inside each.
__device__ inline void tile256_coords(int b, int nt, int G, int& ti, int& tp) {
  for (int r0 = 0; r0 < nt; r0 += G) {
    const int r1 = min(nt, r0 + G);
    for (int p = 0; 2 * p <= r1 - 1; ++p) {
      const int first = max(r0, 2 * p), cnt = r1 - first;
      if (cnt <= 0) continue;
      if (b < cnt) {
        ti = first + b;
        tp = p;
        return;
      }
      b -= cnt;
    }
  }
  ti = nt;
  tp = 0;
}

__host__ inline int tiles256(int nt) {
  int t = 0;
  for (int ti = 0; ti < nt; ++ti) t += ti / 2 + 1;
  return t;
}

__device__ __forceinline__ void drain_bar512() { asm volatile("bar.sync 1, 512;" ::: "memory"); }
// Named barrier 1 over the sixteen drain warps that also returns the AND of `v` over their threads.
__device__ __forceinline__ bool drain_and512(bool v) {
  uint32_t r;
  asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred p, 1, 512, p;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(r)
               : "r"((uint32_t)v)
               : "memory");
  return r != 0;
}

// part >= 0 (complex A): blocks [0, tiles) write the real parts with the weighted planes of `maps`, blocks
// [tiles, 2 tiles) the imaginary parts with those of `maps_im` (one launch for both contractions).
__global__ void __launch_bounds__(w256::NT, 1) tc_syrk256_kernel(const __grid_constant__ Maps maps,
                                                                const __grid_constant__ Maps maps_im, int tiles,
                                                                int n, int k_tiles, int group, void* A_out, int part,
                                                                float* negpi32, unsigned* status) {
  constexpr int BM = w256::BM, BN = w256::BN, BK = w256::BK, SPL = w256::SPL, BPL = w256::BPL;
  constexpr int STAGE = w256::STAGE, STAGES = w256::STAGES, NDRAIN = w256::NDRAIN, LDS = w256::LDS;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ int issued, consumed;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nt = (n + BM - 1) / BM;
  const bool second = part >= 0 && (int)blockIdx.x >= tiles;
  if (part >= 0) part = second ? 1 : 0;
  const Maps* mp = second ? &maps_im : &maps;
  int ti, tp;
  tile256_coords(second ? (int)blockIdx.x - tiles : (int)blockIdx.x, nt, group, ti, tp);
  const int row0 = ti * BM, col0 = tp * BN;
  if (row0 >= n) return;   // past the triangle: the whole CTA leaves before any barrier or allocation

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], NDRAIN);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    issued = 0;
    consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int kt = 0;
    for (; kt < k_tiles; ++kt) {
      const int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)(kt / STAGES - 1) & 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      mbar_expect_tx(&full_bar[s], (uint32_t)STAGE);
      uint8_t* st = smem + s * STAGE;
      const int x = kt * BK;
      tma_load_2d(&mp->sh, &full_bar[s], st, x, row0);
      tma_load_2d(&mp->sl, &full_bar[s], st + SPL, x, row0);
      tma_load_2d(&mp->bh, &full_bar[s], st + 2 * SPL, x, col0);
      tma_load_2d(&mp->bl, &full_bar[s], st + 2 * SPL + BPL, x, col0);
    }
    issued = kt;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer: K-tiles 2c and 2c + 1 form chain c in accumulator c % 2 (columns 256 (c % 2) ..)
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    int kt = 0;
    for (; kt < k_tiles; ++kt) {
      const int s = kt % STAGES, c = kt >> 1, ab = c & 1;
      const bool c_first = (kt & 1) == 0, c_last = (kt & 1) == 1 || kt == k_tiles - 1;
      if (!mbar_wait(&full_bar[s], (uint32_t)(kt / STAGES) & 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      // the drain must have read this accumulator's previous chain (chain c - 2)
      if (c_first && c >= 2 && !mbar_wait(&acc_empty[ab], (uint32_t)(c / 2 - 1) & 1u, &abort_flag)) {
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t base = smem_u32(smem + s * STAGE);
      const uint32_t ah = base, al = base + SPL, bh = base + 2 * SPL, bl = base + 2 * SPL + BPL;
      const uint32_t d = tmem + (uint32_t)(256 * ab);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {   // 16 BF16 = 32 bytes along K inside the 64-byte swizzle row
        const uint32_t ko = kk * 32;
        umma(d, sdesc64(ah + ko), sdesc64(bl + ko), idesc, (c_first && kk == 0) ? 0u : 1u);
        umma(d, sdesc64(al + ko), sdesc64(bh + ko), idesc, 1u);
      }
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) umma(d, sdesc64(ah + kk * 32), sdesc64(bh + kk * 32), idesc, 1u);
      if (c_last) umma_commit(&acc_full[ab]);
      umma_commit(&empty_bar[s]);
    }
    consumed = kt;
    umma_commit(&done_bar);   // arrives once every MMA issued above has completed
  } else if (warp >= 2 && warp < 2 + NDRAIN) {
    // ---- drain: sixteen warps; warp w reads lanes 32 (w % 4) .. + 31 and columns 64 cg .. + 63 of each chain
    const int q = warp & 3, cg = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    float run[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) run[j] = 0.f;
    bool ok = true;
    const int n_chains = (k_tiles + 1) / 2;
    for (int c = 0; c < n_chains; ++c) {
      const int ab = c & 1;
      // accumulator ab's next phase needs this drain's arrival first, so the phase cannot pass unobserved
      ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[ab], (uint32_t)(c / 2) & 1u, &abort_flag));
      if (!ok) break;
      tc_fence_after();
#pragma unroll
      for (int i = 0; i < 4; ++i) {   // one 16-column load at a time: the 64 running sums leave no room for more
        uint32_t v[16];
        tmem_ld16_async(tmem + lane_base + (uint32_t)(256 * ab + 64 * cg + 16 * i), v);
        tmem_wait_ld16(v, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) run[16 * i + j] += __uint_as_float(v[j]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
    }
    if (!ok) abort_flag = 1;
    // every drain warp is done (a timeout in one ends the others' bounded waits too); the verdict is the AND over
    // the sixteen warps, the same in all of them, so the barriers below are reached by all or none
    if (drain_and512(ok && !abort_flag)) {
      // the last chain's commit follows every MMA, so the operand ring is free: stage the tile (row stride
      // BN + 1 floats) and write it out as coalesced row segments
      float* stg = reinterpret_cast<float*>(smem);
#pragma unroll
      for (int j = 0; j < 64; ++j) stg[(q * 32 + lane) * LDS + 64 * cg + j] = run[j];
      drain_bar512();
      const int e = warp - 2;   // rows 8 e .. 8 e + 7 of the tile
      for (int rr = 0; rr < 8; ++rr) {
        const int row = row0 + 8 * e + rr;
        if (row >= n) break;
        const float* src = stg + (8 * e + rr) * LDS;
        for (int j = lane; j < BN; j += 32) {
          const int col = col0 + j;
          if (col > row || col >= n) continue;
          const double diag = col == row ? 1.0 : 0.0;
          if (part < 0) {
            reinterpret_cast<double*>(A_out)[(long)row * n + col] = diag + (double)src[j];
            if (negpi32) negpi32[(long)row * n + col] = src[j];   // -Pi in FP32 for the Pi O product
          } else {
            double* Ac = reinterpret_cast<double*>(A_out) + 2 * ((long)row * n + col) + part;
            *Ac = (part == 0 ? diag : 0.0) + (double)src[j];
          }
        }
      }
      if (part < 0 && negpi32) {
        // the transposed (upper) entries: the 32 lanes hold consecutive rows, so every store is coalesced
        const int row = row0 + q * 32 + lane;
        for (int j = 64 * cg; j < 64 * cg + 64; ++j) {
          const int col = col0 + j;
          if (row < n && col < row) negpi32[(long)col * n + row] = stg[(q * 32 + lane) * LDS + j];
        }
      }
    }
  }
  __syncwarp();

  // every MMA issued has completed before the tensor memory is released, on every path
  const bool done_ok = mbar_wait(&done_bar, 0, nullptr);
  tc_fence_after();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!done_ok || abort_flag) {
      raise_status(status, DEV_ERR_TIMEOUT);
      for (int kt = consumed; kt < issued; ++kt)
        mbar_wait(&full_bar[kt % STAGES], (uint32_t)(kt / STAGES) & 1u, nullptr);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
  }
}

// ---- operand preparation (HBM-bound elementwise passes) ---------------------------------------------------------

__device__ __forceinline__ void split8(const float (&v)[8], uint4& hi, uint4& lo) {
  __nv_bfloat16 h[8], l[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    h[j] = __float2bfloat16_rn(v[j]);
    l[j] = __float2bfloat16_rn(v[j] - __bfloat162float(h[j]));
  }
  hi = *reinterpret_cast<uint4*>(h);
  lo = *reinterpret_cast<uint4*>(l);
}

template <class TIn>
__device__ __forceinline__ void load8(const TIn* row, long k, long n_ov, float (&v)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = (k + j < n_ov) ? (float)row[k + j] : 0.f;
}

// B -> hi/lo planes [n][kpad] (zero padded along K)
template <class TIn>
__global__ void split_kernel(const TIn* __restrict__ B, int n, long n_ov, long kpad, __nv_bfloat16* __restrict__ hi,
                             __nv_bfloat16* __restrict__ lo) {
  const long chunks = kpad / 8, total = (long)n * chunks;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < total; c += (long)gridDim.x * blockDim.x) {
    const long r = c / chunks, k = (c % chunks) * 8;
    float v[8];
    load8(B + r * n_ov, k, n_ov, v);
    uint4 h, l;
    split8(v, h, l);
    *reinterpret_cast<uint4*>(hi + r * kpad + k) = h;
    *reinterpret_cast<uint4*>(lo + r * kpad + k) = l;
  }
}

// per-column weights: imaginary axis  w0 = 4 D / (xi^2 + D^2);  complex  (w0, w1) = -4 D / (z^2 - D^2)
__global__ void weight_kernel(const double* __restrict__ D, long n_ov, long kpad, const double* xi_dev,
                              const cplx* z_dev, float* __restrict__ w0, float* __restrict__ w1) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < kpad; k += (long)gridDim.x * blockDim.x) {
    if (k >= n_ov) {
      w0[k] = 0.f;
      if (w1) w1[k] = 0.f;
      continue;
    }
    const double d = D[k];
    if (xi_dev) {
      const double x = xi_dev[0];
      w0[k] = (float)(4.0 * d / (x * x + d * d));
    } else {
      const cplx z = z_dev[0];
      const cplx w = mkc(-4.0 * d, 0.0) / (z * z - mkc(d * d, 0.0));
      w0[k] = (float)w.x;
      w1[k] = (float)w.y;
    }
  }
}

// S_a = B diag(w_a) -> hi/lo planes, for one (NACC = 1) or two (NACC = 2) weight vectors
template <class TIn, int NACC>
__global__ void scale_split_kernel(const TIn* __restrict__ B, int n, long n_ov, long kpad, const float* __restrict__ w0,
                                   const float* __restrict__ w1, __nv_bfloat16* __restrict__ s0h,
                                   __nv_bfloat16* __restrict__ s0l, __nv_bfloat16* __restrict__ s1h,
                                   __nv_bfloat16* __restrict__ s1l) {
  const long chunks = kpad / 8, total = (long)n * chunks;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < total; c += (long)gridDim.x * blockDim.x) {
    const long r = c / chunks, k = (c % chunks) * 8;
    float v[8], s[8];
    load8(B + r * n_ov, k, n_ov, v);
    const float4 wa = *reinterpret_cast<const float4*>(w0 + k), wb = *reinterpret_cast<const float4*>(w0 + k + 4);
    const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] = v[j] * wv[j];
    uint4 h, l;
    split8(s, h, l);
    *reinterpret_cast<uint4*>(s0h + r * kpad + k) = h;
    *reinterpret_cast<uint4*>(s0l + r * kpad + k) = l;
    if (NACC == 2) {
      const float4 xa = *reinterpret_cast<const float4*>(w1 + k), xb = *reinterpret_cast<const float4*>(w1 + k + 4);
      const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) s[j] = v[j] * xv[j];
      split8(s, h, l);
      *reinterpret_cast<uint4*>(s1h + r * kpad + k) = h;
      *reinterpret_cast<uint4*>(s1l + r * kpad + k) = l;
    }
  }
}

// ---- host side --------------------------------------------------------------------------------------------------

struct Scratch {
  __nv_bfloat16 *bh, *bl, *s0h, *s0l, *s1h, *s1l;
  float *w0, *w1;
  long kpad;
};

long kpad_of(long n_ov) { return ((n_ov + BK - 1) / BK) * BK; }

// Shared region: the BF16 planes of O^{ia} (read by every lane).  Lane region: the weighted planes and weights.
Scratch carve(const void* shared, void* lane, int n, long n_ov) {
  Scratch s;
  const long kp = kpad_of(n_ov);
  const size_t plane = (size_t)n * kp;
  Arena as(const_cast<void*>(shared));
  s.bh = as.take<__nv_bfloat16>(plane);
  s.bl = as.take<__nv_bfloat16>(plane);
  Arena al(lane);   // the second weighted pair comes last: a lane sized for real weights only stops before it
  s.s0h = al.take<__nv_bfloat16>(plane);
  s.s0l = al.take<__nv_bfloat16>(plane);
  s.w0 = al.take<float>(kp);
  s.w1 = al.take<float>(kp);
  s.s1h = al.take<__nv_bfloat16>(plane);
  s.s1l = al.take<__nv_bfloat16>(plane);
  s.kpad = kp;
  return s;
}

bool make_map(CUtensorMap* m, const void* base, int rows, long kpad, int box_rows = BM) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int elementwise_blocks(cdwac_ctx* ctx, long work) {
  long b = (work + 255) / 256;
  long cap = (long)ctx->num_sms * 8;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// TMA map of a plane for the 128 x 256 kernel: 32-column boxes, 64-byte swizzle.
bool make_map64(CUtensorMap* m, const void* base, int rows, long kpad, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)w256::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One launch on 128 x 256 tiles: part < 0 the real A with the weighted planes (sh, sl); part >= 0 both parts of
// the complex A, the real parts with (sh, sl) and the imaginary parts with (sh2, sl2).
cdwac_status run_syrk256(cdwac_ctx* ctx, const Scratch& s, const __nv_bfloat16* sh, const __nv_bfloat16* sl,
                         const __nv_bfloat16* sh2, const __nv_bfloat16* sl2, int n, void* A, int part, float* negpi32,
                         cudaStream_t st) {
  Maps maps, maps_im;
  memset(&maps, 0, sizeof(maps));
  if (!make_map64(&maps.sh, sh, n, s.kpad, w256::BM) || !make_map64(&maps.sl, sl, n, s.kpad, w256::BM) ||
      !make_map64(&maps.bh, s.bh, n, s.kpad, w256::BN) || !make_map64(&maps.bl, s.bl, n, s.kpad, w256::BN))
    return set_error(ctx, CDWAC_ERR_CUDA, "cuTensorMapEncodeTiled failed (n=%d kpad=%ld)", n, s.kpad);
  maps_im = maps;
  if (part >= 0 && (!make_map64(&maps_im.sh, sh2, n, s.kpad, w256::BM) ||
                    !make_map64(&maps_im.sl, sl2, n, s.kpad, w256::BM)))
    return set_error(ctx, CDWAC_ERR_CUDA, "cuTensorMapEncodeTiled failed (n=%d kpad=%ld)", n, s.kpad);
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(tc_syrk256_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           w256::SMEM));
  const int nt = (n + w256::BM - 1) / w256::BM, tiles = tiles256(nt);
  const int group = ctx->pi_group >= 1 && ctx->pi_group <= 64 ? ctx->pi_group : 12;
  tc_syrk256_kernel<<<part >= 0 ? 2 * tiles : tiles, w256::NT, w256::SMEM, st>>>(
      maps, maps_im, tiles, n, (int)(s.kpad / w256::BK), group, A, part, negpi32, ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

// One launch of the contraction with the weighted planes (sh, sl): part as in tc_syrk_kernel; 128 x 256 tiles
// (the context's pi_tile, 256 by default) or 128 x 128 tiles.
cdwac_status run_syrk(cdwac_ctx* ctx, const Scratch& s, const __nv_bfloat16* sh, const __nv_bfloat16* sl, int n,
                      void* A, int part, float* negpi32, cudaStream_t st) {
  if (ctx->pi_tile != 128) return run_syrk256(ctx, s, sh, sl, nullptr, nullptr, n, A, part, negpi32, st);
  Maps maps;
  memset(&maps, 0, sizeof(maps));
  if (!make_map(&maps.sh, sh, n, s.kpad) || !make_map(&maps.sl, sl, n, s.kpad) || !make_map(&maps.bh, s.bh, n, s.kpad) ||
      !make_map(&maps.bl, s.bl, n, s.kpad))
    return set_error(ctx, CDWAC_ERR_CUDA, "cuTensorMapEncodeTiled failed (n=%d kpad=%ld)", n, s.kpad);
  CDWAC_CUDA_TRY(ctx, cudaFuncSetAttribute(tc_syrk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
  const int nt = (n + BM - 1) / BM;
  const int group = ctx->pi_group >= 1 && ctx->pi_group <= 64 ? ctx->pi_group : 12;
  tc_syrk_kernel<<<nt * (nt + 1) / 2, 384, SMEM, st>>>(maps, n, (int)(s.kpad / BK), group, A, part, negpi32,
                                                        ctx->d_status);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

}  // namespace

size_t tc_pi_shared_bytes(int n_aux, long n_ov) {
  const long kp = kpad_of(n_ov);
  return 2 * ((size_t)n_aux * kp * 2 + 256) + 512;
}

size_t tc_pi_lane_bytes(int n_aux, long n_ov, int nacc) {
  const long kp = kpad_of(n_ov);
  return 2 * nacc * ((size_t)n_aux * kp * 2 + 256) + 2 * ((size_t)kp * 4 + 256) + 512;
}

size_t tc_pi_scratch_bytes(int n_aux, long n_ov) {
  return tc_pi_shared_bytes(n_aux, n_ov) + tc_pi_lane_bytes(n_aux, n_ov) + 256;
}

void* tc_pi_lane_part(void* scratch, int n_aux, long n_ov) {
  return static_cast<char*>(scratch) + ((tc_pi_shared_bytes(n_aux, n_ov) + 255) & ~size_t(255));
}

cdwac_status tc_pi_prepare(cdwac_ctx* ctx, const void* O_ia, int dtype, int n_aux, long n_ov, void* scratch,
                           cudaStream_t st) {
  Scratch s = carve(scratch, nullptr, n_aux, n_ov);
  const int blocks = elementwise_blocks(ctx, (long)n_aux * (s.kpad / 8));
  if (dtype == CDWAC_F64)
    split_kernel<double><<<blocks, 256, 0, st>>>((const double*)O_ia, n_aux, n_ov, s.kpad, s.bh, s.bl);
  else
    split_kernel<float><<<blocks, 256, 0, st>>>((const float*)O_ia, n_aux, n_ov, s.kpad, s.bh, s.bl);
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

static cdwac_status scale(cdwac_ctx* ctx, const Scratch& s, const void* O_ia, int dtype, const double* D, int n,
                          long n_ov, const double* xi_dev, const cplx* z_dev, cudaStream_t st) {
  const int wb = elementwise_blocks(ctx, s.kpad);
  weight_kernel<<<wb, 256, 0, st>>>(D, n_ov, s.kpad, xi_dev, z_dev, s.w0, z_dev ? s.w1 : nullptr);
  CDWAC_LAUNCH_CHECK(ctx);
  const int blocks = elementwise_blocks(ctx, (long)n * (s.kpad / 8));
  if (xi_dev) {
    if (dtype == CDWAC_F64)
      scale_split_kernel<double, 1><<<blocks, 256, 0, st>>>((const double*)O_ia, n, n_ov, s.kpad, s.w0, nullptr, s.s0h,
                                                           s.s0l, nullptr, nullptr);
    else
      scale_split_kernel<float, 1><<<blocks, 256, 0, st>>>((const float*)O_ia, n, n_ov, s.kpad, s.w0, nullptr, s.s0h,
                                                          s.s0l, nullptr, nullptr);
  } else {
    if (dtype == CDWAC_F64)
      scale_split_kernel<double, 2><<<blocks, 256, 0, st>>>((const double*)O_ia, n, n_ov, s.kpad, s.w0, s.w1, s.s0h,
                                                           s.s0l, s.s1h, s.s1l);
    else
      scale_split_kernel<float, 2><<<blocks, 256, 0, st>>>((const float*)O_ia, n, n_ov, s.kpad, s.w0, s.w1, s.s0h,
                                                          s.s0l, s.s1h, s.s1l);
  }
  CDWAC_LAUNCH_CHECK(ctx);
  return CDWAC_OK;
}

cdwac_status tc_pi_imag(cdwac_ctx* ctx, const void* shared, void* lane, const void* O_ia, int dtype, const double* D,
                        int n_aux, long n_ov, const double* xi_dev, double* A, float* negpi32, cudaStream_t st) {
  Scratch s = carve(shared, lane, n_aux, n_ov);
  cdwac_status rc;
  {
    ProfScope ps(ctx, PROF_PI_PREP, st);
    rc = scale(ctx, s, O_ia, dtype, D, n_aux, n_ov, xi_dev, nullptr, st);
  }
  if (rc) return rc;
  ProfScope ps(ctx, PROF_PI_TC_IMAG, st);
  return run_syrk(ctx, s, s.s0h, s.s0l, n_aux, A, -1, negpi32, st);
}

cdwac_status tc_pi_complex(cdwac_ctx* ctx, const void* shared, void* lane, const void* O_ia, int dtype,
                           const double* D, int n_aux, long n_ov, const cplx* z_dev, cplx* A, cudaStream_t st) {
  Scratch s = carve(shared, lane, n_aux, n_ov);
  cdwac_status rc;
  {
    ProfScope ps(ctx, PROF_PI_PREP, st);
    rc = scale(ctx, s, O_ia, dtype, D, n_aux, n_ov, nullptr, z_dev, st);
  }
  if (rc) return rc;
  ProfScope ps(ctx, PROF_PI_TC_CPLX, st);
  // real and imaginary parts as two real contractions sharing the B planes (one launch on 128 x 256 tiles)
  if (ctx->pi_tile != 128) return run_syrk256(ctx, s, s.s0h, s.s0l, s.s1h, s.s1l, n_aux, A, 0, nullptr, st);
  if ((rc = run_syrk(ctx, s, s.s0h, s.s0l, n_aux, A, 0, nullptr, st))) return rc;
  return run_syrk(ctx, s, s.s1h, s.s1l, n_aux, A, 1, nullptr, st);
}
