// FP64-equivalent trailing update of the blocked LDL^T on the tcgen05 tensor cores (exact BF16 slice products).
#pragma once
#include <cuda.h>

#include "common.cuh"

struct OzakiPlan {
  CUtensorMap wmap[2], lmap[2];   // slice planes of W (128-row boxes) and of L (column-tile boxes), two buffers
  void* wpl[2];
  void* lpl[2];
  int* ew[2];                     // per-row exponents e (the row's largest magnitude is below 2^e)
  int* el[2];
  int n;
  bool cplx;
};

// Device scratch of one factorisation of order n (two buffers of slice planes and exponents).
size_t ozaki_scratch_bytes(int n, bool cplx);
// Carves the scratch and encodes the tensor maps (host work, once per factorisation).
cdwac_status ozaki_plan(cdwac_ctx* ctx, void* scratch, int n, bool cplx, OzakiPlan* plan);
// Slices rows k0 + 64 .. n - 1 of the panel W (wpanel, row stride 64) and of L (columns k0 .. k0 + 63 of A).
template <class T>
cdwac_status ozaki_slice(cdwac_ctx* ctx, const OzakiPlan& plan, int buf, const T* A, int n, int k0, const T* wpanel,
                         cudaStream_t st);
// A_ij -= sum_c W_ic L_jc over the trailing lower triangle (i >= j >= k0 + 64).  part 0: every tile; part 1: the
// next 64-column block only; part 2: every tile except that block.
template <class T>
cdwac_status ozaki_update(cdwac_ctx* ctx, const OzakiPlan& plan, int buf, T* A, int n, int k0, int part,
                          cudaStream_t st);
