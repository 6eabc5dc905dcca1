// Mixed-precision polarizability on the tcgen05 tensor cores: split-BF16 operands (hi + lo, three products
// hi*hi + hi*lo + lo*hi) with FP32 accumulation in tensor memory, written out as A = I - Pi in FP64.
#pragma once
#include "common.cuh"

// Scratch of the mixed path: a shared region (BF16 planes of O^{ia}, built once per call by tc_pi_prepare) and a
// per-lane region (the weighted planes of one frequency and the weights); tc_pi_scratch_bytes = both, laid out as
// [shared | lane] with tc_pi_lane_part giving the lane part.
size_t tc_pi_shared_bytes(int n_aux, long n_ov);
// nacc = 1: a lane that only serves tc_pi_imag (one weighted pair); 2: also tc_pi_complex.
size_t tc_pi_lane_bytes(int n_aux, long n_ov, int nacc = 2);
size_t tc_pi_scratch_bytes(int n_aux, long n_ov);
void* tc_pi_lane_part(void* scratch, int n_aux, long n_ov);
// Splits O^{ia} into BF16 hi/lo planes in the shared region (once per call).
cdwac_status tc_pi_prepare(cdwac_ctx* ctx, const void* O_ia, int dtype, int n_aux, long n_ov, void* shared,
                           cudaStream_t st);
// A = I - Pi(i xi) (real, lower triangle), xi read from xi_dev[0].  If negpi32 is not null it receives -Pi in
// FP32 (the full symmetric matrix, row-major [n_aux][n_aux]).
cdwac_status tc_pi_imag(cdwac_ctx* ctx, const void* shared, void* lane, const void* O_ia, int dtype, const double* D,
                        int n_aux, long n_ov, const double* xi_dev, double* A, float* negpi32, cudaStream_t st);
// A = I - Pi(z) (complex, lower triangle), z read from z_dev[0].
cdwac_status tc_pi_complex(cdwac_ctx* ctx, const void* shared, void* lane, const void* O_ia, int dtype,
                           const double* D, int n_aux, long n_ov, const cplx* z_dev, cplx* A, cudaStream_t st);
