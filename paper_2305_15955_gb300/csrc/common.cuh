// Shared definitions of libcdwac: the context, error plumbing, the complex scalar, launch helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/cdwac.h"

// Device status bits (OR-ed into the context's status word by kernels).
enum : unsigned {
  DEV_ERR_NOT_SPD = 1u << 0,
  DEV_ERR_SINGULAR = 1u << 1,
  DEV_INFO_PADE_BREAKDOWN = 1u << 2,
  DEV_INFO_QP_NOT_CONVERGED = 1u << 3,
  DEV_ERR_TIMEOUT = 1u << 4,
  DEV_ERR_BOUNDS = 1u << 5,
};

// Kernel classes timed by the optional event profiler (cdwac_profile_enable).
enum ProfClass {
  PROF_GRID = 0,
  PROF_PI_PREP,       // BF16 split / weighted split of the operand planes
  PROF_PI_TC_IMAG,    // tcgen05 Pi(i xi)
  PROF_PI_TC_CPLX,    // tcgen05 Pi(z)
  PROF_PI_SIMT,       // FP64 Pi on the CUDA cores
  PROF_LDLT,          // blocked LDL^T (FP64, real or complex)
  PROF_QUADFORM,      // Pi O product and triangular solves for W
  PROF_THIELE,
  PROF_SIGMA,
  PROF_QP,
  PROF_MLP,           // learned continuation: training step or pole inference
  PROF_LDLT_DIAG,     // fine level: the three launches of each LDL^T block step
  PROF_LDLT_PANEL,
  PROF_LDLT_UPDATE,
  PROF_LDLT_SLICE,    // fine level: digit planes of the panel for the tensor-core updates
  PROF_COUNT
};

struct ProfRecord {
  int cls;
  cudaEvent_t start, stop;
};

struct cdwac_ctx {
  int device = 0;
  int num_sms = 0;
  unsigned* d_status = nullptr;     // device status word
  unsigned* h_status = nullptr;     // pinned mirror
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  unsigned long long scratch_gen = 0;   // bumped whenever the scratch is reallocated (invalidates captured graphs)
  std::string last_error;
  long long launches = 0;           // kernels launched through this context
  bool quiet = false;               // set_error keeps no message (used where no allocation may happen)
  int prof = 0;                     // 0 off, 1 kernel classes, 2 also the launches inside the LDL^T
  cudaStream_t side_stream = nullptr;  // second stream of the LDL^T lookahead (joined before each call returns)
  cudaStream_t own_side = nullptr;     // the side stream this context created (side_stream may be switched off)
  cudaEvent_t ev_panel = nullptr, ev_bulk = nullptr;
  // the LDL^T critical path (panel, next-column update, diagonal block) runs on a high-priority stream so that its
  // single-CTA launches are dispatched ahead of the bulk update's waiting CTAs (side stream, lowest priority)
  cudaStream_t crit_stream = nullptr;
  cudaEvent_t ev_crit_in = nullptr, ev_crit_out = nullptr;
  // batched launch: lane contexts (own scratch and streams, shared status word), fork/join events, graph cache
  bool is_lane = false;
  int freq_lanes = 8;                   // concurrent frequency chains in the W builds (lanes never nest)
  bool lookahead = true;                // LDL^T bulk updates on the side stream (else one stream, no events)
  // tile configuration (chosen by the batch autotuner, or CDWAC_PI_GROUP / CDWAC_UPD_WAVES at creation):
  int pi_group = 12;                    // tensor-core Pi: tiles ordered in pi_group x pi_group groups
  int pi_tile = 256;                    // tensor-core Pi: output tile width, 256 or 128 columns
  int upd_waves = 1;                    // real trailing update: row-strip chunks sized for this many CTA waves
  std::vector<cdwac_ctx*> lanes;
  std::vector<cudaStream_t> lane_streams;
  std::vector<cudaEvent_t> lane_events;
  cudaEvent_t ev_fork = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::string graph_key;
  std::vector<ProfRecord> prof_live;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[PROF_COUNT] = {};
  int prof_n[PROF_COUNT] = {};
};

// Records CUDA events around a region on `st` when profiling is on.
struct ProfScope {
  cdwac_ctx* ctx;
  cudaStream_t st;
  int cls;
  cudaEvent_t stop = nullptr;
  ProfScope(cdwac_ctx* c, int k, cudaStream_t s, int level = 1) : ctx(c), st(s), cls(k) {
    if (ctx->prof < level) return;
    cudaEvent_t a = take(), b = take();
    cudaEventRecord(a, st);
    ctx->prof_live.push_back({cls, a, b});
    stop = b;
  }
  ~ProfScope() {
    if (stop) cudaEventRecord(stop, st);
  }
  cudaEvent_t take() {
    if (!ctx->prof_pool.empty()) {
      cudaEvent_t e = ctx->prof_pool.back();
      ctx->prof_pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
};

// Bump allocator over the context scratch; every region is 256-byte aligned.
struct Arena {
  char* base;
  size_t off = 0;
  explicit Arena(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += n * sizeof(T);
    return p;
  }
};

cdwac_status ensure_scratch(cdwac_ctx* ctx, size_t bytes);
// Creates the LDL^T streams and events of a context (side stream, high-priority critical-path stream); false on
// a CUDA error.
bool create_factor_streams(cdwac_ctx* ctx);
// batch.cu: lane contexts (own scratch, own side stream, the parent's status word) and their streams/events
cdwac_status ensure_lanes(cdwac_ctx* ctx, int n);
cdwac_status set_error(cdwac_ctx* ctx, cdwac_status st, const char* fmt, ...);

#define CDWAC_CUDA_TRY(ctx, expr)                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (expr);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return set_error((ctx), CDWAC_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #expr,         \
                       cudaGetErrorString(e_));                                                   \
  } while (0)

#define CDWAC_LAUNCH_CHECK(ctx)            \
  do {                                     \
    ++(ctx)->launches;                     \
    CDWAC_CUDA_TRY(ctx, cudaGetLastError()); \
  } while (0)

// ---- complex scalar (re, im) with the operations the kernels need ------------------------------------------
struct cplx {
  double x, y;
};
__host__ __device__ inline cplx mkc(double x, double y) { return cplx{x, y}; }
__host__ __device__ inline cplx operator+(cplx a, cplx b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cplx operator-(cplx a, cplx b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cplx operator*(cplx a, cplx b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__host__ __device__ inline cplx operator*(double s, cplx a) { return {s * a.x, s * a.y}; }
// Smith's division (R. L. Smith, CACM 5(8), 1962): scales by the larger component to avoid overflow.
__host__ __device__ inline cplx operator/(cplx a, cplx b) {
  double br = fabs(b.x), bi = fabs(b.y);
  if (br >= bi) {
    if (br == 0.0 && bi == 0.0) return {a.x / br, a.y / br};
    double rat = b.y / b.x, scl = 1.0 / (b.x + b.y * rat);
    return {(a.x + a.y * rat) * scl, (a.y - a.x * rat) * scl};
  }
  double rat = b.x / b.y, scl = 1.0 / (b.y + b.x * rat);
  return {(a.x * rat + a.y) * scl, (a.y * rat - a.x) * scl};
}
__host__ __device__ inline bool finite_c(cplx a) { return isfinite(a.x) && isfinite(a.y); }

// Scalar traits so that one LDL^T / solve template serves the real (imaginary axis) and complex (near-real
// and residue) cases.
template <class T>
struct Num;
template <>
struct Num<double> {
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double one() { return 1.0; }
  __device__ static double fma_(double a, double b, double c) { return fma(a, b, c); }   // a*b + c
  __device__ static double fms(double a, double b, double c) { return fma(-a, b, c); }   // c - a*b
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double div(double a, double b) { return a / b; }
  __device__ static double sub(double a, double b) { return a - b; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double re(double a) { return a; }
  __device__ static double mag(double a) { return fabs(a); }
};
template <>
struct Num<cplx> {
  __host__ __device__ static cplx zero() { return {0.0, 0.0}; }
  __host__ __device__ static cplx one() { return {1.0, 0.0}; }
  __device__ static cplx fma_(cplx a, cplx b, cplx c) {
    return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
  }
  __device__ static cplx fms(cplx a, cplx b, cplx c) {
    return {fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y))};
  }
  __device__ static cplx mul(cplx a, cplx b) { return a * b; }
  __device__ static cplx div(cplx a, cplx b) { return a / b; }
  __device__ static cplx sub(cplx a, cplx b) { return a - b; }
  __device__ static cplx add(cplx a, cplx b) { return a + b; }
  __device__ static double re(cplx a) { return a.x; }
  __device__ static double mag(cplx a) { return hypot(a.x, a.y); }
};

__device__ inline void raise_status(unsigned* status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

inline int ceil_div(long a, long b) { return int((a + b - 1) / b); }

// ---- entry points of the individual translation units (host side, stream ordered) -----------------------
// grid.cu
cdwac_status launch_gauss_legendre(cdwac_ctx* ctx, int n, double omega0, double* xi, double* wxi,
                                   cudaStream_t st);
// pi_simt.cu: A = I - Pi(z) (lower triangle), FP64 SIMT.  B is [n_aux][n_ov] (f64 or f32).
// xi (or z) is read on the device from xi_dev[0] (z_dev[0]), so that host code never waits for it.
// The imaginary-axis kernel also writes -Pi into the strict upper triangle of A (untouched by the LDL^T) and
// the diagonal of Pi into pidiag (may be null), so that Pi O can be formed after the factorisation.
cdwac_status launch_pi_imag_fp64(cdwac_ctx* ctx, const void* B, int dtype, const double* D, int n_aux, int n_ov,
                                 const double* xi_dev, double* A, double* pidiag, cudaStream_t st);
// V = Pi O (FP64) for every state column; V has O_n's layout [n_states][n][ld_o].
cdwac_status launch_pi_times_o(cdwac_ctx* ctx, const double* A, const double* pidiag, int n, const void* O, int dtype,
                               long o_state_stride, long ld_o, int n_states, int cols_per_state, double* V,
                               cudaStream_t st);
cdwac_status launch_pi_complex_fp64(cdwac_ctx* ctx, const void* B, int dtype, const double* D, int n_aux,
                                    int n_ov, const cplx* z_dev, cplx* A, cudaStream_t st);
cdwac_status launch_transition_energies(cdwac_ctx* ctx, const double* eps, int n_occ, int n_virt, double* D,
                                        cudaStream_t st);
// ldlt.cu
template <class T>
cdwac_status ldlt_factor(cdwac_ctx* ctx, T* A, int n, T* dinv, T* linv_blocks, T* wpanel, cudaStream_t st,
                         void* oz_scratch = nullptr);
// Device scratch for ldlt_factor's tensor-core trailing update (oz_scratch; null = FP64 FMA update).
size_t ldlt_tc_scratch_bytes(int n, bool cplx);
template <class T>
size_t ldlt_scratch_elems(int n);
// W[s][m] = sum_P y_Pm^2 / d_P - sum_P o_Pm^2, y = L^{-1} o, for states s < n_states and columns
// m < cols_per_state; o_Pm of state s is O[s * o_state_stride + P * ld_o + m] (element type dtype) and the
// result goes to W_out[s * w_state_stride + m].
template <class T>
cdwac_status ldlt_quadform(cdwac_ctx* ctx, const T* L, const T* dinv, const T* linv_blocks, int n, const void* O,
                           int dtype, long o_state_stride, long ld_o, int n_states, int cols_per_state, T* W_out,
                           long w_state_stride, T* ywork, cudaStream_t st);
template <class T>
size_t quadform_scratch_elems(int n, int n_cols);
// W[s][m] = sum_P y_Pm u_Pm / d_P with y = L^{-1} o, u = L^{-1} v, v = Pi o (real): o^T (I - Pi)^{-1} Pi o without
// the cancellation of |L^{-1} o|^2 / d - |o|^2 when W is small.  V is FP64 with O's layout.
cdwac_status ldlt_quadform_pi(cdwac_ctx* ctx, const double* L, const double* dinv, const double* linv_blocks, int n,
                              const void* O, int dtype, const double* V, long o_state_stride, long ld_o, int n_states,
                              int cols_per_state, double* W_out, long w_state_stride, double* ywork, cudaStream_t st);
// wsolve_tc.cu: mixed-precision W = sum_P y u / d, [y | u] = L^-1 [o | Pi o] as a blocked forward substitution whose
// products run on the tensor cores (split BF16, FP32 sums); Pi from negpi32 (-Pi, FP32, full symmetric).
size_t wsolve_tc_scratch_bytes(int n, int n_cols);
cdwac_status wsolve_tc(cdwac_ctx* ctx, const double* L, const double* dinv, const double* linv, const float* negpi32,
                       int n, const void* O, int dtype, long o_state_stride, long ld_o, int n_states,
                       int cols_per_state, double* W_out, long w_state_stride, void* scratch, cudaStream_t st);
// wsolve_tc.cu, near-real points and residues: W = sum_P y_P^2 / d_P - sum_P o_P^2, y = L^-1 o (complex symmetric
// FP64 factor), blocked forward substitution with tensor-core updates
size_t wsolve_tc_c_scratch_bytes(int n, int n_cols);
cdwac_status wsolve_tc_c(cdwac_ctx* ctx, const cplx* L, const cplx* dinv, const cplx* linv, int n, const void* O,
                         int dtype, long o_state_stride, long ld_o, int n_states, int cols_per_state, cplx* W_out,
                         long w_state_stride, void* scratch, cudaStream_t st);
// thiele.cu
cdwac_status launch_thiele_fit(cdwac_ctx* ctx, int n_states, int n_occ, int n_imag, int n_real, const double* xi,
                               const double* W_imag, int n_basis, const double* z_real, const double* W_real,
                               const cdwac_params* prm, const cdwac_pade* pade, cudaStream_t st);
cdwac_status launch_near_real_points(cdwac_ctx* ctx, const double* eps, int n_occ, const int* states,
                                     int n_states, const cdwac_params* prm, double* z_real, cudaStream_t st);
// sigma.cu
cdwac_status launch_spectral(cdwac_ctx* ctx, const double* eps, const int* states, int n_states, const double* shift,
                             const double* omega, int n_omega, const double* sigma, double* A, cudaStream_t st);
cdwac_status launch_sigma_wac(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                              const double* wxi, const double* W_imag, const cdwac_pade* pade,
                              const double* omega, int n_omega, double* sigma, cudaStream_t st,
                              const double* W_zero = nullptr);
cdwac_status launch_sigma_I_only(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm,
                                 const double* xi, const double* wxi, const double* W_imag, const double* omega,
                                 int n_omega, double* sigma, cudaStream_t st);
// poles: [n_states][n_occ][CDWAC_MLP_POLES][2] (Omega, residue) of the learned continuation, replacing the Thiele
// fits in the residue term when pade is null and poles is not.
cdwac_status launch_sigma_poles(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                                const double* wxi, const double* W_imag, const double* poles, const double* omega,
                                int n_omega, double* sigma, cudaStream_t st);
cdwac_status launch_qp_poles(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                             const double* wxi, const double* W_imag, const double* poles, const double* shift,
                             const double* omega, int n_grid, double tol, int max_iter, double* e_qp, double* Z,
                             int* iters, int* qp_status, cudaStream_t st);
// W_zero [n_states][n_basis] (optional): the I term's W(0) part in closed form; eps_qp (optional): the energies
// eps_n of the QP equation when sys->eps holds those of G (evGW), the fixed point starting from sys->eps.
cdwac_status launch_qp_wac(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                           const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* shift,
                           const double* omega, int n_grid, double tol, int max_iter, double* e_qp, double* Z,
                           int* iters, int* qp_status, cudaStream_t st, const double* W_zero = nullptr,
                           const double* eps_qp = nullptr);
// eps[states[i]] = e[i]
cdwac_status launch_scatter_states(cdwac_ctx* ctx, double* eps, const int* states, const double* e, int n,
                                   cudaStream_t st);
