// C ABI of libcdwac: argument checks, scratch layout and the stream-ordered sequence of kernels of each step
// of the G0W0 procedure with CD and CD-WAC (Sec. 3.4).
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tc_pi.cuh"

// ---- context and errors ----------------------------------------------------------------------------------

cdwac_status set_error(cdwac_ctx* ctx, cdwac_status st, const char* fmt, ...) {
  if (ctx && !ctx->quiet) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return st;
}

cdwac_status ensure_scratch(cdwac_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return CDWAC_OK;
  if (ctx->scratch) {
    CDWAC_CUDA_TRY(ctx, cudaDeviceSynchronize());
    CDWAC_CUDA_TRY(ctx, cudaFree(ctx->scratch));
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
  }
  size_t want = bytes + (bytes >> 4);
  cudaError_t e = cudaMalloc(&ctx->scratch, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->scratch = nullptr;
    return set_error(ctx, CDWAC_ERR_OOM, "scratch allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  ctx->scratch_bytes = want;
  ++ctx->scratch_gen;
  return CDWAC_OK;
}

bool create_factor_streams(cdwac_ctx* ctx) {
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return false;
  if (cudaStreamCreateWithPriority(&ctx->own_side, cudaStreamNonBlocking, least) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->crit_stream, cudaStreamNonBlocking, greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_panel, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_bulk, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_crit_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_crit_out, cudaEventDisableTiming) != cudaSuccess)
    return false;
  ctx->side_stream = ctx->lookahead ? ctx->own_side : nullptr;
  return true;
}

extern "C" {

cdwac_status cdwac_create(cdwac_ctx** out, int device) {
  if (!out) return CDWAC_ERR_ARG;
  *out = nullptr;
  cdwac_ctx* ctx = new cdwac_ctx();
  ctx->device = device;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    delete ctx;
    return CDWAC_ERR_CUDA;
  }
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
    delete ctx;
    return CDWAC_ERR_CUDA;
  }
  if (!(p.major == 10 && p.minor == 3)) {
    delete ctx;
    return CDWAC_ERR_UNSUPPORTED;
  }
  ctx->num_sms = p.multiProcessorCount;
  if (const char* fl = getenv("CDWAC_FREQ_LANES")) ctx->freq_lanes = std::max(1, std::min(16, atoi(fl)));
  if (const char* la = getenv("CDWAC_LOOKAHEAD")) ctx->lookahead = atoi(la) != 0;
  if (const char* pg = getenv("CDWAC_PI_GROUP")) ctx->pi_group = std::max(1, std::min(64, atoi(pg)));
  if (const char* pt = getenv("CDWAC_PI_TILE")) ctx->pi_tile = atoi(pt) == 128 ? 128 : 256;
  if (const char* uw = getenv("CDWAC_UPD_WAVES")) ctx->upd_waves = std::max(1, std::min(8, atoi(uw)));
  if (!create_factor_streams(ctx)) {
    cdwac_destroy(ctx);
    return CDWAC_ERR_CUDA;
  }
  if (cudaMalloc(&ctx->d_status, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(unsigned)) != cudaSuccess) {
    cudaFree(ctx->d_status);
    delete ctx;
    return CDWAC_ERR_CUDA;
  }
  *out = ctx;
  return CDWAC_OK;
}

static const char* kProfNames[PROF_COUNT] = {"grid",      "pi_prep",   "pi_tc_imag", "pi_tc_complex", "pi_fp64_simt",
                                              "ldlt",      "w_solves",  "thiele_fit", "sigma",         "qp_solve",
                                              "mlp",       "ldlt_diag", "ldlt_panel", "ldlt_update", "ldlt_slice"};

void cdwac_profile_enable(cdwac_ctx* ctx, int on) {
  if (ctx) ctx->prof = on < 0 ? 0 : (on > 2 ? 2 : on);
}

static int drain_profile(cdwac_ctx* src, cdwac_ctx* dst) {
  for (auto& r : src->prof_live) {
    if (cudaEventSynchronize(r.stop) != cudaSuccess) return -1;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess) return -1;
    dst->prof_ms[r.cls] += ms;
    dst->prof_n[r.cls] += 1;
    src->prof_pool.push_back(r.start);
    src->prof_pool.push_back(r.stop);
  }
  src->prof_live.clear();
  return 0;
}

int cdwac_profile_read(cdwac_ctx* ctx, cdwac_profile_entry* out, int max_entries) {
  if (!ctx) return -1;
  if (drain_profile(ctx, ctx)) return -1;
  for (auto* l : ctx->lanes)
    if (drain_profile(l, ctx)) return -1;
  int k = 0;
  for (int c = 0; c < PROF_COUNT && k < max_entries; ++c) {
    if (ctx->prof_n[c] == 0) continue;
    out[k].name = kProfNames[c];
    out[k].launches = ctx->prof_n[c];
    out[k].total_ms = ctx->prof_ms[c];
    ++k;
  }
  for (int c = 0; c < PROF_COUNT; ++c) {
    ctx->prof_ms[c] = 0;
    ctx->prof_n[c] = 0;
  }
  return k;
}

long long cdwac_launch_count(const cdwac_ctx* ctx) {
  if (!ctx) return 0;
  long long n = ctx->launches;
  for (auto* l : ctx->lanes) n += l->launches;
  return n;
}

void cdwac_destroy(cdwac_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (auto* l : ctx->lanes) cdwac_destroy(l);
  for (auto s : ctx->lane_streams) cudaStreamDestroy(s);
  for (auto e : ctx->lane_events) cudaEventDestroy(e);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  for (auto& r : ctx->prof_live) {
    cudaEventDestroy(r.start);
    cudaEventDestroy(r.stop);
  }
  for (auto e : ctx->prof_pool) cudaEventDestroy(e);
  if (ctx->ev_panel) cudaEventDestroy(ctx->ev_panel);
  if (ctx->ev_bulk) cudaEventDestroy(ctx->ev_bulk);
  if (ctx->ev_crit_in) cudaEventDestroy(ctx->ev_crit_in);
  if (ctx->ev_crit_out) cudaEventDestroy(ctx->ev_crit_out);
  if (ctx->own_side) cudaStreamDestroy(ctx->own_side);
  if (ctx->crit_stream) cudaStreamDestroy(ctx->crit_stream);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (!ctx->is_lane) {
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
  }
  delete ctx;
}

const char* cdwac_last_error(const cdwac_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

size_t cdwac_scratch_bytes(const cdwac_ctx* ctx) { return ctx ? ctx->scratch_bytes : 0; }

void cdwac_default_params(cdwac_params* p) {
  if (!p) return;
  p->n_imag = 100;
  p->omega0 = 1.0;
  p->n_real = 40;
  p->eta_ref = 1e-3;
  p->real_margin = 0.5;
  p->eta = 1e-3;
  p->pade_M = 64;
  p->greedy_first = 0;
  p->greedy_crit = 0;
  p->precision = CDWAC_PREC_FP64;
  p->pade_tol = 0.0;
  p->real_set = CDWAC_REAL_GENERIC;
  p->n_core = 20;
  p->n_val = 20;
  p->delta_c = 0.5;
  p->delta_v = 0.5;
}

cdwac_status cdwac_sync_status(cdwac_ctx* ctx, void* stream) {
  if (!ctx) return CDWAC_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), st));
  CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  unsigned s = *ctx->h_status;
  if (s & DEV_ERR_TIMEOUT) return set_error(ctx, CDWAC_ERR_TIMEOUT, "a bounded device wait gave up");
  if (s & DEV_ERR_NOT_SPD) return set_error(ctx, CDWAC_ERR_NOT_SPD, "I - Pi(i xi) is not positive definite");
  if (s & DEV_ERR_SINGULAR) return set_error(ctx, CDWAC_ERR_SINGULAR, "I - Pi(z) has a vanishing pivot");
  if (s & DEV_ERR_BOUNDS)
    return set_error(ctx, CDWAC_ERR_ARG, "a frequency outside the range of the continuation (omega above the LUMO)");
  if (s & DEV_INFO_QP_NOT_CONVERGED)
    return set_error(ctx, CDWAC_ERR_QP_NOT_CONVERGED, "a quasiparticle equation did not converge");
  if (s & DEV_INFO_PADE_BREAKDOWN)
    return set_error(ctx, CDWAC_ERR_PADE_BREAKDOWN, "a Thiele fit stopped early (fit truncated)");
  return CDWAC_OK;
}

}  // extern "C"

// ---- shared pieces ------------------------------------------------------------------------------------------

static cdwac_status check_system(cdwac_ctx* ctx, const cdwac_system* s, const cdwac_params* p) {
  if (!ctx) return CDWAC_ERR_ARG;
  if (!s || !p) return set_error(ctx, CDWAC_ERR_ARG, "null system or params");
  if (s->n_basis < 2 || s->n_occ < 1 || s->n_occ >= s->n_basis || s->n_aux < 1 || s->n_states < 1)
    return set_error(ctx, CDWAC_ERR_ARG, "bad sizes n_basis=%d n_occ=%d n_aux=%d n_states=%d", s->n_basis, s->n_occ,
                     s->n_aux, s->n_states);
  if (!s->eps || !s->O_ia || !s->O_n || !s->states) return set_error(ctx, CDWAC_ERR_ARG, "null system pointer");
  if (s->O_dtype != CDWAC_F64 && s->O_dtype != CDWAC_F32) return set_error(ctx, CDWAC_ERR_ARG, "bad O_dtype");
  if (p->n_imag < 1 || p->n_imag > 4096) return set_error(ctx, CDWAC_ERR_ARG, "n_imag out of range");
  if (p->n_real < 0 || p->n_imag + p->n_real > CDWAC_MAX_CANDIDATES)
    return set_error(ctx, CDWAC_ERR_ARG, "n_imag + n_real must be <= %d", CDWAC_MAX_CANDIDATES);
  if (p->pade_M < 1 || p->pade_M > CDWAC_MAX_M) return set_error(ctx, CDWAC_ERR_ARG, "pade_M out of range");
  if (!(p->omega0 > 0) || !(p->eta >= 0) || !(p->eta_ref > 0) || !(p->pade_tol >= 0))
    return set_error(ctx, CDWAC_ERR_ARG, "omega0, eta_ref must be > 0 and eta >= 0");
  if (p->precision != CDWAC_PREC_FP64 && p->precision != CDWAC_PREC_MIXED)
    return set_error(ctx, CDWAC_ERR_ARG, "bad precision");
  if (p->real_set != CDWAC_REAL_GENERIC && p->real_set != CDWAC_REAL_REFINED)
    return set_error(ctx, CDWAC_ERR_ARG, "bad real_set");
  if (p->real_set == CDWAC_REAL_REFINED &&
      (p->n_core < 0 || p->n_val < 0 || p->n_core + p->n_val != p->n_real || !(p->delta_c >= 0) ||
       !(p->delta_v >= 0) || !(p->delta_c < 1e6) || !(p->delta_v < 1e6)))
    return set_error(ctx, CDWAC_ERR_ARG, "refined set: need n_core, n_val >= 0 with n_core + n_val = n_real and "
                                         "finite delta_c, delta_v >= 0");
  if ((long)s->n_aux * s->n_aux > (1L << 31) * 16) return set_error(ctx, CDWAC_ERR_ARG, "n_aux too large");
  return CDWAC_OK;
}

// Dense W build at one frequency: A = I - Pi(z) in `A`, factorised in place.
template <class T>
struct FactorScratch {
  T* A;
  T* dinv;
  T* linv;
  T* wpanel;
  T* ywork;
};

// rhs_sets: right-hand-side vectors solved per column (1, or 2 for the (I - Pi)^-1 Pi form)
template <class T>
static size_t factor_scratch_bytes(int n, int n_cols, int rhs_sets = 1) {
  size_t el = (size_t)n * n + ldlt_scratch_elems<T>(n) + rhs_sets * quadform_scratch_elems<T>(n, n_cols);
  return el * sizeof(T) + 8 * 256;
}

template <class T>
static FactorScratch<T> carve_factor(Arena& ar, int n, int n_cols, int rhs_sets = 1) {
  FactorScratch<T> f;
  f.A = ar.take<T>((size_t)n * n);
  int nblk = (n + 63) / 64;
  f.dinv = ar.take<T>(n);
  f.linv = ar.take<T>((size_t)nblk * 64 * 64);
  f.wpanel = ar.take<T>(2 * (size_t)(nblk + 1) * 64 * 64);
  f.ywork = ar.take<T>(rhs_sets * quadform_scratch_elems<T>(n, n_cols));
  return f;
}

extern "C" {

cdwac_status cdwac_ldlt_factor(cdwac_ctx* ctx, void* A, int n, int is_complex, int method, void* stream) {
  if (!ctx) return CDWAC_ERR_ARG;
  if (!A || n <= 0) return set_error(ctx, CDWAC_ERR_ARG, "null matrix or n <= 0");
  if (method != CDWAC_LDLT_FP64 && method != CDWAC_LDLT_EMULATED)
    return set_error(ctx, CDWAC_ERR_ARG, "unknown factorisation method %d", method);
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const bool cx = is_complex != 0;
  const bool emu = method == CDWAC_LDLT_EMULATED;
  const size_t el = cx ? sizeof(cplx) : sizeof(double);
  size_t bytes = ldlt_scratch_elems<double>(n) * el + 1024;
  if (emu) bytes += ldlt_tc_scratch_bytes(n, cx);
  cdwac_status rc = ensure_scratch(ctx, bytes);
  if (rc) return rc;
  Arena ar(ctx->scratch);
  const int nblk = (n + 63) / 64;
  ProfScope ps(ctx, PROF_LDLT, st);
  if (cx) {
    cplx* dinv = ar.take<cplx>(n);
    cplx* linv = ar.take<cplx>((size_t)nblk * 64 * 64);
    cplx* wpanel = ar.take<cplx>(2 * (size_t)(nblk + 1) * 64 * 64);
    void* oz = emu ? ar.take<char>(ldlt_tc_scratch_bytes(n, true)) : nullptr;
    return ldlt_factor<cplx>(ctx, static_cast<cplx*>(A), n, dinv, linv, wpanel, st, oz);
  }
  double* dinv = ar.take<double>(n);
  double* linv = ar.take<double>((size_t)nblk * 64 * 64);
  double* wpanel = ar.take<double>(2 * (size_t)(nblk + 1) * 64 * 64);
  void* oz = emu ? ar.take<char>(ldlt_tc_scratch_bytes(n, false)) : nullptr;
  return ldlt_factor<double>(ctx, static_cast<double*>(A), n, dinv, linv, wpanel, st, oz);
}

cdwac_status cdwac_spectral(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                            const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* shift,
                            const double* omega, int n_omega, double* sigma, double* A, void* stream) {
  if (!ctx) return CDWAC_ERR_ARG;
  if (!sigma || !A) return set_error(ctx, CDWAC_ERR_ARG, "null output");
  cdwac_status rc = cdwac_sigma(ctx, sys, prm, xi, wxi, W_imag, pade, omega, n_omega, sigma, stream);
  if (rc) return rc;
  return launch_spectral(ctx, sys->eps, sys->states, sys->n_states, shift, omega, n_omega, sigma, A,
                         (cudaStream_t)stream);
}

// ---- frequency lanes: the per-frequency work of one call split over concurrent streams -------------------------
// Each lane owns a context (own scratch, own LDL^T side stream) and takes frequencies k = l, l + L, ...; the
// caller's stream forks to the lanes and joins them.  While one lane walks the sequential diagonal/panel steps of
// its factorisation, the other's bulk trailing update keeps the FP64 units busy.

// Lanes for n_freq frequencies whose per-lane scratch is lane_bytes: at most ctx->freq_lanes, and no more than
// half of the device memory that is free (plus what the lanes already hold) can carry.
static int freq_lanes(cdwac_ctx* ctx, int n_freq, size_t lane_bytes) {
  if (ctx->is_lane) return 1;
  int L = std::max(1, std::min(ctx->freq_lanes, n_freq));
  size_t free_b = 0, total_b = 0;
  if (L > 1 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
    size_t held = 0;
    for (auto* l : ctx->lanes) held += l->scratch_bytes;
    const size_t budget = (free_b + held) / 2;
    const int fit = (int)std::min<size_t>(budget / std::max<size_t>(lane_bytes, 1), 64);
    L = std::max(1, std::min(L, fit));
  }
  return L;
}

static cdwac_status fork_lanes(cdwac_ctx* ctx, int L, cudaStream_t st) {
  cdwac_status rc = ensure_lanes(ctx, L);
  if (rc) return rc;
  CDWAC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, st));
  for (int l = 0; l < L; ++l) {
    ctx->lanes[l]->prof = ctx->prof;
    ctx->lanes[l]->side_stream = ctx->lookahead ? ctx->lanes[l]->own_side : nullptr;
    ctx->lanes[l]->pi_group = ctx->pi_group;
    ctx->lanes[l]->pi_tile = ctx->pi_tile;
    ctx->lanes[l]->upd_waves = ctx->upd_waves;
    CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->lane_streams[l], ctx->ev_fork, 0));
  }
  return CDWAC_OK;
}

static cdwac_status join_lanes(cdwac_ctx* ctx, int L, cudaStream_t st) {
  for (int l = 0; l < L; ++l) {
    CDWAC_CUDA_TRY(ctx, cudaEventRecord(ctx->lane_events[l], ctx->lane_streams[l]));
    CDWAC_CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->lane_events[l], 0));
  }
  return CDWAC_OK;
}

struct ImagBufs {
  FactorScratch<double> f;
  void* oz;
  double* pidiag;
  double* V;
  void* tc_lane;
  float* negpi32;
  void* wsolve;
};

// FP64 path: W = y^T D^-1 u with u = L^-1 Pi o (needs Pi O and a second solve); mixed path: FP32 solves of the
// same form with tensor-core products on the tensor-core Pi (wsolve_tc).
static size_t imag_lane_bytes(const cdwac_system* sys, bool mixed) {
  const int n = sys->n_aux, nb = sys->n_basis, cols = sys->n_states * nb;
  const long n_ov = (long)sys->n_occ * (nb - sys->n_occ);
  size_t b = factor_scratch_bytes<double>(n, cols, mixed ? 0 : 2) + 4096;
  if (!mixed) b += sizeof(double) * ((size_t)n + (size_t)sys->n_states * n * nb);
  if (mixed)
    b += tc_pi_lane_bytes(n, n_ov, 1) + sizeof(float) * (size_t)n * n + wsolve_tc_scratch_bytes(n, cols) +
         ldlt_tc_scratch_bytes(n, false) + 1280;
  return b;
}

static ImagBufs carve_imag(Arena& ar, const cdwac_system* sys, bool mixed) {
  const int n = sys->n_aux, nb = sys->n_basis, cols = sys->n_states * nb;
  const long n_ov = (long)sys->n_occ * (nb - sys->n_occ);
  ImagBufs b;
  b.f = carve_factor<double>(ar, n, cols, mixed ? 0 : 2);
  b.pidiag = mixed ? nullptr : ar.take<double>(n);
  b.V = mixed ? nullptr : ar.take<double>((size_t)sys->n_states * n * nb);
  b.tc_lane = mixed ? ar.take<char>(tc_pi_lane_bytes(n, n_ov, 1)) : nullptr;
  b.negpi32 = mixed ? ar.take<float>((size_t)n * n) : nullptr;
  b.wsolve = mixed ? ar.take<char>(wsolve_tc_scratch_bytes(n, cols)) : nullptr;
  b.oz = mixed ? ar.take<char>(ldlt_tc_scratch_bytes(n, false)) : nullptr;
  return b;
}

static cdwac_status imag_freqs(cdwac_ctx* lc, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                               double* W_imag, const double* D, const void* tc_shared, const ImagBufs& b, int k0,
                               int kstep, cudaStream_t st) {
  const int n = sys->n_aux, nb = sys->n_basis;
  const long n_ov = (long)sys->n_occ * (nb - sys->n_occ);
  const bool mixed = prm->precision == CDWAC_PREC_MIXED;
  cdwac_status rc;
  for (int k = k0; k < prm->n_imag; k += kstep) {
    if (mixed) {
      rc = tc_pi_imag(lc, tc_shared, b.tc_lane, sys->O_ia, sys->O_dtype, D, n, n_ov, xi + k, b.f.A, b.negpi32, st);
    } else {
      ProfScope ps(lc, PROF_PI_SIMT, st);
      rc = launch_pi_imag_fp64(lc, sys->O_ia, sys->O_dtype, D, n, (int)n_ov, xi + k, b.f.A, b.pidiag, st);
    }
    if (rc) return rc;
    {
      ProfScope ps(lc, PROF_LDLT, st);
      if ((rc = ldlt_factor<double>(lc, b.f.A, n, b.f.dinv, b.f.linv, b.f.wpanel, st, b.oz))) return rc;
    }
    ProfScope ps(lc, PROF_QUADFORM, st);
    if (mixed) {
      rc = wsolve_tc(lc, b.f.A, b.f.dinv, b.f.linv, b.negpi32, n, sys->O_n, sys->O_dtype, (long)n * nb, nb,
                    sys->n_states, nb, W_imag + (long)k * nb, (long)prm->n_imag * nb, b.wsolve, st);
    } else {
      if ((rc = launch_pi_times_o(lc, b.f.A, b.pidiag, n, sys->O_n, sys->O_dtype, (long)n * nb, nb, sys->n_states, nb,
                                  b.V, st)))
        return rc;
      rc = ldlt_quadform_pi(lc, b.f.A, b.f.dinv, b.f.linv, n, sys->O_n, sys->O_dtype, b.V, (long)n * nb, nb,
                            sys->n_states, nb, W_imag + (long)k * nb, (long)prm->n_imag * nb, b.f.ywork, st);
    }
    if (rc) return rc;
  }
  return CDWAC_OK;
}

// W_nm(i xi_k) at the prm->n_imag imaginary frequencies xi [device] into W [n_states][n_imag][n_basis].
static cdwac_status build_W_freqs(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                                  double* W_imag, cudaStream_t st) {
  cdwac_status rc;
  const int n = sys->n_aux, nb = sys->n_basis, n_occ = sys->n_occ, n_virt = nb - n_occ;
  const long n_ov = (long)n_occ * n_virt;
  const bool mixed = prm->precision == CDWAC_PREC_MIXED;
  const int L = freq_lanes(ctx, prm->n_imag, imag_lane_bytes(sys, mixed));
  size_t bytes = n_ov * sizeof(double) + (mixed ? tc_pi_shared_bytes(n, n_ov) : 0) + 1024;
  if (L == 1) bytes += imag_lane_bytes(sys, mixed);
  rc = ensure_scratch(ctx, bytes);
  if (rc) return rc;
  if (L > 1) {
    if ((rc = ensure_lanes(ctx, L))) return rc;
    for (int l = 0; l < L; ++l)
      if ((rc = ensure_scratch(ctx->lanes[l], imag_lane_bytes(sys, mixed)))) return set_error(ctx, rc, "lane scratch");
  }
  Arena ar(ctx->scratch);
  double* D = ar.take<double>(n_ov);
  void* tc_shared = mixed ? ar.take<char>(tc_pi_shared_bytes(n, n_ov)) : nullptr;
  {
    ProfScope ps(ctx, PROF_GRID, st);
    if ((rc = launch_transition_energies(ctx, sys->eps, n_occ, n_virt, D, st))) return rc;
  }
  if (mixed) {
    ProfScope ps(ctx, PROF_PI_PREP, st);
    if ((rc = tc_pi_prepare(ctx, sys->O_ia, sys->O_dtype, n, n_ov, tc_shared, st))) return rc;
  }
  if (L == 1) {
    ImagBufs b = carve_imag(ar, sys, mixed);
    return imag_freqs(ctx, sys, prm, xi, W_imag, D, tc_shared, b, 0, 1, st);
  }
  if ((rc = fork_lanes(ctx, L, st))) return rc;
  // frequencies are enqueued round robin over the lanes: the host's launch queue is bounded, so enqueueing one
  // lane's whole share first would let it drain alone before the next lane's work even arrives
  for (int k = 0; k < prm->n_imag; ++k) {
    const int l = k % L;
    Arena al(ctx->lanes[l]->scratch);
    ImagBufs b = carve_imag(al, sys, mixed);
    rc = imag_freqs(ctx->lanes[l], sys, prm, xi, W_imag, D, tc_shared, b, k, prm->n_imag, ctx->lane_streams[l]);
    if (rc) return set_error(ctx, rc, "lane %d: %s", l, ctx->lanes[l]->last_error.c_str());
  }
  return join_lanes(ctx, L, st);
}

cdwac_status cdwac_build_W_imag(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, double* xi,
                                double* wxi, double* W_imag, void* stream) {
  cdwac_status rc = check_system(ctx, sys, prm);
  if (rc) return rc;
  if (!xi || !wxi || !W_imag) return set_error(ctx, CDWAC_ERR_ARG, "null output");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  {
    ProfScope ps(ctx, PROF_GRID, st);
    if ((rc = launch_gauss_legendre(ctx, prm->n_imag, prm->omega0, xi, wxi, st))) return rc;
  }
  return build_W_freqs(ctx, sys, prm, xi, W_imag, st);
}

struct RealBufs {
  FactorScratch<cplx> f;
  void* oz;
  void* tc_lane;
  void* wsc;
};

static size_t real_lane_bytes(const cdwac_system* sys, bool mixed) {
  const int n = sys->n_aux, ns = sys->n_states, n_occ = sys->n_occ;
  const long n_ov = (long)n_occ * (sys->n_basis - n_occ);
  size_t b = factor_scratch_bytes<cplx>(n, ns * n_occ) + 2048;
  if (mixed) b += tc_pi_lane_bytes(n, n_ov) + wsolve_tc_c_scratch_bytes(n, ns * n_occ) + ldlt_tc_scratch_bytes(n, true) + 768;
  return b;
}

static RealBufs carve_real(Arena& ar, const cdwac_system* sys, bool mixed) {
  const int n = sys->n_aux, ns = sys->n_states, n_occ = sys->n_occ;
  const long n_ov = (long)n_occ * (sys->n_basis - n_occ);
  RealBufs b;
  b.f = carve_factor<cplx>(ar, n, ns * n_occ);
  b.tc_lane = mixed ? ar.take<char>(tc_pi_lane_bytes(n, n_ov)) : nullptr;
  b.wsc = mixed ? ar.take<char>(wsolve_tc_c_scratch_bytes(n, ns * n_occ)) : nullptr;
  b.oz = mixed ? ar.take<char>(ldlt_tc_scratch_bytes(n, true)) : nullptr;
  return b;
}

static cdwac_status real_points(cdwac_ctx* lc, const cdwac_system* sys, const cdwac_params* prm, const cplx* zr,
                                cplx* Wr, const double* D, const void* tc_shared, const RealBufs& b, int j0, int jstep,
                                cudaStream_t st) {
  const int n = sys->n_aux, nb = sys->n_basis, n_occ = sys->n_occ, ns = sys->n_states, nr = prm->n_real;
  const long n_ov = (long)n_occ * (nb - n_occ);
  const bool mixed = prm->precision == CDWAC_PREC_MIXED;
  cdwac_status rc;
  for (int j = j0; j < nr; j += jstep) {
    if (mixed) {
      rc = tc_pi_complex(lc, tc_shared, b.tc_lane, sys->O_ia, sys->O_dtype, D, n, n_ov, zr + j, b.f.A, st);
    } else {
      ProfScope ps(lc, PROF_PI_SIMT, st);
      rc = launch_pi_complex_fp64(lc, sys->O_ia, sys->O_dtype, D, n, (int)n_ov, zr + j, b.f.A, st);
    }
    if (rc) return rc;
    {
      ProfScope ps(lc, PROF_LDLT, st);
      if ((rc = ldlt_factor<cplx>(lc, b.f.A, n, b.f.dinv, b.f.linv, b.f.wpanel, st, b.oz))) return rc;
    }
    ProfScope ps(lc, PROF_QUADFORM, st);
    if (mixed)
      rc = wsolve_tc_c(lc, b.f.A, b.f.dinv, b.f.linv, n, sys->O_n, sys->O_dtype, (long)n * nb, nb, ns, n_occ,
                      Wr + (long)j * n_occ, (long)nr * n_occ, b.wsc, st);
    else
      rc = ldlt_quadform<cplx>(lc, b.f.A, b.f.dinv, b.f.linv, n, sys->O_n, sys->O_dtype, (long)n * nb, nb, ns, n_occ,
                               Wr + (long)j * n_occ, (long)nr * n_occ, b.f.ywork, st);
    if (rc) return rc;
  }
  return CDWAC_OK;
}

cdwac_status cdwac_fit_pade(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                            const double* W_imag, double* z_real, double* W_real, const cdwac_pade* pade,
                            void* stream) {
  cdwac_status rc = check_system(ctx, sys, prm);
  if (rc) return rc;
  if (!xi || !W_imag || !pade || !pade->a || !pade->z2 || !pade->nodes || !pade->n_used)
    return set_error(ctx, CDWAC_ERR_ARG, "null input or pade array");
  if (pade->n_states != sys->n_states || pade->n_occ != sys->n_occ || pade->M < prm->pade_M)
    return set_error(ctx, CDWAC_ERR_ARG, "pade arrays sized for (%d, %d, %d), need (%d, %d, >= %d)", pade->n_states,
                     pade->n_occ, pade->M, sys->n_states, sys->n_occ, prm->pade_M);
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int n = sys->n_aux, nb = sys->n_basis, n_occ = sys->n_occ, n_virt = nb - n_occ;
  const long n_ov = (long)n_occ * n_virt;
  const int nr = prm->n_real, ns = sys->n_states;
  const bool mixed = prm->precision == CDWAC_PREC_MIXED;
  const int L = nr > 0 ? freq_lanes(ctx, nr, real_lane_bytes(sys, mixed)) : 1;
  size_t bytes = n_ov * sizeof(double) + 2 * sizeof(cplx) * (size_t)ns * nr * (n_occ + 1) + 4096;
  if (mixed && nr > 0) bytes += tc_pi_shared_bytes(n, n_ov);
  if (nr > 0 && L == 1) bytes += real_lane_bytes(sys, mixed);
  rc = ensure_scratch(ctx, bytes);
  if (rc) return rc;
  if (nr > 0 && L > 1) {
    if ((rc = ensure_lanes(ctx, L))) return rc;
    for (int l = 0; l < L; ++l)
      if ((rc = ensure_scratch(ctx->lanes[l], real_lane_bytes(sys, mixed)))) return set_error(ctx, rc, "lane scratch");
  }
  Arena ar(ctx->scratch);
  double* D = ar.take<double>(n_ov);
  cplx* zr = z_real ? reinterpret_cast<cplx*>(z_real) : ar.take<cplx>((size_t)ns * nr + 1);
  cplx* Wr = W_real ? reinterpret_cast<cplx*>(W_real) : ar.take<cplx>((size_t)ns * nr * n_occ + 1);
  if (nr > 0) {
    void* tc_shared = mixed ? ar.take<char>(tc_pi_shared_bytes(n, n_ov)) : nullptr;
    if ((rc = launch_transition_energies(ctx, sys->eps, n_occ, n_virt, D, st))) return rc;
    if ((rc = launch_near_real_points(ctx, sys->eps, n_occ, sys->states, ns, prm, reinterpret_cast<double*>(zr),
                                      st)))
      return rc;
    if (mixed) {
      ProfScope ps(ctx, PROF_PI_PREP, st);
      if ((rc = tc_pi_prepare(ctx, sys->O_ia, sys->O_dtype, n, n_ov, tc_shared, st))) return rc;
    }
    if (L == 1) {
      RealBufs b = carve_real(ar, sys, mixed);
      if ((rc = real_points(ctx, sys, prm, zr, Wr, D, tc_shared, b, 0, 1, st))) return rc;
    } else {
      if ((rc = fork_lanes(ctx, L, st))) return rc;
      for (int j = 0; j < nr; ++j) {   // round robin over the lanes, as for the imaginary axis
        const int l = j % L;
        Arena al(ctx->lanes[l]->scratch);
        RealBufs b = carve_real(al, sys, mixed);
        rc = real_points(ctx->lanes[l], sys, prm, zr, Wr, D, tc_shared, b, j, nr, ctx->lane_streams[l]);
        if (rc) return set_error(ctx, rc, "lane %d: %s", l, ctx->lanes[l]->last_error.c_str());
      }
      if ((rc = join_lanes(ctx, L, st))) return rc;
    }
  }
  ProfScope ps(ctx, PROF_THIELE, st);
  return launch_thiele_fit(ctx, ns, n_occ, prm->n_imag, nr, xi, W_imag, nb, reinterpret_cast<const double*>(zr),
                           reinterpret_cast<const double*>(Wr), prm, pade, st);
}

}  // extern "C"

// Plain CD: Sigma[s][j] += f_m W_{n_s m}(|eps_m - omega_j| + i eta) for every residue, W built directly.
__global__ static void add_residue_kernel(cplx* sigma, int n_omega, int j, int n_states, double f, const cplx* W,
                                          long w_stride) {
  int s = threadIdx.x;
  if (s < n_states) {
    cplx w = W[s * w_stride];
    sigma[(long)s * n_omega + j] = sigma[(long)s * n_omega + j] + f * w;
  }
}

__global__ static void set_z_kernel(cplx* z, double x, double eta) { z[0] = mkc(x, eta); }

static cdwac_status plain_cd_residues(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm,
                                      const std::vector<double>& eps, const std::vector<double>& omega, double* sigma,
                                      int n_omega_stride, int j_offset, cudaStream_t st) {
  const int n = sys->n_aux, nb = sys->n_basis, n_occ = sys->n_occ, n_virt = nb - n_occ;
  const long n_ov = (long)n_occ * n_virt;
  const int ns = sys->n_states;
  const bool mixed = prm->precision == CDWAC_PREC_MIXED;
  size_t bytes = n_ov * sizeof(double) + factor_scratch_bytes<cplx>(n, ns) + sizeof(cplx) * (ns + 2) + 2048;
  if (mixed) bytes += tc_pi_scratch_bytes(n, n_ov) + wsolve_tc_c_scratch_bytes(n, ns) + ldlt_tc_scratch_bytes(n, true) + 512;
  cdwac_status rc = ensure_scratch(ctx, bytes);
  if (rc) return rc;
  Arena ar(ctx->scratch);
  double* D = ar.take<double>(n_ov);
  FactorScratch<cplx> f = carve_factor<cplx>(ar, n, ns);
  cplx* zdev = ar.take<cplx>(1);
  cplx* Wv = ar.take<cplx>(ns);
  void* tcs = mixed ? ar.take<char>(tc_pi_scratch_bytes(n, n_ov)) : nullptr;
  void* wsc = mixed ? ar.take<char>(wsolve_tc_c_scratch_bytes(n, ns)) : nullptr;
  void* oz = mixed ? ar.take<char>(ldlt_tc_scratch_bytes(n, true)) : nullptr;
  if ((rc = launch_transition_energies(ctx, sys->eps, n_occ, n_virt, D, st))) return rc;
  if (mixed && (rc = tc_pi_prepare(ctx, sys->O_ia, sys->O_dtype, n, n_ov, tcs, st))) return rc;
  for (size_t j = 0; j < omega.size(); ++j) {
    const double w = omega[j];
    for (int m = 0; m < nb; ++m) {
      double th_occ = eps[m] > w ? 1.0 : (eps[m] < w ? 0.0 : 0.5);
      double th_vir = w > eps[m] ? 1.0 : (w < eps[m] ? 0.0 : 0.5);
      double fm = m < n_occ ? -th_occ : th_vir;
      if (fm == 0.0) continue;
      set_z_kernel<<<1, 1, 0, st>>>(zdev, fabs(eps[m] - w), prm->eta);
      CDWAC_LAUNCH_CHECK(ctx);
      if (mixed)
        rc = tc_pi_complex(ctx, tcs, tc_pi_lane_part(tcs, n, n_ov), sys->O_ia, sys->O_dtype, D, n, n_ov, zdev, f.A, st);
      else
        rc = launch_pi_complex_fp64(ctx, sys->O_ia, sys->O_dtype, D, n, (int)n_ov, zdev, f.A, st);
      if (rc) return rc;
      if ((rc = ldlt_factor<cplx>(ctx, f.A, n, f.dinv, f.linv, f.wpanel, st, oz))) return rc;
      // column m of every state's O_n
      const void* Om = sys->O_dtype == CDWAC_F64 ? (const void*)((const double*)sys->O_n + m)
                                                 : (const void*)((const float*)sys->O_n + m);
      if (mixed)
        rc = wsolve_tc_c(ctx, f.A, f.dinv, f.linv, n, Om, sys->O_dtype, (long)n * nb, nb, ns, 1, Wv, 1, wsc, st);
      else
        rc = ldlt_quadform<cplx>(ctx, f.A, f.dinv, f.linv, n, Om, sys->O_dtype, (long)n * nb, nb, ns, 1, Wv, 1,
                                 f.ywork, st);
      if (rc) return rc;
      add_residue_kernel<<<1, 32 * ((ns + 31) / 32), 0, st>>>(reinterpret_cast<cplx*>(sigma), n_omega_stride,
                                                              (int)j + j_offset, ns, fm, Wv, 1);
      CDWAC_LAUNCH_CHECK(ctx);
    }
  }
  return CDWAC_OK;
}

extern "C" {

cdwac_status cdwac_sigma(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                         const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* omega,
                         int n_omega, double* sigma, void* stream) {
  cdwac_status rc = check_system(ctx, sys, prm);
  if (rc) return rc;
  if (!xi || !wxi || !W_imag || !omega || !sigma || n_omega < 0) return set_error(ctx, CDWAC_ERR_ARG, "bad sigma args");
  if (pade && (pade->n_states != sys->n_states || pade->n_occ != sys->n_occ))
    return set_error(ctx, CDWAC_ERR_ARG, "pade arrays do not match the system");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (n_omega == 0) return CDWAC_OK;
  {
    ProfScope ps(ctx, PROF_SIGMA, st);
    if ((rc = launch_sigma_wac(ctx, sys, prm, xi, wxi, W_imag, pade, omega, n_omega, sigma, st))) return rc;
  }
  if (pade) return CDWAC_OK;
  // plain CD: residues need the frequencies and eigenvalues on the host
  std::vector<double> w(n_omega), e(sys->n_basis);
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(w.data(), omega, sizeof(double) * n_omega, cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(e.data(), sys->eps, sizeof(double) * sys->n_basis, cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return plain_cd_residues(ctx, sys, prm, e, w, sigma, n_omega, 0, st);
}

// Plain-CD quasiparticle solve for one state: host-driven fixed point, one Sigma evaluation per iteration.
// One state's QP equation with plain CD; eps (host) are the energies of G, en the eps_n of the equation.
// Optional (evGW): sub_W, whose device energies give W's transition energies (default: sub's); W_zero_s, the
// state's W_nm(0) row for the closed-form part of the I term.  The fixed point starts from en.
static cdwac_status qp_plain_cd_state(cdwac_ctx* ctx, const cdwac_system* sub, const cdwac_params* prm,
                                      const double* xi, const double* wxi, const double* W_imag_s,
                                      const std::vector<double>& eps, double en, double sh,
                                      const std::vector<double>& grid, double tol, int max_iter, double* out_e,
                                      double* out_z, int* out_it, int* out_st, double* dsig, cudaStream_t st,
                                      const cdwac_system* sub_W = nullptr, const double* W_zero_s = nullptr) {
  auto resig = [&](double w, double* val) -> cdwac_status {
    cdwac_status r;
    std::vector<double> wv(1, w);
    // omega must be on the device for the I term: reuse dsig[2..] as the frequency slot
    CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(dsig + 2, &w, sizeof(double), cudaMemcpyHostToDevice, st));
    if ((r = launch_sigma_wac(ctx, sub, prm, xi, wxi, W_imag_s, nullptr, dsig + 2, 1, dsig, st, W_zero_s))) return r;
    if ((r = plain_cd_residues(ctx, sub_W ? sub_W : sub, prm, eps, wv, dsig, 1, 0, st))) return r;
    double h[2];
    CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(h, dsig, sizeof(h), cudaMemcpyDeviceToHost, st));
    CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    *val = h[0];
    return CDWAC_OK;
  };
  const double hstep = 1e-5;
  auto zfac = [&](double e, double* z) -> cdwac_status {
    double a = 0.0, b = 0.0;
    cdwac_status r;
    if ((r = resig(e + hstep, &a))) return r;
    if ((r = resig(e - hstep, &b))) return r;
    *z = 1.0 / (1.0 - (a - b) / (2.0 * hstep));
    return CDWAC_OK;
  };
  cdwac_status rc;
  double e = en, e_new = e, s = 0.0;
  for (int it = 1; it <= max_iter; ++it) {
    if ((rc = resig(e, &s))) return rc;
    e_new = en + sh + s;
    if (fabs(e_new - e) < tol) {
      *out_e = e_new;
      *out_it = it;
      *out_st = 0;
      return zfac(e_new, out_z);
    }
    e = e_new;
  }
  *out_it = max_iter;
  bool found = false;
  double be = 0, bz = 0;
  auto f = [&](double w, double* v) -> cdwac_status {
    double sv = 0.0;
    cdwac_status r = resig(w, &sv);
    *v = w - en - sh - sv;
    return r;
  };
  double fprev;
  if ((rc = f(grid[0], &fprev))) return rc;
  for (size_t j = 0; j + 1 < grid.size(); ++j) {
    double fnext;
    if ((rc = f(grid[j + 1], &fnext))) return rc;
    if (fprev == 0.0 || fprev * fnext < 0.0) {
      double lo = grid[j], hi = grid[j + 1], flo = fprev;
      for (int b = 0; b < 200 && hi - lo > 1e-9; ++b) {
        double mid = 0.5 * (lo + hi), fm;
        if ((rc = f(mid, &fm))) return rc;
        if (fm * flo <= 0.0) {
          hi = mid;
        } else {
          lo = mid;
          flo = fm;
        }
      }
      double r = 0.5 * (lo + hi), fr;
      if ((rc = f(r, &fr))) return rc;
      if (fabs(fr) < 1e-6) {
        double zr;
        if ((rc = zfac(r, &zr))) return rc;
        if (zr > 0.0 && zr <= 1.0 && (!found || zr > bz)) {
          found = true;
          be = r;
          bz = zr;
        }
      }
    }
    fprev = fnext;
  }
  if (found) {
    *out_e = be;
    *out_z = bz;
    *out_st = 1;
    return CDWAC_OK;
  }
  *out_e = e;
  *out_st = 2;
  return zfac(e, out_z);
}

cdwac_status cdwac_qp_solve(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                            const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* shift,
                            const double* omega, int n_grid, double tol, int max_iter, double* e_qp, double* Z,
                            int* iters, int* qp_status, void* stream) {
  cdwac_status rc = check_system(ctx, sys, prm);
  if (rc) return rc;
  if (!xi || !wxi || !W_imag || !omega || n_grid < 2 || !e_qp || !Z || !iters || !qp_status || max_iter < 1 ||
      !(tol > 0))
    return set_error(ctx, CDWAC_ERR_ARG, "bad qp_solve args");
  if (pade && (pade->n_states != sys->n_states || pade->n_occ != sys->n_occ))
    return set_error(ctx, CDWAC_ERR_ARG, "pade arrays do not match the system");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (pade) {
    ProfScope ps(ctx, PROF_QP, st);
    return launch_qp_wac(ctx, sys, prm, xi, wxi, W_imag, pade, shift, omega, n_grid, tol, max_iter, e_qp, Z, iters,
                         qp_status, st);
  }
  // plain CD: host-driven iteration per state
  const int ns = sys->n_states, nb = sys->n_basis;
  std::vector<double> e(nb), grid(n_grid), sh(ns, 0.0);
  std::vector<int> states(ns);
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(e.data(), sys->eps, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(grid.data(), omega, sizeof(double) * n_grid, cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(states.data(), sys->states, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
  if (shift) CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(sh.data(), shift, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  double* dsig = nullptr;
  CDWAC_CUDA_TRY(ctx, cudaMalloc(&dsig, 4 * sizeof(double)));
  std::vector<double> he(ns), hz(ns);
  std::vector<int> hit(ns), hst(ns);
  for (int s = 0; s < ns && rc == CDWAC_OK; ++s) {
    cdwac_system sub = *sys;
    sub.n_states = 1;
    sub.states = sys->states + s;
    sub.O_n = sys->O_dtype == CDWAC_F64 ? (const void*)((const double*)sys->O_n + (long)s * sys->n_aux * nb)
                                        : (const void*)((const float*)sys->O_n + (long)s * sys->n_aux * nb);
    rc = qp_plain_cd_state(ctx, &sub, prm, xi, wxi, W_imag + (long)s * prm->n_imag * nb, e, e[states[s]], sh[s],
                           grid, tol, max_iter, &he[s], &hz[s], &hit[s], &hst[s], dsig, st);
  }
  cudaFree(dsig);
  if (rc) return rc;
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(e_qp, he.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(Z, hz.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(iters, hit.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(qp_status, hst.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
  CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return CDWAC_OK;
}

}  // extern "C"

// ---- eigenvalue self-consistency beyond G0W0 (evGW0, evGW) -------------------------------------------------

namespace {
struct EvBufs {
  double *epsG, *xi, *wxi, *W, *W0, *zero, *dsig;
  cplx *pa, *pz2;
  int *nodes, *used, *iters;
};

void carve_ev(Arena& a, EvBufs& b, int nb, int ns, int ni, int n_occ, int M) {
  b.epsG = a.take<double>(nb);
  b.xi = a.take<double>(ni);
  b.wxi = a.take<double>(ni);
  b.W = a.take<double>((size_t)ns * ni * nb);
  b.W0 = a.take<double>((size_t)ns * nb);
  b.zero = a.take<double>(1);
  b.dsig = a.take<double>(4);
  b.pa = a.take<cplx>((size_t)ns * n_occ * M);
  b.pz2 = a.take<cplx>((size_t)ns * n_occ * M);
  b.nodes = a.take<int>((size_t)ns * n_occ * M);
  b.used = a.take<int>((size_t)ns * n_occ);
  b.iters = a.take<int>(ns);
}

// Frees a call's own device tables once the work queued on its stream (lanes and side streams are joined back to
// it before each internal call returns) has finished, on every return path.
struct StreamFree {
  void* p;
  cudaStream_t st;
  ~StreamFree() {
    if (!p) return;
    cudaStreamSynchronize(st);
    cudaFree(p);
  }
};
}  // namespace

extern "C" cdwac_status cdwac_evgw(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, int mode,
                                   int plain_cd, const double* shift, const double* omega, int n_grid,
                                   double cycle_tol, int max_cycles, double* e_qp, double* Z, int* qp_status,
                                   int* cycles, void* stream) {
  cdwac_status rc = check_system(ctx, sys, prm);
  if (rc) return rc;
  if ((mode != CDWAC_EVGW0 && mode != CDWAC_EVGW) || (plain_cd != 0 && plain_cd != 1) || !omega || n_grid < 2 ||
      !e_qp || !Z || !qp_status || !cycles || !(cycle_tol > 0) || max_cycles < 1)
    return set_error(ctx, CDWAC_ERR_ARG, "bad evgw args");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int ns = sys->n_states, nb = sys->n_basis, n_occ = sys->n_occ, ni = prm->n_imag, M = prm->pade_M;
  // each cycle's QP equation is solved ten times tighter than the self-consistency it is judged by
  const double inner_tol = std::min(1e-7, 0.1 * cycle_tol);
  // tables kept across the cycles (the W builds use the context scratch for their own work)
  Arena dry(nullptr);
  EvBufs b;
  carve_ev(dry, b, nb, ns, ni, n_occ, M);
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, dry.off + 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, CDWAC_ERR_OOM, "evgw tables (%zu bytes): %s", dry.off, cudaGetErrorString(e));
  }
  StreamFree guard{buf, st};
  Arena ar(buf);
  carve_ev(ar, b, nb, ns, ni, n_occ, M);
  std::vector<double> hG(nb), hK(nb), he(ns), hz(ns), hsh(ns, 0.0), hgrid(n_grid);
  std::vector<int> hs(ns), hst(ns), hit(ns);
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(b.epsG, sys->eps, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st));
  CDWAC_CUDA_TRY(ctx, cudaMemsetAsync(b.zero, 0, sizeof(double), st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(hK.data(), sys->eps, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(hs.data(), sys->states, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(hgrid.data(), omega, sizeof(double) * n_grid, cudaMemcpyDeviceToHost, st));
  if (shift) CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(hsh.data(), shift, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
  CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  hG = hK;
  for (int s = 0; s < ns; ++s)
    if (hs[s] < 0 || hs[s] >= nb) return set_error(ctx, CDWAC_ERR_ARG, "state index %d out of range", hs[s]);
  cdwac_system sysG = *sys;   // G from eps_G
  sysG.eps = b.epsG;
  cdwac_pade pade{ns, n_occ, M, reinterpret_cast<double*>(b.pa), reinterpret_cast<double*>(b.pz2), b.nodes, b.used};
  cdwac_params p0 = *prm;     // W(0): one frequency at xi = 0
  p0.n_imag = 1;
  // evGW0 keeps W (and for CD-WAC the near-real references and fits) of the KS energies; evGW rebuilds them
  // from eps_G every cycle
  const cdwac_system* sw = mode == CDWAC_EVGW ? &sysG : sys;
  int cyc = 1, outcome = 0;   // 1 self-consistent, 2 a QP equation without solution, 3 a level crossed eps_F
  for (; cyc <= max_cycles; ++cyc) {
    if (cyc == 1 || mode == CDWAC_EVGW) {
      if ((rc = cdwac_build_W_imag(ctx, sw, prm, b.xi, b.wxi, b.W, st))) return rc;
      if ((rc = build_W_freqs(ctx, sw, &p0, b.zero, b.W0, st))) return rc;
      if (!plain_cd && (rc = cdwac_fit_pade(ctx, sw, prm, b.xi, b.W, nullptr, nullptr, &pade, st))) return rc;
    }
    if (!plain_cd) {
      {
        ProfScope ps(ctx, PROF_QP, st);
        if ((rc = launch_qp_wac(ctx, &sysG, prm, b.xi, b.wxi, b.W, &pade, shift, omega, n_grid, inner_tol, 100,
                                e_qp, Z, b.iters, qp_status, st, b.W0, sys->eps)))
          return rc;
      }
      CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(he.data(), e_qp, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
      CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(hst.data(), qp_status, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
      CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    } else {
      // plain CD, one state at a time: I term on G's energies, residues with W of sw's transition energies
      for (int s = 0; s < ns; ++s) {
        cdwac_system subG = sysG;
        subG.n_states = 1;
        subG.states = sys->states + s;
        subG.O_n = sys->O_dtype == CDWAC_F64 ? (const void*)((const double*)sys->O_n + (long)s * sys->n_aux * nb)
                                             : (const void*)((const float*)sys->O_n + (long)s * sys->n_aux * nb);
        cdwac_system subW = subG;
        subW.eps = sw->eps;
        if ((rc = qp_plain_cd_state(ctx, &subG, prm, b.xi, b.wxi, b.W + (long)s * ni * nb, hG, hK[hs[s]], hsh[s],
                                    hgrid, inner_tol, 100, &he[s], &hz[s], &hit[s], &hst[s], b.dsig, st, &subW,
                                    b.W0 + (long)s * nb)))
          return rc;
      }
      CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(e_qp, he.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st));
      CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(Z, hz.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st));
      CDWAC_CUDA_TRY(ctx, cudaMemcpyAsync(qp_status, hst.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, st));
      CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    }
    double dmax = 0.0;
    for (int s = 0; s < ns; ++s) {
      if (hst[s] == 2) outcome = 2;
      dmax = fmax(dmax, fabs(he[s] - hG[hs[s]]));
    }
    if (outcome == 2) break;
    if (dmax < cycle_tol) {
      outcome = 1;
      break;
    }
    for (int s = 0; s < ns; ++s) hG[hs[s]] = he[s];
    // every transition energy eps_a - eps_i must stay positive
    const double top_occ = *std::max_element(hG.begin(), hG.begin() + n_occ);
    const double low_virt = *std::min_element(hG.begin() + n_occ, hG.end());
    if (!(top_occ < low_virt)) {
      outcome = 3;
      break;
    }
    if ((rc = launch_scatter_states(ctx, b.epsG, sys->states, e_qp, ns, st))) return rc;
  }
  *cycles = cyc > max_cycles ? max_cycles : cyc;
  CDWAC_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (outcome == 1) return CDWAC_OK;
  return set_error(ctx, CDWAC_ERR_QP_NOT_CONVERGED,
                   outcome == 2   ? "evgw: a QP equation has no solution (cycle %d)"
                   : outcome == 3 ? "evgw: an updated level crossed the Fermi level (cycle %d)"
                                  : "evgw: not self-consistent after %d cycles",
                   *cycles);
}

// ---- learned continuation in the residue term -------------------------------------------------------------

extern "C" cdwac_status cdwac_sigma_poles(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm,
                                          const double* xi, const double* wxi, const double* W_imag,
                                          const double* poles, const double* omega, int n_omega, double* sigma,
                                          void* stream) {
  cdwac_status rc = check_system(ctx, sys, prm);
  if (rc) return rc;
  if (!xi || !wxi || !W_imag || !poles || !omega || !sigma || n_omega < 0)
    return set_error(ctx, CDWAC_ERR_ARG, "bad sigma_poles args");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  if (n_omega == 0) return CDWAC_OK;
  ProfScope ps(ctx, PROF_SIGMA, (cudaStream_t)stream);
  return launch_sigma_poles(ctx, sys, prm, xi, wxi, W_imag, poles, omega, n_omega, sigma, (cudaStream_t)stream);
}

extern "C" cdwac_status cdwac_qp_solve_poles(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm,
                                             const double* xi, const double* wxi, const double* W_imag,
                                             const double* poles, const double* shift, const double* omega,
                                             int n_grid, double tol, int max_iter, double* e_qp, double* Z, int* iters,
                                             int* qp_status, void* stream) {
  cdwac_status rc = check_system(ctx, sys, prm);
  if (rc) return rc;
  if (!xi || !wxi || !W_imag || !poles || !omega || n_grid < 2 || !e_qp || !Z || !iters || !qp_status ||
      max_iter < 1 || !(tol > 0))
    return set_error(ctx, CDWAC_ERR_ARG, "bad qp_solve_poles args");
  CDWAC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
  ProfScope ps(ctx, PROF_QP, (cudaStream_t)stream);
  return launch_qp_poles(ctx, sys, prm, xi, wxi, W_imag, poles, shift, omega, n_grid, tol, max_iter, e_qp, Z, iters,
                         qp_status, (cudaStream_t)stream);
}
