// cdwac_build_W_imag_noalloc: the FP64 W_nm(i xi) build with its scratch in a fixed device array.
//
// Some callers cannot call cudaMalloc while they run: a host application that hands a library a fixed device
// budget up front and forbids it from growing, or a latency-critical loop that cannot afford the device-wide
// synchronisation an allocation may cause.  For them this entry point takes no context and allocates nothing:
// the caller passes the system, the outputs and a device status word, and every intermediate (Pi, the LDL^T
// factor and its panels, Pi O, the solve vectors) lives in one file-scope __device__ array of
// CDWAC_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until the process exits.
//
// Set-up: the array's name is only a host-side stand-in in host code, so the first call on each device, with
// that device current, asks the runtime for the array's device address (cudaGetSymbolAddress) and keeps it.
// Make that first call before any stream capture.  All calls on a device share the one array and it keeps the
// last call's contents; nothing in it has to start at zero (every kernel writes what it later reads).  Two calls
// whose work overlaps on the GPU (different streams, no ordering between them) race on the array.
#include "common.cuh"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[CDWAC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_noalloc_addr[kMaxDevices] = {};

}  // namespace

extern "C" cdwac_status cdwac_build_W_imag_noalloc(const cdwac_system* sys, const cdwac_params* prm, double* xi,
                                                   double* wxi, double* W_imag, unsigned* dev_status, void* stream) {
  if (!sys || !prm || !xi || !wxi || !W_imag) return CDWAC_ERR_ARG;
  if (sys->n_basis < 2 || sys->n_occ < 1 || sys->n_occ >= sys->n_basis || sys->n_aux < 1 || sys->n_states < 1)
    return CDWAC_ERR_ARG;
  if (!sys->eps || !sys->O_ia || !sys->O_n || !sys->states) return CDWAC_ERR_ARG;
  if (sys->O_dtype != CDWAC_F64 && sys->O_dtype != CDWAC_F32) return CDWAC_ERR_ARG;
  if (prm->n_imag < 1 || prm->n_imag > 4096 || !(prm->omega0 > 0)) return CDWAC_ERR_ARG;
  if (prm->precision != CDWAC_PREC_FP64) return CDWAC_ERR_ARG;

  // scratch layout (same regions as the context path) and the size check, before anything is launched
  const int n = sys->n_aux, nb = sys->n_basis, n_occ = sys->n_occ, n_virt = nb - n_occ;
  const long n_ov = (long)n_occ * n_virt;
  const int cols = sys->n_states * nb;
  const int nblk = (n + 63) / 64;
  Arena probe(nullptr);
  probe.take<double>(n_ov);                                      // D
  probe.take<double>((size_t)n * n);                             // A = I - Pi (and -Pi above the diagonal)
  probe.take<double>(n);                                         // D^-1
  probe.take<double>((size_t)nblk * 64 * 64);                    // inverses of the diagonal blocks
  probe.take<double>(2 * (size_t)(nblk + 1) * 64 * 64);          // panels
  probe.take<double>(2 * quadform_scratch_elems<double>(n, cols));  // solve vectors
  probe.take<double>(n);                                         // diagonal of Pi
  probe.take<double>((size_t)sys->n_states * n * nb);            // Pi O
  if (probe.off > (size_t)CDWAC_NOALLOC_SCRATCH_BYTES) return CDWAC_ERR_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CDWAC_ERR_CUDA;
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CDWAC_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }

  cdwac_ctx ctx;          // stack context: no scratch, no profiler, no messages
  ctx.quiet = true;
  ctx.device = dev;
  ctx.d_status = dev_status;
  cudaDeviceGetAttribute(&ctx.num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = (cudaStream_t)stream;

  Arena ar(g_noalloc_addr[dev]);
  double* D = ar.take<double>(n_ov);
  double* A = ar.take<double>((size_t)n * n);
  double* dinv = ar.take<double>(n);
  double* linv = ar.take<double>((size_t)nblk * 64 * 64);
  double* wpanel = ar.take<double>(2 * (size_t)(nblk + 1) * 64 * 64);
  double* ywork = ar.take<double>(2 * quadform_scratch_elems<double>(n, cols));
  double* pidiag = ar.take<double>(n);
  double* V = ar.take<double>((size_t)sys->n_states * n * nb);

  cdwac_status rc;
  if ((rc = launch_gauss_legendre(&ctx, prm->n_imag, prm->omega0, xi, wxi, st))) return rc;
  if ((rc = launch_transition_energies(&ctx, sys->eps, n_occ, n_virt, D, st))) return rc;
  for (int k = 0; k < prm->n_imag; ++k) {
    if ((rc = launch_pi_imag_fp64(&ctx, sys->O_ia, sys->O_dtype, D, n, (int)n_ov, xi + k, A, pidiag, st))) return rc;
    if ((rc = ldlt_factor<double>(&ctx, A, n, dinv, linv, wpanel, st))) return rc;
    if ((rc = launch_pi_times_o(&ctx, A, pidiag, n, sys->O_n, sys->O_dtype, (long)n * nb, nb, sys->n_states, nb, V, st)))
      return rc;
    if ((rc = ldlt_quadform_pi(&ctx, A, dinv, linv, n, sys->O_n, sys->O_dtype, V, (long)n * nb, nb, sys->n_states, nb,
                               W_imag + (long)k * nb, (long)prm->n_imag * nb, ywork, st)))
      return rc;
  }
  return CDWAC_OK;
}
