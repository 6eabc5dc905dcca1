/*
 * cdwac.h -- C ABI of libcdwac.so: contour-deformation G0W0 self-energy of core levels with the analytic
 * continuation of W (CD-WAC), on one NVIDIA GB300 (sm_103a).
 *
 * The calls follow the paper's problem statement (Panades-Barrueta & Golze, arXiv 2305.15955):
 *   cdwac_build_W_imag  -- the wmatrix(F_Im) step of the G0W0 procedure (Sec. 3.4): Pi(i xi) (Eq. piriv),
 *                          Lambda = (I - Pi)^-1 - I (Eq. bigLambda) and W_nm(i xi) (Eq. wriv) on the
 *                          modified Gauss-Legendre grid (Sec. 4).
 *   cdwac_fit_pade      -- the wmatrix(F_real) and AC steps (Secs. 3.3, 3.4): W_nm at near-real reference
 *                          points, then one greedy Thiele continued fraction per (n, occupied m)
 *                          (Eqs. pade, pre_rec, rec_eq; Sec. 3.2).
 *   cdwac_sigma         -- Sigma^c_n(omega) = R_n(omega) - I_n(omega) (Eqs. In_term, Rn_term, ffact, cdselfe),
 *                          with R_n from the continued fraction (CD-WAC) or from W built directly at every
 *                          residue (plain CD).
 *   cdwac_qp_solve      -- the quasiparticle equation e = eps_n + Re Sigma_n(e) - v^xc_n (Eq. qp_eq) by
 *                          fixed-point iteration with a bracketed-bisection fallback.
 *
 * Conventions shared by every call
 *   - Units are Hartree.  Complex numbers are stored as two doubles (re, im).
 *   - Every pointer in cdwac_system, cdwac_pade and in the argument lists is DEVICE memory on the context's
 *     device unless stated otherwise.  The caller owns all inputs and outputs; the context owns its scratch.
 *   - Calls are asynchronous and ordered on the given CUDA stream (0 = legacy default stream).  The returned
 *     status reports argument and launch errors.  Errors found on the device (a non-positive Cholesky pivot,
 *     a singular complex pivot, a wait that ran out) are OR-ed into a device status word; cdwac_sync_status
 *     waits for the stream and returns the first of them.  No call aborts, traps or waits without a bound.
 *   - A context serves one device and one stream at a time; calls that overlap on two streams race on its
 *     scratch.  Internally a call may fork work from that stream onto the context's own streams (frequency
 *     lanes, the factorisation's critical-path and side streams) and joins them back before it returns.
 *   - Tuning read once when a context is created: CDWAC_FREQ_LANES (concurrent frequency lanes of a W build,
 *     1..16, default 8, further limited to half of the free device memory), CDWAC_LOOKAHEAD (0 runs the
 *     factorisation's bulk updates in line instead of on a side stream; default 1), CDWAC_PI_TILE (width of the
 *     tensor-core Pi tiles, 256 or 128; default 256), CDWAC_PI_GROUP (row blocks per group in the order of the Pi
 *     tiles, 1..64; default 12) and CDWAC_UPD_WAVES (CTA waves of the real trailing update's row-strip chunks,
 *     1..8; default 1); none of the last three changes a result beyond FP32 rounding in Pi.  A process that runs
 *     the default eight lanes does best with CUDA_DEVICE_MAX_CONNECTIONS=32 set before CUDA initialises
 *     (bench.py does so).
 */
#ifndef CDWAC_H
#define CDWAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CDWAC_OK = 0,
  CDWAC_ERR_ARG = 1,               /* bad argument: sizes, null pointers, unsupported combination */
  CDWAC_ERR_CUDA = 2,              /* a CUDA runtime call failed; cdwac_last_error has the text */
  CDWAC_ERR_NOT_SPD = 3,           /* I - Pi(i xi) had a non-positive Cholesky pivot */
  CDWAC_ERR_SINGULAR = 4,          /* I - Pi(z) had a (near) zero pivot in the complex LDL^T */
  CDWAC_ERR_PADE_BREAKDOWN = 5,    /* a Thiele fit stopped early (informational; the fit is still usable) */
  CDWAC_ERR_QP_NOT_CONVERGED = 6,  /* at least one state did not converge (per-state status has details) */
  CDWAC_ERR_TIMEOUT = 7,           /* a bounded device wait gave up */
  CDWAC_ERR_OOM = 8,               /* scratch allocation failed */
  CDWAC_ERR_UNSUPPORTED = 9        /* operation not available on this device / build */
} cdwac_status;

typedef enum { CDWAC_F64 = 0, CDWAC_F32 = 1 } cdwac_dtype;

/* Arithmetic of the W build.  FP64: every contraction in FP64 (parity path).  MIXED: Pi and the near-real
 * Pi(z) as split-BF16 (hi/lo, three products) tcgen05 tensor-core contractions with FP32 accumulation; the
 * Cholesky / LDL^T stays FP64-accurate (diagonal blocks and panels on the FP64 units, trailing updates as exact
 * BF16 digit products on the tensor cores, CDWAC_LDLT_EMULATED below); the W solves are blocked forward
 * substitutions on the FP64 factor whose products run as split-BF16 tensor-core GEMMs (FP32 block solves, FP64
 * sums of W); the Thiele fit and the residue sum stay FP64; the I_n quadrature terms are FP32 with FP64 partial
 * sums.  The mixed form's W(z) error is the BF16x3 error of Pi (~2e-5 relative) times cond(I - Pi(z)): large for
 * near-real points that lie among a strongly coupled system's excitations. */
typedef enum { CDWAC_PREC_FP64 = 0, CDWAC_PREC_MIXED = 1 } cdwac_precision;

/* Near-real reference set F_real of the core-state CD-WAC (Sec. 3.3); every point is x_j + i eta_ref with x_j >= 0
 * (first quadrant), one set per system shared by its requested states.
 *   GENERIC  omega_G: n_real equidistant x_j on [0, max_n |eps_F - eps_n| + real_margin], both ends included.
 *   REFINED  omega_C U omega_V, n_real = n_core + n_val: n_core equidistant x_j on the core neighbourhood
 *            [0, max_n eps_n - min_n eps_n + delta_c] (radius delta_c around the core-level residues |eps_n' - eps_n|
 *            at omega = eps_n, 0 for one state), then n_val equidistant x_j on the valence neighbourhood
 *            [max(0, min_n r_n - delta_v), max_n r_n + delta_v], r_n = |eps_F - eps_n|.  A region of one point
 *            holds the middle of its centres; an empty region holds none.
 * eps_F = (eps_HOMO + eps_LUMO) / 2 and n runs over the requested states. */
typedef enum { CDWAC_REAL_GENERIC = 0, CDWAC_REAL_REFINED = 1 } cdwac_real_set;

typedef struct cdwac_ctx cdwac_ctx;

/* One closed-shell system in the RI-V representation (Sec. 2.2).
 *   eps    [n_basis]                      ascending orbital energies; orbitals 0..n_occ-1 are occupied.
 *   O_ia   [n_aux][n_occ * n_virt]        O^{ia}_P with column ia = i * n_virt + a (a counts virtuals from 0),
 *                                         row-major, element type O_dtype; n_virt = n_basis - n_occ.
 *   O_n    [n_states][n_aux][n_basis]     O^{n m}_P of each requested state n for every orbital m, O_dtype.
 *   states [n_states] (int32)             orbital index n of each requested state.
 * The O^{ia} block and the occupied-virtual entries of O_n must describe one tensor (O^{nm} = O^{mn}). */
typedef struct {
  int n_basis, n_occ, n_aux, n_states;
  int O_dtype;                 /* cdwac_dtype */
  const double* eps;
  const void* O_ia;
  const void* O_n;
  const int* states;
} cdwac_system;

/* Method parameters (Secs. 3.2-3.4, 4).  cdwac_default_params fills the defaults noted here. */
typedef struct {
  int n_imag;          /* imaginary-axis Gauss-Legendre points (100) */
  double omega0;       /* grid map xi = omega0 (1 + x) / (1 - x) (1.0 Ha) */
  int n_real;          /* near-real reference points per state (40; 0 = imaginary only), set chosen by real_set */
  double eta_ref;      /* imaginary part of the near-real points (1e-3 Ha) */
  double real_margin;  /* GENERIC points span [0, |eps_F - eps_n| + real_margin] (0.5 Ha) */
  double eta;          /* broadening i*eta in I_n and R_n (1e-3 Ha) */
  int pade_M;          /* continued-fraction nodes per fit (64), at most n_imag + n_real and CDWAC_MAX_M */
  int greedy_first;    /* first node: 0 = argmax |W|, 1 = argmax Re W, 2 = candidate 0 */
  int greedy_crit;     /* later nodes: 0 = largest L1 error of the current convergent, 1 = smallest */
  int precision;       /* cdwac_precision */
  double pade_tol;     /* optional early end of a fit: stop once every remaining candidate is reproduced to an
                          L1 error below pade_tol * max|W| (0 = off, the paper's fixed M; default 0) */
  int real_set;        /* cdwac_real_set (GENERIC) */
  int n_core, n_val;   /* REFINED region sizes, n_core + n_val must equal n_real (20, 20: the paper's
                          CD-WAC(20, 20, N_Im) of Sec. 5.1); ignored by GENERIC */
  double delta_c;      /* REFINED core and valence neighbourhood radii (0.5 Ha, 0.5 Ha; Sec. 3.3 leaves them to */
  double delta_v;      /*   tuning) */
} cdwac_params;

#define CDWAC_MAX_M 256          /* largest continued fraction the fit kernel holds */
#define CDWAC_MAX_CANDIDATES 512 /* largest n_imag + n_real */

/* Thiele model of every (state n, occupied m): caller-owned device arrays sized from n_states, n_occ, M. */
typedef struct {
  int n_states, n_occ, M;      /* capacity the arrays were allocated for; M >= params.pade_M */
  double* a;                   /* [n_states][n_occ][M][2] coefficients a_p */
  double* z2;                  /* [n_states][n_occ][M][2] node values zt_p^2 */
  int* nodes;                  /* [n_states][n_occ][M] candidate index of node p: 0..n_imag-1 = i xi_k,
                                  n_imag + j = near-real point j */
  int* n_used;                 /* [n_states][n_occ] nodes actually used (< pade_M after a breakdown) */
} cdwac_pade;

/* ---- context ------------------------------------------------------------------------------------------ */

/* Creates a context on CUDA device `device` (makes it current for the calling thread).  *out is set to NULL
 * on failure.  Returns CDWAC_ERR_UNSUPPORTED if the device is not compute capability 10.3. */
cdwac_status cdwac_create(cdwac_ctx** out, int device);
/* Frees the context's scratch.  Waits for nothing: the caller must have synchronised its streams. */
void cdwac_destroy(cdwac_ctx* ctx);
/* Text of the last error on this context (static storage owned by the context, never NULL). */
const char* cdwac_last_error(const cdwac_ctx* ctx);
/* Fills *p with the defaults listed in cdwac_params. */
void cdwac_default_params(cdwac_params* p);
/* Waits for `stream`, reads and clears the device status word; returns CDWAC_OK or the first device error. */
cdwac_status cdwac_sync_status(cdwac_ctx* ctx, void* stream);
/* Bytes of context scratch currently held (grows on demand, released by cdwac_destroy). */
size_t cdwac_scratch_bytes(const cdwac_ctx* ctx);

/* ---- tracing ------------------------------------------------------------------------------------------ */

/* One kernel class of the event profiler: name (static string), launches of the class and their summed device
 * time (CUDA events recorded on the call's stream around each launch or launch group). */
typedef struct {
  const char* name;
  int launches;
  double total_ms;
} cdwac_profile_entry;

/* Per-kernel-class CUDA-event timers: on = 0 off (default), 1 kernel classes, 2 also each launch of the LDL^T
 * block steps (diag / panel / update).  Adds two event records per timed region and no synchronisation. */
void cdwac_profile_enable(cdwac_ctx* ctx, int on);
/* Waits for the recorded events, writes up to max_entries classes into out (classes never timed are skipped),
 * clears the accumulated times and returns the number written (negative on a CUDA error). */
int cdwac_profile_read(cdwac_ctx* ctx, cdwac_profile_entry* out, int max_entries);
/* Kernels launched through this context since it was created. */
long long cdwac_launch_count(const cdwac_ctx* ctx);

/* ---- the four steps ----------------------------------------------------------------------------------- */

/* W_nm(i xi_k) on the imaginary grid: the wmatrix(F_Im) step (Sec. 3.4; Eqs. piriv, bigLambda, wriv).
 *   xi, wxi  [n_imag]                        out: nodes xi_k (ascending) and quadrature weights of the
 *                                            modified Gauss-Legendre grid (Sec. 4), Jacobian included.
 *   W_imag   [n_states][n_imag][n_basis]     out: W^c_nm(i xi_k) for every m (real).
 * Pi(i xi) = -4 sum_ia O^ia_P O^ia_Q D_ia / (xi^2 + D_ia^2) (spin factor 2), I - Pi is factorised by FP64
 * Cholesky and W_nm = |L^-1 o_nm|^2 - |o_nm|^2 = o^T Lambda o.  Device error: CDWAC_ERR_NOT_SPD. */
cdwac_status cdwac_build_W_imag(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, double* xi,
                                double* wxi, double* W_imag, void* stream);

/* Near-real reference points, W there, and the greedy Thiele fits: the wmatrix(F_real) and AC steps.
 *   xi, W_imag                               in: output of cdwac_build_W_imag with the same prm.
 *   z_real   [n_states][n_real][2]           out (may be NULL): x_j + i eta_ref, the generic or refined set
 *                                            of prm->real_set (cdwac_real_set above).
 *   W_real   [n_states][n_real][n_occ][2]    out (may be NULL): W_nm(z_j) for the occupied m.
 *   pade                                     out: one fit per (n, occupied m) over the n_imag + n_real
 *                                            candidates (greedy ordering of Sec. 3.2).
 * Device error: CDWAC_ERR_SINGULAR.  A fit that breaks down keeps its first n_used nodes. */
cdwac_status cdwac_fit_pade(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                            const double* W_imag, double* z_real, double* W_real, const cdwac_pade* pade,
                            void* stream);

/* Sigma^c_n(omega_j) = R_n - I_n (Eq. cdselfe without the static exchange).
 *   xi, wxi, W_imag                          in: output of cdwac_build_W_imag.
 *   pade                                     in: CD-WAC model, or NULL for plain CD (W built directly at each
 *                                            residue |eps_m - omega| + i eta: one Pi(z) and one complex
 *                                            LDL^T per residue, the O(N^5) route).
 *   omega    [n_omega]                       in: real frequencies.  CD-WAC needs omega < eps_LUMO.
 *   sigma    [n_states][n_omega][2]          out. */
cdwac_status cdwac_sigma(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                         const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* omega,
                         int n_omega, double* sigma, void* stream);

/* Quasiparticle energies (Eq. qp_eq): e = eps_n + shift_n + Re Sigma^c_n(e), shift_n = Sigma^x_n - v^xc_n.
 *   shift    [n_states]                      in (may be NULL = 0).
 *   omega    [n_grid]                        in: bracketing grid of the bisection fallback.
 *   e_qp, Z  [n_states]                      out: solution and renormalisation 1 / (1 - dRe Sigma/d omega)
 *                                            (central difference, step 1e-5 Ha).
 *   iters, qp_status [n_states] (int32)      out: fixed-point iterations; 0 = fixed point converged
 *                                            (|e_k+1 - e_k| < tol), 1 = bracketed bisection, 2 = not converged.
 * CD-WAC (pade != NULL) runs entirely on the device.  Plain CD (pade == NULL) drives one residue build per
 * occupied orbital per iteration from the host and synchronises the stream between iterations. */
cdwac_status cdwac_qp_solve(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                            const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* shift,
                            const double* omega, int n_grid, double tol, int max_iter, double* e_qp, double* Z,
                            int* iters, int* qp_status, void* stream);

/* Eigenvalue self-consistency beyond G0W0 (Sec. 5.4) for the requested states, by CD-WAC (plain_cd 0) or by plain
 * CD (plain_cd 1: every residue builds W from the cycle's transition energies; the reference CD-WAC is judged by).
 * Cycle k solves the QP equation e_n = eps_n + shift_n + Re Sigma^c_n(e_n) (eps_n: sys->eps) of every requested
 * state with G built from eps_G: sys->eps with the requested entries replaced by the QP energies of cycle k-1
 * (cycle 1 is G0W0); every other orbital keeps its energy.
 *   mode CDWAC_EVGW0  W (imaginary grid, near-real references, residues) and the Thiele fits from sys->eps, built once.
 *        CDWAC_EVGW   W, the near-real references (placed from eps_G) and the fits rebuilt every cycle from eps_G.
 * The I term carries W_nm(0) in closed form (its Lorentzian integrates to sgn(omega - eps_m) pi / 2 whatever the
 * grid), since at self-consistency Sigma_n is evaluated at its own G energy, closer to it than the grid resolves.
 *   shift       [n_states]  in (device, may be NULL): Sigma^x_n - v^xc_n
 *   omega       [n_grid]    in (device): bracketing grid of the QP solver, as in cdwac_qp_solve (n_grid >= 2)
 *   cycle_tol               self-consistency reached when no requested state moves by cycle_tol (Ha) or more
 *   max_cycles              at least 1
 *   e_qp, Z, qp_status [n_states] out (device): the last cycle's QP solutions (qp_status as cdwac_qp_solve)
 *   cycles      [1]         out (HOST int): cycles run
 * Every cycle's QP fixed point starts from eps_n (the KS level, as in G0W0) and stops at |e_k+1 - e_k| <
 * min(1e-7, cycle_tol / 10) Ha, at most 100 iterations.
 * Host-driven: the call synchronises `stream` once per cycle.  Returns CDWAC_ERR_QP_NOT_CONVERGED (cdwac_last_error
 * says which) when a QP equation has no solution, when an updated level crosses the Fermi level (the transition
 * energies of W must stay positive) or when max_cycles pass without self-consistency; *cycles and the outputs then
 * hold the last cycle run.  Allocates its tables (eps_G, W, W(0), fits) for the call. */
typedef enum { CDWAC_EVGW0 = 0, CDWAC_EVGW = 1 } cdwac_ev_mode;
cdwac_status cdwac_evgw(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, int mode, int plain_cd,
                        const double* shift, const double* omega, int n_grid, double cycle_tol, int max_cycles,
                        double* e_qp, double* Z, int* qp_status, int* cycles, void* stream);

/* Diagonal spectral function (Sec. 5.5): A_nn(omega_j) = |Im[(omega_j - eps_n - shift_n - Sigma^c_n(omega_j))^-1]|
 * / pi, the imaginary part of the Green's function (normalised so that one quasiparticle pole carries weight one).
 * Sigma^c as in cdwac_sigma: CD-WAC from the continued fractions (pade != NULL) or plain CD (pade == NULL), which
 * the paper compares for a 50 eV window at 0.01 eV spacing (5000 points).
 *   shift    [n_states]                      in (may be NULL = 0): Sigma^x_n - v^xc_n.
 *   omega    [n_omega]                       in: real frequencies (CD-WAC needs omega < eps_LUMO).
 *   sigma    [n_states][n_omega][2]          out: Sigma^c_n(omega_j).
 *   A        [n_states][n_omega]             out. */
cdwac_status cdwac_spectral(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                            const double* wxi, const double* W_imag, const cdwac_pade* pade, const double* shift,
                            const double* omega, int n_omega, double* sigma, double* A, void* stream);

/* ---- the factorisation step on its own -------------------------------------------------------------- */

/* Trailing-update arithmetic of the LDL^T factorisation. */
typedef enum {
  CDWAC_LDLT_FP64 = 0,      /* every update on the FP64 FMA units */
  CDWAC_LDLT_EMULATED = 1   /* rank-64 trailing updates on the tcgen05 tensor cores from exact BF16 digits of
                               the FP64 operands (per row 7 digits of 8 bits, complex 8 of 7 bits; exact FP32
                               level sums recombined in 64-bit integers): FP64-equivalent accuracy */
} cdwac_ldlt_method;

/* Square-root-free Cholesky factorisation A = L D L^T of the symmetric matrix I - Pi of Eq. bigLambda (real
 * symmetric positive definite on the imaginary axis, complex symmetric without pivoting near the real axis).
 *   A  [n][n] device, row-major, FP64 (is_complex = 0) or interleaved complex FP64 (is_complex = 1).  Only the
 *      lower triangle is read; on return it holds the unit-lower L below the diagonal and D on the diagonal.
 *      The strict upper triangle is not touched.  The caller owns A; the context owns the scratch.
 * A non-positive real pivot (CDWAC_ERR_NOT_SPD) or a vanishing complex pivot (CDWAC_ERR_SINGULAR) goes to the
 * device status word and the factorisation continues with a unit pivot. */
cdwac_status cdwac_ldlt_factor(cdwac_ctx* ctx, void* A, int n, int is_complex, int method, void* stream);

/* ---- batched launch ------------------------------------------------------------------------------------ */

/* One system of a batch and its outputs (all device pointers; layouts as in the single-system calls). */
typedef struct {
  cdwac_system sys;
  double* xi;            /* [n_imag] */
  double* wxi;           /* [n_imag] */
  double* W_imag;        /* [n_states][n_imag][n_basis] */
  double* z_real;        /* [n_states][n_real][2] or NULL */
  double* W_real;        /* [n_states][n_real][n_occ][2] or NULL */
  cdwac_pade pade;       /* fits of this system (arrays sized for it) */
  const double* omega;   /* [n_omega] Sigma grid (n_omega may be 0) */
  int n_omega;
  double* sigma;         /* [n_states][n_omega][2] */
  const double* shift;   /* [n_states] or NULL */
  const double* qp_grid; /* [n_grid] bracketing grid of the QP fallback */
  int n_grid;
  double* e_qp;          /* [n_states] */
  double* Z;             /* [n_states] */
  int* iters;            /* [n_states] */
  int* qp_status;        /* [n_states] */
} cdwac_batch_item;

#define CDWAC_BATCH_GRAPH 1u     /* capture the whole batch into one CUDA graph and replay it */
#define CDWAC_BATCH_AUTOTUNE 2u  /* choose lanes, LDL^T lookahead and tile configuration by timing candidates
                                    (cached per size bucket) */

/* CD-WAC for many systems of uneven size in one stream-ordered call: the systems are spread over up to
 * `max_lanes` concurrent lanes (streams with their own scratch), largest first, and each runs W(i xi), the
 * near-real points, the Thiele fits, Sigma on its grid and the QP equation.  With CDWAC_BATCH_GRAPH the batch is
 * captured once into a CUDA graph (keyed on the item array's contents) and later calls with the same items
 * replay it: the items' buffers must stay valid.  With CDWAC_BATCH_AUTOTUNE the first call for a size bucket
 * times every lane count in {1, 2, 4, 8} <= max_lanes with and without the LDL^T lookahead, then, from the
 * fastest, the tile configuration of the tensor-core kernels: the Pi output tile width (128 x 256 or 128 x 128),
 * its tile-group size (output tiles ordered in groups of G row blocks; G in {4, 8, 12, 16}) and the number of CTA
 * waves (1, 2 or 3) the real trailing update's 128-row strips are cut into; it keeps the fastest.  The group size
 * and the waves change no result bit; the two Pi tile widths sum the same products in differently chunked FP32
 * accumulations (FP32 rounding).  Choices are appended to the file named by the environment
 * variable CDWAC_TUNE_CACHE (if set) and read back by later processes.  `chosen` (may be NULL; five ints)
 * receives {lanes, lookahead, Pi tile-group size, Pi tile width, update waves}.  The precision and parameters
 * are the same for every item. */
cdwac_status cdwac_batch_run(cdwac_ctx* ctx, const cdwac_batch_item* items, int n_items, const cdwac_params* prm,
                             double tol, int max_iter, int max_lanes, unsigned flags, int* chosen, void* stream);

/* ---- learned continuation (pole-residue MLP) ----------------------------------------------------------- */
/* Not in the paper: an alternative to the Thiele continuation in the residue term R_n (Eq. Rn_term).  A network
 * 32 -> 3 x 256 (GELU) -> 16 maps x_k = W_nm(i xi_{3k}) / s (k < 32, s = |W_nm(i xi_1)|) to 8 poles
 * Omega_s = softplus(o_s) + 0.05 Ha and residues r_s = softplus(o_{8+s}); the model is the sum-over-poles form of W
 * behind Eq. sigma_pole, W(z) = -s sum_s r_s 2 Omega_s / (Omega_s^2 - z^2) (<= 0 on the imaginary axis). */
#define CDWAC_MLP_IN 32
#define CDWAC_MLP_HIDDEN 256
#define CDWAC_MLP_POLES 8
/* FP32 parameters, per layer row-major weights [in][out] then bias: 32x256,256 | 256x256,256 | 256x256,256 | 256x16,16 */
#define CDWAC_MLP_NPARAMS (32 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 16 + 16)

/* Features and training targets of every (state, occupied m) pair, b = s * n_occ + m (B = n_states * n_occ):
 *   x [B][32] float, scale [B] float, z_ref and w_ref [B][32 + n_real][2]: the 32 imaginary nodes i xi_{3k} with
 *   W(i xi_{3k}), then the near-real points z_real[s][j] with W_real[s][j][m] (outputs of cdwac_build_W_imag and
 *   cdwac_fit_pade).  Needs n_imag >= 94. */
cdwac_status cdwac_mlp_features(cdwac_ctx* ctx, const double* xi, const double* W_imag, int n_states, int n_imag,
                                int n_basis, int n_occ, const double* z_real, const double* W_real, int n_real,
                                float* x, float* scale, double* z_ref, double* w_ref, void* stream);
/* One training gradient (FP32): loss = mean_b (1/J) sum_j |W_model(z_j) - w_ref_j|^2 / (scale_b^2 + |w_ref_j|^2)
 * (written to *loss, a device double) and its gradient with respect to params (grad [CDWAC_MLP_NPARAMS] float). */
cdwac_status cdwac_mlp_loss_grad(cdwac_ctx* ctx, const float* params, int batch, const float* x, const float* scale,
                                 int n_ref, const double* z_ref, const double* w_ref, float* grad, double* loss,
                                 void* stream);
/* Adam step on params with moments m, v (all [CDWAC_MLP_NPARAMS] float); step counts from 1. */
cdwac_status cdwac_mlp_adam(cdwac_ctx* ctx, float* params, const float* grad, float* m, float* v, int step, float lr,
                            float beta1, float beta2, float eps, void* stream);
/* Inference with BF16 copies of the weights: poles [batch][8][2] = (Omega_s, r_s * scale) in Ha. */
cdwac_status cdwac_mlp_poles(cdwac_ctx* ctx, const float* params, int batch, const float* x, const float* scale,
                             double* poles, void* stream);
/* cdwac_sigma / cdwac_qp_solve with the residue term from poles [n_states][n_occ][8][2] instead of Thiele fits. */
cdwac_status cdwac_sigma_poles(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                               const double* wxi, const double* W_imag, const double* poles, const double* omega,
                               int n_omega, double* sigma, void* stream);
cdwac_status cdwac_qp_solve_poles(cdwac_ctx* ctx, const cdwac_system* sys, const cdwac_params* prm, const double* xi,
                                  const double* wxi, const double* W_imag, const double* poles, const double* shift,
                                  const double* omega, int n_grid, double tol, int max_iter, double* e_qp, double* Z,
                                  int* iters, int* qp_status, void* stream);

/* ---- allocation-free variant ------------------------------------------------------------------------ */

/* Fixed device scratch of cdwac_build_W_imag_noalloc (held by every GPU that loads the library). */
#define CDWAC_NOALLOC_SCRATCH_BYTES (16u << 20)

/* cdwac_build_W_imag with precision CDWAC_PREC_FP64, for callers that must not allocate device memory while
 * they run (a host program that grants the library a fixed device budget, a latency-critical loop that cannot
 * take an allocation's device-wide synchronisation).  No context: the caller passes the system, the outputs
 * (same layouts as cdwac_build_W_imag) and `dev_status`, a device word into which pivot errors are OR-ed
 * (bit 0: I - Pi not positive definite; may be NULL).  Every intermediate lives in one fixed device array of
 * CDWAC_NOALLOC_SCRATCH_BYTES; a system whose intermediates do not fit (about n_aux^2 + n_occ*n_virt
 * + 3*n_states*n_basis*n_aux doubles; n_aux = 500 with one state of 600 orbitals fits) is rejected with
 * CDWAC_ERR_ARG before anything runs, as is precision != CDWAC_PREC_FP64.  The first call on a device (that device
 * current) looks up the array's device address; make it before any stream capture.  Calls share the array:
 * calls that overlap on the GPU race.  Calls no cudaMalloc/cudaFree.  The paper has no counterpart: this is an
 * interface variant of the wmatrix(F_Im) step only. */
cdwac_status cdwac_build_W_imag_noalloc(const cdwac_system* sys, const cdwac_params* prm, double* xi, double* wxi,
                                        double* W_imag, unsigned* dev_status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CDWAC_H */
