/*
 * fh.h -- C ABI of the GB300 FFT/CG homogenization library (libfh.so).
 *
 * The library solves the trigonometric-collocation Lippmann-Schwinger system
 * of Zeman et al., "Accelerating a FFT-based solver for numerical
 * homogenization of periodic media by conjugate gradients":
 *
 *     (I + B) e = e0,   B = F^-1 Gamma0 F dL          (Eq. linear_system, Eq. mtrx_B)
 *
 * for the periodic field e on a grid N = (N_0, ..., N_{d-1}) under a
 * prescribed macroscopic field E (Eq. problem_def_2), with
 *   dL(x)     = L(x) - L0                              (Eq. current_decomp)
 *   Gamma0(k) = xi (x) xi / (xi . L0 . xi), Gamma0(0)=0, xi_a = k_a / Y_a  (Section 2.1)
 * for k in Z^N (Section 2.2).  The paper's grids are odd; on an even axis the
 * library takes Gamma0 = 0 at every frequency with a Nyquist component
 * k_a = N_a / 2 (the solution is then the equilibrium solution among the
 * trigonometric polynomials without Nyquist modes)
 * and returns the effective tensor L_eff[:, b] = <L e^(b)> (nodal mean).
 *
 * Conventions for every call:
 *  - Status codes only; nothing aborts or throws across the ABI.  On error
 *    fh_last_error(ctx) returns a message.
 *  - Fields are component-major ("SoA") [d][N_0]...[N_{d-1}], C-order, the
 *    last axis contiguous; node i sits at pixel coordinate i.
 *  - Pointers documented as "device" must be CUDA device (or managed)
 *    memory owned by the caller; "host" pointers are ordinary host memory.
 *    The library never frees caller memory and keeps no caller pointer
 *    after a call returns.
 *  - The context owns every internal device buffer (spectra, Krylov vectors,
 *    scalars); it is allocated in fh_create and freed in fh_destroy.
 *  - All device work is enqueued on the CUDA stream given to fh_create.
 *    fh_apply does not synchronise.  fh_solve synchronises on the stream
 *    only to read its small status word between iteration chunks, and
 *    before returning.
 *  - One context must not be used from two host threads at once.
 */
#ifndef FH_H_
#define FH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fh_ctx fh_ctx;

typedef enum {
  FH_OK = 0,
  FH_ERR_ARG = 1,            /* invalid argument (null pointer, bad d/N/tol ...) */
  FH_ERR_EVEN_N = 2,         /* reserved: even axis lengths are accepted (Nyquist
                                frequencies carry no Green operator, see above) */
  FH_ERR_NOT_SPD = 3,        /* a phase tensor or L0 is not symmetric positive definite */
  FH_ERR_OOM = 4,            /* device allocation failed */
  FH_ERR_CUDA = 5,           /* a CUDA runtime call failed */
  FH_ERR_NOT_CONVERGED = 6,  /* iteration cap reached before the tolerance */
  FH_ERR_BREAKDOWN = 7,      /* (A p, p) <= 0, a zero BiCG denominator, or a non-finite scalar */
  FH_ERR_TIMEOUT = 8,        /* a bounded device wait expired */
  FH_ERR_UNSUPPORTED = 9     /* size/precision without a compiled FFT plan */
} fh_status;

typedef enum {
  FH_CG = 0,           /* conjugate gradients, Saad Alg. 6.18 (Section 2.3) */
  FH_BICG = 1,         /* biconjugate gradients, Saad Alg. 7.3, shadow r0* = r0 (Section 3) */
  FH_FIXED_POINT = 2   /* Moulinec-Suquet Neumann iteration, Eq. (orig_fft) */
} fh_method;

typedef enum {
  FH_FP64 = 0,         /* every vector and FFT in float64 */
  FH_FP32 = 1,         /* float32 vectors and FFTs, float64 scalars (no refinement) */
  FH_FP32_REFINED = 2  /* float32 inner solves on A d = r, float64 outer residual
                          r = e0 - A x and float64 x += d until the float64 residual
                          meets the tolerance.  The outer residual's fields and
                          pointwise work are float64; in 2-D its FFTs run in
                          double-float arithmetic (two float32 parts, ~48 bits:
                          residual accurate to ~1e-14 |e0| instead of ~1e-16) */
} fh_precision;

/* Per-solve report.  history/history_cap are inputs (a host buffer for the
 * relative recursive residual of every inner iteration; may be NULL/0). */
typedef struct {
  int iters;              /* inner iterations over all refinement steps */
  int outer_iters;        /* float64 refinement steps (0 unless FH_FP32_REFINED) */
  int matvecs;            /* applications of A or A^T */
  int status;             /* fh_status of this solve */
  double rel_res_true;    /* ||e0 - A e||_2 / ||e0||_2 recomputed at exit (float64 for
                             FH_FP64 and FH_FP32_REFINED, float32 pipeline for FH_FP32) */
  double rel_res;         /* last recursive relative residual of the inner solver */
  double eta_r;           /* Eq. (errR_def) as printed: ||L0 (e_{m+1} - e_m)|| / ||e0|| */
  double eta_e;           /* Eq. (errE_def) of the returned field (float64), when
                             flags has FH_INFO_ETA_E; NaN otherwise */
  double* history;        /* in: host buffer or NULL */
  int history_cap;        /* in: its capacity */
  int history_len;        /* out: entries written */
  long long launches;     /* out: CUDA kernels this call launched (graph replays included) */
  int flags;              /* in: FH_INFO_ETA_E requests eta_e (one float64 operator pass) */
  int ct_plans;           /* out: FH_CT_* bits of the compile-time FFT plans whose kernels
                             ran every pass of the float32 CG iterations of this call
                             (0: run-time-plan kernels, or no float32 CG iteration) */
  /* Per-iteration norms of Section 3, FH_FP64 and FH_FP32 contexts (fh_solve
   * only; ignored for FH_FP32_REFINED, whose inner iterates are corrections):
   * host buffers of history_cap doubles, or NULL.  eta_e_history[m] is
   * Eq. (errE_def) of the iterate after m iterations (one more operator-pass
   * set per iteration); eta_r_history[m] is Eq. (errR_def) as printed,
   * ||L0 (e_{m+1} - e_m)|| / ||e0||, for an isotropic L0 (NaN otherwise). */
  double* eta_e_history;
  double* eta_r_history;
  int eta_e_len;          /* out: entries of eta_e_history written */
  int eta_r_len;          /* out: entries of eta_r_history written */
} fh_info;

/* fh_info.flags bits */
#define FH_INFO_ETA_E 1

/* fh_info.ct_plans bits: compile-time plans of the float32 CG-iteration passes */
#define FH_CT_2187 1      /* 2-D, one load per launch, 2187 = 27 * 27 * 3 along both axes */
#define FH_CT_729 2       /* 2-D, two loads per launch, 729 = 27 * 27 along both axes */
#define FH_CT_243 4       /* 3-D, one or three loads per launch, 243 = 27 * 9 along every axis */

/* fh_create -- build a solver context for one microstructure.
 *
 * Problem statement of Section 2.1 / 2.2: cell Y = prod (-Y_a, Y_a), grid N,
 * phase image, per-phase conductivity tensors L, reference medium L0.
 *
 *  out        host; receives the context (NULL on failure).
 *  d          2 or 3.
 *  N          host, d ints, each >= 3; supported lengths are those that
 *             factor into 2, 3, 5, 7, 11, 13 and 17 (an even length, or one
 *             with a factor 11, 13 or 17 such as the 255 = 3 * 5 * 17 grid of
 *             Section 3, runs the extended-radix kernels one load per launch).
 *  Y          host, d half side lengths (> 0), or NULL for all ones.
 *  phase      |N| bytes in C order, phase id per node (< nphase); a host
 *             pointer if phase_on_device == 0, else a device pointer.
 *             Copied into the context.
 *  nphase     1..256.
 *  L          host, nphase*d*d float64, row-major tensor per phase, each SPD.
 *  L0         host, d*d float64 SPD, or NULL for Eq. (opt_ref):
 *             (lambda_min + lambda_max)/2 I over all phase eigenvalues.
 *  precision  an fh_precision; decides which buffers are allocated
 *             (FH_FP32_REFINED allocates both float32 and float64 paths).
 *  stream     cudaStream_t (as void*), or NULL for the legacy default stream.
 *
 * Errors: FH_ERR_ARG, FH_ERR_NOT_SPD, FH_ERR_UNSUPPORTED, FH_ERR_OOM,
 * FH_ERR_CUDA.  On error nothing is leaked. */
fh_status fh_create(fh_ctx** out, int d, const int* N, const double* Y,
                    const uint8_t* phase, int phase_on_device, int nphase,
                    const double* L, const double* L0, int precision, void* stream);

/* fh_set_phase -- replace the phase image (same grid, same phase table).
 * phase: |N| bytes, host (phase_on_device == 0) or device.  Enqueued on the
 * context stream; a host source is copied synchronously. */
fh_status fh_set_phase(fh_ctx* ctx, const uint8_t* phase, int phase_on_device);

/* fh_apply -- one matrix-free product (Eq. linear_system, Eq. mtrx_B):
 *   transpose == 0:  e_out = (I + B) e_in   = e_in + F^-1 Gamma0 F (dL e_in)
 *   transpose != 0:  e_out = (I + B^T) e_in = e_in + dL F^-1 Gamma0 F e_in
 *  e_in, e_out  device, d*|N| elements [d][N...]; dtype FH_FP64 (double) or
 *               FH_FP32 (float).  e_in == e_out is allowed.
 *  dtype        FH_FP64 needs a context created with FH_FP64 or
 *               FH_FP32_REFINED; FH_FP32 needs FH_FP32 or FH_FP32_REFINED.
 * Asynchronous on the context stream.  Errors: FH_ERR_ARG, FH_ERR_CUDA. */
fh_status fh_apply(fh_ctx* ctx, const void* e_in, void* e_out, int transpose, int dtype);

/* fh_solve -- solve (I + B) e = e0 with e0 = E at every node.
 *  E          host, d float64 (the macroscopic field of Eq. problem_def_2).
 *  tol        > 0: stop when ||e0 - A e||_2 / ||e0||_2 <= tol.  The inner
 *             solver tests its recursive residual; FH_FP64 and FH_FP32_REFINED
 *             confirm with a float64 true residual before returning FH_OK.
 *  method     an fh_method.
 *  max_iter   cap on inner iterations (all refinement steps together).
 *  e_init     device float64 [d][N...] initial field, or NULL for e = E.
 *  e_out      device float64 [d][N...] for the solution, or NULL.
 *  Leff_col   host, d float64 for <L e> (column of L_eff for unit E), or NULL.
 *  info       host, or NULL.
 * The iterations of an inner solve run on the device in one graph launch
 * (a while node over chunks of iterations).  With the environment variable
 * FH_HOST_LOOP set (not "0") the same iterations are issued as ordinary
 * stream launches, one chunk at a time with the host testing the stop
 * conditions in between: slower, but visible launch by launch to profilers
 * that cannot look inside graphs with conditional nodes.
 * Returns FH_OK, FH_ERR_NOT_CONVERGED (the iteration cap, or the host's
 * iteration guard ran out without a device status; e_out still holds the
 * last iterate), FH_ERR_BREAKDOWN, FH_ERR_ARG, FH_ERR_CUDA, or FH_ERR_TIMEOUT
 * (a bounded device wait expired; the context stays usable). */
fh_status fh_solve(fh_ctx* ctx, const double* E, double tol, int method, int max_iter,
                   const double* e_init, double* e_out, double* Leff_col, fh_info* info);

/* fh_solve_all -- the full d x d effective tensor: the d unit loads E = e_1
 * ... e_d are solved together, each kernel launch carrying all d loads (for
 * FH_FP64 and FH_FP32_REFINED contexts; an FH_FP32 context solves them one by
 * one).  The first call allocates a second set of buffers sized for d loads,
 * kept until fh_destroy; grids with an axis that has a factor 11, 13 or 17
 * solve the loads one by one.  Leff receives L_eff row-major (column b from
 * load b).
 * infos: host array of d fh_info (iters, outer_iters, status, rel_res_true,
 * launches are filled), or NULL.  Returns the first non-OK status (the
 * statuses of fh_solve, FH_ERR_TIMEOUT included). */
fh_status fh_solve_all(fh_ctx* ctx, double tol, int method, int max_iter,
                       double* Leff, fh_info* infos);

/* fh_effective_column -- col[a] = mean over nodes of (L(x) e(x))_a, float64.
 *  e: device float64 [d][N...]; col: host, d doubles.  Synchronises. */
fh_status fh_effective_column(fh_ctx* ctx, const double* e, double* col);

/* fh_eta_e -- equilibrium norm of Eq. (errE_def) for field e (device float64):
 *   eta_e^2 = sum_k |xi . j^(k)|^2 / |j^(0)|^2,  j = L e.  Synchronises. */
fh_status fh_eta_e(fh_ctx* ctx, const double* e, double* eta);

/* fh_profile -- measurement hook (no counterpart in the paper; used to state
 * achieved bandwidth against the HBM roofline).  Times `reps` back-to-back
 * launches of one piece of the CG iteration on the context stream with CUDA
 * events after 3 warm-up launches, and writes the average milliseconds per
 * launch to *ms.  The context's Krylov vectors are overwritten (zeroed); any
 * solve state is lost.
 *  dtype  FH_FP64 or FH_FP32 (pipeline to time)
 *  what   0 row-forward pass (p = r + beta p, dL p, forward line FFTs)
 *         1 column passes with the Green projection
 *         2 row-inverse pass (inverse line FFTs, A p = p + y, (p, A p))
 *         3 CG vector update (x += alpha p, r -= alpha A p, (r, r))
 *         5 one full operator application (all passes of fh_apply)
 * Synchronises.  Errors: FH_ERR_ARG, FH_ERR_CUDA. */
fh_status fh_profile(fh_ctx* ctx, int dtype, int what, int reps, double* ms);

/* fh_autotune -- choose the launch shapes of the context's pipeline of the
 * given precision (FH_FP32 or FH_FP64) by timing candidates: half-spectrum
 * tile width, lines per CTA of the row passes, and the radix plan (threads per
 * line / column FFT).  Each candidate is a temporary set of buffers of the
 * same size as the context's; its four CG-iteration pass kernels are timed
 * with CUDA events (10 launches each).  If a faster shape is found the
 * pipeline is rebuilt with it (its Krylov vectors are reallocated, so any
 * solve state is lost).  When the environment variable FH_TUNE_CACHE names a
 * file, the result is appended to it, and fh_create reads that file to start
 * every later context of the same shape with the tuned launch shapes.
 *  ms_before / ms_after  host, may be NULL: summed pass time per CG iteration
 *                        before and after.
 * Synchronises.  Errors: FH_ERR_ARG, FH_ERR_OOM, FH_ERR_CUDA, FH_ERR_UNSUPPORTED. */
fh_status fh_autotune(fh_ctx* ctx, int dtype, double* ms_before, double* ms_after);

/* fh_autotune_loads -- the same search for the pipeline of fh_solve_all,
 * which carries all d unit loads in every launch (float32; FH_FP32 and
 * FH_FP32_REFINED contexts).  The best shapes are appended to the tuning
 * cache under this grid with d loads, and the next fh_solve_all uses them.
 * ms_before / ms_after (host, or NULL): float32 CG-iteration time of the
 * default and of the chosen shapes.  Errors: FH_ERR_ARG (FH_FP64 context),
 * FH_ERR_OOM, FH_ERR_CUDA. */
fh_status fh_autotune_loads(fh_ctx* ctx, double* ms_before, double* ms_after);

/* ---- Batches of independent 2-D cells (serving-style sweeps) ------------
 *
 * fh_batch_create -- many independent 2-D cells, possibly of different odd
 * sizes, solved together.  Cells of one size form a group; each group runs
 * every kernel over all of its cells in one launch (per-cell phase tables,
 * per-cell reference medium L0 = Eq. (opt_ref) of that cell's phases,
 * per-(cell, load) Krylov scalars; converged cells are skipped inside the
 * kernels), and the groups iterate concurrently on their own streams in
 * CUDA-graph chunks.
 *  out        host; receives the batch.
 *  ncells     >= 1.
 *  N          host, 2*ncells ints (N_0, N_1 of each cell; >= 3, factors
 *             3/5/7, or also 2/11/13/17 when nloads == 1).
 *  phase      host array of ncells host pointers, cell c has N_0*N_1 bytes.
 *  nphase     host, ncells ints in 1..256.
 *  L          host array of ncells host pointers, cell c has nphase[c]*4
 *             float64 (SPD 2x2 tensors, row-major).
 *  nloads     1 or 2 loads solved per cell.
 *  precision  FH_FP64 or FH_FP32_REFINED.
 * Everything is copied; the batch owns its device memory (one stream per
 * group).  Errors: FH_ERR_ARG, FH_ERR_NOT_SPD, FH_ERR_OOM, FH_ERR_CUDA,
 * FH_ERR_UNSUPPORTED. */
typedef struct fh_batch fh_batch;
fh_status fh_batch_create(fh_batch** out, int ncells, const int* N, const uint8_t* const* phase,
                          const int* nphase, const double* const* L, int nloads, int precision);

/* fh_batch_solve -- solve every (cell, load) to the float64 true relative
 * residual tol (Section 2.3 solvers; FP32 inner solves with float64
 * refinement for FH_FP32_REFINED).
 *  E        host, 2*nloads float64: the loads, E[2*l + a].
 *  Leff     host, ncells*2*nloads float64: Leff[(c*2 + a)*nloads + l] is
 *           component a of <L e> of cell c under load l (a column of the
 *           cell's effective tensor for a unit load).
 *  status   host, ncells*nloads fh_status per (cell, load), or NULL.
 *  iters    host, ncells*nloads inner iterations per (cell, load), or NULL.
 *  summary  host, or NULL: total iterations, refinement steps, worst true
 *           residual, kernels launched.
 * Returns FH_OK if every (cell, load) converged, else the first failure
 * status (FH_ERR_TIMEOUT when a bounded device wait expired,
 * FH_ERR_NOT_CONVERGED when the host's round guard ran out).  Synchronises. */
fh_status fh_batch_solve(fh_batch* b, const double* E, double tol, int method, int max_iter,
                         double* Leff, int* status, int* iters, fh_info* summary);

/* fh_batch_autotune -- pick the launch shapes of every size group's float32
 * pipeline (FH_FP32_REFINED batches) by timing a bounded set of candidates
 * on the group itself, as fh_autotune does for one cell.  ms_before /
 * ms_after (host, or NULL): the summed float32 CG-iteration time of all
 * groups before and after.  Synchronises.  Errors: FH_ERR_ARG, FH_ERR_OOM,
 * FH_ERR_CUDA. */
fh_status fh_batch_autotune(fh_batch* b, double* ms_before, double* ms_after);

/* Last error message of a batch (never NULL). */
const char* fh_batch_last_error(const fh_batch* b);

/* fh_batch_destroy -- free a batch.  NULL is a no-op. */
void fh_batch_destroy(fh_batch* b);

/* fh_apply_noalloc -- fh_apply for callers that cannot allocate device memory
 * (the paper has no counterpart; this is a deployment convenience).
 *
 * Some callers cannot call cudaMalloc: a host framework that owns all device
 * memory through its own pool and forbids outside allocations, a latency-
 * critical loop where cudaMalloc's implicit device synchronisation is not
 * acceptable, or an embedded user with a device-memory budget fixed at load
 * time.  This call computes the same float64 product as fh_apply,
 *   transpose == 0:  e_out = e_in + F^-1 Gamma0 F (dL e_in)
 *   transpose != 0:  e_out = e_in + dL F^-1 Gamma0 F e_in
 * without a context and without allocating: its spectrum scratch and its
 * twiddle and dL tables live in fixed arrays inside the library, about
 * 16.1 MiB that every GPU loading the library keeps until the process exits.
 *
 *  d, N, Y     as fh_create (d = 2 or 3, each axis <= 2187 and built from
 *              2, 3, 5, 7, 11, 13 and 17; Y may be NULL).  Grids whose float64 half
 *              spectrum exceeds 16 MiB (for example 2-D above ~1000^2, 3-D
 *              above ~85^3) are rejected with FH_ERR_UNSUPPORTED.
 *  phase       device, |N| bytes; ids >= nphase act as L = L0 (dL = 0).
 *  nphase, L   host, as fh_create.
 *  L0          host, d*d, required here (no default).
 *  e_in,e_out  device float64 [d][N...]; e_in == e_out is allowed.
 *  stream      cudaStream_t as void*, or NULL for the legacy default stream.
 *  errbuf      optional host buffer for a message (errlen bytes), may be NULL.
 *
 * All calls on one device share the fixed arrays and leave their contents
 * behind; every element is written before it is read within a call, so no
 * clearing is needed, but calls whose GPU work overlaps (different streams or
 * host threads) race and give wrong results: order them.  The first call on
 * each device (with that device current) performs a one-time set-up -- it
 * looks up the arrays' device addresses and raises the kernels' shared-memory
 * limit, both kept until the process exits -- and should come before any
 * stream capture on that device; resetting the device (cudaDeviceReset)
 * after that first call is not supported.  Every call is asynchronous on
 * `stream`: its twiddle and dL tables are filled by a kernel on that stream
 * (nothing is copied from host memory).  Errors: FH_ERR_ARG,
 * FH_ERR_NOT_SPD, FH_ERR_UNSUPPORTED, FH_ERR_CUDA. */
fh_status fh_apply_noalloc(int d, const int* N, const double* Y, const uint8_t* phase,
                           int nphase, const double* L, const double* L0, const double* e_in,
                           double* e_out, int transpose, void* stream, char* errbuf,
                           size_t errlen);

/* fh_set_wait_limit -- limit, in seconds, of the library's bounded device
 * waits (the persistent Green pass's bulk-copy waits, the tensor-core
 * convolution's commit waits): a wait that runs out ends its kernel with a
 * device error word, and the call that launched it returns FH_ERR_TIMEOUT
 * with its context still usable.  0 restores the default (2 s).  Applies to
 * kernels launched, and CUDA graphs captured, after the call; a context keeps
 * the graphs it captured earlier.  Process-wide.  (A failure-detection
 * setting; the paper has no counterpart.)  Errors: FH_ERR_ARG. */
fh_status fh_set_wait_limit(double seconds);

/* fh_wait_selftest -- runs one bounded wait of `seconds` on an mbarrier that
 * nothing completes, on `stream` (cudaStream_t as void*, NULL = legacy
 * default stream), and reports it: FH_ERR_TIMEOUT when the wait gave up as it
 * must (nothing is in flight, so the device stays usable), FH_OK if it
 * completed.  Synchronises the stream.  Errors: FH_ERR_ARG (seconds outside
 * (0, 60]), FH_ERR_CUDA. */
fh_status fh_wait_selftest(double seconds, void* stream);

/* fh_project_compatible -- out = Q in with Q = F^-1 Gamma0 F L0 (Section 2.1):
 * the projection onto the compatible (curl-free, zero-mean) fields along the
 * complement on which I + B acts as the identity.  A warm start x0 for the
 * load E is admissible for CG when x0 - E is compatible; use
 * x0 = E + Q (guess - E).  in, out: device float64 [d][N...] (in == out
 * allowed).  Float64 pipeline (float32 for FH_FP32 contexts).  Asynchronous.
 * Errors: FH_ERR_ARG, FH_ERR_CUDA. */
fh_status fh_project_compatible(fh_ctx* ctx, const double* in, double* out);

/* fh_destroy -- free the context and every buffer it owns.  NULL is a no-op. */
void fh_destroy(fh_ctx* ctx);

/* Human-readable name of a status code (static storage). */
const char* fh_status_string(int status);

/* Last error message recorded on ctx (static or context storage, never NULL). */
const char* fh_last_error(const fh_ctx* ctx);

/* Library version string. */
const char* fh_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FH_H_ */
