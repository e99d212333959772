/*
 * mlba.h — C ABI of the GB300 (sm_103a) library for the preconditioned
 * modified linearized Bregman algorithm (MLBA) for frame-based image
 * deblurring with reduced boundary artifacts (Cai, Donatelli, Bianchi,
 * Huang, arXiv 1504.07234).
 *
 * The model is g = A f + eta (Section 1, Eq. modeld): an n x n observed image
 * g, a p x p PSF (p odd, centred at ((p-1)/2, (p-1)/2)), noise norm
 * delta = ||eta||.  A is either the rectangular n^2 x m^2 "valid" operator
 * (m = n + p - 1, Section 2.1, Eq. Arect) or the square operator obtained by
 * imposing zero / periodic / reflective boundary conditions (Section 2.2,
 * Table 1).  One iteration (Eq. MLBA2 and Algorithms 1-4, 4-NS) is
 *
 *     r  = g - A f                                   (residual, FP64 norm)
 *     stop when ||r|| <= gamma*delta (n > 0)  or  ||r|| <= tau*delta (4-NS)
 *     t  = P r                                       (preconditioner)
 *     u  = A^T t      (Algorithms 1-3)   or  u = C^T (CC^T+alpha I)^{-1} r (4)
 *     z <- z + W u;   x = S_mu(z);   f = W^T x      (framelets, Section 6.1)
 *
 * Conventions
 *  - Images are dense row-major arrays without padding: g, r, t are n x n;
 *    f is N_f x N_f with N_f = m (rectangular A) or n (boundary conditions).
 *  - The element type of images is double (MLBA_F64) or float (MLBA_F32),
 *    chosen by mlba_opts.dtype.  The Bregman variable z is stored as
 *    (8*levels + 1) planes of N_f x N_f in mlba_opts.z_store precision, band
 *    order: the 8 high-pass bands (i,j) != (0,0) of level 1 in lexicographic
 *    order, then level 2, ..., then the final low-pass band.
 *  - "on_device" arguments: 1 = the pointer is device memory valid on the
 *    context's stream, 0 = host memory (the call then synchronises).
 *  - Every function returns MLBA_OK (0) or a negative status; nothing throws.
 *  - All work is queued on mlba_opts.stream (a cudaStream_t; NULL makes the
 *    library create and own a non-blocking stream, because the legacy
 *    default stream cannot be captured into a CUDA graph).  The library owns
 *    the device memory it allocates at create time (cudaMalloc) and frees it
 *    at destroy.
 *  - Calls on one context or batch are not thread-safe; distinct contexts
 *    are independent.
 */
#ifndef MLBA_H
#define MLBA_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MLBA_OK            0
#define MLBA_E_INVAL      (-1)  /* bad argument (p even, p > n, alpha <= 0, Algorithm 4 with rectangular A, ...) */
#define MLBA_E_NOMEM      (-2)  /* device or host allocation failed */
#define MLBA_E_CUDA       (-3)  /* a CUDA runtime call failed */
#define MLBA_E_TIMEOUT    (-4)  /* a bounded device-side wait expired */
#define MLBA_E_DIVERGED   (-5)  /* ||r|| became NaN or Inf */
#define MLBA_E_STATE      (-6)  /* call out of order (e.g. iterate before set_data) */
#define MLBA_E_UNSUPPORTED (-7) /* size not supported (a preconditioned n must be <= 4096; p <= MLBA_MAX_P) */

/* ---- enumerations ---------------------------------------------------- */
enum mlba_bc {                 /* Section 2, Table 1 */
  MLBA_BC_ZERO = 0,            /* Dirichlet: zero outside the field of view */
  MLBA_BC_PERIODIC = 1,        /* A is BCCB */
  MLBA_BC_REFLECTIVE = 2,      /* fliplr / flipud mirror (Neumann) */
  MLBA_RECT = 3,               /* rectangular n^2 x m^2 valid operator, Eq. Arect */
  MLBA_BC_ANTIREFLECTIVE = 4   /* 2 F(edge) - F(mirror) pad, corners antireflected row then
                                  column (Section 2.2); A^T is replaced by the reblurring
                                  matrix A' (the same BCs on the PSF rotated by 180 degrees).
                                  Algorithms 1, 3, 4 and 4-NS and P = I; not Algorithm 2 (the
                                  paper finds it of no use there). */
};

enum mlba_precond {            /* Sections 3-5 */
  MLBA_P_NONE = 0,             /* P = I: linearized Bregman, Eq. iterLinBreg (lambda = 1) */
  MLBA_P_BCCB = 1,             /* Algorithm 1: P = (CC^T + alpha I)^{-1}, Eq. Alg1 */
  MLBA_P_KRYLOV = 2,           /* Algorithm 2: PCG for (AA^T + alpha I) t = r, Eqs. syscg, psys, bet */
  MLBA_P_SYM = 3,              /* Algorithm 3: Q from the symmetrised PSF, Eq. Alg3 */
  MLBA_P_TIKH = 4,             /* Algorithm 4: z += W C^T (CC^T + alpha I)^{-1} r, Eq. Alg4 */
  MLBA_P_TIKH_NS = 5           /* Algorithm 4-NS: alpha_n from Eq. Alg4_rev_7 */
};

enum mlba_dtype { MLBA_F32 = 0, MLBA_F64 = 1, MLBA_BF16 = 2 };

enum mlba_transform {          /* diagonalising transform of C (Section 4.1) */
  MLBA_TR_AUTO = 0,            /* DFT for periodic BC (C = A); antireflective BC: the antireflective
                                  transform (C = A) for a quadrantally symmetric PSF outside 4-NS,
                                  else DFT; otherwise DCT for a quadrantally symmetric PSF, else DFT */
  MLBA_TR_DFT = 1,             /* C = periodic-BC (Strang) matrix */
  MLBA_TR_DCT = 2,             /* C = reflective-BC matrix; PSF must be quadrantally symmetric */
  MLBA_TR_AR = 3               /* C = antireflective-BC matrix (antireflective BCs only, Section 2.2):
                                  the sine basis of length n - 2 plus the constant and linear
                                  vectors; PSF quadrantally symmetric; not with 4-NS (the transform
                                  is not unitary) nor Algorithm 2; n <= 2049.  Algorithm 3 with
                                  antireflective BCs always uses it (Q from H~, Section 4.3). */
};

/* ---- options --------------------------------------------------------- */
typedef struct mlba_opts {
  double mu;          /* soft-threshold parameter, Eq. soft */
  double alpha;       /* regularisation of P (Algorithms 1-4); floor of alpha_n for the rectangular 4-NS hybrid */
  double gamma;       /* discrepancy factor of Eq. discrpr (default 1 + 1e-15) */
  double q;           /* Algorithm 4-NS safeguard q in (2 rho, 1) (default 0.5) */
  double rho;         /* Algorithm 4-NS rho in (0, 1/2) (default 1e-4) */
  double pcg_tol;     /* Algorithm 2 relative tolerance (default 1e-3) */
  int levels;         /* framelet levels L >= 1; z has 8L+1 bands */
  int max_iter;       /* iteration budget */
  int pcg_max;        /* Algorithm 2 cap on PCG steps (default 5, Eq. bet) */
  int dtype;          /* MLBA_F32 or MLBA_F64 */
  int z_store;        /* MLBA_F32 or MLBA_BF16 with F32; MLBA_F64 with F64 */
  int transform;      /* enum mlba_transform */
  int stop;           /* 1: stop on the discrepancy principle; 0: run max_iter iterations */
  int rect_ns_hybrid; /* 1: allow MLBA_P_TIKH_NS with MLBA_RECT (A^T (CC^T + alpha_n I)^{-1}) */
  void* stream;       /* cudaStream_t */
  int two_group;      /* batches of >= 2 problems: 1 (default) runs two groups of about equal
                         work half a step apart on two streams, so that one group's framelet
                         update overlaps the other's residual and preconditioner; 0 advances
                         the whole batch launch by launch.  The iterates are the same. */
  int autotune;       /* tile shape of the framelet kernel (FP32, levels <= 2): 0 (default) the
                         built-in shape; 1 measure every candidate shape at create on the
                         batch's own buffers and keep the fastest, reusing an earlier
                         measurement from the on-disk cache (MLBA_TUNE_CACHE, else
                         $XDG_CACHE_HOME/mlba_tune.txt, else $HOME/.cache/mlba_tune.txt; an
                         unwritable cache is skipped); 2 measure, ignoring the cache.  Every
                         shape computes the same values; only the time differs. */
  int frame_shape;    /* -1 (default): as autotune says; 0 .. MLBA_FRAME_SHAPES - 1: force it */
  int blur_path;      /* how A and A^T (A' for antireflective BCs) are applied (Sections 2.1,
                         2.2): 0 (default) direct stencils with the BCs in the index math;
                         1 FFT convolution on a 2^a 3^b 5^c size M >= n + p - 1 (the input
                         padded by the BCs, the PSF's DFT as the multiplier) for every problem
                         where M <= 4096 and the algorithm is not 2 (its PCG keeps the
                         stencils); 2 per problem the faster of the two, measured at create.
                         Both compute the same operator (to rounding). */
  int formulation;    /* 0 (default) the synthesis MLBA of Eq. MLBA2; 1 the balanced approach
                         the paper names as the other use of its preconditioners (Section 1,
                         Conclusions), in proximal form x^{n+1} = S_mu(W (W^T x^n + u^n)) with
                         u^n the same preconditioned correction; z then holds W (f^n + u^n). */
  int persistent;     /* 1: iterate(k) is ONE cooperative launch (a CUDA graph of a memset of
                         the barrier words and the kernel) that runs the k steps of the
                         whole batch, stage by stage, with grid barriers between the stages
                         (CTAs resident on every SM take the items of a stage in turn); 0
                         (default) the captured graphs of separate launches.  The iterates are
                         the same.  Supported with dtype F32, levels <= 2, direct stencils
                         (blur_path 0) and the DFT/DCT preconditioners or none (not Algorithm
                         2, not the antireflective transform); otherwise create returns
                         MLBA_E_UNSUPPORTED.  The framelet tile shape is the built-in one. */
  double wait_s;      /* persistent: longest wait of a CTA at a grid barrier (default 1 s).  When
                         it expires the launch ends and every problem of the batch stops with
                         status MLBA_E_TIMEOUT (0: a CTA that is not the last to arrive gives up
                         at once, so that the first barrier times out). */
} mlba_opts;

#define MLBA_FRAME_SHAPES 8

/* Fill defaults: mu = 10/255, alpha = 0.05, gamma = 1 + 1e-15, q = 0.5,
 * rho = 1e-4, pcg_tol = 1e-3, levels = 1, max_iter = 200, pcg_max = 5,
 * dtype = F32, z_store = F32, transform = AUTO, stop = 1, hybrid = 0,
 * stream = NULL, two_group = 1, autotune = 0, frame_shape = -1, blur_path = 0,
 * formulation = 0, persistent = 0, wait_s = 1. */
void mlba_opts_default(mlba_opts* o);

/* ---- statistics ------------------------------------------------------- */
typedef struct mlba_stats {
  int iter;           /* z-updates done; the current f is f^iter */
  int stopped;        /* 1 once the context stopped (rule fired, budget used, or diverged) */
  int stop_iter;      /* first n at which the discrepancy rule held, -1 if never */
  int status;         /* MLBA_OK, MLBA_E_DIVERGED or MLBA_E_TIMEOUT */
  double resnorm;     /* ||r^k|| of the last residual computed */
  double alpha_n;     /* last alpha used (alpha_n for 4-NS) */
  int beta_n;         /* last PCG step count (Algorithm 2) */
  int nres;           /* residuals computed so far (history length) */
} mlba_stats;

/* ---- single problem --------------------------------------------------- */
typedef struct mlba_ctx mlba_ctx;

/* Largest PSF side accepted by mlba_create / mlba_batch_create (the stencil
 * tile holds 64 + p - 1 <= 128 columns). */
#define MLBA_MAX_P 65

/* Create a context for one problem.  psf: host, p*p doubles, row-major,
 * nonnegative; the library copies it.  n: observed size (n >= p); p odd and
 * at most MLBA_MAX_P (else MLBA_E_UNSUPPORTED).
 * Validates the combination (Algorithm 4 needs a square A, Section 5), builds
 * the PSF tap list and its rank-one test, the FFT plans for length n and the
 * spectrum of C / Q in FP64 on the device (Section 4.1, 4.3), allocates all
 * device buffers and captures one iteration into a CUDA graph.
 * Errors: MLBA_E_INVAL, MLBA_E_UNSUPPORTED, MLBA_E_NOMEM, MLBA_E_CUDA. */
int mlba_create(const double* psf, int p, int n, int bc, int precond,
                const mlba_opts* opts, mlba_ctx** out);

/* Upload g (n x n, dtype of the context) and the noise level delta, and
 * reset the iteration (z = 0, f = 0, counters cleared). */
int mlba_set_data(mlba_ctx* ctx, const void* g, int g_on_device, double delta);

/* Queue k steps on the stream.  A step computes r^n = g - A f^n and its FP64
 * norm, applies the stop rule, and (unless stopped) performs the update to
 * z^{n+1}, f^{n+1}.  Once stopped, further steps do nothing.  Asynchronous. */
int mlba_iterate(mlba_ctx* ctx, int k);

/* Copy f (N_f x N_f, dtype of the context) out.  Host destination: syncs. */
int mlba_result(mlba_ctx* ctx, void* f_out, int on_device);

/* Synchronise the stream and read the counters. */
int mlba_stats_get(mlba_ctx* ctx, mlba_stats* st);

/* Residual-norm (and alpha_n, beta_n) history, up to cap entries each (host
 * arrays; any may be NULL).  Returns the number of entries written. */
int mlba_history(mlba_ctx* ctx, double* resnorm, double* alpha, int* beta, int cap);

/* Copy the Bregman variable z out / in ((8L+1) x N_f x N_f, z_store type). */
int mlba_get_z(mlba_ctx* ctx, void* z_out, int on_device);

/* Checkpoint / resume.  The iteration of Eq. MLBA2 is fully determined by
 * z^n (f^n = W^T S_mu(z^n) is kept with it so that no synthesis has to be
 * re-run), the counters, the stop record, ||r^{n-1}||, alpha_{n-1} and the
 * log-alpha warm start of Algorithm 4-NS; the state also carries the
 * histories.  The state is a host blob of mlba_state_size() bytes: a header
 * (sizes, dtype, z storage, max_iter, preconditioner, transform, stop flag,
 * PCG cap, formulation, and mu, alpha, gamma, delta, q, rho, pcg_tol), the scalars, the
 * histories (max_iter + 2 entries each), f (N_f x N_f, dtype) and z
 * (band-major planes, z_store type).  mlba_get_state synchronises the stream
 * and copies it out; mlba_set_state loads it into a context created with the
 * same PSF size, n, boundary treatment, levels, dtype, z storage, max_iter,
 * preconditioner, transform and parameters, whose mlba_set_data gave the same
 * delta (else MLBA_E_INVAL: a state taken under another preconditioner or
 * parameter set would silently continue a different iteration).  Call
 * mlba_set_data first (it resets the state): the observation g is not part of
 * the state.  The next mlba_iterate
 * continues from the saved iteration exactly as the original context would
 * have.  bytes: the caller's buffer size (>= mlba_state_size, else
 * MLBA_E_INVAL).  No counterpart in the paper. */
int mlba_state_size(mlba_ctx* ctx, size_t* bytes);
int mlba_get_state(mlba_ctx* ctx, void* blob, size_t bytes);
int mlba_set_state(mlba_ctx* ctx, const void* blob, size_t bytes);

void mlba_destroy(mlba_ctx* ctx);
const char* mlba_strerror(int status);

/* ---- operator entry points (one kernel pass each, on a context) ------------
 * All arrays are in the context dtype; on_device as above. */
/* out = A f   (f: N_f x N_f, out: n x n)  Section 2, Table 1, Eq. Arect. */
int mlba_op_blur(mlba_ctx* ctx, const void* f, void* out, int on_device);
/* out = A^T t (t: n x n, out: N_f x N_f)  exact transpose of mlba_op_blur;
 * for antireflective BCs the reblurring matrix A' t (Section 2.2). */
int mlba_op_blur_adjoint(mlba_ctx* ctx, const void* t, void* out, int on_device);
/* out = (CC^T + alpha I)^{-1} r (which = 0, Eq. Alg1/Alg3) or
 * C^T (CC^T + alpha I)^{-1} r (which = 1, Eq. Alg4); r, out: n x n.
 * Uses the context's C (DFT or DCT) through the batched transform kernels. */
int mlba_op_precond(mlba_ctx* ctx, const void* r, void* out, double alpha, int which, int on_device);
/* One fused framelet pass: z_out = z_in + W u, f = W^T S_mu(z_out)
 * (Eq. MLBA2 second half; Section 6.1).  z_*: z_store type; u, f: N_f x N_f. */
int mlba_op_frame(mlba_ctx* ctx, const void* z_in, const void* u, void* z_out,
                  void* f, double mu, int on_device);
/* alpha solving alpha ||(CC^T + alpha I)^{-1} r|| = qn ||r|| (Eq. Alg4_rev_7);
 * r: n x n; result written to *alpha_out (host). */
int mlba_op_ns_alpha(mlba_ctx* ctx, const void* r, double qn, double* alpha_out, int on_device);
/* Spectrum of C (or Q) as the library stores it: DFT: n x (n/2+1) complex
 * (interleaved re, im doubles), DCT: n x n doubles.  Host output. */
int mlba_op_spectrum(mlba_ctx* ctx, double* out, int* rows, int* cols, int* is_complex);

/* ---- batch of independent problems (one graph launch per step) ---------- */
typedef struct mlba_problem {
  const double* psf;  /* host p*p */
  int p, n, bc, precond, transform, max_iter;
  double mu, alpha, delta;
  const void* g;      /* n x n in the batch dtype */
  int g_on_device;
} mlba_problem;

typedef struct mlba_batch mlba_batch;

/* Problems share opts.dtype, z_store, levels, stop, gamma, q, rho, pcg_*,
 * stream; each has its own size, PSF, BC, preconditioner, mu, alpha, delta
 * and budget.  Each problem stops on its own rule. */
int mlba_batch_create(const mlba_problem* probs, int count, const mlba_opts* opts, mlba_batch** out);
/* Enqueue k steps on the batch stream (asynchronous).  Every live problem
 * advances by k iterations, whatever opts.two_group says.  With
 * opts.persistent the k steps are one launch; a grid barrier that waited
 * longer than opts.wait_s shows as status MLBA_E_TIMEOUT in every problem's
 * stats. */
int mlba_batch_iterate(mlba_batch* b, int k);
/* Number of problems not yet stopped (synchronises). */
int mlba_batch_active(mlba_batch* b, int* n_active);
int mlba_batch_result(mlba_batch* b, int i, void* f_out, int on_device);
int mlba_batch_stats(mlba_batch* b, int i, mlba_stats* st);
/* Re-arm every problem: z = 0, f = 0, counters cleared (data kept). */
int mlba_batch_reset(mlba_batch* b);
/* Replace problem i's observed image g (n x n, batch dtype) and delta; the
 * iteration state is left as it is (call mlba_batch_reset to restart).
 * Host source: synchronises. */
int mlba_batch_set_data(mlba_batch* b, int i, const void* g, int g_on_device, double delta);
/* Every problem at once (the observation g = A f + eta and the noise level
 * delta of the paper's problem statement, Section 2 and Eq. discrpr):
 * g[i] is problem i's n_i x n_i observed image (batch dtype, row-major, host
 * or device memory as g_on_device says), delta[i] its delta.  All copies are
 * enqueued on the batch stream and the call synchronises once, at the end,
 * so the caller may reuse the host buffers after it returns (pinned host
 * memory gives asynchronous copies).  Arguments are checked for every
 * problem before anything is copied (MLBA_E_INVAL, nothing changed); the
 * iteration state is left as it is. */
int mlba_batch_set_data_all(mlba_batch* b, const void* const* g, int g_on_device,
                            const double* delta);
/* f~ of every problem at once: f_out[i] receives problem i's N_f,i x N_f,i
 * result (batch dtype, row-major; caller-owned host or device memory as
 * on_device says), with one synchronisation at the end for host
 * destinations (device destinations: stream-ordered, no synchronisation). */
int mlba_batch_result_all(mlba_batch* b, void* const* f_out, int on_device);
/* Time one stage of the step on the batch stream with CUDA events: stage 0 =
 * the whole captured step (graph launch), 1 = residual stencil, 2 =
 * spectral preconditioner passes, 3 = adjoint correlation, 4 = fused
 * framelet kernel.  Launches it `reps` times and writes the mean time per
 * launch in milliseconds.  Stages 1-4 run outside the graph and advance the
 * per-problem state arbitrarily: call mlba_batch_reset before using results. */
int mlba_batch_profile(mlba_batch* b, int stage, int reps, float* ms_per_rep);
/* Kernel launches per step: the kernel nodes of the captured step graph (with
 * the two-group schedule, of the body graph, which holds one step of each
 * group). */
int mlba_batch_graph_kernels(mlba_batch* b, int* n_kernels);
void mlba_batch_destroy(mlba_batch* b);

/* Tile shape of the framelet launch: shape index, tile columns x rows, z
 * prefetch distance in rows, how it was chosen (0 built-in default, 1
 * measured at create, 2 read from the tuning cache, 3 forced by
 * opts.frame_shape) and the measured microseconds per launch (1, 2).  Shapes
 * apply to levels <= 2; with more levels tile_x = tile_y = prefetch = 0.
 * Any output pointer may be NULL.  No counterpart in the paper. */
int mlba_batch_tiles(mlba_batch* b, int* frame_shape, int* tile_x, int* tile_y, int* prefetch,
                     int* how, float* us);
int mlba_tiles(mlba_ctx* ctx, int* frame_shape, int* tile_x, int* tile_y, int* prefetch, int* how,
               float* us);
/* Whether problem i applies A and A^T by FFT convolution (opts.blur_path) and
 * the convolution size M (0 on the direct path).  No counterpart in the paper
 * beyond Section 2's remark that A is applied by FFTs after padding. */
int mlba_batch_blur_fft(mlba_batch* b, int i, int* uses_fft, int* size);

/* ---- entry point that allocates no device memory ------------------------
 * The paper has no counterpart: this is a service for callers that cannot
 * call cudaMalloc (a host framework that owns all device memory, a fixed
 * memory budget, or a loop where the implicit synchronisation of
 * cudaMalloc/cudaFree is not acceptable).
 *
 * r = g - A f and *norm2 = ||r||^2 (FP64 accumulation, fixed summation
 * order), the residual stencil of one iteration, in FP32.  All pointers are
 * device memory on the current device: f (N_f x N_f, N_f = n + p - 1 for
 * MLBA_RECT else n), g and r (n x n), psf (p x p row-major floats, centred),
 * norm2 (one double).  bc is an enum mlba_bc value; work is queued on
 * `stream` (a cudaStream_t, NULL = legacy default stream).
 *
 * Scratch: a fixed array in device memory of the library, 8 bytes per
 * 32 x 32 tile for n up to MLBA_NOALLOC_MAX_N (about 128 KiB), which every
 * GPU that loads the library holds until the process exits.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call shares the
 * array: calls whose kernels overlap on the GPU (other streams, concurrent
 * graph replays) race and must be serialised by the caller.  Nothing is
 * allocated or freed.
 * Errors: MLBA_E_INVAL (null pointer, even p, n < p, bad bc),
 * MLBA_E_UNSUPPORTED (n > MLBA_NOALLOC_MAX_N or p > MLBA_NOALLOC_MAX_P),
 * MLBA_E_CUDA (launch or symbol lookup failed). */
#define MLBA_NOALLOC_MAX_N 4096
#define MLBA_NOALLOC_MAX_P 41
int mlba_residual_noalloc(const float* f, const float* g, const float* psf, int p, int n, int bc,
                          float* r, double* norm2, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MLBA_H */
