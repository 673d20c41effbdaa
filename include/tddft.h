/*
 * tddft.h - C ABI of the GB300 rid-preconditioned Davidson solver for the
 * TDDFT response problem (arXiv 2404.17133).
 *
 * The library solves, on one GPU:
 *   - the Tamm-Dancoff eigenproblem  A X = Omega X            (Eq. TDA)
 *   - the Casida eigenproblem [[A,B],[B,A]](X;Y) = Omega diag(1,-1)(X;Y)
 *                                                              (Eq. Casida)
 *   - the dynamic polarizability alpha_vu(omega) of Eq. TDDFT_polar
 * by the preconditioned Davidson algorithm of Sec. 2.1 (Eqs. 1-4,
 * Eq. residual, Eq. precondition), with either the diagonal preconditioner
 * or the rid preconditioner (Sec. 3: an inner Krylov solve with the
 * minimal-auxiliary ris operator, Eq. TDDFT-ris_approx, (l_J, l_K) = (d, s),
 * exchange energy window t_cut of Sec. 3.1).
 *
 * Operator (Eq. hessian with f^xc = 0 and density-fitted integrals,
 * (pq|rs) = sum_P L^P_pq L^P_rs, Eq. pqrs / Eq. pqrs_approx):
 *   A   = Delta + c_J (ia|jb) - a_x (ij|ab)
 *   B   = c_J (ia|jb) - a_x (ib|ja)
 *   Delta_ia = eps_a - eps_i
 * c_J is `coulomb_factor`: 2 is the restricted-singlet convention (default),
 * 1 reproduces Eq. hessian as printed (2(ia|jb) in A+B).
 *
 * Conventions for every call:
 *   - Index order: a singles vector is [n_occ][n_vir] row-major, ia = i*n_vir+a.
 *     Factor blocks are [P][p][q] row-major and symmetric in (p,q) for each P.
 *   - Ownership: input arrays stay owned by the caller; tddft_create copies
 *     and converts them, so they may be freed when it returns.  Output arrays
 *     are caller-allocated.  The context owns every device allocation it makes.
 *   - Errors: every call returns a tddft_status and never aborts the process;
 *     tddft_last_error() returns a message for the last failing call on that
 *     context.  TDDFT_ERR_NOCONV still fills the outputs with the last Ritz data.
 *   - Threading: a context is used by one host thread at a time, except that
 *     tddft_submit/tddft_poll may be called from any thread.
 *   - Environment (read at call time; none changes a result):
 *       TDDFT_TRACE=1 one line per outer iteration on stderr; =2 also times
 *         the solver's phases (stream-synchronised: diagnostics only);
 *       TDDFT_TC_CLUSTER=0 runs the split-operand tensor-core contractions
 *         without CTA clusters, TDDFT_TC_QUAD=0 in pairs only (not 2 x 2):
 *         every launch shape gives the same bits;
 *       TDDFT_BATCH_VARIANT=i makes tddft_solve_tda_batch keep SIMT tile
 *         variant i after timing them all (same bits from each variant).
 */
#ifndef TDDFT_H
#define TDDFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tddft_ctx tddft_ctx;

typedef enum {
  TDDFT_OK = 0,
  TDDFT_PENDING = 1,          /* tddft_poll: request not finished yet          */
  TDDFT_ERR_ARG = -1,         /* bad argument (null pointer, size, option)     */
  TDDFT_ERR_OOM = -2,         /* device memory budget or allocation exceeded   */
  TDDFT_ERR_CUDA = -3,        /* a CUDA runtime call failed                    */
  TDDFT_ERR_NOCONV = -4,      /* max_iter reached; outputs hold the last data  */
  TDDFT_ERR_INDEFINITE = -5,  /* A-B or A+B (projected) not positive definite, */
                              /* or non-finite values in the inputs / Ritz data*/
  TDDFT_ERR_TIMEOUT = -6,     /* tddft_poll waited timeout_ms without result   */
  TDDFT_ERR_BUSY = -7         /* request queue full                            */
} tddft_status;

typedef enum { TDDFT_F64 = 0, TDDFT_F32 = 1 } tddft_dtype;

typedef enum { TDDFT_PRECOND_DIAG = 0, TDDFT_PRECOND_RID = 1 } tddft_precond;

/* Arithmetic of the solve.
 * PLAIN: every step in FP64 (factors, products, subspace algebra).
 * MIXED: exact products with FP32 factors and FP32 accumulation, or, when
 *        `tensor_cores` is set, on the tcgen05 tensor cores with every operand
 *        (factors, trial vectors, the first contraction's results) scaled by
 *        a power of two and split into FP16 hi + lo parts (22 significand
 *        bits; three products hi*hi + hi*lo + lo*hi, FP32 accumulation) --
 *        FP32-accurate products either way; the ris inner solve on BF16
 *        factors with FP32 accumulation; FP64 for the subspace eigenproblem,
 *        Gram-Schmidt and the residuals, which are recomputed at the end from
 *        fresh products of the converged vectors ("certification").        */
typedef enum { TDDFT_PLAIN = 0, TDDFT_MIXED = 1 } tddft_precision;

typedef struct {
  int n_occ, n_vir;           /* occupied / virtual orbitals                  */
  int n_aux;                  /* exact auxiliary functions P                  */
  int n_aux_ris_J;            /* ris auxiliary functions (Coulomb, 9/atom)    */
  int n_aux_ris_K;            /* ris exchange rows (s functions, 1/atom)      */
  double a_x;                 /* exact-exchange fraction c_x                  */
  double coulomb_factor;      /* c_J, see above (2.0 default)                 */
  double t_cut_ha;            /* exchange energy cutoff, Hartree (40 eV)      */
  int precisions;             /* bit0: keep FP64 factors (PLAIN solves);      */
                              /* bit1: keep FP32/BF16 factors (MIXED solves)  */
  double hbm_budget_gb;       /* refuse create (TDDFT_ERR_OOM) above this;    */
                              /* 0 = free device memory minus 2 GB            */
} tddft_desc;

typedef struct {
  int precond;                /* tddft_precond                                */
  int n_states;               /* roots wanted                                 */
  int n_extra_guess;          /* -1: paper rule (rid: +min(n,3), diag: +8)    */
  double tol;                 /* outer residual threshold (1e-5, Sec. 3)      */
  double inner_tol;           /* ris inner solve, relative (1e-2, Sec. 3.1)   */
  double guess_tol;           /* ris initial-guess solve (1e-3, Sec. 3.1)     */
  int max_iter;               /* outer iterations (50)                        */
  int inner_max_iter;         /* ris inner iterations (20, Sec. 3.1)          */
  int max_subspace;           /* collapse above this many vectors (0: auto)   */
  int precision;              /* tddft_precision                              */
  int tensor_cores;           /* MIXED only: tcgen05 FP16 hi+lo exchange      */
  int outputs_on_device;      /* 1: omega/X/Y/resid/alpha are device pointers */
  int ris_fp8;                /* MIXED + tensor_cores: the ris exchange products of
                               * the rid preconditioner (Eq. TDDFT-ris_approx) in
                               * FP8 e4m3 with one scale per auxiliary row,
                               * FP32 accumulation; 0: BF16 ris factors        */
} tddft_opts;

typedef struct {
  int n_iter;                 /* outer Davidson iterations                    */
  int n_matvec;               /* exact operator products (vectors)            */
  int n_ris_matvec;           /* ris operator products (vectors)              */
  int converged;              /* 1 if every root / system met tol             */
  int n_restart;              /* subspace collapses                           */
  int gpu_launches;           /* kernels launched by this solve               */
  double max_resid;           /* largest final residual norm                  */
  double max_resid_certified; /* MIXED: the final residuals recomputed from   */
                              /* fresh FP32-accurate products (-1: PLAIN)     */
  double t_total_s, t_matvec_s, t_precond_s;  /* wall times (host clock)     */
  double t_guess_s;           /* initial guess (Davidson on the ris operator)  */
  double t_certify_s;         /* MIXED: that recomputation                     */
} tddft_stats;

/* Fill `opts` with the paper's defaults (Sec. 3.1-3.2): rid, tol 1e-5,
 * inner tol 1e-2 / 20 iterations, guess tol 1e-3, N_init rule, PLAIN.      */
void tddft_default_opts(tddft_opts* opts);

/* Fill `desc` defaults: a_x 0.25, c_J 2, t_cut 40 eV, both precisions.     */
void tddft_default_desc(tddft_desc* desc);

/* Create a context: upload and convert the orbital energies and factors.
 *   eps_occ [n_occ], eps_vir [n_vir]      ascending orbital energies (FP64)
 *   L_oo [n_aux][n_occ][n_occ], L_ov [n_aux][n_occ][n_vir],
 *   L_vv [n_aux][n_vir][n_vir]            exact factors (Eq. pqrs_approx)
 *   Lr_ov [n_aux_ris_J][n_occ][n_vir]     ris Coulomb factors (all rows)
 *   Lr_oo [n_aux_ris_K][n_occ][n_occ],
 *   Lr_vv [n_aux_ris_K][n_vir][n_vir]     ris exchange factors (s rows only)
 *   ris_K_index [n_aux_ris_K]             row of Lr_ov that each exchange row
 *                                         is (its ov block for (ib|ja))
 *   dtype                                 element type of all factor arrays
 *   inputs_on_device                      1: every array pointer is device memory;
 *                                         the library reads it on cuda_stream (or
 *                                         its own stream) after the work already
 *                                         queued on the legacy default stream;
 *                                         writes queued on other streams must be
 *                                         complete or ordered before cuda_stream
 *   cuda_stream                           cudaStream_t to run on (NULL: own one)
 * The t_cut window is applied here to the ris exchange rows.
 * Returns TDDFT_ERR_ARG on bad sizes or null pointers, TDDFT_ERR_OOM when the
 * resident factor copies exceed desc->hbm_budget_gb or the free memory.    */
tddft_status tddft_create(const tddft_desc* desc, const double* eps_occ, const double* eps_vir,
                          const void* L_oo, const void* L_ov, const void* L_vv,
                          const void* Lr_oo, const void* Lr_ov, const void* Lr_vv,
                          const int* ris_K_index, tddft_dtype dtype, int inputs_on_device,
                          void* cuda_stream, tddft_ctx** out);

/* TDA excitation energies (Eq. TDA).  omega [n_states] ascending, X
 * [n_states][n_occ*n_vir] unit-norm eigenvectors (may be NULL), resid
 * [n_states] final |R_n| (may be NULL), stats may be NULL.                 */
tddft_status tddft_solve_tda(tddft_ctx* ctx, const tddft_opts* opts, double* omega, double* X,
                             double* resid, tddft_stats* stats);

/* Casida excitation energies (Eq. Casida), X and Y normalised so that
 * X^T X - Y^T Y = 1 (each may be NULL).  The residual of root n is
 * sqrt(|(A+B)(X+Y) - Omega(X-Y)|^2 + |(A-B)(X-Y) - Omega(X+Y)|^2).         */
tddft_status tddft_solve_rpa(tddft_ctx* ctx, const tddft_opts* opts, double* omega, double* X,
                             double* Y, double* resid, tddft_stats* stats);

/* Dynamic polarizability (Eq. TDDFT_polar) for n_dip dipole vectors mu
 * [n_dip][n_occ*n_vir] at n_freq frequencies omega [n_freq] (Hartree):
 * alpha [n_freq][n_dip][n_dip], alpha_vu = mu_v^T (X_u + Y_u).  The system
 * residual is divided by |2 mu_u| before the tol test.                    */
tddft_status tddft_solve_polar(tddft_ctx* ctx, const tddft_opts* opts, const double* mu,
                               int n_dip, const double* omega, int n_freq, double* alpha,
                               tddft_stats* stats);

/* Variant terms of Eq. hessian for other functionals (the paper's benchmarks
 * include a range-separated hybrid; the terms keep the same kernels).  Each
 * may be added once per context, before or between solves; they enter the
 * exact operator (every product and residual) and not the ris
 * preconditioner T.
 *
 * tddft_add_exchange: a second exchange factor set M (the long-range,
 * erf-attenuated exchange integrals (pq|rs)_LR = sum_Q M^Q_pq M^Q_rs of a
 * range-separated hybrid) with weight b_x:
 *   A -= b_x (ij|ab)_LR,  B -= b_x (ib|ja)_LR.
 *   M_oo [n_aux_lr][n_occ][n_occ], M_ov [n_aux_lr][n_occ][n_vir],
 *   M_vv [n_aux_lr][n_vir][n_vir] in `dtype`, copied in the precisions the
 *   context keeps (the caller keeps ownership).
 * tddft_add_kernel: a low-rank response kernel in place of f^xc,
 *   (ia|f|jb) = sum_g w_g F^g_ia F^g_jb, added to A and to B with the Coulomb
 *   prefactor (c_J (ia|f|jb), as Eq. hessian adds 2 f^xc next to 2 (ia|jb)).
 *   w [n_g] FP64 (any sign; host or device as inputs_on_device says),
 *   F_ov [n_g][n_occ][n_vir] in `dtype`.
 * Errors: TDDFT_ERR_ARG (bad sizes, null pointers, non-finite weight, the term
 * already present), TDDFT_ERR_INDEFINITE (non-finite factor values).        */
tddft_status tddft_add_exchange(tddft_ctx* ctx, double b_x, int n_aux_lr, const void* M_oo,
                                const void* M_ov, const void* M_vv, tddft_dtype dtype,
                                int inputs_on_device);
tddft_status tddft_add_kernel(tddft_ctx* ctx, int n_g, const double* w, const void* F_ov,
                              tddft_dtype dtype, int inputs_on_device);

/* One operator product on m vectors (for tests and measurement):
 *   kind 0: A X (exact), 1: ((A+B)X, (A-B)X) exact, 2: T_A X (ris),
 *   kind 3: ((T_A+T_B)X, (T_A-T_B)X) ris.
 * X [m][ov]; out0 [m][ov]; out1 [m][ov] for kinds 1 and 3 (else NULL).
 * precision / tensor_cores as in tddft_opts (exact kinds: the scaled FP16
 * hi + lo products; ris kinds: two products, trial vectors as BF16 hi + lo
 * against the BF16 ris rows); tensor_cores = 2 runs the ris kinds' exchange
 * contractions with the FP8 e4m3 ris rows (tddft_opts.ris_fp8) and the exact
 * kinds as 1; other values: TDDFT_ERR_ARG; on_device: pointers are device
 * memory.
 * Results are FP64.                                                        */
tddft_status tddft_apply(tddft_ctx* ctx, int kind, int precision, int tensor_cores,
                         const double* X, int m, double* out0, double* out1, int on_device);

/* Asynchronous requests.  kind: 0 TDA, 1 RPA, 2 polar.  `req` points to a
 * tddft_request whose arrays must stay valid until tddft_poll returns a final
 * status for the ticket.  A worker thread owned by the context runs the
 * requests in arrival order.  tddft_poll waits at most timeout_ms (0: do not
 * wait) and returns TDDFT_PENDING, TDDFT_ERR_TIMEOUT, or the request's status. */
typedef struct {
  tddft_opts opts;
  double* omega; double* X; double* Y; double* resid;      /* eigen requests */
  const double* mu; int n_dip; const double* freqs; int n_freq; double* alpha;  /* polar */
  tddft_stats stats;                                       /* filled on completion */
} tddft_request;

tddft_status tddft_submit(tddft_ctx* ctx, int kind, tddft_request* req,
                          unsigned long long* ticket);
tddft_status tddft_poll(tddft_ctx* ctx, unsigned long long ticket, int timeout_ms);

/* ---- Serving (no counterpart in the paper, which solves one molecule at a
 * time; this is the library's interface for many independent problems).
 * A server runs up to max_active requests at once, each on a CUDA stream of
 * its own, so the kernels of different requests overlap on the device.  A
 * request either brings its own problem (the server creates a context from
 * the desc and arrays when the request is admitted, on the slot's stream, and
 * destroys it when the solve ends) or names an existing context in `ctx`,
 * whose factors stay resident between requests (solves on one context run
 * one at a time).  Admission is first in, first out: the oldest waiting
 * request starts as soon as a slot is free and its charge fits into the
 * budget minus the charges of the running requests.  The charge is
 * tddft_estimate_bytes (factor copies + workspace; workspace only for a
 * request on an existing context).  A request whose charge exceeds the whole
 * budget is refused at submit with TDDFT_ERR_OOM.
 * Every array a request points to must stay valid until tddft_server_poll
 * returns its final status. */
typedef struct tddft_server tddft_server;

typedef struct {
  tddft_ctx* ctx;             /* non-NULL: solve on this context; the problem
                                 fields below (desc ... inputs_on_device) are
                                 then ignored                                 */
  tddft_desc desc;            /* problem, as for tddft_create                 */
  const double* eps_occ; const double* eps_vir;
  const void* L_oo; const void* L_ov; const void* L_vv;
  const void* Lr_oo; const void* Lr_ov; const void* Lr_vv;
  const int* ris_K_index;
  tddft_dtype dtype; int inputs_on_device;
  int kind;                   /* 0 TDA, 1 Casida, 2 polarizability            */
  tddft_request req;          /* options, outputs and statistics (as for
                                 tddft_submit)                                */
  /* filled by the server */
  unsigned long long charged_bytes;   /* admission charge                     */
  double t_submit_s, t_start_s, t_end_s;  /* seconds since server creation:
                                 queued, admitted, finished                  */
  char error[256];            /* message when the final status is an error   */
} tddft_serve_request;

typedef struct {
  unsigned long long budget_bytes, in_use_bytes, peak_in_use_bytes;  /* charges */
  int active, max_active, queued;
  unsigned long long completed;
  /* the device's default stream-ordered memory pool, from which every device
   * buffer of the library comes: bytes in use when the server was created and
   * the high-water mark since then (other users of that pool included)     */
  unsigned long long pool_used_at_create_bytes, pool_high_bytes;
} tddft_server_state;

/* Device-memory charge of one request: the factor copies tddft_create makes
 * for desc (factor_bytes, may be NULL) and a bound on the solve's work
 * buffers (work_bytes, may be NULL): the outer subspace and its work vectors,
 * the rid inner space, the operator's P-chunk intermediates (at most three
 * of 512 MiB) and 64 MiB for the small algebra.  n_dip / n_freq are used for
 * kind 2 only.  TDDFT_ERR_ARG on bad sizes or kind.                        */
tddft_status tddft_estimate_bytes(const tddft_desc* desc, int kind, const tddft_opts* opts, int n_dip,
                                  int n_freq, unsigned long long* factor_bytes,
                                  unsigned long long* work_bytes);

/* hbm_budget_gb: total charge allowed at once (0: free memory at creation
 * minus 2 GB; larger values are capped at that); max_active: 1..64 slots.  */
tddft_status tddft_server_create(double hbm_budget_gb, int max_active, tddft_server** out);

/* Queue a request; fills *ticket.  TDDFT_ERR_OOM if its charge exceeds the
 * budget, TDDFT_ERR_ARG on a bad kind or desc, TDDFT_ERR_BUSY when the queue
 * holds 65536 requests or the server is shutting down.                     */
tddft_status tddft_server_submit(tddft_server* server, tddft_serve_request* req,
                                 unsigned long long* ticket);

/* Wait at most timeout_ms (0: do not wait).  TDDFT_PENDING / TDDFT_ERR_TIMEOUT
 * while queued or running; else the request's final status (once: the ticket
 * is then forgotten).                                                      */
tddft_status tddft_server_poll(tddft_server* server, unsigned long long ticket, int timeout_ms);

/* Budget, charges and queue length now; peak_in_use_bytes since creation.  */
tddft_status tddft_server_info(const tddft_server* server, tddft_server_state* state);

/* Run every queued request to its end, then release the slots and streams. */
void tddft_server_destroy(tddft_server* server);

/* The tddft_desc a context was created with.                              */
tddft_status tddft_ctx_desc(const tddft_ctx* ctx, tddft_desc* desc);

/* Release every device allocation and the worker thread. NULL is a no-op.  */
void tddft_destroy(tddft_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failing create when
 * ctx is NULL).  Valid until the next call on the same context.            */
const char* tddft_last_error(const tddft_ctx* ctx);

/* Device resident bytes held by the context (factor copies + workspace).   */
unsigned long long tddft_device_bytes(const tddft_ctx* ctx);

/* tddft_apply without device allocation.  (No counterpart in the paper: this
 * is an interface for callers of this library.)  Some callers cannot allocate
 * device memory when they need a product -- another runtime owns the device's
 * memory pool, a real-time loop cannot take an allocation's latency or its
 * out-of-memory failure, or allocation calls are not allowed in the calling
 * context.  This entry point computes the same products as tddft_apply
 * (kinds 0-3, PLAIN = FP64 or MIXED = FP32 SIMT; no tensor-core path; a
 * context with variant terms is refused with TDDFT_ERR_ARG) and keeps
 * every intermediate in one 64 MiB array of device memory that the library
 * declares statically: every GPU that loads the library holds those 64 MiB
 * until the process exits.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *   X, out0, out1: DEVICE pointers, [m][ov] FP64 (out1 for kinds 1 and 3).
 * The work is queued on the context's stream, which does not wait for any
 * other stream: X must be complete before the call (synchronise the stream
 * that wrote it, or make the context's stream wait on an event recorded
 * after the write).  Results are valid once the context's stream has been
 * synchronised.  Every call whose stream is not being captured looks up the
 * array's device address with the context's device current (so an address
 * from before a cudaDeviceReset or from another CUDA context is never used);
 * a call made during stream capture reuses the address of the last
 * uncaptured call on that device, so make the first call on a device before
 * any stream capture.  All calls in the process
 * share the one array and it keeps the previous call's contents, so calls
 * whose work overlaps on the GPU (for example from two contexts on different
 * streams) race with each other.  A product whose intermediates do not fit in
 * 64 MiB is rejected with TDDFT_ERR_ARG (use tddft_apply).                  */
tddft_status tddft_apply_noalloc(tddft_ctx* ctx, int kind, int precision, const double* X, int m,
                                 double* out0, double* out1);

/* ---- Batched TDA solves (no counterpart in the paper, which solves one
 * molecule at a time; this is the library's interface for many small
 * independent problems).  The n contexts' TDA problems (opts[i] for
 * ctxs[i]; a context may appear more than once, its factors are only read)
 * are advanced together, one Davidson iteration (Sec. 2.1) of every problem
 * at a time: every step of an iteration is one launch for all problems (a
 * persistent grouped GEMM walking a device task list; row operations from a
 * device list; one CTA per problem for the small matrices), and the exact
 * operator product of an iteration is replayed from a captured CUDA graph.
 * The exact operator's lists run on a grouped tensor-core tile kernel (each
 * operand split into three BF16 parts, six products per K step: FP32-
 * accurate); the other lists' SIMT tile shape is chosen by a measured
 * autotune on the first ris product (every variant gives the same bits).
 * Precision: trial vectors in FP32, exact products FP32-accurate, ris
 * factors in BF16 (FP32 accumulation), projected matrices and small solves
 * in FP64; stats[i].max_resid_certified is -1 (no separate recomputation);
 * a timed-out wait of the tensor-core kernel is TDDFT_ERR_CUDA; contexts need the MIXED
 * factor copies; opts[i].precision / tensor_cores / ris_fp8 are ignored,
 * n_states <= 32; contexts with variant terms are refused (TDDFT_ERR_ARG).
 *   omega, resid: HOST arrays of sum_i min(opts[i].n_states, ov_i) entries,
 *                 problem after problem (resid may be NULL);
 *   stats: HOST [n] (may be NULL); info: HOST (may be NULL).
 * All contexts must be on one device; the work runs on ctxs[0]'s stream.
 * Returns TDDFT_ERR_NOCONV when some problem did not converge (its results
 * are the last Ritz data); errors are reported on ctxs[0].                */
typedef struct {
  int n_variants;             /* grouped-GEMM tile variants timed             */
  int variant;                /* the variant kept (index), -1 if none         */
  double autotune_ms[8];      /* measured time of each variant (ms), -1: not run */
  int outer_iterations;       /* lockstep outer iterations (slowest problem)  */
  int graph_nodes;            /* kernel nodes of the captured operator graph  */
  long long launches;         /* kernel launches of the whole batch (incl. graph nodes) */
  long long graph_launches;   /* CUDA graph replays                           */
  double t_total_s;           /* wall time of the call                        */
} tddft_batch_info;

tddft_status tddft_solve_tda_batch(tddft_ctx* const* ctxs, int n, const tddft_opts* opts,
                                   double* omega, double* resid, tddft_stats* stats,
                                   tddft_batch_info* info);

/* Device memory pool query for tests and callers that track allocations.
 * (No counterpart in the paper.)  Reads the current and the high-water
 * "used" byte counts of `device`'s default stream-ordered memory pool, from
 * which every work buffer of this library is allocated; with reset_high
 * nonzero the high-water mark is then restarted at the current use.
 * used_current / used_high may be NULL.  Bad device: TDDFT_ERR_ARG.        */
tddft_status tddft_pool_usage(int device, unsigned long long* used_current,
                              unsigned long long* used_high, int reset_high);

/* Kernel timing for measurement.  tddft_profile(ctx, 1) starts recording
 * CUDA events on the context's stream around every launch of the dominant
 * contraction -- the exchange term K1's second contraction
 * sum_(P,a) Z[(n,i)][(P,a)] L^P_ab of the exact operator -- and resets the
 * totals; 0 stops.  tddft_profile_read returns, for that contraction, the
 * number of launches, their summed device time (ms) and the algorithmic
 * flops (2*M*N*K per launch) since the last reset: which = 0 for the
 * tcgen05 kernel (tensor_cores on), 1 for the SIMT kernel (tensor cores
 * off).  Other values:
 * TDDFT_ERR_ARG.                                                          */
tddft_status tddft_profile(tddft_ctx* ctx, int enable);
tddft_status tddft_profile_read(const tddft_ctx* ctx, int which, long long* launches,
                                double* ms, double* flops);

/* Per-launch records of the same kernel family since tddft_profile(ctx, 1):
 * device time (ms), algorithmic flops (2 M N K) and algorithmic bytes (each
 * operand read once in its stored type, the result written once in its
 * working type and read back when a P-chunk accumulates into it) of each
 * launch, oldest first, the
 * first 131072 launches at most.  Writes min(max_records, available) entries
 * of ms, flops and bytes and sets *count to the number available.          */
tddft_status tddft_profile_records(const tddft_ctx* ctx, int which, int max_records, double* ms,
                                   double* flops, double* bytes, int* count);

#ifdef __cplusplus
}
#endif
#endif /* TDDFT_H */
